"""The slab decomposition of one large cell across ranks (the multi-GPU design: the paper's
domain partitioning with ghost layers, Sec. 3.3), checked on the CPU with two gloo ranks.

Each rank holds a slab of z planes and one ghost plane on each side and advances it with
the FP64 oracle; after every step it sends to each neighbour only the five populations
whose e_kz points at that neighbour, of the fluid cells of its boundary plane, which land
in the neighbour's ghost plane.  That exchange plan suffices for SBB and CLI walls and the
periodic pressure drop: the slabs together equal the undivided cell bit for bit, and the
all-reduced moment sums equal its sums.  (A multi-GPU run is not possible here; this checks
the plan the GPU path would follow: which planes and which directions travel.)"""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, NZ, STEPS = 14, 12, 16, 24
SPHERES = [[7.2, 6.1, 7.6, 4.3], [2.0, 10.5, 15.2, 3.6]]   # one across the slab boundary, one across z = 0


def _setup():
    sys.path.insert(0, ROOT)
    import oracle
    oracle.set_threads(1)
    g = np.array(SPHERES)
    solid = oracle.voxelize((NZ, NY, NX), g)
    q = oracle.wall_distances(solid, g)
    _, w, _ = oracle.lattice()
    f0 = w[:, None, None, None] * (1.0 + 1e-3 * np.random.default_rng(3).uniform(-1, 1, (19, NZ, NY, NX)))
    f0[:, solid == 1] = 0.0
    return oracle, solid, q, f0


def exchange_plan(e):
    """Directions sent up (e_kz = +1: the plane above pulls them) and down (e_kz = -1)."""
    up = [k for k in range(19) if e[k, 2] == 1]
    down = [k for k in range(19) if e[k, 2] == -1]
    return up, down


def _rank(rank, world, port, wall, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle, solid, q, f0 = _setup()
    e, _, _ = oracle.lattice()
    up, down = exchange_plan(e)
    nzl = NZ // world
    z0 = rank * nzl
    planes = [(z0 - 1 + i) % NZ for i in range(nzl + 2)]   # ghost, interior..., ghost
    s = np.ascontiguousarray(solid[planes])
    qs = np.ascontiguousarray(q[:, planes])
    f = np.ascontiguousarray(f0[:, planes])
    kw = dict(q=qs, tau=0.7, delta_rho=3e-4, magic_lambda=3 / 16, collision=oracle.TRT, wall=wall)
    above, below = (rank + 1) % world, (rank - 1) % world
    fluid_top_ghost = s[nzl + 1] == 0
    fluid_bottom_ghost = s[0] == 0
    for _ in range(STEPS):
        f, _, _ = oracle.run(s, f, 1, **kw)
        # top interior plane's upward populations -> the slab above's bottom ghost; bottom
        # interior plane's downward populations -> the slab below's top ghost
        send_up = torch.from_numpy(np.ascontiguousarray(f[up][:, nzl]))
        send_down = torch.from_numpy(np.ascontiguousarray(f[down][:, 1]))
        recv_from_below = torch.empty_like(send_up)
        recv_from_above = torch.empty_like(send_down)
        reqs = [dist.isend(send_up, above, tag=1), dist.isend(send_down, below, tag=2),
                dist.irecv(recv_from_below, below, tag=1), dist.irecv(recv_from_above, above, tag=2)]
        for r in reqs:
            r.wait()
        for i, k in enumerate(up):
            f[k, 0][fluid_bottom_ghost] = recv_from_below.numpy()[i][fluid_bottom_ghost]
        for i, k in enumerate(down):
            f[k, nzl + 1][fluid_top_ghost] = recv_from_above.numpy()[i][fluid_top_ghost]
    interior = f[:, 1:nzl + 1]
    e64 = e.astype(np.float64)
    fl = interior[:, s[1:nzl + 1] == 0]
    sums = torch.tensor([fl.sum(), (e64[:, 0] @ fl).sum(), (e64[:, 1] @ fl).sum(), (e64[:, 2] @ fl).sum()],
                        dtype=torch.float64)
    dist.all_reduce(sums)
    out.put((rank, interior, sums.numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("wall", [0, 1])
def test_two_slabs_equal_the_undivided_cell(wall):
    oracle, solid, q, f0 = _setup()
    ref, _, _ = oracle.run(solid, f0, STEPS, q=q, tau=0.7, delta_rho=3e-4, magic_lambda=3 / 16,
                           collision=oracle.TRT, wall=wall)
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = 29700 + (os.getpid() % 200) + 7 * wall
    procs = [ctx.Process(target=_rank, args=(r, 2, port, wall, qu)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((qu.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = np.concatenate([r[1] for r in res], axis=1)
    assert np.array_equal(whole, ref)
    e, _, _ = oracle.lattice()
    fl = ref[:, solid == 0]
    ref_sums = np.array([fl.sum(), *(e.astype(np.float64).T @ fl).sum(axis=1)])
    for _, _, sums in res:
        assert np.allclose(sums, ref_sums, rtol=1e-12, atol=1e-15)
