// lbm_tma.cuh -- the fused step of a single instance in the A-B layout with its pulls
// staged in shared memory by the Tensor Memory Accelerator.
//
// The box is cut into bricks of kBrickX x kBrickY x kBrickZ cells (kBrickX = 32: one warp
// per x row); the bricks holding fluid form the work list.  A persistent block takes bricks
// b, b + B, b + 2B, ... (B = blocks in the grid) through a ring of kBrickStages stages: one
// thread issues, per brick and direction k, one tiled TMA copy of the brick shifted by -e_k
// (its x origin rounded down to a 16-byte boundary, the box kBrickX + XA wide for e_kx != 0)
// into the stage, completing on the stage's mbarrier; while a brick is being finished the
// copies of the next one are in flight, so the number of bytes in flight no longer depends
// on registers.  Pull sources outside the box (the periodic images across a face) are read
// directly by the lanes concerned.  Each cell then runs exactly the arithmetic of the tile
// kernel (finish_item), so both kernels give bit-identical states; the step that reduces
// the moments always runs the tile kernel.
//
// Runs on request (block_cells = kBrickCells).  On the 128^3 and 256^3 sphere cells it is
// slower than the tile kernel over fluid cells (14.5k and 18.6k against 23.3k and 28.0k
// MLUPS, FP32): a third (128^3) or an eighth (256^3) of a brick's threads hold solid cells,
// which the fluid-cell work list never schedules, and a brick costs about half as many
// instructions again in staging and synchronisation.  A dense box without walls staged this
// way reached 5.2-6.0 TB/s.
#pragma once

#include <cuda.h>

#include "lbm_step.cuh"

namespace lbm {


// Elements by which the x origin of a shifted box is rounded down (16 bytes).
template <int STORE> constexpr int brick_xa() { return 16 / (int)sizeof(typename Store<STORE>::T); }

// Shared-memory layout of one stage: direction k's box in a slot aligned to 128 bytes.
template <int STORE> struct BrickStage {
    using T = typename Store<STORE>::T;
    static constexpr int XA = brick_xa<STORE>();
    static constexpr int W0 = kBrickX, W1 = kBrickX + XA;  // box widths: e_kx = 0, e_kx != 0
    static constexpr int S0 = W0 * kBrickY * kBrickZ, S1 = W1 * kBrickY * kBrickZ;
    static constexpr int AL = 128 / (int)sizeof(T);
    static constexpr int P0 = (S0 + AL - 1) / AL * AL, P1 = (S1 + AL - 1) / AL * AL;
    __host__ __device__ static constexpr int off(int k)
    {
        int o = 0;
        for (int j = 0; j < k; ++j) o += ex(j) == 0 ? P0 : P1;
        return o;
    }
    static constexpr int ELEMS = 9 * P0 + 10 * P1;
    static constexpr int TX_BYTES = (9 * S0 + 10 * S1) * (int)sizeof(T);  // bytes one brick's copies deliver
    static constexpr int SMEM_BYTES = kBrickStages * ELEMS * (int)sizeof(T) + kBrickStages * 8 + 128;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
// Bounded wait for phase `parity` of barrier b: false if it did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity, long long limit)
{
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(smem_addr(b)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_box4(void *dst, const CUtensorMap *map, int x, int y, int z, int k, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(k), "r"(smem_addr(bar))
        : "memory");
}

// Limit of a stage wait: far above any copy's latency; reaching it flags an error.
constexpr long long kBrickWaitLimit = 1ll << 24;

// Blocks per multiprocessor the registers are sized for: 3 of 256 threads (85 registers a
// thread) for the 32- and 16-bit formats, 1 for FP64.
template <int STORE> constexpr int tma_min_blocks() { return STORE == ST_F64 ? 1 : 3; }

template <int COLL, int STORE, bool WX>
__global__ void __launch_bounds__(kBrickCells, tma_min_blocks<STORE>())
    step_kernel_tma(const __grid_constant__ InstanceDev I, const __grid_constant__ CUtensorMap map0_w0,
                    const __grid_constant__ CUtensorMap map0_w1, const __grid_constant__ CUtensorMap map1_w0,
                    const __grid_constant__ CUtensorMap map1_w1, const uint32_t *__restrict__ bricks, int nbricks,
                    int flip, unsigned *__restrict__ error)
{
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    using L = BrickStage<STORE>;
    extern __shared__ unsigned char smem_raw[];
    T *stage0 = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    uint64_t *full = reinterpret_cast<uint64_t *>(stage0 + kBrickStages * L::ELEMS);
    allow_next_step();
    const int tid = threadIdx.x;
    const int cx = tid % kBrickX, cy = (tid / kBrickX) % kBrickY, cz = tid / (kBrickX * kBrickY);
    if (tid == 0) {
        for (int s = 0; s < kBrickStages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const Par<R> P = load_par<R>(I);
    R rates[Q];
    load_rates<COLL>(I, rates);
    const int cur = I.phase ^ flip;
    const T *fs = reinterpret_cast<const T *>(cur ? I.f1 : I.f0);
    T *fd = reinterpret_cast<T *>(cur ? I.f0 : I.f1);
    const CUtensorMap *mw0 = cur ? &map1_w0 : &map0_w0;
    const CUtensorMap *mw1 = cur ? &map1_w1 : &map0_w1;
    // brick list entries pack the brick's coordinates: bx | by << 10 | bz << 21
    auto brick_origin = [&](uint32_t p, int &x0, int &y0, int &z0) {
        x0 = (int)(p & 1023u) * kBrickX;
        y0 = (int)((p >> 10) & 2047u) * kBrickY;
        z0 = (int)(p >> 21) * kBrickZ;
    };
    auto issue = [&](int brick, int s) {  // one thread: the 19 shifted boxes of a brick
        int x0, y0, z0;
        brick_origin(bricks[brick], x0, y0, z0);
        T *st = stage0 + s * L::ELEMS;
        mbar_expect_tx(&full[s], L::TX_BYTES);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int xo = ex(k) == 1 ? x0 - L::XA : x0;
            tma_box4(st + L::off(k), ex(k) == 0 ? mw0 : mw1, xo, y0 - ey(k), z0 - ez(k), k, &full[s]);
        }
    };
    // what a thread needs of its cell in a brick, read from tables no step writes: loaded
    // one brick ahead, while the previous brick is being finished
    auto locate = [&](int brick, WarpItem &m) {
        int x0, y0, z0;
        brick_origin(bricks[brick], x0, y0, z0);
        const uint32_t x = (uint32_t)(x0 + cx), y = (uint32_t)(y0 + cy), z = (uint32_t)(z0 + cz);
        const uint32_t cell = x + P.nx * (y + P.ny * z);
        const bool in_box = checked(I, cell, I.n32);
        // solid, boundary bits, boundary-table base of the row
        const uint4 sg = in_box ? I.seg[cell >> 5] : make_uint4(~0u, 0u, 0u, 0u);
        const bool live = !((sg.x >> cx) & 1u);
        m.cell = live ? cell : 0xFFFFFFFFu;
        m.xf = (x == 0 ? 1u : 0u) | (x == P.nx - 1 ? 2u : 0u);
        m.wm = 0u;
        m.off = 0u;
        m.inner = (y - 1u < P.ny - 2u) && (z - 1u < P.nz - 2u);
        m.wd = make_uint2(y, z);
        if (live && ((sg.y >> cx) & 1u)) {
            const uint32_t bi = sg.z + __popc(sg.y & ((1u << cx) - 1u));
            if (checked(I, bi, I.n_boundary)) {
                m.wm = I.bmask[bi];
                m.off = I.boff[bi];
                if (!checked(I, m.off + __popc(m.wm), I.n_links + 1u)) m.wm = 0u;
            }
        }
    };

    __shared__ int failed;
    if (tid == 0) failed = 0;
    WarpItem meta;
    if ((int)blockIdx.x < nbricks) locate((int)blockIdx.x, meta);
    wait_previous_step();  // the copies read what the previous step wrote
    if (tid == 0)
        for (int s = 0; s < kBrickStages; ++s)
            if ((int)blockIdx.x + s * (int)gridDim.x < nbricks) issue((int)blockIdx.x + s * (int)gridDim.x, s);

    int it = 0;
    for (int brick = blockIdx.x; brick < nbricks; brick += gridDim.x, ++it) {
        const int s = it % kBrickStages;
        const uint32_t parity = (uint32_t)(it / kBrickStages) & 1u;
        const bool live = meta.cell != 0xFFFFFFFFu;
        const uint32_t xf = meta.xf, y = meta.wd.x, z = meta.wd.y;
        // pulls whose source lies across a face: outside the box, read directly
        T raw[Q];
        uint32_t wrap = 0u;
        if (live && (xf != 0u || y == 0 || y == P.ny - 1 || z == 0 || z == P.nz - 1)) {
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const bool w = (ex(k) == 1 && (xf & 1u)) || (ex(k) == -1 && (xf & 2u)) || (ey(k) == 1 && y == 0) ||
                               (ey(k) == -1 && y == P.ny - 1) || (ez(k) == 1 && z == 0) ||
                               (ez(k) == -1 && z == P.nz - 1);
                wrap |= (w ? 1u : 0u) << k;
            }
            const Coord co = coord_of(P, meta.cell);
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if ((wrap >> k) & 1u) raw[k] = __ldg(fs + ((uint32_t)k * P.ks + co.pull(k)));
        }
        if (!mbar_wait_bounded(&full[s], parity, kBrickWaitLimit)) failed = 1;
        const T *st = stage0 + s * L::ELEMS;
        if (live) {
            const int row = cz * kBrickY + cy;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                if ((wrap >> k) & 1u) continue;
                const int xi = ex(k) == 0 ? cx : (ex(k) == 1 ? cx - 1 + L::XA : cx + 1);
                raw[k] = st[L::off(k) + row * (ex(k) == 0 ? L::W0 : L::W1) + xi];
            }
        }
        __syncthreads();  // stage s read by every thread (or a copy never completed)
        if (failed) {     // flag it, let the other stages' copies land, stop
            if (tid == 0) atomicOr(error, STATUS_TIMEOUT);
            for (int j = 1; j < kBrickStages; ++j)
                mbar_wait_bounded(&full[(it + j) % kBrickStages], (uint32_t)((it + j) / kBrickStages) & 1u,
                                  kBrickWaitLimit);
            return;
        }
        if (tid == 0) {  // refill stage s with the brick after next
            const int nb = brick + kBrickStages * (int)gridDim.x;
            if (nb < nbricks) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(nb, s);
            }
        }
        const WarpItem now = meta;
        if (brick + (int)gridDim.x < nbricks) locate(brick + (int)gridDim.x, meta);
        RedAcc<R> acc{};
        finish_item<COLL, STORE, KIND_AB, false, WX, R>(I, P, rates, raw, now, cx, fs, fd, nullptr, acc);
    }
}

}  // namespace lbm
