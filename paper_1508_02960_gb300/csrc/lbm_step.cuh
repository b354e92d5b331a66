// lbm_step.cuh -- the fused D3Q19 time step (Sec. 2: stream first, then collide, the two
// fused so that macroscopic values are never stored).
//
// Work decomposition.  An instance's cells are grouped in 32-cell segments; only the
// segments holding fluid are listed (all-solid segments cost nothing).  A warp takes
// chunks of consecutive list entries from a global counter; one lane per cell.
//
// Per fluid cell x and direction k (all arithmetic on deviations g = f - w rho0):
//   pull      g_k <- g~_k(x - e_k), plus +w_k delta_rho when the pull crosses the x
//             boundary from right to left and -w_k delta_rho the other way (Sec. 2.2.2,
//             Eqs. Periodicfunkown, PeriodicfunkownRight);
//   wall      if x - e_k is solid: SBB g_k <- g~_kbar(x) (Eq. noslip), or CLI
//             g_k <- c (g_kbar^in - g~_k(x)) + g~_kbar(x), c = (1-2q)/(1+2q) (Eq. CLI;
//             g_kbar^in is the streamed value from x_f2 = x + e_k);
//   moments   drho = sum g_k, u = rho0^-1 sum e_k g_k (Eq. Macro);
//   collide   SRT, TRT or MRT relaxation towards Eq. equilibrium;
//   store     A-B: to the other buffer; AA: in place (see below).
//
// Staged loads.  When rows are a multiple of 32 cells, every segment lies in one row, and
// the 32 pull sources of direction k are one contiguous run of the source row (shifted
// by one cell when e_kx != 0).  Lanes 0..18 then each issue one bulk asynchronous copy
// (cp.async.bulk, completion counted on an mbarrier) of their direction's run into a
// shared-memory ring of kStages segments, so the next segments' populations are in flight
// while the current one is collided, without holding registers.  Only the first and last
// cell of a row read their x-wrapped source directly.  Other boxes use direct loads.
//
// AA layout (in-place, one buffer).  PULL steps read g~_k(x - e_k) from slot kbar of
// x - e_k and push g~_k(x) into slot k of x + e_k; LOCAL steps read slot k and write
// slot kbar of x itself.  Every slot is then read and written by one thread only.  A
// push into a solid cell goes to the own slot kbar instead, which is exactly where the
// next step's bounce-back reads it.  CLI's own value g~_k(x) would be overwritten by the
// neighbour x + e_k in either step, so each CLI link keeps it in a side buffer (linkB).
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kStages = 2;                       // segments in flight per warp
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // bounded mbarrier wait: 2 s

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared-memory window layout of one segment: 19 direction slots of W elements; the 32
// cells of the segment sit at [H, H + 32), H elements (16 bytes) of halo on each side.
template <int STORE> struct Window {
    using T = typename Store<STORE>::T;
    static constexpr int H = 16 / (int)sizeof(T);
    static constexpr int W = 32 + 2 * H;
    static constexpr int stage_bytes = Q * W * (int)sizeof(T);
    // bytes copied per segment: e_kx == 0 -> 32 cells, else 32 + 2H cells
    static constexpr int bytes_pull = (9 * 32 + 10 * W) * (int)sizeof(T);
    static constexpr int bytes_local = Q * 32 * (int)sizeof(T);
};

inline size_t step_smem_bytes(int storage, int warps)
{
    const int stage = storage == ST_F64 ? Window<ST_F64>::stage_bytes
                      : storage == ST_F32 ? Window<ST_F32>::stage_bytes
                                          : Window<ST_F16>::stage_bytes;
    return (size_t)warps * (kStages * stage + kStages * 8);
}

// ---- inline PTX: mbarrier and bulk copies --------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity, at most kWaitLimitNs; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Collision of one cell, in place on g[] (deviations).  rho0 enters the equilibrium.
template <int COLL, typename R>
__device__ __forceinline__ void collide(R (&g)[Q], const InstanceDev &I, R drho, R ux, R uy, R uz)
{
    const R rho0 = R(I.rho0);
    const R uu = ux * ux + uy * uy + uz * uz;
    if constexpr (COLL == COLL_SRT) {
        const R om = R(I.omega);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R eu = R(ex(k)) * ux + R(ey(k)) * uy + R(ez(k)) * uz;
            const R geq = R(weight(k)) * (drho + rho0 * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu));
            g[k] = g[k] - om * (g[k] - geq);
        }
    } else if constexpr (COLL == COLL_TRT) {
        const R wp = R(I.omega), wm = R(I.omega_m);
        {
            const R geq0 = R(weight(0)) * (drho - rho0 * R(1.5) * uu);
            g[0] = g[0] - wp * (g[0] - geq0);
        }
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const int kb = k + 1;
            const R eu = R(ex(k)) * ux + R(ey(k)) * uy + R(ez(k)) * uz;
            const R eqp = R(weight(k)) * (drho + rho0 * (R(4.5) * eu * eu - R(1.5) * uu));
            const R eqm = R(weight(k)) * (rho0 * R(3) * eu);
            const R gp = R(0.5) * (g[k] + g[kb]);
            const R gm = R(0.5) * (g[k] - g[kb]);
            const R dp = wp * (gp - eqp);
            const R dm = wm * (gm - eqm);
            g[k] = g[k] - dp - dm;
            g[kb] = g[kb] - dp + dm;
        }
    } else {  // MRT: g~ = g - M^-1 S M (g - g^eq), M^-1 = M^T diag(1/|M_i|^2)
        R neq[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R eu = R(ex(k)) * ux + R(ey(k)) * uy + R(ez(k)) * uz;
            neq[k] = g[k] - R(weight(k)) * (drho + rho0 * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu));
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (i == 0 || i == 3 || i == 5 || i == 7) continue;  // conserved: m^neq = 0
            R m = R(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int c = mrt_m(i, k);
                if (c == 1) m += neq[k];
                else if (c == -1) m -= neq[k];
                else if (c != 0) m += R(c) * neq[k];
            }
            const R dm = R(I.s[i]) * m * (R(1) / R(mrt_norm2(i)));
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const int c = mrt_m(i, k);
                if (c == 1) g[k] -= dm;
                else if (c == -1) g[k] += dm;
                else if (c != 0) g[k] -= R(c) * dm;
            }
        }
    }
}

// Issue the bulk copies of one segment's pull windows into a stage (whole warp calls).
// Lane k < 19 copies direction k: the 32 sources of the segment's cells (A-B: array k at
// x - e_k; AA pull: array kbar at x - e_k; AA local: array k at x), widened by H cells on
// each side when e_kx != 0 so that every copy starts and ends on a 16-byte boundary.
template <int STORE, int KIND>
__device__ __forceinline__ void issue_segment(const InstanceDev &I, const typename Store<STORE>::T *fs, uint32_t seg,
                                              uint32_t stage_smem, uint32_t bar, int lane)
{
    using T = typename Store<STORE>::T;
    using Wn = Window<STORE>;
    const uint32_t cell0 = seg * 32u;
    const uint32_t row = fast_div(cell0, I.div_nx);
    const uint32_t x0 = cell0 - row * (uint32_t)I.nx;
    const uint32_t z = fast_div(row, I.div_ny);
    const uint32_t y = row - z * (uint32_t)I.ny;
    if (lane == 0) mbar_arrive_expect_tx(bar, KIND == KIND_AA_LOCAL ? Wn::bytes_local : Wn::bytes_pull);
    __syncwarp();
    if (lane < Q) {
        const int k = lane;
        uint32_t src_row = row;
        int arr = k, shift = 0;
        if (KIND != KIND_AA_LOCAL) {
            const int ky = ey_rt(k), kz = ez_rt(k);
            const uint32_t ny = I.ny, nz = I.nz;
            const uint32_t ys = ky == 1 ? (y == 0 ? ny - 1 : y - 1) : (ky == -1 ? (y == ny - 1 ? 0 : y + 1) : y);
            const uint32_t zs = kz == 1 ? (z == 0 ? nz - 1 : z - 1) : (kz == -1 ? (z == nz - 1 ? 0 : z + 1) : z);
            src_row = ys + ny * zs;
            if (KIND == KIND_AA_PULL) arr = opp_rt(k);
            shift = ex_rt(k) != 0;
        }
        const uint32_t start = (uint32_t)arr * I.n32 + src_row * (uint32_t)I.nx + x0 - (shift ? Wn::H : 0);
        const uint32_t n = shift ? Wn::W : 32;
        const uint32_t dst = stage_smem + (uint32_t)(k * Wn::W + (shift ? 0 : Wn::H)) * (uint32_t)sizeof(T);
        bulk_g2s(dst, fs + start, n * (uint32_t)sizeof(T), bar);
    }
}

// The fused step.  flip selects the A-B buffer pair (src = f[phase ^ flip]); reduce != 0
// makes every chunk write its FP64 partial sums (drho, u_x, u_y, u_z) and flags diverged
// cells in status[instance].  sched[0] is the chunk counter, sched[1] counts finished
// blocks; the last block resets both for the next launch.
template <int COLL, int STORE, int KIND>
__global__ void __launch_bounds__(256) step_kernel(const InstanceDev *__restrict__ table,
                                                   const TileDev *__restrict__ chunks, int nchunks, int chunk_segs,
                                                   int flip, int reduce, unsigned *__restrict__ status,
                                                   unsigned *__restrict__ sched)
{
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    using Wn = Window<STORE>;
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned char *wbase = smem_raw + (size_t)warp * kStages * Wn::stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)nwarps * kStages * Wn::stage_bytes) +
                     warp * kStages;
    if (lane == 0)
        for (int s = 0; s < kStages; ++s) mbar_init(smem_addr(&bars[s]), 1);
    mbar_fence_init();
    __syncwarp();
    uint32_t parity = 0;  // bit s: parity of the phase awaited next on stage s
    bool failed = false;

    while (!failed) {
        int c = 0;
        if (lane == 0) c = (int)atomicAdd(&sched[0], 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= nchunks) break;
        const TileDev chunk = chunks[c];
        const InstanceDev &I = table[chunk.inst];
        const uint32_t e0 = (uint32_t)chunk.seg0;
        const int n_e = min(chunk_segs, (int)(I.n_active - e0));
        const uint4 meta_l = lane < n_e ? I.aseg[e0 + lane] : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
        const uint32_t N = I.n32;
        const uint32_t nx = I.nx, ny = I.ny, nz = I.nz;
        const float sc = I.scale, isc = I.inv_scale;
        T *fs;  // state read this step
        T *fd;  // state written this step
        if constexpr (KIND == KIND_AB) {
            const int cur = I.phase ^ flip;
            fs = reinterpret_cast<T *>(cur ? I.f1 : I.f0);
            fd = reinterpret_cast<T *>(cur ? I.f0 : I.f1);
        } else {
            fs = fd = reinterpret_cast<T *>(I.f0);
        }
        const bool staged = I.staged != 0;
        const R dshift = R(I.delta_rho);
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;

        if (staged)
            for (int i = 0; i < kStages && i < n_e; ++i) {
                const uint32_t seg_i = __shfl_sync(0xffffffffu, meta_l.w, i);
                issue_segment<STORE, KIND>(I, fs, seg_i, smem_addr(wbase + i * Wn::stage_bytes),
                                           smem_addr(&bars[i]), lane);
            }

        for (int i = 0; i < n_e; ++i) {
            const int st = i % kStages;
            uint4 meta;
            meta.x = __shfl_sync(0xffffffffu, meta_l.x, i);
            meta.y = __shfl_sync(0xffffffffu, meta_l.y, i);
            meta.z = __shfl_sync(0xffffffffu, meta_l.z, i);
            meta.w = __shfl_sync(0xffffffffu, meta_l.w, i);
            const T *win = reinterpret_cast<const T *>(wbase + st * Wn::stage_bytes);
            if (staged) {
                const bool ok = mbar_wait(smem_addr(&bars[st]), (parity >> st) & 1u);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) atomicOr(status + chunk.inst, STATUS_TIMEOUT);
                    failed = true;
                    break;
                }
                parity ^= 1u << st;
            }

            if (!((meta.x >> lane) & 1u)) {
                const uint32_t cell = meta.w * 32u + lane;
                const uint32_t yz = fast_div(cell, I.div_nx);
                const uint32_t x = cell - yz * nx;
                const uint32_t z = fast_div(yz, I.div_ny);
                const uint32_t y = yz - z * ny;
                const uint32_t nxy = nx * ny;
                const uint32_t X[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
                const uint32_t Y[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
                const uint32_t Z[3] = {(z == 0 ? nz - 1 : z - 1) * nxy, z * nxy, (z == nz - 1 ? 0 : z + 1) * nxy};
                // pull source of direction k: x - e_k
                auto src_of = [&](int k) -> uint32_t { return X[1 - ex(k)] + Y[1 - ey(k)] + Z[1 - ez(k)]; };

                uint32_t wm = 0u, off = 0u;
                if ((meta.y >> lane) & 1u) {
                    const uint32_t b = meta.z + __popc(meta.y & ((1u << lane) - 1u));
                    wm = I.bmask[b];
                    off = I.boff[b];
                }

                R g[Q];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    if ((wm >> k) & 1u) {
                        g[k] = R(0);
                        continue;
                    }
                    const int arr = KIND == KIND_AA_PULL ? opp(k) : k;
                    R v;
                    if (staged) {
                        if (KIND == KIND_AA_LOCAL) {
                            v = S::cvt(win[k * Wn::W + Wn::H + lane], isc);
                        } else if ((ex(k) == 1 && x == 0) || (ex(k) == -1 && x == nx - 1)) {
                            v = S::load(fs + ((uint32_t)arr * N + src_of(k)), isc);  // x-wrapped source
                        } else {
                            v = S::cvt(win[k * Wn::W + Wn::H + lane - ex(k)], isc);
                        }
                    } else {
                        if constexpr (KIND == KIND_AA_LOCAL) v = S::load(fs + ((uint32_t)k * N + cell), isc);
                        else v = S::load(fs + ((uint32_t)arr * N + src_of(k)), isc);
                    }
                    if (ex(k) == 1 && x == 0) v += R(weight(k)) * dshift;
                    if (ex(k) == -1 && x == nx - 1) v -= R(weight(k)) * dshift;
                    g[k] = v;
                }
                if (wm) {
                    const R *linkc = reinterpret_cast<const R *>(I.linkc);
                    const T *linkB = reinterpret_cast<const T *>(I.linkB);
#pragma unroll
                    for (int k = 1; k < Q; ++k) {
                        if (!((wm >> k) & 1u)) continue;
                        const int kb = opp(k);
                        // own post-collision g~_kbar(x)
                        R C;
                        if constexpr (KIND == KIND_AB) C = S::load(fs + ((uint32_t)kb * N + cell), isc);
                        else C = S::load(fs + ((uint32_t)k * N + cell), isc);
                        R v = C;
                        if (I.wall == 1) {
                            const uint32_t l = off + __popc(wm & ((1u << k) - 1u));
                            const R c = linkc[l];
                            if (c != R(0)) {
                                R B;  // own post-collision g~_k(x)
                                if constexpr (KIND == KIND_AB) B = S::load(fs + ((uint32_t)k * N + cell), isc);
                                else B = S::load(linkB + l, isc);
                                v = c * (g[kb] - B) + C;
                            }
                        }
                        g[k] = v;
                    }
                }

                R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    drho += g[k];
                    if (ex(k)) jx += ex(k) > 0 ? g[k] : -g[k];
                    if (ey(k)) jy += ey(k) > 0 ? g[k] : -g[k];
                    if (ez(k)) jz += ez(k) > 0 ? g[k] : -g[k];
                }
                const R irho0 = R(1) / R(I.rho0);
                const R ux = jx * irho0, uy = jy * irho0, uz = jz * irho0;
                if (reduce) {
                    a0 += (double)drho;
                    a1 += (double)ux;
                    a2 += (double)uy;
                    a3 += (double)uz;
                    const R uu = ux * ux + uy * uy + uz * uz;
                    if (!(uu < R(0.09)) || !(drho == drho)) atomicOr(status + chunk.inst, STATUS_DIVERGED);
                }

                collide<COLL, R>(g, I, drho, ux, uy, uz);

#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const T v = S::pack(g[k], sc);
                    if constexpr (KIND == KIND_AB) {
                        fd[(uint32_t)k * N + cell] = v;
                    } else if constexpr (KIND == KIND_AA_LOCAL) {
                        fd[(uint32_t)opp(k) * N + cell] = v;
                    } else {
                        // push to x + e_k = pull source of kbar, or bounce into the own slot
                        if ((wm >> opp(k)) & 1u) fd[(uint32_t)opp(k) * N + cell] = v;
                        else fd[(uint32_t)k * N + src_of(opp(k))] = v;
                    }
                }
                if constexpr (KIND != KIND_AB) {
                    if (wm && I.wall == 1) {
                        T *linkB = reinterpret_cast<T *>(I.linkB);
#pragma unroll
                        for (int k = 1; k < Q; ++k) {
                            if (!((wm >> k) & 1u)) continue;
                            linkB[off + __popc(wm & ((1u << k) - 1u))] = S::pack(g[k], sc);
                        }
                    }
                }
            }
            // the stage is free once every lane has read it: refill it with segment i + kStages
            __syncwarp();
            if (staged && i + kStages < n_e) {
                const uint32_t seg_n = __shfl_sync(0xffffffffu, meta_l.w, i + kStages);
                issue_segment<STORE, KIND>(I, fs, seg_n, smem_addr(wbase + st * Wn::stage_bytes),
                                           smem_addr(&bars[st]), lane);
            }
        }
        if (failed) {
            // let copies still in flight land before the block leaves (bounded again)
            for (int s = 0; s < kStages; ++s) mbar_wait(smem_addr(&bars[s]), (parity >> s) & 1u);
            break;
        }
        if (reduce) {  // deterministic: per-lane sums over the chunk, then a fixed shuffle tree
            a0 = warp_sum(a0);
            a1 = warp_sum(a1);
            a2 = warp_sum(a2);
            a3 = warp_sum(a3);
            if (lane == 0) {
                double *p = I.partials + (size_t)chunk.local * 4;
                p[0] = a0;
                p[1] = a1;
                p[2] = a2;
                p[3] = a3;
            }
        }
    }

    // the last block to finish resets the work counter for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&sched[1], 1u);
        if (done == gridDim.x - 1) {
            sched[0] = 0u;
            sched[1] = 0u;
            __threadfence();
        }
    }
}

}  // namespace lbm
