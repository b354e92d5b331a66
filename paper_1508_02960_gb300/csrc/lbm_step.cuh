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
// Staged loads.  Each lane copies its cell's 19 pull sources with per-thread asynchronous
// copies (cp.async) into its own slots of a per-warp shared-memory ring of kStages
// segments, kStages - 1 segments ahead of the one being collided.  Populations in flight
// therefore hold no registers, and no lane reads another lane's slots.  16-bit formats
// copy the aligned 32-bit word holding the population and keep which half it is.
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

constexpr int kStages = 3;  // segments per warp: kStages - 1 in flight while one is collided

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One stage of a warp's ring: [19][32] copied words (8 bytes for FP64, else 4), then for
// 16-bit formats one 19-bit mask per lane telling which half of each word is wanted.
template <int STORE> struct Stage {
    using T = typename Store<STORE>::T;
    static constexpr int word = sizeof(T) == 8 ? 8 : 4;
    static constexpr bool halves = sizeof(T) == 2;
    static constexpr int bytes = Q * 32 * word + (halves ? 32 * 4 : 0);
};

inline size_t step_smem_bytes(int storage, int warps)
{
    const int stage = storage == ST_F64 ? Stage<ST_F64>::bytes
                      : storage == ST_F32 ? Stage<ST_F32>::bytes
                                          : Stage<ST_F16>::bytes;
    return (size_t)warps * kStages * stage;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Cell coordinates and the periodic x-1/x/x+1 offsets, row offsets y-1/y/y+1 and plane
// offsets z-1/z/z+1 (32-bit element counts).
struct Coord {
    uint32_t x, y, z;
    uint32_t X[3], Y[3], Z[3];
    __device__ __forceinline__ uint32_t pull(int k) const { return X[1 - ex(k)] + Y[1 - ey(k)] + Z[1 - ez(k)]; }
};
__device__ __forceinline__ Coord coord_of(const InstanceDev &I, uint32_t cell)
{
    Coord c;
    const uint32_t nx = I.nx, ny = I.ny, nz = I.nz, nxy = nx * ny;
    const uint32_t yz = fast_div(cell, I.div_nx);
    c.x = cell - yz * nx;
    c.z = fast_div(yz, I.div_ny);
    c.y = yz - c.z * ny;
    c.X[0] = c.x == 0 ? nx - 1 : c.x - 1;
    c.X[1] = c.x;
    c.X[2] = c.x == nx - 1 ? 0 : c.x + 1;
    c.Y[0] = (c.y == 0 ? ny - 1 : c.y - 1) * nx;
    c.Y[1] = c.y * nx;
    c.Y[2] = (c.y == ny - 1 ? 0 : c.y + 1) * nx;
    c.Z[0] = (c.z == 0 ? nz - 1 : c.z - 1) * nxy;
    c.Z[1] = c.z * nxy;
    c.Z[2] = (c.z == nz - 1 ? 0 : c.z + 1) * nxy;
    return c;
}

// Element index of the population a cell pulls for direction k: A-B array k at x - e_k;
// AA pull array kbar at x - e_k; AA local array k at x.
template <int KIND>
__device__ __forceinline__ uint32_t pull_index(uint32_t N, uint32_t cell, const Coord &c, int k)
{
    if constexpr (KIND == KIND_AA_LOCAL) return (uint32_t)k * N + cell;
    else if constexpr (KIND == KIND_AA_PULL) return (uint32_t)opp(k) * N + c.pull(k);
    else return (uint32_t)k * N + c.pull(k);
}

// Queue the asynchronous copies of one lane's 19 pull sources into a stage.
template <int STORE, int KIND>
__device__ __forceinline__ void issue_cell(const InstanceDev &I, const typename Store<STORE>::T *fs, uint4 meta,
                                           int lane, unsigned char *stage)
{
    using St = Stage<STORE>;
    if ((meta.x >> lane) & 1u) return;
    const uint32_t cell = meta.w * 32u + lane;
    const Coord c = coord_of(I, cell);
    const uint32_t base = smem_addr(stage) + (uint32_t)lane * St::word;
    uint32_t hmask = 0u;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const uint32_t idx = pull_index<KIND>(I.n32, cell, c, k);
        if constexpr (St::halves) {
            hmask |= (idx & 1u) << k;
            cp_async<4>(base + (uint32_t)(k * 32 * 4), fs + (idx & ~1u));
        } else {
            cp_async<St::word>(base + (uint32_t)(k * 32 * St::word), fs + idx);
        }
    }
    if constexpr (St::halves) reinterpret_cast<uint32_t *>(stage + Q * 32 * 4)[lane] = hmask;
}

// Read back population k of a lane from a stage.
template <int STORE>
__device__ __forceinline__ typename Store<STORE>::R staged_value(const unsigned char *stage, int k, int lane,
                                                                   uint32_t hmask, float isc)
{
    using S = Store<STORE>;
    using T = typename S::T;
    if constexpr (Stage<STORE>::halves) {
        const uint32_t w = reinterpret_cast<const uint32_t *>(stage)[k * 32 + lane];
        const unsigned short h = (unsigned short)(((hmask >> k) & 1u) ? (w >> 16) : (w & 0xFFFFu));
        T v;
        memcpy(&v, &h, 2);
        return S::cvt(v, isc);
    } else {
        return S::cvt(reinterpret_cast<const T *>(stage)[k * 32 + lane], isc);
    }
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
    using St = Stage<STORE>;
    extern __shared__ __align__(128) unsigned char smem_raw[];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *ring = smem_raw + (size_t)warp * kStages * St::bytes;

    while (true) {
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
        const uint32_t nx = I.nx;
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
        const R dshift = R(I.delta_rho);
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;

        auto meta_at = [&](int i) {
            uint4 m;
            m.x = __shfl_sync(0xffffffffu, meta_l.x, i);
            m.y = __shfl_sync(0xffffffffu, meta_l.y, i);
            m.z = __shfl_sync(0xffffffffu, meta_l.z, i);
            m.w = __shfl_sync(0xffffffffu, meta_l.w, i);
            return m;
        };
        // prologue: kStages - 1 segments in flight
#pragma unroll
        for (int i = 0; i < kStages - 1; ++i) {
            if (i < n_e) issue_cell<STORE, KIND>(I, fs, meta_at(i), lane, ring + i * St::bytes);
            cp_commit();
        }

        for (int i = 0; i < n_e; ++i) {
            const int j = i + kStages - 1;
            if (j < n_e) issue_cell<STORE, KIND>(I, fs, meta_at(j), lane, ring + (j % kStages) * St::bytes);
            cp_commit();
            cp_wait<kStages - 1>();  // this lane's copies of segment i have landed
            const uint4 meta = meta_at(i);
            const unsigned char *stage = ring + (i % kStages) * St::bytes;

            if (!((meta.x >> lane) & 1u)) {
                const uint32_t cell = meta.w * 32u + lane;
                const Coord co = coord_of(I, cell);
                const uint32_t x = co.x;
                uint32_t hmask = 0u;
                if constexpr (St::halves) hmask = reinterpret_cast<const uint32_t *>(stage + Q * 32 * 4)[lane];

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
                    R v = staged_value<STORE>(stage, k, lane, hmask, isc);
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
                            const R cq = linkc[l];
                            if (cq != R(0)) {
                                R B;  // own post-collision g~_k(x)
                                if constexpr (KIND == KIND_AB) B = S::load(fs + ((uint32_t)k * N + cell), isc);
                                else B = S::load(linkB + l, isc);
                                v = cq * (g[kb] - B) + C;
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
                        else fd[(uint32_t)k * N + co.pull(opp(k))] = v;
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
    cp_wait<0>();

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
