// lbm_step.cuh -- the fused D3Q19 time step (Sec. 2: stream first, then collide, the two
// fused so that macroscopic values are never stored).  One thread per cell, one warp
// per 32-cell segment, one thread block per tile of segments; the grid is persistent
// and strides over the tile list, which may span many independent instances.
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
// AA layout (in-place, one buffer).  PULL steps read g~_k(x - e_k) from slot kbar of
// x - e_k and push g~_k(x) into slot k of x + e_k; LOCAL steps read slot k and write
// slot kbar of x itself.  Every slot is then read and written by one thread only.  A
// push into a solid cell goes to the own slot kbar instead, which is exactly where the
// next step's bounce-back reads it.  CLI's own value g~_k(x) would be overwritten by the
// neighbour x + e_k in either step, so each CLI link keeps it in a side buffer (linkB).
#pragma once

#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
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
// makes every tile write its FP64 partial sums (drho, u_x, u_y, u_z) and flags diverged
// cells in *status.
template <int COLL, int STORE, int KIND>
__global__ void __launch_bounds__(256) step_kernel(const InstanceDev *__restrict__ table,
                                                   const TileDev *__restrict__ tiles, int ntiles,
                                                   int flip, int reduce, unsigned *__restrict__ status)
{
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    __shared__ double red[32][4];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const TileDev tile = tiles[t];
        const InstanceDev &I = table[tile.inst];
        const uint32_t N = I.n32;
        const uint32_t nx = I.nx, ny = I.ny, nz = I.nz;
        const float sc = I.scale, isc = I.inv_scale;
        const uint4 meta = I.aseg[(uint32_t)tile.seg0 + warp];  // {solid, boundary, base, segment}
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;

        if (!((meta.x >> lane) & 1u)) {
            const uint32_t cell = meta.w * 32u + lane;
            const uint32_t yz = fast_div(cell, I.div_nx);
            const uint32_t x = cell - yz * nx;
            const uint32_t z = fast_div(yz, I.div_ny);
            const uint32_t y = yz - z * ny;
            // x-1, x, x+1 (periodic) and the row / plane offsets, all 32-bit element counts
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

            R g[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                if ((wm >> k) & 1u) {
                    g[k] = R(0);
                    continue;
                }
                const T *p;
                if constexpr (KIND == KIND_AB) p = fs + ((uint32_t)k * N + src_of(k));
                else if constexpr (KIND == KIND_AA_PULL) p = fs + ((uint32_t)opp(k) * N + src_of(k));
                else p = fs + ((uint32_t)k * N + cell);
                R v = S::load(p, isc);
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
                a0 = (double)drho;
                a1 = (double)ux;
                a2 = (double)uy;
                a3 = (double)uz;
                const R uu = ux * ux + uy * uy + uz * uz;
                if (!(uu < R(0.09)) || !(drho == drho)) atomicOr(status + tile.inst, STATUS_DIVERGED);
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

        if (reduce) {  // deterministic: fixed shuffle tree, then warps in order
            a0 = warp_sum(a0);
            a1 = warp_sum(a1);
            a2 = warp_sum(a2);
            a3 = warp_sum(a3);
            if (lane == 0) {
                red[warp][0] = a0;
                red[warp][1] = a1;
                red[warp][2] = a2;
                red[warp][3] = a3;
            }
            __syncthreads();
            if (threadIdx.x < 4) {
                double s = 0.0;
                for (int w = 0; w < nwarps; ++w) s += red[w][threadIdx.x];
                I.partials[(long long)tile.local * 4 + threadIdx.x] = s;
            }
            __syncthreads();
        }
    }
}

}  // namespace lbm
