// lbm_step.cuh -- the fused D3Q19 time step (Sec. 2: stream first, then collide, the two
// fused so that macroscopic values are never stored).
//
// Work decomposition.  An instance's cells are grouped in 32-cell segments; only the
// segments holding fluid are listed (all-solid segments cost nothing).  One block per
// tile of consecutive list entries; each warp (one lane per cell) takes kSegsPerWarp of
// them and issues all their pulls before finishing the first, for load/compute overlap.
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
// The 19 pulls are issued unconditionally (a solid source slot holds 0 and is then
// replaced by the wall rule), so no load waits on the boundary table; the wall code runs
// only in warps whose segment holds a boundary cell.
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

// The step kernel uses no dynamic shared memory.
inline size_t step_smem_bytes(int, int) { return 0; }

// Instance parameters held in registers for the duration of a chunk.
template <typename R> struct Par {
    uint32_t ks, nx, ny, nz;
    FastDiv dnx, dny;
    R omega, omega_m, rho0, irho0, dshift;
    float sc, isc;
    int wall;
};

template <typename R> __device__ __forceinline__ Par<R> load_par(const InstanceDev &I)
{
    Par<R> p;
    p.ks = I.ks;
    p.nx = I.nx;
    p.ny = I.ny;
    p.nz = I.nz;
    p.dnx = I.div_nx;
    p.dny = I.div_ny;
    p.omega = R(I.omega);
    p.omega_m = R(I.omega_m);
    p.rho0 = R(I.rho0);
    p.irho0 = R(1) / R(I.rho0);
    p.dshift = R(I.delta_rho);
    p.sc = I.scale;
    p.isc = I.inv_scale;
    p.wall = I.wall;
    return p;
}

// Cell coordinates with the periodic x-1/x/x+1 offsets, row offsets y-1/y/y+1 and plane
// offsets z-1/z/z+1 (32-bit element counts).
struct Coord {
    uint32_t x;
    uint32_t X[3], Y[3], Z[3];
    __device__ __forceinline__ uint32_t pull(int k) const { return X[1 - ex(k)] + Y[1 - ey(k)] + Z[1 - ez(k)]; }
    __device__ __forceinline__ uint32_t push(int k) const { return X[1 + ex(k)] + Y[1 + ey(k)] + Z[1 + ez(k)]; }
};
template <typename R> __device__ __forceinline__ Coord coord_of(const Par<R> &p, uint32_t cell)
{
    Coord c;
    const uint32_t nx = p.nx, ny = p.ny, nz = p.nz, nxy = nx * ny;
    const uint32_t yz = fast_div(cell, p.dnx);
    c.x = cell - yz * nx;
    const uint32_t z = fast_div(yz, p.dny);
    const uint32_t y = yz - z * ny;
    c.X[0] = c.x == 0 ? nx - 1 : c.x - 1;
    c.X[1] = c.x;
    c.X[2] = c.x == nx - 1 ? 0 : c.x + 1;
    c.Y[0] = (y == 0 ? ny - 1 : y - 1) * nx;
    c.Y[1] = y * nx;
    c.Y[2] = (y == ny - 1 ? 0 : y + 1) * nx;
    c.Z[0] = (z == 0 ? nz - 1 : z - 1) * nxy;
    c.Z[1] = z * nxy;
    c.Z[2] = (z == nz - 1 ? 0 : z + 1) * nxy;
    return c;
}

// Blocks per multiprocessor the register allocation is sized for.
template <int STORE, int KIND> constexpr int step_min_blocks() { return STORE == ST_F64 ? 2 : 8; }

// Moments of the incoming populations (Eq. Macro), in deviation form.
template <typename R>
__device__ __forceinline__ void moments(const R (&g)[Q], R irho0, R &drho, R &ux, R &uy, R &uz)
{
    // sums and differences of opposite pairs: drho = g_0 + sum s_p, j = sum e_p d_p
    R d_sum = g[0], jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const R sp = g[k] + g[k + 1], dp = g[k] - g[k + 1];
        d_sum += sp;
        if (ex(k)) jx += ex(k) > 0 ? dp : -dp;
        if (ey(k)) jy += ey(k) > 0 ? dp : -dp;
        if (ez(k)) jz += ez(k) > 0 ? dp : -dp;
    }
    drho = d_sum;
    ux = jx * irho0;
    uy = jy * irho0;
    uz = jz * irho0;
}

// Collision of one cell, in place on g[] (deviations), Eqs. SRT, TRT, MRT with the
// equilibrium of Eq. equilibrium.  rates: the 19 MRT rates (MRT only).
template <int COLL, typename R>
__device__ __forceinline__ void collide(R (&g)[Q], const Par<R> &p, const R *rates, R drho, R ux, R uy, R uz)
{
    const R rho0 = p.rho0;
    const R uu = ux * ux + uy * uy + uz * uz;
    if constexpr (COLL == COLL_SRT) {
        const R om = p.omega;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R eu = R(ex(k)) * ux + R(ey(k)) * uy + R(ez(k)) * uz;
            const R geq = R(weight(k)) * (drho + rho0 * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu));
            g[k] = g[k] - om * (g[k] - geq);
        }
    } else if constexpr (COLL == COLL_TRT) {
        // symmetric part relaxes with omega+, antisymmetric part with omega- (Eq. TRT)
        const R wp = p.omega, wm = p.omega_m;
        const R base = drho - R(1.5) * rho0 * uu;     // drho + rho0 (-3/2 u.u)
        g[0] = g[0] - wp * (g[0] - R(weight(0)) * base);
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const int kb = k + 1;
            const R w = R(weight(k));
            const R eu = R(ex(k)) * ux + R(ey(k)) * uy + R(ez(k)) * uz;
            const R eqp = w * (base + R(4.5) * rho0 * eu * eu);   // (f_k^eq + f_kbar^eq) / 2
            const R eqm = (w * R(3) * rho0) * eu;                  // (f_k^eq - f_kbar^eq) / 2
            const R dp = wp * (R(0.5) * (g[k] + g[kb]) - eqp);
            const R dm = wm * (R(0.5) * (g[k] - g[kb]) - eqm);
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
            const R dm = rates[i] * m;  // rates[] already divided by |M_i|^2
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

// Process one cell whose 19 pulled populations are in g[] (already shifted): walls,
// moments, collision, stores.  Returns the moments for the reduction through rd..rz.
template <int COLL, int STORE, int KIND, typename R>
__device__ __forceinline__ void finish_cell(R (&g)[Q], const Par<R> &P, const R *rates, uint32_t cell, uint32_t x,
                                            const uint32_t *push_off, uint32_t wm, uint32_t off,
                                            const typename Store<STORE>::T *fs, typename Store<STORE>::T *fd,
                                            const R *linkc, typename Store<STORE>::T *linkB, int reduce,
                                            unsigned *status, R &rd, R &rx, R &ry, R &rz)
{
    using S = Store<STORE>;
    using T = typename S::T;
    const uint32_t KS = P.ks;
    if (wm) {  // walls: the solid sources read for these directions held 0
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (!((wm >> k) & 1u)) continue;
            const int kb = opp(k);
            // own post-collision g~_kbar(x)
            R C;
            if constexpr (KIND == KIND_AB) C = S::load(fs + ((uint32_t)kb * KS + cell), P.isc);
            else C = S::load(fs + ((uint32_t)k * KS + cell), P.isc);
            R v = C;
            if (P.wall == 1) {
                const uint32_t l = off + __popc(wm & ((1u << k) - 1u));
                const R cq = linkc[l];
                if (cq != R(0)) {
                    R B;  // own post-collision g~_k(x)
                    if constexpr (KIND == KIND_AB) B = S::load(fs + ((uint32_t)k * KS + cell), P.isc);
                    else B = S::load(linkB + l, P.isc);
                    v = cq * (g[kb] - B) + C;
                }
            }
            g[k] = v;
        }
    }

    R drho, ux, uy, uz;
    moments(g, P.irho0, drho, ux, uy, uz);
    if (reduce) {
        rd = drho;
        rx = ux;
        ry = uy;
        rz = uz;
        const R uu = ux * ux + uy * uy + uz * uz;
        if (!(uu < R(1)) || !(drho == drho)) atomicOr(status, STATUS_DIVERGED);
    }

    collide<COLL, R>(g, P, rates, drho, ux, uy, uz);

    // 16-bit formats round stochastically (see Store); wider formats round to nearest
    constexpr bool sr = sizeof(T) == 2;
    const uint32_t h = sr ? cell_hash(cell) : 0u;
    T packed[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k)
        packed[k] = sr ? S::pack_sr(g[k], P.sc, round_bits(h, k, float(g[k]))) : S::pack(g[k], P.sc);
    if constexpr (KIND == KIND_AA_PULL) {
        if (push_off) {  // interior cell: x + e_k is cell + e_k, except across the x faces
            const uint32_t cxm = x == 0 ? P.nx : 0u, cxp = x == P.nx - 1 ? P.nx : 0u;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                uint32_t idx = cell + push_off[k];
                if (ex(k) == 1) idx -= cxp;
                if (ex(k) == -1) idx += cxm;
                // push to x + e_k, or bounce into the own slot kbar when x + e_k is solid
                if ((wm >> opp(k)) & 1u) idx = (uint32_t)opp(k) * KS + cell;
                fd[idx] = packed[k];
            }
        } else {
            const Coord co = coord_of(P, cell);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                if ((wm >> opp(k)) & 1u) fd[(uint32_t)opp(k) * KS + cell] = packed[k];
                else fd[(uint32_t)k * KS + co.push(k)] = packed[k];
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if constexpr (KIND == KIND_AB) fd[(uint32_t)k * KS + cell] = packed[k];
            else fd[(uint32_t)opp(k) * KS + cell] = packed[k];
        }
    }
    if constexpr (KIND != KIND_AB) {
        if (wm && P.wall == 1) {
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                if (!((wm >> k) & 1u)) continue;
                linkB[off + __popc(wm & ((1u << k) - 1u))] = packed[k];
            }
        }
    }
}

// Instance parameters: from the device table (batches), or from a kernel argument in the
// constant bank (a single instance).
template <bool BATCH>
__device__ __forceinline__ const InstanceDev &instance_of(const InstanceDev *table, const InstanceDev &one, int i)
{
    if constexpr (BATCH) return table[i];
    else return one;
}

// The fused step.  One block per tile: kStepWarps warps, each taking kSegsPerWarp
// consecutive entries of the instance's active-segment list.  A warp first issues the
// pulls of all its segments, then finishes them one after the other.  Warps whose cells
// are all away from the y and z faces use precomputed offsets (cell + pull_off[k], with a
// fix-up on the first and last cell of a row); the others index through their periodic
// neighbours.  flip selects the A-B buffer pair (src = f[phase ^ flip]); reduce != 0 makes
// every tile write its FP64 partial sums (drho, u_x, u_y, u_z) and flags diverged cells in
// status[instance].
template <int COLL, int STORE, int KIND, bool BATCH>
__global__ void __launch_bounds__(kStepWarps * 32, step_min_blocks<STORE, KIND>())
    step_kernel(const InstanceDev *__restrict__ table, const __grid_constant__ InstanceDev one,
                const TileDev *__restrict__ tiles, int ntiles, int flip, int reduce, unsigned *__restrict__ status)
{
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    constexpr int NS = kSegsPerWarp;
    __shared__ double red[kStepWarps][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    const TileDev tile = tiles[t];
    const InstanceDev &I = instance_of<BATCH>(table, one, tile.inst);
    const Par<R> P = load_par<R>(I);
    R rates[Q];
    if constexpr (COLL == COLL_MRT) {
#pragma unroll
        for (int i = 0; i < Q; ++i) rates[i] = R(I.s[i]) / R(mrt_norm2(i));
    }
    const uint32_t KS = P.ks;
    T *fs;  // state read this step
    T *fd;  // state written this step
    if constexpr (KIND == KIND_AB) {
        const int cur = I.phase ^ flip;
        fs = reinterpret_cast<T *>(cur ? I.f1 : I.f0);
        fd = reinterpret_cast<T *>(cur ? I.f0 : I.f1);
    } else {
        fs = fd = reinterpret_cast<T *>(I.f0);
    }

    // descriptors of this warp's segments (entries past the list are all solid)
    const uint32_t e0 = (uint32_t)tile.seg0 + (uint32_t)(warp * NS);
    uint4 meta[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s)
        meta[s] = e0 + s < I.n_active ? I.aseg[e0 + s] : make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);

    // issue every pull of the warp's cells (unconditional: solid sources hold 0)
    R g[NS][Q];
    uint32_t cell[NS], xs[NS];
    bool inner[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        cell[s] = meta[s].w * 32u + lane;
        const uint32_t yz = fast_div(cell[s], P.dnx);
        const uint32_t x = cell[s] - yz * P.nx;
        const uint32_t z = fast_div(yz, P.dny);
        const uint32_t y = yz - z * P.ny;
        xs[s] = x;
        // every lane away from the y and z faces (solid lanes do not matter)
        const bool in_yz = ((meta[s].x >> lane) & 1u) || (y - 1u < P.ny - 2u && z - 1u < P.nz - 2u);
        inner[s] = __all_sync(0xffffffffu, in_yz);
        if ((meta[s].x >> lane) & 1u) continue;
        if (KIND != KIND_AA_LOCAL && inner[s]) {
            const uint32_t cxm = x == 0 ? P.nx : 0u, cxp = x == P.nx - 1 ? P.nx : 0u;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                uint32_t idx = cell[s] + I.pull_off[k];
                if (ex(k) == 1) idx += cxm;   // x - 1 wraps to the end of the row
                if (ex(k) == -1) idx -= cxp;  // x + 1 wraps to the start of the row
                g[s][k] = S::load(fs + idx, P.isc);
            }
        } else {
            const Coord co = coord_of(P, cell[s]);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                uint32_t idx;
                if constexpr (KIND == KIND_AA_LOCAL) idx = (uint32_t)k * KS + cell[s];
                else if constexpr (KIND == KIND_AA_PULL) idx = (uint32_t)opp(k) * KS + co.pull(k);
                else idx = (uint32_t)k * KS + co.pull(k);
                g[s][k] = S::load(fs + idx, P.isc);
            }
        }
        // pressure shift of pulls that cross the x boundary
        if (x == 0) {
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (ex(k) == 1) g[s][k] += R(weight(k)) * P.dshift;
        }
        if (x == P.nx - 1) {
#pragma unroll
            for (int k = 0; k < Q; ++k)
                if (ex(k) == -1) g[s][k] -= R(weight(k)) * P.dshift;
        }
    }

    R rd = R(0), rx = R(0), ry = R(0), rz = R(0);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if ((meta[s].x >> lane) & 1u) continue;
        uint32_t wm = 0u, off = 0u;
        if ((meta[s].y >> lane) & 1u) {
            const uint32_t b = meta[s].z + __popc(meta[s].y & ((1u << lane) - 1u));
            wm = I.bmask[b];
            off = I.boff[b];
        }
        finish_cell<COLL, STORE, KIND, R>(g[s], P, rates, cell[s], xs[s], inner[s] ? I.push_off : nullptr, wm, off,
                                          fs, fd, reinterpret_cast<const R *>(I.linkc),
                                          reinterpret_cast<T *>(I.linkB), reduce, status + tile.inst, rd, rx, ry,
                                          rz);
        if (reduce) {  // lane sums over the warp's segments, in order
            a0 += (double)rd;
            a1 += (double)rx;
            a2 += (double)ry;
            a3 += (double)rz;
        }
    }

    if (reduce) {  // deterministic: fixed shuffle tree, then the block's warps in order
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
            double sum = 0.0;
            for (int w = 0; w < kStepWarps; ++w) sum += red[w][threadIdx.x];
            I.partials[(size_t)tile.local * 4 + threadIdx.x] = sum;
        }
    }
}

}  // namespace lbm
