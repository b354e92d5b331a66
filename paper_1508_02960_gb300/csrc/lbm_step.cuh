// lbm_step.cuh -- the fused D3Q19 time step (Sec. 2: stream first, then collide, the two
// fused so that macroscopic values are never stored).
//
// Work decomposition.  An instance's fluid cells, in cell order, are dealt out 32 per
// warp (solid cells cost nothing and every lane has a cell, up to the last warp); runs of
// consecutive fluid cells keep the loads of a warp coalesced.  One block per tile of
// kStepWarps such work items, one per warp (one lane per cell).
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
// The 19 pulls are issued unconditionally: a solid source slot holds the own-cell part
// of the wall rule (A-B layout, see finish_cell) or is replaced by the wall rule (AA), so
// no pull waits on the boundary table; the wall code runs only for boundary cells.
//
// AA layout (in-place, one buffer).  PULL steps read g~_k(x - e_k) from slot kbar of
// x - e_k and push g~_k(x) into slot k of x + e_k; LOCAL steps read slot k and write
// slot kbar of x itself.  Every slot is then read and written by one thread only.
// Walls.  No fluid cell owns a slot of a solid cell, and slot kbar of the solid cell
// s = x - e_k belongs to the link (x, k) alone: a PULL step of x pulls direction k from
// it and pushes g~_kbar(x) into it (x + e_kbar = s).  Each step leaves the own-cell part S
// of the link's wall rule (wall_own_part, from the post-collision values in registers)
// where the next step's ordinary pull of direction k finds it: a LOCAL step stores S into
// slot kbar of s; a PULL step stores it into the own slot k, which no other cell reads or
// writes in a PULL step, besides its ordinary push of g~_kbar(x) into slot kbar of s.
// So the wall rule needs no load beyond the 19 pulls, as in the A-B layout, and the two
// layouts agree bit for bit.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Loads of population values.  An A-B step reads a buffer that no thread of the step
// writes, through the read-only (non-coherent) path.  The AA steps update their buffer, and
// the CLI link buffer, in place: a non-coherent load there is not allowed (the compiler may
// then order it after a store of the same thread), so they load plainly.
template <int KIND, typename T> __device__ __forceinline__ T ld_pop(const T *p)
{
    if constexpr (KIND == KIND_AB) return __ldg(p);
    else return *p;
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
    if constexpr (sizeof(R) == sizeof(float)) {
        p.omega = I.omega_f;
        p.omega_m = I.omega_m_f;
        p.rho0 = I.rho0_f;
        p.irho0 = I.irho0_f;
        p.dshift = I.delta_rho_f;
    } else {
        p.omega = I.omega;
        p.omega_m = I.omega_m;
        p.rho0 = I.rho0;
        p.irho0 = I.irho0;
        p.dshift = I.delta_rho;
    }
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

// The static tables a step reads (work list, boundary table, wall-rule coefficients) are
// small next to the populations streaming through L2 every step; they are loaded with an
// evict-last L2 policy so that they stay resident from one step to the next.
__device__ __forceinline__ uint64_t l2_keep_policy()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t *a, uint64_t pol)
{
    uint32_t v;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_keep(const float *a, uint64_t pol)
{
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *a, uint64_t pol)
{
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ld_keep(const uint2 *a, uint64_t pol)
{
    uint2 v;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(pol));
    return v;
}

// Blocks per multiprocessor the register allocation is sized for.  The plain SRT and TRT
// step of the 32- and 16-bit formats: 36 warps (56 registers a thread; measured 1-6 %
// faster than 32 warps at 64 registers, and 40 warps spill).  MRT, the reducing and
// interpolated-wall variants and the in-place 16-bit steps keep 32 warps (64 registers),
// where 56 would spill (MRT at 56 spills 136 bytes and ran 3 % slower).  FP64: 8 warps.
#ifndef LBM_STEP_WARPS_PER_SM
#define LBM_STEP_WARPS_PER_SM 36
#endif
template <int STORE, int COLL, bool RED, bool WX, int WARPS = kStepWarps, int KIND = KIND_AB, bool BATCH = false>
constexpr int step_min_blocks()
{
    // the in-place steps of the 16-bit formats (stochastic rounding, scaling) spill at 56
    // registers: 32 warps, measured 0.3-3 % faster than 36; so does a batch's local step,
    // whose parameters come from the instance table instead of the constant bank (60 bytes
    // at 56 registers; 32 warps measured 3-6 % faster on batches of 2-4 cells)
    constexpr bool wide = RED || WX || COLL == COLL_MRT || ((STORE == ST_F16 || STORE == ST_BF16) && KIND != KIND_AB) ||
                          (BATCH && KIND == KIND_AA_LOCAL);
    return (STORE == ST_F64 ? 8 : wide ? 32 : LBM_STEP_WARPS_PER_SM) / WARPS;
}

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
        // Every row of M is even or odd in e (mrt_even), so a moment takes the sums (even
        // rows) or the differences (odd rows) of the opposite pairs of g - g^eq, and the
        // relaxation goes back to a pair as its even part plus or minus its odd part: the
        // same matrix in half the operations of the full 19 x 19 products.
        R sp[Q / 2 + 1], dp[Q / 2 + 1];
        sp[0] = g[0] - R(weight(0)) * (drho - R(1.5) * rho0 * uu);
        dp[0] = R(0);
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const R w = R(weight(k));
            const R eu = R(ex(k)) * ux + R(ey(k)) * uy + R(ez(k)) * uz;
            const R eqs = w * (drho + rho0 * (R(4.5) * eu * eu - R(1.5) * uu));  // even part of f^eq
            const R eqd = w * rho0 * R(3) * eu;                                  // odd part of f^eq
            const R nk = g[k] - (eqs + eqd), nkb = g[k + 1] - (eqs - eqd);
            sp[(k + 1) / 2] = nk + nkb;
            dp[(k + 1) / 2] = nk - nkb;
        }
        R dm[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            dm[i] = R(0);
            if (i == 0 || i == 3 || i == 5 || i == 7) continue;  // conserved: m^neq = 0
            R m = R(0);
#pragma unroll
            for (int p = 0; p <= Q / 2; ++p) {
                const int c = mrt_m(i, p == 0 ? 0 : 2 * p - 1);
                const R v = mrt_even(i) ? sp[p] : dp[p];
                if (c == 1) m += v;
                else if (c == -1) m -= v;
                else if (c != 0) m += R(c) * v;
            }
            dm[i] = rates[i] * m;  // rates[] already divided by |M_i|^2
        }
#pragma unroll
        for (int p = 0; p <= Q / 2; ++p) {
            const int k = p == 0 ? 0 : 2 * p - 1;
            R ev = R(0), od = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (i == 0 || i == 3 || i == 5 || i == 7) continue;
                const int c = mrt_m(i, k);
                if (c == 0) continue;
                const R t = c == 1 ? dm[i] : (c == -1 ? -dm[i] : R(c) * dm[i]);
                if (mrt_even(i)) ev += t;
                else od += t;
            }
            if (p == 0) {
                g[0] -= ev;
            } else {
                g[k] -= ev + od;
                g[k + 1] -= ev - od;
            }
        }
    }
}

// Periodic wrap of c + d into [0, n) for |d| <= 2 (any n >= 1).
__device__ __forceinline__ int wrap2(int c, int n)
{
    if (c < 0) c += n;
    if (c < 0) c += n;
    if (c >= n) c -= n;
    if (c >= n) c -= n;
    return c;
}

// Cells of the periodic images of x + e_k and x + 2 e_k (x_f2, x_f3 of the link (x, kbar));
// xv2 / xv3 receive their virtual x coordinates (outside [0, nx) across an x face).
template <typename R>
__device__ __forceinline__ void link_neighbours(const Par<R> &P, uint32_t cell, int k, uint32_t &c2, int &xv2,
                                                uint32_t &c3, int &xv3)
{
    const uint32_t yz = fast_div(cell, P.dnx);
    const int x = (int)(cell - yz * P.nx);
    const uint32_t zz = fast_div(yz, P.dny);
    const int y = (int)(yz - zz * P.ny), z = (int)zz;
    const int nx = (int)P.nx, ny = (int)P.ny, nz = (int)P.nz;
    xv2 = x + ex(k);
    xv3 = x + 2 * ex(k);
    c2 = (uint32_t)wrap2(xv2, nx) + P.nx * ((uint32_t)wrap2(y + ey(k), ny) + P.ny * (uint32_t)wrap2(z + ez(k), nz));
    c3 = (uint32_t)wrap2(xv3, nx) +
         P.nx * ((uint32_t)wrap2(y + 2 * ey(k), ny) + P.ny * (uint32_t)wrap2(z + 2 * ez(k), nz));
}

// Population of direction m read at a virtual x coordinate: the pressure shift of a value
// that crossed an x face (Sec. 2.2.2, as for the pulls).
template <typename R> __device__ __forceinline__ R shifted(R v, int xv, int nx, R w_dshift)
{
    return xv < 0 ? v + w_dshift : (xv >= nx ? v - w_dshift : v);
}

// The neighbour terms alpha P2 + beta P3 + delta B2 + zeta J2 of an interpolated wall rule
// (kLinkW) of link (x, kbar), x - e_k solid, added to v (which holds S).  The loads the
// rule may need are issued before its coefficients arrive (a coefficient of 0 -- a
// fallback -- multiplies a finite value read from a solid cell's slot).
template <int STORE, typename R>
__device__ __forceinline__ R wall_neighbour_terms(const Par<R> &P, int wall, const R *lw, int k, uint32_t cell,
                                                  const R (&g)[Q], const typename Store<STORE>::T *fs, R v)
{
    using S = Store<STORE>;
    const int kb = opp(k);
    const uint64_t keep = l2_keep_policy();
    if (wall == 3 || wall == 5) {  // QIBB, MR: P3 = g~_kbar(x_f3), B2 = g~_k(x_f2)
        int xv2, xv3;
        uint32_t c2, c3;
        link_neighbours(P, cell, k, c2, xv2, c3, xv3);
        const R b2 = shifted(S::load(fs + ((uint32_t)k * P.ks + c2), P.isc), xv2, (int)P.nx,
                             R(weight(k)) * P.dshift);
        const R p3 = shifted(S::load(fs + ((uint32_t)kb * P.ks + c3), P.isc), xv3, (int)P.nx,
                             R(weight(kb)) * P.dshift);
        v = fma_r(ld_keep(lw + LW_ALPHA, keep), g[kb], v);
        v = fma_r(ld_keep(lw + LW_BETA, keep), p3, v);
        v = fma_r(ld_keep(lw + LW_DELTA, keep), b2, v);
    } else if (wall == 4) {  // IEBB: J2 = e_kbar . (momentum of x_f2); the shift carries none
        int xv2, xv3;
        uint32_t c2, c3;
        link_neighbours(P, cell, k, c2, xv2, c3, xv3);
        R j2 = R(0);
#pragma unroll
        for (int m = 1; m < Q; ++m) {
            const int d = ex(kb) * ex(m) + ey(kb) * ey(m) + ez(kb) * ez(m);
            if (d == 0) continue;
            const R gm = S::load(fs + ((uint32_t)m * P.ks + c2), P.isc);
            j2 += d > 0 ? (d == 1 ? gm : R(d) * gm) : (d == -1 ? -gm : R(d) * gm);
        }
        v = fma_r(ld_keep(lw + LW_ZETA, keep), j2, v);
    } else {  // LIBB
        v = fma_r(ld_keep(lw + LW_ALPHA, keep), g[kb], v);
    }
    return v;
}

// The own-cell part S of an interpolated wall rule (kLinkW) from the cell's post-collision
// values g[] and its moments drho, u at this step.
template <typename R>
__device__ __forceinline__ R wall_own_part_w(const Par<R> &P, const R *lw, int k, const R (&g)[Q], R drho, R ux, R uy,
                                             R uz)
{
    const int kb = opp(k);
    const uint64_t keep = l2_keep_policy();
    R sv = fma_r(ld_keep(lw + LW_GAMMA, keep), g[k], ld_keep(lw + LW_EPS, keep) * g[kb]);
    const R X = ld_keep(lw + LW_X, keep);
    if (X != R(0)) {
        const R eu = R(ex(kb)) * ux + R(ey(kb)) * uy + R(ez(kb)) * uz;
        const R uu = ux * ux + uy * uy + uz * uz;
        const R fst = drho + P.rho0 * (ld_keep(lw + LW_THETA, keep) * eu + R(4.5) * eu * eu - R(1.5) * uu);
        sv = fma_r(X * R(weight(kb)), fst, sv);
    }
    return sv;
}

// Process one cell whose 19 pulled populations are in g[] (already shifted, except the
// wall directions): walls, moments, collision, stores.  When RED is set, returns the
// moments through rd..rz and the momentum the cell's wall links hand to the solid in this
// step through fm[3]: a link (x, kbar) with x - e_k solid carries g~_kbar(x) into the wall
// and brings the new g_k back, so the solid gains e_kbar (g~_kbar(x) + g_k).  (Deviations
// suffice: the 2 w rho0 of full populations sums to zero over a periodic domain.)
//
// Walls in the A-B layout.  The pull of a wall direction k reads slot k of the solid cell
// x - e_k, which no fluid cell owns; every step leaves there the own-cell part S of the
// wall rule for the next step (wall_own_part, from its post-collision values in
// registers), so SBB needs no wall code at all and CLI adds c g_kbar^in, g_kbar^in being
// the cell's ordinary pull from x_f2 = x + e_k.  A state set from outside (initial state,
// imported populations) gets these slots from wall_prepare_kernel.
// Walls in the AA layout: the same, with S where the AA layout's pull reads (see above).
template <int COLL, int STORE, int KIND, bool RED, bool WX, typename R>
__device__ __forceinline__ void finish_cell(const InstanceDev &I, R (&g)[Q], const Par<R> &P, const R *rates,
                                            uint32_t cell, uint32_t xf,
                                            bool inner, const uint32_t *pull_off, const uint32_t *push_off,
                                            uint32_t wm, uint32_t off, const typename Store<STORE>::T *fs,
                                            typename Store<STORE>::T *fd, const R *linkc, const R *linkw,
                                            unsigned *status, R &rd, R &rx, R &ry, R &rz, R (&fm)[3])
{
    using S = Store<STORE>;
    using T = typename S::T;
    const uint32_t KS = P.ks;
    if (wm) {
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (!((wm >> k) & 1u)) continue;
            const int kb = opp(k);
            const uint32_t l = off + __popc(wm & ((1u << k) - 1u));
            const R cq = P.wall == 1 ? ld_keep(linkc + l, l2_keep_policy()) : R(0);
            R v, C;
            v = g[k];  // S, left by the previous step where this pull reads
            if (WX && KIND == KIND_AB && P.wall >= 2)
                v = wall_neighbour_terms<STORE>(P, P.wall, linkw + (size_t)l * kLinkW, k, cell, g, fs, v);
            else if (cq != R(0)) v = fma_r(cq, g[kb], v);
            if constexpr (RED) {
                // the own post-collision g~_kbar(x) of the previous step (momentum exchange):
                // A-B: own slot kbar; AA after a LOCAL step: own slot k; AA after a PULL
                // step: where it was pushed, slot kbar of x - e_k
                uint32_t ci;
                if constexpr (KIND == KIND_AB) ci = (uint32_t)kb * KS + cell;
                else if constexpr (KIND == KIND_AA_PULL) ci = (uint32_t)k * KS + cell;
                else ci = (uint32_t)kb * KS + coord_of(P, cell).pull(k);
                C = checked(I, ci - (KIND == KIND_AA_PULL ? (uint32_t)k : (uint32_t)kb) * KS, I.n32)
                        ? S::cvt(ld_pop<KIND>(fs + ci), P.isc)
                        : R(0);
            }
            g[k] = v;
            if constexpr (RED) {  // e_kbar = -e_k
                const R m = C + v;
                if (ex(k)) fm[0] += ex(k) > 0 ? -m : m;
                if (ey(k)) fm[1] += ey(k) > 0 ? -m : m;
                if (ez(k)) fm[2] += ez(k) > 0 ? -m : m;
            }
        }
    }

    R drho, ux, uy, uz;
    moments(g, P.irho0, drho, ux, uy, uz);
    if constexpr (RED) {
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
            const uint32_t cxm = (xf & 1u) ? P.nx : 0u, cxp = (xf & 2u) ? P.nx : 0u;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                uint32_t idx = cell + push_off[k];
                if (ex(k) == 1) idx -= cxp;
                if (ex(k) == -1) idx += cxm;
                if (checked(I, idx - (uint32_t)k * KS, I.n32)) fd[idx] = packed[k];
            }
        } else {
            const Coord co = coord_of(P, cell);
#pragma unroll
            for (int k = 0; k < Q; ++k) fd[(uint32_t)k * KS + co.push(k)] = packed[k];
        }
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if constexpr (KIND == KIND_AB) fd[(uint32_t)k * KS + cell] = packed[k];
            else fd[(uint32_t)opp(k) * KS + cell] = packed[k];
        }
    }
    if constexpr (KIND == KIND_AA_PULL) {
        // the own-cell part of every wall rule into the own slot k, which the next (LOCAL)
        // step's pull of direction k reads
        if (wm) {
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                if (!((wm >> k) & 1u)) continue;
                const uint32_t l = off + __popc(wm & ((1u << k) - 1u));
                const R cq = P.wall == 1 ? ld_keep(linkc + l, l2_keep_policy()) : R(0);
                const R sv = wall_own_part(P.wall, cq, g[opp(k)], g[k]);
                fd[(uint32_t)k * KS + cell] = sr ? S::pack_sr(sv, P.sc, round_bits(h, k, float(sv))) : S::pack(sv, P.sc);
            }
        }
    }
    if constexpr (KIND != KIND_AA_PULL) {
        // A-B, and AA LOCAL steps: the own-cell part of every wall rule into the solid slot
        // the next step's pull of direction k reads (A-B: slot k of x - e_k in the other
        // buffer; AA: slot kbar of x - e_k)
        if (wm) {
            const uint32_t cxm = (xf & 1u) ? P.nx : 0u, cxp = (xf & 2u) ? P.nx : 0u;
            Coord co;
            if (!inner) co = coord_of(P, cell);
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                if (!((wm >> k) & 1u)) continue;
                const uint32_t l = off + __popc(wm & ((1u << k) - 1u));
                R sv;
                if (WX && P.wall >= 2) {
                    sv = wall_own_part_w(P, linkw + (size_t)l * kLinkW, k, g, drho, ux, uy, uz);
                } else {
                    const R cq = P.wall == 1 ? ld_keep(linkc + l, l2_keep_policy()) : R(0);
                    sv = wall_own_part(P.wall, cq, g[opp(k)], g[k]);
                }
                // the slot direction: k in A-B, kbar in AA (pull_off of an AA instance
                // addresses slot kbar of x - e_k)
                const uint32_t d = KIND == KIND_AB ? (uint32_t)k : (uint32_t)opp(k);
                uint32_t idx;
                if (inner) {
                    idx = cell + pull_off[k];
                    if (ex(k) == 1) idx += cxm;
                    if (ex(k) == -1) idx -= cxp;
                } else {
                    idx = d * KS + co.pull(k);
                }
                if (checked(I, idx - d * KS, I.n32))
                    fd[idx] = sr ? S::pack_sr(sv, P.sc, round_bits(h, k, float(sv))) : S::pack(sv, P.sc);
            }
        }
    }
}

// One warp's work item: 32 fluid cells of the work list (w = its index), their raw pulled
// values (see pull_item) and what the finish needs.
struct WarpItem {
    uint32_t cell;     // this lane's cell (0xFFFFFFFF: padding lane)
    uint32_t xf;       // bit 0: x = 0, bit 1: x = nx - 1 (pulls and pushes across the x faces)
    uint32_t wm, off;  // boundary cell: wall mask (bit k: x - e_k solid) and first link; else 0
    uint2 wd;          // tiles: the warp's entry (.y its first link); bricks: y and z of the cell
    bool inner;        // every lane away from the y and z faces
};

// Locate one work item: this lane's cell, its x-face flags, wall mask and links, and
// whether every lane is away from the y and z faces, all precomputed in the work list (one
// entry per warp and one per lane, no dependent load and no division), which no step writes.
template <typename R>
__device__ __forceinline__ void locate_item(const InstanceDev &I, const Par<R> &P, const uint2 *flane,
                                            const uint2 *fwarp, uint32_t w, int lane, WarpItem &it)
{
    const uint64_t keep = l2_keep_policy();
    const bool w_ok = checked(I, w, I.n_fwarps_padded);
    it.wd = w_ok ? ld_keep(fwarp + w, keep) : make_uint2(0u, 0u);
    const uint2 e = w_ok ? ld_keep(flane + (w * 32u + (uint32_t)lane), keep) : make_uint2(0xFFFFFFFFu, 0u);
    const bool live = e.x != 0xFFFFFFFFu;
    it.cell = live ? (e.x & 0x0FFFFFFFu) : 0xFFFFFFFFu;
    if (live && !checked(I, it.cell, I.n32)) it.cell = 0xFFFFFFFFu;
    it.xf = (e.x >> 28) & 3u;
    it.inner = ((e.x >> 30) & 1u) != 0u;  // the same in all live lanes of the item
    it.wm = e.y & 0x7FFFFu;
    it.off = it.wd.y + (e.y >> 19);
    // every link of the cell within the link tables
    if (it.wm && !checked(I, it.off + __popc(it.wm), I.n_links + 1u)) it.wm = 0u;
}

// Issue the 19 pulls of a located work item into raw[] (storage type, converted in
// finish_item).  Unconditional: solid sources hold 0.  Warps whose cells are all away from
// the y and z faces index through precomputed offsets (cell + pull_off[k], with a fix-up on
// the first and last cell of a row); the others through their periodic neighbours.
template <int STORE, int KIND, typename R>
__device__ __forceinline__ void pull_item(const InstanceDev &I, const Par<R> &P, const typename Store<STORE>::T *fs,
                                          const WarpItem &it, typename Store<STORE>::T (&raw)[Q])
{
    if (it.cell == 0xFFFFFFFFu) return;
    if (KIND != KIND_AA_LOCAL && it.inner) {
        const uint32_t cxm = (it.xf & 1u) ? P.nx : 0u, cxp = (it.xf & 2u) ? P.nx : 0u;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            uint32_t idx = it.cell + I.pull_off[k];
            if (ex(k) == 1) idx += cxm;   // x - 1 wraps to the end of the row
            if (ex(k) == -1) idx -= cxp;  // x + 1 wraps to the start of the row
            const uint32_t d = KIND == KIND_AA_PULL ? (uint32_t)opp(k) : (uint32_t)k;
            raw[k] = checked(I, idx - d * P.ks, I.n32) ? ld_pop<KIND>(fs + idx) : typename Store<STORE>::T{};
        }
    } else {
        const Coord co = coord_of(P, it.cell);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            uint32_t idx;
            if constexpr (KIND == KIND_AA_LOCAL) idx = (uint32_t)k * P.ks + it.cell;
            else if constexpr (KIND == KIND_AA_PULL) idx = (uint32_t)opp(k) * P.ks + co.pull(k);
            else idx = (uint32_t)k * P.ks + co.pull(k);
            const uint32_t d = KIND == KIND_AA_PULL ? (uint32_t)opp(k) : (uint32_t)k;
            raw[k] = checked(I, idx - d * P.ks, I.n32) ? ld_pop<KIND>(fs + idx) : typename Store<STORE>::T{};
        }
    }
}

// Per-lane values of the reduction (RED steps) in the compute type: one cell a lane.
template <typename R> struct RedAcc {
    R v[RED_F + 3];
};

// Finish one work item pulled by pull_item: convert, pressure shift of the pulls that
// crossed the x boundary, walls, collision, stores; with RED, add the lane's moments and
// momentum exchange to acc.
template <int COLL, int STORE, int KIND, bool RED, bool WX, typename R>
__device__ __forceinline__ void finish_item(const InstanceDev &I, const Par<R> &P, const R *rates,
                                            const typename Store<STORE>::T (&raw)[Q], const WarpItem &it, int lane,
                                            const typename Store<STORE>::T *fs, typename Store<STORE>::T *fd,
                                            unsigned *status, RedAcc<R> &acc)
{
    using S = Store<STORE>;
    using T = typename S::T;
    if (it.cell == 0xFFFFFFFFu) return;
    R g[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) g[k] = S::cvt(raw[k], P.isc);
    // pressure shift of the pulls that crossed the x boundary (wall directions take their
    // value from the wall rule instead)
    const uint32_t wm = it.wm;
    if (it.xf & 1u) {
#pragma unroll
        for (int k = 0; k < Q; ++k)
            if (ex(k) == 1 && !((wm >> k) & 1u)) g[k] += R(weight(k)) * P.dshift;
    }
    if (it.xf & 2u) {
#pragma unroll
        for (int k = 0; k < Q; ++k)
            if (ex(k) == -1 && !((wm >> k) & 1u)) g[k] -= R(weight(k)) * P.dshift;
    }
    R rd = R(0), rx = R(0), ry = R(0), rz = R(0);
    R fm[3] = {R(0), R(0), R(0)};
    finish_cell<COLL, STORE, KIND, RED, WX, R>(I, g, P, rates, it.cell, it.xf, it.inner, I.pull_off,
                                               it.inner ? I.push_off : nullptr, wm, it.off, fs, fd,
                                               reinterpret_cast<const R *>(I.linkc),
                                               reinterpret_cast<const R *>(I.linkw), status, rd, rx, ry, rz, fm);
    if constexpr (RED) {
        acc.v[RED_DRHO] += rd;
        acc.v[RED_U + 0] += rx;
        acc.v[RED_U + 1] += ry;
        acc.v[RED_U + 2] += rz;
#pragma unroll
        for (int d = 0; d < 3; ++d) acc.v[RED_F + d] += fm[d];
    }
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Warp sum of float-float values hi + lo (fixed butterfly; every lane ends with the same
// pair, the exact TwoSum error being unique).  Each addition keeps its rounding error, so
// hi + lo is the sum to about 2^-48 of the magnitudes added, close to an FP64 sum, on the
// FP32 pipes (GB300's FP64 rate made the FP64 butterfly the cost of the reducing step).
__device__ __forceinline__ void warp_sum_ff(float &hi, float &lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        float sh, se;
        two_sum(hi, h2, sh, se);
        se = __fadd_rn(se, __fadd_rn(lo, l2));
        two_sum(sh, se, hi, lo);
    }
}

// Block sum of the lanes' values of one tile (fixed shuffle tree, then the warps in order)
// to partials[tile] in FP64; every thread of the block calls it.  FP64 lanes sum in FP64;
// FP32 lanes sum in float-float within the warp, then in FP64.
template <typename R>
__device__ __forceinline__ void reduce_tile(const RedAcc<R> &acc, double *partials, long long tile)
{
    __shared__ double red[kStepWarps][RED_F + 3];  // the reducing step runs kStepWarps-warp blocks
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[RED_F + 3];
#pragma unroll
    for (int d = 0; d < RED_F + 3; ++d) {
        if constexpr (sizeof(R) == sizeof(double)) {
            v[d] = warp_sum((double)acc.v[d]);
        } else {
            float hi = (float)acc.v[d], lo = 0.0f;
            warp_sum_ff(hi, lo);
            v[d] = (double)hi + (double)lo;
        }
    }
    if (lane == 0)
#pragma unroll
        for (int d = 0; d < RED_F + 3; ++d) red[warp][d] = v[d];
    __syncthreads();
    if (threadIdx.x < RED_F + 3) {
        double sum = 0.0;
        for (int w = 0; w < kStepWarps; ++w) sum += red[w][threadIdx.x];
        partials[tile * kRedSlots + threadIdx.x] = sum;
    }
}

template <int COLL, typename R> __device__ __forceinline__ void load_rates(const InstanceDev &I, R (&rates)[Q])
{
    if constexpr (COLL == COLL_MRT) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if constexpr (sizeof(R) == sizeof(float)) rates[i] = I.rate_f[i];
            else rates[i] = I.rate_d[i];
        }
    }
}

// Programmatic dependent launch (sm_90 and later): a step lets the next step's blocks be
// scheduled as soon as all of its own blocks are running, and a step waits for the
// previous one to complete (with its memory visible) only before its first population
// load.  Between the two, a block reads its tile and work list, which no step writes.
__device__ __forceinline__ void allow_next_step() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_previous_step() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <bool BATCH>
__device__ __forceinline__ const InstanceDev &instance_of(const InstanceDev *table, const InstanceDev &one, int i)
{
    if constexpr (BATCH) return table[i];
    else return one;
}

// The fused step.  One block of WARPS warps per tile of WARPS work items (32 fluid cells
// each), one item per warp.  Each cell's arithmetic does not depend on WARPS, so every block
// shape gives the same state bit for bit; the reducing step always runs kStepWarps-warp
// tiles.  A single instance's parameters travel by value (constant bank); a batch's come
// from the device table.  flip selects the A-B buffer pair (src = f[phase ^ flip]).  The RED
// variant (the step that ends a chunk) also makes every tile write its FP64 partial sums
// (the kRedSlots slots: drho, u_x, u_y, u_z and the momentum exchanged with the solid) and
// flags diverged cells in status[instance]; the other steps carry none of that code.  The WX
// variant (A-B only) also runs the interpolated wall rules LIBB, QIBB, IEBB and MR.
template <int COLL, int STORE, int KIND, bool BATCH, bool RED, bool WX, int WARPS = kStepWarps>
__global__ void __launch_bounds__(WARPS * 32, step_min_blocks<STORE, COLL, RED, WX, WARPS, KIND, BATCH>())
    step_kernel(const InstanceDev *__restrict__ table, const __grid_constant__ InstanceDev one,
                const __grid_constant__ MapArg<BATCH> map, const TileDev *__restrict__ tiles, int ntiles, int flip,
                unsigned *__restrict__ status)
{
    static_assert(!RED || WARPS == kStepWarps, "the reducing step runs kStepWarps-warp tiles");
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    allow_next_step();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = blockIdx.x;
    if (t >= ntiles) return;
    // a single instance's tiles are consecutive: tile t holds work items WARPS t ... (its
    // table entry holds the same, so that no load precedes the work list's)
    TileDev tile;
    if constexpr (BATCH) {
        if (map.n > 0) {  // the instance whose tiles hold t: the last i with tile_start[i] <= t
            int lo = 0, hi = map.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (map.tile_start[mid] <= t) lo = mid;
                else hi = mid - 1;
            }
            const int local = t - map.tile_start[lo];
            tile = TileDev{lo, local, (long long)local * WARPS, map.flane[lo], map.fwarp[lo]};
        } else {
            tile = tiles[t];
        }
    } else {
        tile = TileDev{0, t, (long long)t * WARPS, nullptr, nullptr};
    }
    const InstanceDev &I = instance_of<BATCH>(table, one, tile.inst);
    const Par<R> P = load_par<R>(I);
    R rates[Q];
    load_rates<COLL>(I, rates);
    const T *fs;  // state read this step
    T *fd;        // state written this step
    if constexpr (KIND == KIND_AB) {
        const int cur = I.phase ^ flip;
        fs = reinterpret_cast<const T *>(cur ? I.f1 : I.f0);
        fd = reinterpret_cast<T *>(cur ? I.f0 : I.f1);
    } else {
        fd = reinterpret_cast<T *>(I.f0);
        fs = fd;
    }
    WarpItem it;
    locate_item<R>(I, P, BATCH ? tile.flane : I.flane, BATCH ? tile.fwarp : I.fwarp,
                   (uint32_t)tile.seg0 + (uint32_t)warp, lane, it);
    wait_previous_step();
    T raw[Q];
    pull_item<STORE, KIND, R>(I, P, fs, it, raw);
    RedAcc<R> acc{};
    finish_item<COLL, STORE, KIND, RED, WX, R>(I, P, rates, raw, it, lane, fs, fd, status + tile.inst, acc);
    if constexpr (RED) reduce_tile(acc, I.partials, tile.local);
}

}  // namespace lbm
