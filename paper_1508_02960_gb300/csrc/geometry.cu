// geometry.cu -- device construction of the solid flags, the per-segment cell tables,
// the boundary-cell table and the wall distance q of every cut link (Sec. 2.2.1 and
// Sec. 3: for a non-deforming medium they are computed once before time stepping).
//
// Steps (all on the device, deterministic):
//   1. solid[cell]: a cell is solid when its centre (i+1/2, j+1/2, k+1/2) lies within r
//      of the nearest periodic image of a sphere centre (or copied from a flag field);
//   2. wm[cell]: bit k set when the fluid cell's pull source x - e_k is solid;
//   3. per 32-cell segment: solid/out-of-range bits, boundary bits, boundary count;
//   4. exclusive scan of the counts -> first boundary index of every segment; the list
//      of segments holding fluid; the fluid cells in cell order, 32 per warp;
//   5. boundary table (mask, cell) and link counts; scan -> first link of every cell;
//   6. per link: q from the ray x_f1 + t e_kbar against the spheres (nearest crossing),
//      or from a caller-supplied q field, and the CLI coefficient (1-2q)/(1+2q), set
//      to 0 (simple bounce-back) when x_f2 = x + e_k is solid.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
namespace {

// Nearest periodic image of a displacement along an axis of length n.
__device__ double min_image(double d, int n)
{
    const double h = 0.5 * n;
    while (d > h) d = __dsub_rn(d, (double)n);
    while (d < -h) d = __dadd_rn(d, (double)n);
    return d;
}

__device__ double dist2_rn(double a, double b, double c)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

__global__ void voxelize_kernel(int nx, int ny, int nz, const double4 *__restrict__ sph, int ns,
                                uint8_t *__restrict__ solid)
{
    const long long n = (long long)nx * ny * nz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const long long yz = c / nx;
        const int y = (int)(yz % ny), z = (int)(yz / ny);
        uint8_t s = 0;
        for (int i = 0; i < ns; ++i) {
            const double4 sp = sph[i];
            const double dx = min_image(__dsub_rn(x + 0.5, sp.x), nx);
            const double dy = min_image(__dsub_rn(y + 0.5, sp.y), ny);
            const double dz = min_image(__dsub_rn(z + 0.5, sp.z), nz);
            if (dist2_rn(dx, dy, dz) <= __dmul_rn(sp.w, sp.w)) s = 1;
        }
        solid[c] = s;
    }
}

__global__ void wallmask_kernel(int nx, int ny, int nz, const uint8_t *__restrict__ solid,
                                uint32_t *__restrict__ wm)
{
    const long long n = (long long)nx * ny * nz;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        uint32_t m = 0u;
        if (!solid[c]) {
            const int x = (int)(c % nx);
            const long long yz = c / nx;
            const int y = (int)(yz % ny), z = (int)(yz / ny);
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                const int xs = (x - ex(k) + nx) % nx, ys = (y - ey(k) + ny) % ny, zs = (z - ez(k) + nz) % nz;
                if (solid[xs + (long long)nx * (ys + (long long)ny * zs)]) m |= 1u << k;
            }
        }
        wm[c] = m;
    }
}

// One warp per segment.  count[s] = boundary cells; fluid count accumulated atomically.
__global__ void segment_kernel(long long n, long long nseg_padded, const uint8_t *__restrict__ solid,
                               const uint32_t *__restrict__ wm, uint4 *__restrict__ seg,
                               unsigned long long *__restrict__ count, unsigned long long *__restrict__ nfluid)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg_padded;
         s += warps) {
        const long long c = s * 32 + lane;
        const bool in = c < n;
        const bool sol = !in || solid[c];
        const bool bnd = in && !sol && wm[c] != 0u;
        const unsigned sb = __ballot_sync(0xffffffffu, sol);
        const unsigned bb = __ballot_sync(0xffffffffu, bnd);
        if (lane == 0) {
            seg[s] = make_uint4(sb, bb, 0u, 0u);
            count[s] = __popc(bb);
            const int nf = 32 - __popc(sb);
            if (nf) atomicAdd(nfluid, (unsigned long long)nf);
        }
    }
}

__global__ void active_count_kernel(long long nseg, const uint4 *__restrict__ seg,
                                    unsigned long long *__restrict__ act)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
         s += (long long)gridDim.x * blockDim.x)
        act[s] = seg[s].x != 0xFFFFFFFFu ? 1ull : 0ull;
}

// aseg[i] = segment entry of the i-th segment that holds fluid, with .w = its index;
// entries past n_active (padding) have every cell marked solid.
__global__ void active_scatter_kernel(long long nseg, long long n_active_padded, const uint4 *__restrict__ seg,
                                      const unsigned long long *__restrict__ act,
                                      const unsigned long long *__restrict__ pos, uint4 *__restrict__ aseg,
                                      long long n_active)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
         s += (long long)gridDim.x * blockDim.x)
        if (act[s]) {
            uint4 m = seg[s];
            m.w = (uint32_t)s;
            aseg[pos[s]] = m;
        }
    for (long long i = n_active + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_active_padded;
         i += (long long)gridDim.x * blockDim.x)
        aseg[i] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
}

// Fluid cells in cell order: count per segment, then each fluid cell's rank -> fcell.
__global__ void fluid_count_kernel(long long nseg, const uint4 *__restrict__ seg, unsigned long long *__restrict__ cnt)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
         s += (long long)gridDim.x * blockDim.x)
        cnt[s] = 32u - __popc(seg[s].x);
}

__global__ void fluid_scatter_kernel(long long n, const uint4 *__restrict__ seg,
                                     const unsigned long long *__restrict__ fbase, uint32_t *__restrict__ fcell)
{
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const uint32_t lane = (uint32_t)(c & 31);
        const uint32_t sb = seg[c >> 5].x;
        if (!((sb >> lane) & 1u)) fcell[fbase[c >> 5] + __popc(~sb & ((1u << lane) - 1u))] = (uint32_t)c;
    }
}

// The step kernels' per-lane work-list entries, one warp per work item w (its cells
// icell[32w .. 32w+31] in cell order, padding lanes 0xFFFFFFFF), so that a step finds what
// it needs of a cell without a dependent load or a division: flane[32w + l] = {x, y},
//   x: the cell (bits 0-27; cells < 2^28 since 19 direction strides fit 32 bits), bit 28
//      x = 0, bit 29 x = nx - 1 (the pulls and pushes that cross the x faces), bit 30 every
//      cell of the item away from the y and z faces (the same in all its lanes);
//      0xFFFFFFFF for a padding lane;
//   y: bits 0-18 the wall mask (bit k: x - e_k solid), bits 19-31 the cell's first link
//      minus the item's first link;
// and fwarp[w] = {boundary bits of the lanes, the item's first link (0 when it has no
// boundary cell)}.  Links are numbered in cell order, and an item's cells lie within
// kItemSpan + 1 consecutive cells of at most 18 links each, so the offset fits 13 bits.
static_assert(18 * (kItemSpan + 1) < (1 << 13), "link offset field of the work-list entries");
__global__ void flane_kernel(long long nw, int nx, int ny, int nz, const uint32_t *__restrict__ icell,
                             const uint4 *__restrict__ seg, const uint32_t *__restrict__ bmask,
                             const uint32_t *__restrict__ boff, uint2 *__restrict__ fwarp, uint2 *__restrict__ flane)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nw; w += warps) {
        const uint32_t c = icell[w * 32 + lane];
        const bool live = c != 0xFFFFFFFFu;
        const uint4 m = live ? seg[c >> 5] : make_uint4(0u, 0u, 0u, 0u);
        const bool bnd = live && ((m.y >> (c & 31u)) & 1u);
        uint32_t wm = 0u, off = 0u;
        if (bnd) {  // the boundary table lists boundary cells in cell order
            const uint32_t b = m.z + __popc(m.y & ((1u << (c & 31u)) - 1u));
            wm = bmask[b];
            off = boff[b];
        }
        const unsigned bb = __ballot_sync(0xffffffffu, bnd);
        const uint32_t base = bb ? __shfl_sync(0xffffffffu, off, __ffs(bb) - 1) : 0u;
        uint32_t ex = 0xFFFFFFFFu;
        bool in_yz = true;
        if (live) {
            const uint32_t x = c % (uint32_t)nx, yz = c / (uint32_t)nx;
            const uint32_t y = yz % (uint32_t)ny, z = yz / (uint32_t)ny;
            ex = c | (x == 0 ? 1u << 28 : 0u) | (x == (uint32_t)nx - 1u ? 1u << 29 : 0u);
            in_yz = y >= 1 && y + 2 <= (uint32_t)ny && z >= 1 && z + 2 <= (uint32_t)nz;
        }
        if (__all_sync(0xffffffffu, in_yz) && live) ex |= 1u << 30;
        flane[w * 32 + lane] = make_uint2(ex, wm | ((bnd ? off - base : 0u) << 19));
        if (lane == 0) fwarp[w] = make_uint2(bb, base);
    }
}

// The step kernels' work items (one warp each) from the fluid cells in cell order.  A
// box segment of 32 cells that are all fluid is an item of its own: aligned to 128-byte
// lines, each of its loads and stores touches one line (two for the directions with
// e_kx != 0).  The fluid cells of the other segments are packed 32 to an item in cell
// order, an item spanning at most kItemSpan + 1 cells (the link-offset field above).  On
// the r = 60 sphere cell this cuts the cache lines a step touches by a fifth at the same
// number of items, where 32 consecutive fluid cells to an item straddle two lines almost
// always.
static std::vector<uint32_t> pack_items(const std::vector<uint32_t> &cells, long long *n_items)
{
    std::vector<uint32_t> out, pend;
    out.reserve(cells.size() + cells.size() / 8 + 64);
    pend.reserve(32);
    auto flush = [&]() {
        if (pend.empty()) return;
        out.insert(out.end(), pend.begin(), pend.end());
        out.insert(out.end(), 32 - pend.size(), 0xFFFFFFFFu);
        pend.clear();
    };
    size_t j = 0;
    while (j < cells.size()) {
        const uint32_t sg = cells[j] >> 5;
        size_t k = j + 1;
        while (k < cells.size() && (cells[k] >> 5) == sg) ++k;
        if (k - j == 32) {
            out.insert(out.end(), cells.begin() + (long)j, cells.begin() + (long)k);
        } else {
            for (size_t i = j; i < k; ++i) {
                if (pend.size() == 32 || (!pend.empty() && (long long)cells[i] - (long long)pend[0] > kItemSpan))
                    flush();
                pend.push_back(cells[i]);
            }
        }
        j = k;
    }
    flush();
    *n_items = (long long)(out.size() / 32);
    return out;
}

__global__ void seg_base_kernel(long long nseg, uint4 *__restrict__ seg, const unsigned long long *__restrict__ base)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
         s += (long long)gridDim.x * blockDim.x)
        seg[s].z = (uint32_t)base[s];
}

__global__ void boundary_kernel(long long n, const uint4 *__restrict__ seg, const uint32_t *__restrict__ wm,
                                uint32_t *__restrict__ bmask, long long *__restrict__ bcell,
                                unsigned long long *__restrict__ nlink)
{
    const int lane = threadIdx.x & 31;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const uint4 m = seg[c >> 5];
        if ((m.y >> lane) & 1u) {
            const uint32_t b = m.z + __popc(m.y & ((1u << lane) - 1u));
            bmask[b] = wm[c];
            bcell[b] = c;
            nlink[b] = __popc(wm[c]);
        }
    }
}

__global__ void to_u32_kernel(long long n, const unsigned long long *__restrict__ in, uint32_t *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (uint32_t)in[i];
}

// Coefficients of the rule of one cut link (see kLinkW in lbm_device.cuh): q its wall
// distance, f2 / f3 whether x_f2 / x_f3 are fluid, kd the link direction (into the wall).
// The rules are Sec. 2.2.1's, rewritten for the unknown g_k (k = kbar of the paper's link
// direction); fallbacks where a node a rule reads is solid: SBB when it needs x_f2, QIBB
// to LIBB and MR to CLI when only x_f3 is solid.  MR's first coefficient is taken over
// (1+q)^2, like its second: as printed over (1+2q)^2 the rule is not consistent.
__device__ void rule_coefficients(int wall, double q, bool f2, bool f3, double tau, int kd, double *w)
{
    for (int i = 0; i < kLinkW; ++i) w[i] = 0.0;
    const bool lo = q < 0.5;
    auto sbb = [&] { w[LW_EPS] = 1.0; };
    auto cli = [&] {
        const double c = __ddiv_rn(__dsub_rn(1.0, 2.0 * q), __dadd_rn(1.0, 2.0 * q));
        w[LW_EPS] = 1.0;
        w[LW_GAMMA] = -c;
        w[LW_ALPHA] = c;
    };
    auto libb = [&] {
        if (lo) {
            w[LW_ALPHA] = 1.0 - 2.0 * q;
            w[LW_EPS] = 2.0 * q;
        } else {
            w[LW_GAMMA] = 1.0 - 1.0 / (2.0 * q);
            w[LW_EPS] = 1.0 / (2.0 * q);
        }
    };
    switch (wall) {
    case 2:  // LIBB
        if (lo && !f2) sbb();
        else libb();
        break;
    case 3:  // QIBB
        if (!f2) {
            if (lo) sbb();
            else libb();
        } else if (lo && !f3) {
            libb();
        } else if (lo) {
            w[LW_EPS] = q * (1.0 + 2.0 * q);
            w[LW_ALPHA] = 1.0 - 4.0 * q * q;
            w[LW_BETA] = -q * (1.0 - 2.0 * q);
        } else {
            w[LW_GAMMA] = (2.0 * q - 1.0) / q;
            w[LW_EPS] = 1.0 / (q * (2.0 * q + 1.0));
            w[LW_DELTA] = (1.0 - 2.0 * q) / (2.0 * q + 1.0);
        }
        break;
    case 4:  // IEBB: (1 - X) C + X f*, f* = w {rho + rho0 [3 e.u_bf + 9/2 (e.u1)^2 - 3/2 u1.u1]}
        if (lo && !f2) {
            sbb();
        } else if (lo) {  // u_bf = u(x_f2): its e.u term waits for step t+1
            const double X = (2.0 * q - 1.0) / (tau - 2.0);
            w[LW_X] = X;
            w[LW_EPS] = 1.0 - X;
            w[LW_ZETA] = 3.0 * X * weight(kd);
        } else {  // u_bf = (1 - 3/(2q)) u(x_f1)
            const double X = (2.0 * q - 1.0) / (tau + 0.5);
            w[LW_X] = X;
            w[LW_EPS] = 1.0 - X;
            w[LW_THETA] = 3.0 * (1.0 - 3.0 / (2.0 * q));
        }
        break;
    case 5:  // MR
        if (!f2) {
            sbb();
        } else if (!f3) {
            cli();
        } else {
            const double a = (1.0 - 2.0 * q - 2.0 * q * q) / ((1.0 + q) * (1.0 + q));
            const double b = q * q / ((1.0 + q) * (1.0 + q));
            w[LW_EPS] = 1.0;
            w[LW_ALPHA] = a;
            w[LW_GAMMA] = -a;
            w[LW_BETA] = b;
            w[LW_DELTA] = -b;
        }
        break;
    default: sbb(); break;
    }
}

template <typename R>
__global__ void link_kernel(long long nb, int nx, int ny, int nz, const double4 *__restrict__ sph, int ns,
                            const double *__restrict__ qfield, const uint8_t *__restrict__ solid,
                            const uint32_t *__restrict__ bmask, const uint32_t *__restrict__ boff,
                            const long long *__restrict__ bcell, double *__restrict__ linkq, R *__restrict__ linkc,
                            unsigned long long *__restrict__ ncli, int wall, double tau, R *__restrict__ linkw)
{
    const long long n = (long long)nx * ny * nz;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const long long c = bcell[b];
        const uint32_t m = bmask[b];
        const int x = (int)(c % nx);
        const long long yz = c / nx;
        const int y = (int)(yz % ny), z = (int)(yz / ny);
        uint32_t l = boff[b];
        int cli = 0;
        for (int k = 1; k < Q; ++k) {
            if (!((m >> k) & 1u)) continue;
            const int kd = opp(k);  // link direction from x_f1 into the wall
            double q = 0.5;
            if (sph) {
                // solid end point x_b = x + e_kd; nearest crossing of the segment x_f1 -> x_b
                const double bx = x + ex(kd) + 0.5, by = y + ey(kd) + 0.5, bz = z + ez(kd) + 0.5;
                double best = INFINITY;
                for (int i = 0; i < ns; ++i) {
                    const double4 sp = sph[i];
                    const double cx = __dsub_rn(bx, min_image(__dsub_rn(bx, sp.x), nx));
                    const double cy = __dsub_rn(by, min_image(__dsub_rn(by, sp.y), ny));
                    const double cz = __dsub_rn(bz, min_image(__dsub_rn(bz, sp.z), nz));
                    if (dist2_rn(__dsub_rn(bx, cx), __dsub_rn(by, cy), __dsub_rn(bz, cz)) > __dmul_rn(sp.w, sp.w))
                        continue;
                    const double px = __dsub_rn(x + 0.5, cx), py = __dsub_rn(y + 0.5, cy), pz = __dsub_rn(z + 0.5, cz);
                    const double a = (double)speed2(kd);
                    const double hb = __dadd_rn(__dadd_rn(__dmul_rn(px, (double)ex(kd)), __dmul_rn(py, (double)ey(kd))),
                                                __dmul_rn(pz, (double)ez(kd)));
                    const double cc = __dsub_rn(dist2_rn(px, py, pz), __dmul_rn(sp.w, sp.w));
                    double disc = __dsub_rn(__dmul_rn(hb, hb), __dmul_rn(a, cc));
                    if (disc < 0.0) disc = 0.0;
                    const double t = __ddiv_rn(__dsub_rn(-hb, __dsqrt_rn(disc)), a);
                    if (t < best) best = t;
                }
                if (best < INFINITY) q = best;
            } else if (qfield) {
                q = qfield[(long long)kd * n + c];
                if (!(q == q)) q = 0.5;
            }
            if (q < 1e-6) q = 1e-6;
            if (q > 1.0) q = 1.0;
            // x_f2 = x_f1 - e_kd = x + e_k must be fluid for CLI (else simple bounce-back)
            const int x2 = (x + ex(k) + nx) % nx, y2 = (y + ey(k) + ny) % ny, z2 = (z + ez(k) + nz) % nz;
            const bool f2 = !solid[x2 + (long long)nx * (y2 + (long long)ny * z2)];
            const double cq = f2 ? __ddiv_rn(__dsub_rn(1.0, 2.0 * q), __dadd_rn(1.0, 2.0 * q)) : 0.0;
            linkq[l] = q;
            linkc[l] = (R)cq;
            if (linkw) {  // x_f3 = x + 2 e_k
                const int x3 = (x + 2 * ex(k) + 2 * nx) % nx, y3 = (y + 2 * ey(k) + 2 * ny) % ny,
                          z3 = (z + 2 * ez(k) + 2 * nz) % nz;
                const bool f3 = f2 && !solid[x3 + (long long)nx * (y3 + (long long)ny * z3)];
                double wv[kLinkW];
                rule_coefficients(wall, q, f2, f3, tau, kd, wv);
                for (int i = 0; i < kLinkW; ++i) linkw[(long long)l * kLinkW + i] = (R)wv[i];
            }
            cli += f2;
            ++l;
        }
        if (cli) atomicAdd(ncli, (unsigned long long)cli);
    }
}

__global__ void scatter_q_kernel(long long nb, int kdir, const uint32_t *__restrict__ bmask,
                                 const uint32_t *__restrict__ boff, const long long *__restrict__ bcell,
                                 const double *__restrict__ linkq, double *__restrict__ qk)
{
    const int k = opp(kdir);  // pull direction whose source is the wall
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const uint32_t m = bmask[b];
        if ((m >> k) & 1u) qk[bcell[b]] = linkq[boff[b] + __popc(m & ((1u << k) - 1u))];
    }
}

__global__ void fill_kernel(long long n, double v, double *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = v;
}

// ---- exclusive scan of unsigned 64-bit counts (deterministic, recursive) ----------------
__global__ void scan_block_kernel(const unsigned long long *__restrict__ in, unsigned long long *__restrict__ out,
                                  unsigned long long *__restrict__ bsum, long long n)
{
    __shared__ unsigned long long ws[32];
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long v = i < n ? in[i] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const unsigned long long excl = x - v + (warp ? ws[warp - 1] : 0ull);
    if (i < n) out[i] = excl;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = excl + v;
}

__global__ void scan_add_kernel(unsigned long long *__restrict__ out, const unsigned long long *__restrict__ boff,
                                long long n)
{
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

cudaError_t exclusive_scan(const unsigned long long *in, unsigned long long *out, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long nb = (n + 1023) / 1024;
    unsigned long long *bsum = nullptr, *bscan = nullptr;
    cudaError_t e = dev_alloc(&bsum, sizeof(unsigned long long) * nb);
    if (e != cudaSuccess) return e;
    scan_block_kernel<<<(unsigned)nb, 1024, 0, s>>>(in, out, bsum, n);
    e = cudaGetLastError();
    if (e == cudaSuccess && nb > 1) {
        e = dev_alloc(&bscan, sizeof(unsigned long long) * nb);
        if (e == cudaSuccess) e = exclusive_scan(bsum, bscan, nb, s);
        if (e == cudaSuccess) {
            scan_add_kernel<<<(unsigned)nb, 1024, 0, s>>>(out, bscan, n);
            e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    cudaFree(bsum);
    if (bscan) cudaFree(bscan);
    return e;
}

int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

void free_geometry(GeometryDev *g)
{
    cudaFree(g->solid);
    cudaFree(g->seg);
    cudaFree(g->aseg);
    cudaFree(g->fcell);
    cudaFree(g->flane);
    cudaFree(g->fwarp);
    cudaFree(g->bmask);
    cudaFree(g->boff);
    cudaFree(g->bcell);
    cudaFree(g->linkq);
    cudaFree(g->linkc);
    cudaFree(g->linkw);
    *g = GeometryDev();
}

#define GEO_CHECK(x)                                                                  \
    do {                                                                              \
        e = (x);                                                                      \
        if (e != cudaSuccess) {                                                       \
            *err = std::string("geometry: ") + #x + ": " + cudaGetErrorString(e);     \
            goto fail;                                                                \
        }                                                                             \
    } while (0)

std::vector<uint32_t> pack_work_items(const std::vector<uint32_t> &cells, long long *n_items)
{
    return pack_items(cells, n_items);
}

cudaError_t build_geometry(int nx, int ny, int nz, const double *spheres, int n_spheres, const uint8_t *flags,
                           const double *q_host, bool c_double, int wall, double tau, cudaStream_t s, GeometryDev *g,
                           std::string *err)
{
    cudaError_t e = cudaSuccess;
    const long long n = (long long)nx * ny * nz;
    if (n >= (1ll << 28)) {  // the work-list entries keep a cell in 28 bits
        *err = "geometry: box of 2^28 cells or more";
        return cudaErrorInvalidValue;
    }
    double4 *d_sph = nullptr;
    double *d_q = nullptr;
    uint32_t *d_wm = nullptr, *d_icell = nullptr;  // d_icell: the work items' cells, [32 n_fwarps_padded]
    unsigned long long *d_cnt = nullptr, *d_base = nullptr, *d_nl = nullptr, *d_lbase = nullptr, *d_ctr = nullptr;
    unsigned long long h_ctr[2] = {0ull, 0ull};
    unsigned long long h_last[2];
    *g = GeometryDev();
    g->ncells = n;
    g->nseg = (n + 31) / 32;
    g->nseg_padded = (g->nseg + kMaxWarpsPerBlock - 1) / kMaxWarpsPerBlock * kMaxWarpsPerBlock;

    GEO_CHECK(dev_alloc(&g->solid, n));
    GEO_CHECK(dev_alloc(&g->seg, sizeof(uint4) * g->nseg_padded));
    GEO_CHECK(dev_alloc(&d_wm, sizeof(uint32_t) * n));
    GEO_CHECK(dev_alloc(&d_cnt, sizeof(unsigned long long) * g->nseg_padded));
    GEO_CHECK(dev_alloc(&d_base, sizeof(unsigned long long) * g->nseg_padded));
    GEO_CHECK(dev_alloc(&d_ctr, sizeof(unsigned long long) * 2));
    GEO_CHECK(cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long) * 2, s));

    if (spheres && n_spheres > 0) {
        GEO_CHECK(dev_alloc(&d_sph, sizeof(double4) * n_spheres));
        GEO_CHECK(cudaMemcpyAsync(d_sph, spheres, sizeof(double4) * n_spheres, cudaMemcpyHostToDevice, s));
        voxelize_kernel<<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, d_sph, n_spheres, g->solid);
        GEO_CHECK(cudaGetLastError());
    } else if (flags) {
        GEO_CHECK(cudaMemcpyAsync(g->solid, flags, n, cudaMemcpyHostToDevice, s));
    } else {
        GEO_CHECK(cudaMemsetAsync(g->solid, 0, n, s));
    }
    wallmask_kernel<<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, g->solid, d_wm);
    GEO_CHECK(cudaGetLastError());
    segment_kernel<<<grid_for(g->nseg_padded * 32, 256), 256, 0, s>>>(n, g->nseg_padded, g->solid, d_wm, g->seg,
                                                                       d_cnt, d_ctr);
    GEO_CHECK(cudaGetLastError());
    GEO_CHECK(exclusive_scan(d_cnt, d_base, g->nseg_padded, s));
    GEO_CHECK(cudaMemcpy(&h_last[0], d_base + g->nseg_padded - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    GEO_CHECK(cudaMemcpy(&h_last[1], d_cnt + g->nseg_padded - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    g->n_boundary = (long long)(h_last[0] + h_last[1]);
    if (g->n_boundary >= (1ll << 32)) {
        *err = "geometry: too many boundary cells for 32-bit indices";
        e = cudaErrorInvalidValue;
        goto fail;
    }
    seg_base_kernel<<<grid_for(g->nseg_padded, 256), 256, 0, s>>>(g->nseg_padded, g->seg, d_base);
    GEO_CHECK(cudaGetLastError());

    // list of the segments that hold fluid (the kernels' work list), padded to 32 entries
    active_count_kernel<<<grid_for(g->nseg_padded, 256), 256, 0, s>>>(g->nseg_padded, g->seg, d_cnt);
    GEO_CHECK(cudaGetLastError());
    GEO_CHECK(exclusive_scan(d_cnt, d_base, g->nseg_padded, s));
    GEO_CHECK(cudaMemcpy(&h_last[0], d_base + g->nseg_padded - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    GEO_CHECK(cudaMemcpy(&h_last[1], d_cnt + g->nseg_padded - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    g->n_active = (long long)(h_last[0] + h_last[1]);
    g->n_active_padded = std::max<long long>(kMaxWarpsPerBlock,
        (g->n_active + kMaxWarpsPerBlock - 1) / kMaxWarpsPerBlock * kMaxWarpsPerBlock);
    GEO_CHECK(dev_alloc(&g->aseg, sizeof(uint4) * g->n_active_padded));
    active_scatter_kernel<<<grid_for(g->nseg_padded, 256), 256, 0, s>>>(g->nseg_padded, g->n_active_padded, g->seg,
                                                                         d_cnt, d_base, g->aseg, g->n_active);
    GEO_CHECK(cudaGetLastError());

    // the fluid cells in cell order (fcell, the state kernels' list), then the step kernels'
    // work items packed from it on the host (pack_items)
    fluid_count_kernel<<<grid_for(g->nseg_padded, 256), 256, 0, s>>>(g->nseg_padded, g->seg, d_cnt);
    GEO_CHECK(cudaGetLastError());
    GEO_CHECK(exclusive_scan(d_cnt, d_base, g->nseg_padded, s));
    GEO_CHECK(cudaMemcpy(&h_last[0], d_base + g->nseg_padded - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    GEO_CHECK(cudaMemcpy(&h_last[1], d_cnt + g->nseg_padded - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    g->n_fcell = (long long)(h_last[0] + h_last[1]);
    g->n_fcell_padded = std::max<long long>(32, (g->n_fcell + 31) / 32 * 32);
    GEO_CHECK(dev_alloc(&g->fcell, sizeof(uint32_t) * g->n_fcell_padded));
    GEO_CHECK(cudaMemsetAsync(g->fcell, 0xFF, sizeof(uint32_t) * g->n_fcell_padded, s));
    fluid_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, g->seg, d_base, g->fcell);
    GEO_CHECK(cudaGetLastError());
    {
        std::vector<uint32_t> cells((size_t)g->n_fcell);
        if (g->n_fcell > 0)
            GEO_CHECK(cudaMemcpyAsync(cells.data(), g->fcell, sizeof(uint32_t) * cells.size(), cudaMemcpyDeviceToHost,
                                      s));
        GEO_CHECK(cudaStreamSynchronize(s));
        const std::vector<uint32_t> items = pack_items(cells, &g->n_fwarps);
        g->n_fwarps_padded = std::max<long long>(kMaxWarpsPerBlock,
            (g->n_fwarps + kMaxWarpsPerBlock - 1) / kMaxWarpsPerBlock * kMaxWarpsPerBlock);
        GEO_CHECK(dev_alloc(&d_icell, sizeof(uint32_t) * 32 * g->n_fwarps_padded));
        GEO_CHECK(cudaMemsetAsync(d_icell, 0xFF, sizeof(uint32_t) * 32 * g->n_fwarps_padded, s));
        if (!items.empty())
            GEO_CHECK(cudaMemcpyAsync(d_icell, items.data(), sizeof(uint32_t) * items.size(), cudaMemcpyHostToDevice,
                                      s));
        GEO_CHECK(cudaStreamSynchronize(s));  // before items goes out of scope
    }
    GEO_CHECK(dev_alloc(&g->fwarp, sizeof(uint2) * g->n_fwarps_padded));

    if (g->n_boundary > 0) {
        const long long nb = g->n_boundary;
        GEO_CHECK(dev_alloc(&g->bmask, sizeof(uint32_t) * nb));
        GEO_CHECK(dev_alloc(&g->boff, sizeof(uint32_t) * nb));
        GEO_CHECK(dev_alloc(&g->bcell, sizeof(long long) * nb));
        GEO_CHECK(dev_alloc(&d_nl, sizeof(unsigned long long) * nb));
        GEO_CHECK(dev_alloc(&d_lbase, sizeof(unsigned long long) * nb));
        boundary_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, g->seg, d_wm, g->bmask, g->bcell, d_nl);
        GEO_CHECK(cudaGetLastError());
        GEO_CHECK(exclusive_scan(d_nl, d_lbase, nb, s));
        GEO_CHECK(cudaMemcpy(&h_last[0], d_lbase + nb - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        GEO_CHECK(cudaMemcpy(&h_last[1], d_nl + nb - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        g->n_links = (long long)(h_last[0] + h_last[1]);
        if (g->n_links >= (1ll << 32)) {
            *err = "geometry: too many cut links for 32-bit indices";
            e = cudaErrorInvalidValue;
            goto fail;
        }
        to_u32_kernel<<<grid_for(nb, 256), 256, 0, s>>>(nb, d_lbase, g->boff);
        GEO_CHECK(cudaGetLastError());
        if (g->n_links > 0) {
            GEO_CHECK(dev_alloc(&g->linkq, sizeof(double) * g->n_links));
            GEO_CHECK(dev_alloc(&g->linkc, (c_double ? 8 : 4) * g->n_links));
            if (wall >= 2) GEO_CHECK(dev_alloc(&g->linkw, (c_double ? 8 : 4) * kLinkW * g->n_links));
            if (q_host && !(spheres && n_spheres > 0)) {
                GEO_CHECK(dev_alloc(&d_q, sizeof(double) * Q * n));
                GEO_CHECK(cudaMemcpyAsync(d_q, q_host, sizeof(double) * Q * n, cudaMemcpyHostToDevice, s));
            }
            const double4 *sp = (spheres && n_spheres > 0) ? d_sph : nullptr;
            if (c_double)
                link_kernel<double><<<grid_for(nb, 128), 128, 0, s>>>(nb, nx, ny, nz, sp, n_spheres, d_q, g->solid,
                                                                      g->bmask, g->boff, g->bcell, g->linkq,
                                                                      (double *)g->linkc, d_ctr + 1, wall, tau,
                                                                      (double *)g->linkw);
            else
                link_kernel<float><<<grid_for(nb, 128), 128, 0, s>>>(nb, nx, ny, nz, sp, n_spheres, d_q, g->solid,
                                                                     g->bmask, g->boff, g->bcell, g->linkq,
                                                                     (float *)g->linkc, d_ctr + 1, wall, tau,
                                                                     (float *)g->linkw);
            GEO_CHECK(cudaGetLastError());
        }
    }
    // per-lane entries of the step kernels' work list (needs the boundary table's links)
    GEO_CHECK(dev_alloc(&g->flane, sizeof(uint2) * 32 * g->n_fwarps_padded));
    flane_kernel<<<grid_for(g->n_fwarps_padded * 32, 256), 256, 0, s>>>(g->n_fwarps_padded, nx, ny, nz, d_icell,
                                                                          g->seg, g->bmask, g->boff, g->fwarp,
                                                                          g->flane);
    GEO_CHECK(cudaGetLastError());
    GEO_CHECK(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(h_ctr), cudaMemcpyDeviceToHost, s));
    GEO_CHECK(cudaStreamSynchronize(s));
    g->n_fluid = (long long)h_ctr[0];
    g->n_links_cli = (long long)h_ctr[1];
    g->bytes = n + sizeof(uint4) * (g->nseg_padded + g->n_active_padded) + sizeof(uint32_t) * g->n_fcell_padded +
               (sizeof(uint2) * 32 + sizeof(uint2)) * g->n_fwarps_padded +
               (sizeof(uint32_t) * 2 + sizeof(long long)) * g->n_boundary +
               (sizeof(double) + (c_double ? 8 : 4) * (wall >= 2 ? 1 + kLinkW : 1)) * g->n_links;

    cudaFree(d_sph);
    cudaFree(d_q);
    cudaFree(d_wm);
    cudaFree(d_cnt);
    cudaFree(d_base);
    cudaFree(d_nl);
    cudaFree(d_lbase);
    cudaFree(d_ctr);
    cudaFree(d_icell);
    return cudaSuccess;
fail:
    cudaStreamSynchronize(s);
    cudaFree(d_sph);
    cudaFree(d_q);
    cudaFree(d_wm);
    cudaFree(d_cnt);
    cudaFree(d_base);
    cudaFree(d_nl);
    cudaFree(d_lbase);
    cudaFree(d_ctr);
    cudaFree(d_icell);
    free_geometry(g);
    return e == cudaSuccess ? cudaErrorUnknown : e;
}

cudaError_t export_wall_distances(const GeometryDev &g, int kdir, double *qk, cudaStream_t s)
{
    fill_kernel<<<grid_for(g.ncells, 256), 256, 0, s>>>(g.ncells, NAN, qk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || g.n_links == 0 || kdir == 0) return e;
    scatter_q_kernel<<<grid_for(g.n_boundary, 256), 256, 0, s>>>(g.n_boundary, kdir, g.bmask, g.boff, g.bcell,
                                                                  g.linkq, qk);
    return cudaGetLastError();
}

// ---- deterministic final reduction of tile partials ---------------------------------------
// kFinalSlices blocks per instance each sum one fixed, contiguous range of the instance's
// tile partials (strided over the threads, then a fixed tree) into scratch; the last of
// them to finish (the instance's counter) adds the slices in order into out and resets the
// counter.  The result depends only on the partials and their count, never on timing;
// spreading the FP64 additions over many SMs matters on GB300, whose FP64 rate made one
// block per instance the cost of the check.
__global__ void final_reduce_kernel(const InstanceDev *__restrict__ table, const int *__restrict__ tile_count,
                                    double *__restrict__ out, double *__restrict__ scratch,
                                    unsigned *__restrict__ counter)
{
    constexpr int D = RED_F + 3;  // slots in use
    __shared__ double sm[256][D];
    __shared__ bool last;
    const int inst = blockIdx.x / kFinalSlices, slice = blockIdx.x % kFinalSlices;
    const double *p = table[inst].partials;
    const int nt = tile_count[inst];
    const int per = (nt + kFinalSlices - 1) / kFinalSlices;
    const int t0 = slice * per, t1 = min(nt, t0 + per);
    double a[D];
    for (int d = 0; d < D; ++d) a[d] = 0.0;
    for (int t = t0 + (int)threadIdx.x; t < t1; t += blockDim.x)
        for (int d = 0; d < D; ++d) a[d] += p[(long long)t * kRedSlots + d];
    for (int d = 0; d < D; ++d) sm[threadIdx.x][d] = a[d];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int d = 0; d < D; ++d) sm[threadIdx.x][d] += sm[threadIdx.x + w][d];
        __syncthreads();
    }
    double *row = scratch + ((long long)inst * kFinalSlices + slice) * D;
    if (threadIdx.x < D) row[threadIdx.x] = sm[0][threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&counter[inst], 1u) == (unsigned)kFinalSlices - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < kRedSlots) {
        double sum = 0.0;
        if (threadIdx.x < D)
            for (int k = 0; k < kFinalSlices; ++k)
                sum += __ldcg(scratch + ((long long)inst * kFinalSlices + k) * D + threadIdx.x);
        out[(long long)inst * kRedSlots + threadIdx.x] = sum;
    }
    if (threadIdx.x == 0) counter[inst] = 0u;
}

cudaError_t launch_final_reduce(const InstanceDev *table, const int *tile_count, int n_inst, double *out,
                                double *scratch, unsigned *counter, cudaStream_t s)
{
    final_reduce_kernel<<<n_inst * kFinalSlices, 256, 0, s>>>(table, tile_count, out, scratch, counter);
    return cudaGetLastError();
}

}  // namespace lbm
