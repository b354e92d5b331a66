// lbm_device.cuh -- device-side definitions shared by the kernels of the GB300 D3Q19
// sphere-pack library: the D3Q19 lattice (Sec. 2), population storage formats, the
// per-instance parameter table and the tile work list.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 19;

// D3Q19 velocities: rest, six axis links, twelve face diagonals, opposites adjacent.
__host__ __device__ constexpr int ex(int k)
{
    constexpr int v[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[k];
}
__host__ __device__ constexpr int ey(int k)
{
    constexpr int v[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[k];
}
__host__ __device__ constexpr int ez(int k)
{
    constexpr int v[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[k];
}
// Opposite direction k-bar (e_kbar = -e_k); also valid for a run-time k.
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }
__host__ __device__ __forceinline__ constexpr int opp_rt(int k) { return opp(k); }

// Velocity components for a run-time k (lane-indexed code): 2 bits per direction.
__host__ __device__ constexpr unsigned long long pack_component(int a)
{
    unsigned long long m = 0ull;
    for (int k = 0; k < 19; ++k)
        m |= (unsigned long long)((a == 0 ? ex(k) : a == 1 ? ey(k) : ez(k)) + 1) << (2 * k);
    return m;
}
__device__ __forceinline__ int ex_rt(int k) { return (int)((pack_component(0) >> (2 * k)) & 3ull) - 1; }
__device__ __forceinline__ int ey_rt(int k) { return (int)((pack_component(1) >> (2 * k)) & 3ull) - 1; }
__device__ __forceinline__ int ez_rt(int k) { return (int)((pack_component(2) >> (2 * k)) & 3ull) - 1; }
// Squared speed and lattice weight (c_s^2 = 1/3 isotropic set).
__host__ __device__ constexpr int speed2(int k) { return ex(k) * ex(k) + ey(k) * ey(k) + ez(k) * ez(k); }
__host__ __device__ constexpr double weight(int k)
{
    return speed2(k) == 0 ? 1.0 / 3.0 : (speed2(k) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// MRT moment basis (Sec. 2.1, Eq. MRT): d'Humieres' integer polynomials in e_k, which
// are already mutually orthogonal over the 19 velocities (the Gram-Schmidt result up
// to row scaling).  Row order: rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx,
// 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z.
__host__ __device__ constexpr int mrt_m(int i, int k)
{
    const int x = ex(k), y = ey(k), z = ez(k), n2 = speed2(k);
    switch (i) {
    case 0: return 1;
    case 1: return 19 * n2 - 30;
    case 2: return (21 * n2 * n2 - 53 * n2 + 24) / 2;
    case 3: return x;
    case 4: return (5 * n2 - 9) * x;
    case 5: return y;
    case 6: return (5 * n2 - 9) * y;
    case 7: return z;
    case 8: return (5 * n2 - 9) * z;
    case 9: return 3 * x * x - n2;
    case 10: return (3 * n2 - 5) * (3 * x * x - n2);
    case 11: return y * y - z * z;
    case 12: return (3 * n2 - 5) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
    }
}
// Row i of M is even in e (M[i][kbar] = M[i][k] for every k) or odd (M[i][kbar] = -M[i][k],
// M[i][0] = 0): its moment needs only the sums, or only the differences, of the opposite
// pairs (k, k + 1).  mrt_even is written out (rows 0-2 and 9-15 even) so that the unrolled
// loops of the collision fold it to a constant; the check below derives it from the rows.
__host__ __device__ constexpr bool mrt_even(int i) { return i <= 2 || (i >= 9 && i <= 15); }
__host__ __device__ constexpr bool mrt_row_parity_holds(int i)
{
    for (int k = 1; k < Q; k += 2) {
        const int a = mrt_m(i, k), b = mrt_m(i, k + 1);
        if (mrt_even(i) ? (b != a) : (b != -a)) return false;
    }
    return mrt_even(i) || mrt_m(i, 0) == 0;
}
__host__ __device__ constexpr bool mrt_parities_hold()
{
    for (int i = 0; i < Q; ++i)
        if (!mrt_row_parity_holds(i)) return false;
    return true;
}
static_assert(mrt_parities_hold(), "mrt_even matches the rows of M");
__host__ __device__ constexpr int mrt_norm2(int i)
{
    int s = 0;
    for (int k = 0; k < Q; ++k) s += mrt_m(i, k) * mrt_m(i, k);
    return s;
}

// ------------------------------------------------------------------------------------
// Storage formats.  Every format stores the deviation g_k = f_k - w_k rho0; R is the
// arithmetic type of the collision.
//
// The 16-bit formats store with stochastic rounding: a per-step change of a population
// that is below half a unit of the stored format would otherwise round to no change at
// all, and a run started from rest then stops short of its steady state.  The random bits
// come from a multiplicative hash of the cell, the direction and the value itself, so a
// run is reproducible, a true fixed point stays fixed, and the rounding is unbiased over
// the changing values of a flow that is still evolving.
// ------------------------------------------------------------------------------------
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }

// The own-cell part of the wall rule of link (x, kbar), x - e_k solid, from the cell's own
// post-collision values C = g~_kbar(x) and B = g~_k(x): SBB S = C (Eq. noslip); CLI
// S = C - c B, so that the new g_k = S + c g_kbar^in (Eq. CLI; c = 0 where CLI falls back
// to SBB).
template <typename R> __device__ __forceinline__ R wall_own_part(int wall, R cq, R C, R B)
{
    return (wall == 1 && cq != R(0)) ? fma_r(-cq, B, C) : C;
}

template <int S> struct Store;
template <> struct Store<ST_F64> {
    using T = double;
    using R = double;
    __device__ static R load(const T *p, float) { return __ldg(p); }
    __device__ static R cvt(T v, float) { return v; }
    __device__ static T pack(R v, float) { return v; }
    __device__ static T pack_sr(R v, float, uint32_t) { return v; }
};
template <> struct Store<ST_F32> {
    using T = float;
    using R = float;
    __device__ static R load(const T *p, float) { return __ldg(p); }
    __device__ static R cvt(T v, float) { return v; }
    __device__ static T pack(R v, float) { return v; }
    __device__ static T pack_sr(R v, float, uint32_t) { return v; }
};
// FP16 deviation with a power-of-two scale 2^s: stored = g * 2^s (exact scaling).
template <> struct Store<ST_F16> {
    using T = __half;
    using R = float;
    __device__ static R load(const T *p, float inv_scale) { return __half2float(__ldg(p)) * inv_scale; }
    __device__ static R cvt(T v, float inv_scale) { return __half2float(v) * inv_scale; }
    __device__ static T pack(R v, float scale) { return __float2half_rn(v * scale); }
    // stochastic rounding: 13 random bits added below the FP16 mantissa, then truncation
    __device__ static T pack_sr(R v, float scale, uint32_t rnd)
    {
        const float x = v * scale;
        return __float2half_rz(__uint_as_float(__float_as_uint(x) + (rnd >> 19)));
    }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    using R = float;
    __device__ static R load(const T *p, float) { return __bfloat162float(__ldg(p)); }
    __device__ static R cvt(T v, float) { return __bfloat162float(v); }
    __device__ static T pack(R v, float) { return __float2bfloat16_rn(v); }
    // stochastic rounding: 16 random bits added below the BF16 mantissa, then truncation
    __device__ static T pack_sr(R v, float, uint32_t rnd)
    {
        const uint32_t b = __float_as_uint(v) + (rnd >> 16);
        return __ushort_as_bfloat16((unsigned short)(b >> 16));
    }
};

// Random bits for the stochastic rounding of population k of a cell: cell_hash mixes the
// cell index once (SplitMix-style finaliser), then one multiply per direction folds in the
// value's own bits.
__device__ __forceinline__ uint32_t cell_hash(uint32_t cell)
{
    uint32_t h = cell * 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    return h ^ (h >> 16);
}
__device__ __forceinline__ uint32_t round_bits(uint32_t h, int k, float v)
{
    return (h ^ __float_as_uint(v)) * (0x9E3779B1u + 0x6A09E666u * (uint32_t)k);
}

inline size_t storage_bytes(int s) { return s == ST_F64 ? 8 : (s == ST_F32 ? 4 : 2); }

// ------------------------------------------------------------------------------------
// Unsigned 32-bit division by a run-time invariant divisor d >= 1 with one multiply-high
// (Granlund & Montgomery, "Division by invariant integers using multiplication", PLDI
// 1994, the round-up method with an N+1-bit multiplier): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n), n / d = (t + ((n - t) >> sh1)) >> sh2
// with sh1 = min(l, 1), sh2 = max(l - 1, 0).  Exact for every 32-bit n.
// ------------------------------------------------------------------------------------
struct FastDiv {
    uint32_t d, m, sh1, sh2;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    f.sh1 = l < 1 ? l : 1;
    f.sh2 = l > 1 ? l - 1 : 0;
    return f;
}

__host__ __device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv &f)
{
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(n, f.m);
#else
    const uint32_t t = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
    return (t + ((n - t) >> f.sh1)) >> f.sh2;
}

// Status word bits: a reduction saw a diverged cell; a bounded wait ran out; (checked
// build) a kernel met an index outside its arrays and skipped the access.
enum { STATUS_DIVERGED = 1u, STATUS_TIMEOUT = 2u, STATUS_BOUNDS = 4u };

// ------------------------------------------------------------------------------------
// Per-instance parameters, read by every kernel from a device table so that one launch
// can advance many independent cells (the batched sweep) or just one.
//
// Geometry is described per 32-cell segment (cells 32s .. 32s+31 of the linear index):
//   seg[s].x  bit l set: cell 32s+l is solid or beyond the box (no work)
//   seg[s].y  bit l set: cell 32s+l is fluid with at least one solid pull source
//   seg[s].z  index of the first such boundary cell of the segment in the boundary table
// fcell[j] is the j-th fluid cell in cell order (the state kernels' list).  The step kernels
// take work items of one warp each (geometry.cu, pack_items): a box segment whose 32 cells
// are all fluid, or up to 32 fluid cells of partly solid segments in cell order, the lanes
// after an item's last cell padding.  For item w: fwarp[w].x bit l set when lane l's cell is
// a boundary cell, fwarp[w].y the index of the item's first link; flane[32w + l] = {x, y}:
// x the cell (bits 0-27) with bit 28 x = 0, bit 29 x = nx - 1, bit 30 all the item's cells
// away from the y and z faces (0xFFFFFFFF: padding lane); y the wall mask (bits 0-18, as
// bmask below, 0 for other cells) and the cell's first link - fwarp[w].y (bits 19-31), so
// that a step needs no dependent load and no division to find a cell's walls and its
// periodic fix-ups.
// Boundary cell b: bmask[b] bit k set when x - e_k is solid (the pull of direction k hits
// the wall), boff[b] the index of its first link; its links are ordered by k.  Link l:
// linkc[l] = CLI coefficient (1-2q)/(1+2q) (0 where CLI falls back to SBB).
// ------------------------------------------------------------------------------------
struct InstanceDev {
    void *f0, *f1;           // populations [19][ks] (direction k at k * ks); AA uses f0 only
    const uint4 *seg;        // [nseg]
    const uint4 *aseg;       // [n_active_padded]: seg entries of segments holding fluid, .w = segment
    const uint32_t *fcell;   // [n_fluid] (padded)
    const uint2 *flane;      // [32 n_fwarps_padded]
    const uint2 *fwarp;      // [n_fwarps_padded]
    const uint32_t *bmask;   // [n_boundary]
    const uint32_t *boff;    // [n_boundary]
    const void *linkc;       // [n_links], type R
    const void *linkw;       // [n_links][kLinkW], type R (walls >= LBM_LIBB), else NULL
    double *partials;        // [n_tiles of this instance][kRedSlots]
    long long ncells;
    uint32_t n32;            // ncells
    uint32_t ks;             // elements between consecutive direction arrays (>= ncells; 19 ks < 2^32)
    uint32_t n_active;       // entries of aseg
    uint32_t n_fwarps;       // step work items (entries of fwarp before the padding)
    // interior cells (no periodic wrap): element offset of the pulled population of
    // direction k relative to the cell, and (AA) of the pushed one (mod 2^32)
    uint32_t pull_off[Q];
    uint32_t push_off[Q];
    FastDiv div_nx, div_ny;  // division by nx and ny
    int nx, ny, nz;
    int wall;                // 0 = SBB, 1 = CLI, 2 = LIBB, 3 = QIBB, 4 = IEBB, 5 = MR
    int phase;               // A-B: buffer holding the current state when flip == 0
    float scale, inv_scale;  // FP16 deviation scaling
    double omega;            // SRT omega = 1/tau; TRT omega+
    double omega_m;          // TRT omega-
    double s[Q];             // MRT relaxation rates
    double delta_rho, rho0;
    // the same parameters as the step kernels use them, computed on the host so that no
    // thread converts or divides them: single precision for the formats that collide in FP32
    // (each the correctly rounded single of the double above, 1/rho0 the correctly rounded
    // quotient), and the MRT rates divided by |M_i|^2 in both precisions
    float omega_f, omega_m_f, rho0_f, irho0_f, delta_rho_f;
    double irho0;
    float rate_f[Q];
    double rate_d[Q];
    // sizes the checked build tests indices against, and the batch's sticky error word
    // (STATUS_BOUNDS, STATUS_TIMEOUT), which the host reads with the reductions
    uint32_t n_fwarps_padded, n_boundary, n_links;
    unsigned *error;
};

#ifdef LBM_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// Index test of the checked build (LBM_CHECKED): true when i < n; otherwise it sets
// STATUS_BOUNDS in the batch error word and returns false, and the caller skips the
// access.  The default build compiles it to true.
__device__ __forceinline__ bool checked(const InstanceDev &I, uint32_t i, uint32_t n)
{
    if constexpr (kChecked) {
        if (i >= n) {
            atomicOr(I.error, STATUS_BOUNDS);
            return false;
        }
    }
    return true;
}

// Coefficients of the interpolated wall rules LIBB, QIBB, IEBB and MR (Sec. 2.2.1), one
// row of kLinkW values per cut link (x, kbar), x - e_k solid, in the compute type.  With
// C = g~_kbar(x), B = g~_k(x) (own post-collision values at t), P2 = g~_kbar(x_f2),
// P3 = g~_kbar(x_f3), B2 = g~_k(x_f2) (x_f2 = x + e_k, x_f3 = x + 2 e_k, read across the x
// faces with the pressure shift), J2 = e_kbar . sum_m e_m g~_m(x_f2) and the cell's moments
// drho, u at t, the new g_k is
//   S + alpha P2 + beta P3 + delta B2 + zeta J2,
//   S = eps C + gamma B + X w_kbar (drho + rho0 (theta e_kbar.u + 9/2 (e_kbar.u)^2 - 3/2 u.u)),
// S being the own-cell part each step leaves in the solid slot for the next.  The
// fallbacks of a rule whose x_f2 or x_f3 is solid are folded into the coefficients.
enum { LW_EPS = 0, LW_GAMMA, LW_ALPHA, LW_BETA, LW_DELTA, LW_X, LW_THETA, LW_ZETA, kLinkW };

// A tile: consecutive entries of one instance's work list, processed by one thread block:
// for the step kernels kTileSegs fluid warps (seg0 = the first), for the other kernels
// blockDim/32 entries of the active-segment list (the segments holding fluid).  A batch's
// step tiles also carry the instance's fluid work list, so that a block's work-list loads
// do not wait for its instance's table entry (they are issued together with the table's).
struct TileDev {
    int inst;
    int local;           // tile index within its instance (partials slot)
    long long seg0;      // first entry of the work list
    const uint2 *flane;  // step tiles: the instance's flane and fwarp; else NULL
    const uint2 *fwarp;
};

enum { KIND_AB = 0, KIND_AA_PULL = 1, KIND_AA_LOCAL = 2 };

// The tiles of a batched step launch, as a kernel parameter (constant bank) for batches of up
// to kBatchMapMax instances: instance i owns tiles tile_start[i] .. tile_start[i + 1] - 1 of
// the launch, and its work list is flane[i], fwarp[i].  A block finds its instance by a
// binary search there instead of loading its tile record first, which the work-list loads
// would wait for.  n = 0: the launch reads its tile records (larger batches).
constexpr int kBatchMapMax = 64;
struct BatchMap {
    int n;
    int tile_start[kBatchMapMax + 1];
    const uint2 *flane[kBatchMapMax];
    const uint2 *fwarp[kBatchMapMax];
};
struct NoBatchMap {};
template <bool BATCH> struct MapArgT { using type = NoBatchMap; };
template <> struct MapArgT<true> { using type = BatchMap; };
template <bool BATCH> using MapArg = typename MapArgT<BATCH>::type;

// TMA brick kernel (lbm_tma.cuh): bricks of kBrickX x kBrickY x kBrickZ cells, one thread
// per cell, kBrickStages shared-memory stages per block.
constexpr int kBrickX = 32, kBrickY = 2, kBrickZ = 4;
constexpr int kBrickCells = kBrickX * kBrickY * kBrickZ;
constexpr int kBrickStages = 2;

// Step-kernel tiling: a tile is kTileSegs consecutive work items (32 fluid cells each), one
// per warp of a kStepWarps-warp block.  kTileApiCells is the block_cells value of the C ABI
// that selects this kernel.
constexpr int kStepWarps = 4;
constexpr int kTileSegs = kStepWarps;
constexpr int kTileApiCells = 32 * kTileSegs;
enum { COLL_SRT = 0, COLL_TRT = 1, COLL_MRT = 2 };

// FP64 reduction slots per tile and per instance: sum of (rho - rho0), of u_x, u_y, u_z
// over fluid cells, then the x, y, z momentum exchanged with the solid in the step
// (drag force, Sec. 3), and one unused slot (64-byte rows).
enum { RED_DRHO = 0, RED_U = 1, RED_F = 4, kRedSlots = 8 };

}  // namespace lbm
