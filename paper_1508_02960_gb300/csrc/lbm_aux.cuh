// lbm_aux.cuh -- kernels around the time step: initial state, import/export of the
// populations as FP64, velocity field and moment sums of the stored state.  All of
// them see the state through canonical(): the post-collision population g~_k(x) in
// either layout.
#pragma once

#include "lbm_device.cuh"
#include "lbm_step.cuh"

namespace lbm {

// Where g~_k(x) of a fluid cell lives.  A-B: slot k of the current buffer.  AA after a
// LOCAL step (or import): own slot kbar.  AA after a PULL step: slot k of x + e_k (a
// solid cell's slot when x + e_k is solid: the link's own slot there).
template <int STORE>
__device__ __forceinline__ long long canonical_index(const InstanceDev &I, int layout, int aa_phase,
                                                     int cur, long long cell, int k, uint32_t wm,
                                                     const long long (&X)[3], const long long (&Y)[3],
                                                     const long long (&Z)[3], int &buf)
{
    const long long N = I.ks;
    if (layout == 0) {
        buf = cur;
        return (long long)k * N + cell;
    }
    buf = 0;
    (void)wm;
    if (aa_phase == 0) return (long long)opp(k) * N + cell;
    return (long long)k * N + X[1 + ex(k)] + Y[1 + ey(k)] + Z[1 + ez(k)];
}

struct CellGeom {
    long long cell;
    int x, y, z;
    long long X[3], Y[3], Z[3];
    uint32_t wm, off;
};

__device__ __forceinline__ void cell_geom(const InstanceDev &I, long long cell, uint4 meta, int lane,
                                          CellGeom &c)
{
    const int nx = I.nx, ny = I.ny, nz = I.nz;
    c.cell = cell;
    c.x = (int)(cell % nx);
    const long long yz = cell / nx;
    c.y = (int)(yz % ny);
    c.z = (int)(yz / ny);
    const long long nxy = (long long)nx * ny;
    c.X[0] = c.x == 0 ? nx - 1 : c.x - 1;
    c.X[1] = c.x;
    c.X[2] = c.x == nx - 1 ? 0 : c.x + 1;
    c.Y[0] = (long long)(c.y == 0 ? ny - 1 : c.y - 1) * nx;
    c.Y[1] = (long long)c.y * nx;
    c.Y[2] = (long long)(c.y == ny - 1 ? 0 : c.y + 1) * nx;
    c.Z[0] = (long long)(c.z == 0 ? nz - 1 : c.z - 1) * nxy;
    c.Z[1] = (long long)c.z * nxy;
    c.Z[2] = (long long)(c.z == nz - 1 ? 0 : c.z + 1) * nxy;
    c.wm = 0u;
    c.off = 0u;
    if ((meta.y >> lane) & 1u) {
        const uint32_t b = meta.z + __popc(meta.y & ((1u << lane) - 1u));
        c.wm = I.bmask[b];
        c.off = I.boff[b];
    }
}

// SplitMix64 finaliser (Steele, Lea & Flood 2014) as a counter-based hash.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double hash_uniform_pm1(unsigned long long seed, long long cell, int comp)
{
    const unsigned long long h = mix64(seed ^ mix64((unsigned long long)cell * 3ull + (unsigned long long)comp));
    return ((double)(h >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

// Equilibrium initial state g_k = f^eq_k(rho0, u) - w_k rho0 for fluid cells (u = 0 or a
// seeded perturbation of amplitude amp), 0 in solid cells.  Writes the layout's
// post-collision form (A-B buffer `cur`, or AA phase 0); the wall terms follow from
// wall_prepare_kernel.
template <int STORE>
__global__ void init_kernel(const InstanceDev *__restrict__ table, int inst, int layout, int cur,
                            double amp, unsigned long long seed)
{
    using S = Store<STORE>;
    using T = typename S::T;
    const InstanceDev &I = table[inst];
    const long long N = I.ncells;
    const int lane = threadIdx.x & 31;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < N;
         cell += (long long)gridDim.x * blockDim.x) {
        const uint4 meta = I.seg[cell >> 5];
        T *f = reinterpret_cast<T *>(layout == 0 ? (cur ? I.f1 : I.f0) : I.f0);
        if ((meta.x >> lane) & 1u) {
#pragma unroll
            for (int k = 0; k < Q; ++k) f[(long long)k * I.ks + cell] = S::pack(0.0f, I.scale);
            continue;
        }
        double u[3] = {0.0, 0.0, 0.0};
        if (amp != 0.0)
            for (int a = 0; a < 3; ++a) u[a] = amp * hash_uniform_pm1(seed, cell, a);
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const double eu = ex(k) * u[0] + ey(k) * u[1] + ez(k) * u[2];
            const double g = weight(k) * I.rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
            f[(long long)(layout == 0 ? k : opp(k)) * I.ks + cell] = S::pack((typename S::R)g, I.scale);
        }
    }
}

// The own-cell part S of every wall rule (wall_own_part), from the stored post-collision
// state, into the solid slot the next step's pull of direction k reads (the steps
// themselves leave S there for the step after them): A-B, from buffer cur into slot k of
// the solid cell x - e_k; AA at phase 0 (the state after a LOCAL step, where own slot m
// holds g~_mbar), into slot kbar of x - e_k.  For a state set from outside: the initial
// state, imported populations.  One thread per boundary cell; every solid slot belongs to
// one link only.
template <int STORE>
__global__ void wall_prepare_kernel(const InstanceDev *__restrict__ table, int inst, long long nb,
                                    const long long *__restrict__ bcell, int layout, int cur)
{
    using S = Store<STORE>;
    using T = typename S::T;
    using R = typename S::R;
    const InstanceDev &I = table[inst];
    T *f = reinterpret_cast<T *>(layout == 0 && cur ? I.f1 : I.f0);
    const R *linkc = reinterpret_cast<const R *>(I.linkc);
    const long long ks = I.ks, nx = I.nx, ny = I.ny, nz = I.nz;
    constexpr bool sr = sizeof(T) == 2;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
         b += (long long)gridDim.x * blockDim.x) {
        const long long cell = bcell[b];
        const uint32_t wm = I.bmask[b], off = I.boff[b];
        const long long x = cell % nx, yz = cell / nx, y = yz % ny, z = yz / ny;
        const uint32_t h = sr ? cell_hash((uint32_t)cell) : 0u;
        // the cell's moments at t (for IEBB): the post-collision state conserves them
        R drho = R(0), u[3] = {R(0), R(0), R(0)};
        if (I.wall == 4) {
            for (int m = 0; m < Q; ++m) {
                const R gm = S::load(f + (long long)(layout == 0 ? m : opp(m)) * ks + cell, I.inv_scale);
                drho += gm;
                u[0] += R(ex(m)) * gm;
                u[1] += R(ey(m)) * gm;
                u[2] += R(ez(m)) * gm;
            }
            for (int a = 0; a < 3; ++a) u[a] /= R(I.rho0);
        }
        const R *linkw = reinterpret_cast<const R *>(I.linkw);
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (!((wm >> k) & 1u)) continue;
            const int kb = opp(k);
            // C = g~_kbar(x), B = g~_k(x): slots kbar and k in A-B, k and kbar in AA
            const R C = S::load(f + (long long)(layout == 0 ? kb : k) * ks + cell, I.inv_scale);
            const R B = S::load(f + (long long)(layout == 0 ? k : kb) * ks + cell, I.inv_scale);
            const uint32_t l = off + __popc(wm & ((1u << k) - 1u));
            R sv;
            if (I.wall >= 2) {  // as wall_own_part_w in the step kernel
                const R *lw = linkw + (size_t)l * kLinkW;
                sv = fma_r(lw[LW_GAMMA], B, lw[LW_EPS] * C);
                const R X = lw[LW_X];
                if (X != R(0)) {
                    const R eu = R(ex(kb)) * u[0] + R(ey(kb)) * u[1] + R(ez(kb)) * u[2];
                    const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                    const R fst = drho + R(I.rho0) * (lw[LW_THETA] * eu + R(4.5) * eu * eu - R(1.5) * uu);
                    sv = fma_r(X * R(weight(kb)), fst, sv);
                }
            } else {
                const R cq = I.wall == 1 ? linkc[l] : R(0);
                sv = wall_own_part(I.wall, cq, C, B);
            }
            const long long src = (x - ex(k) + nx) % nx + nx * ((y - ey(k) + ny) % ny + ny * ((z - ez(k) + nz) % nz));
            f[(long long)(layout == 0 ? k : kb) * ks + src] =
                sr ? S::pack_sr(sv, I.scale, round_bits(h, k, float(sv))) : S::pack(sv, I.scale);
        }
    }
}

// Import direction k from FP64 f (cells of one direction): g = f - w rho0.
template <int STORE>
__global__ void import_kernel(const InstanceDev *__restrict__ table, int inst, int layout, int cur, int k,
                              const double *__restrict__ fk)
{
    using S = Store<STORE>;
    using T = typename S::T;
    const InstanceDev &I = table[inst];
    const long long N = I.ncells;
    const int lane = threadIdx.x & 31;
    const double wr = weight(k) * I.rho0;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < N;
         cell += (long long)gridDim.x * blockDim.x) {
        const uint4 meta = I.seg[cell >> 5];
        T *f = reinterpret_cast<T *>(layout == 0 ? (cur ? I.f1 : I.f0) : I.f0);
        const long long slot = (long long)(layout == 0 ? k : opp(k)) * I.ks + cell;
        if ((meta.x >> lane) & 1u) {
            f[slot] = S::pack(0.0f, I.scale);
            continue;
        }
        f[slot] = S::pack((typename S::R)(fk[cell] - wr), I.scale);
    }
}

// Export direction k as FP64 f = w rho0 + g~ (0 in solid cells).
template <int STORE>
__global__ void export_kernel(const InstanceDev *__restrict__ table, int inst, int layout, int cur,
                              int aa_phase, int k, double *__restrict__ fk)
{
    using S = Store<STORE>;
    using T = typename S::T;
    const InstanceDev &I = table[inst];
    const long long N = I.ncells;
    const int lane = threadIdx.x & 31;
    const double wr = weight(k) * I.rho0;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < N;
         cell += (long long)gridDim.x * blockDim.x) {
        const uint4 meta = I.seg[cell >> 5];
        if ((meta.x >> lane) & 1u) {
            fk[cell] = 0.0;
            continue;
        }
        CellGeom c;
        cell_geom(I, cell, meta, lane, c);
        int buf;
        const long long idx = canonical_index<STORE>(I, layout, aa_phase, cur, cell, k, c.wm, c.X, c.Y, c.Z, buf);
        const T *f = reinterpret_cast<const T *>(buf ? I.f1 : I.f0);
        fk[cell] = wr + (double)S::load(f + idx, I.inv_scale);
    }
}

// The stored state of directions k0 + blockIdx.y of the fluid cells, bit for bit, in the
// storage type: out[blockIdx.y * nf + j] = the stored g~_k of fluid cell j (cells in cell
// order, from the work list), read where the layout keeps it (as export_kernel).
template <int STORE>
__global__ void state_gather_kernel(const InstanceDev *__restrict__ table, int inst, int layout, int cur,
                                    int aa_phase, int k0, long long nf, typename Store<STORE>::T *__restrict__ out)
{
    using T = typename Store<STORE>::T;
    const InstanceDev &I = table[inst];
    const int k = k0 + (int)blockIdx.y;
    out += (long long)blockIdx.y * nf;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nf;
         j += (long long)gridDim.x * blockDim.x) {
        const long long cell = I.fcell[j];
        const int lane = (int)(cell & 31);
        CellGeom c;
        cell_geom(I, cell, I.seg[cell >> 5], lane, c);
        int buf;
        const long long idx = canonical_index<STORE>(I, layout, aa_phase, cur, cell, k, c.wm, c.X, c.Y, c.Z, buf);
        out[j] = reinterpret_cast<const T *>(buf ? I.f1 : I.f0)[idx];
    }
}

// The inverse for a state set from outside (as import_kernel, without conversion):
// direction k = k0 + blockIdx.y of fluid cell j from in[blockIdx.y * nf + j] into its slot
// of the step-0 arrangement.  Solid cells are left alone (their wall terms are rebuilt by
// wall_prepare_kernel).
template <int STORE>
__global__ void state_scatter_kernel(const InstanceDev *__restrict__ table, int inst, int layout, int cur, int k0,
                                     long long nf, const typename Store<STORE>::T *__restrict__ in)
{
    using T = typename Store<STORE>::T;
    const InstanceDev &I = table[inst];
    const int k = k0 + (int)blockIdx.y;
    in += (long long)blockIdx.y * nf;
    T *f = reinterpret_cast<T *>(layout == 0 ? (cur ? I.f1 : I.f0) : I.f0);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nf;
         j += (long long)gridDim.x * blockDim.x) {
        const long long cell = I.fcell[j];
        f[(long long)(layout == 0 ? k : opp(k)) * I.ks + cell] = in[j];
    }
}

// Moments of the stored post-collision state of every fluid cell, one warp per work
// chunk.  mode 0: write the velocity component `comp` to out[cell] of fluid cells (the
// caller clears out first).  mode 1: chunk partial sums (drho, u_x, u_y, u_z) into
// I.partials, in FP64 in a fixed order; the force slots, which only a step defines, are
// written as 0.
template <int STORE>
__global__ void __launch_bounds__(256) moments_kernel(const InstanceDev *__restrict__ table,
                                                      const TileDev *__restrict__ chunks, int nchunks, int chunk_segs,
                                                      int layout, int cur, int aa_phase, int mode, int comp,
                                                      double *__restrict__ out)
{
    using S = Store<STORE>;
    using T = typename S::T;
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * (long long)blockDim.x) >> 5);
    for (int c = gw; c < nchunks; c += nw) {
        const TileDev chunk = chunks[c];
        const InstanceDev &I = table[chunk.inst];
        const int n_e = min(chunk_segs, (int)(I.n_active - (uint32_t)chunk.seg0));
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < n_e; ++i) {
            const uint4 meta = I.aseg[chunk.seg0 + i];
            const long long cell = (long long)meta.w * 32 + lane;
            if ((meta.x >> lane) & 1u) continue;
            CellGeom c;
            cell_geom(I, cell, meta, lane, c);
            double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                int buf;
                const long long idx =
                    canonical_index<STORE>(I, layout, aa_phase, cur, cell, k, c.wm, c.X, c.Y, c.Z, buf);
                const T *f = reinterpret_cast<const T *>(buf ? I.f1 : I.f0);
                const double g = (double)S::load(f + idx, I.inv_scale);
                drho += g;
                j[0] += ex(k) * g;
                j[1] += ey(k) * g;
                j[2] += ez(k) * g;
            }
            if (mode == 0) {
                out[cell] = j[comp] / I.rho0;
            } else {
                a[0] += drho;
                for (int d = 0; d < 3; ++d) a[1 + d] += j[d] / I.rho0;
            }
        }
        if (mode == 1) {
#pragma unroll
            for (int d = 0; d < 4; ++d) a[d] = warp_sum(a[d]);
            if (lane == 0)
                for (int d = 0; d < kRedSlots; ++d) I.partials[(long long)chunk.local * kRedSlots + d] = d < 4 ? a[d] : 0.0;
        }
    }
}

}  // namespace lbm
