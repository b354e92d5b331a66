// lbm_format_impl.cuh -- instantiates every kernel of one storage format and exposes
// them through a FormatOps table.  Included once per format translation unit, so the
// formats compile in parallel.
#pragma once

#include <utility>

#include "lbm_aux.cuh"
#include "lbm_internal.h"
#include "lbm_step.cuh"
#include "lbm_tma.cuh"

namespace lbm {
namespace detail {

// Launch of a step kernel with programmatic stream serialisation: the kernel may start
// (up to its wait on the previous step) while the previous kernel of the stream is still
// running.  Captured into a graph, this becomes a programmatic dependency edge.
template <typename... P, typename... A>
cudaError_t launch_step(void (*kernel)(P...), const Launch &L, A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)L.grid);
    cfg.blockDim = dim3((unsigned)L.block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

template <int STORE, int COLL, int KIND, bool RED, bool WX, int WARPS>
cudaError_t step_red(const Launch &L, int flip, unsigned *status, const InstanceDev *one)
{
    cudaError_t e;
    if (one) {  // a single instance: parameters travel in the constant bank
        e = launch_step(step_kernel<COLL, STORE, KIND, false, RED, WX, WARPS>, L, L.table, *one, NoBatchMap{}, L.tiles,
                        L.ntiles, flip, status);
    } else {  // a batch: parameters from the device table, the tiles' instances from the map
        static const InstanceDev unused{};
        static const BatchMap no_map{};  // n = 0: tile records
        e = launch_step(step_kernel<COLL, STORE, KIND, true, RED, WX, WARPS>, L, L.table, unused,
                        L.map ? *L.map : no_map, L.tiles, L.ntiles, flip, status);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// wx: some instance uses an interpolated wall rule (LIBB, QIBB, IEBB, MR; A-B only).
// warps: warps per block of a non-reducing SBB/CLI step (2, 4 or 8); the reducing and the
// interpolated-wall steps run kStepWarps.
template <int STORE, int COLL, int KIND>
cudaError_t step_one(const Launch &L, int flip, int reduce, unsigned *status, const InstanceDev *one, int wx,
                     int warps)
{
    if constexpr (KIND == KIND_AB) {
        if (wx)
            return reduce ? step_red<STORE, COLL, KIND, true, true, kStepWarps>(L, flip, status, one)
                          : step_red<STORE, COLL, KIND, false, true, kStepWarps>(L, flip, status, one);
    } else {
        if (wx) return cudaErrorInvalidValue;
    }
    if (reduce) return step_red<STORE, COLL, KIND, true, false, kStepWarps>(L, flip, status, one);
    switch (warps) {
    case 2: return step_red<STORE, COLL, KIND, false, false, 2>(L, flip, status, one);
    case 8: return step_red<STORE, COLL, KIND, false, false, 8>(L, flip, status, one);
    default: return step_red<STORE, COLL, KIND, false, false, kStepWarps>(L, flip, status, one);
    }
}

template <int STORE>
cudaError_t step(int coll, int kind, const Launch &L, int flip, int reduce, unsigned *status, const InstanceDev *one,
                 int wx, int warps)
{
    switch (coll * 3 + kind) {
    case COLL_SRT * 3 + KIND_AB: return step_one<STORE, COLL_SRT, KIND_AB>(L, flip, reduce, status, one, wx, warps);
    case COLL_SRT * 3 + KIND_AA_PULL:
        return step_one<STORE, COLL_SRT, KIND_AA_PULL>(L, flip, reduce, status, one, wx, warps);
    case COLL_SRT * 3 + KIND_AA_LOCAL:
        return step_one<STORE, COLL_SRT, KIND_AA_LOCAL>(L, flip, reduce, status, one, wx, warps);
    case COLL_TRT * 3 + KIND_AB: return step_one<STORE, COLL_TRT, KIND_AB>(L, flip, reduce, status, one, wx, warps);
    case COLL_TRT * 3 + KIND_AA_PULL:
        return step_one<STORE, COLL_TRT, KIND_AA_PULL>(L, flip, reduce, status, one, wx, warps);
    case COLL_TRT * 3 + KIND_AA_LOCAL:
        return step_one<STORE, COLL_TRT, KIND_AA_LOCAL>(L, flip, reduce, status, one, wx, warps);
    case COLL_MRT * 3 + KIND_AB: return step_one<STORE, COLL_MRT, KIND_AB>(L, flip, reduce, status, one, wx, warps);
    case COLL_MRT * 3 + KIND_AA_PULL:
        return step_one<STORE, COLL_MRT, KIND_AA_PULL>(L, flip, reduce, status, one, wx, warps);
    case COLL_MRT * 3 + KIND_AA_LOCAL:
        return step_one<STORE, COLL_MRT, KIND_AA_LOCAL>(L, flip, reduce, status, one, wx, warps);
    default: return cudaErrorInvalidValue;
    }
}

template <int STORE, int COLL, bool WX> auto tma_kernel() { return step_kernel_tma<COLL, STORE, WX>; }

template <int STORE, int COLL, bool WX>
cudaError_t step_tma_one(const TmaLaunch &T, const InstanceDev &one, int flip)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)T.grid);
    cfg.blockDim = dim3((unsigned)kBrickCells);
    cfg.dynamicSmemBytes = BrickStage<STORE>::SMEM_BYTES;
    cfg.stream = T.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, tma_kernel<STORE, COLL, WX>(), one, T.map[0][0], T.map[0][1],
                                       T.map[1][0], T.map[1][1], T.bricks, T.nbricks, flip, T.error);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int STORE>
cudaError_t step_tma(int coll, int wx, const TmaLaunch &T, const InstanceDev &one, int flip)
{
    switch (coll * 2 + (wx ? 1 : 0)) {
    case COLL_SRT * 2: return step_tma_one<STORE, COLL_SRT, false>(T, one, flip);
    case COLL_SRT * 2 + 1: return step_tma_one<STORE, COLL_SRT, true>(T, one, flip);
    case COLL_TRT * 2: return step_tma_one<STORE, COLL_TRT, false>(T, one, flip);
    case COLL_TRT * 2 + 1: return step_tma_one<STORE, COLL_TRT, true>(T, one, flip);
    case COLL_MRT * 2: return step_tma_one<STORE, COLL_MRT, false>(T, one, flip);
    case COLL_MRT * 2 + 1: return step_tma_one<STORE, COLL_MRT, true>(T, one, flip);
    default: return cudaErrorInvalidValue;
    }
}

template <int STORE, int COLL, bool WX> int tma_prepare_one()
{
    const int smem = BrickStage<STORE>::SMEM_BYTES;
    if (cudaFuncSetAttribute(tma_kernel<STORE, COLL, WX>(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tma_kernel<STORE, COLL, WX>(), kBrickCells, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <int STORE> int tma_prepare(int coll, int wx)
{
    switch (coll * 2 + (wx ? 1 : 0)) {
    case COLL_SRT * 2: return tma_prepare_one<STORE, COLL_SRT, false>();
    case COLL_SRT * 2 + 1: return tma_prepare_one<STORE, COLL_SRT, true>();
    case COLL_TRT * 2: return tma_prepare_one<STORE, COLL_TRT, false>();
    case COLL_TRT * 2 + 1: return tma_prepare_one<STORE, COLL_TRT, true>();
    case COLL_MRT * 2: return tma_prepare_one<STORE, COLL_MRT, false>();
    case COLL_MRT * 2 + 1: return tma_prepare_one<STORE, COLL_MRT, true>();
    default: return 0;
    }
}

inline int flat_grid(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

template <int STORE>
cudaError_t init(const InstanceDev *table, int inst, long long n, int layout, int cur, double amp,
                 unsigned long long seed, cudaStream_t s)
{
    init_kernel<STORE><<<flat_grid(n, 256), 256, 0, s>>>(table, inst, layout, cur, amp, seed);
    return cudaGetLastError();
}

template <int STORE>
cudaError_t import_dir(const InstanceDev *table, int inst, long long n, int layout, int cur, int k,
                       const double *fk, cudaStream_t s)
{
    import_kernel<STORE><<<flat_grid(n, 256), 256, 0, s>>>(table, inst, layout, cur, k, fk);
    return cudaGetLastError();
}

template <int STORE>
cudaError_t export_dir(const InstanceDev *table, int inst, long long n, int layout, int cur, int aa_phase,
                       int k, double *fk, cudaStream_t s)
{
    export_kernel<STORE><<<flat_grid(n, 256), 256, 0, s>>>(table, inst, layout, cur, aa_phase, k, fk);
    return cudaGetLastError();
}

template <int STORE>
cudaError_t state_dir(const InstanceDev *table, int inst, long long nf, int layout, int cur, int aa_phase, int k,
                      int nk, void *buf, int to_host, cudaStream_t s)
{
    if (nf <= 0 || nk <= 0) return cudaSuccess;
    using T = typename Store<STORE>::T;
    const dim3 grid((unsigned)flat_grid(nf, 256), (unsigned)nk);
    if (to_host)
        state_gather_kernel<STORE>
            <<<grid, 256, 0, s>>>(table, inst, layout, cur, aa_phase, k, nf, static_cast<T *>(buf));
    else
        state_scatter_kernel<STORE><<<grid, 256, 0, s>>>(table, inst, layout, cur, k, nf, static_cast<const T *>(buf));
    return cudaGetLastError();
}

template <int STORE>
cudaError_t moments(const Launch &L, int layout, int cur, int aa_phase, int mode, int comp, double *out)
{
    moments_kernel<STORE><<<L.grid, L.block, 0, L.stream>>>(L.table, L.tiles, L.ntiles, L.chunk_segs, layout, cur,
                                                            aa_phase, mode, comp, out);
    return cudaGetLastError();
}

template <int STORE>
cudaError_t wall_prepare(const InstanceDev *table, int inst, long long nb, const long long *bcell, int layout,
                         int cur, cudaStream_t s)
{
    if (nb <= 0) return cudaSuccess;
    wall_prepare_kernel<STORE><<<flat_grid(nb, 128), 128, 0, s>>>(table, inst, nb, bcell, layout, cur);
    return cudaGetLastError();
}

template <int STORE>
FormatOps make_ops()
{
    FormatOps o;
    o.step = &step<STORE>;
    o.init = &init<STORE>;
    o.import_dir = &import_dir<STORE>;
    o.export_dir = &export_dir<STORE>;
    o.state_dir = &state_dir<STORE>;
    o.moments = &moments<STORE>;
    o.wall_prepare = &wall_prepare<STORE>;
    o.step_tma = &step_tma<STORE>;
    o.tma_prepare = &tma_prepare<STORE>;
    return o;
}

}  // namespace detail
}  // namespace lbm
