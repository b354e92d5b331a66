// lbm_format_impl.cuh -- instantiates every kernel of one storage format and exposes
// them through a FormatOps table.  Included once per format translation unit, so the
// formats compile in parallel.
#pragma once

#include "lbm_aux.cuh"
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbm {
namespace detail {

template <int STORE, int COLL, int KIND>
cudaError_t step_one(const Launch &L, int flip, int reduce, unsigned *status, const InstanceDev *one)
{
    if (one) {  // a single instance: parameters travel in the constant bank
        step_kernel<COLL, STORE, KIND, false><<<L.grid, L.block, 0, L.stream>>>(L.table, *one, L.tiles, L.ntiles, flip,
                                                                               reduce, status);
    } else if constexpr (KIND == KIND_AB) {
        static const InstanceDev unused{};
        step_kernel<COLL, STORE, KIND, true><<<L.grid, L.block, 0, L.stream>>>(L.table, unused, L.tiles, L.ntiles, flip,
                                                                              reduce, status);
    } else {
        return cudaErrorInvalidValue;  // the AA layout runs single instances only
    }
    return cudaGetLastError();
}

template <int STORE>
cudaError_t step(int coll, int kind, const Launch &L, int flip, int reduce, unsigned *status, const InstanceDev *one)
{
    switch (coll * 3 + kind) {
    case COLL_SRT * 3 + KIND_AB: return step_one<STORE, COLL_SRT, KIND_AB>(L, flip, reduce, status, one);
    case COLL_SRT * 3 + KIND_AA_PULL: return step_one<STORE, COLL_SRT, KIND_AA_PULL>(L, flip, reduce, status, one);
    case COLL_SRT * 3 + KIND_AA_LOCAL: return step_one<STORE, COLL_SRT, KIND_AA_LOCAL>(L, flip, reduce, status, one);
    case COLL_TRT * 3 + KIND_AB: return step_one<STORE, COLL_TRT, KIND_AB>(L, flip, reduce, status, one);
    case COLL_TRT * 3 + KIND_AA_PULL: return step_one<STORE, COLL_TRT, KIND_AA_PULL>(L, flip, reduce, status, one);
    case COLL_TRT * 3 + KIND_AA_LOCAL: return step_one<STORE, COLL_TRT, KIND_AA_LOCAL>(L, flip, reduce, status, one);
    case COLL_MRT * 3 + KIND_AB: return step_one<STORE, COLL_MRT, KIND_AB>(L, flip, reduce, status, one);
    case COLL_MRT * 3 + KIND_AA_PULL: return step_one<STORE, COLL_MRT, KIND_AA_PULL>(L, flip, reduce, status, one);
    case COLL_MRT * 3 + KIND_AA_LOCAL: return step_one<STORE, COLL_MRT, KIND_AA_LOCAL>(L, flip, reduce, status, one);
    default: return cudaErrorInvalidValue;
    }
}

template <int STORE>
const void *step_ptr(int coll, int kind)
{
    switch (coll * 3 + kind) {
    case COLL_SRT * 3 + KIND_AB: return (const void *)step_kernel<COLL_SRT, STORE, KIND_AB, false>;
    case COLL_SRT * 3 + KIND_AA_PULL: return (const void *)step_kernel<COLL_SRT, STORE, KIND_AA_PULL, false>;
    case COLL_SRT * 3 + KIND_AA_LOCAL: return (const void *)step_kernel<COLL_SRT, STORE, KIND_AA_LOCAL, false>;
    case COLL_TRT * 3 + KIND_AB: return (const void *)step_kernel<COLL_TRT, STORE, KIND_AB, false>;
    case COLL_TRT * 3 + KIND_AA_PULL: return (const void *)step_kernel<COLL_TRT, STORE, KIND_AA_PULL, false>;
    case COLL_TRT * 3 + KIND_AA_LOCAL: return (const void *)step_kernel<COLL_TRT, STORE, KIND_AA_LOCAL, false>;
    case COLL_MRT * 3 + KIND_AB: return (const void *)step_kernel<COLL_MRT, STORE, KIND_AB, false>;
    case COLL_MRT * 3 + KIND_AA_PULL: return (const void *)step_kernel<COLL_MRT, STORE, KIND_AA_PULL, false>;
    case COLL_MRT * 3 + KIND_AA_LOCAL: return (const void *)step_kernel<COLL_MRT, STORE, KIND_AA_LOCAL, false>;
    default: return nullptr;
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
cudaError_t moments(const Launch &L, int layout, int cur, int aa_phase, int mode, int comp, double *out)
{
    moments_kernel<STORE><<<L.grid, L.block, 0, L.stream>>>(L.table, L.tiles, L.ntiles, L.chunk_segs, layout, cur,
                                                            aa_phase, mode, comp, out);
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
    o.moments = &moments<STORE>;
    o.step_kernel_ptr = &step_ptr<STORE>;
    return o;
}

}  // namespace detail
}  // namespace lbm
