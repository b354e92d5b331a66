// lbm_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lbm_gb300.h"
#include "lbm_device.cuh"

namespace lbm {

// Every device buffer the library owns is allocated here, so that the fault injection of
// lbm_debug_fail_alloc_after reaches every out-of-memory path.
cudaError_t dev_alloc(void **p, size_t bytes);
template <typename T> cudaError_t dev_alloc(T **p, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}

// NVTX range for profilers (a no-op unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
};

// Arguments of one launch over a tile list (each tile: up to chunk_segs consecutive
// entries of one instance's active-segment list).
struct Launch {
    const InstanceDev *table;
    const TileDev *tiles;
    int ntiles;
    int chunk_segs;
    int grid, block;
    cudaStream_t stream;
    const BatchMap *map = nullptr;  // a batched step launch: its tiles' instances (n = 0: none)
};

// Arguments of one launch of the TMA brick kernel (single instance, A-B layout): tensor
// maps of the two population buffers (box widths kBrickX and kBrickX + 16 bytes), the
// device list of bricks holding fluid, and an error word for bounded waits that ran out.
struct TmaLaunch {
    CUtensorMap map[2][2];  // [buffer f0 / f1][box narrow / wide]
    const uint32_t *bricks;
    int nbricks;
    int grid;
    unsigned *error;
    cudaStream_t stream;
};

// Per-storage-format kernel entry points (one translation unit per format).
struct FormatOps {
    // one: host copy of the only instance's parameters (passed by value), or NULL for a batch;
    // wx: some instance uses LIBB, QIBB, IEBB or MR (A-B layout)
    // warps: warps per block of a non-reducing SBB/CLI step (2, 4 or 8; the reducing and the
    // interpolated-wall steps run kStepWarps); L.block must be warps * 32
    cudaError_t (*step)(int coll, int kind, const Launch &L, int flip, int reduce, unsigned *status,
                        const InstanceDev *one, int wx, int warps);
    cudaError_t (*init)(const InstanceDev *table, int inst, long long ncells, int layout, int cur,
                        double amp, unsigned long long seed, cudaStream_t s);
    cudaError_t (*import_dir)(const InstanceDev *table, int inst, long long ncells, int layout, int cur,
                              int k, const double *fk, cudaStream_t s);
    cudaError_t (*export_dir)(const InstanceDev *table, int inst, long long ncells, int layout, int cur,
                              int aa_phase, int k, double *fk, cudaStream_t s);
    // fluid-cell state of directions k .. k + nk - 1 in the storage type: to_host = 1
    // gathers them into buf [nk][n_fluid], 0 scatters them from buf (the step-0 arrangement)
    cudaError_t (*state_dir)(const InstanceDev *table, int inst, long long n_fluid, int layout, int cur,
                             int aa_phase, int k, int nk, void *buf, int to_host, cudaStream_t s);
    cudaError_t (*moments)(const Launch &L, int layout, int cur, int aa_phase, int mode, int comp,
                           double *out);
    // TMA brick step (non-reducing, single instance, A-B); one: the instance's parameters
    cudaError_t (*step_tma)(int coll, int wx, const TmaLaunch &T, const InstanceDev &one, int flip);
    // once per kernel, before any launch or capture: opt in to its shared memory; returns
    // the blocks per multiprocessor it can hold (0 on error)
    int (*tma_prepare)(int coll, int wx);
    // wall terms of the stored state into the solid slots (wall_prepare_kernel; layout 0 =
    // A-B from buffer cur, 1 = AA at phase 0)
    cudaError_t (*wall_prepare)(const InstanceDev *table, int inst, long long n_boundary, const long long *bcell,
                                int layout, int cur, cudaStream_t s);
};

const FormatOps &format_ops(int storage);
extern const FormatOps ops_f64, ops_f32, ops_f16, ops_bf16;

// Geometry built on the device for one instance (Sec. 3: flags and wall distances are
// computed once before time stepping).
struct GeometryDev {
    long long ncells = 0, nseg = 0, nseg_padded = 0;
    long long n_fluid = 0, n_boundary = 0, n_links = 0, n_links_cli = 0;
    uint8_t *solid = nullptr;      // [ncells]
    uint4 *seg = nullptr;          // [nseg_padded]
    uint4 *aseg = nullptr;         // [n_active_padded] segments holding fluid: {x, y, z, segment}
    long long n_active = 0, n_active_padded = 0;
    uint32_t *fcell = nullptr;     // [n_fcell_padded] fluid cells in cell order (pad 0xFFFFFFFF)
    long long n_fcell = 0, n_fcell_padded = 0;
    uint2 *flane = nullptr;        // [32 n_fwarps_padded] the step work items' cells with their
                                   // wall masks, link offsets and face flags (lbm_device.cuh)
    uint2 *fwarp = nullptr;        // [n_fwarps_padded] per work item: boundary bits, first link
    long long n_fwarps = 0, n_fwarps_padded = 0;
    uint32_t *bmask = nullptr;     // [n_boundary]
    uint32_t *boff = nullptr;      // [n_boundary]
    long long *bcell = nullptr;    // [n_boundary] cell index of each boundary cell
    double *linkq = nullptr;       // [n_links] wall distance q (FP64)
    void *linkc = nullptr;         // [n_links] CLI coefficient, compute type
    void *linkw = nullptr;         // [n_links][kLinkW] rule coefficients (LIBB, QIBB, IEBB, MR)
    size_t bytes = 0;
};

// Builds the geometry tables.  spheres (host, n*4 doubles) or flags (host [ncells]);
// q_host optional [19][ncells] wall distances indexed by link direction.  linkc (and, for
// walls >= LBM_LIBB, linkw: the coefficients of the rule, see lbm_device.cuh) are written
// as double when c_double, else float; tau enters IEBB's coefficients.  Returns a CUDA error or cudaSuccess;
// *err receives a message on failure.
// The step kernels' work items (32 entries each, padding 0xFFFFFFFF) from the fluid cells in
// increasing cell order (geometry.cu).  Host code.
std::vector<uint32_t> pack_work_items(const std::vector<uint32_t> &cells, long long *n_items);
cudaError_t build_geometry(int nx, int ny, int nz, const double *spheres, int n_spheres,
                           const uint8_t *flags, const double *q_host, bool c_double, int wall, double tau,
                           cudaStream_t s, GeometryDev *g, std::string *err);
void free_geometry(GeometryDev *g);
// Scatter link q values into qk[ncells] for link direction kdir (NaN elsewhere).
cudaError_t export_wall_distances(const GeometryDev &g, int kdir, double *qk, cudaStream_t s);

// Deterministic final sum of each instance's tile partials: out[kRedSlots] = the sum over
// its tile_count tiles of partials[t][...], in a fixed order.  kFinalSlices blocks per
// instance; scratch: kFinalSlices * (RED_F + 3) doubles and counter: one zeroed word per
// instance (the kernel leaves it zero again).
constexpr int kFinalSlices = 32;
cudaError_t launch_final_reduce(const InstanceDev *table, const int *tile_count, int n_inst, double *out,
                                double *scratch, unsigned *counter, cudaStream_t s);

// Error helpers
void set_error(const std::string &msg);

constexpr int kMaxWarpsPerBlock = 32;
// A step work item packed from partly solid box segments spans at most kItemSpan + 1
// consecutive cells (pack_items in geometry.cu).
constexpr long long kItemSpan = 448;
constexpr int kMinChunkSegs = kStepWarps;  // smallest tile (work items) of any kernel: sizes the partial sums
constexpr long long kDirPad = 0;       // extra elements between direction arrays
// Sphere centres may lie at most this many box lengths from the origin along each axis
// (the voxeliser folds displacements into the box one box length at a time).
constexpr int kMaxCentreBoxes = 64;
long long direction_stride(long long ncells);

}  // namespace lbm
