// batch.h -- host runtime object behind contexts, batches and the server: a set of
// independent periodic cells that share storage format, collision operator and layout
// and advance together, one kernel launch per time step over the tiles of all of them.
#pragma once

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "lbm_internal.h"

namespace lbm {

struct Instance {
    lbm_desc desc{};               // copy; pointer members cleared
    std::vector<double> mrt_rates; // explicit MRT rates when given
    GeometryDev geo;
    void *f0 = nullptr, *f1 = nullptr;
    double *partials = nullptr;
    long long partial_capacity = 0;  // tiles
    int phase = 0;                   // A-B buffer holding the state when the batch flip is 0
    int dev_scale_log2 = 0;
    double d_p = 0.0;
    double r_sum = 0.0, area_sum = 0.0;  // sum of sphere radii and of pi r^2 (0: flag geometry)
    long long steps = 0;
    // results of the last reduction (slots RED_DRHO, RED_U.., RED_F..)
    double sums[kRedSlots] = {};
    unsigned status = 0;
    bool have_sums = false;
    bool have_force = false;         // sums[RED_F..] come from a step (not a state reduction)
    bool sums_pending = false;       // the last queued step reduced the moments
    size_t bytes_pop = 0;
    long long ks = 0;                // elements between direction arrays

    Instance() = default;
    Instance(const Instance &) = delete;
    Instance &operator=(const Instance &) = delete;
    ~Instance();                     // frees the instance's device memory
};

// Block shape of the non-reducing SBB/CLI step: warps per block, one tile of that many work
// items per block.
struct StepShape {
    int warps = kStepWarps;
};
constexpr int kShapeWarps[] = {4, 2, 8};  // the candidates, in the order they are timed
static_assert(kShapeWarps[0] == kStepWarps, "shape 0 is the reducing step's (its tile map serves both)");
constexpr int kShapeWarpsN = 3;

class Batch {
public:
    ~Batch();
    // Validates and builds one instance (geometry + memory).  Does not initialise state.
    static lbm_status make_instance(const lbm_desc &d, cudaStream_t s, std::unique_ptr<Instance> *out);
    // Footprint estimate (bytes) of an instance before building it.
    static size_t footprint(const lbm_desc &d);

    lbm_status init(cudaStream_t user_stream, int storage, int collision, int layout);
    // AA batches: after an even number of steps only (the instances share one arrangement)
    lbm_status add(std::unique_ptr<Instance> inst);
    lbm_status remove(int i);                          // releases device memory of instance i
    int size() const { return (int)inst_.size(); }
    Instance &at(int i) { return *inst_[i]; }

    lbm_status init_equilibrium(int i);                // i < 0: all
    lbm_status step(long long n);                      // queue n steps (+ final reduction)
    lbm_status moment_sums_now(int i, double *sums);   // sums[4] of the stored state (synchronises)
    lbm_status fetch_sums();                           // copy last reduction to host (synchronises)
    lbm_status get_f64(int i, double *host);
    lbm_status set_f64(int i, const double *host);
    // fluid-cell state in the storage type, bit for bit ([19][n_fluid]; see lbm_get_state)
    lbm_status state_io(int i, void *host, size_t bytes, bool to_host);
    // prefetched states ([19][n_fluid] each): copy into staging now, apply later
    lbm_status stage_state(int i, const void *host, size_t bytes);
    lbm_status apply_staged_state(int i);
    lbm_status get_velocity(int i, double *host);
    lbm_status get_flags(int i, uint8_t *host);
    lbm_status get_q(int i, double *host);
    lbm_status save(int i, const char *path);
    lbm_status load(int i, const char *path);
    lbm_status sync();
    void fill_info(int i, lbm_info *out) const;
    long long launches() const { return launches_; }
    int block_cells() const { return tma_ ? kBrickCells : kTileApiCells; }
    int aa_phase() const { return aa_phase_; }
    cudaStream_t stream() const { return stream_; }
    long long fluid_cells() const;
    lbm_status set_block(int block_cells);
    // how the step kernel was chosen (0 = given, 1 = measured now, 2 = from the autotuner
    // cache) and the ms per step measured for the tiles and the bricks
    void set_tuning(int source, double ms_tiles, double ms_bricks)
    {
        tune_src_ = source;
        tune_ms_[0] = ms_tiles;
        tune_ms_[1] = ms_bricks;
    }
    lbm_status prepare();              // upload tables and choose the step kernel now if pending

private:
    struct GraphKey {
        long long steps_red;
        int flip, aa, shape;
        bool operator<(const GraphKey &o) const
        {
            return std::tie(steps_red, flip, aa, shape) < std::tie(o.steps_red, o.flip, o.aa, o.shape);
        }
    };
    struct CachedGraph {
        cudaGraphExec_t exec;
        long long used;
    };
    static constexpr size_t kGraphCache = 16;  // instantiated step graphs kept per batch
    Launch shaped_launch(const StepShape &sh, int kind) const;
    lbm_status graph_for(long long m, bool red, const StepShape &sh, int wx, cudaGraphExec_t *out);
    void lookup_shape();                // the cached shape of this batch, or tuning pending
    lbm_status tune_shape(int wx);      // time every candidate shape on the live state
    lbm_status rebuild();          // upload table and tiles, drop graphs
    lbm_status aa_restart(int i);  // instance i (i < 0: all) set from outside: AA arrangement of step 0
    int cur_of(const Instance &in) const { return in.phase ^ flip_; }
    const FormatOps &ops() const { return format_ops(storage_); }

    std::vector<std::unique_ptr<Instance>> inst_;
    int tune_src_ = 0;
    double tune_ms_[2] = {0.0, 0.0};
    int storage_ = 0, collision_ = 0, layout_ = 0;
    cudaStream_t stream_ = nullptr;   // user stream (launches)
    cudaStream_t cap_ = nullptr;      // private stream for graph capture
    InstanceDev *d_table_ = nullptr;
    std::vector<InstanceDev> h_table_;  // host copy (the single-instance launch passes it by value)
    TileDev *d_tiles_ = nullptr;      // tiles of the active-segment lists (state kernels)
    int *d_tile_count_ = nullptr;
    TileDev *d_stiles_ = nullptr;     // tiles of the fluid-warp lists (step kernels)
    int *d_stile_count_ = nullptr;
    int nstiles_ = 0;
    double *d_sums_ = nullptr;        // [n][kRedSlots]
    unsigned *d_status_ = nullptr;    // [n]
    double *h_sums_ = nullptr;        // pinned [n][kRedSlots]
    unsigned *h_status_ = nullptr;    // pinned [n]
    int capacity_ = 0;
    int ntiles_ = 0;
    int block_ = 32 * kStepWarps;      // cells per chunk of the state kernels
    int step_mode_ = 0;               // 0 (default) and 1: tiles of fluid cells; 2: TMA bricks
    // TMA brick kernel (single instance, A-B layout, box a multiple of the brick)
    bool tma_ = false;
    TmaLaunch tma_launch_{};
    uint32_t *d_bricks_ = nullptr;
    unsigned *d_error_ = nullptr;
    lbm_status setup_tma();           // decides tma_ and builds maps and brick list
    int grid_ = 0;                    // step-kernel blocks (one per step tile)
    int aux_grid_ = 1;
    int flip_ = 0;
    int aa_phase_ = 0;
    bool dirty_ = true;
    long long launches_ = 0;
    std::map<GraphKey, CachedGraph> graphs_;
    long long graph_clock_ = 0;
    // tiles of every block shape of the non-reducing step
    TileDev *d_wtiles_[kShapeWarpsN] = {nullptr, nullptr, nullptr};
    int nwtiles_[kShapeWarpsN] = {0, 0, 0};
    // the same tiles as kernel-parameter maps (batches of 2 .. kBatchMapMax instances)
    BatchMap maps_[kShapeWarpsN] = {};
    StepShape shape_;
    int shape_src_ = 0;                // 0 default, 1 measured by this batch, 2 from the cache
    double shape_ms_[kShapeWarpsN] = {0, 0, 0};
    bool tune_shape_ = false;
    int sms_ = 0;
    double *d_stage_ = nullptr;       // FP64 staging for import/export (one direction)
    long long stage_cells_ = 0;
    // state transfers: two staging buffers of one direction each, a copy stream, and
    // events: ev_[b] buffer b filled, ev_[2 + b] buffer b free again
    void *d_sstage_[2] = {nullptr, nullptr};
    // final reduction: per instance kFinalSlices rows of partial sums and a block counter
    double *d_fscratch_ = nullptr;
    unsigned *d_fcount_ = nullptr;
    size_t sstage_bytes_ = 0;
    cudaStream_t copy_ = nullptr;
    cudaEvent_t ev_[4] = {nullptr, nullptr, nullptr, nullptr};
    // prefetched states: two full staging buffers used in turn; ev_staged_[b] copy into b
    // done, ev_free_[b] the scatter out of b done; n_staged_ states waiting from slot head_
    void *d_pstage_[2] = {nullptr, nullptr};
    size_t pstage_bytes_ = 0;
    cudaEvent_t ev_staged_[2] = {nullptr, nullptr}, ev_free_[2] = {nullptr, nullptr};
    bool pstage_used_[2] = {false, false};
    int n_staged_ = 0, head_ = 0, staged_inst_[2] = {0, 0};
    lbm_status ensure_copy_stream();
};

lbm_status fail(lbm_status st, const std::string &msg);
// Checks a descriptor without touching the GPU.
lbm_status validate_desc(const lbm_desc &d);
// Observables of an instance's last reduction (Eqs. Darcy, Forchheimer, frictionFactor).
void compute_obs(const Instance &in, double K_D, lbm_obs *out);
// Step kernel of a single-instance batch chosen by measurement (block_cells = LBM_BLOCK_AUTO).
lbm_status autotune_block(Batch &b, const lbm_desc &d, cudaStream_t s);
lbm_status cuda_fail(cudaError_t e, const char *what);

}  // namespace lbm
