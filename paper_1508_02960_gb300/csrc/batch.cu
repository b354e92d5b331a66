// batch.cu -- runtime of a set of independent periodic cells advanced together.
//
// One time step of every instance is one launch of the fused step kernel over a tile
// list of work chunks (chunks never span two instances and their partial sums are kept
// per chunk, so each instance's reduction order is the same alone or in a mix).  Repeated step sequences are captured once as CUDA graphs
// (n steps + the final FP64 reduction) and replayed on the caller's stream.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>

#include "batch.h"
#include "lbm_step.cuh"

namespace lbm {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
const char *last_error_cstr() { return g_last_error.c_str(); }

lbm_status fail(lbm_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

lbm_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_NO_MEMORY : LBM_ERR_CUDA;
}

const FormatOps &format_ops(int storage)
{
    switch (storage) {
    case ST_F64: return ops_f64;
    case ST_F32: return ops_f32;
    case ST_F16: return ops_f16;
    default: return ops_bf16;
    }
}

#define CK(x)                                                 \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x);      \
    } while (0)

// ------------------------------------------------------------------------------------
// Descriptor validation and defaults
// ------------------------------------------------------------------------------------
lbm_status validate_desc(const lbm_desc &d)
{
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return fail(LBM_ERR_ARG, "nx, ny, nz must be >= 1");
    const long long n = (long long)d.nx * d.ny * d.nz;
    // the kernels address populations with 32-bit element offsets: 19 * stride < 2^32
    if (19 * direction_stride(n) >= (1ll << 32))
        return fail(LBM_ERR_ARG, "box too large: 19 * nx * ny * nz must be below 2^32");
    if (!(d.tau > 0.5) || !std::isfinite(d.tau)) return fail(LBM_ERR_ARG, "tau must be a finite value > 1/2");
    if (!std::isfinite(d.delta_rho)) return fail(LBM_ERR_ARG, "delta_rho must be finite");
    if (d.rho0 < 0 || !std::isfinite(d.rho0)) return fail(LBM_ERR_ARG, "rho0 must be >= 0 (0 = 1)");
    if (d.collision < LBM_SRT || d.collision > LBM_MRT) return fail(LBM_ERR_ARG, "unknown collision operator");
    if (d.wall < LBM_SBB || d.wall > LBM_MR) return fail(LBM_ERR_ARG, "unknown wall rule");
    if (d.wall >= LBM_LIBB && d.layout != LBM_LAYOUT_AB)
        return fail(LBM_ERR_ARG, "LIBB, QIBB, IEBB and MR walls need the A-B layout");
    if (d.wall == LBM_IEBB && std::fabs(d.tau - 2.0) < 1e-12)
        return fail(LBM_ERR_ARG, "IEBB needs tau != 2 (its q < 1/2 weight is (2q-1)/(tau-2))");
    if (d.storage < LBM_F64 || d.storage > LBM_BF16DEV) return fail(LBM_ERR_ARG, "unknown storage format");
    if (d.layout < LBM_LAYOUT_AB || d.layout > LBM_LAYOUT_AA) return fail(LBM_ERR_ARG, "unknown layout");
    if (d.n_spheres < 0) return fail(LBM_ERR_ARG, "n_spheres < 0");
    if (d.n_spheres > 0 && !d.spheres) return fail(LBM_ERR_ARG, "n_spheres > 0 but spheres is NULL");
    for (int i = 0; i < d.n_spheres; ++i) {
        const lbm_sphere &s = d.spheres[i];
        if (!std::isfinite(s.cx) || !std::isfinite(s.cy) || !std::isfinite(s.cz) || !(s.r > 0) || !std::isfinite(s.r))
            return fail(LBM_ERR_ARG, "sphere " + std::to_string(i) + " has a non-finite centre or radius <= 0");
        // the device folds a displacement into the box one box length at a time: a centre
        // far outside it would take that many iterations per cell (or never end, once
        // d - n rounds back to d)
        if (std::fabs(s.cx) > kMaxCentreBoxes * d.nx || std::fabs(s.cy) > kMaxCentreBoxes * d.ny ||
            std::fabs(s.cz) > kMaxCentreBoxes * d.nz)
            return fail(LBM_ERR_ARG, "sphere " + std::to_string(i) + " has a centre more than " +
                                         std::to_string(kMaxCentreBoxes) + " box lengths from the origin");
    }
    if (d.magic_lambda < 0 || !std::isfinite(d.magic_lambda)) return fail(LBM_ERR_ARG, "magic_lambda must be >= 0");
    if (d.mrt_energy_ratio < 0 || !std::isfinite(d.mrt_energy_ratio))
        return fail(LBM_ERR_ARG, "mrt_energy_ratio must be >= 0");
    if (d.block_cells != 0 && d.block_cells != LBM_BLOCK_AUTO && d.block_cells != kTileApiCells &&
        d.block_cells != kBrickCells)
        return fail(LBM_ERR_ARG, "block_cells: 0 or 128 (tiles of fluid cells), 256 (TMA bricks) or -1 (autotune)");
    if (d.block_cells == kBrickCells &&
        (d.layout != LBM_LAYOUT_AB || d.nx % kBrickX || d.ny % kBrickY || d.nz % kBrickZ))
        return fail(LBM_ERR_ARG, "TMA bricks need the A-B layout and nx, ny, nz multiples of 32, 2, 4");
    if (d.dev_scale_log2 != LBM_DEV_SCALE_AUTO && (d.dev_scale_log2 < -60 || d.dev_scale_log2 > 60))
        return fail(LBM_ERR_ARG, "dev_scale_log2 out of [-60, 60]");
    if (!std::isfinite(d.perturb_u) || std::fabs(d.perturb_u) > 0.3) return fail(LBM_ERR_ARG, "|perturb_u| > 0.3");
    if (d.d_p < 0 || !std::isfinite(d.d_p)) return fail(LBM_ERR_ARG, "d_p must be >= 0");
    return LBM_OK;
}

// Elements between consecutive direction arrays: the cell count rounded up to 64 elements
// plus kDirPad, so that the 19 read and 19 write streams of a step do not all start at
// the same power-of-two offset.
long long direction_stride(long long ncells)
{
    return (ncells + 63) / 64 * 64 + kDirPad;
}

static int auto_dev_scale(const lbm_desc &d)
{
    if (d.storage != LBM_F16DEV) return 0;
    if (d.dev_scale_log2 != LBM_DEV_SCALE_AUTO) return d.dev_scale_log2;
    // the largest deviations are of the order of the density drop; map it near 2^12
    const double dr = std::max(std::fabs(d.delta_rho), 1e-12);
    int s = (int)std::floor(std::log2(4096.0 / dr));
    return std::min(40, std::max(0, s));
}

size_t Batch::footprint(const lbm_desc &d)
{
    const size_t n = (size_t)d.nx * d.ny * d.nz;
    const size_t es = storage_bytes(d.storage);
    const size_t bufs = d.layout == LBM_LAYOUT_AA ? 1 : 2;
    // populations + solid flags + segment table + partials + a boundary-table allowance
    return bufs * Q * (size_t)direction_stride((long long)n) * es + n + (n / 32 + 64) * (16 + 16) + n / 8 +
           (1u << 20);
}

lbm_status Batch::make_instance(const lbm_desc &d0, cudaStream_t s, std::unique_ptr<Instance> *out)
{
    TraceRange trace("lbm.make_instance");
    lbm_status st = validate_desc(d0);
    if (st != LBM_OK) return st;
    std::unique_ptr<Instance> in(new Instance());
    in->desc = d0;
    lbm_desc &d = in->desc;
    if (d.rho0 == 0) d.rho0 = 1.0;
    if (d.magic_lambda == 0) d.magic_lambda = 3.0 / 16.0;
    if (d.mrt_energy_ratio == 0) d.mrt_energy_ratio = 4.6;
    if (d0.mrt_rates) in->mrt_rates.assign(d0.mrt_rates, d0.mrt_rates + Q);
    in->dev_scale_log2 = auto_dev_scale(d0);
    d.dev_scale_log2 = in->dev_scale_log2;
    if (d.d_p > 0) {
        in->d_p = d.d_p;
    } else if (d0.n_spheres > 0) {
        double m3 = 0;
        for (int i = 0; i < d0.n_spheres; ++i) m3 += std::pow(d0.spheres[i].r, 3.0);
        in->d_p = 2.0 * std::cbrt(m3 / d0.n_spheres);
    }
    for (int i = 0; i < d0.n_spheres; ++i) {  // drag normalisation (Eq. AnalyticForce, Sec. 4)
        in->r_sum += d0.spheres[i].r;
        in->area_sum += M_PI * d0.spheres[i].r * d0.spheres[i].r;
    }
    std::vector<double> sph;
    for (int i = 0; i < d0.n_spheres; ++i) {
        sph.push_back(d0.spheres[i].cx);
        sph.push_back(d0.spheres[i].cy);
        sph.push_back(d0.spheres[i].cz);
        sph.push_back(d0.spheres[i].r);
    }
    std::string err;
    cudaError_t e = build_geometry(d.nx, d.ny, d.nz, sph.empty() ? nullptr : sph.data(), d0.n_spheres,
                                   d0.n_spheres > 0 ? nullptr : d0.flags, d0.q, d.storage == LBM_F64, d.wall, d.tau,
                                   s, &in->geo, &err);
    d.spheres = nullptr;
    d.flags = nullptr;
    d.q = nullptr;
    d.mrt_rates = nullptr;
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_NO_MEMORY : LBM_ERR_CUDA, err);

    const long long n = in->geo.ncells;
    const size_t es = storage_bytes(d.storage);
    // 16 bytes of slack: 16-bit formats copy the aligned 32-bit word holding a population
    in->ks = direction_stride(n);
    const size_t pop = (size_t)Q * in->ks * es + 16;
    auto cleanup = [&](cudaError_t ce, const char *what) {  // in's destructor frees the memory
        return cuda_fail(ce, what);
    };
    // Canaries: the padding after each direction's ncells values (and the slack) holds
    // all-ones bytes, a NaN in every storage format, so that a kernel reading there by
    // mistake turns its results non-finite (the divergence flag, the parity tests).
    auto clear = [&](void *f) {
        cudaError_t ce = cudaMemsetAsync(f, 0xFF, pop, s);
        for (int k = 0; k < Q && ce == cudaSuccess; ++k)
            ce = cudaMemsetAsync(static_cast<char *>(f) + (size_t)k * in->ks * es, 0, (size_t)n * es, s);
        return ce;
    };
    if ((e = dev_alloc(&in->f0, pop)) != cudaSuccess) return cleanup(e, "dev_alloc(populations)");
    if ((e = clear(in->f0)) != cudaSuccess) return cleanup(e, "cudaMemset");
    if (d.layout == LBM_LAYOUT_AB) {
        if ((e = dev_alloc(&in->f1, pop)) != cudaSuccess) return cleanup(e, "dev_alloc(populations)");
        if ((e = clear(in->f1)) != cudaSuccess) return cleanup(e, "cudaMemset");
    }
    // partial sums: one row of kRedSlots doubles per tile at the smallest tile size, of the
    // active-segment chunks (state kernels) and of the step work items alike
    in->partial_capacity =
        std::max(1ll, (std::max(in->geo.n_active, in->geo.n_fwarps) + kMinChunkSegs - 1) / kMinChunkSegs);
    if ((e = dev_alloc(&in->partials, sizeof(double) * kRedSlots * in->partial_capacity)) != cudaSuccess)
        return cleanup(e, "dev_alloc(partials)");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cleanup(e, "cudaStreamSynchronize");
    in->bytes_pop = pop * (d.layout == LBM_LAYOUT_AB ? 2 : 1);
    *out = std::move(in);
    return LBM_OK;
}

// ------------------------------------------------------------------------------------
// Batch
// ------------------------------------------------------------------------------------
Instance::~Instance()
{
    cudaFree(f0);
    cudaFree(f1);
    cudaFree(partials);
    free_geometry(&geo);
}

Batch::~Batch()
{
    if (stream_ || cap_) cudaStreamSynchronize(stream_);
    for (auto &kv : graphs_) cudaGraphExecDestroy(kv.second.exec);
    inst_.clear();
    for (int w = 0; w < kShapeWarpsN; ++w) cudaFree(d_wtiles_[w]);
    cudaFree(d_table_);
    cudaFree(d_tiles_);
    cudaFree(d_tile_count_);
    cudaFree(d_stiles_);
    cudaFree(d_stile_count_);
    cudaFree(d_bricks_);
    cudaFree(d_error_);
    cudaFree(d_sums_);
    cudaFree(d_status_);
    cudaFree(d_stage_);
    if (h_sums_) cudaFreeHost(h_sums_);
    if (h_status_) cudaFreeHost(h_status_);
    if (cap_) cudaStreamDestroy(cap_);
    if (copy_) cudaStreamSynchronize(copy_);  // no copy still reads a caller's buffer
    cudaFree(d_sstage_[0]);
    cudaFree(d_sstage_[1]);
    cudaFree(d_pstage_[0]);
    cudaFree(d_pstage_[1]);
    for (int b = 0; b < 2; ++b) {
        if (ev_staged_[b]) cudaEventDestroy(ev_staged_[b]);
        if (ev_free_[b]) cudaEventDestroy(ev_free_[b]);
    }
    cudaFree(d_fscratch_);
    cudaFree(d_fcount_);
    if (copy_) cudaStreamDestroy(copy_);
    for (cudaEvent_t e : ev_)
        if (e) cudaEventDestroy(e);
}

lbm_status Batch::init(cudaStream_t user_stream, int storage, int collision, int layout)
{
    stream_ = user_stream;
    storage_ = storage;
    collision_ = collision;
    layout_ = layout;
    CK(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
    return LBM_OK;
}

lbm_status Batch::add(std::unique_ptr<Instance> in)
{
    const lbm_desc &d = in->desc;
    if (d.storage != storage_ || d.collision != collision_ || d.layout != layout_)
        return fail(LBM_ERR_ARG, "instances of a batch must share storage, collision and layout");
    // the instances of an AA batch share one in-place arrangement: a new one joins when the
    // batch is back in the arrangement of step 0 (after an even number of steps)
    if (layout_ == LBM_LAYOUT_AA && !inst_.empty() && aa_phase_ != 0)
        return fail(LBM_ERR_STATE, "an AA batch takes new instances after an even number of steps only");
    in->phase = 0;
    inst_.push_back(std::move(in));
    dirty_ = true;
    return LBM_OK;
}

lbm_status Batch::remove(int i)
{
    if (i < 0 || i >= size()) return fail(LBM_ERR_ARG, "instance index out of range");
    CK(cudaStreamSynchronize(stream_));
    inst_.erase(inst_.begin() + i);  // the instance frees its device memory
    dirty_ = true;
    return LBM_OK;
}

lbm_status Batch::set_block(int block_cells)
{
    int mode;
    if (block_cells == 0) mode = 0;
    else if (block_cells == kTileApiCells) mode = 1;
    else if (block_cells == kBrickCells) mode = 2;
    else return fail(LBM_ERR_ARG, "block_cells: 0 or 128 (tiles of fluid cells) or 256 (TMA bricks)");
    if (mode != step_mode_) {
        step_mode_ = mode;
        dirty_ = true;
    }
    return LBM_OK;
}

lbm_status Batch::prepare()
{
    if (!dirty_ || size() == 0) return LBM_OK;
    return rebuild();
}

long long Batch::fluid_cells() const
{
    long long s = 0;
    for (auto &p : inst_) s += p->geo.n_fluid;
    return s;
}

static void fill_dev(const Instance &in, InstanceDev &D)
{
    const lbm_desc &d = in.desc;
    std::memset(&D, 0, sizeof(D));
    D.f0 = in.f0;
    D.f1 = in.f1;
    D.seg = in.geo.seg;
    D.aseg = in.geo.aseg;
    D.n_active = (uint32_t)in.geo.n_active;
    D.fcell = in.geo.fcell;
    D.flane = in.geo.flane;
    D.fwarp = in.geo.fwarp;
    D.n_fwarps = (uint32_t)in.geo.n_fwarps;
    D.n_fwarps_padded = (uint32_t)in.geo.n_fwarps_padded;
    D.n_boundary = (uint32_t)in.geo.n_boundary;
    D.n_links = (uint32_t)in.geo.n_links;
    for (int k = 0; k < Q; ++k) {
        const long long dk = ex(k) + (long long)ey(k) * d.nx + (long long)ez(k) * d.nx * d.ny;  // e_k as an offset
        const long long arr = d.layout == LBM_LAYOUT_AA ? opp(k) : k;
        D.pull_off[k] = (uint32_t)(arr * in.ks - dk);
        D.push_off[k] = (uint32_t)((long long)k * in.ks + dk);
    }
    D.bmask = in.geo.bmask;
    D.boff = in.geo.boff;
    D.linkc = in.geo.linkc;
    D.linkw = in.geo.linkw;
    D.partials = in.partials;
    D.ncells = in.geo.ncells;
    D.n32 = (uint32_t)in.geo.ncells;
    D.ks = (uint32_t)in.ks;
    D.div_nx = make_fastdiv((uint32_t)d.nx);
    D.div_ny = make_fastdiv((uint32_t)d.ny);
    D.nx = d.nx;
    D.ny = d.ny;
    D.nz = d.nz;
    D.wall = d.wall;
    D.phase = in.phase;
    D.scale = std::ldexp(1.0f, in.dev_scale_log2);
    D.inv_scale = std::ldexp(1.0f, -in.dev_scale_log2);
    const double tau = d.tau;
    D.omega = 1.0 / tau;
    D.omega_m = 1.0 / (0.5 + d.magic_lambda / (tau - 0.5));
    if (!in.mrt_rates.empty()) {
        for (int i = 0; i < Q; ++i) D.s[i] = in.mrt_rates[i];
    } else {
        // Sec. 2.1: s_nu = 1/tau on the viscous modes, s_zeta = 8(2-s_nu)/(8-s_nu) on the
        // kinetic modes, energy modes by the ratio rule, conserved modes 0.
        const double snu = 1.0 / tau;
        const double sz = 8.0 * (2.0 - snu) / (8.0 - snu);
        const double se = 1.0 / (0.5 + (tau - 0.5) / d.mrt_energy_ratio);
        for (int i = 0; i < Q; ++i) D.s[i] = sz;
        D.s[0] = D.s[3] = D.s[5] = D.s[7] = 0.0;
        D.s[9] = D.s[11] = D.s[13] = D.s[14] = D.s[15] = snu;
        D.s[1] = D.s[2] = se;
    }
    D.delta_rho = d.delta_rho;
    D.rho0 = d.rho0;
    D.omega_f = (float)D.omega;
    D.omega_m_f = (float)D.omega_m;
    D.rho0_f = (float)D.rho0;
    D.irho0_f = 1.0f / D.rho0_f;
    D.delta_rho_f = (float)D.delta_rho;
    D.irho0 = 1.0 / D.rho0;
    for (int i = 0; i < Q; ++i) {
        D.rate_f[i] = (float)D.s[i] / (float)mrt_norm2(i);
        D.rate_d[i] = D.s[i] / (double)mrt_norm2(i);
    }
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to the driver library)
typedef CUresult (*TensorMapEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                         const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                         CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                         CUtensorMapFloatOOBfill);

static TensorMapEncodeTiled tensor_map_encoder()
{
    static std::mutex mu;
    static TensorMapEncodeTiled fn = nullptr;
    static bool tried = false;
    std::lock_guard<std::mutex> lk(mu);
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TensorMapEncodeTiled>(p);
    }
    return fn;
}

lbm_status Batch::setup_tma()
{
    tma_ = false;
    cudaFree(d_bricks_);
    d_bricks_ = nullptr;
    // the brick kernel runs on request only (block_cells = kBrickCells): on the sphere cells
    // measured here the tile kernel over fluid cells is faster (see lbm_tma.cuh)
    auto not_here = [&](const char *why) { return fail(LBM_ERR_ARG, why); };
    if (step_mode_ != 2) return LBM_OK;
    if (size() != 1 || layout_ != LBM_LAYOUT_AB) return not_here("TMA bricks run single A-B instances only");
    Instance &in = *inst_[0];
    const lbm_desc &d = in.desc;
    if (d.nx % kBrickX || d.ny % kBrickY || d.nz % kBrickZ)
        return not_here("TMA bricks need nx, ny, nz multiples of 32, 2, 4");
    if (d.nx / kBrickX > 1024 || d.ny / kBrickY > 2048 || d.nz / kBrickZ > 2048)
        return not_here("box too large for the brick list (nx <= 32768, ny <= 4096, nz <= 8192)");
    TensorMapEncodeTiled enc = tensor_map_encoder();
    if (!enc) return not_here("cuTensorMapEncodeTiled is not available");
    const int wx = d.wall >= LBM_LIBB;
    const int per_sm = ops().tma_prepare(collision_, wx);
    if (per_sm <= 0) return not_here("the TMA brick kernel does not fit on a multiprocessor");
    // bricks holding fluid, from the 32-cell segment table
    const long long nseg = in.geo.nseg;
    std::vector<uint4> seg((size_t)nseg);
    CK(cudaMemcpy(seg.data(), in.geo.seg, sizeof(uint4) * nseg, cudaMemcpyDeviceToHost));
    const int bx_n = d.nx / kBrickX, by_n = d.ny / kBrickY, bz_n = d.nz / kBrickZ;
    std::vector<uint32_t> list;
    for (int bz = 0; bz < bz_n; ++bz)
        for (int by = 0; by < by_n; ++by)
            for (int bx = 0; bx < bx_n; ++bx) {
                bool fluid = false;
                for (int dz = 0; dz < kBrickZ && !fluid; ++dz)
                    for (int dy = 0; dy < kBrickY && !fluid; ++dy) {
                        const long long y = (long long)by * kBrickY + dy, z = (long long)bz * kBrickZ + dz;
                        fluid = seg[(size_t)(bx + (long long)bx_n * (y + (long long)d.ny * z))].x != 0xFFFFFFFFu;
                    }
                if (fluid) list.push_back((uint32_t)bx | (uint32_t)by << 10 | (uint32_t)bz << 21);
            }
    if (list.empty()) return not_here("no fluid");
    CK(dev_alloc(&d_bricks_, sizeof(uint32_t) * list.size()));
    CK(cudaMemcpy(d_bricks_, list.data(), sizeof(uint32_t) * list.size(), cudaMemcpyHostToDevice));
    // tensor maps [nz][ny][nx] x 19 directions of both buffers, boxes kBrickX and kBrickX + 16 B wide
    const size_t es = storage_bytes(storage_);
    const CUtensorMapDataType dt = storage_ == LBM_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : storage_ == LBM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : storage_ == LBM_F16DEV ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[4] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {(cuuint64_t)d.nx * es, (cuuint64_t)d.nx * d.ny * es, (cuuint64_t)in.ks * es};
    const cuuint32_t boxes[2][4] = {{(cuuint32_t)kBrickX, kBrickY, kBrickZ, 1},
                                    {(cuuint32_t)(kBrickX + 16 / es), kBrickY, kBrickZ, 1}};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int b = 0; b < 2; ++b)
        for (int w = 0; w < 2; ++w) {
            const CUresult r = enc(&tma_launch_.map[b][w], dt, 4, b ? in.f1 : in.f0, dims, strides, boxes[w], estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return not_here("cuTensorMapEncodeTiled rejected the population layout");
        }
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    tma_launch_.bricks = d_bricks_;
    tma_launch_.nbricks = (int)list.size();
    tma_launch_.grid = (int)std::min<long long>((long long)list.size(), (long long)per_sm * sms);
    tma_launch_.error = d_error_;
    tma_launch_.stream = stream_;
    tma_ = true;
    return LBM_OK;
}

lbm_status Batch::rebuild()
{
    CK(cudaStreamSynchronize(stream_));
    const int n = size();
    const int CS = block_ / 32;  // segments per work chunk
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!d_error_) {  // the batch's sticky error word (bounded waits, checked build)
        CK(dev_alloc(&d_error_, sizeof(unsigned)));
        CK(cudaMemset(d_error_, 0, sizeof(unsigned)));
    }
    std::vector<InstanceDev> table(std::max(n, 1));
    std::vector<TileDev> tiles, stiles, wtiles[kShapeWarpsN];
    std::vector<int> tc(std::max(n, 1)), sc(std::max(n, 1));  // tiles of each instance
    for (int i = 0; i < n; ++i) {
        Instance &in = *inst_[i];
        fill_dev(in, table[i]);
        table[i].error = d_error_;
        // state kernels: chunks of the active-segment list
        const long long nt = std::max(1ll, (in.geo.n_active + CS - 1) / CS);
        // step kernels: kTileSegs fluid warps per tile (the list is padded to whole tiles)
        const long long ns = std::max(1ll, (in.geo.n_fwarps + kTileSegs - 1) / kTileSegs);
        if (nt > in.partial_capacity || ns > in.partial_capacity) return fail(LBM_ERR_STATE, "partials too small");
        if (ns * kTileSegs > in.geo.n_fwarps_padded) return fail(LBM_ERR_STATE, "fluid work list too short");
        tc[i] = (int)nt;
        for (long long t = 0; t < nt; ++t) tiles.push_back(TileDev{i, (int)t, t * CS, nullptr, nullptr});
        sc[i] = (int)ns;
        for (long long t = 0; t < ns; ++t)
            stiles.push_back(TileDev{i, (int)t, t * kTileSegs, in.geo.flane, in.geo.fwarp});
        // tiles of the other block shapes of the non-reducing step (no partial sums)
        for (int w = 0; w < kShapeWarpsN; ++w) {
            const int W = kShapeWarps[w];
            // at least one tile, as for the reducing step, whose tiles the kShapeWarps[0]
            // map also describes (an instance without fluid has one tile of padding)
            const long long nw = std::max(1ll, (in.geo.n_fwarps + W - 1) / W);
            if (i < kBatchMapMax) {
                maps_[w].tile_start[i] = (int)wtiles[w].size();
                maps_[w].flane[i] = in.geo.flane;
                maps_[w].fwarp[i] = in.geo.fwarp;
            }
            if (nw * W > in.geo.n_fwarps_padded) return fail(LBM_ERR_STATE, "fluid work list too short");
            for (long long t = 0; t < nw; ++t)
                wtiles[w].push_back(TileDev{i, (int)t, t * W, in.geo.flane, in.geo.fwarp});
        }
    }
    if (tiles.size() > (size_t)INT32_MAX || stiles.size() > (size_t)INT32_MAX)
        return fail(LBM_ERR_ARG, "too many tiles");
    for (int w = 0; w < kShapeWarpsN; ++w) {  // maps for batches of 2 .. kBatchMapMax instances
        maps_[w].n = (n >= 2 && n <= kBatchMapMax) ? n : 0;
        if (maps_[w].n) maps_[w].tile_start[n] = (int)wtiles[w].size();
    }
    ntiles_ = (int)tiles.size();
    nstiles_ = (int)stiles.size();
    cudaFree(d_table_);
    cudaFree(d_tiles_);
    cudaFree(d_tile_count_);
    cudaFree(d_stiles_);
    cudaFree(d_stile_count_);
    d_table_ = nullptr;
    d_tiles_ = d_stiles_ = nullptr;
    d_tile_count_ = d_stile_count_ = nullptr;
    h_table_ = table;
    CK(dev_alloc(&d_table_, sizeof(InstanceDev) * table.size()));
    CK(cudaMemcpy(d_table_, table.data(), sizeof(InstanceDev) * table.size(), cudaMemcpyHostToDevice));
    if (ntiles_ > 0) {
        CK(dev_alloc(&d_tiles_, sizeof(TileDev) * tiles.size()));
        CK(cudaMemcpy(d_tiles_, tiles.data(), sizeof(TileDev) * tiles.size(), cudaMemcpyHostToDevice));
    }
    CK(dev_alloc(&d_tile_count_, sizeof(int) * tc.size()));
    CK(cudaMemcpy(d_tile_count_, tc.data(), sizeof(int) * tc.size(), cudaMemcpyHostToDevice));
    if (nstiles_ > 0) {
        CK(dev_alloc(&d_stiles_, sizeof(TileDev) * stiles.size()));
        CK(cudaMemcpy(d_stiles_, stiles.data(), sizeof(TileDev) * stiles.size(), cudaMemcpyHostToDevice));
    }
    for (int w = 0; w < kShapeWarpsN; ++w) {
        cudaFree(d_wtiles_[w]);
        d_wtiles_[w] = nullptr;
        nwtiles_[w] = (int)wtiles[w].size();
        if (nwtiles_[w] > 0) {
            CK(dev_alloc(&d_wtiles_[w], sizeof(TileDev) * wtiles[w].size()));
            CK(cudaMemcpy(d_wtiles_[w], wtiles[w].data(), sizeof(TileDev) * wtiles[w].size(),
                          cudaMemcpyHostToDevice));
        }
    }
    CK(dev_alloc(&d_stile_count_, sizeof(int) * sc.size()));
    CK(cudaMemcpy(d_stile_count_, sc.data(), sizeof(int) * sc.size(), cudaMemcpyHostToDevice));
    if (n > capacity_) {
        cudaFree(d_sums_);
        cudaFree(d_status_);
        cudaFree(d_fscratch_);
        cudaFree(d_fcount_);
        d_fscratch_ = nullptr;
        d_fcount_ = nullptr;
        if (h_sums_) cudaFreeHost(h_sums_);
        if (h_status_) cudaFreeHost(h_status_);
        d_sums_ = nullptr;
        d_status_ = nullptr;
        h_sums_ = nullptr;
        h_status_ = nullptr;
        capacity_ = std::max(n, 2 * capacity_);
        CK(dev_alloc(&d_sums_, sizeof(double) * kRedSlots * capacity_));
        CK(dev_alloc(&d_status_, sizeof(unsigned) * capacity_));
        CK(cudaMemset(d_status_, 0, sizeof(unsigned) * capacity_));
        CK(dev_alloc(&d_fscratch_, sizeof(double) * (RED_F + 3) * kFinalSlices * capacity_));
        CK(dev_alloc(&d_fcount_, sizeof(unsigned) * capacity_));
        CK(cudaMemset(d_fcount_, 0, sizeof(unsigned) * capacity_));
        CK(cudaMallocHost(&h_sums_, sizeof(double) * kRedSlots * capacity_));
        CK(cudaMallocHost(&h_status_, sizeof(unsigned) * capacity_));
    }
    // one step block per tile; the hardware block scheduler balances the tiles
    grid_ = std::max(1, nstiles_);
    sms_ = sms;
    for (auto &kv : graphs_) cudaGraphExecDestroy(kv.second.exec);
    graphs_.clear();
    shape_ = StepShape{};
    shape_src_ = 0;
    aux_grid_ = std::max(1, std::min(sms * 8, (ntiles_ + 7) / 8));
    lbm_status st = setup_tma();
    if (st != LBM_OK) return st;
    lookup_shape();
    dirty_ = false;
    return LBM_OK;
}

// A state set from outside is written in the AA arrangement of step 0.  In a batch of
// several AA instances that is possible only while the others are in it too.
lbm_status Batch::aa_restart(int i)
{
    if (layout_ != LBM_LAYOUT_AA || aa_phase_ == 0) return LBM_OK;
    if (i >= 0 && size() > 1)
        return fail(LBM_ERR_STATE, "an AA batch sets one instance's state after an even number of steps only");
    aa_phase_ = 0;
    return LBM_OK;
}

lbm_status Batch::init_equilibrium(int i)
{
    {
        lbm_status st = aa_restart(i);
        if (st != LBM_OK) return st;
    }
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    for (int j = 0; j < size(); ++j) {
        if (i >= 0 && j != i) continue;
        Instance &in = *inst_[j];
        CK(ops().init(d_table_, j, in.geo.ncells, layout_, cur_of(in), in.desc.perturb_u,
                      (unsigned long long)in.desc.seed, stream_));
        ++launches_;
        if (in.geo.n_boundary > 0) {
            CK(ops().wall_prepare(d_table_, j, in.geo.n_boundary, in.geo.bcell, layout_, cur_of(in), stream_));
            ++launches_;
        }
        in.have_sums = false;
        in.have_force = false;
        in.sums_pending = false;
        in.steps = 0;
    }
    return LBM_OK;
}

struct StepQueue {
    const FormatOps *ops;
    Launch L;                // the reducing step (kStepWarps-warp tiles, one block each)
    Launch Ln[2];            // the non-reducing steps (the tuned shape), by AA kind (A-B: [0])
    int warps;               // warps per block of Ln
    const InstanceDev *one;  // single instance: its parameters by value; else NULL
    int wx;                  // some instance uses an interpolated wall rule
    const TmaLaunch *tma;    // non-reducing steps on the TMA brick kernel; else NULL
    int collision, layout;
    unsigned *status;
    int n_status;
    const int *tile_count;
    double *sums;
    int n_inst;
    double *fscratch;
    unsigned *fcount;
};

// Queue n steps on stream s starting from (flip, aa); returns launches queued.
static cudaError_t queue_steps(const StepQueue &q, cudaStream_t s, long long n, bool reduce_last, int &flip,
                               int &aa, long long &launches)
{
    Launch L = q.L;
    L.stream = s;
    for (long long i = 0; i < n; ++i) {
        const bool red = reduce_last && i == n - 1;
        if (red) {
            cudaError_t e = cudaMemsetAsync(q.status, 0, sizeof(unsigned) * q.n_status, s);
            if (e != cudaSuccess) return e;
        }
        const int kind = q.layout == LBM_LAYOUT_AB ? KIND_AB : (aa == 0 ? KIND_AA_PULL : KIND_AA_LOCAL);
        cudaError_t e;
        if (!red && q.tma) {  // the reducing step always runs the tile kernel
            TmaLaunch T = *q.tma;
            T.stream = s;
            e = q.ops->step_tma(q.collision, q.wx, T, *q.one, flip);
        } else if (red || q.wx) {  // the reducing and interpolated-wall steps: kStepWarps tiles
            e = q.ops->step(q.collision, kind, L, flip, red ? 1 : 0, q.status, q.one, q.wx, kStepWarps);
        } else {
            Launch Ls = q.Ln[kind == KIND_AA_LOCAL ? 1 : 0];
            Ls.stream = s;
            e = q.ops->step(q.collision, kind, Ls, flip, 0, q.status, q.one, 0, q.warps);
        }
        if (e != cudaSuccess) return e;
        ++launches;
        if (q.layout == LBM_LAYOUT_AB) flip ^= 1;
        else aa ^= 1;
    }
    if (reduce_last && n > 0) {
        cudaError_t e = launch_final_reduce(q.L.table, q.tile_count, q.n_inst, q.sums, q.fscratch, q.fcount, s);
        if (e != cudaSuccess) return e;
        ++launches;
    }
    return cudaSuccess;
}

// Launch of the non-reducing step of AA kind (or A-B) `kind` in block shape sh.
Launch Batch::shaped_launch(const StepShape &sh, int kind) const
{
    int w = 0;
    while (w < kShapeWarpsN && kShapeWarps[w] != sh.warps) ++w;
    (void)kind;
    const int nt = nwtiles_[w];
    return Launch{d_table_, d_wtiles_[w], nt, sh.warps, std::max(1, nt), sh.warps * 32, stream_, &maps_[w]};
}

// The graph of m steps (+ the reduction when red) from (flip_, aa_phase_) in shape sh,
// instantiated on first use and kept in a small least-recently-used cache.
lbm_status Batch::graph_for(long long m, bool red, const StepShape &sh, int wx, cudaGraphExec_t *out)
{
    const GraphKey key{m * 2 + (red ? 1 : 0), flip_, aa_phase_, sh.warps};
    auto it = graphs_.find(key);
    if (it != graphs_.end()) {
        it->second.used = ++graph_clock_;
        *out = it->second.exec;
        return LBM_OK;
    }
    if (graphs_.size() >= kGraphCache) {  // evict the least recently used graph
        auto lru = graphs_.begin();
        for (auto g = graphs_.begin(); g != graphs_.end(); ++g)
            if (g->second.used < lru->second.used) lru = g;
        cudaGraphExecDestroy(lru->second.exec);
        graphs_.erase(lru);
    }
    StepQueue q{&ops(),
                Launch{d_table_, d_stiles_, nstiles_, kTileSegs, grid_, kStepWarps * 32, stream_, &maps_[0]},
                {shaped_launch(sh, layout_ == LBM_LAYOUT_AB ? KIND_AB : KIND_AA_PULL),
                 shaped_launch(sh, KIND_AA_LOCAL)},
                sh.warps,
                size() == 1 ? &h_table_[0] : nullptr,
                wx,
                tma_ ? &tma_launch_ : nullptr,
                collision_,
                layout_,
                d_status_,
                size(),
                d_stile_count_,
                d_sums_,
                size(),
                d_fscratch_,
                d_fcount_};
    int f = flip_, a = aa_phase_;
    long long dummy = 0;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = queue_steps(q, cap_, m, red, f, a, dummy);
    cudaError_t e2 = cudaStreamEndCapture(cap_, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e, "capture of step kernels");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    graphs_[key] = CachedGraph{exec, ++graph_clock_};
    *out = exec;
    return LBM_OK;
}

// Block shapes of the non-reducing step, tuned online: every shape gives the same state bit
// for bit (the cells' arithmetic does not depend on how the tiles are grouped), so the first
// steps of a batch time each candidate on the live state.  The choice is cached per
// (storage, collision, layout, instance count, total fluid cells, multiprocessor count) for
// the process.
namespace {
struct ShapeKey {
    int storage, collision, layout, n_inst, sms;
    long long n_fluid;
    bool operator<(const ShapeKey &o) const
    {
        return std::tie(storage, collision, layout, n_inst, sms, n_fluid) <
               std::tie(o.storage, o.collision, o.layout, o.n_inst, o.sms, o.n_fluid);
    }
};
std::mutex g_shape_mu;
std::map<ShapeKey, StepShape> g_shapes;
const StepShape kShapeCandidates[] = {{kShapeWarps[0]}, {kShapeWarps[1]}, {kShapeWarps[2]}};
constexpr int kTuneSteps = 16;  // steps timed per candidate (even: flip and AA phase return)
}  // namespace

void Batch::lookup_shape()
{
    tune_shape_ = false;
    if (tma_ || size() == 0) return;
    for (auto &p : inst_)
        if (p->desc.wall >= LBM_LIBB) return;  // the interpolated-wall step has one shape
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shapes.find(ShapeKey{storage_, collision_, layout_, size(), sms_, fluid_cells()});
    if (it != g_shapes.end()) {
        shape_ = it->second;
        shape_src_ = 2;
    } else {
        tune_shape_ = true;
    }
}

lbm_status Batch::tune_shape(int wx)
{
    const int nc = (int)(sizeof(kShapeCandidates) / sizeof(kShapeCandidates[0]));
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    double best = 0.0;
    StepShape pick = shape_;
    lbm_status st = LBM_OK;
    for (int c = 0; c < nc && st == LBM_OK; ++c) {
        const StepShape &sh = kShapeCandidates[c];
        cudaGraphExec_t exec = nullptr;
        if ((st = graph_for(kTuneSteps, false, sh, wx, &exec)) != LBM_OK) break;
        cudaError_t e = cudaEventRecord(ev[0], stream_);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, stream_);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], stream_);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "timing of a step shape");
            break;
        }
        launches_ += kTuneSteps;
        shape_ms_[c] = ms / kTuneSteps;
        if (c == 0 || ms < best) {
            best = ms;
            pick = sh;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != LBM_OK) return st;
    shape_ = pick;
    shape_src_ = 1;
    tune_shape_ = false;
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes[ShapeKey{storage_, collision_, layout_, size(), sms_, fluid_cells()}] = pick;
    return LBM_OK;
}

lbm_status Batch::step(long long n)
{
    TraceRange trace("lbm.step");
    if (n < 0) return fail(LBM_ERR_ARG, "n_steps < 0");
    if (n == 0 || size() == 0) return LBM_OK;
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    int wx = 0;
    for (auto &p : inst_) wx |= p->desc.wall >= LBM_LIBB;
    const int nc = (int)(sizeof(kShapeCandidates) / sizeof(kShapeCandidates[0]));
    long long left = n;
    if (tune_shape_ && n > (long long)nc * kTuneSteps) {  // the first steps time the shapes
        lbm_status st = tune_shape(wx);
        if (st != LBM_OK) return st;
        left -= (long long)nc * kTuneSteps;
    }
    const long long kChunk = 1000;
    while (left > 0) {
        const long long m = left > 2 * kChunk ? kChunk : left;
        const bool red = (m == left);
        cudaGraphExec_t exec = nullptr;
        lbm_status st = graph_for(m, red, shape_, wx, &exec);
        if (st != LBM_OK) return st;
        CK(cudaGraphLaunch(exec, stream_));
        launches_ += m + (red ? 1 : 0);
        if (layout_ == LBM_LAYOUT_AB) flip_ ^= (int)(m & 1);
        else aa_phase_ ^= (int)(m & 1);
        left -= m;
    }
    for (auto &p : inst_) {
        p->steps += n;
        p->have_sums = false;
        p->have_force = false;
        p->sums_pending = true;
    }
    return LBM_OK;
}

lbm_status Batch::fetch_sums()
{
    const int n = size();
    if (n == 0) return LBM_OK;
    CK(cudaMemcpyAsync(h_sums_, d_sums_, sizeof(double) * kRedSlots * n, cudaMemcpyDeviceToHost, stream_));
    CK(cudaMemcpyAsync(h_status_, d_status_, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, stream_));
    unsigned err = 0;
    if (d_error_) CK(cudaMemcpyAsync(&err, d_error_, sizeof(unsigned), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (err & STATUS_TIMEOUT) return fail(LBM_ERR_TIMEOUT, "a TMA brick copy did not complete within its wait limit");
    if (err & STATUS_BOUNDS)
        return fail(LBM_ERR_BOUNDS, "checked build: a step kernel met an index outside its arrays (access skipped)");
    for (int i = 0; i < n; ++i) {
        Instance &in = *inst_[i];
        for (int d = 0; d < kRedSlots; ++d) in.sums[d] = h_sums_[kRedSlots * i + d];
        in.status = h_status_[i];
        if (in.sums_pending) in.have_sums = in.have_force = true;
        in.sums_pending = false;
    }
    return LBM_OK;
}

lbm_status Batch::moment_sums_now(int i, double *sums)
{
    if (i < 0 || i >= size()) return fail(LBM_ERR_ARG, "instance index out of range");
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    Instance &in = *inst_[i];
    std::vector<int> tb(size());
    {
        int acc = 0;
        for (int j = 0; j < size(); ++j) {
            tb[j] = acc;
            acc += (int)std::max(1ll, (inst_[j]->geo.n_active + block_ / 32 - 1) / (block_ / 32));
        }
    }
    const int nt = (int)std::max(1ll, (in.geo.n_active + block_ / 32 - 1) / (block_ / 32));
    Launch L{d_table_, d_tiles_ + tb[i], nt, block_ / 32, std::max(1, std::min(aux_grid_, (nt + 7) / 8)), 256,
             stream_};
    CK(ops().moments(L, layout_, cur_of(in), aa_phase_, 1, 0, nullptr));
    double *ds = d_sums_ + (size_t)kRedSlots * i;
    double *hs = h_sums_ + (size_t)kRedSlots * i;
    CK(launch_final_reduce(d_table_ + i, d_tile_count_ + i, 1, ds, d_fscratch_ + (size_t)i * kFinalSlices * (RED_F + 3),
                           d_fcount_ + i, stream_));
    launches_ += 2;
    CK(cudaMemcpyAsync(hs, ds, sizeof(double) * 4, cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    for (int d = 0; d < 4; ++d) sums[d] = hs[d];
    return LBM_OK;
}

static cudaError_t ensure_stage(double **buf, long long *cap, long long n)
{
    if (*cap >= n) return cudaSuccess;
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = dev_alloc(buf, sizeof(double) * n);
    if (e == cudaSuccess) *cap = n;
    return e;
}

lbm_status Batch::get_f64(int i, double *host)
{
    if (i < 0 || i >= size() || !host) return fail(LBM_ERR_ARG, "bad instance index or NULL buffer");
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    Instance &in = *inst_[i];
    const long long n = in.geo.ncells;
    CK(ensure_stage(&d_stage_, &stage_cells_, n));
    for (int k = 0; k < Q; ++k) {
        CK(ops().export_dir(d_table_, i, n, layout_, cur_of(in), aa_phase_, k, d_stage_, stream_));
        ++launches_;
        CK(cudaMemcpyAsync(host + (long long)k * n, d_stage_, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
    }
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

lbm_status Batch::set_f64(int i, const double *host)
{
    if (i < 0 || i >= size() || !host) return fail(LBM_ERR_ARG, "bad instance index or NULL buffer");
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    {
        lbm_status st = aa_restart(i);
        if (st != LBM_OK) return st;
    }
    Instance &in = *inst_[i];
    const long long n = in.geo.ncells;
    CK(ensure_stage(&d_stage_, &stage_cells_, n));
    for (int k = 0; k < Q; ++k) {
        CK(cudaMemcpyAsync(d_stage_, host + (long long)k * n, sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
        CK(ops().import_dir(d_table_, i, n, layout_, cur_of(in), k, d_stage_, stream_));
        ++launches_;
    }
    if (in.geo.n_boundary > 0) {
        CK(ops().wall_prepare(d_table_, i, in.geo.n_boundary, in.geo.bcell, layout_, cur_of(in), stream_));
        ++launches_;
    }
    in.have_sums = false;
    in.have_force = false;
    in.sums_pending = false;
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

lbm_status Batch::state_io(int i, void *host, size_t bytes, bool to_host)
{
    if (i < 0 || i >= size() || !host) return fail(LBM_ERR_ARG, "bad instance index or NULL buffer");
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    Instance &in = *inst_[i];
    const long long nf = in.geo.n_fluid;
    const size_t dir_bytes = (size_t)nf * storage_bytes(storage_);
    if (bytes != (size_t)Q * dir_bytes) return fail(LBM_ERR_ARG, "state buffer must hold 19 * n_fluid elements");
    if (!to_host) {
        lbm_status st = aa_restart(i);
        if (st != LBM_OK) return st;
    }
    if (nf > 0) {
        lbm_status cs = ensure_copy_stream();
        if (cs != LBM_OK) return cs;
        if (sstage_bytes_ < dir_bytes) {
            cudaFree(d_sstage_[0]);
            cudaFree(d_sstage_[1]);
            d_sstage_[0] = d_sstage_[1] = nullptr;
            sstage_bytes_ = 0;
            CK(dev_alloc(&d_sstage_[0], dir_bytes));
            CK(dev_alloc(&d_sstage_[1], dir_bytes));
            sstage_bytes_ = dir_bytes;
        }
        const int cur = cur_of(in);
        char *h = static_cast<char *>(host);
        // direction k through staging buffer k % 2: the copy of one direction overlaps the
        // gather or scatter of the other
        for (int k = 0; k < Q; ++k) {
            const int b = k & 1;
            void *st = d_sstage_[b];
            if (to_host) {
                if (k >= 2) CK(cudaStreamWaitEvent(stream_, ev_[2 + b], 0));
                CK(ops().state_dir(d_table_, i, nf, layout_, cur, aa_phase_, k, 1, st, 1, stream_));
                CK(cudaEventRecord(ev_[b], stream_));
                CK(cudaStreamWaitEvent(copy_, ev_[b], 0));
                CK(cudaMemcpyAsync(h + k * dir_bytes, st, dir_bytes, cudaMemcpyDeviceToHost, copy_));
                CK(cudaEventRecord(ev_[2 + b], copy_));
            } else {
                if (k >= 2) CK(cudaStreamWaitEvent(copy_, ev_[2 + b], 0));
                CK(cudaMemcpyAsync(st, h + k * dir_bytes, dir_bytes, cudaMemcpyHostToDevice, copy_));
                CK(cudaEventRecord(ev_[b], copy_));
                CK(cudaStreamWaitEvent(stream_, ev_[b], 0));
                CK(ops().state_dir(d_table_, i, nf, layout_, cur, aa_phase_, k, 1, st, 0, stream_));
                CK(cudaEventRecord(ev_[2 + b], stream_));
            }
            ++launches_;
        }
    }
    if (to_host) {
        if (copy_) CK(cudaStreamSynchronize(copy_));
        return LBM_OK;
    }
    if (in.geo.n_boundary > 0) {
        CK(ops().wall_prepare(d_table_, i, in.geo.n_boundary, in.geo.bcell, layout_, cur_of(in), stream_));
        ++launches_;
    }
    in.have_sums = false;
    in.have_force = false;
    in.sums_pending = false;
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

lbm_status Batch::ensure_copy_stream()
{
    if (!copy_) CK(cudaStreamCreateWithFlags(&copy_, cudaStreamNonBlocking));
    for (cudaEvent_t &e : ev_)
        if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        if (!ev_staged_[b]) CK(cudaEventCreateWithFlags(&ev_staged_[b], cudaEventDisableTiming));
        if (!ev_free_[b]) CK(cudaEventCreateWithFlags(&ev_free_[b], cudaEventDisableTiming));
    }
    return LBM_OK;
}

lbm_status Batch::stage_state(int i, const void *host, size_t bytes)
{
    if (i < 0 || i >= size() || !host) return fail(LBM_ERR_ARG, "bad instance index or NULL buffer");
    const Instance &in = *inst_[i];
    const size_t total = (size_t)Q * (size_t)in.geo.n_fluid * storage_bytes(storage_);
    if (bytes != total) return fail(LBM_ERR_ARG, "state buffer must hold 19 * n_fluid elements");
    if (n_staged_ == 2) return fail(LBM_ERR_STATE, "two states are staged already: apply one first");
    lbm_status cs = ensure_copy_stream();
    if (cs != LBM_OK) return cs;
    if (pstage_bytes_ < total) {
        if (n_staged_ > 0) return fail(LBM_ERR_STATE, "a staged state of another size is pending");
        CK(cudaStreamSynchronize(stream_));  // no scatter still reads the old buffers
        cudaFree(d_pstage_[0]);
        cudaFree(d_pstage_[1]);
        d_pstage_[0] = d_pstage_[1] = nullptr;
        pstage_bytes_ = 0;
        pstage_used_[0] = pstage_used_[1] = false;
        CK(dev_alloc(&d_pstage_[0], total));
        CK(dev_alloc(&d_pstage_[1], total));
        pstage_bytes_ = total;
    }
    const int b = (head_ + n_staged_) & 1;
    if (pstage_used_[b]) CK(cudaStreamWaitEvent(copy_, ev_free_[b], 0));  // its last scatter is done
    if (total > 0) CK(cudaMemcpyAsync(d_pstage_[b], host, total, cudaMemcpyHostToDevice, copy_));
    CK(cudaEventRecord(ev_staged_[b], copy_));
    staged_inst_[b] = i;
    ++n_staged_;
    return LBM_OK;
}

lbm_status Batch::apply_staged_state(int i)
{
    if (i < 0 || i >= size()) return fail(LBM_ERR_ARG, "bad instance index");
    if (n_staged_ == 0) return fail(LBM_ERR_STATE, "no state is staged");
    const int b = head_;
    if (staged_inst_[b] != i) return fail(LBM_ERR_STATE, "the oldest staged state belongs to another instance");
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    Instance &in = *inst_[i];
    const long long nf = in.geo.n_fluid;
    {
        lbm_status st = aa_restart(i);
        if (st != LBM_OK) return st;
    }
    CK(cudaStreamWaitEvent(stream_, ev_staged_[b], 0));
    const int cur = cur_of(in);
    if (nf > 0) {  // all 19 directions in one launch
        CK(ops().state_dir(d_table_, i, nf, layout_, cur, aa_phase_, 0, Q, d_pstage_[b], 0, stream_));
        ++launches_;
    }
    if (in.geo.n_boundary > 0) {
        CK(ops().wall_prepare(d_table_, i, in.geo.n_boundary, in.geo.bcell, layout_, cur, stream_));
        ++launches_;
    }
    CK(cudaEventRecord(ev_free_[b], stream_));
    pstage_used_[b] = true;
    head_ = (head_ + 1) & 1;
    --n_staged_;
    in.have_sums = false;
    in.have_force = false;
    in.sums_pending = false;
    return LBM_OK;
}

lbm_status Batch::get_velocity(int i, double *host)
{
    if (i < 0 || i >= size() || !host) return fail(LBM_ERR_ARG, "bad instance index or NULL buffer");
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    Instance &in = *inst_[i];
    const long long n = in.geo.ncells;
    CK(ensure_stage(&d_stage_, &stage_cells_, n));
    std::vector<int> tb(size());
    int acc = 0;
    for (int j = 0; j < size(); ++j) {
        tb[j] = acc;
        acc += (int)std::max(1ll, (inst_[j]->geo.n_active + block_ / 32 - 1) / (block_ / 32));
    }
    const int nt = (int)std::max(1ll, (in.geo.n_active + block_ / 32 - 1) / (block_ / 32));
    Launch L{d_table_, d_tiles_ + tb[i], nt, block_ / 32, std::max(1, std::min(aux_grid_, (nt + 7) / 8)), 256,
             stream_};
    for (int c = 0; c < 3; ++c) {
        // all-solid segments are not in the work list: clear the whole field first
        CK(cudaMemsetAsync(d_stage_, 0, sizeof(double) * n, stream_));
        CK(ops().moments(L, layout_, cur_of(in), aa_phase_, 0, c, d_stage_));
        ++launches_;
        CK(cudaMemcpyAsync(host + (long long)c * n, d_stage_, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
    }
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

lbm_status Batch::get_flags(int i, uint8_t *host)
{
    if (i < 0 || i >= size() || !host) return fail(LBM_ERR_ARG, "bad instance index or NULL buffer");
    Instance &in = *inst_[i];
    CK(cudaMemcpyAsync(host, in.geo.solid, in.geo.ncells, cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

lbm_status Batch::get_q(int i, double *host)
{
    if (i < 0 || i >= size() || !host) return fail(LBM_ERR_ARG, "bad instance index or NULL buffer");
    Instance &in = *inst_[i];
    const long long n = in.geo.ncells;
    CK(ensure_stage(&d_stage_, &stage_cells_, n));
    for (int k = 0; k < Q; ++k) {
        CK(export_wall_distances(in.geo, k, d_stage_, stream_));
        launches_ += 2;
        CK(cudaMemcpyAsync(host + (long long)k * n, d_stage_, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_));
    }
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

lbm_status Batch::sync()
{
    CK(cudaStreamSynchronize(stream_));
    return LBM_OK;
}

void Batch::fill_info(int i, lbm_info *out) const
{
    std::memset(out, 0, sizeof(*out));
    for (int j = 0; j < size(); ++j) {
        if (i >= 0 && j != i) continue;
        const Instance &in = *inst_[j];
        out->n_cells += in.geo.ncells;
        out->n_fluid += in.geo.n_fluid;
        out->n_boundary += in.geo.n_boundary;
        out->n_links += in.geo.n_links;
        out->n_links_cli += in.geo.n_links_cli;
        out->bytes_populations += (int64_t)in.bytes_pop;
        out->bytes_geometry += (int64_t)in.geo.bytes;
        out->steps = in.steps;
        out->dev_scale_log2 = in.dev_scale_log2;
        out->wall = in.desc.wall;
    }
    out->kernel_launches = launches_;
    out->block_cells = block_cells();
    out->storage = storage_;
    out->layout = layout_;
    out->collision = collision_;
    out->autotune = tune_src_;
    out->tune_ms_tiles = tune_ms_[0];
    out->tune_ms_bricks = tune_ms_[1];
    out->step_warps = tma_ ? 0 : shape_.warps;
    out->shape_source = shape_src_;
    for (int c = 0; c < kShapeWarpsN; ++c) out->shape_ms[c] = shape_ms_[c];
}

// ------------------------------------------------------------------------------------
// Checkpoint: native-format state of one instance.
// ------------------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int32_t version, nx, ny, nz, storage, layout, collision, wall, aa_phase, dev_scale_log2;
    int64_t steps, n_links, elem_bytes, stride;
};

lbm_status Batch::save(int i, const char *path)
{
    if (i < 0 || i >= size() || !path) return fail(LBM_ERR_ARG, "bad instance index or NULL path");
    Instance &in = *inst_[i];
    CK(cudaStreamSynchronize(stream_));
    const size_t es = storage_bytes(storage_);
    const size_t pop = (size_t)Q * in.ks * es;
    std::vector<char> buf(pop);
    const void *src = (layout_ == LBM_LAYOUT_AB) ? (cur_of(in) ? in.f1 : in.f0) : in.f0;
    CK(cudaMemcpy(buf.data(), src, pop, cudaMemcpyDeviceToHost));
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "LBMGB300", 8);
    h.version = 3;  // 3: the solid slots of either layout hold the wall terms of the next step
    h.nx = in.desc.nx;
    h.ny = in.desc.ny;
    h.nz = in.desc.nz;
    h.storage = storage_;
    h.layout = layout_;
    h.collision = collision_;
    h.wall = in.desc.wall;
    h.aa_phase = aa_phase_;
    h.dev_scale_log2 = in.dev_scale_log2;
    h.steps = in.steps;
    h.n_links = 0;  // no per-link buffer
    h.elem_bytes = (int64_t)es;
    h.stride = in.ks;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(LBM_ERR_IO, std::string("write failed: ") + path);
    return LBM_OK;
}

lbm_status Batch::load(int i, const char *path)
{
    if (i < 0 || i >= size() || !path) return fail(LBM_ERR_ARG, "bad instance index or NULL path");
    if (dirty_) {
        lbm_status st = rebuild();
        if (st != LBM_OK) return st;
    }
    Instance &in = *inst_[i];
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    CkptHeader h;
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "LBMGB300", 8) != 0 || h.version != 3) {
        std::fclose(f);
        return fail(LBM_ERR_IO, "not a checkpoint of this library");
    }
    const size_t es = storage_bytes(storage_);
    if (h.nx != in.desc.nx || h.ny != in.desc.ny || h.nz != in.desc.nz || h.storage != storage_ ||
        h.layout != layout_ || h.collision != collision_ || h.wall != in.desc.wall || h.elem_bytes != (int64_t)es ||
        h.dev_scale_log2 != in.dev_scale_log2 || h.n_links != 0 ||
        h.stride != in.ks) {
        std::fclose(f);
        return fail(LBM_ERR_ARG, "checkpoint does not match this context's descriptor");
    }
    const size_t pop = (size_t)Q * in.ks * es;
    std::vector<char> buf(pop);
    bool ok = std::fread(buf.data(), 1, pop, f) == pop;
    std::fclose(f);
    if (!ok) return fail(LBM_ERR_IO, "checkpoint truncated");
    CK(cudaStreamSynchronize(stream_));
    if (layout_ == LBM_LAYOUT_AA && size() > 1 && h.aa_phase != aa_phase_)
        return fail(LBM_ERR_STATE, "the checkpoint's AA arrangement differs from the batch's");
    if (layout_ == LBM_LAYOUT_AA) aa_phase_ = h.aa_phase;
    void *dst = (layout_ == LBM_LAYOUT_AB) ? (cur_of(in) ? in.f1 : in.f0) : in.f0;
    CK(cudaMemcpy(dst, buf.data(), pop, cudaMemcpyHostToDevice));
    in.steps = h.steps;
    in.have_sums = false;
    in.have_force = false;
    in.sums_pending = false;
    return LBM_OK;
}

}  // namespace lbm
