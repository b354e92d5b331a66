// capi.cu -- extern "C" entry points for contexts and batches, and the host arithmetic
// of the observables (Eqs. Darcy, Forchheimer, frictionFactor) and the convergence test.
#include <cmath>
#include <cstring>
#include <limits>
#include <new>

#include "batch.h"

using namespace lbm;

namespace lbm {
const char *last_error_cstr();
}

struct lbm_ctx {
    Batch b;
};
struct lbm_batch {
    Batch b;
};

namespace lbm {

// Observables in lattice units with rho = rho0: mu = rho0 (tau - 1/2)/3, nu = (tau - 1/2)/3,
// delta_p = delta_rho / 3 (p = rho c_s^2), gradP = delta_p / L_x, K = mu U / gradP
// (Eq. Darcy), Re_p = U d_p / nu, and with K_D: beta = (gradP - mu U / K_D)/(rho U^2)
// (Eq. Forchheimer), C_F = beta sqrt(K_D), F_K = gradP sqrt(K_D)/(rho U^2),
// Re_K = rho U sqrt(K_D)/mu (Eq. frictionFactor).  Drag: F_D = the momentum handed to the
// solid in the last reducing step, C_D = F_x / (6 pi mu U r) with r the sum of the sphere
// radii (Eq. AnalyticForce) and C_D_A = F_x / (rho0 A U^2) with A the sum of pi r^2 (Sec. 4).
void compute_obs(const Instance &in, double K_D, lbm_obs *o)
{
    const lbm_desc &d = in.desc;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    const double ncell = (double)in.geo.ncells, nf = (double)in.geo.n_fluid;
    std::memset(o, 0, sizeof(*o));
    o->U_sup = in.sums[1] / ncell;
    o->U_int = nf > 0 ? in.sums[1] / nf : nan;
    o->mass = nf * d.rho0 + in.sums[0];
    o->porosity = nf / ncell;
    const double mu = d.rho0 * (d.tau - 0.5) / 3.0, nu = (d.tau - 0.5) / 3.0;
    const double gradP = (d.delta_rho / 3.0) / d.nx;
    const double U = o->U_sup;
    o->K = gradP != 0 ? mu * U / gradP : nan;
    o->K_app = o->K;
    o->Re_p = in.d_p > 0 ? U * in.d_p / nu : nan;
    if (K_D > 0) {
        const double sk = std::sqrt(K_D);
        o->beta = (gradP - mu * U / K_D) / (d.rho0 * U * U);
        o->C_F = o->beta * sk;
        o->F_K = gradP * sk / (d.rho0 * U * U);
        o->Re_K = d.rho0 * U * sk / mu;
    } else {
        o->beta = o->C_F = o->F_K = o->Re_K = nan;
    }
    o->u_max = 0.0;
    if (in.have_force) {
        o->F_x = in.sums[RED_F + 0];
        o->F_y = in.sums[RED_F + 1];
        o->F_z = in.sums[RED_F + 2];
    } else {
        o->F_x = o->F_y = o->F_z = nan;
    }
    o->C_D = in.r_sum > 0 ? o->F_x / (6.0 * M_PI * mu * U * in.r_sum) : nan;
    o->C_D_A = in.area_sum > 0 ? o->F_x / (d.rho0 * in.area_sum * U * U) : nan;
    o->K_star = K_D > 0 ? o->K_app / K_D : nan;
    o->steps = in.steps;
    o->n_fluid = in.geo.n_fluid;
}

}  // namespace lbm

namespace {

lbm_status create_batch(Batch &b, const lbm_desc *descs, int n, cudaStream_t s)
{
    for (int i = 0; i < n; ++i) {
        lbm_status v = validate_desc(descs[i]);
        if (v != LBM_OK) return v;
        if (descs[i].storage != descs[0].storage || descs[i].collision != descs[0].collision ||
            descs[i].layout != descs[0].layout)
            return fail(LBM_ERR_ARG, "instances of a batch must share storage, collision and layout");
    }
    lbm_status st = b.init(s, descs[0].storage, descs[0].collision, descs[0].layout);
    if (st != LBM_OK) return st;
    int block = 0;
    bool tune = false;
    for (int i = 0; i < n; ++i) {
        std::unique_ptr<Instance> in;
        st = Batch::make_instance(descs[i], s, &in);
        if (st != LBM_OK) return st;
        if (descs[i].block_cells == LBM_BLOCK_AUTO) tune = true;
        else if (descs[i].block_cells) block = descs[i].block_cells;
        st = b.add(std::move(in));
        if (st != LBM_OK) return st;
    }
    if (tune && !block) {
        st = autotune_block(b, descs[0], s);
        if (st != LBM_OK) return st;
    } else if (block) {
        st = b.set_block(block);
        if (st != LBM_OK) return st;
    }
    return b.prepare();  // tables and the step kernel chosen now: errors surface at create
}

}  // namespace

extern "C" {

const char *lbm_last_error(void) { return last_error_cstr(); }
const char *lbm_version(void) { return "lbm_gb300 0.1 (sm_103a)"; }

unsigned lbm_build_flags(void) { return kChecked ? LBM_BUILD_CHECKED : 0u; }

lbm_status lbm_debug_pack_work_items(const uint32_t *cells, int64_t n_cells, uint32_t *out, int64_t out_cap,
                                     int64_t *n_items)
{
    if (!n_items || n_cells < 0 || (n_cells > 0 && !cells)) return fail(LBM_ERR_ARG, "NULL or negative argument");
    std::vector<uint32_t> c(cells, cells + n_cells);
    for (int64_t j = 1; j < n_cells; ++j)
        if (c[(size_t)j] <= c[(size_t)j - 1]) return fail(LBM_ERR_ARG, "cells must be strictly increasing");
    for (int64_t j = 0; j < n_cells; ++j)
        if (c[(size_t)j] >= (1u << 28)) return fail(LBM_ERR_ARG, "cell index beyond 2^28");
    long long ni = 0;
    const std::vector<uint32_t> items = pack_work_items(c, &ni);
    *n_items = (int64_t)ni;
    if (!out || out_cap < (int64_t)items.size()) return fail(LBM_ERR_ARG, "out holds fewer than 32 n_items entries");
    std::copy(items.begin(), items.end(), out);
    return LBM_OK;
}

lbm_status lbm_debug_corrupt_worklist(lbm_ctx *ctx)
{
    if (!ctx || ctx->b.size() != 1) return fail(LBM_ERR_ARG, "ctx is NULL");
    if (!kChecked) return fail(LBM_ERR_STATE, "only the checked build (LBM_CHECKED) tests its indices");
    const Instance &in = ctx->b.at(0);
    if (!in.geo.flane || in.geo.n_fwarps < 1) return fail(LBM_ERR_STATE, "no fluid cells");
    const uint32_t bad = (uint32_t)in.geo.ncells;  // one past the last cell
    // the cell of the step kernels' first work-list entry (flane[0].x)
    cudaError_t e = cudaMemcpyAsync(in.geo.flane, &bad, sizeof(bad), cudaMemcpyHostToDevice, ctx->b.stream());
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->b.stream());
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "cudaMemcpyAsync");
}

lbm_status lbm_create(const lbm_desc *desc, void *cuda_stream, lbm_ctx **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(LBM_ERR_ARG, "desc is NULL");
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ERR_NO_MEMORY, "host allocation failed");
    lbm_status st = create_batch(c->b, desc, 1, (cudaStream_t)cuda_stream);
    if (st != LBM_OK) {
        delete c;
        return st;
    }
    *out = c;
    set_error("");
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx) { delete ctx; }

lbm_status lbm_init_equilibrium(lbm_ctx *ctx)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.init_equilibrium(-1);
}

lbm_status lbm_step(lbm_ctx *ctx, int64_t n_steps)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.step(n_steps);
}

lbm_status lbm_observables(lbm_ctx *ctx, double K_darcy, lbm_obs *out)
{
    if (!ctx || !out) return fail(LBM_ERR_ARG, "NULL argument");
    Instance &in = ctx->b.at(0);
    if (!in.have_sums) {
        lbm_status st;
        if (in.sums_pending) {
            st = ctx->b.fetch_sums();
        } else {  // no step since the state was set: reduce the stored state
            st = ctx->b.moment_sums_now(0, in.sums);
            in.status = 0;
            in.have_sums = (st == LBM_OK);
            in.have_force = false;
        }
        if (st != LBM_OK) return st;
    }
    compute_obs(in, K_darcy, out);
    if (in.status & STATUS_DIVERGED) return fail(LBM_ERR_DIVERGED, "the last reduction saw a diverged cell");
    return LBM_OK;
}

lbm_status lbm_run_to_convergence(lbm_ctx *ctx, double tol, int64_t check_interval, int64_t max_steps,
                                  int64_t *steps_done)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    if (!(tol > 0) || check_interval < 1 || max_steps < 0) return fail(LBM_ERR_ARG, "bad tol/check_interval/max_steps");
    Instance &in = ctx->b.at(0);
    int64_t done = 0;
    double U_old = std::numeric_limits<double>::quiet_NaN();
    lbm_status result = LBM_ERR_NOT_CONVERGED;
    while (done < max_steps) {
        const int64_t m = std::min<int64_t>(check_interval, max_steps - done);
        lbm_status st = ctx->b.step(m);
        if (st != LBM_OK) return st;
        done += m;
        st = ctx->b.fetch_sums();
        if (st != LBM_OK) return st;
        if (in.status & STATUS_DIVERGED) {
            result = fail(LBM_ERR_DIVERGED, "diverged (non-finite moments or |u| > 1)");
            break;
        }
        const double U = in.sums[1] / (double)in.geo.ncells;
        if (!std::isnan(U_old) && std::fabs(U - U_old) < tol * std::fabs(U)) {
            result = LBM_OK;
            break;
        }
        U_old = U;
    }
    if (steps_done) *steps_done = done;
    if (result == LBM_ERR_NOT_CONVERGED) set_error("max_steps reached before convergence");
    return result;
}

lbm_status lbm_average(lbm_ctx *ctx, int64_t n_samples, int64_t sample_interval, double K_darcy, lbm_obs *out)
{
    if (!ctx || !out) return fail(LBM_ERR_ARG, "NULL argument");
    if (n_samples < 1 || sample_interval < 1) return fail(LBM_ERR_ARG, "n_samples and sample_interval must be >= 1");
    Instance &in = ctx->b.at(0);
    double acc[kRedSlots] = {};
    int64_t done = 0;
    lbm_status result = LBM_OK;
    for (int64_t i = 0; i < n_samples; ++i) {
        lbm_status st = ctx->b.step(sample_interval);
        if (st != LBM_OK) return st;
        st = ctx->b.fetch_sums();
        if (st != LBM_OK) return st;
        for (int d = 0; d < kRedSlots; ++d) acc[d] += in.sums[d];
        ++done;
        if (in.status & STATUS_DIVERGED) {
            result = fail(LBM_ERR_DIVERGED, "a sample saw a diverged cell");
            break;
        }
    }
    double keep[kRedSlots];
    for (int d = 0; d < kRedSlots; ++d) {
        keep[d] = in.sums[d];
        in.sums[d] = acc[d] / (double)done;
    }
    compute_obs(in, K_darcy, out);
    for (int d = 0; d < kRedSlots; ++d) in.sums[d] = keep[d];
    return result;
}

lbm_status lbm_run_developed(lbm_ctx *ctx, const lbm_develop_opts *o, double K_darcy, lbm_develop_result *out)
{
    TraceRange trace("lbm.run_developed");
    if (!ctx || !o || !out) return fail(LBM_ERR_ARG, "NULL argument");
    if (o->samples_per_ft < 1 || !(o->min_spinup_ft >= 0) || !(o->max_spinup_ft >= o->min_spinup_ft) ||
        !(o->average_ft > 0) || !(o->drag_tol > 0) || o->max_steps < 1)
        return fail(LBM_ERR_ARG, "bad developed-average options");
    std::memset(out, 0, sizeof(*out));
    Instance &in = ctx->b.at(0);
    const double nx = (double)in.desc.nx, ncell = (double)in.geo.ncells;
    int64_t total = 0;
    // one sample: advance n steps, reduce; the sums describe the last of them
    auto sample = [&](int64_t n) -> lbm_status {
        lbm_status st = ctx->b.step(n);
        if (st != LBM_OK) return st;
        st = ctx->b.fetch_sums();
        if (st != LBM_OK) return st;
        total += n;
        if (in.status & STATUS_DIVERGED) return fail(LBM_ERR_DIVERGED, "diverged (non-finite moments or |u| > 1)");
        return LBM_OK;
    };
    auto ft_steps = [&](double &T) -> lbm_status {  // T = nx / U_sup of the latest sample
        const double U = in.sums[RED_U] / ncell;
        if (!(std::fabs(U) > 0) || !std::isfinite(U)) return fail(LBM_ERR_ARG, "no flow: U_sup is 0");
        T = std::max(1.0, nx / std::fabs(U));
        return LBM_OK;
    };
    // spin-up: the first sample (nx steps) gives the first flow-through time
    lbm_status st = sample(std::max<int64_t>(1, (int64_t)nx));
    if (st != LBM_OK) return st;
    double T = 0.0;
    if ((st = ft_steps(T)) != LBM_OK) return st;
    double spin_ft = 1.0 * (double)total / T, prev = std::numeric_limits<double>::quiet_NaN(), change = 1.0;
    int64_t spin_steps = total;
    for (;;) {
        const int64_t sub = std::max<int64_t>(1, (int64_t)std::llround(T / o->samples_per_ft));
        if (total + sub * o->samples_per_ft > o->max_steps) {
            out->spinup_steps = spin_steps;
            out->spinup_ft = spin_ft;
            out->drag_change = change;
            return fail(LBM_ERR_NOT_CONVERGED, "max_steps reached during the spin-up");
        }
        double wsum = 0.0;
        for (int i = 0; i < o->samples_per_ft; ++i) {
            if ((st = sample(sub)) != LBM_OK) return st;
            wsum += in.sums[RED_F];
        }
        spin_steps += sub * o->samples_per_ft;
        spin_ft += (double)(sub * o->samples_per_ft) / T;
        const double W = wsum / o->samples_per_ft;
        change = std::isnan(prev) ? 1.0 : std::fabs(W - prev) / std::max(std::fabs(W), 1e-300);
        prev = W;
        if ((st = ft_steps(T)) != LBM_OK) return st;
        if (spin_ft >= o->min_spinup_ft && change < o->drag_tol) {
            out->developed = 1;
            break;
        }
        if (spin_ft >= o->max_spinup_ft) break;
    }
    out->spinup_steps = spin_steps;
    out->spinup_ft = spin_ft;
    out->drag_change = change;
    // averaging over average_ft flow-through times
    const int64_t sub = std::max<int64_t>(1, (int64_t)std::llround(T / o->samples_per_ft));
    const int64_t n_samples = std::max<int64_t>(1, (int64_t)std::llround(o->average_ft * o->samples_per_ft));
    double acc[kRedSlots] = {};
    int64_t done = 0;
    lbm_status result = LBM_OK;
    for (int64_t i = 0; i < n_samples; ++i) {
        if (total + sub > o->max_steps) {
            result = fail(LBM_ERR_NOT_CONVERGED, "max_steps reached during the averaging");
            break;
        }
        if ((st = sample(sub)) != LBM_OK) return st;
        for (int d = 0; d < kRedSlots; ++d) acc[d] += in.sums[d];
        ++done;
    }
    if (done == 0) return result == LBM_OK ? fail(LBM_ERR_NOT_CONVERGED, "no averaging sample") : result;
    double keep[kRedSlots];
    for (int d = 0; d < kRedSlots; ++d) {
        keep[d] = in.sums[d];
        in.sums[d] = acc[d] / (double)done;
    }
    const bool hf = in.have_force;
    in.have_force = true;
    compute_obs(in, K_darcy, &out->avg);
    in.have_force = hf;
    for (int d = 0; d < kRedSlots; ++d) in.sums[d] = keep[d];
    out->average_steps = done * sub;
    out->flow_through_steps = out->avg.U_sup != 0 ? nx / std::fabs(out->avg.U_sup) : 0.0;
    out->average_ft = out->flow_through_steps > 0 ? (double)out->average_steps / out->flow_through_steps : 0.0;
    return result;
}

lbm_status lbm_moment_sums(lbm_ctx *ctx, double *sums)
{
    if (!ctx || !sums) return fail(LBM_ERR_ARG, "NULL argument");
    return ctx->b.moment_sums_now(0, sums);
}

lbm_status lbm_get_populations_f64(lbm_ctx *ctx, double *host_out)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.get_f64(0, host_out);
}

lbm_status lbm_set_populations_f64(lbm_ctx *ctx, const double *host_in)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.set_f64(0, host_in);
}

lbm_status lbm_get_state(lbm_ctx *ctx, void *host_out, size_t bytes)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.state_io(0, host_out, bytes, true);
}

lbm_status lbm_set_state(lbm_ctx *ctx, const void *host_in, size_t bytes)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.state_io(0, const_cast<void *>(host_in), bytes, false);
}

lbm_status lbm_stage_state(lbm_ctx *ctx, const void *host_in, size_t bytes)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.stage_state(0, host_in, bytes);
}

lbm_status lbm_apply_staged_state(lbm_ctx *ctx)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.apply_staged_state(0);
}

lbm_status lbm_get_velocity_f64(lbm_ctx *ctx, double *host_out)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.get_velocity(0, host_out);
}

lbm_status lbm_get_flags(lbm_ctx *ctx, uint8_t *host_out)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.get_flags(0, host_out);
}

lbm_status lbm_get_wall_distances(lbm_ctx *ctx, double *host_out)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.get_q(0, host_out);
}

lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *out)
{
    if (!ctx || !out) return fail(LBM_ERR_ARG, "NULL argument");
    lbm_status st = ctx->b.prepare();
    if (st != LBM_OK) return st;
    ctx->b.fill_info(0, out);
    return LBM_OK;
}

lbm_status lbm_synchronize(lbm_ctx *ctx)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.sync();
}

lbm_status lbm_save(lbm_ctx *ctx, const char *path)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.save(0, path);
}

lbm_status lbm_load(lbm_ctx *ctx, const char *path)
{
    if (!ctx) return fail(LBM_ERR_ARG, "ctx is NULL");
    return ctx->b.load(0, path);
}

// Solve gradP = mu U / K_D + (C_F / sqrt(K_D)) rho U^2 for the U of the target Re_p
// (U = Re_p nu / d_p) and return delta_rho = 3 L gradP.
double lbm_delta_rho_for_re_p(double re_p, double tau, double d_p, int32_t lx, double K_D, double C_F, double rho0)
{
    if (rho0 <= 0) rho0 = 1.0;
    const double nu = (tau - 0.5) / 3.0, mu = rho0 * nu;
    const double U = re_p * nu / d_p;
    const double gradP = mu * U / K_D + (K_D > 0 ? C_F / std::sqrt(K_D) : 0.0) * rho0 * U * U;
    return 3.0 * lx * gradP;
}

// ---- batches ---------------------------------------------------------------------------
lbm_status lbm_batch_create(const lbm_desc *descs, int32_t n, void *cuda_stream, lbm_batch **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || n < 1) return fail(LBM_ERR_ARG, "need at least one descriptor");
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return fail(LBM_ERR_NO_MEMORY, "host allocation failed");
    lbm_status st = create_batch(b->b, descs, n, (cudaStream_t)cuda_stream);
    if (st != LBM_OK) {
        delete b;
        return st;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) { delete b; }

lbm_status lbm_batch_init_equilibrium(lbm_batch *b)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    return b->b.init_equilibrium(-1);
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t n_steps)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    return b->b.step(n_steps);
}

lbm_status lbm_batch_observables(lbm_batch *b, int32_t i, double K_darcy, lbm_obs *out)
{
    if (!b || !out) return fail(LBM_ERR_ARG, "NULL argument");
    if (i < 0 || i >= b->b.size()) return fail(LBM_ERR_ARG, "instance index out of range");
    Instance &in = b->b.at(i);
    if (!in.have_sums) {
        lbm_status st;
        if (in.sums_pending) {
            st = b->b.fetch_sums();
        } else {
            st = b->b.moment_sums_now(i, in.sums);
            in.status = 0;
            in.have_sums = (st == LBM_OK);
            in.have_force = false;
        }
        if (st != LBM_OK) return st;
    }
    compute_obs(in, K_darcy, out);
    if (in.status & STATUS_DIVERGED) return fail(LBM_ERR_DIVERGED, "the last reduction saw a diverged cell");
    return LBM_OK;
}

lbm_status lbm_batch_get_populations_f64(lbm_batch *b, int32_t i, double *host_out)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    return b->b.get_f64(i, host_out);
}

lbm_status lbm_batch_set_populations_f64(lbm_batch *b, int32_t i, const double *host_in)
{
    if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
    return b->b.set_f64(i, host_in);
}

lbm_status lbm_batch_get_info(lbm_batch *b, lbm_info *out)
{
    if (!b || !out) return fail(LBM_ERR_ARG, "NULL argument");
    lbm_status st = b->b.prepare();
    if (st != LBM_OK) return st;
    b->b.fill_info(-1, out);
    return LBM_OK;
}

}  // extern "C"
