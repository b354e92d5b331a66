// models.cu -- host-side fits of the macroscopic flow laws of Sec. 1 to simulated data.
//
// Barree-Conway apparent permeability (Eq. AppPer), normalised by the Darcy permeability
// (Eq. normalizedPermeability):
//     K*(Re) = m + (1 - m) / (1 + (a Re)^F)^E,
// m = K_min / K_D, a = l_T / d_p (a Re_p is the transition Reynolds number Re_T), E, F the
// exponents.  Least squares by Levenberg-Marquardt over theta = (logit m, ln a, ln E, ln F),
// which keeps m in (0, 1) and a, E, F positive, with the analytic Jacobian; fixed iteration
// order, so the fit is deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "batch.h"

namespace lbm {
namespace {

struct BCModel {
    // value and gradient (d/dtheta) of K* at re for theta = (logit m, ln a, ln E, ln F)
    static double eval(double re, const double *th, double *grad)
    {
        const double m = 1.0 / (1.0 + std::exp(-th[0])), la = th[1], E = std::exp(th[2]), F = std::exp(th[3]);
        const double lar = la + std::log(re);     // ln(a re)
        const double z = std::exp(F * lar);       // (a re)^F
        const double g = std::exp(-E * std::log1p(z));  // (1 + z)^-E
        if (grad) {
            const double gD = g / (1.0 + z);  // (1 + z)^(-E-1)
            grad[0] = (1.0 - g) * m * (1.0 - m);
            grad[1] = (1.0 - m) * (-E * F * z * gD);
            grad[2] = (1.0 - m) * (-E * std::log1p(z) * g);
            grad[3] = (1.0 - m) * (-E * F * z * lar * gD);
        }
        return m + (1.0 - m) * g;
    }
};

double cost(const std::vector<double> &re, const std::vector<double> &k, const double *th)
{
    double c = 0.0;
    for (size_t i = 0; i < re.size(); ++i) {
        const double r = BCModel::eval(re[i], th, nullptr) - k[i];
        c += r * r;
    }
    return c;
}

// Solve the 4x4 system A x = b (Gaussian elimination with partial pivoting); false if singular.
bool solve4(double A[4][4], double b[4], double x[4])
{
    int p[4] = {0, 1, 2, 3};
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (std::fabs(A[p[r]][c]) > std::fabs(A[p[piv]][c])) piv = r;
        std::swap(p[c], p[piv]);
        const double d = A[p[c]][c];
        if (!(std::fabs(d) > 1e-300)) return false;
        for (int r = c + 1; r < 4; ++r) {
            const double f = A[p[r]][c] / d;
            for (int j = c; j < 4; ++j) A[p[r]][j] -= f * A[p[c]][j];
            b[p[r]] -= f * b[p[c]];
        }
    }
    for (int c = 3; c >= 0; --c) {
        double s = b[p[c]];
        for (int j = c + 1; j < 4; ++j) s -= A[p[c]][j] * x[j];
        x[c] = s / A[p[c]][c];
    }
    return true;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_fit_barree_conway(const double *re, const double *kstar, int32_t n, const double *init,
                                            double *params_out, double *rms_out)
{
    if (!re || !kstar || !params_out) return fail(LBM_ERR_ARG, "NULL argument");
    if (n < 4) return fail(LBM_ERR_ARG, "the Barree-Conway model has 4 parameters: n >= 4 points needed");
    std::vector<double> R(re, re + n), K(kstar, kstar + n);
    for (int i = 0; i < n; ++i)
        if (!(R[i] > 0) || !std::isfinite(R[i]) || !std::isfinite(K[i]))
            return fail(LBM_ERR_ARG, "points need Re > 0 and finite K*");
    double th[4];
    if (init) {
        if (!(init[0] > 0 && init[0] < 1) || !(init[1] > 0) || !(init[2] > 0) || !(init[3] > 0))
            return fail(LBM_ERR_ARG, "init needs 0 < m < 1 and a, E, F > 0");
        th[0] = std::log(init[0] / (1.0 - init[0]));
        th[1] = std::log(init[1]);
        th[2] = std::log(init[2]);
        th[3] = std::log(init[3]);
    } else {  // m below the smallest K*, transition at the median Re, E = F = 1
        std::vector<double> s(R);
        std::sort(s.begin(), s.end());
        const double m0 = std::min(0.9, std::max(0.01, 0.9 * *std::min_element(K.begin(), K.end())));
        th[0] = std::log(m0 / (1.0 - m0));
        th[1] = -std::log(s[n / 2]);
        th[2] = 0.0;
        th[3] = 0.0;
    }
    double c = cost(R, K, th), lambda = 1e-3;
    bool converged = false;
    for (int it = 0; it < 1000 && !converged; ++it) {
        double JtJ[4][4] = {}, Jtr[4] = {};
        for (int i = 0; i < n; ++i) {
            double gr[4];
            const double r = BCModel::eval(R[i], th, gr) - K[i];
            for (int a = 0; a < 4; ++a) {
                Jtr[a] += gr[a] * r;
                for (int b = 0; b < 4; ++b) JtJ[a][b] += gr[a] * gr[b];
            }
        }
        bool stepped = false;
        for (int tries = 0; tries < 30 && !stepped; ++tries) {
            double A[4][4], b[4], d[4];
            for (int a = 0; a < 4; ++a) {
                for (int bb = 0; bb < 4; ++bb) A[a][bb] = JtJ[a][bb];
                A[a][a] += lambda * std::max(JtJ[a][a], 1e-30);
                b[a] = -Jtr[a];
            }
            if (!solve4(A, b, d)) {
                lambda *= 10.0;
                continue;
            }
            double tn[4];
            for (int a = 0; a < 4; ++a) tn[a] = th[a] + d[a];
            const double cn = cost(R, K, tn);
            if (std::isfinite(cn) && cn < c) {
                const double rel = (c - cn) / std::max(c, 1e-300);
                for (int a = 0; a < 4; ++a) th[a] = tn[a];
                c = cn;
                lambda = std::max(lambda / 3.0, 1e-15);
                stepped = true;
                converged = rel < 1e-15;
            } else {
                lambda *= 4.0;
            }
        }
        if (!stepped) break;
    }
    params_out[0] = 1.0 / (1.0 + std::exp(-th[0]));
    params_out[1] = std::exp(th[1]);
    params_out[2] = std::exp(th[2]);
    params_out[3] = std::exp(th[3]);
    if (rms_out) *rms_out = std::sqrt(c / n);
    return LBM_OK;
}
