// Host-only planning of (M, L) for Algorithm 2 (Section 2.3).
#include <cmath>
#include <limits>

#include "../../include/xyz.h"

namespace {

// 1 - (1 - beta)^L without cancellation for tiny beta.
double hit_prob(double beta, double L)
{
    if (beta >= 1.0)
        return L > 0 ? 1.0 : 0.0;
    return -std::expm1(L * std::log1p(-beta));
}

}  // namespace

extern "C" {

// eq. eta: a pair of strength gamma lands in one run's equal pairs with
// probability gamma^M, so L independent runs find it with 1-(1-gamma^M)^L.
double xyz_eta(double gamma, int32_t M, int64_t L)
{
    if (!(gamma >= 0.0 && gamma <= 1.0) || M < 0 || L < 0)
        return std::numeric_limits<double>::quiet_NaN();
    return hit_prob(std::pow(gamma, (double)M), (double)L);
}

// eq. L_choice: least L with 1 - (1 - beta)^L >= eta.
int64_t xyz_runs_for_recall(double beta, double eta)
{
    if (!(beta > 0.0) || !(eta > 0.0 && eta < 1.0))
        return -1;
    if (beta >= 1.0)
        return 1;
    double Lr = std::log1p(-eta) / std::log1p(-beta);
    if (!(Lr < 9.0e18))
        return -1;
    int64_t L = (int64_t)std::ceil(Lr);
    if (L < 1)
        L = 1;
    while (hit_prob(beta, (double)L) < eta)
        ++L;
    while (L > 1 && hit_prob(beta, (double)(L - 1)) >= eta)
        --L;
    return L;
}

// eq. bestM with the plug-in estimate of sum_{j != k} gamma_jk^M from
// sampled pairs (Section 2.3, last paragraph).
int xyz_best_M(int64_t n, int64_t p, double gamma, const int32_t *agree, int64_t count,
               int32_t max_M, int32_t *M_out, double *cost_out)
{
    if (n < 1 || p < 2 || !(gamma > 0.0 && gamma < 1.0) || !agree || count < 1 || max_M < 1 ||
        max_M > XYZ_MAX_M || !M_out)
        return XYZ_EINVAL;
    const double pd = (double)p, nd = (double)n;
    double best = std::numeric_limits<double>::infinity();
    int32_t bestM = 1;
    for (int32_t M = 1; M <= max_M; ++M) {
        double mean = 0.0;
        for (int64_t t = 0; t < count; ++t)
            mean += std::pow((double)agree[t] / nd, (double)M);
        mean /= (double)count;
        const double S = pd * (pd - 1.0) * mean;
        const double retain = std::pow(gamma, (double)M);
        const double denom = -std::log1p(-retain);
        if (!(denom > 0.0))
            continue;
        const double cost = (M * pd + pd * std::log(pd) + nd * S) / denom;
        if (cost < best) {
            best = cost;
            bestM = M;
        }
    }
    *M_out = bestM;
    if (cost_out)
        *cost_out = best;
    return XYZ_OK;
}

// gamma_0 = p^(-1/M) near gamma0  <=>  M near log p / log(1/gamma0).
int32_t xyz_M_for_gamma0(int64_t p, double gamma0)
{
    if (p < 2 || !(gamma0 > 0.0 && gamma0 < 1.0))
        return -1;
    double M = std::log((double)p) / std::log(1.0 / gamma0);
    int32_t r = (int32_t)std::lround(M);
    if (r < 1)
        r = 1;
    if (r > XYZ_MAX_M)
        r = XYZ_MAX_M;
    return r;
}

}  // extern "C"
