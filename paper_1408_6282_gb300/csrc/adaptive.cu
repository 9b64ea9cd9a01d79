// Adaptive error estimation for SKIM (Section 4.3.2, Eq. chernoff): a
// confidence bound on the sum over iterations of the discrepancy, the gap
// between the largest marginal coverage in the residual problem and the
// coverage of the seed that was selected.  Host-only FP64 arithmetic over what
// skim_greedy_ex recorded on the device (delta, tau, k').
//
// Per iteration j: if the true maximum were delta_j + d, that node would hold
// in expectation mu = tau_j (delta_j + d) of the processed ranks, yet no node
// other than the seed held more than k'_j of them.  The lower Chernoff tail
// bounds the chance of that:
//     P[D_j > d] <= B_j(d) = (exp(-nu) / (1 - nu)^(1 - nu))^mu,
//     nu = 1 - k'_j / mu,   and B_j(d) = 1 where mu <= k'_j,
// evaluated as exp(k' - mu + k' ln(mu / k')) (exp(-mu) for k' = 0).
// D_j is dominated by a variable on the grid {0, h, 2h, ...}: value (i+1)h
// with probability B_j(ih) - B_j((i+1)h), 0 with 1 - B_j(0); mass beyond the
// last cell is kept apart as an overflow cell that counts as unbounded.  The
// sum of discrepancies is bounded by the convolution of these variables over
// the iterations (treated as independent).
#include <cmath>
#include <cstdint>
#include <vector>

#include "skim.h"

namespace {

double tail_bound(double mu, int32_t kp) {
    if (!(mu > kp)) return 1.0;
    if (kp == 0) return std::exp(-mu);
    const double k = kp;
    return std::exp(k - mu + k * std::log1p((mu - k) / k));
}

}  // namespace

extern "C" int skim_discrepancy_bound(uint32_t s, const uint64_t *delta, const uint64_t *tau,
                                      const int32_t *kprime, double step, uint32_t bins, uint32_t n_conf,
                                      const double *conf, double *bound_out, double *ccdf_out) {
    if (s && (!delta || !tau || !kprime)) return SKIM_EINVAL;
    if (n_conf && (!conf || !bound_out)) return SKIM_EINVAL;
    if (!(step > 0) || !std::isfinite(step) || bins == 0) return SKIM_EINVAL;
    for (uint32_t c = 0; c < n_conf; c++)
        if (!(conf[c] > 0 && conf[c] < 1)) return SKIM_EINVAL;
    for (uint32_t j = 0; j < s; j++)
        if (kprime[j] < -1) return SKIM_EINVAL;

    // running distribution of the sum: cells 0..bins-1 and the overflow
    std::vector<double> r(bins, 0.0), q(bins), nr(bins), qsuf(bins + 1);
    r[0] = 1.0;
    double ovf = 0.0;
    for (uint32_t j = 0; j < s; j++) {
        if (kprime[j] < 0) continue;  // exact selection: a point mass at 0
        const double t = std::ldexp(static_cast<double>(tau[j]), -64);
        const double dl = static_cast<double>(delta[j]);
        double prev = tail_bound(t * dl, kprime[j]);
        q[0] = 1.0 - prev;
        uint32_t len = 1;
        for (uint32_t i = 1; i < bins; i++) {
            const double b = tail_bound(t * (dl + static_cast<double>(i) * step), kprime[j]);
            q[i] = prev - b;
            prev = b;
            if (q[i] != 0.0) len = i + 1;
        }
        const double qovf = prev;  // B_j((bins - 1) h)
        // qsuf[i] = sum of q[i..len)
        qsuf[len] = 0.0;
        for (uint32_t i = len; i-- > 0;) qsuf[i] = qsuf[i + 1] + q[i];
        double beyond = 0.0;
        for (uint32_t a = 0; a < bins; a++)  // r[a] q[b] with a + b >= bins leaves the grid
            if (r[a] != 0.0 && bins - a < len) beyond += r[a] * qsuf[bins - a];
        for (uint32_t t2 = 0; t2 < bins; t2++) {
            double acc = 0.0;
            const uint32_t bmax = t2 + 1 < len ? t2 + 1 : len;
            for (uint32_t b = 0; b < bmax; b++) acc += r[t2 - b] * q[b];
            nr[t2] = acc;
        }
        ovf = ovf + qovf - ovf * qovf + beyond;
        r.swap(nr);
    }
    // ccdf[i] = P[sum > i h] = mass in cells above i plus the overflow
    std::vector<double> ccdf(bins + 1);
    ccdf[bins] = ovf;
    double acc = ovf;
    for (uint32_t i = bins; i-- > 0;) {
        ccdf[i] = acc;
        acc += r[i];
    }
    if (ccdf_out)
        for (uint32_t i = 0; i <= bins; i++) ccdf_out[i] = ccdf[i];
    for (uint32_t c = 0; c < n_conf; c++) {
        const double allow = 1.0 - conf[c];
        double b = HUGE_VAL;
        for (uint32_t i = 0; i < bins; i++)
            if (ccdf[i] <= allow) {
                b = static_cast<double>(i) * step;
                break;
            }
        bound_out[c] = b;
    }
    return SKIM_OK;
}
