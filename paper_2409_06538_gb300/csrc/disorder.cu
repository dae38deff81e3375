// Disorder averages of per-realization thermal means (Sec. III.C), host code behind the C ABI.
//
// [A] is the plain mean of A over realizations and its standard error the sample standard
// deviation divided by sqrt(R).  The Binder ratios take ratios of disorder means,
// U_m = [<m^4>] / [<m^2>]^2 and Q_q = [<q^4>] / [<q^2>]^2 (Eq. eq:binderEA with its denominator
// read as the square of the disorder mean; [<q^2>^2], the other reading, is returned beside it);
// the overlap susceptibility is chi_q = (L^2/T) ([<q^2>] - [<q>]^2) as printed in Eq. eq:susEA
// (square of the disorder mean of q), and the edge susceptibility chi_edge = L [<m_edge^2>].
// Realizations whose proposals met a doubly clamped site (status TNMC_ERR_NUMERIC) are skipped.
#include <cmath>
#include <cstring>
#include <limits>

#include "../../include/tnmc.h"

namespace {

double obs_field(const tnmc_obs& o, int k) {
  switch (k) {
    case TNMC_DIS_E: return o.E;
    case TNMC_DIS_E2: return o.E2;
    case TNMC_DIS_MABS: return o.m_abs;
    case TNMC_DIS_M2: return o.m2;
    case TNMC_DIS_M4: return o.m4;
    case TNMC_DIS_Q: return o.q;
    case TNMC_DIS_QABS: return o.q_abs;
    case TNMC_DIS_Q2: return o.q2;
    case TNMC_DIS_Q4: return o.q4;
    case TNMC_DIS_MEDGE: return o.m_edge;
    case TNMC_DIS_MEDGEABS: return o.m_edge_abs;
    default: return o.m_edge2;
  }
}

}  // namespace

extern "C" tnmc_status tnmc_disorder_average(const tnmc_obs* obs, int n_real, int L, double beta,
                                             tnmc_disorder* out) {
  if (!obs || !out || n_real < 1 || L < 2 || !(beta > 0.0) || !std::isfinite(beta)) return TNMC_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  const double nan = std::numeric_limits<double>::quiet_NaN();
  int used = 0;
  for (int r = 0; r < n_real; ++r) {
    if (obs[r].status != TNMC_OK) { ++out->n_dropped; continue; }
    ++used;
    out->n_prop += obs[r].n_prop;
    out->n_tests += obs[r].n_tests;
    out->n_acc += obs[r].n_acc;
    out->clamps += obs[r].clamps;
  }
  out->n_used = used;
  if (used == 0) {
    for (int k = 0; k < TNMC_DIS_N; ++k) { out->mean[k] = nan; out->se[k] = nan; }
    out->U_m = out->Q_q = out->q2_sq = out->chi_q = out->chi_edge = out->acceptance = nan;
    return TNMC_ERR_NUMERIC;
  }
  // two passes per quantity: the mean, then the sum of squared deviations from it
  for (int k = 0; k < TNMC_DIS_N; ++k) {
    double s = 0.0;
    for (int r = 0; r < n_real; ++r)
      if (obs[r].status == TNMC_OK) s += obs_field(obs[r], k);
    const double mean = s / used;
    double ss = 0.0;
    for (int r = 0; r < n_real; ++r)
      if (obs[r].status == TNMC_OK) { const double d = obs_field(obs[r], k) - mean; ss += d * d; }
    out->mean[k] = mean;
    out->se[k] = used > 1 ? std::sqrt(ss / (used - 1)) / std::sqrt((double)used) : 0.0;
  }
  double q2sq = 0.0;
  for (int r = 0; r < n_real; ++r)
    if (obs[r].status == TNMC_OK) q2sq += obs[r].q2 * obs[r].q2;
  out->q2_sq = q2sq / used;
  const double m2 = out->mean[TNMC_DIS_M2], q2 = out->mean[TNMC_DIS_Q2];
  out->U_m = m2 > 0.0 ? out->mean[TNMC_DIS_M4] / (m2 * m2) : nan;
  out->Q_q = q2 > 0.0 ? out->mean[TNMC_DIS_Q4] / (q2 * q2) : nan;
  const double q1 = out->mean[TNMC_DIS_Q];
  out->chi_q = (double)L * L * beta * (q2 - q1 * q1);
  out->chi_edge = (double)L * out->mean[TNMC_DIS_MEDGE2];
  out->acceptance = out->n_tests > 0 ? (double)out->n_acc / (double)out->n_tests : nan;
  return TNMC_OK;
}

// Inverse temperature on the Nishimori line of the +-J model (Sec. III.A): the gauge symmetry
// of P(J) = (1-p) delta(J-1) + p delta(J+1) gives exp(-2 beta) = p / (1-p), so
// beta = (1/2) ln((1-p)/p) for 0 < p < 1/2.
extern "C" tnmc_status tnmc_nishimori_beta(double p, double* beta_out) {
  if (!beta_out || !(p > 0.0 && p < 0.5)) return TNMC_ERR_ARG;
  *beta_out = 0.5 * std::log((1.0 - p) / p);
  return TNMC_OK;
}
