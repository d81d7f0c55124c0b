// Host side of the learned step controller: the network's input features from the history of
// accepted steps and the training targets taken from the plain controller's traces.  The
// formulas are stated with the declarations in ers.h.
#include "controller.h"

#include <algorithm>
#include <cmath>

namespace ers {

namespace {
inline double clampd(double v, double lo, double hi) { return std::min(hi, std::max(lo, v)); }
inline double log10_floor(double v, double lo) {
  return (v > 0.0 && std::isfinite(v)) ? std::max(lo, std::log10(v)) : lo;
}
}  // namespace

void ctrl_features(const ers_step_record* recs, int count, float* out) {
  for (int j = 0; j < ERS_CTRL_HISTORY; ++j) {
    const ers_step_record& r = recs[std::max(count - 1 - j, 0)];
    double hr = r.h_max > 0.0 ? r.h / r.h_max : 1.0;
    out[4 * j + 0] = (float)(clampd(log10_floor(hr, -6.0), -6.0, 0.0) / 3.0);
    out[4 * j + 1] = (float)(r.m_max > 0 ? (double)r.m / r.m_max : 0.0);
    double er = r.E > 0.0 ? r.err / r.E : 0.0;
    out[4 * j + 2] = (float)(clampd(log10_floor(er, -6.0), -6.0, 1.0) / 3.0);
    out[4 * j + 3] = (float)((clampd(log10_floor(r.dF, -12.0), -12.0, 0.0) + 6.0) / 6.0);
  }
}

bool ctrl_target(const ers_step_record* recs, int count, const ers_step_record& next, float* t) {
  if (next.landed || !(next.h > 0.0)) return false;
  const ers_step_record& r = recs[count - 1];
  double head = next.err > 0.0 ? 0.8 * std::sqrt(next.E / next.err) : 2.0;
  head = clampd(head, 1.0, 2.0);
  double t0 = std::log2(next.h / r.h) + std::log2(head);
  t[0] = (float)clampd(t0, -3.0, 2.0);
  t[1] = (float)(next.m_max > 0 ? (double)next.m / next.m_max : 0.0);
  return std::isfinite(t0);
}

void ctrl_propose(const float* y, double h_k, double h_max, int m_min, int m_max, double margin,
                  double err_ratio, double* h_next, int* m_start) {
  double l2 = std::isfinite(y[0]) ? clampd(y[0] - margin, -3.0, 2.0) : 1.0;
  // safety band from the local error model err ~ h^2: r* = (E / err)^(1/2) is the ratio that
  // would land on the budget; the proposal stays within [min(1, r*/2), max(1, 2 r*)]
  double lr = (err_ratio > 0.0 && std::isfinite(err_ratio)) ? -0.5 * std::log2(err_ratio) : 6.0;
  lr = clampd(lr, -3.0, 6.0);
  l2 = clampd(l2, std::min(0.0, lr - 1.0), std::max(0.0, lr + 1.0));
  *h_next = std::min(h_k * std::exp2(l2), h_max);
  double mm = std::isfinite(y[1]) ? y[1] * m_max : (double)m_min;
  int ms = (int)std::floor(mm + 0.5) - 1;
  *m_start = std::min(m_max, std::max(m_min, ms));
}

}  // namespace ers

extern "C" {

ers_status ers_ctrl_features(const ers_step_record* recs, int32_t count, float* out) {
  if (!recs || count < 1 || !out) return ERS_ERR_INVALID;
  ers::ctrl_features(recs, count, out);
  return ERS_OK;
}

ers_status ers_ctrl_target(const ers_step_record* recs, int32_t count, const ers_step_record* next,
                           float* t) {
  if (!recs || count < 1 || !next || !t) return ERS_ERR_INVALID;
  return ers::ctrl_target(recs, count, *next, t) ? ERS_OK : ERS_ERR_INVALID;
}

ers_status ers_ctrl_propose(const float* y, const ers_step_record* last, double margin,
                            int32_t m_min, double* h_next, int32_t* m_start) {
  if (!y || !last || !h_next || !m_start || !(margin >= 0.0) || m_min < 1 || last->m_max < m_min)
    return ERS_ERR_INVALID;
  int ms = 0;
  double ratio = last->E > 0.0 ? last->err / last->E : 0.0;
  ers::ctrl_propose(y, last->h, last->h_max, m_min, last->m_max, margin, ratio, h_next, &ms);
  *m_start = ms;
  return ERS_OK;
}

}  // extern "C"
