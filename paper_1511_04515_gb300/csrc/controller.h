// Host-side featurisation and proposal rule of the learned step controller.
#pragma once
#include "../../include/ers.h"

namespace ers {

// network input (ERS_CTRL_FEATURES floats) from the last min(count, 8) accepted steps
void ctrl_features(const ers_step_record* recs, int count, float* out);
// training target (2 floats) of the step that followed recs[count-1]; false if unusable
bool ctrl_target(const ers_step_record* recs, int count, const ers_step_record& next, float* t);
// network output -> next step size and the first Krylov dimension at which the residual test
// runs (in [m_min, m_max]); the rule is stated with ers_ctrl_propose in ers.h
void ctrl_propose(const float* y, double h_k, double h_max, int m_min, int m_max, double margin,
                  double err_ratio, double* h_next, int* m_start);

}  // namespace ers
