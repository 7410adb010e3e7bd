// prune_rule.cuh -- the pruning rule of Def. 2 / Eq. 1 as the prune and merge kernels take it:
// FP32 constants for the fast decision, FP64 constants for the near-tie re-decision, and the
// alpha grid of adaptive pruning (Alg. 4).
#pragma once

#include "cng_internal.h"
#include "device_common.cuh"

namespace cng {

struct RuleArgs {
  float alpha32, t32, band;
  double alpha64, t64;
  int R;   // out-degree bound
  int rs;  // row stride of the final adjacency (R + connectivity slots)
  // adaptive pruning (Alg. 4): alpha_i = alpha0 + i * dalpha for i = 0 .. imax; imax < 0: fixed
  double alpha0, dalpha, tau64;
  int imax;
};

// The rule at step i of Alg. 4, in the oracle's operation order (no contraction).
CNG_DEV RuleArgs rule_step(const RuleArgs& ra, int i) {
  RuleArgs r = ra;
  r.alpha64 = __dadd_rn(ra.alpha0, __dmul_rn((double)i, ra.dalpha));
  r.t64 = __dmul_rn(__dadd_rn(r.alpha64, 1.0), ra.tau64);
  r.alpha32 = (float)r.alpha64;
  r.t32 = (float)r.t64;
  return r;
}

// Alg. 2 with the fixed alpha, or Alg. 4: sweeps with alpha_0, alpha_1, ... until the kept set
// holds at least R/2 points (its first R are kept) or alpha_max was tried.  `sweep(rule)` runs
// one Alg. 2 pass and returns |S| (uniform over the CTA).  *steps receives the last i.
template <typename F>
CNG_DEV int prune_with_rule(const RuleArgs& ra, F&& sweep, int* steps) {
  int ns = 0, i = 0;
  for (;; ++i) {
    ns = sweep(ra.imax >= 0 ? rule_step(ra, i) : ra);
    if (ra.imax < 0 || 2 * ns >= ra.R || i >= ra.imax) break;
  }
  *steps = ra.imax >= 0 ? i : 0;
  return ns;
}

inline RuleArgs rule_args(double alpha, double tau, int R, float band, int rs, const AlphaGrid& g) {
  RuleArgs ra;
  ra.rs = rs;
  ra.alpha64 = alpha;
  ra.t64 = (alpha + 1.0) * tau;
  ra.alpha32 = (float)alpha;
  ra.t32 = (float)ra.t64;
  ra.band = band;
  ra.R = R;
  ra.alpha0 = g.alpha0;
  ra.dalpha = g.dalpha;
  ra.tau64 = tau;
  ra.imax = g.imax;
  return ra;
}

}  // namespace cng
