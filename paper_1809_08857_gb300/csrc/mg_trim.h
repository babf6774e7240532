// Inner V-cycles of the next refinement step of a mixed-precision solve.
//
// Every step runs the context's inner_cycles FP32 V-cycles, except that from
// the second finished step on, the contraction per V-cycle measured over the
// step that just finished may say that fewer reach tol: then the next step
// runs only that many.  The measured rate is taken 15 % weaker in its
// logarithm, so that a step that varies a little from the last one still
// lands below tol; if it does not, the step after it runs the full count
// again.  The fixed point and the stopping test are unchanged: only the
// number of V-cycles in the last step can shrink.  (An answer that meets tol
// is as close to the exact discrete solution as its problem's conditioning
// allows: the error of the 512^3 gap Poisson answer is up to 30 times its
// relative residual, since the boundary lift dominates ||b||; a stricter aim
// than tol removed every trimmed V-cycle of the benchmark's set.)  The first
// step is not used: it starts from the first pass's residual, whose
// contraction differs from the later steps' (for the Poisson problem of the
// benchmark 0.09 per V-cycle against 0.23).
//
// Host-only and free of CUDA, so that the rule is tested on its own by a
// small C++ program.
#pragma once

#include <algorithm>
#include <cmath>

namespace mg {

// full: inner_cycles; fixed: mg_options.fixed_cycles; steps: refinement
// steps finished; last: V-cycles of the step that just finished; rel_prev,
// rel: relative residuals before and after it; tol: the stopping tolerance.
inline int trimmed_inner_cycles(int full, bool fixed, int steps, int last, double rel_prev,
                                double rel, double tol) {
  if (fixed || steps < 2 || last < 1 || !(rel_prev > 0.0) || !(rel > 0.0) || !(rel < rel_prev))
    return full;
  const double per_cycle = std::log(rel / rel_prev) / last;  // < 0
  const double need = std::log(tol / rel) / (0.85 * per_cycle);
  if (!(need > 0.0) || need >= full) return full;
  return std::max(1, (int)std::ceil(need));
}

}  // namespace mg
