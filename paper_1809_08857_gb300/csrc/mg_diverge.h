// Divergence rule of the solvers' outer loops (FP64 V-cycles, mixed-precision
// refinement steps, FAC iterations of a composite solve).
//
// A solve stops with MG_ERR_DIVERGED once its relative residual has risen at
// each of the last three cycles and is more than twice what it was three
// cycles ago.  A multigrid cycle with a sound coarse operator contracts the
// residual by a fixed factor per cycle (Sec. 2: one V-cycle per solve in the
// paper's runs), so three rises in a row mean the iteration amplifies some
// error component; with a coarse operator that loses a thin electrode, the
// growth per step was 3.7.  A residual that only wanders at the round-off
// floor of the iteration (tol below what the precision reaches) seldom rises
// three times in a row and almost never doubles while doing so: such a solve
// still ends at max_cycles with MG_ERR_NOT_CONVERGED.
//
// Host-only and free of CUDA, so that the rule is tested on its own by a
// small C++ program.
#pragma once

namespace mg {

struct Growth {
  double r[4] = {0.0, 0.0, 0.0, 0.0};  // the last four residuals, r[3] the newest
  int n = 0;                           // how many of them are set

  // Records the relative residual after a cycle (the initial one first);
  // true when the solve diverges by the rule above.
  bool push(double rel) {
    r[0] = r[1];
    r[1] = r[2];
    r[2] = r[3];
    r[3] = rel;
    if (n < 4) ++n;
    return n == 4 && r[1] > r[0] && r[2] > r[1] && r[3] > r[2] && r[3] > 2.0 * r[0];
  }
};

}  // namespace mg
