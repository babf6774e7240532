"""The last-step trimming rule of the mixed-precision solve (host logic, no
GPU): from the second finished refinement step on, the contraction per
V-cycle measured over the step that just finished, taken 15 % weaker in its
logarithm, sets how many V-cycles the next step needs to reach tol; fewer
than inner_cycles are run only when that count is smaller.  The rule's
header is compiled into a small C++ program; the cases are the residual
histories of the benchmark's 512^3 set (whose V-cycle counts 14, 12, 11, 8
for steps of 4 the line reports) and the rule's guards."""
import math
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_08857_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstdlib>
#include "mg_trim.h"
// argv: full fixed steps last rel_prev rel tol; prints the next step's V-cycles
int main(int argc, char** argv) {
  if (argc != 8) return 2;
  std::printf("%d\n", mg::trimmed_inner_cycles(std::atoi(argv[1]), std::atoi(argv[2]) != 0,
                                               std::atoi(argv[3]), std::atoi(argv[4]),
                                               std::strtod(argv[5], nullptr),
                                               std::strtod(argv[6], nullptr),
                                               std::strtod(argv[7], nullptr)));
  return 0;
}
"""


@pytest.fixture(scope="module")
def trim(tmp_path_factory):
    d = tmp_path_factory.mktemp("trim")
    src = d / "trim.cpp"
    src.write_text(PROG)
    exe = d / "trim"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(full, fixed, steps, last, rel_prev, rel, tol):
        out = subprocess.run([str(exe), str(full), str(int(fixed)), str(steps), str(last),
                              repr(float(rel_prev)), repr(float(rel)), repr(float(tol))],
                             check=True, capture_output=True, text=True).stdout
        return int(out)

    return run


def replay(trim, hist, full=4, tol=1e-10):
    """V-cycles per step that the rule gives for a residual history (the
    first pass's residual first, then the residual after each step)."""
    cycles = []
    last = full
    for s in range(1, len(hist)):
        cycles.append(last)
        if s < len(hist) - 1:
            last = trim(full, False, s, last, hist[s - 1], hist[s], tol)
    return cycles


def test_benchmark_histories_give_the_reported_cycles(trim):
    """The four residual histories of one 512^3 benchmark set (Poisson with
    the slab and the shell, three Helmholtz problems): the rule trims the
    Poisson problem's fourth step to 2 V-cycles and the second Helmholtz
    problem's third step to 3, and leaves the others full, which is 14, 12,
    11 and 8 V-cycles."""
    hists = [
        [1.0, 7.493e-05, 1.921e-07, 5.366e-10, 2.643e-11],
        [1.0, 0.0003702, 1.109e-07, 3.634e-11],
        [1.0, 0.0001171, 1.518e-08, 1.903e-11],
        [1.0, 1.444e-07, 9.891e-15],
    ]
    got = [replay(trim, h) for h in hists]
    assert got == [[4, 4, 4, 2], [4, 4, 4], [4, 4, 3], [4, 4]]
    assert [sum(c) for c in got] == [14, 12, 11, 8]


def test_need_from_the_weakened_rate(trim):
    """The count is ceil(log(tol / rel) / (0.85 log(rel / rel_prev) / last)),
    worked by hand here for one case: rel_prev 1e-4, rel 1e-8 after 4
    V-cycles (1e-1 per cycle, weakened to 10^-0.85); reaching 1e-10 from 1e-8
    needs 2 / 0.85 = 2.35, so 3 V-cycles; to 1e-9, 1 / 0.85 = 1.18, so 2."""
    assert trim(4, False, 2, 4, 1e-4, 1e-8, 1e-10) == 3
    assert trim(4, False, 2, 4, 1e-4, 1e-8, 1e-9) == 2
    # just above tol: at least one V-cycle
    assert trim(4, False, 2, 4, 1e-4, 1.0000001e-10, 1e-10) == 1
    # a count of full or more stays full (never more than inner_cycles)
    assert trim(4, False, 2, 4, 1e-4, 1e-6, 1e-10) == 4
    assert trim(6, False, 3, 6, 1e-2, 1e-5, 1e-10) == 6


@pytest.mark.parametrize("case", [
    dict(fixed=True),                       # mg_options.fixed_cycles
    dict(steps=1),                          # the first step's rate is not used
    dict(steps=0),
    dict(last=0),
    dict(rel_prev=0.0),
    dict(rel=0.0),
    dict(rel=2e-8, rel_prev=1e-8),          # the residual rose
    dict(rel=1e-8, rel_prev=1e-8),          # or stayed
    dict(rel=float("nan")),
    dict(rel_prev=float("nan")),
])
def test_guards_keep_the_full_count(trim, case):
    """Where no rate can be measured, or the rule is switched off, the next
    step runs inner_cycles."""
    a = dict(full=4, fixed=False, steps=2, last=4, rel_prev=1e-4, rel=1e-8, tol=1e-10)
    a.update(case)
    assert trim(a["full"], a["fixed"], a["steps"], a["last"], a["rel_prev"], a["rel"],
                a["tol"]) == 4


def test_trimmed_step_reaches_tol_at_the_measured_rate(trim):
    """Whenever the rule trims, a step that contracts at the measured rate
    (not the weakened one) ends below tol: the cycles given are at least the
    exact count log(tol / rel) / log(rate)."""
    for rp, r, last in [(3.7e-4, 1.1e-7, 4), (1.2e-4, 1.5e-8, 4), (1.9e-7, 5.4e-10, 4),
                        (1e-3, 2e-7, 3), (5e-5, 1e-9, 2)]:
        c = trim(4, False, 2, last, rp, r, 1e-10)
        rate = (r / rp) ** (1.0 / last)
        assert r * rate ** c <= 1e-10 or c == 4
        assert c >= math.log(1e-10 / r) / math.log(rate) - 1e-12 or c == 4
