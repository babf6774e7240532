"""The solvers' divergence rule (host logic, no GPU): a solve stops with
MG_ERR_DIVERGED once its relative residual has risen at each of the last three
cycles and is over twice what it was three cycles earlier.  The rule's header
is compiled into a small C++ program that replays residual sequences; the C
layouts of the statistics and options records are checked against the
binding's."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_08857_gb300", "csrc")

REPLAY = r"""
#include <cstdio>
#include <cstdlib>
#include "mg_diverge.h"
// argv: residuals in order (the initial one first); prints the index of the
// first cycle at which the rule fires, or -1
int main(int argc, char** argv) {
  mg::Growth g;
  for (int i = 1; i < argc; ++i)
    if (g.push(std::strtod(argv[i], nullptr))) { std::printf("%d\n", i - 1); return 0; }
  std::printf("-1\n");
  return 0;
}
"""

LAYOUT = r"""
#include <stdio.h>
#include <stddef.h>
#include "mg.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(mg_stats), offsetof(mg_stats, vcycles),
         offsetof(mg_stats, diverged), sizeof(mg_options));
  return 0;
}
"""


@pytest.fixture(scope="module")
def replay(tmp_path_factory):
    d = tmp_path_factory.mktemp("diverge")
    src = d / "replay.cpp"
    src.write_text(REPLAY)
    exe = d / "replay"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(seq):
        out = subprocess.run([str(exe)] + [repr(float(x)) for x in seq], check=True,
                             capture_output=True, text=True).stdout
        return int(out)

    return run


def test_contracting_solve_never_fires(replay):
    seq = [1.0 * 0.15 ** k for k in range(40)]
    assert replay(seq) == -1


def test_growth_of_three_point_seven_per_step_fires_at_the_third_rise(replay):
    # a good first step, then the growth of a coarse operator that lost an
    # electrode: the rule fires after three rises (cycle 4 here)
    seq = [1.0, 0.2, 0.2 * 3.7, 0.2 * 3.7 ** 2, 0.2 * 3.7 ** 3, 0.2 * 3.7 ** 4]
    assert replay(seq) == 4


def test_two_rises_then_a_drop_do_not_fire(replay):
    seq = [1.0, 0.1, 0.3, 0.9, 0.05, 0.01, 0.03, 0.09, 0.001]
    assert replay(seq) == -1


def test_floor_wander_does_not_fire(replay):
    # three small rises at the round-off floor: under a factor of two in all
    seq = [1.0, 1e-4, 1e-8, 1e-11, 1.2e-11, 1.4e-11, 1.6e-11, 1.5e-11]
    assert replay(seq) == -1


def test_slow_rise_fires_only_once_doubled(replay):
    # rises of 1.2 per cycle: 1.2^3 = 1.73 < 2, then 1.2^4 over three cycles
    # is not counted either (the window is three cycles), so it never fires
    seq = [1.0 * 1.2 ** k for k in range(10)]
    assert replay(seq) == -1
    # rises of 1.3 per cycle double in three (2.197): fires at cycle 3
    seq = [1.0 * 1.3 ** k for k in range(10)]
    assert replay(seq) == 3


def test_status_and_layouts_match_the_binding(tmp_path):
    from paper_1809_08857_gb300 import mg

    header = open(os.path.join(ROOT, "include", "mg.h")).read()
    assert int(re.search(r"MG_ERR_DIVERGED\s*=\s*(\d+)", header).group(1)) == mg.MG_ERR_DIVERGED
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-O1", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    size, off_v, off_d, osize = map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.split())
    assert size == ctypes.sizeof(mg.Stats)
    assert off_v == mg.Stats.vcycles.offset and off_d == mg.Stats.diverged.offset
    assert osize == ctypes.sizeof(mg.Options)


def test_error_string(tmp_path):
    from paper_1809_08857_gb300 import build, mg

    build.build()
    lib = mg.load()
    assert lib.mg_error_string(mg.MG_ERR_DIVERGED).startswith(b"diverged")
