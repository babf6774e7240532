"""Host logic of the autotune cache (no GPU): keys, round trip, and that a
cached entry is installed without searching again."""
from paper_1809_08857_gb300 import autotune


class FakeSolver:
    shape = (64, 48, 32)

    def __init__(self):
        self.set_calls = []
        self.tunes = 0

    def set_options(self, **kw):
        self.set_calls.append(kw)

    def autotune(self, rho, S, kappa, tol):
        self.tunes += 1
        return {"nu1": 2, "nu2": 1, "inner_cycles": 3, "ir_zchunk": 32, "sweep_zchunk": 16}, 12.5


def test_signature_distinguishes_problem_classes():
    a = autotune.signature("GB300", (8, 8, 8), True, False, 1, 1e-10)
    assert a != autotune.signature("GB300", (8, 8, 8), False, False, 1, 1e-10)
    assert a != autotune.signature("GB300", (8, 8, 16), True, False, 1, 1e-10)
    assert a != autotune.signature("B200", (8, 8, 8), True, False, 1, 1e-10)
    assert "32x48x64" in autotune.signature("X", (64, 48, 32), 0, 0, 1, 1e-10)


def test_tune_then_hit_cache(tmp_path):
    path = str(tmp_path / "cache.json")
    s1 = FakeSolver()
    e1, hit1 = autotune.tuned(s1, None, None, (1, 2, 3), has_eps=True, cache_path=path, device="D")
    assert not hit1 and s1.tunes == 1 and e1["inner_cycles"] == 3
    s2 = FakeSolver()
    e2, hit2 = autotune.tuned(s2, None, None, (1, 2, 3), has_eps=True, cache_path=path, device="D")
    assert hit2 and s2.tunes == 0
    assert s2.set_calls == [{"nu1": 2, "nu2": 1, "inner_cycles": 3, "ir_zchunk": 32,
                             "sweep_zchunk": 16}]
    s3 = FakeSolver()
    _, hit3 = autotune.tuned(s3, None, None, (1, 2, 3), has_eps=False, cache_path=path, device="D")
    assert not hit3 and s3.tunes == 1


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "cache.json"
    path.write_text("{not json")
    s = FakeSolver()
    _, hit = autotune.tuned(s, None, None, (1, 2, 3), cache_path=str(path), device="D")
    assert not hit and s.tunes == 1


def test_entry_without_tile_installs_the_automatic_tile(tmp_path):
    """Entries written before the refinement-pass tile and the staged
    half-sweep's planes were tuned install ir_zchunk = sweep_zchunk = 0
    (automatic)."""
    path = str(tmp_path / "cache.json")
    key = autotune.signature("D", FakeSolver.shape, True, False, 1, 1e-10)
    autotune.store(path, key, {"nu1": 1, "nu2": 1, "inner_cycles": 2, "ms": 3.0})
    s = FakeSolver()
    _, hit = autotune.tuned(s, None, None, (1, 2, 3), has_eps=True, cache_path=path, device="D")
    assert hit and s.set_calls == [{"nu1": 1, "nu2": 1, "inner_cycles": 2, "ir_zchunk": 0,
                                    "sweep_zchunk": 0}]
