"""GPU parity of the configuration the benchmark times, and of the options
it can choose.

The benchmark solves one set (the Poisson problem with the dielectric slab
and the streamer-shell charge, the three radiative-transfer problems with the
smoothed source) at 512^3 through mg_solve_set with four problems in flight,
CUDA-graph steps and the options mg_autotune installs (on GB300: V(2,1), three
inner V-cycles per refinement step, 128-plane refinement tile).  Here the same
set is solved with those options and with the autotuner's own choice, and
every answer is compared with the oracle's solution iterated to its
round-off floor (1e-9 relative L2) and checked by the oracle's FP64
residual; the FP64-mode GPU answer of the same set meets the same bars.  Smaller
cases sweep every settable refinement tile against the converged oracle,
check the per-term amplitudes of the three-term radiative-transfer solve
(Eq. 3) and the plain FP64 residual norms the benchmark reports.
"""
import numpy as np
import pytest

import oracle
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-10
PARITY = 1e-9
KAPPAS = (10.0, 100.0, 1000.0)


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08857_gb300 import build, mg as _mg

    build.build()
    _mg.load()
    return _mg


@pytest.fixture(scope="module")
def set512():
    n = 512
    return {"n": n, "rho": W.streamer_shell(n, 0), "eps": W.dielectric_slab(n),
            "S": W.ionization_source(n, 0)}


@pytest.fixture(scope="module")
def ref512(set512):
    """The oracle's solutions of the four problems of the set, iterated to its
    round-off floor (about a minute on the host cores): the exact discrete
    answers the GPU answers are compared with."""
    n = set512["n"]
    out = []
    for p, f in problems(set512):
        u, _, rel, _ = p.solve(f, tol=1e-13, max_cycles=200)
        assert rel < 1e-12
        out.append(u)
    return out


def problems(inp):
    n = inp["n"]
    h = 1.0 / n
    probs = [(oracle.poisson((n, n, n), h, eps_r=inp["eps"]), inp["rho"] / oracle.EPS0)]
    probs += [(oracle.helmholtz((n, n, n), h, k), inp["S"]) for k in KAPPAS]
    return probs


def solve_set(mg, inp, prec, options=None, tune_cache=None):
    n = inp["n"]
    dev = "cuda"
    rho = torch.from_numpy(inp["rho"]).to(dev)
    S = torch.from_numpy(inp["S"]).to(dev)
    s = mg.Solver((n, n, n), 1.0 / n, eps_r=torch.from_numpy(inp["eps"]).to(dev), precision=prec,
                  concurrency=4)
    if options:
        s.set_options(**options)
    tuned = None
    if tune_cache is not None:
        from paper_1809_08857_gb300 import autotune

        tuned, _ = autotune.tuned(s, rho, S, KAPPAS, TOL, has_eps=True, precision=prec,
                                  cache_path=tune_cache)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
    psi = [torch.zeros_like(phi) for _ in KAPPAS]
    st = s.solve_set(rho, phi, S, psi, KAPPAS, TOL)
    norms = [s.residual_norms("poisson", rho, phi)]
    norms += [s.residual_norms("helmholtz", S, p, k) for p, k in zip(psi, KAPPAS)]
    s.close()
    out = [phi.cpu().numpy()] + [p.cpu().numpy() for p in psi]
    del phi, psi, rho, S
    torch.cuda.empty_cache()
    return out, st, norms, tuned


def oracle_checks(inp, answers, norms, refs):
    """Each answer is within 1e-9 (relative L2) of the oracle's converged
    solution, its relative residual by the oracle (FP64, its own operator and
    lifts) is <= 1.01 tol, and the library's plain FP64 norms agree with the
    oracle's."""
    rels = []
    errs = [oracle.rel_l2(u, ref) for u, ref in zip(answers, refs)]
    print("rel_l2 vs oracle:", errs)
    assert max(errs) <= PARITY, errs
    for (p, f), u, (rn_lib, bn_lib) in zip(problems(inp), answers, norms):
        _, rn = p.residual(f, u)
        bn = p.rhs_norm(f, np.zeros_like(u))
        rels.append(rn / bn)
        assert rn / bn <= 1.01 * TOL, rels
        assert bn_lib == pytest.approx(bn, rel=1e-12)
        assert rn_lib == pytest.approx(rn, rel=1e-6, abs=1e-3 * TOL * bn)
    return rels


def test_bench_set_512_tuned_options(mg, set512, ref512):
    """The set with the options the benchmark runs on GB300 (V(2,1), three
    inner V-cycles, 128-plane refinement tile, four problems in flight,
    graph steps), and the same set in FP64 mode: every answer within 1e-9 of
    the oracle's converged solution and at <= 1e-10 by the oracle's FP64
    residual."""
    opts = {"nu1": 2, "nu2": 1, "inner_cycles": 3, "ir_zchunk": 128}
    mixed, st, norms, _ = solve_set(mg, set512, mg.MG_PREC_MIXED, opts)
    assert all(x["converged"] for x in st)
    oracle_checks(set512, mixed, norms, ref512)
    fp64, st64, norms64, _ = solve_set(mg, set512, mg.MG_PREC_FP64)
    assert all(x["converged"] for x in st64)
    oracle_checks(set512, fp64, norms64, ref512)


def test_bench_set_512_autotuned(mg, set512, ref512, tmp_path):
    """The set with whatever mg_autotune installs from an empty cache (as
    the benchmark does on a fresh machine): every answer within 1e-9 of the
    oracle's converged solution and at <= 1e-10 by its FP64 residual."""
    mixed, st, norms, tuned = solve_set(mg, set512, mg.MG_PREC_MIXED,
                                        tune_cache=str(tmp_path / "tune.json"))
    assert tuned is not None and tuned["ir_zchunk"] in (0, 16, 32, 64, 128)
    assert all(x["converged"] for x in st)
    oracle_checks(set512, mixed, norms, ref512)


@pytest.mark.parametrize("zchunk", [0, 16, 32, 64, 128])
def test_refinement_tiles_match_oracle(mg, zchunk):
    """Every settable tile of the refinement pass (z planes per CTA column;
    0 = automatic) on a non-cubic box whose 200 planes leave a ragged last
    chunk for each of them, with a dielectric slab, a shell charge, an
    electrode block, and one Helmholtz problem: converged answers within 1e-9
    of the oracle."""
    shape = (200, 40, 48)  # (nz, ny, nx)
    nz, ny, nx = shape
    h = 1.0 / nz
    rng = np.random.default_rng(11)
    eps = np.where((np.arange(nz) + 0.5)[:, None, None] * h < 0.2, 4.0, 1.0) * np.ones(shape)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[150:170, 12:22, 20:30] = 1
    mval = np.where(mask, 1.0, 0.0)
    rho = W.EPS0 * rng.standard_normal(shape) * 200
    S = np.abs(rng.standard_normal(shape))
    dev = "cuda"
    s = mg.Solver(shape, h, eps_r=torch.from_numpy(eps).to(dev),
                  mask=torch.from_numpy(mask).to(dev), mask_value=torch.from_numpy(mval).to(dev),
                  bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE, precision=mg.MG_PREC_MIXED,
                  max_cycles=400)
    s.set_options(ir_zchunk=zchunk, nu1=2, nu2=1, inner_cycles=2)
    phi = torch.zeros(shape, dtype=torch.float64, device=dev)
    psi = torch.zeros_like(phi)
    st = mg.solve_batch([{"solver": s, "kind": "poisson", "rhs": torch.from_numpy(rho).to(dev),
                          "u": phi},
                         {"solver": s, "kind": "helmholtz", "rhs": torch.from_numpy(S).to(dev),
                          "u": psi, "kappa": 30.0}], TOL)
    s.close()
    assert all(x["converged"] for x in st)
    P = oracle.Problem(shape, h, 0.0, eps, mask, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    ref, _, rel, _ = P.solve(rho / oracle.EPS0, u0=mval, max_cycles=2000)
    assert rel < 1e-12
    assert oracle.rel_l2(phi.cpu().numpy(), ref, mask) <= PARITY
    refh, _, rel, _ = oracle.helmholtz(shape, h, 30.0, mask=mask).solve(S, max_cycles=2000)
    assert rel < 1e-12
    assert oracle.rel_l2(psi.cpu().numpy(), refh, mask) <= PARITY


@pytest.mark.parametrize("prec", [0, 1])
def test_photoionization_amplitudes(mg, prec):
    """(kappa_j^2 - lap) Psi_j = A_j S with a different amplitude per term
    (one of them negative), from a nonzero guess: each answer within 1e-9 of
    the oracle's solution for the scaled source."""
    n = 48
    h = 1.0 / n
    S = W.ionization_source(n, 4)
    amp = (0.37, 1.0, -2.5)
    kap = (15.0, 150.0, 40.0)
    s = mg.Solver((n, n, n), h, precision=prec)
    psi = [torch.full((n, n, n), 0.5, dtype=torch.float64, device="cuda") for _ in range(3)]
    st = s.solve_photoionization(torch.from_numpy(S).cuda(), psi, kap, amp, TOL)
    s.close()
    for j in range(3):
        got = psi[j].cpu().numpy()
        assert st[j]["converged"]
        ref, _, rel, _ = oracle.helmholtz((n, n, n), h, kap[j]).solve(S * amp[j])
        assert rel < 1e-12
        assert oracle.rel_l2(got, ref) <= PARITY, j


def test_fp64_residual_norms_match_oracle(mg):
    """mg_residual_norms (plain FP64) against the oracle's residual and ||b||
    for the three problem kinds, with electrodes, a dielectric and the gap
    faces, on a random iterate."""
    shape = (24, 20, 28)
    nz, ny, nx = shape
    h = 1.0 / 28
    rng = np.random.default_rng(12)
    eps = rng.uniform(1.0, 4.0, shape)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[10:14, 5:9, 8:12] = 1
    mval = np.where(mask, 0.6, 0.0)
    f = rng.standard_normal(shape)
    u = rng.standard_normal(shape)
    dev = "cuda"
    s = mg.Solver(shape, h, eps_r=torch.from_numpy(eps).to(dev),
                  mask=torch.from_numpy(mask).to(dev), mask_value=torch.from_numpy(mval).to(dev),
                  bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE)
    cases = [("poisson", 0.0, oracle.Problem(shape, h, 0.0, eps, mask, W.GAP_BC_KIND,
                                             W.GAP_BC_VALUE), f * W.EPS0, f, np.where(mask, 0.6, u)),
             ("screened", 7.5, oracle.Problem(shape, h, 7.5, eps, mask, W.GAP_BC_KIND,
                                              W.GAP_BC_VALUE), f, f, np.where(mask, 0.6, u)),
             ("helmholtz", 20.0, oracle.helmholtz(shape, h, 20.0, mask=mask), f, f,
              np.where(mask, 0.0, u))]
    for kind, param, P, rhs, fo, uu in cases:
        rn, bn = s.residual_norms(kind, torch.from_numpy(rhs).to(dev),
                                  torch.from_numpy(uu).to(dev), param)
        _, rn_ref = P.residual(fo, uu)
        bn_ref = P.rhs_norm(fo, np.where(mask, uu, 0.0))
        assert rn == pytest.approx(rn_ref, rel=1e-12), kind
        assert bn == pytest.approx(bn_ref, rel=1e-12), kind
    s.close()


def test_two_cell_and_one_cell_refinement_kernels_agree(mg):
    """The refinement residual runs two x-adjacent cells per thread (FP32x2
    double-float arithmetic) when nx is even and every array sits on a
    16-byte boundary, else one cell per thread.  The residual norm of the same
    iterate through an aligned array and through an array offset by one FP64
    (8 bytes, so the one-cell kernel runs) agree to the FP32 summation order,
    and both agree with the oracle; the same for an odd nx (one-cell kernel
    either way)."""
    for shape in ((40, 36, 48), (24, 20, 27)):
        nz, ny, nx = shape
        h = 1.0 / nz
        rng = np.random.default_rng(31)
        mask_np = np.zeros(shape, dtype=np.uint8)
        mask_np[10:14, 5:11, 8:16] = 1
        rho_np = W.EPS0 * rng.standard_normal(shape) * 50
        u_np = np.where(mask_np == 1, 0.5, rng.standard_normal(shape))
        n = u_np.size
        buf_u = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        buf_r = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        u_al = torch.from_numpy(u_np).cuda()
        r_al = torch.from_numpy(rho_np).cuda()
        u_off = buf_u[1:].view(shape)
        r_off = buf_r[1:].view(shape)
        u_off.copy_(u_al)
        r_off.copy_(r_al)
        assert u_off.data_ptr() % 16 == 8
        mask = torch.from_numpy(mask_np).cuda()
        out = []
        for u, r in ((u_al, r_al), (u_off, r_off)):
            o = mg.residual_norm_noalloc(u, r, h, alpha=3.0, rhs_scale=1.0 / W.EPS0, mask=mask,
                                         bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE)
            torch.cuda.synchronize()
            out.append(o.item())
        P = oracle.Problem(shape, h, 3.0, None, mask_np, W.GAP_BC_KIND, W.GAP_BC_VALUE)
        _, rn = P.residual(rho_np / oracle.EPS0, u_np)
        assert out[0] == pytest.approx(out[1], rel=1e-6), (shape, out)
        assert out[0] == pytest.approx(rn, rel=1e-6), (shape, out, rn)


def test_trimmed_last_step_reaches_tol_with_fewer_vcycles(mg, set512, ref512):
    """The benchmark's set at 512^3 with V(2,1) and three inner V-cycles per
    step: with the last step trimmed to the V-cycles its measured rate needs
    (the default) every problem still meets 1e-10 in no more steps and no
    more V-cycles than with every step at three, fewer V-cycles in all (the
    Poisson and kappa L = 100 problems end far below tol with three), and
    every answer is within 1e-9 of the oracle's converged solution."""
    opts = {"nu1": 2, "nu2": 1, "inner_cycles": 3}
    st = {}
    for fixed in (1, 0):
        answers, st[fixed], norms, _ = solve_set(mg, set512, mg.MG_PREC_MIXED,
                                                 dict(opts, fixed_cycles=fixed))
        assert all(x["converged"] for x in st[fixed])
        oracle_checks(set512, answers, norms, ref512)
    for a, b in zip(st[0], st[1]):
        assert a["cycles"] <= b["cycles"] and a["vcycles"] <= b["vcycles"]
        assert b["vcycles"] == 3 * b["cycles"]
    assert sum(x["vcycles"] for x in st[0]) < sum(x["vcycles"] for x in st[1]), (
        [x["vcycles"] for x in st[0]], [x["vcycles"] for x in st[1]])


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_and_nonzero_guess_first_pass(mg, prec):
    """A cold start (zero guess, no electrode cells) takes a pointwise first
    pass (the residual is b); a guess with one nonzero entry takes the
    stencil pass.  Both reach the oracle's answer to 1e-9 and the zero guess
    starts at relative residual exactly 1; a nonzero guess (the oracle's
    answer plus a perturbation) converges to it too."""
    n = 48
    h = 1.0 / n
    rho, eps, S = W.streamer_shell(n, 3), W.dielectric_slab(n), W.ionization_source(n, 3)
    P = oracle.poisson((n, n, n), h, eps_r=eps)
    ref, _, rel, _ = P.solve(rho / oracle.EPS0)
    assert rel < 1e-12
    refh = [oracle.helmholtz((n, n, n), h, k).solve(S)[0] for k in KAPPAS]
    rng = np.random.default_rng(21)
    guesses = {"zero": (np.zeros((n, n, n)), [np.zeros((n, n, n))] * 3)}
    one = np.zeros((n, n, n))
    one[7, 9, 11] = 1e-300
    guesses["one entry"] = (one, [one] * 3)
    guesses["near"] = (ref + 1e-3 * rng.standard_normal((n, n, n)),
                       [r + 1e-3 * rng.standard_normal((n, n, n)) for r in refh])
    s = mg.Solver((n, n, n), h, eps_r=torch.from_numpy(eps).cuda(), precision=prec)
    for name, (g, gh) in guesses.items():
        phi = torch.from_numpy(g.copy()).cuda()
        psi = [torch.from_numpy(x.copy()).cuda() for x in gh]
        st = s.solve_set(torch.from_numpy(rho).cuda(), phi, torch.from_numpy(S).cuda(), psi,
                         KAPPAS, TOL)
        assert all(x["converged"] for x in st), name
        if name == "zero":
            assert all(x["hist"][0] == 1.0 for x in st)
        assert oracle.rel_l2(phi.cpu().numpy(), ref) <= PARITY, name
        for p, r in zip(psi, refh):
            assert oracle.rel_l2(p.cpu().numpy(), r) <= PARITY, name
    s.close()
