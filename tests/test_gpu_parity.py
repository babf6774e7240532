"""GPU parity: the CUDA multigrid (through the C ABI) against the FP64 oracle.

Bar: relative L2 error over free cells <= 1e-9 for phi and each Psi_j at a
solver tolerance of 1e-10 relative residual, in both precision modes (FP64
V-cycles; FP32 V-cycles inside FP64 iterative refinement).  The oracle is
iterated to its round-off floor, so it stands for the exact discrete solution.
"""
import numpy as np
import pytest

import oracle
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARITY = 1e-9
TOL = 1e-10
PRECS = [0, 1]  # MG_PREC_FP64, MG_PREC_MIXED


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08857_gb300 import build, mg as _mg

    build.build()
    _mg.load()
    return _mg


def cuda(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_poisson(mg, shape, h, rho, eps=None, mask=None, mask_value=None, prec=0,
                bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE, tol=TOL, **kw):
    s = mg.Solver(shape, h, eps_r=cuda(eps), mask=cuda(mask), mask_value=cuda(mask_value),
                  bc_kind=bc_kind, bc_value=bc_value, precision=prec, **kw)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st = s.solve_poisson(cuda(rho), phi, tol)
    out = phi.cpu().numpy()
    s.close()
    return out, st


def oracle_poisson(shape, h, rho, eps=None, mask=None, mask_value=None,
                   bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE):
    p = oracle.Problem(shape, h, 0.0, eps, mask, bc_kind, bc_value)
    u0 = np.zeros(shape)
    if mask is not None:
        u0[mask != 0] = 0.0 if mask_value is None else mask_value[mask != 0]
    u, cyc, rel, _ = p.solve(rho / oracle.EPS0, u0=u0)
    assert rel < 1e-12
    return u, p


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1])
def test_gaussian_blobs_64(mg, prec, seed):
    """Plain Poisson on 64^3, 4 Gaussian blobs, gap BCs."""
    n = 64
    h = 1.0 / n
    rho = W.gaussian_blobs(n, seed)
    phi, st = gpu_poisson(mg, (n, n, n), h, rho, prec=prec)
    ref, p = oracle_poisson((n, n, n), h, rho)
    assert st["converged"] and st["rel_resid"] <= TOL
    # independent check of the reported residual by the oracle's operator
    bn = p.rhs_norm(rho / oracle.EPS0, np.zeros_like(phi))
    _, rn = p.residual(rho / oracle.EPS0, phi)
    assert rn / bn <= 1.01 * TOL
    assert oracle.rel_l2(phi, ref) <= PARITY


@pytest.mark.parametrize("prec", PRECS)
def test_variable_eps_mask_nonCubic(mg, prec):
    """Dielectric slab, an electrode block at potential 1, a non-cubic box
    (axes distinguishable) whose coarsest grid is 6 x 10 x 12 cells (x, y, z)."""
    shape = (48, 40, 24)  # (nz, ny, nx)
    nz, ny, nx = shape
    h = 1.0 / nz
    rng = np.random.default_rng(5)
    eps = np.where((np.arange(nz) + 0.5)[:, None, None] * h < 0.3, 4.0, 1.0) * np.ones(shape)
    eps *= rng.uniform(0.9, 1.1, shape)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[30:40, 15:22, 8:14] = 1
    mval = np.where(mask, 1.0, 0.0)
    rho = W.EPS0 * rng.standard_normal(shape) * 50
    phi, st = gpu_poisson(mg, shape, h, rho, eps, mask, mval, prec=prec, max_cycles=400)
    ref, _ = oracle_poisson(shape, h, rho, eps, mask, mval)
    assert st["converged"]
    assert np.all(phi[mask == 1] == 1.0)
    assert oracle.rel_l2(phi, ref, mask) <= PARITY


@pytest.mark.parametrize("prec", PRECS)
def test_all_dirichlet_odd_coarsest(mg, prec):
    """Dirichlet on all six faces with distinct values; 40^3 coarsens to 5^3."""
    n = 40
    h = 1.0 / n
    rho = W.gaussian_blobs(n, 3)
    kind = (0,) * 6
    val = (0.1, -0.2, 0.3, 0.4, -0.5, 0.6)
    phi, st = gpu_poisson(mg, (n, n, n), h, rho, prec=prec, bc_kind=kind, bc_value=val)
    ref, _ = oracle_poisson((n, n, n), h, rho, bc_kind=kind, bc_value=val)
    assert oracle.rel_l2(phi, ref) <= PARITY


@pytest.mark.parametrize("prec", PRECS)
def test_single_level_grid(mg, prec):
    """A 6 x 4 x 5 box cannot coarsen: the dense coarsest solve is the whole
    solver."""
    shape = (5, 4, 6)
    h = 0.2
    rng = np.random.default_rng(1)
    eps = rng.uniform(1, 3, shape)
    rho = W.EPS0 * rng.standard_normal(shape)
    phi, st = gpu_poisson(mg, shape, h, rho, eps, prec=prec)
    ref, _ = oracle_poisson(shape, h, rho, eps)
    assert st["cycles"] <= 3
    assert oracle.rel_l2(phi, ref) <= PARITY


@pytest.mark.parametrize("prec", PRECS)
def test_helmholtz_batch_64(mg, prec):
    n = 64
    h = 1.0 / n
    S = W.ionization_source(n, 0)
    kappas = W.helmholtz_kappas()
    s = mg.Solver((n, n, n), h, precision=prec)
    psi = [torch.zeros((n, n, n), dtype=torch.float64, device="cuda") for _ in range(3)]
    st = s.solve_helmholtz_batch(cuda(S), psi, kappas, TOL)
    s.close()
    for j, kap in enumerate(kappas):
        ref, _, rel, _ = oracle.helmholtz((n, n, n), h, kap).solve(S)
        assert st[j]["converged"]
        assert oracle.rel_l2(psi[j].cpu().numpy(), ref) <= PARITY, (j, kap)


@pytest.mark.parametrize("prec", PRECS)
def test_helmholtz_with_electrode(mg, prec):
    """Electrode cells hold Psi = 0 in the radiative-transfer solves."""
    n = 32
    h = 1.0 / n
    S = W.ionization_source(n, 1)
    mask = W.needle_mask(n, tip_z=0.6, tip_radius_cells=2.0)
    s = mg.Solver((n, n, n), h, mask=cuda(mask), precision=prec, max_cycles=400)
    psi = [torch.full((n, n, n), 3.0, dtype=torch.float64, device="cuda") for _ in range(3)]
    st = s.solve_helmholtz_batch(cuda(S), psi, (10.0, 100.0, 1000.0), TOL)
    s.close()
    for j, kap in enumerate((10.0, 100.0, 1000.0)):
        ref, _, _, _ = oracle.helmholtz((n, n, n), h, kap, mask=mask).solve(S)
        got = psi[j].cpu().numpy()
        assert np.all(got[mask == 1] == 0.0)
        assert oracle.rel_l2(got, ref, mask) <= PARITY


def test_zero_problem_returns_immediately(mg):
    n = 16
    phi, st = gpu_poisson(mg, (n, n, n), 1.0 / n, np.zeros((n, n, n)), bc_value=(0,) * 6)
    assert st["cycles"] == 0 and np.all(phi == 0)


def test_nonfinite_input_is_reported(mg):
    n = 16
    rho = np.zeros((n, n, n))
    rho[3, 4, 5] = np.nan
    with pytest.raises(mg.MGError) as ei:
        gpu_poisson(mg, (n, n, n), 1.0 / n, rho)
    assert ei.value.status == mg.MG_ERR_NONFINITE


def test_cycle_cap_reports_not_converged_with_stats(mg):
    n = 32
    rho = W.gaussian_blobs(n, 0)
    s = mg.Solver((n, n, n), 1.0 / n, max_cycles=2)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    st = s.solve_poisson(cuda(rho), phi, 1e-14, raise_on_nonconvergence=False)
    s.close()
    assert st["status"] == mg.MG_ERR_NOT_CONVERGED
    assert st["cycles"] == 2 and not st["converged"]
    assert st["hist"][2] < st["hist"][1] < st["hist"][0]


def test_mixed_and_fp64_agree_512_streamer(mg):
    """Full-size 512^3 streamer shell in the dielectric gap: both precision
    modes reach 1e-10; the oracle's own FP64 residual of each GPU answer is
    <= 1e-10 (a property that holds at any size), and they agree to 1e-9."""
    n = 512
    h = 1.0 / n
    rho = W.streamer_shell(n, 0)
    eps = W.dielectric_slab(n)
    out = {}
    for prec in PRECS:
        out[prec], st = gpu_poisson(mg, (n, n, n), h, rho, eps, prec=prec)
        assert st["converged"]
    p = oracle.poisson((n, n, n), h, eps_r=eps)
    f = rho / oracle.EPS0
    bn = p.rhs_norm(f, np.zeros((n, n, n)))
    for prec in PRECS:
        _, rn = p.residual(f, out[prec])
        assert rn / bn <= 1.05 * TOL, (prec, rn / bn)
    assert oracle.rel_l2(out[1], out[0]) <= PARITY


@pytest.mark.parametrize("graphs", [True, False])
def test_solve_set_concurrent_matches_oracle(mg, graphs):
    """Poisson + three Helmholtz solves of one time step in one call, run
    concurrently (with and without CUDA-graph steps; the Helmholtz problems
    stacked, or each on its own stream), against the oracle; without the
    stack the concurrent answers equal the one-at-a-time answers bit for bit
    (the stack runs each step with the most inner V-cycles any member needs,
    so its answers differ from those within the tolerance)."""
    n = 48
    h = 1.0 / n
    rho = W.streamer_shell(n, 2) + W.gaussian_blobs(n, 2)
    eps = W.dielectric_slab(n)
    S = W.ionization_source(n, 3)
    kap = W.helmholtz_kappas()
    out = {}
    for conc, no_stack in ((4, 0), (4, 1), (1, 0)):
        s = mg.Solver((n, n, n), h, eps_r=cuda(eps), precision=1, inner_cycles=2,
                      concurrency=conc, graphs=graphs)
        s.set_options(stack=1 - no_stack)
        phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
        psi = [torch.zeros_like(phi) for _ in range(3)]
        st = s.solve_set(cuda(rho), phi, cuda(S), psi, kap, TOL)
        s.close()
        assert all(x["converged"] for x in st)
        out[(conc, no_stack)] = [phi.cpu().numpy()] + [p.cpu().numpy() for p in psi]
    ref_phi, _ = oracle_poisson((n, n, n), h, rho, eps)
    refs = [ref_phi] + [oracle.helmholtz((n, n, n), h, k).solve(S)[0] for k in kap]
    for key in ((4, 0), (4, 1)):
        for got, ref in zip(out[key], refs):
            assert oracle.rel_l2(got, ref) <= PARITY, key
    for a, b in zip(out[(4, 1)], out[(1, 0)]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[(4, 0)][0], out[(1, 0)][0])  # the Poisson problem is alone


def test_repeated_solves_reuse_graphs(mg):
    """The same context solves twice (graphs replayed, ping-pong parity in
    either state) and gives the same answer as a fresh context."""
    n = 32
    h = 1.0 / n
    rho = W.gaussian_blobs(n, 4)
    s = mg.Solver((n, n, n), h, precision=1, inner_cycles=1)
    res = []
    for _ in range(3):
        phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
        st = s.solve_poisson(cuda(rho), phi, TOL)
        res.append((st["cycles"], phi.cpu().numpy()))
    s.close()
    assert res[0][0] == res[1][0] == res[2][0]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[1][1], res[2][1])


def test_autotune_picks_a_converging_configuration(mg, tmp_path):
    """mg_autotune on a small solve set returns a candidate from its grid that
    converges; the cache then reinstalls it without searching."""
    from paper_1809_08857_gb300 import autotune

    n = 32
    h = 1.0 / n
    rho, eps, S = W.streamer_shell(n, 1), W.dielectric_slab(n), W.ionization_source(n, 1)
    s = mg.Solver((n, n, n), h, eps_r=cuda(eps), precision=1)
    path = str(tmp_path / "tune.json")
    entry, hit = autotune.tuned(s, cuda(rho), cuda(S), W.helmholtz_kappas(), TOL, has_eps=True,
                                cache_path=path)
    assert not hit
    assert (entry["nu1"], entry["nu2"]) in [(1, 1), (2, 1), (2, 2), (3, 3)]
    assert 1 <= entry["inner_cycles"] <= 4
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    psi = [torch.zeros_like(phi) for _ in range(3)]
    st = s.solve_set(cuda(rho), phi, cuda(S), psi, W.helmholtz_kappas(), TOL)
    assert all(x["converged"] for x in st)
    ref, _ = oracle_poisson((n, n, n), h, rho, eps)
    assert oracle.rel_l2(phi.cpu().numpy(), ref) <= PARITY
    s2 = mg.Solver((n, n, n), h, eps_r=cuda(eps), precision=1)
    _, hit2 = autotune.tuned(s2, cuda(rho), cuda(S), W.helmholtz_kappas(), TOL, has_eps=True,
                             cache_path=path)
    assert hit2 and s2.options.inner_cycles == entry["inner_cycles"]
    s.close()
    s2.close()
