"""GPU tests of the composite AMR path (mg_amr_*): the composite residual
kernel against the FP64 oracle cell by cell, and composite solves (Poisson
with permittivity and electrodes, screened, Helmholtz; two and three levels;
FP64 and mixed precision) against the oracle's sparse direct solution."""
import numpy as np
import pytest

import oracle
from oracle import amr as oamr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARITY = 1e-9
TOL = 1e-10
POISSON_BC = ((1, 1, 1, 1, 0, 0), (0.0, 0.0, 0.0, 0.0, 0.0, 1.0))
NEUMANN = ((1,) * 6, (0.0,) * 6)

# three levels on a 16^3 base (two level-1 boxes, one level-2 box)
SMALL = ((16, 16, 16), [(1, (8, 8, 8), (12, 16, 8)), (1, (6, 20, 18), (8, 6, 10)),
                        (2, (20, 20, 20), (8, 8, 8))])
# three levels on a 24^3 base, about 22k unknowns
MEDIUM = ((24, 24, 24), [(1, (10, 10, 10), (16, 16, 16)), (1, (30, 8, 30), (12, 12, 12)),
                         (2, (24, 24, 24), (16, 16, 16))])
# two levels
TWO = ((16, 24, 16), [(1, (8, 10, 6), (16, 20, 12))])


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


def shapes_of(layout):
    base, boxes = layout
    return [tuple(base)] + [tuple(b[2]) for b in boxes]


def coefficients(layout, seed, spread=0.5):
    rng = np.random.default_rng(seed)
    return [np.exp(spread * rng.standard_normal(s)) for s in shapes_of(layout)]


def smooth_source(H, seed):
    """A few Gaussian blobs sampled at the cell centres of every box."""
    rng = np.random.default_rng(seed)
    cs = rng.uniform(0.25, 0.75, (4, 3))
    amp = rng.uniform(0.5, 2.0, 4)
    out = []
    for q in range(len(H.boxes)):
        z, y, x = H.cell_centres(q)
        v = np.zeros(z.shape)
        for c, a in zip(cs, amp):
            v += a * np.exp(-((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2) / (2 * 0.08 ** 2))
        out.append(v)
    return out


def electrode(base):
    m = np.zeros(base, np.uint8)
    m[1:3, base[1] - 6:base[1] - 3, 2:5] = 1
    return m


def make(mg, layout, beta=None, mask=None, mask_value=None, bc=POISSON_BC, precision=0,
         inner_cycles=1, max_cycles=100):
    base, boxes = layout
    return mg.Amr(base, 1.0 / base[0], boxes,
                  eps_r=None if beta is None else [cuda(b) for b in beta],
                  mask=cuda(mask), mask_value=cuda(mask_value), bc_kind=bc[0], bc_value=bc[1],
                  precision=precision, inner_cycles=inner_cycles, max_cycles=max_cycles)


def oracle_of(layout, alpha, beta=None, mask=None, mask_value=None, bc=POISSON_BC):
    base, boxes = layout
    return oamr.Hierarchy(base, 1.0 / base[0], boxes, alpha=alpha, beta=beta, mask=mask,
                          mask_value=mask_value, bc_kind=bc[0], bc_value=bc[1])


@pytest.mark.parametrize("kind", ["screened", "poisson", "helmholtz"])
def test_composite_residual_matches_oracle(mg, kind):
    """mg_amr_residual of a random iterate: every valid cell equals the
    oracle's composite residual (FP64), covered cells the mean of their
    children, electrode cells 0, and the norm."""
    rng = np.random.default_rng(11)
    layout = SMALL
    shapes = shapes_of(layout)
    beta = None if kind == "helmholtz" else coefficients(layout, 12)
    mask = electrode(layout[0]) if kind != "screened" else None
    mv = np.where(mask != 0, 0.7, 0.0) if (mask is not None and kind == "poisson") else None
    bc = NEUMANN if kind == "screened" else POISSON_BC
    alpha, param = {"screened": (3.0, 3.0), "poisson": (0.0, 0.0),
                    "helmholtz": (49.0, 7.0)}[kind]
    if kind == "helmholtz":
        bc_o = ((0,) * 6, (0.0,) * 6)
    else:
        bc_o = bc
    H = oracle_of(layout, alpha, beta, mask, mv, bc_o)
    u = [rng.standard_normal(s) for s in shapes]
    if mask is not None:
        u[0][mask != 0] = 0.0 if mv is None else mv[mask != 0]
    f = [rng.standard_normal(s) for s in shapes]
    A = make(mg, layout, beta, mask, mv, bc)
    rhs = [cuda(x * (oracle.EPS0 if kind == "poisson" else 1.0)) for x in f]
    r, norm = A.residual(kind, rhs, [cuda(x) for x in u], param=param)
    A.close()
    r = [t.cpu().numpy() for t in r]
    ref, ref_norm = H.residual(f, u)
    ref = H.average_down(ref)
    scale = max(np.abs(x).max() for x in ref)
    for q in range(len(shapes)):
        np.testing.assert_allclose(r[q], ref[q], rtol=0, atol=1e-12 * scale)
    # r^2 is summed in FP32 per thread (FP64 across blocks)
    assert abs(norm - ref_norm) <= 1e-6 * ref_norm


def test_composite_residual_conserves_flux(mg):
    """Neumann faces, alpha = 0, random coefficient: the volume-weighted sum
    of A u over the valid cells is zero (r = -A u for rhs 0)."""
    rng = np.random.default_rng(13)
    layout = SMALL
    shapes = shapes_of(layout)
    beta = coefficients(layout, 14, 1.0)
    A = make(mg, layout, beta, bc=NEUMANN)
    u = [cuda(rng.standard_normal(s)) for s in shapes]
    r, _ = A.residual("screened", [torch.zeros_like(t) for t in u], u, param=0.0)
    A.close()
    H = oracle_of(layout, 0.0, beta, bc=NEUMANN)
    y = H.gather([t.cpu().numpy() for t in r]) * H.volumes()
    assert abs(y.sum()) <= 1e-12 * np.abs(y).sum()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("layout", [TWO, SMALL, MEDIUM], ids=["two", "small", "medium"])
def test_poisson_solve_matches_oracle(mg, precision, layout):
    """Composite Poisson solve (permittivity on every box, an electrode held
    at 0.6, Dirichlet z faces) against the oracle's sparse direct solution."""
    beta = coefficients(layout, 21, 0.4)
    mask = electrode(layout[0])
    mv = np.where(mask != 0, 0.6, 0.0)
    H = oracle_of(layout, 0.0, beta, mask, mv)
    rho = smooth_source(H, 22)
    ref = H.solve(rho)
    A = make(mg, layout, beta, mask, mv, precision=precision)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in shapes_of(layout)]
    st = A.solve("poisson", [cuda(x * oracle.EPS0) for x in rho], u, tol=TOL)
    A.close()
    u = [t.cpu().numpy() for t in u]
    assert st["converged"] and st["cycles"] <= 25
    assert H.rel_l2(u, ref) <= PARITY
    # the oracle's own residual of the GPU solution
    _, rn = H.residual(rho, u)
    assert rn <= 1.01 * TOL * H.rhs_norm(rho)
    np.testing.assert_array_equal(u[0][mask != 0], 0.6)
    # covered cells hold the mean of their children
    back = H.average_down(u)
    for q in range(len(u)):
        np.testing.assert_allclose(u[q], back[q], rtol=0, atol=1e-14 * np.abs(back[q]).max())


@pytest.mark.parametrize("precision", [0, 1])
def test_screened_and_helmholtz_solves_match_oracle(mg, precision):
    layout = SMALL
    beta = coefficients(layout, 31, 0.3)
    # screened: alpha u - div(beta grad u) = f, Neumann faces
    H = oracle_of(layout, 40.0, beta, bc=NEUMANN)
    f = smooth_source(H, 32)
    ref = H.solve(f)
    A = make(mg, layout, beta, bc=NEUMANN, precision=precision)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in shapes_of(layout)]
    st = A.solve("screened", [cuda(x) for x in f], u, tol=TOL, param=40.0)
    assert st["converged"]
    assert H.rel_l2([t.cpu().numpy() for t in u], ref) <= PARITY
    # Helmholtz kappa = 12: beta = 1, Psi = 0 on the faces (the context's
    # coefficient is not used)
    Hh = oracle_of(layout, 144.0, None, bc=((0,) * 6, (0.0,) * 6))
    S = smooth_source(Hh, 33)
    ref = Hh.solve(S)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in shapes_of(layout)]
    st = A.solve("helmholtz", [cuda(x) for x in S], u, tol=TOL, param=12.0)
    A.close()
    assert st["converged"]
    assert Hh.rel_l2([t.cpu().numpy() for t in u], ref) <= PARITY


def test_without_refined_boxes_it_is_the_single_grid_solve(mg):
    """No refined boxes: the AMR solve equals the single-grid solver's
    (Poisson, electrode, permittivity) to the parity bound."""
    base = (16, 24, 32)
    rng = np.random.default_rng(41)
    beta = np.exp(0.4 * rng.standard_normal(base))
    mask = electrode(base)
    mv = np.where(mask != 0, 0.6, 0.0)
    rho = rng.standard_normal(base) * oracle.EPS0
    A = mg.Amr(base, 1.0 / 16, [], eps_r=[cuda(beta)], mask=cuda(mask), mask_value=cuda(mv))
    u = [torch.zeros(base, dtype=torch.float64, device="cuda")]
    A.solve("poisson", [cuda(rho)], u, tol=TOL)
    A.close()
    ref, _, _, _ = oracle.poisson(base, 1.0 / 16, beta, mask).solve(rho / oracle.EPS0,
                                                                     u0=mv)
    assert oracle.rel_l2(u[0].cpu().numpy(), ref, mask) <= PARITY


def test_warm_start_from_the_solution_takes_no_iteration(mg):
    layout = TWO
    H = oracle_of(layout, 5.0, None, bc=NEUMANN)
    f = smooth_source(H, 51)
    ref = H.solve(f)
    A = make(mg, layout, None, bc=NEUMANN)
    u = [cuda(x) for x in ref]
    st = A.solve("screened", [cuda(x) for x in f], u, tol=1e-9, param=5.0)
    A.close()
    assert st["cycles"] == 0 and st["converged"]


def test_bad_hierarchies_are_rejected(mg):
    base = (16, 16, 16)
    mask = np.zeros(base, np.uint8)
    mask[8, 3, 8] = 1  # next to the box below
    with pytest.raises(mg.MGError) as e:
        mg.Amr(base, 1.0 / 16, [(1, (8, 8, 8), (8, 8, 8))], mask=cuda(mask))
    assert e.value.status == mg.MG_ERR_INVALID_ARG
    A = mg.Amr(base, 1.0 / 16, [(1, (8, 8, 8), (8, 8, 8))], rte_bc=mg.MG_RTE_BC_MARSHAK)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in A.shapes]
    with pytest.raises(mg.MGError) as e:
        A.solve("helmholtz", u, [torch.zeros_like(t) for t in u], param=3.0)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
    A.close()


@pytest.mark.parametrize("n0", [64, 128])
def test_streamer_hierarchy_meets_tol_by_the_oracle(mg, n0):
    """The nested streamer-head hierarchy of the benchmark (three refined
    levels around the channel and head, dielectric slab on the base, shell
    charge sampled on every level) at a reduced base size, mixed precision
    with two inner V-cycles as timed: the oracle's FP64 composite residual of
    the GPU solution meets the tolerance, and the library's residual norm of
    that solution agrees with the oracle's."""
    from paper_1809_08857_gb300 import workloads as W

    h0 = 1.0 / n0
    boxes = W.streamer_amr_layout(n0)
    eps = [W.dielectric_slab(n0)] + [None] * len(boxes)
    rho = [W.streamer_shell_box((n0,) * 3, h0, (0, 0, 0), 0, thickness=h0)]
    for q, b in enumerate(boxes):
        o, h = W.amr_box_origin(h0, b)
        rho.append(W.streamer_shell_box(b[2], h, o, q + 1, thickness=h0))
    A = mg.Amr((n0,) * 3, h0, boxes, eps_r=[cuda(e) for e in eps], bc_kind=W.GAP_BC_KIND,
               bc_value=W.GAP_BC_VALUE, precision=1, inner_cycles=2)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in A.shapes]
    rhs = [cuda(r) for r in rho]
    st = A.solve("poisson", rhs, u, tol=TOL)
    _, gpu_norm = A.residual("poisson", rhs, u)
    A.close()
    assert st["converged"] and st["cycles"] <= 12
    H = oamr.Hierarchy((n0,) * 3, h0, boxes, beta=eps, bc_kind=W.GAP_BC_KIND,
                       bc_value=W.GAP_BC_VALUE)
    f = [r / oracle.EPS0 for r in rho]
    un = [t.cpu().numpy() for t in u]
    _, rn = H.residual(f, un)
    bn = H.rhs_norm(f)
    assert rn <= 1.01 * TOL * bn
    # the library's residual (double-float rows on the interior cells) agrees
    # with the oracle's to its rounding floor, far below the tolerance
    assert abs(gpu_norm - rn) <= 1e-11 * bn
    back = H.average_down(un)
    for q in range(len(un)):
        np.testing.assert_allclose(un[q], back[q], rtol=0, atol=1e-14 * np.abs(back[q]).max())


# margin of exactly one base cell (shell cells on the domain faces), the
# smallest box (2^3 fine cells: its whole grid is the dense coarsest solve)
# and a level-2 box at the smallest margin inside a refined parent (two cells)
EDGE = ((12, 12, 12), [(1, (2, 2, 2), (8, 10, 6)), (1, (14, 14, 16), (2, 2, 2)),
                       (2, (8, 8, 8), (4, 4, 4))])


@pytest.mark.parametrize("precision", [0, 1])
def test_edge_hierarchy_matches_oracle(mg, precision):
    """A box whose grown footprint reaches the domain faces, a 2x2x2 box and
    a level-2 box two cells inside the first: residual cell by cell and the
    solve against the oracle (Dirichlet z faces, variable coefficient)."""
    layout = EDGE
    beta = coefficients(layout, 61, 0.4)
    H = oracle_of(layout, 0.0, beta)
    rho = smooth_source(H, 62)
    rng = np.random.default_rng(63)
    u = [rng.standard_normal(s) for s in shapes_of(layout)]
    A = make(mg, layout, beta, precision=precision)
    rhs = [cuda(x * oracle.EPS0) for x in rho]
    r, _ = A.residual("poisson", rhs, [cuda(x) for x in u])
    ref, _ = H.residual(rho, u)
    ref = H.average_down(ref)
    scale = max(np.abs(x).max() for x in ref)
    for q in range(len(u)):
        np.testing.assert_allclose(r[q].cpu().numpy(), ref[q], rtol=0, atol=1e-12 * scale)
    sol = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in shapes_of(layout)]
    st = A.solve("poisson", rhs, sol, tol=TOL)
    A.close()
    assert st["converged"]
    assert H.rel_l2([t.cpu().numpy() for t in sol], H.solve(rho)) <= PARITY


def test_zero_problem_takes_no_iteration(mg):
    """b = 0 and a zero guess: converged before any iteration, u stays 0."""
    A = make(mg, TWO, None, bc=NEUMANN)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in A.shapes]
    st = A.solve("screened", [torch.zeros_like(t) for t in u], u, tol=TOL, param=3.0)
    A.close()
    assert st["cycles"] == 0 and st["converged"]
    assert all(bool((t == 0).all()) for t in u)


def test_nonfinite_input_is_reported(mg):
    A = make(mg, TWO, None, bc=NEUMANN)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in A.shapes]
    f = [torch.ones_like(t) for t in u]
    f[1][3, 4, 5] = float("nan")
    with pytest.raises(mg.MGError) as e:
        A.solve("screened", f, u, tol=TOL, param=3.0)
    A.close()
    assert e.value.status == mg.MG_ERR_NONFINITE


def test_iteration_cap_reports_not_converged_with_stats(mg):
    """max_cycles = 2: status not converged, two iterations, a decreasing
    history, and the iterate of the last iteration returned."""
    H = oracle_of(TWO, 5.0, None, bc=NEUMANN)
    f = smooth_source(H, 71)
    A = make(mg, TWO, None, bc=NEUMANN, max_cycles=2)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in A.shapes]
    st = A.solve("screened", [cuda(x) for x in f], u, tol=TOL, param=5.0,
                 raise_on_nonconvergence=False)
    A.close()
    assert not st["converged"] and st["cycles"] == 2
    h = st["hist"]
    assert len(h) == 3 and h[0] == 1.0 and h[2] < h[1] < h[0]
    _, rn = H.residual(f, [t.cpu().numpy() for t in u])
    assert abs(rn / H.rhs_norm(f) - st["rel_resid"]) <= 1e-6 * st["rel_resid"]
