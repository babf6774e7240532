"""One multigrid cycle on the GPU against one cycle of the oracle.

A converged solve only shows that the answer is right; inside the mixed
path the FP32 V-cycle is a preconditioner, so a wrong weight in a smoother,
restriction or prolongation kernel would only slow convergence down.  These
tests stop both sides after exactly one cycle from a zero guess (tol = 0,
max_cycles = 1, one inner cycle), where the GPU iterate is the V-cycle's
output itself:

  * FP64 path: the same V(nu1, nu2) cycle as the oracle (Sec. 2's red-black
    Gauss-Seidel, 8-child restriction, trilinear prolongation, exact coarsest
    solve), equal to rounding;
  * mixed path: the FP32 V-cycle applied to the FP64 residual, equal to the
    oracle's FP64 cycle to FP32 rounding (the tolerance below; a dropped or
    misplaced stencil weight moves the result by 1e-3 or more).

Several (nu1, nu2) pairs (both >= 1: an option value of 0 selects the
default, 2) and shapes that reach odd coarse extents (a coarse level of
5 x 6 x 4 cells under an even one, hence odd packed widths).
"""
import numpy as np
import pytest

import oracle
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12
FP32_TOL = 2e-5
NUS = [(2, 2), (1, 1), (3, 1), (1, 3)]


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


def blobs(shape, seed):
    """Smooth random charge on a box of the given (nz, ny, nx) shape."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = [(np.arange(m) + 0.5) / m for m in (nz, ny, nx)]
    rho = np.zeros(shape)
    for _ in range(4):
        c = rng.uniform(0.2, 0.8, 3)
        a = rng.standard_normal()
        rho += a * np.exp(-((z[:, None, None] - c[2]) ** 2 + (y[None, :, None] - c[1]) ** 2
                            + (x[None, None, :] - c[0]) ** 2) / (2 * 0.08**2))
    return rho * W.EPS0


def one_cycle_gpu(mg, prec, shape, h, nu, rho=None, eps=None, mask=None, mask_value=None,
                  kappa=None, S=None, bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE,
                  alpha=None, rte_bc=0, coarse_op=1, visits=1):
    """One cycle on the GPU.  coarse_op defaults to the cell rule
    (MG_COARSE_CELL) and visits to one V-cycle on the first coarse level, the
    oracle's V-cycle, so that the cycle can be compared with the oracle's."""
    s = mg.Solver(shape, h, eps_r=cuda(eps), mask=cuda(mask), mask_value=cuda(mask_value),
                  bc_kind=bc_kind, bc_value=bc_value, precision=prec, nu1=nu[0], nu2=nu[1],
                  max_cycles=1, inner_cycles=1, rte_bc=rte_bc, coarse_op=coarse_op)
    s.set_options(coarse_visits=visits)
    try:
        if alpha is not None:
            u = torch.zeros(shape, dtype=torch.float64, device="cuda")
            st = s.solve_screened(alpha, cuda(rho), u, 0.0, raise_on_nonconvergence=False)
            assert st["cycles"] == 1
            return u.cpu().numpy()
        if kappa is None:
            u = torch.zeros(shape, dtype=torch.float64, device="cuda")
            st = s.solve_poisson(cuda(rho), u, 0.0, raise_on_nonconvergence=False)
            assert st["cycles"] == 1
            return u.cpu().numpy()
        psi = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        st = s.solve_helmholtz_batch(cuda(S), psi, kappa, 0.0, raise_on_nonconvergence=False)
        assert all(x["cycles"] == 1 for x in st)
        return [p.cpu().numpy() for p in psi]
    finally:
        s.close()


def one_cycle_oracle(prob, f, nu, u0=None):
    u, cyc, _, _ = prob.solve(f, u0=u0, tol=0.0, max_cycles=1, nu1=nu[0], nu2=nu[1])
    assert cyc == 1
    return u


def check(got, ref, prec):
    err = oracle.rel_l2(got, ref)
    assert err <= (FP64_TOL if prec == 0 else FP32_TOL), err


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nu", NUS)
def test_one_cycle_poisson_slab(mg, prec, nu):
    """Variable permittivity, gap boundary conditions, a non-cubic box whose
    hierarchy is 32x48x40 -> 16x24x20 -> 8x12x10 -> 4x6x5 (x, y, z)."""
    shape = (40, 48, 32)
    h = 1.0 / 48
    rho = blobs(shape, 3)
    eps = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.3)
    got = one_cycle_gpu(mg, prec, shape, h, nu, rho=rho, eps=eps)
    p = oracle.Problem(shape, h, 0.0, eps, None, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    check(got, one_cycle_oracle(p, rho / oracle.EPS0, nu), prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nu", [(2, 2), (3, 1)])
def test_one_cycle_odd_coarse_width(mg, prec, nu):
    """40 x 48 x 32 (x, y, z): the coarsest level has 5 cells along x, so the
    level above it has an odd packed width (5 per colour and row)."""
    shape = (32, 48, 40)
    h = 1.0 / 48
    rho = blobs(shape, 4)
    eps = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.25)
    bc_kind = (0, 1, 1, 0, 0, 0)
    bc_value = (0.2, 0.0, 0.0, -0.3, 0.0, 1.0)
    got = one_cycle_gpu(mg, prec, shape, h, nu, rho=rho, eps=eps, bc_kind=bc_kind,
                        bc_value=bc_value)
    p = oracle.Problem(shape, h, 0.0, eps, None, bc_kind, bc_value)
    check(got, one_cycle_oracle(p, rho / oracle.EPS0, nu), prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nu", [(2, 2), (1, 3)])
def test_one_cycle_electrode(mg, prec, nu):
    """Needle electrode at potential 1 (masked cells) in the gap."""
    n = 32
    h = 1.0 / n
    mask = W.needle_mask(n, tip_z=0.6, tip_radius_cells=3.0)
    mv = mask.astype(np.float64)
    rho = blobs((n, n, n), 5)
    eps = W.dielectric_slab(n)
    got = one_cycle_gpu(mg, prec, (n, n, n), h, nu, rho=rho, eps=eps, mask=mask, mask_value=mv)
    p = oracle.Problem((n, n, n), h, 0.0, eps, mask, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    u0 = np.where(mask != 0, mv, 0.0)
    check(got, one_cycle_oracle(p, rho / oracle.EPS0, nu, u0=u0), prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nu", [(2, 2), (1, 1), (3, 1)])
def test_one_cycle_helmholtz(mg, prec, nu):
    """Constant-coefficient screened Poisson (all-Dirichlet, zero data), the
    three photon groups of one source."""
    shape = (32, 24, 40)
    h = 1.0 / 40
    S = np.abs(blobs(shape, 6)) / W.EPS0
    kap = W.helmholtz_kappas()
    got = one_cycle_gpu(mg, prec, shape, h, nu, kappa=kap, S=S)
    for g, k in zip(got, kap):
        check(g, one_cycle_oracle(oracle.helmholtz(shape, h, k), S, nu), prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nu", [(2, 2), (1, 3)])
def test_one_cycle_screened(mg, prec, nu):
    """Variable coefficient and alpha > 0 together (mg_solve_screened), Neumann
    on the sides and Dirichlet data on z."""
    shape = (24, 32, 40)
    h = 1.0 / 40
    f = blobs(shape, 7) / W.EPS0
    beta = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.3) * (
        1.0 + 0.5 * np.random.default_rng(8).random(shape))
    got = one_cycle_gpu(mg, prec, shape, h, nu, rho=f, eps=beta, alpha=400.0)
    p = oracle.Problem(shape, h, 400.0, beta, None, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    check(got, one_cycle_oracle(p, f, nu), prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nu", [(2, 2), (1, 1)])
def test_one_cycle_marshak(mg, prec, nu):
    """Robin (Marshak) faces on every level: the face factor and the
    prolongation ghost follow each level's h."""
    shape = (32, 24, 40)
    h = 1.0 / 40
    S = np.abs(blobs(shape, 9)) / W.EPS0
    kap = W.helmholtz_kappas()
    got = one_cycle_gpu(mg, prec, shape, h, nu, kappa=kap, S=S, rte_bc=1)
    for g, k in zip(got, kap):
        check(g, one_cycle_oracle(oracle.helmholtz(shape, h, k, marshak=True), S, nu), prec)


# ---- the finest level at a width that takes the staged half-sweep ---------
#
# Levels whose packed width W = nx / 2 is at least 128 run the half-sweep
# whose planes arrive in shared memory by tensor copies (tiles of 128 packed
# entries x 8 rows, 32 planes per CTA).  264 x 20 x 40 cells (x, y, z): W =
# 132, so the second x-tile holds one active quad and its halo lies past the
# level's edge; 20 rows end in a half-empty row tile; 40 planes are a chunk of
# 32 and one of 8.  The level below (W = 66) runs the register-fed kernel.

TMA_SHAPE = (40, 20, 264)


@pytest.mark.parametrize("nu", [(2, 2), (2, 1)])
def test_one_cycle_staged_sweep_poisson_slab_electrode(mg, nu):
    """Variable permittivity and an electrode block that reaches into the
    last x-tile: the FP32 cycle equals the oracle's FP64 cycle to FP32
    rounding."""
    shape = TMA_SHAPE
    nz, ny, nx = shape
    h = 1.0 / nx
    rho = blobs(shape, 31)
    eps = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.07)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[18:27, 6:13, 250:262] = 1
    mv = np.where(mask != 0, 0.5, 0.0)
    got = one_cycle_gpu(mg, 1, shape, h, nu, rho=rho, eps=eps, mask=mask, mask_value=mv)
    p = oracle.Problem(shape, h, 0.0, eps, mask, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    check(got, one_cycle_oracle(p, rho / oracle.EPS0, nu, u0=mv), 1)


@pytest.mark.parametrize("nu", [(2, 2), (1, 1)])
def test_one_cycle_staged_sweep_helmholtz(mg, nu):
    """Constant coefficient (the staged kernel without coefficient arrays)."""
    shape = TMA_SHAPE
    h = 1.0 / shape[2]
    S = np.abs(blobs(shape, 32)) / W.EPS0
    kap = W.helmholtz_kappas()
    got = one_cycle_gpu(mg, 1, shape, h, nu, kappa=kap, S=S)
    for g, k in zip(got, kap):
        check(g, one_cycle_oracle(oracle.helmholtz(shape, h, k), S, nu), 1)


@pytest.mark.parametrize("zchunk", [0, -1, 8, 16, 32])
def test_staged_sweep_converges_to_oracle(mg, zchunk):
    """The same box solved to 1e-10 in mixed precision with the slab, the
    electrode and Neumann sides, for every settable sweep_zchunk (0
    automatic, -1 the register-fed kernel, 8 / 16 / 32 planes per CTA: 40
    planes leave a ragged last chunk for each): within 1e-9 of the oracle's
    answer."""
    shape = TMA_SHAPE
    nz, ny, nx = shape
    h = 1.0 / nx
    rho = blobs(shape, 33)
    eps = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.07)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[18:27, 6:13, 250:262] = 1
    mv = np.where(mask != 0, 0.5, 0.0)
    bc_kind = (1, 1, 1, 1, 0, 0)
    bc_value = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    s = mg.Solver(shape, h, eps_r=cuda(eps), mask=cuda(mask), mask_value=cuda(mv),
                  bc_kind=bc_kind, bc_value=bc_value, precision=1)
    s.set_options(sweep_zchunk=zchunk)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st = s.solve_poisson(cuda(rho), u, 1e-10)
    s.close()
    assert st["converged"]
    p = oracle.Problem(shape, h, 0.0, eps, mask, bc_kind, bc_value)
    ref, _, rel, _ = p.solve(rho / oracle.EPS0, u0=mv, tol=1e-13)
    assert rel < 1e-12
    assert oracle.rel_l2(u.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("ir_zchunk", [0, 16, 32, 128])
def test_staged_refinement_helmholtz_converges_to_oracle(mg, ir_zchunk):
    """The three Helmholtz problems of the staged-sweep box solved to 1e-10:
    their refinement steps run the two-cell pass whose planes arrive by
    tensor copies (5 CTA columns of 60 cells over 264, the last with 24;
    2 row tiles of 14 over 20; chunks of 8, 16, 40 or the automatic run over
    40 planes).  Each answer within 1e-9 of the oracle's."""
    shape = TMA_SHAPE
    h = 1.0 / shape[2]
    S = np.abs(blobs(shape, 34)) / W.EPS0
    kap = W.helmholtz_kappas()
    s = mg.Solver(shape, h, precision=1, nu1=2, nu2=1, inner_cycles=2)
    s.set_options(ir_zchunk=ir_zchunk)
    psi = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    st = s.solve_helmholtz_batch(cuda(S), psi, kap, 1e-10)
    s.close()
    assert all(x["converged"] and x["cycles"] >= 2 for x in st)
    for p, k in zip(psi, kap):
        ref, _, rel, _ = oracle.helmholtz(shape, h, k).solve(S, tol=1e-13)
        assert rel < 1e-12
        assert oracle.rel_l2(p.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("ir_zchunk", [0, 16, 128])
def test_staged_refinement_poisson_converges_to_oracle(mg, ir_zchunk):
    """The Poisson problem of the staged-sweep box (slab, electrode block in
    the last x-tile, Neumann sides) solved to 1e-10: its refinement steps run
    the one-cell face-array pass whose planes arrive by tensor copies (9 CTA
    columns of 30 cells over 264, the last with 24; 2 row tiles of 14 over
    20; chunks of 10, 16 with a ragged 8, or all 40 planes).  Within 1e-9 of
    the oracle's answer."""
    shape = TMA_SHAPE
    nz, ny, nx = shape
    h = 1.0 / nx
    rho = blobs(shape, 36)
    eps = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.07)
    mask = np.zeros(shape, dtype=np.uint8)
    mask[18:27, 6:13, 250:262] = 1
    mv = np.where(mask != 0, 0.5, 0.0)
    bc_kind = (1, 1, 1, 1, 0, 0)
    bc_value = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    s = mg.Solver(shape, h, eps_r=cuda(eps), mask=cuda(mask), mask_value=cuda(mv),
                  bc_kind=bc_kind, bc_value=bc_value, precision=1, nu1=2, nu2=1,
                  inner_cycles=2)
    s.set_options(ir_zchunk=ir_zchunk)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st = s.solve_poisson(cuda(rho), u, 1e-10)
    s.close()
    assert st["converged"] and st["cycles"] >= 2
    p = oracle.Problem(shape, h, 0.0, eps, mask, bc_kind, bc_value)
    ref, _, rel, _ = p.solve(rho / oracle.EPS0, u0=mv, tol=1e-13)
    assert rel < 1e-12
    assert oracle.rel_l2(u.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("shape", [(24, 16, 64), (20, 24, 72)])
def test_staged_poisson_refinement_smallest_boxes(mg, shape):
    """The staged face-array refinement step at the smallest planes it takes
    (64 x 16: three CTA columns of 30 cells, the last with 4; two row tiles
    of 14, the last with 2) and at 72 x 24 (columns of 30, 30, 12; rows of
    14 and 10), with the slab and Neumann sides: within 1e-9 of the oracle.
    (Sizes whose halvings reach a coarsest level of at most 4096 cells.)"""
    nz, ny, nx = shape
    h = 1.0 / nx
    rho = blobs(shape, 39)
    eps = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.3 * nz * h)
    bc_kind = (1, 1, 1, 1, 0, 0)
    bc_value = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    s = mg.Solver(shape, h, eps_r=cuda(eps), bc_kind=bc_kind, bc_value=bc_value,
                  precision=1, nu1=2, nu2=1, inner_cycles=2)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    st = s.solve_poisson(cuda(rho), u, 1e-10)
    s.close()
    assert st["converged"] and st["cycles"] >= 2
    p = oracle.Problem(shape, h, 0.0, eps, None, bc_kind, bc_value)
    ref, _, rel, _ = p.solve(rho / oracle.EPS0, tol=1e-13)
    assert rel < 1e-12
    assert oracle.rel_l2(u.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("shape", [(16, 16, 128), (16, 20, 136)])
def test_staged_helmholtz_refinement_smallest_boxes(mg, shape):
    """The staged two-cell refinement step at the smallest planes it takes
    (128 x 16: three CTA columns of 60 cells, the last with 8; two row tiles)
    and at 136 x 20 (columns of 60, 60, 16; rows of 14 and 6): each of the
    three Helmholtz answers within 1e-9 of the oracle's."""
    h = 1.0 / shape[2]
    S = np.abs(blobs(shape, 40)) / W.EPS0
    kap = W.helmholtz_kappas()
    s = mg.Solver(shape, h, precision=1, nu1=2, nu2=1, inner_cycles=2)
    psi = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    st = s.solve_helmholtz_batch(cuda(S), psi, kap, 1e-10)
    s.close()
    assert all(x["converged"] and x["cycles"] >= 2 for x in st)
    for p, k in zip(psi, kap):
        ref, _, rel, _ = oracle.helmholtz(shape, h, k).solve(S, tol=1e-13)
        assert rel < 1e-12
        assert oracle.rel_l2(p.cpu().numpy(), ref) <= 1e-9


@pytest.mark.parametrize("nu", [(2, 1), (1, 1)])
def test_stacked_helmholtz_matches_oracle_and_unstacked(mg, nu):
    """The three Helmholtz problems of one context run their FP32 V-cycles
    stacked along z (one launch per level step for all three; the problems
    converge after different numbers of steps, so the stack runs on with
    fewer members).  On the staged-sweep box (levels of 40, 20, 10 planes)
    each answer is within 1e-9 of the oracle's, the same problems solved one
    by one (stack off) agree with it, and the stacked solve launches fewer
    kernels."""
    shape = TMA_SHAPE
    h = 1.0 / shape[2]
    S = np.abs(blobs(shape, 35)) / W.EPS0
    kap = W.helmholtz_kappas()
    out, launches, steps = {}, {}, {}
    for no_stack in (0, 1):
        s = mg.Solver(shape, h, precision=1, nu1=nu[0], nu2=nu[1], inner_cycles=3)
        s.set_options(stack=1 - no_stack)
        psi = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        s.solve_helmholtz_batch(cuda(S), psi, kap, 1e-10)  # graphs, coarse inverses
        for p in psi:
            p.zero_()
        torch.cuda.synchronize()
        l0 = mg.launch_count()
        st = s.solve_helmholtz_batch(cuda(S), psi, kap, 1e-10)
        torch.cuda.synchronize()
        launches[no_stack] = mg.launch_count() - l0
        s.close()
        assert all(x["converged"] for x in st)
        out[no_stack] = [p.cpu().numpy() for p in psi]
        steps[no_stack] = [x["cycles"] for x in st]
    for j, k in enumerate(kap):
        ref, _, rel, _ = oracle.helmholtz(shape, h, k).solve(S, tol=1e-13)
        assert rel < 1e-12
        for no_stack in (0, 1):
            assert oracle.rel_l2(out[no_stack][j], ref) <= 1e-9, (j, no_stack)
    assert launches[0] < launches[1], (launches, steps)


# ---- the face-rule coarse operator (MG_COARSE_FACE, the default) ----------
#
# Its coarse faces are built from the finer level's face weights (series along
# the face normal, parallel across), which the oracle's cycle does not use.
# Where the coefficient is constant the rule gives the oracle's coarse
# operator, so one cycle equals the oracle's; elsewhere the FP32 face kernels
# (mg_faces32.cu) are checked against the FP64 natural-layout kernels, which
# read the same FP64 face weights, and the converged answers against the
# oracle (the parity tests, which run with the default rule).


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nu", [(2, 2), (2, 1)])
def test_face_rule_constant_coefficient_equals_oracle_cycle(mg, prec, nu):
    """eps_r = 2.5 everywhere, gap faces: the face rule's coarse faces are the
    cell rule's, so one cycle matches the oracle's."""
    shape = (40, 48, 32)
    h = 1.0 / 48
    rho = blobs(shape, 13)
    eps = np.full(shape, 2.5)
    got = one_cycle_gpu(mg, prec, shape, h, nu, rho=rho, eps=eps, coarse_op=0)
    p = oracle.Problem(shape, h, 0.0, eps, None, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    check(got, one_cycle_oracle(p, rho / oracle.EPS0, nu), prec)


@pytest.mark.parametrize("visits", [1, 2])
@pytest.mark.parametrize("case", ["slab", "electrode", "odd", "screened"])
def test_face_rule_fp32_cycle_matches_fp64_cycle(mg, case, visits):
    """One mixed-precision cycle (FP32 split face kernels on the coarse
    levels) against one FP64 cycle (natural-layout FP64 kernels on the same
    face-rule operators), within FP32 rounding: a slab not aligned with the
    coarse cells, a needle electrode with a dielectric, an odd coarse packed
    width (40 x 48 x 32 -> 5 x 6 x 4) and the screened problem."""
    nu = (2, 1)
    kw = {}
    if case == "slab":
        shape, h = (40, 48, 32), 1.0 / 48
        rho = blobs(shape, 14)
        kw["eps"] = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.37)
    elif case == "electrode":
        n = 32
        shape, h = (n, n, n), 1.0 / n
        mask = W.needle_mask(n, tip_z=0.6, tip_radius_cells=3.0)
        kw.update(eps=W.dielectric_slab(n, z_top=0.33), mask=mask,
                  mask_value=mask.astype(np.float64))
        rho = blobs(shape, 15)
    elif case == "odd":
        shape, h = (32, 48, 40), 1.0 / 48
        rho = blobs(shape, 16)
        kw["eps"] = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.29) * (
            1.0 + np.random.default_rng(17).random(shape))
        kw.update(bc_kind=(0, 1, 1, 0, 0, 0), bc_value=(0.2, 0.0, 0.0, -0.3, 0.0, 1.0))
    else:
        shape, h = (24, 32, 40), 1.0 / 40
        rho = blobs(shape, 18) / W.EPS0
        kw["eps"] = W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.31) * (
            1.0 + 0.5 * np.random.default_rng(19).random(shape))
        kw["alpha"] = 400.0
    u64 = one_cycle_gpu(mg, 0, shape, h, nu, rho=rho, coarse_op=0, visits=visits, **kw)
    u32 = one_cycle_gpu(mg, 1, shape, h, nu, rho=rho, coarse_op=0, visits=visits, **kw)
    mask = kw.get("mask")
    assert oracle.rel_l2(u32, u64, mask) <= FP32_TOL
    # and the face rule (and the second visit) really change the cycle here
    ucell = one_cycle_gpu(mg, 0, shape, h, nu, rho=rho, coarse_op=1, **kw)
    assert oracle.rel_l2(ucell, u64, mask) > 10 * FP32_TOL
    if visits == 2:
        uv1 = one_cycle_gpu(mg, 0, shape, h, nu, rho=rho, coarse_op=0, visits=1, **kw)
        assert oracle.rel_l2(uv1, u64, mask) > 10 * FP32_TOL


def test_face_rule_converges_faster_on_the_slab(mg):
    """The reason for the face rule and for the second cycle on the first
    coarse level: on the dielectric slab (eps_r = 4 below z = 0.2, an
    interface inside coarse cells from the second coarse level on) FP64
    V(2,1)-cycles from zero reach 1e-10 in fewer cycles with the face rule
    than with the cell rule, and in fewer still with two visits to the first
    coarse level; every answer meets 1e-10 by the oracle's residual."""
    n = 128
    h = 1.0 / n
    rho = W.streamer_shell(n, 0)
    eps = W.dielectric_slab(n)
    out, cyc = {}, {}
    for rule, visits in ((0, 1), (1, 1), (0, 2)):
        s = mg.Solver((n, n, n), h, eps_r=cuda(eps), precision=0, nu1=2, nu2=1,
                      coarse_op=rule)
        s.set_options(coarse_visits=visits)
        u = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
        st = s.solve_poisson(cuda(rho), u, 1e-10)
        s.close()
        out[(rule, visits)], cyc[(rule, visits)] = u.cpu().numpy(), st["cycles"]
    assert cyc[(0, 2)] < cyc[(0, 1)] < cyc[(1, 1)], cyc
    P = oracle.poisson((n, n, n), h, eps_r=eps)
    f = rho / oracle.EPS0
    bn = P.rhs_norm(f, np.zeros((n, n, n)))
    for u in out.values():
        assert P.residual(f, u)[1] <= 1.01e-10 * bn
