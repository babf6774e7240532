"""GPU tests of the variable-coefficient screened solve
alpha u - div(beta grad u) = f (mg_solve_screened): one factor (I - mu L) of
the semi-implicit diffusion advance of Sec. 2.2 (alpha = 1/mu, beta = the
diffusion coefficient), against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARITY = 1e-9
TOL = 1e-10
NEUMANN = (1,) * 6


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


def smooth_field(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = [(np.arange(m) + 0.5) / m for m in (nz, ny, nx)]
    out = np.zeros(shape)
    for _ in range(5):
        c = rng.uniform(0.15, 0.85, 3)
        out += rng.uniform(0.5, 2.0) * np.exp(
            -((z[:, None, None] - c[2]) ** 2 + (y[None, :, None] - c[1]) ** 2
              + (x[None, None, :] - c[0]) ** 2) / (2 * 0.07**2))
    return out


def diffusion_coefficient(shape, h, seed):
    """A cell-wise diffusion coefficient: the dielectric-slab jump times a
    lognormal factor per cell."""
    rng = np.random.default_rng(seed)
    return W.dielectric_slab_box(shape, h, (0.0, 0.0, 0.0), z_top=0.35) * np.exp(
        0.3 * rng.standard_normal(shape))


def gpu_screened(mg, shape, h, beta, alpha, f, prec, bc_kind=NEUMANN, bc_value=(0.0,) * 6,
                 mask=None, mask_value=None, u0=None):
    s = mg.Solver(shape, h, eps_r=cuda(beta), mask=cuda(mask), mask_value=cuda(mask_value),
                  bc_kind=bc_kind, bc_value=bc_value, precision=prec)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda") if u0 is None else cuda(u0)
    st = s.solve_screened(alpha, cuda(f), u, TOL)
    s.close()
    return u.cpu().numpy(), st


@pytest.mark.parametrize("prec", [0, 1])
def test_screened_neumann_matches_oracle(mg, prec):
    """Diffusion factor with Neumann faces, a jumping lognormal coefficient,
    alpha = 1/mu for a step mu = 0.4 h^2 / max(beta)."""
    shape = (40, 48, 32)
    h = 1.0 / 48
    beta = diffusion_coefficient(shape, h, 1)
    alpha = 1.0 / (0.4 * h * h / beta.max())
    f = alpha * smooth_field(shape, 2)
    u, st = gpu_screened(mg, shape, h, beta, alpha, f, prec)
    p = oracle.Problem(shape, h, alpha, beta, None, NEUMANN)
    ref, _, rel, _ = p.solve(f)
    assert rel < 1e-12 and st["converged"]
    bn = p.rhs_norm(f, np.zeros(shape))
    assert p.residual(f, u)[1] / bn <= 1.01 * TOL
    assert oracle.rel_l2(u, ref) <= PARITY


@pytest.mark.parametrize("prec", [0, 1])
def test_screened_dirichlet_and_electrode(mg, prec):
    """Gap boundary conditions (Dirichlet values lifted into b) and a needle
    electrode held at 1, small alpha."""
    n = 48
    h = 1.0 / n
    beta = diffusion_coefficient((n, n, n), h, 3)
    mask = W.needle_mask(n, tip_z=0.7, tip_radius_cells=3.0)
    mv = mask.astype(np.float64)
    alpha = 2.0
    f = smooth_field((n, n, n), 4)
    kw = dict(bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE)
    s = mg.Solver((n, n, n), h, eps_r=cuda(beta), mask=cuda(mask), mask_value=cuda(mv),
                  precision=prec, max_cycles=400, **kw)
    u = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    st = s.solve_screened(alpha, cuda(f), u, TOL)
    s.close()
    u = u.cpu().numpy()
    p = oracle.Problem((n, n, n), h, alpha, beta, mask, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    u0 = mv.copy()
    ref, _, rel, _ = p.solve(f, u0=u0)
    assert st["converged"]
    assert oracle.rel_l2(u, ref) <= PARITY
    np.testing.assert_array_equal(u[mask != 0], 1.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_two_factor_diffusion_advance(mg, prec):
    """(I - mu1 L)(I - mu2 L) n = (I + mu3 L) n_dagger (the diffusion advance
    of Sec. 2.2, L = div(D grad)) as two screened solves on the GPU, against
    the same two solves by the oracle; the Neumann advance keeps the total."""
    shape = (32, 32, 48)
    h = 1.0 / 48
    D = diffusion_coefficient(shape, h, 5)
    dt = 2.0 * h * h / D.max()
    a = 2.0 - np.sqrt(2.0)  # TGA: mu1 = mu2 = a dt / 2, mu3 = (1 - a) dt
    mu1 = mu2 = a * dt / 2
    mu3 = (1.0 - a) * dt
    nd = smooth_field(shape, 6)
    lap = -oracle.Problem(shape, h, 0.0, D, None, NEUMANN).apply(nd)
    g = nd + mu3 * lap
    # oracle
    p1 = oracle.Problem(shape, h, 1.0 / mu1, D, None, NEUMANN)
    p2 = oracle.Problem(shape, h, 1.0 / mu2, D, None, NEUMANN)
    y_ref, _, _, _ = p1.solve(g / mu1)
    n_ref, _, _, _ = p2.solve(y_ref / mu2)
    # GPU
    s = mg.Solver(shape, h, eps_r=cuda(D), bc_kind=NEUMANN, precision=prec)
    y = torch.zeros(shape, dtype=torch.float64, device="cuda")
    s.solve_screened(1.0 / mu1, cuda(g / mu1), y, TOL)
    n = torch.zeros_like(y)
    s.solve_screened(1.0 / mu2, y / mu2, n, TOL)
    s.close()
    n = n.cpu().numpy()
    assert oracle.rel_l2(n, n_ref) <= PARITY
    assert abs(n.sum() - nd.sum()) <= 1e-8 * np.abs(nd).sum()


@pytest.mark.parametrize("prec", [0, 1])
def test_screened_in_a_batch(mg, prec):
    """mg_solve_batch with a screened problem next to a Poisson and a
    Helmholtz problem on another grid."""
    shape = (32, 32, 32)
    h = 1.0 / 32
    beta = diffusion_coefficient(shape, h, 7)
    alpha = 30.0
    f = smooth_field(shape, 8)
    s1 = mg.Solver(shape, h, eps_r=cuda(beta), bc_kind=NEUMANN, precision=prec)
    s2 = mg.Solver((16, 24, 32), 1.0 / 32, precision=prec)
    rho = W.gaussian_blobs(32, 3)[:16, :24, :32].copy()
    S = np.abs(rho) / W.EPS0
    us = [torch.zeros(sh, dtype=torch.float64, device="cuda")
          for sh in (shape, (16, 24, 32), (16, 24, 32))]
    st = mg.solve_batch([
        {"solver": s1, "kind": "screened", "alpha": alpha, "rhs": cuda(f), "u": us[0]},
        {"solver": s2, "kind": "poisson", "rhs": cuda(rho), "u": us[1]},
        {"solver": s2, "kind": "helmholtz", "kappa": 10.0, "rhs": cuda(S), "u": us[2]},
    ], tol=TOL)
    s1.close()
    s2.close()
    assert all(x["converged"] for x in st)
    ref, _, _, _ = oracle.Problem(shape, h, alpha, beta, None, NEUMANN).solve(f)
    assert oracle.rel_l2(us[0].cpu().numpy(), ref) <= PARITY
    ref, _, _, _ = oracle.poisson((16, 24, 32), 1.0 / 32).solve(rho / oracle.EPS0)
    assert oracle.rel_l2(us[1].cpu().numpy(), ref) <= PARITY
    ref, _, _, _ = oracle.helmholtz((16, 24, 32), 1.0 / 32, 10.0).solve(S)
    assert oracle.rel_l2(us[2].cpu().numpy(), ref) <= PARITY
