"""GPU test of mg_residual_norm_noalloc, the entry point that allocates no
device memory (its partial sums live in a static device array inside libmg).

It is meant for callers that cannot call cudaMalloc during the call, such as
codes whose device memory is owned by their own pool allocator.  The test
calls it through the C ABI on two calls in a row (so that the shared scratch
array is reused) and checks each result twice: against the FP64 CPU oracle's
own residual norm of the same iterate (an independent operator, lifts and
reduction), and against the residual norms the ordinary solver entry points
report (a solve whose tolerance the initial guess already meets returns the
initial relative residual ||b - A u|| / ||b||).  This file is collected last
on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the solver's first pass sums r^2 one cell per thread, this entry point
# (constant coefficients, even nx, aligned arrays) two cells per thread: the
# same r, FP32 per-thread sums in another order
NORM_RTOL = 1e-6
# against the oracle: r in double-float arithmetic, rounded to FP32 and squared
# and summed per thread in FP32 (about 2^-24 relative per term)
ORACLE_RTOL = 1e-6


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_08857_gb300 import build, mg as _mg

    build.build()
    _mg.load()
    return _mg


def test_noalloc_matches_helmholtz_entry_point(mg):
    n = 64
    h = 1.0 / n
    kappa = 100.0
    S = torch.from_numpy(W.ionization_source(n, 2)).cuda()
    mask_np = W.needle_mask(n, tip_z=0.7, tip_radius_cells=3.0)
    mask = torch.from_numpy(mask_np).cuda()
    rng = np.random.default_rng(8)
    u_np = rng.standard_normal((n, n, n))
    u_np[mask_np == 1] = 0.0
    u = torch.from_numpy(u_np).cuda()
    zero = torch.zeros_like(u)
    kind, val = (0,) * 6, (0.0,) * 6

    solver = mg.Solver((n, n, n), h, mask=mask)
    psi = [u.clone() for _ in range(3)]
    st = solver.solve_helmholtz_batch(S, psi, (kappa, kappa, kappa), tol=1e300)
    solver.close()
    expected = st[0]["rel_resid"]

    P = oracle.helmholtz((n, n, n), h, kappa, mask=mask_np)
    _, rn_ref = P.residual(S.cpu().numpy(), u_np)
    bn_ref = P.rhs_norm(S.cpu().numpy(), np.zeros_like(u_np))

    out_r = torch.empty(1, dtype=torch.float64, device="cuda")
    out_b = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        mg.residual_norm_noalloc(u, S, h, alpha=kappa**2, mask=mask, bc_kind=kind, bc_value=val,
                                 out=out_r)
        mg.residual_norm_noalloc(zero, S, h, alpha=kappa**2, mask=mask, bc_kind=kind,
                                 bc_value=val, out=out_b)
        torch.cuda.synchronize()
        assert out_r.item() == pytest.approx(rn_ref, rel=ORACLE_RTOL)
        assert out_b.item() == pytest.approx(bn_ref, rel=ORACLE_RTOL)
        got = out_r.item() / out_b.item()
        assert got == pytest.approx(expected, rel=NORM_RTOL)


def test_noalloc_matches_poisson_entry_point(mg):
    shape = (48, 40, 24)
    h = 1.0 / 48
    rng = np.random.default_rng(9)
    rho_np = W.EPS0 * rng.standard_normal(shape) * 30
    mask_np = np.zeros(shape, dtype=np.uint8)
    mask_np[30:38, 10:20, 4:12] = 1
    mval_np = np.where(mask_np == 1, 0.75, 0.0)
    u_np = rng.standard_normal(shape)
    u_np[mask_np == 1] = 0.75
    rho = torch.from_numpy(rho_np).cuda()
    mask = torch.from_numpy(mask_np).cuda()
    u = torch.from_numpy(u_np).cuda()
    u0 = torch.from_numpy(mval_np).cuda()

    solver = mg.Solver(shape, h, mask=mask, mask_value=u0.clone(), bc_kind=W.GAP_BC_KIND,
                       bc_value=W.GAP_BC_VALUE)
    phi = u.clone()
    st = solver.solve_poisson(rho, phi, tol=1e300)
    solver.close()
    expected = st["rel_resid"]

    P = oracle.poisson(shape, h, mask=mask_np)
    _, rn_ref = P.residual(rho_np / oracle.EPS0, u_np)
    bn_ref = P.rhs_norm(rho_np / oracle.EPS0, mval_np)

    out_r = torch.empty(1, dtype=torch.float64, device="cuda")
    out_b = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        mg.residual_norm_noalloc(u, rho, h, rhs_scale=1.0 / W.EPS0, mask=mask,
                                 bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE, out=out_r)
        mg.residual_norm_noalloc(u0, rho, h, rhs_scale=1.0 / W.EPS0, mask=mask,
                                 bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE, out=out_b)
        torch.cuda.synchronize()
        assert out_r.item() == pytest.approx(rn_ref, rel=ORACLE_RTOL)
        assert out_b.item() == pytest.approx(bn_ref, rel=ORACLE_RTOL)
        assert out_r.item() / out_b.item() == pytest.approx(expected, rel=NORM_RTOL)


def test_noalloc_rejects_oversized_grid(mg):
    """A residual kernel of more than 16384 thread blocks (partial sums) is
    refused up front, with the count it would need (no kernel runs, so no
    memory is touched)."""
    import ctypes

    lib = mg.load()
    g = mg.Grid(4096, 4096, 1, 1.0, (ctypes.c_double * 3)())
    bc = mg.BC((ctypes.c_int * 6)(*(0,) * 6), (ctypes.c_double * 6)())
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = lib.mg_residual_norm_noalloc(ctypes.byref(g), ctypes.byref(bc), 0.0, dummy, 1.0, None,
                                      dummy, dummy, None)
    assert st == mg.MG_ERR_UNSUPPORTED
    msg = lib.mg_last_error()
    assert b"16384" in msg and b"40141" in msg  # 137 * 293 * 1 blocks
