"""GPU tests of mg_efield (E = -grad phi and the relaxation time
eps0 |E| / |J| of Sec. 1) against the numpy oracle."""
import numpy as np
import pytest

from oracle import efield as EF
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


@pytest.mark.parametrize("shape", [(32, 32, 32), (20, 36, 52), (8, 8, 296)])
def test_efield_and_relaxation_time_match_oracle(mg, shape):
    """Gap boundary conditions, a needle electrode, a current density with a
    hole (|J| = 0 cells are skipped); several x extents (ragged thread
    blocks)."""
    rng = np.random.default_rng(sum(shape))
    nz, ny, nx = shape
    h = 1.0 / max(shape)
    phi = rng.standard_normal(shape) + np.linspace(0, 1, nz)[:, None, None]
    mask = np.zeros(shape, dtype=np.uint8)
    mask[nz // 2:, ny // 3:ny // 3 + 2, nx // 2:nx // 2 + 3] = 1
    phi[mask != 0] = 1.0
    J = rng.standard_normal((3,) + shape) * 1e-9
    J[:, : nz // 4] = 0.0
    s = mg.Solver(shape, h, mask=cuda(mask), mask_value=cuda(mask.astype(np.float64)),
                  bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE)
    E = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    dt = s.efield(cuda(phi), cuda(J), E)
    s.close()
    E_ref = EF.efield(phi, h, W.GAP_BC_KIND, W.GAP_BC_VALUE, mask)
    np.testing.assert_allclose(E.cpu().numpy(), E_ref, rtol=1e-14, atol=1e-12)
    # the ratio is formed in FP32 on the GPU
    assert dt == pytest.approx(EF.relaxation_time(E_ref, J, mask), rel=2e-6)


def test_efield_without_current_and_zero_current(mg):
    n = 16
    h = 1.0 / n
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((n, n, n))
    s = mg.Solver((n, n, n), h)
    E = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    assert s.efield(cuda(phi), None, E) is None
    np.testing.assert_allclose(E.cpu().numpy(),
                               EF.efield(phi, h, W.GAP_BC_KIND, W.GAP_BC_VALUE),
                               rtol=1e-14, atol=1e-12)
    assert s.efield(cuda(phi), torch.zeros((3, n, n, n), dtype=torch.float64,
                                           device="cuda")) == float("inf")
    s.close()


def test_efield_of_a_solved_potential(mg):
    """After a 64^3 Poisson solve (streamer shell, dielectric slab), the GPU
    field of the GPU potential equals the oracle's field of that potential,
    and the relaxation time of a synthetic conduction current J = sigma E
    with sigma = 1e-3 eps0 is 1000 s wherever |E| > 0."""
    n = 64
    h = 1.0 / n
    rho = W.streamer_shell(n, 1)
    eps = W.dielectric_slab(n)
    s = mg.Solver((n, n, n), h, eps_r=cuda(eps), precision=1)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    s.solve_poisson(cuda(rho), phi, 1e-10)
    E = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    s.efield(phi, None, E)
    J = E * (1e-3 * EF.EPS0)
    dt = s.efield(phi, J)
    s.close()
    E_ref = EF.efield(phi.cpu().numpy(), h, W.GAP_BC_KIND, W.GAP_BC_VALUE)
    np.testing.assert_allclose(E.cpu().numpy(), E_ref, rtol=1e-13, atol=1e-10)
    assert dt == pytest.approx(1000.0, rel=1e-5)
