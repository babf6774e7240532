"""GPU tests of the radiative-transfer solves with the Marshak condition on
the domain faces (mg_options.rte_bc = MG_RTE_BC_MARSHAK): the Robin face
n.grad Psi + (sqrt(3)/2) kappa Psi = 0 of the Eddington closure of Eq. 3,
against the FP64 oracle's Robin faces."""
import numpy as np
import pytest

import oracle
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARITY = 1e-9
TOL = 1e-10


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


@pytest.mark.parametrize("prec", [0, 1])
def test_marshak_batch_matches_oracle(mg, prec):
    """The three photon groups (kappa L = 10, 100, 1000) of the smoothed
    ionisation source at 64^3 on a Marshak context."""
    n = 64
    h = 1.0 / n
    S = W.ionization_source(n, 1)
    s = mg.Solver((n, n, n), h, precision=prec, rte_bc=mg.MG_RTE_BC_MARSHAK)
    psi = [torch.zeros((n, n, n), dtype=torch.float64, device="cuda") for _ in range(3)]
    kap = W.helmholtz_kappas()
    st = s.solve_helmholtz_batch(cuda(S), psi, kap, TOL)
    s.close()
    for p, k, x in zip(psi, kap, st):
        assert x["converged"]
        prob = oracle.helmholtz((n, n, n), h, k, marshak=True)
        ref, _, rel, _ = prob.solve(S)
        assert rel < 1e-12
        got = p.cpu().numpy()
        assert oracle.rel_l2(got, ref) <= PARITY
        bn = prob.rhs_norm(S, np.zeros_like(got))
        assert prob.residual(S, got)[1] / bn <= 1.01 * TOL


@pytest.mark.parametrize("prec", [0, 1])
def test_marshak_differs_from_dirichlet_near_faces(mg, prec):
    """A source touching the faces: the Marshak answer is larger on the
    boundary cells than the Psi = 0 answer (radiation leaves through a
    partially reflecting face), and equal to the oracle's."""
    shape = (32, 40, 48)
    h = 1.0 / 48
    rng = np.random.default_rng(4)
    S = rng.uniform(0.5, 1.5, shape)
    kappa = 10.0
    out = {}
    for bc in (mg.MG_RTE_BC_DIRICHLET, mg.MG_RTE_BC_MARSHAK):
        s = mg.Solver(shape, h, precision=prec, rte_bc=bc)
        psi = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
        s.solve_helmholtz_batch(cuda(S), psi, (kappa,) * 3, TOL)
        s.close()
        out[bc] = psi[0].cpu().numpy()
    ref, _, _, _ = oracle.helmholtz(shape, h, kappa, marshak=True).solve(S)
    assert oracle.rel_l2(out[mg.MG_RTE_BC_MARSHAK], ref) <= PARITY
    m, d = out[mg.MG_RTE_BC_MARSHAK], out[mg.MG_RTE_BC_DIRICHLET]
    assert (m[0] > d[0]).all() and (m[:, :, -1] > d[:, :, -1]).all()


@pytest.mark.parametrize("prec", [0, 1])
def test_marshak_with_electrode_in_a_set(mg, prec):
    """mg_solve_set on a Marshak context with a needle electrode (Psi = 0 on
    its cells) and the dielectric slab for the Poisson problem."""
    n = 48
    h = 1.0 / n
    mask = W.needle_mask(n, tip_z=0.7, tip_radius_cells=3.0)
    eps = W.dielectric_slab(n)
    rho = W.streamer_shell(n, 2)
    S = W.ionization_source(n, 2)
    kap = W.helmholtz_kappas()
    s = mg.Solver((n, n, n), h, eps_r=cuda(eps), mask=cuda(mask),
                  mask_value=cuda(mask.astype(np.float64)), precision=prec, max_cycles=400,
                  rte_bc=mg.MG_RTE_BC_MARSHAK)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    psi = [torch.zeros_like(phi) for _ in range(3)]
    st = s.solve_set(cuda(rho), phi, cuda(S), psi, kap, TOL)
    s.close()
    assert all(x["converged"] for x in st)
    ref, _, _, _ = oracle.poisson((n, n, n), h, eps_r=eps, mask=mask).solve(
        rho / oracle.EPS0, u0=mask.astype(np.float64))
    assert oracle.rel_l2(phi.cpu().numpy(), ref) <= PARITY
    for p, k in zip(psi, kap):
        ref, _, _, _ = oracle.helmholtz((n, n, n), h, k, mask=mask, marshak=True).solve(S)
        assert oracle.rel_l2(p.cpu().numpy(), ref) <= PARITY


def test_marshak_rejects_face_data_and_option_change(mg):
    n = 16
    s = mg.Solver((n, n, n), 1.0 / n, rte_bc=mg.MG_RTE_BC_MARSHAK)
    u = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    faces = torch.zeros(mg.face_count((n, n, n)), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError):
        mg.solve_batch([{"solver": s, "kind": "helmholtz", "kappa": 10.0,
                         "rhs": torch.ones_like(u), "u": u, "faces": faces}])
    with pytest.raises(mg.MGError):
        s.set_options(rte_bc=mg.MG_RTE_BC_DIRICHLET)
    s.close()
