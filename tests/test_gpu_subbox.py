"""GPU tests of refined sub-boxes (the stand-in for the paper's patch-based
grid hierarchy, Sec. 4): Dirichlet face data from the parent solution, and
batched solves of uneven sub-boxes against the FP64 oracle.

The sub-box boundary data is pinned independently by scipy's
RegularGridInterpolator (trilinear on the parent's cell centres); for the
solve parity both sides get the same face array, computed from the oracle's
parent solution.
"""
import numpy as np
import pytest

import oracle
from paper_1809_08857_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PARITY = 1e-9
TOL = 1e-10
ALL_DIR = (0,) * 6


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


def face_points(origin, dims, hp):
    """Physical (z, y, x) coordinates of the boundary face centres of a ratio-2
    sub-box, in the packed face order."""
    nx, ny, nz = dims
    hf = hp / 2
    o = np.array(origin, dtype=np.float64) * hp
    x = o[0] + (np.arange(nx) + 0.5) * hf
    y = o[1] + (np.arange(ny) + 0.5) * hf
    z = o[2] + (np.arange(nz) + 0.5) * hf
    pts = []
    for f in range(6):
        if f < 2:
            Z, Y = np.meshgrid(z, y, indexing="ij")
            X = np.full_like(Z, o[0] + (0 if f == 0 else nx * hf))
        elif f < 4:
            Z, X = np.meshgrid(z, x, indexing="ij")
            Y = np.full_like(Z, o[1] + (0 if f == 2 else ny * hf))
        else:
            Y, X = np.meshgrid(y, x, indexing="ij")
            Z = np.full_like(Y, o[2] + (0 if f == 4 else nz * hf))
        pts.append(np.stack([Z.ravel(), Y.ravel(), X.ravel()], axis=1))
    return np.concatenate(pts)


def interp_faces(parent_u, hp, origin, dims):
    from scipy.interpolate import RegularGridInterpolator

    nz, ny, nx = parent_u.shape
    grid = ((np.arange(nz) + 0.5) * hp, (np.arange(ny) + 0.5) * hp, (np.arange(nx) + 0.5) * hp)
    return RegularGridInterpolator(grid, parent_u, method="linear")(face_points(origin, dims, hp))


def test_subbox_bc_matches_trilinear_interpolation(mg):
    n = 32
    hp = 1.0 / n
    c = (np.arange(n) + 0.5) * hp
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    u = np.sin(3 * X + 1) * np.cos(2 * Y) * np.exp(Z) + X * Y
    s = mg.Solver((n, n, n), hp)
    for origin, dims in [((5, 7, 9), (16, 12, 20)), ((1, 1, 1), (60, 2, 4)), ((20, 3, 12), (8, 8, 8))]:
        got = s.subbox_bc(cuda(u), origin, dims).cpu().numpy()
        ref = interp_faces(u, hp, origin, dims)
        assert got.shape == (mg.face_count(dims[::-1]),)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    with pytest.raises(mg.MGError):
        s.subbox_bc(cuda(u), (0, 3, 3), (8, 8, 8))  # touches the parent face
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_face_data_reproduces_linear_potential(mg, prec):
    """GPU with per-face Dirichlet data: a linear potential is reproduced to
    round-off (the oracle's pin, here on the GPU)."""
    shape = (20, 12, 16)
    h = 0.05
    nz, ny, nx = shape
    lin = lambda x, y, z: 0.3 + 1.1 * x - 2.3 * y + 0.7 * z
    pts = face_points((0, 0, 0), (nx, ny, nz), 2 * h)
    fd = lin(pts[:, 2], pts[:, 1], pts[:, 0])
    Z, Y, X = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h,
                          (np.arange(nx) + 0.5) * h, indexing="ij")
    exact = lin(X, Y, Z)
    s = mg.Solver(shape, h, eps_r=cuda(np.full(shape, 2.5)), bc_kind=ALL_DIR, precision=prec)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    mg.solve_batch([{"solver": s, "kind": "poisson", "rhs": cuda(np.zeros(shape)), "u": u,
                     "faces": cuda(fd)}], tol=1e-13)
    s.close()
    np.testing.assert_allclose(u.cpu().numpy(), exact, rtol=0, atol=1e-11)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_uneven_subboxes_match_oracle(mg, prec):
    """Parent 64^3 Poisson + Helmholtz solves (oracle), then a batch of uneven
    refined sub-boxes (16^3, 24^3, 32^3 fine cells and a non-cubic one), each a
    Poisson and a Helmholtz problem with Dirichlet data interpolated from the
    parent solutions, solved concurrently on the GPU and compared with the
    oracle on the same face data."""
    n = 64
    hp = 1.0 / n
    rho = W.streamer_shell(n, 5)
    eps = W.dielectric_slab(n)
    S = W.ionization_source(n, 5)
    kappa = 100.0
    phi_p, _, _, _ = oracle.poisson((n, n, n), hp, eps_r=eps).solve(rho / oracle.EPS0)
    psi_p, _, _, _ = oracle.helmholtz((n, n, n), hp, kappa).solve(S)
    boxes = [((20, 22, 20), (16, 16, 16)), ((8, 10, 6), (24, 24, 24)),
             ((30, 28, 26), (32, 32, 32)), ((12, 40, 9), (16, 24, 32))]
    solvers, probs, refs = [], [], []
    hf = hp / 2
    for b, (origin, dims) in enumerate(boxes):
        nx, ny, nz = dims
        shape = (nz, ny, nx)
        o = tuple(v * hp for v in origin)
        rho_b = W.streamer_shell_box(shape, hf, o, 10 + b)
        eps_b = W.dielectric_slab_box(shape, hf, o)
        S_b = np.abs(W.streamer_shell_box(shape, hf, o, 20 + b)) / W.EPS0
        fd_phi = interp_faces(phi_p, hp, origin, dims)
        fd_psi = interp_faces(psi_p, hp, origin, dims)
        s = mg.Solver(shape, hf, eps_r=cuda(eps_b), bc_kind=ALL_DIR, precision=prec)
        solvers.append(s)
        uphi = torch.zeros(shape, dtype=torch.float64, device="cuda")
        upsi = torch.zeros(shape, dtype=torch.float64, device="cuda")
        probs.append({"solver": s, "kind": "poisson", "rhs": cuda(rho_b), "u": uphi,
                      "faces": cuda(fd_phi)})
        probs.append({"solver": s, "kind": "helmholtz", "kappa": kappa, "rhs": cuda(S_b),
                      "u": upsi, "faces": cuda(fd_psi)})
        rp, _, _, _ = oracle.Problem(shape, hf, 0.0, eps_b, None, ALL_DIR, (0.0,) * 6,
                                     fd_phi).solve(rho_b / oracle.EPS0)
        rh, _, _, _ = oracle.Problem(shape, hf, kappa**2, None, None, ALL_DIR, (0.0,) * 6,
                                     fd_psi).solve(S_b)
        refs += [rp, rh]
    st = mg.solve_batch(probs, tol=TOL)
    for s in solvers:
        s.close()
    for pr, ref, stt in zip(probs, refs, st):
        assert stt["converged"]
        assert oracle.rel_l2(pr["u"].cpu().numpy(), ref) <= PARITY


def test_config3_parent_set_and_16_subboxes(mg):
    """The full-size sub-box configuration: the Poisson + three Helmholtz set on
    the 256^3 parent, then 16 sub-boxes of sizes drawn from {32, 48, 64, 96,
    128}^3 (ratio 2), each with its Poisson and three Helmholtz problems on
    Dirichlet data interpolated from the parent answers, all 64 solved in one
    batch.  Every sub-box answer meets 1e-10 by the oracle's FP64 residual on
    the same face data; the smallest and the largest box's four answers are
    within 1e-9 of the oracle's converged solutions; the parent answers meet
    1e-10 by the oracle's residual."""
    from paper_1809_08857_gb300 import subboxes

    c = subboxes.Config3(n=256, count=16, seed=0)
    st_parent, st_boxes = c.run()
    torch.cuda.synchronize()
    assert all(x["converged"] for x in st_parent) and all(x["converged"] for x in st_boxes)
    assert sorted({b["dims"][0] for b in c.boxes}) == [32, 48, 64, 96, 128]
    n = c.n
    hp = 1.0 / n
    P = oracle.poisson((n, n, n), hp, eps_r=c.eps.cpu().numpy())
    f = c.rho.cpu().numpy() / oracle.EPS0
    _, rn = P.residual(f, c.phi.cpu().numpy())
    assert rn <= 1.01 * TOL * P.rhs_norm(f, np.zeros((n, n, n)))
    S = c.S.cpu().numpy()
    for k, psi in zip(subboxes.KAPPAS, c.psi):
        H = oracle.helmholtz((n, n, n), hp, k)
        _, rn = H.residual(S, psi.cpu().numpy())
        assert rn <= 1.01 * TOL * H.rhs_norm(S, np.zeros((n, n, n)))
    sizes = [int(np.prod(b["shape"])) for b in c.boxes]
    full = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    hf = hp / 2
    for q, b in enumerate(c.boxes):
        shape = b["shape"]
        rhs = [b["rho"].cpu().numpy() / oracle.EPS0] + [b["S"].cpu().numpy()] * 3
        alphas = [0.0] + [k * k for k in subboxes.KAPPAS]
        betas = [b["eps"], None, None, None]
        for j in range(4):
            fd = b["faces"][j].cpu().numpy()
            Pb = oracle.Problem(shape, hf, alphas[j], betas[j], None, ALL_DIR, (0.0,) * 6, fd)
            u = b["u"][j].cpu().numpy()
            _, rn = Pb.residual(rhs[j], u)
            assert rn <= 1.01 * TOL * Pb.rhs_norm(rhs[j], np.zeros(shape)), (q, j)
            if q in full:
                ref, _, rel, _ = Pb.solve(rhs[j])
                assert rel < 1e-12
                assert oracle.rel_l2(u, ref) <= PARITY, (q, j)
    c.close()
