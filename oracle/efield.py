"""Plain numpy reference of the electric field and the dielectric relaxation
time (TEST INFRASTRUCTURE ONLY: used by tests/ and nothing else).

E = -grad phi at cell centres by centred differences: per axis
(phi(c - 1) - phi(c + 1)) / (2h), where outside the box phi is the face ghost
of the boundary condition (Dirichlet value g: 2g - phi_c; Neumann: phi_c), the
same ghost the discrete operator of Eq. 2 uses (Sec. 2 items (ii)-(iii)).
Electrode cells get E = 0.  The relaxation time of Sec. 1 is
Delta t_E = eps0 |E| / |J|, minimised over the free cells with |J| > 0.

Arrays are (nz, ny, nx); faces are -x, +x, -y, +y, -z, +z.  Pinned by
tests/test_efield_oracle_pins.py (linear and quadratic potentials, brute-force
loops on a small box).
"""
import numpy as np

EPS0 = 8.8541878128e-12


def _padded(phi, bc_kind, bc_value):
    """phi with one ghost layer per face (corners unused)."""
    nz, ny, nx = phi.shape
    p = np.zeros((nz + 2, ny + 2, nx + 2))
    p[1:-1, 1:-1, 1:-1] = phi
    faces = [
        (np.s_[1:-1, 1:-1, 0], phi[:, :, 0]), (np.s_[1:-1, 1:-1, -1], phi[:, :, -1]),
        (np.s_[1:-1, 0, 1:-1], phi[:, 0, :]), (np.s_[1:-1, -1, 1:-1], phi[:, -1, :]),
        (np.s_[0, 1:-1, 1:-1], phi[0, :, :]), (np.s_[-1, 1:-1, 1:-1], phi[-1, :, :]),
    ]
    for f, (sl, inner) in enumerate(faces):
        p[sl] = 2.0 * bc_value[f] - inner if bc_kind[f] == 0 else inner
    return p


def efield(phi, h, bc_kind, bc_value, mask=None):
    """(Ex, Ey, Ez) as an array of shape (3, nz, ny, nx)."""
    phi = np.asarray(phi, dtype=np.float64)
    p = _padded(phi, bc_kind, bc_value)
    ex = (p[1:-1, 1:-1, :-2] - p[1:-1, 1:-1, 2:]) / (2 * h)
    ey = (p[1:-1, :-2, 1:-1] - p[1:-1, 2:, 1:-1]) / (2 * h)
    ez = (p[:-2, 1:-1, 1:-1] - p[2:, 1:-1, 1:-1]) / (2 * h)
    E = np.stack([ex, ey, ez])
    if mask is not None:
        E[:, mask != 0] = 0.0
    return E


def relaxation_time(E, J, mask=None):
    """min over free cells with |J| > 0 of eps0 |E| / |J| (inf if none)."""
    en = np.sqrt((E ** 2).sum(axis=0))
    jn = np.sqrt((np.asarray(J) ** 2).sum(axis=0))
    ok = jn > 0
    if mask is not None:
        ok &= mask == 0
    if not ok.any():
        return np.inf
    return float((EPS0 * en[ok] / jn[ok]).min())
