"""FP64 CPU oracle for the elliptic hot path of arXiv:1809.08857.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

The oracle is a plain multigrid written in C (``mg_oracle.c``) for the
second-order cell-centred discretisation of the Poisson equation (Eq. 2,
generalised to a cell-wise relative permittivity) and of the screened-Helmholtz
radiative-transfer equations (Eq. 3), with red-black Gauss-Seidel smoothing as
named in Sec. 2 item (ii).  It is iterated to its round-off floor so that it
stands for the exact discrete solution.

Arrays are numpy, shape (nz, ny, nx), x fastest.  Faces are ordered
-x, +x, -y, +y, -z, +z; ``bc_kind`` 0 = Dirichlet (value in ``bc_value``),
1 = homogeneous Neumann, 2 = Robin n.grad u + a u = 0 (a in ``bc_value``).

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` (closed-form eigenmode solves, layered-dielectric
and electrode-plane exact solutions, O(h^2) convergence, symmetry, Gauss law,
dense brute force, multigrid step identities).
"""
import ctypes
import os

import numpy as np

from . import build as _build

EPS0 = 8.8541878128e-12  # F/m, CODATA 2018 (the paper prints no value)


class _Grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("h", ctypes.c_double),
        ("bc_kind", ctypes.c_int * 6),
        ("bc_value", ctypes.c_double * 6),
        ("face_data", ctypes.c_void_p),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        G = ctypes.POINTER(_Grid)
        D = ctypes.c_double
        I = ctypes.c_int
        lib.or_residual.argtypes = [G, D, P, P, P, P, P, I]
        lib.or_residual.restype = D
        lib.or_rbgs.argtypes = [G, D, P, P, P, P, I, I]
        lib.or_restrict.argtypes = [G, P, G, P]
        lib.or_prolong_add.argtypes = [G, P, P, G, P, P]
        lib.or_coarsen.argtypes = [G, P, P, G, P, P]
        lib.or_rhs_norm.argtypes = [G, D, P, P, P, P]
        lib.or_rhs_norm.restype = D
        lib.or_solve.argtypes = [G, D, P, P, P, P, D, I, I, I, P, P]
        lib.or_solve.restype = I
        lib.or_apply.argtypes = [G, D, P, P, P, P, I]
        lib.or_num_levels.argtypes = [G]
        lib.or_num_levels.restype = I
        _lib = lib
    return _lib


def grid(shape, h, bc_kind=(0,) * 6, bc_value=(0.0,) * 6, face_data=None):
    """Build the C grid descriptor for an array of shape (nz, ny, nx).
    face_data (optional, numpy float64, packed per face as in ``face_count``)
    gives the Dirichlet value at every boundary face centre; the caller keeps
    the array alive."""
    nz, ny, nx = shape
    g = _Grid()
    g.nx, g.ny, g.nz, g.h = int(nx), int(ny), int(nz), float(h)
    for d in range(6):
        g.bc_kind[d] = int(bc_kind[d])
        g.bc_value[d] = float(bc_value[d])
    g.face_data = None if face_data is None else face_data.ctypes.data
    return g


def face_count(shape):
    """Length of the packed face data: faces -x, +x (ny*nz, index k*ny + j),
    -y, +y (nx*nz, index k*nx + i), -z, +z (nx*ny, index j*nx + i)."""
    nz, ny, nx = shape
    return 2 * (ny * nz + nx * nz + nx * ny)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


class Problem:
    """One discrete elliptic problem L(u) = f (Sec. 2 items (ii)-(iii)).

    alpha: zeroth-order coefficient (0 for Poisson, kappa^2 for Helmholtz).
    beta: cell coefficient (relative permittivity for Poisson, 1 for
    Helmholtz); None means 1 everywhere.
    mask: nonzero marks electrode cells whose value in ``u`` is held fixed.
    """

    def __init__(self, shape, h, alpha=0.0, beta=None, mask=None,
                 bc_kind=(0,) * 6, bc_value=(0.0,) * 6, face_data=None):
        self.shape = tuple(int(s) for s in shape)
        self.h = float(h)
        self.alpha = float(alpha)
        self.beta = _f64(beta)
        self.mask = _u8(mask)
        self.bc_kind = tuple(bc_kind)
        self.bc_value = tuple(bc_value)
        self.face_data = None if face_data is None else _f64(face_data)
        if self.face_data is not None and self.face_data.size != face_count(self.shape):
            raise ValueError("face_data has the wrong length")
        self.g = grid(self.shape, h, bc_kind, bc_value, self.face_data)

    def residual(self, f, u, homog=False):
        """r = f - L(u) on free cells (0 on electrode cells); returns (r, ||r||_2)."""
        lib = _load()
        f, u = _f64(f), _f64(u)
        r = np.empty(self.shape)
        ss = lib.or_residual(ctypes.byref(self.g), self.alpha, _p(self.beta), _p(self.mask),
                             _p(f), _p(u), _p(r), int(homog))
        return r, float(np.sqrt(ss))

    def apply(self, u, homog=False):
        """L(u) on free cells, 0 on electrode cells."""
        lib = _load()
        u = _f64(u)
        out = np.empty(self.shape)
        lib.or_apply(ctypes.byref(self.g), self.alpha, _p(self.beta), _p(self.mask),
                     _p(u), _p(out), int(homog))
        return out

    def rbgs(self, f, u, color, homog=False):
        """One red-black Gauss-Seidel half-sweep (in place on a copy); returns u."""
        lib = _load()
        f = _f64(f)
        u = np.array(u, dtype=np.float64, copy=True)
        lib.or_rbgs(ctypes.byref(self.g), self.alpha, _p(self.beta), _p(self.mask),
                    _p(f), _p(u), int(color), int(homog))
        return u

    def rhs_norm(self, f, u):
        """||b||_2: residual norm of the zero guess (electrode values kept)."""
        lib = _load()
        return lib.or_rhs_norm(ctypes.byref(self.g), self.alpha, _p(self.beta), _p(self.mask),
                               _p(_f64(f)), _p(_f64(u)))

    def solve(self, f, u0=None, tol=1e-13, max_cycles=1000, nu1=2, nu2=2):
        """Multigrid V(nu1,nu2) solve to ``tol`` or to the round-off floor.

        Returns (u, cycles, final relative residual, history)."""
        lib = _load()
        f = _f64(f)
        u = np.zeros(self.shape) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
        hist = np.zeros(max_cycles + 1)
        rel = ctypes.c_double(0.0)
        cyc = lib.or_solve(ctypes.byref(self.g), self.alpha, _p(self.beta), _p(self.mask),
                           _p(f), _p(u), float(tol), int(max_cycles), int(nu1), int(nu2),
                           _p(hist), ctypes.byref(rel))
        if cyc < 0:
            raise RuntimeError("oracle: coarsest-grid factorisation failed (singular operator)")
        return u, cyc, rel.value, hist[: cyc + 1].copy()

    def num_levels(self):
        return _load().or_num_levels(ctypes.byref(self.g))


def restrict(rf, coarse_shape):
    """Coarse value = mean of the 8 fine children."""
    lib = _load()
    rf = _f64(rf)
    out = np.empty(coarse_shape)
    gf, gc = grid(rf.shape, 1.0), grid(coarse_shape, 2.0)
    lib.or_restrict(ctypes.byref(gf), _p(rf), ctypes.byref(gc), _p(out))
    return out


def prolong_add(ec, cmask, bc_kind, uf, fmask=None):
    """uf + trilinear interpolation of the coarse correction ec (homogeneous
    ghosts per bc_kind; masked coarse cells read as zero)."""
    lib = _load()
    ec = _f64(ec)
    uf = np.array(uf, dtype=np.float64, copy=True)
    gc = grid(ec.shape, 2.0, bc_kind)
    gf = grid(uf.shape, 1.0, bc_kind)
    lib.or_prolong_add(ctypes.byref(gc), _p(_u8(cmask)), _p(ec), ctypes.byref(gf),
                       _p(_u8(fmask)), _p(uf))
    return uf


def coarsen(beta_f, mask_f, shape_f):
    """Coarse (beta, mask): masked iff at least 3 of the 8 children are masked,
    beta = mean of the free children."""
    lib = _load()
    nz, ny, nx = shape_f
    cshape = (nz // 2, ny // 2, nx // 2)
    bc = np.empty(cshape)
    mc = np.empty(cshape, dtype=np.uint8)
    lib.or_coarsen(ctypes.byref(grid(shape_f, 1.0)), _p(_f64(beta_f)), _p(_u8(mask_f)),
                   ctypes.byref(grid(cshape, 2.0)), _p(bc), _p(mc))
    return bc, mc


def poisson(shape, h, eps_r=None, mask=None, bc_kind=(1, 1, 1, 1, 0, 0),
            bc_value=(0.0, 0.0, 0.0, 0.0, 0.0, 1.0)):
    """Poisson problem -div(eps_r grad phi) = rho/eps0 (Eq. 2 with a cell-wise
    relative permittivity).  Default BCs: phi = 0 at z = 0, phi = 1 at z = 1,
    homogeneous Neumann on the sides (the needle-plane/rod-plane setting of
    Secs. 3 and 4)."""
    return Problem(shape, h, 0.0, eps_r, mask, bc_kind, bc_value)


def marshak_coefficient(kappa):
    """Robin coefficient a of the Marshak condition n.grad Psi + a Psi = 0 for
    the Helmholtz form (kappa^2 - lap) Psi = S: the paper's Eq. 3 with the
    Eddington closure has n.grad Psi + (3 kappa_p / 2) Psi = 0, and
    kappa = sqrt(3) kappa_p, so a = (sqrt(3)/2) kappa."""
    return 0.5 * np.sqrt(3.0) * float(kappa)


def helmholtz(shape, h, kappa, mask=None, marshak=False):
    """Screened Helmholtz (kappa^2 - lap) Psi = S (Eq. 3 in the form
    kappa^2 Psi - lap Psi = S), Psi = 0 on electrode cells; on every domain
    face Psi = 0, or with marshak=True the Robin condition of
    marshak_coefficient(kappa)."""
    if marshak:
        a = marshak_coefficient(kappa)
        return Problem(shape, h, float(kappa) ** 2, None, mask, (2,) * 6, (a,) * 6)
    return Problem(shape, h, float(kappa) ** 2, None, mask, (0,) * 6, (0.0,) * 6)


def rel_l2(u, ref, mask=None):
    """Relative L2 error over free cells (the paper's step error norm with
    volume fraction 1 on free cells and 0 on electrode cells, Sec. 3)."""
    d = np.asarray(u, dtype=np.float64) - np.asarray(ref, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if mask is not None:
        keep = np.asarray(mask) == 0
        d, ref = d[keep], ref[keep]
    den = np.sqrt(np.sum(ref * ref))
    return float(np.sqrt(np.sum(d * d)) / (den if den > 0 else 1.0))
