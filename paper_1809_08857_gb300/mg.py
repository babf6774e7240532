"""ctypes binding of libmg.so (include/mg.h).

Argument marshalling only: torch tensors are passed as raw device pointers and
the current torch CUDA stream is handed to the library.  Every step of the
solve runs in libmg's CUDA kernels; there is no CPU fallback, and loading
fails loudly when libmg.so is missing.
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmg.so")

MG_OK = 0
MG_ERR_INVALID_ARG = 1
MG_ERR_CUDA = 2
MG_ERR_OOM = 3
MG_ERR_NOT_CONVERGED = 4
MG_ERR_NONFINITE = 5
MG_ERR_UNSUPPORTED = 6
MG_ERR_DIVERGED = 7
# statuses a solve call returns with its outputs holding the last iterate
_NONCONVERGED = (MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED)

MG_BC_DIRICHLET = 0
MG_BC_NEUMANN = 1
MG_PREC_FP64 = 0
MG_PREC_MIXED = 1
MG_RTE_BC_DIRICHLET = 0
MG_RTE_BC_MARSHAK = 1
MG_COARSE_FACE = 0
MG_COARSE_CELL = 1

EXPORTS = [
    "mg_default_options", "mg_create", "mg_solve_poisson", "mg_solve_helmholtz_batch",
    "mg_solve_set",
    "mg_set_stream", "mg_level_info", "mg_destroy", "mg_error_string", "mg_last_error",
    "mg_profile_enable", "mg_profile_read", "mg_launch_count", "mg_residual_norm_noalloc",
    "mg_face_count", "mg_solve_batch", "mg_subbox_bc", "mg_set_options", "mg_autotune",
    "mg_unet_create", "mg_unet_destroy", "mg_unet_set_scales", "mg_unet_get_scales",
    "mg_unet_train_step", "mg_unet_predict", "mg_unet_grads", "mg_unet_num_params",
    "mg_unet_get_params", "mg_unet_set_params", "mg_unet_save", "mg_unet_load", "mg_nn_conv3d",
    "mg_nn_conv3d_stalled", "mg_nn_conv3d_wgrad", "mg_warmstart_attach", "mg_warmstart_load", "mg_warmstart_predict",
    "mg_poisson_residual", "mg_solve_screened", "mg_efield", "mg_solve_photoionization",
    "mg_residual_norms",
    "mg_amr_create", "mg_amr_solve", "mg_amr_residual", "mg_amr_destroy",
]

MG_PROBLEM_POISSON = 0
MG_PROBLEM_HELMHOLTZ = 1
MG_PROBLEM_SCREENED = 2
_KINDS = {"poisson": MG_PROBLEM_POISSON, "helmholtz": MG_PROBLEM_HELMHOLTZ,
          "screened": MG_PROBLEM_SCREENED}

KCLASSES = ["smooth", "restrict", "prolong", "resid64", "coarse"]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("origin", ctypes.c_double * 3)]


class BC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 6), ("value", ctypes.c_double * 6)]


class Options(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("precision", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("concurrency", ctypes.c_int), ("no_graphs", ctypes.c_int),
                ("rte_bc", ctypes.c_int), ("ir_zchunk", ctypes.c_int),
                ("coarse_op", ctypes.c_int), ("fixed_cycles", ctypes.c_int),
                ("coarse_visits", ctypes.c_int), ("sweep_zchunk", ctypes.c_int),
                ("stack", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_resid", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("hist", ctypes.c_double * 64), ("vcycles", ctypes.c_int),
                ("diverged", ctypes.c_int)]

    def as_dict(self):
        n = min(self.cycles + 1, 64)
        return {"cycles": self.cycles, "converged": bool(self.converged),
                "rel_resid": self.rel_resid, "time_ms": self.time_ms,
                "hist": list(self.hist[:n]), "vcycles": self.vcycles,
                "diverged": bool(self.diverged)}


class Problem(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("kind", ctypes.c_int), ("kappa", ctypes.c_double),
                ("rhs", ctypes.c_void_p), ("faces", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("alpha", ctypes.c_double)]


class AmrBox(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("lo", ctypes.c_int * 3), ("n", ctypes.c_int * 3)]


class KProf(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class MGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libmg status {status}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libmg.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmg.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.mg_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.mg_default_options.restype = None
    lib.mg_create.argtypes = [ctypes.POINTER(Grid), P, P, P, ctypes.POINTER(BC),
                              ctypes.POINTER(Options), P, ctypes.POINTER(P)]
    lib.mg_create.restype = ctypes.c_int
    lib.mg_solve_poisson.argtypes = [P, P, P, ctypes.c_double, ctypes.POINTER(Stats)]
    lib.mg_solve_poisson.restype = ctypes.c_int
    lib.mg_solve_screened.argtypes = [P, ctypes.c_double, P, P, ctypes.c_double,
                                      ctypes.POINTER(Stats)]
    lib.mg_solve_screened.restype = ctypes.c_int
    lib.mg_efield.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_double)]
    lib.mg_efield.restype = ctypes.c_int
    lib.mg_solve_helmholtz_batch.argtypes = [P, P, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_double, ctypes.POINTER(Stats)]
    lib.mg_solve_helmholtz_batch.restype = ctypes.c_int
    lib.mg_solve_set.argtypes = [P, P, P, P, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_double),
                                 ctypes.c_double, ctypes.POINTER(Stats)]
    lib.mg_solve_set.restype = ctypes.c_int
    lib.mg_solve_photoionization.argtypes = [P, P, ctypes.POINTER(P),
                                             ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                             ctypes.POINTER(Stats)]
    lib.mg_solve_photoionization.restype = ctypes.c_int
    lib.mg_residual_norms.argtypes = [P, ctypes.c_int, ctypes.c_double, P, P,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.mg_residual_norms.restype = ctypes.c_int
    lib.mg_set_stream.argtypes = [P, P]
    lib.mg_set_stream.restype = ctypes.c_int
    lib.mg_level_info.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    lib.mg_level_info.restype = ctypes.c_int
    lib.mg_destroy.argtypes = [P]
    lib.mg_destroy.restype = None
    lib.mg_error_string.argtypes = [ctypes.c_int]
    lib.mg_error_string.restype = ctypes.c_char_p
    lib.mg_last_error.argtypes = []
    lib.mg_last_error.restype = ctypes.c_char_p
    lib.mg_profile_enable.argtypes = [P, ctypes.c_int]
    lib.mg_profile_enable.restype = ctypes.c_int
    lib.mg_profile_read.argtypes = [P, ctypes.POINTER(KProf), ctypes.c_int]
    lib.mg_profile_read.restype = ctypes.c_int
    lib.mg_launch_count.argtypes = []
    lib.mg_launch_count.restype = ctypes.c_longlong
    lib.mg_residual_norm_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(BC),
                                             ctypes.c_double, P, ctypes.c_double, P, P, P, P]
    lib.mg_residual_norm_noalloc.restype = ctypes.c_int
    lib.mg_face_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.mg_face_count.restype = ctypes.c_longlong
    lib.mg_solve_batch.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_double,
                                   ctypes.POINTER(Stats)]
    lib.mg_solve_batch.restype = ctypes.c_int
    lib.mg_subbox_bc.argtypes = [P, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), P]
    lib.mg_subbox_bc.restype = ctypes.c_int
    lib.mg_set_options.argtypes = [P, ctypes.POINTER(Options)]
    lib.mg_set_options.restype = ctypes.c_int
    lib.mg_autotune.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_double)]
    lib.mg_autotune.restype = ctypes.c_int
    I, D, F = ctypes.c_int, ctypes.c_double, ctypes.c_float
    FP = ctypes.POINTER(ctypes.c_float)
    lib.mg_unet_create.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(P)]
    lib.mg_unet_destroy.argtypes = [P]
    lib.mg_unet_destroy.restype = None
    lib.mg_unet_set_scales.argtypes = [P, D, D, D]
    lib.mg_unet_get_scales.argtypes = [P, ctypes.POINTER(D)]
    lib.mg_unet_train_step.argtypes = [P, P, P, P, I, I, I, I, F, FP, P]
    lib.mg_unet_predict.argtypes = [P, P, P, P, I, I, I, I, P]
    lib.mg_unet_grads.argtypes = [P, P, P, P, I, I, I, I, FP, FP]
    lib.mg_unet_num_params.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.mg_unet_get_params.argtypes = [P, FP]
    lib.mg_unet_set_params.argtypes = [P, FP]
    lib.mg_unet_save.argtypes = [P, ctypes.c_char_p]
    lib.mg_unet_load.argtypes = [P, ctypes.c_char_p]
    lib.mg_nn_conv3d.argtypes = [P, I, P, I, P, P, I, I, I, I, I, I, P, P]
    lib.mg_nn_conv3d_stalled.argtypes = lib.mg_nn_conv3d.argtypes
    lib.mg_nn_conv3d_wgrad.argtypes = [P, I, P, I, P, I, I, I, I, I, P, P, P]
    lib.mg_warmstart_attach.argtypes = [P, P]
    lib.mg_warmstart_load.argtypes = [P, ctypes.c_char_p]
    lib.mg_warmstart_predict.argtypes = [P, P, P, P, ctypes.POINTER(I)]
    lib.mg_poisson_residual.argtypes = [P, P, P, P]
    lib.mg_poisson_residual.restype = ctypes.c_int
    PP = ctypes.POINTER(P)
    lib.mg_amr_create.argtypes = [ctypes.POINTER(Grid), I, ctypes.POINTER(AmrBox), PP, P, P,
                                  ctypes.POINTER(BC), ctypes.POINTER(Options), P, ctypes.POINTER(P)]
    lib.mg_amr_create.restype = ctypes.c_int
    lib.mg_amr_solve.argtypes = [P, I, D, PP, PP, D, ctypes.POINTER(Stats)]
    lib.mg_amr_solve.restype = ctypes.c_int
    lib.mg_amr_residual.argtypes = [P, I, D, PP, PP, PP, ctypes.POINTER(D)]
    lib.mg_amr_residual.restype = ctypes.c_int
    lib.mg_amr_destroy.argtypes = [P]
    lib.mg_amr_destroy.restype = None
    for name in ("mg_unet_create", "mg_unet_set_scales", "mg_unet_get_scales",
                 "mg_unet_train_step", "mg_unet_predict", "mg_unet_grads", "mg_unet_num_params",
                 "mg_unet_get_params", "mg_unet_set_params", "mg_unet_save", "mg_unet_load",
                 "mg_nn_conv3d", "mg_nn_conv3d_stalled", "mg_nn_conv3d_wgrad",
                 "mg_warmstart_attach",
                 "mg_warmstart_load", "mg_warmstart_predict"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, allow=()):
    if status == MG_OK or status in allow:
        return status
    lib = load()
    raise MGError(status, f"{lib.mg_error_string(status).decode()}: {lib.mg_last_error().decode()}")


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def launch_count():
    """Process-wide number of kernel launches issued by libmg."""
    return load().mg_launch_count()


def residual_norm_noalloc(u, rhs, h, alpha=0.0, rhs_scale=1.0, mask=None,
                          bc_kind=(1, 1, 1, 1, 0, 0), bc_value=(0, 0, 0, 0, 0, 1), out=None,
                          stream=None):
    """||b - A u||_2 for a constant-coefficient problem without any device
    allocation inside libmg (mg_residual_norm_noalloc).  `out` is a CUDA
    float64 tensor of one element that receives the norm (allocated here by
    torch if not given); the call is asynchronous on the stream."""
    lib = load()
    if u.dim() != 3:
        raise ValueError(f"u must be a 3-D (nz, ny, nx) field, got shape {tuple(u.shape)}")
    if tuple(rhs.shape) != tuple(u.shape):
        raise ValueError(f"rhs shape {tuple(rhs.shape)} != u shape {tuple(u.shape)}")
    if mask is not None and tuple(mask.shape) != tuple(u.shape):
        raise ValueError(f"mask shape {tuple(mask.shape)} != u shape {tuple(u.shape)}")
    if out is not None and out.numel() < 1:
        raise ValueError("out must hold at least one element")
    for name, t in (("rhs", rhs), ("mask", mask), ("out", out)):
        if t is not None and t.device != u.device:
            raise ValueError(f"{name} is on {t.device}, u on {u.device}")
    nz, ny, nx = (int(s) for s in u.shape)
    g = Grid(nx, ny, nz, float(h), (ctypes.c_double * 3)(0.0, 0.0, 0.0))
    bc = BC((ctypes.c_int * 6)(*[int(k) for k in bc_kind]),
            (ctypes.c_double * 6)(*[float(v) for v in bc_value]))
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=u.device)
    _check(lib.mg_residual_norm_noalloc(ctypes.byref(g), ctypes.byref(bc), float(alpha),
                                        _ptr(rhs, torch.float64), float(rhs_scale),
                                        _ptr(mask, torch.uint8), _ptr(u, torch.float64),
                                        _ptr(out, torch.float64), _stream_handle(stream)))
    return out


def face_count(shape):
    """Entries of the packed Dirichlet face data of a (nz, ny, nx) box."""
    nz, ny, nx = shape
    return load().mg_face_count(int(nx), int(ny), int(nz))


def solve_batch(problems, tol=1e-10, raise_on_nonconvergence=True):
    """Solve a list of problems, possibly on different Solvers (grids):
    each item is a dict with keys solver, kind ("poisson", "helmholtz" or
    "screened"), rhs, u, and optionally kappa (helmholtz), alpha (screened)
    and faces (packed Dirichlet data, CUDA float64)."""
    lib = load()
    arr = (Problem * len(problems))()
    for q, pr in enumerate(problems):
        sv = pr["solver"]
        sv._check_field(pr["rhs"])
        sv._check_field(pr["u"])
        sv.set_stream()
        faces = pr.get("faces")
        if faces is not None and faces.numel() != face_count(sv.shape):
            raise ValueError("faces has the wrong length")
        arr[q] = Problem(sv._ctx.value, _KINDS[pr["kind"]], float(pr.get("kappa", 0.0)),
                         _ptr(pr["rhs"], torch.float64).value,
                         None if faces is None else _ptr(faces, torch.float64).value,
                         _ptr(pr["u"], torch.float64).value, float(pr.get("alpha", 0.0)))
    st = (Stats * max(1, len(problems)))()
    status = lib.mg_solve_batch(arr, len(problems), float(tol), st)
    _check(status, () if raise_on_nonconvergence else _NONCONVERGED)
    return [st[q].as_dict() for q in range(len(problems))]


def default_options():
    opt = Options()
    load().mg_default_options(ctypes.byref(opt))
    return opt


class Solver:
    """One grid with its multigrid hierarchy (mg_create).

    shape: (nz, ny, nx); h: cell size; eps_r, mask, mask_value: CUDA tensors
    of that shape (float64, uint8, float64) or None; bc_kind/bc_value: the
    Poisson boundary conditions per face (-x,+x,-y,+y,-z,+z); rte_bc: domain
    faces of the Helmholtz problems (Psi = 0 or the Marshak condition).
    """

    def __init__(self, shape, h, eps_r=None, mask=None, mask_value=None,
                 bc_kind=(1, 1, 1, 1, 0, 0), bc_value=(0, 0, 0, 0, 0, 1),
                 precision=MG_PREC_FP64, nu1=2, nu2=2, max_cycles=100, inner_cycles=1,
                 concurrency=4, graphs=True, stream=None, rte_bc=MG_RTE_BC_DIRICHLET,
                 coarse_op=None):
        lib = load()
        nz, ny, nx = (int(s) for s in shape)
        self.shape = (nz, ny, nx)
        g = Grid(nx, ny, nz, float(h), (ctypes.c_double * 3)(0.0, 0.0, 0.0))
        bc = BC((ctypes.c_int * 6)(*[int(k) for k in bc_kind]),
                (ctypes.c_double * 6)(*[float(v) for v in bc_value]))
        opt = Options(nu1, nu2, max_cycles, precision, inner_cycles, concurrency,
                      0 if graphs else 1, rte_bc, 0,
                      MG_COARSE_FACE if coarse_op is None else coarse_op)
        for t in (eps_r, mask, mask_value):
            if t is not None and tuple(t.shape) != self.shape:
                raise ValueError("coefficient shape mismatch")
        ctx = ctypes.c_void_p()
        st = lib.mg_create(ctypes.byref(g), _ptr(eps_r, torch.float64), _ptr(mask, torch.uint8),
                           _ptr(mask_value, torch.float64), ctypes.byref(bc), ctypes.byref(opt),
                           _stream_handle(stream), ctypes.byref(ctx))
        _check(st)
        self._ctx = ctx
        self._lib = lib
        self.options = opt

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.mg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        _check(self._lib.mg_set_stream(self._ctx, _stream_handle(stream)))

    def levels(self):
        n = ctypes.c_int()
        out = []
        _check(self._lib.mg_level_info(self._ctx, 0, ctypes.byref(n), None))
        for l in range(n.value):
            d = (ctypes.c_int * 3)()
            _check(self._lib.mg_level_info(self._ctx, l, None, d))
            out.append((d[2], d[1], d[0]))
        return out

    def profile(self, enable=True):
        """Bracket every fine-level kernel launch with CUDA events (instrumentation)."""
        _check(self._lib.mg_profile_enable(self._ctx, 1 if enable else 0))

    def profile_read(self, reset=False):
        """Per kernel class: launches, event-timed ms, algorithmic bytes."""
        arr = (KProf * len(KCLASSES))()
        _check(self._lib.mg_profile_read(self._ctx, arr, 1 if reset else 0))
        return {k: {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes}
                for i, k in enumerate(KCLASSES)}

    def set_options(self, **kw):
        """Change any field of mg_options by name (nu1, nu2, max_cycles,
        inner_cycles, concurrency, ir_zchunk, fixed_cycles, coarse_visits,
        sweep_zchunk, ...; graphs=bool sets no_graphs).  The precision,
        rte_bc and coarse_op are fixed at creation (the library refuses a
        change)."""
        o = Options.from_buffer_copy(self.options)
        names = {f[0] for f in Options._fields_}
        for k, v in kw.items():
            if k == "graphs":
                o.no_graphs = 0 if v else 1
            elif k in names:
                setattr(o, k, int(v))
            else:
                raise TypeError(f"unknown option {k!r}")
        _check(self._lib.mg_set_options(self._ctx, ctypes.byref(o)))
        self.options = o

    def autotune(self, rho, S, kappa, tol=1e-10):
        """Time the sweep / inner-cycle candidates on this problem (mg_autotune)
        and install the fastest.  Returns (options dict, device ms)."""
        self.set_stream()
        best = Options()
        ms = ctypes.c_double()
        kap = (ctypes.c_double * 3)(*[float(k) for k in kappa])
        _check(self._lib.mg_autotune(self._ctx, _ptr(rho, torch.float64), _ptr(S, torch.float64),
                                     kap, float(tol), ctypes.byref(best), ctypes.byref(ms)))
        self.options = best
        return ({"nu1": best.nu1, "nu2": best.nu2, "inner_cycles": best.inner_cycles,
                 "ir_zchunk": best.ir_zchunk, "sweep_zchunk": best.sweep_zchunk}, ms.value)

    def poisson_residual(self, rho, phi, out=None):
        """r = b - A phi in FP64 (electrode cells of phi are set first)."""
        self._check_field(rho)
        self._check_field(phi)
        if out is None:
            out = torch.empty_like(phi)
        self.set_stream()
        _check(self._lib.mg_poisson_residual(self._ctx, _ptr(rho, torch.float64),
                                             _ptr(phi, torch.float64), _ptr(out, torch.float64)))
        return out

    def warmstart_attach(self, net):
        """Use a UNet for mg_warmstart_predict (None detaches)."""
        self._net = net
        _check(self._lib.mg_warmstart_attach(self._ctx, None if net is None else net._p))

    def warmstart_predict(self, rho, phi_prev, out=None):
        """Judged network guess for the Poisson solve; returns (guess, used_net)."""
        self._check_field(rho)
        self._check_field(phi_prev)
        if out is None:
            out = torch.empty_like(phi_prev)
        self.set_stream()
        used = ctypes.c_int()
        _check(self._lib.mg_warmstart_predict(self._ctx, _ptr(rho, torch.float64),
                                              _ptr(phi_prev, torch.float64),
                                              _ptr(out, torch.float64), ctypes.byref(used)))
        return out, bool(used.value)

    def subbox_bc(self, parent_u, origin, dims, out=None):
        """Dirichlet face data of a ratio-2 sub-box: origin = parent cell index
        (x, y, z) of its lower corner, dims = sub-box size in fine cells
        (x, y, z).  Returns the packed face array (CUDA float64)."""
        self._check_field(parent_u)
        nx, ny, nz = (int(d) for d in dims)
        if out is None:
            out = torch.empty(face_count((nz, ny, nx)), dtype=torch.float64, device=parent_u.device)
        self.set_stream()
        o = (ctypes.c_int * 3)(*[int(v) for v in origin])
        d = (ctypes.c_int * 3)(nx, ny, nz)
        _check(self._lib.mg_subbox_bc(self._ctx, _ptr(parent_u, torch.float64), o, d,
                                      _ptr(out, torch.float64)))
        return out

    def _check_field(self, t):
        if tuple(t.shape) != self.shape:
            raise ValueError(f"field shape {tuple(t.shape)} != grid {self.shape}")

    def solve_poisson(self, rho, phi, tol=1e-10, raise_on_nonconvergence=True):
        """Solve Eq. 2 in place on phi (CUDA float64).  Returns stats dict."""
        self._check_field(rho)
        self._check_field(phi)
        self.set_stream()
        st = Stats()
        status = self._lib.mg_solve_poisson(self._ctx, _ptr(rho, torch.float64),
                                            _ptr(phi, torch.float64), float(tol), ctypes.byref(st))
        _check(status, () if raise_on_nonconvergence else _NONCONVERGED)
        d = st.as_dict()
        d["status"] = status
        return d

    def efield(self, phi, J=None, E=None):
        """E = -grad phi at cell centres into E (CUDA float64 (3, nz, ny, nx),
        optional) and, with J (same layout), the relaxation time
        min eps0 |E| / |J| over free cells (mg_efield); returns it or None."""
        self._check_field(phi)
        for t in (J, E):
            if t is not None and (tuple(t.shape) != (3,) + self.shape or not t.is_contiguous()):
                raise ValueError("J and E must be contiguous (3, nz, ny, nx)")
        self.set_stream()
        dt = ctypes.c_double()
        _check(self._lib.mg_efield(self._ctx, _ptr(phi, torch.float64), _ptr(J, torch.float64),
                                   _ptr(E, torch.float64),
                                   ctypes.byref(dt) if J is not None else None))
        return dt.value if J is not None else None

    def solve_screened(self, alpha, f, u, tol=1e-10, raise_on_nonconvergence=True):
        """alpha u - div(beta grad u) = f in place on u, beta = this Solver's
        eps_r (mg_solve_screened)."""
        self._check_field(f)
        self._check_field(u)
        self.set_stream()
        st = Stats()
        status = self._lib.mg_solve_screened(self._ctx, ctypes.c_double(float(alpha)),
                                             _ptr(f, torch.float64), _ptr(u, torch.float64),
                                             ctypes.c_double(float(tol)), ctypes.byref(st))
        _check(status, () if raise_on_nonconvergence else _NONCONVERGED)
        d = st.as_dict()
        d["status"] = status
        return d

    def solve_helmholtz_batch(self, S, psi, kappa, tol=1e-10, raise_on_nonconvergence=True):
        """Solve the three Helmholtz problems of Eq. 3 in place on psi[0..2]."""
        self._check_field(S)
        if len(psi) != 3 or len(kappa) != 3:
            raise ValueError("need three psi arrays and three kappas")
        for p in psi:
            self._check_field(p)
        self.set_stream()
        ptrs = (ctypes.c_void_p * 3)(*[p.data_ptr() for p in psi])
        for p in psi:
            _ptr(p, torch.float64)
        kap = (ctypes.c_double * 3)(*[float(k) for k in kappa])
        st = (Stats * 3)()
        status = self._lib.mg_solve_helmholtz_batch(self._ctx, _ptr(S, torch.float64), ptrs, kap,
                                                    float(tol), st)
        _check(status, () if raise_on_nonconvergence else _NONCONVERGED)
        return [s.as_dict() for s in st]

    def solve_photoionization(self, S, psi, kappa, amp, tol=1e-10,
                              raise_on_nonconvergence=True):
        """(kappa_j^2 - lap) Psi_j = amp_j S in place on psi[0..2]
        (mg_solve_photoionization)."""
        self._check_field(S)
        if len(psi) != 3 or len(kappa) != 3 or len(amp) != 3:
            raise ValueError("need three psi arrays, three kappas and three amplitudes")
        for p in psi:
            self._check_field(p)
        self.set_stream()
        ptrs = (ctypes.c_void_p * 3)(*[p.data_ptr() for p in psi])
        for p in psi:
            _ptr(p, torch.float64)
        kap = (ctypes.c_double * 3)(*[float(k) for k in kappa])
        am = (ctypes.c_double * 3)(*[float(a) for a in amp])
        st = (Stats * 3)()
        status = self._lib.mg_solve_photoionization(self._ctx, _ptr(S, torch.float64), ptrs, kap,
                                                    am, float(tol), st)
        _check(status, () if raise_on_nonconvergence else _NONCONVERGED)
        return [s.as_dict() for s in st]

    def residual_norms(self, kind, rhs, u, param=0.0):
        """(||b - A u||_2, ||b||_2) over the free cells in plain FP64
        (mg_residual_norms); kind "poisson", "helmholtz" (param = kappa) or
        "screened" (param = alpha)."""
        self._check_field(rhs)
        self._check_field(u)
        self.set_stream()
        out = (ctypes.c_double * 2)()
        _check(self._lib.mg_residual_norms(self._ctx, _KINDS[kind], float(param),
                                           _ptr(rhs, torch.float64), _ptr(u, torch.float64),
                                           out))
        return out[0], out[1]

    def solve_set(self, rho, phi, S, psi, kappa, tol=1e-10, raise_on_nonconvergence=True):
        """Poisson (in place on phi) and the three Helmholtz problems (in place
        on psi[0..2]) of one time step in one call (mg_solve_set)."""
        for t in (rho, phi, S, *psi):
            self._check_field(t)
        if len(psi) != 3 or len(kappa) != 3:
            raise ValueError("need three psi arrays and three kappas")
        self.set_stream()
        ptrs = (ctypes.c_void_p * 3)(*[p.data_ptr() for p in psi])
        for p in psi:
            _ptr(p, torch.float64)
        kap = (ctypes.c_double * 3)(*[float(k) for k in kappa])
        st = (Stats * 4)()
        status = self._lib.mg_solve_set(self._ctx, _ptr(rho, torch.float64), _ptr(phi, torch.float64),
                                        _ptr(S, torch.float64), ptrs, kap, float(tol), st)
        _check(status, () if raise_on_nonconvergence else _NONCONVERGED)
        return [s.as_dict() for s in st]

    # ---- host-buffer convenience (end-to-end path) -------------------------

    def solve_poisson_host(self, rho_host, phi_host, tol=1e-10):
        """Host (pinned) buffers in and out: H2D copy, device solve, D2H copy."""
        dev = torch.device("cuda")
        rho = rho_host.to(dev, non_blocking=True)
        phi = phi_host.to(dev, non_blocking=True)
        st = self.solve_poisson(rho, phi, tol)
        phi_host.copy_(phi, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return st


UNET_CHANNELS = (16, 32, 48, 64)


def unet_conv_flops(n, d, h, w):
    """FLOPs (2 per multiply-add) of the 3x3x3 convolutions of one U-Net
    forward pass on a batch of n volumes d x h x w: per level l (grid >> l)
    two encoder convolutions (input 16 channels at level 0, the level above's
    width below), and on the way up an upsampling convolution from the level
    below, a convolution of the concatenated skip and one more."""
    C = UNET_CHANNELS
    total = 0
    for l in range(4):
        vox = n * (d >> l) * (h >> l) * (w >> l)
        cin = 16 if l == 0 else C[l - 1]
        layers = [(cin, C[l]), (C[l], C[l])]
        if l < 3:
            layers += [(C[l + 1], C[l]), (2 * C[l], C[l]), (C[l], C[l])]
        total += sum(2 * 27 * ci * co * vox for ci, co in layers)
    return total


class UNet:
    """The warm-start U-Net of libmg (mg_unet_*): fields are CUDA float64
    tensors of shape (n, d, h, w) or (d, h, w) with d, h, w multiples of 8."""

    def __init__(self, seed=0):
        self._lib = load()
        p = ctypes.c_void_p()
        _check(self._lib.mg_unet_create(int(seed), ctypes.byref(p)))
        self._p = p

    def close(self):
        if getattr(self, "_p", None):
            self._lib.mg_unet_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _dims(t):
        if t.dim() == 3:
            return (1,) + tuple(t.shape)
        if t.dim() == 4:
            return tuple(t.shape)
        raise ValueError("expected (d, h, w) or (n, d, h, w)")

    def set_scales(self, s_rho, s_phi, s_out):
        _check(self._lib.mg_unet_set_scales(self._p, float(s_rho), float(s_phi), float(s_out)))

    def scales(self):
        out = (ctypes.c_double * 3)()
        _check(self._lib.mg_unet_get_scales(self._p, out))
        return tuple(out)

    def train_step(self, rho, prev, phi, lr=1e-3, stream=None):
        n, d, h, w = self._dims(rho)
        loss = ctypes.c_float()
        _check(self._lib.mg_unet_train_step(self._p, _ptr(rho, torch.float64),
                                            _ptr(prev, torch.float64), _ptr(phi, torch.float64),
                                            n, d, h, w, float(lr), ctypes.byref(loss),
                                            _stream_handle(stream)))
        return loss.value

    def predict(self, rho, prev, out=None, stream=None):
        n, d, h, w = self._dims(rho)
        if out is None:
            out = torch.empty_like(prev)
        _check(self._lib.mg_unet_predict(self._p, _ptr(rho, torch.float64),
                                         _ptr(prev, torch.float64), _ptr(out, torch.float64),
                                         n, d, h, w, _stream_handle(stream)))
        return out

    def num_params(self):
        n = ctypes.c_longlong()
        _check(self._lib.mg_unet_num_params(self._p, ctypes.byref(n)))
        return n.value

    def get_params(self):
        import numpy as np

        a = np.empty(self.num_params(), dtype=np.float32)
        _check(self._lib.mg_unet_get_params(self._p, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return a

    def set_params(self, a):
        import numpy as np

        a = np.ascontiguousarray(a, dtype=np.float32)
        if a.size != self.num_params():
            raise ValueError("parameter count mismatch")
        _check(self._lib.mg_unet_set_params(self._p, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def grads(self, rho, prev, phi):
        import numpy as np

        n, d, h, w = self._dims(rho)
        g = np.empty(self.num_params(), dtype=np.float32)
        loss = ctypes.c_float()
        _check(self._lib.mg_unet_grads(self._p, _ptr(rho, torch.float64), _ptr(prev, torch.float64),
                                       _ptr(phi, torch.float64), n, d, h, w,
                                       g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       ctypes.byref(loss)))
        return g, loss.value

    def save(self, path):
        _check(self._lib.mg_unet_save(self._p, str(path).encode()))

    def load_file(self, path):
        _check(self._lib.mg_unet_load(self._p, str(path).encode()))


def conv3d(x1, w, bias=None, x2=None, relu=False, stream=None, stalled=False):
    """One network convolution (mg_nn_conv3d): x1/x2 channels-last bfloat16
    CUDA tensors (n, d, h, w, c), w bfloat16 (cout, 27, c1 + c2), bias float32.
    stalled=True runs the bounded-wait self-check (mg_nn_conv3d_stalled),
    which raises MGError with MG_ERR_CUDA when the check works."""
    n, d, h, ww, c1 = x1.shape
    c2 = 0 if x2 is None else x2.shape[-1]
    cout = w.shape[0]
    y = torch.empty((n, d, h, ww, cout), dtype=torch.bfloat16, device=x1.device)
    fn = load().mg_nn_conv3d_stalled if stalled else load().mg_nn_conv3d
    _check(fn(_ptr(x1, torch.bfloat16), c1, None if x2 is None else _ptr(x2, torch.bfloat16),
              c2, _ptr(w, torch.bfloat16), None if bias is None else _ptr(bias, torch.float32),
              1 if relu else 0, cout, n, d, h, ww, _ptr(y, torch.bfloat16),
              _stream_handle(stream)))
    return y


def conv3d_wgrad(dy, x1, x2=None, stream=None, bias=False):
    """Weight gradient (mg_nn_conv3d_wgrad) as float32 (cout, 27, c1 + c2);
    with bias=True also the bias gradient, float32 (cout,): (dw, db)."""
    n, d, h, ww, cout = dy.shape
    c1 = x1.shape[-1]
    c2 = 0 if x2 is None else x2.shape[-1]
    dw = torch.empty((cout, 27, c1 + c2), dtype=torch.float32, device=dy.device)
    db = torch.empty((cout,), dtype=torch.float32, device=dy.device) if bias else None
    _check(load().mg_nn_conv3d_wgrad(_ptr(dy, torch.bfloat16), cout, _ptr(x1, torch.bfloat16), c1,
                                     None if x2 is None else _ptr(x2, torch.bfloat16), c2, n, d, h,
                                     ww, _ptr(dw, torch.float32),
                                     None if db is None else _ptr(db, torch.float32),
                                     _stream_handle(stream)))
    return (dw, db) if bias else dw


class Amr:
    """A ratio-2 composite AMR hierarchy (mg_amr_create).

    base_shape (nz, ny, nx) and h: the level-0 grid.  boxes: the refined
    boxes as (level, lo, shape), lo and shape in (z, y, x) cells of that
    level.  Per-box arrays are lists with the base box first, then the
    refined boxes in the given order: eps_r (None, or one CUDA float64 tensor
    or None per box); rhs, u and r of solve() and residual().  mask and
    mask_value belong to the base box.  The library works on the stream that
    is current at construction.
    """

    def __init__(self, base_shape, h, boxes=(), eps_r=None, mask=None, mask_value=None,
                 bc_kind=(1, 1, 1, 1, 0, 0), bc_value=(0, 0, 0, 0, 0, 1),
                 precision=MG_PREC_FP64, nu1=2, nu2=2, max_cycles=100, inner_cycles=1,
                 stream=None, rte_bc=MG_RTE_BC_DIRICHLET):
        lib = load()
        nz, ny, nx = (int(v) for v in base_shape)
        self.shapes = [(nz, ny, nx)] + [tuple(int(v) for v in b[2]) for b in boxes]
        g = Grid(nx, ny, nz, float(h), (ctypes.c_double * 3)(0.0, 0.0, 0.0))
        bc = BC((ctypes.c_int * 6)(*[int(k) for k in bc_kind]),
                (ctypes.c_double * 6)(*[float(v) for v in bc_value]))
        opt = Options(nu1, nu2, max_cycles, precision, inner_cycles, 1, 1, rte_bc)
        arr = (AmrBox * max(1, len(boxes)))()
        for q, (lev, lo, shape) in enumerate(boxes):
            arr[q] = AmrBox(int(lev), (ctypes.c_int * 3)(*[int(v) for v in reversed(lo)]),
                            (ctypes.c_int * 3)(*[int(v) for v in reversed(shape)]))
        eps = None
        if eps_r is not None:
            if len(eps_r) != len(self.shapes):
                raise ValueError("eps_r needs one entry per box")
            for t, sh in zip(eps_r, self.shapes):
                if t is not None and tuple(t.shape) != sh:
                    raise ValueError("eps_r shape mismatch")
            eps = (ctypes.c_void_p * len(eps_r))(*[None if t is None else _ptr(t, torch.float64).value
                                                   for t in eps_r])
        for t in (mask, mask_value):
            if t is not None and tuple(t.shape) != self.shapes[0]:
                raise ValueError("mask shape mismatch")
        amr = ctypes.c_void_p()
        st = lib.mg_amr_create(ctypes.byref(g), len(boxes), arr, eps, _ptr(mask, torch.uint8),
                               _ptr(mask_value, torch.float64), ctypes.byref(bc),
                               ctypes.byref(opt), _stream_handle(stream), ctypes.byref(amr))
        _check(st)
        self._amr = amr
        self._lib = lib

    def close(self):
        if getattr(self, "_amr", None):
            self._lib.mg_amr_destroy(self._amr)
            self._amr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, ts):
        if len(ts) != len(self.shapes):
            raise ValueError("need one array per box")
        for t, sh in zip(ts, self.shapes):
            if tuple(t.shape) != sh:
                raise ValueError("box array shape mismatch")
        return (ctypes.c_void_p * len(ts))(*[_ptr(t, torch.float64).value for t in ts])

    def solve(self, kind, rhs, u, tol=1e-10, param=0.0, raise_on_nonconvergence=True):
        """mg_amr_solve: kind "poisson" (rhs = rho), "screened" (param =
        alpha, rhs = f) or "helmholtz" (param = kappa, rhs = S); u is updated
        in place.  Returns the stats as a dict."""
        st = Stats()
        status = self._lib.mg_amr_solve(self._amr, _KINDS[kind], float(param), self._arrays(rhs),
                                        self._arrays(u), float(tol), ctypes.byref(st))
        _check(status, () if raise_on_nonconvergence else _NONCONVERGED)
        return st.as_dict()

    def residual(self, kind, rhs, u, param=0.0):
        """mg_amr_residual: per-box composite residuals and ||r||_2 over the
        valid cells."""
        r = [torch.empty(sh, dtype=torch.float64, device=u[0].device) for sh in self.shapes]
        norm = ctypes.c_double()
        _check(self._lib.mg_amr_residual(self._amr, _KINDS[kind], float(param), self._arrays(rhs),
                                         self._arrays(u), self._arrays(r), ctypes.byref(norm)))
        return r, norm.value
