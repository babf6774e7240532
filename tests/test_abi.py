"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function include/mg.h declares, and argument validation
rejects bad input before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_08857_gb300 import build, mg

    build.build()
    return mg.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "mg_create" in names and "mg_solve_poisson" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_1809_08857_gb300 import mg

    assert sorted(mg.EXPORTS) == sorted(n for n in declared_functions())


def test_create_rejects_bad_arguments_without_gpu(lib):
    from paper_1809_08857_gb300 import mg

    ctx = ctypes.c_void_p()
    bc = mg.BC((ctypes.c_int * 6)(1, 1, 1, 1, 0, 0), (ctypes.c_double * 6)(0, 0, 0, 0, 0, 1))
    bad = mg.Grid(0, 8, 8, 0.1, (ctypes.c_double * 3)())
    assert lib.mg_create(ctypes.byref(bad), None, None, None, ctypes.byref(bc), None, None,
                         ctypes.byref(ctx)) == mg.MG_ERR_INVALID_ARG
    assert b"sizes" in lib.mg_last_error()
    good = mg.Grid(8, 8, 8, -1.0, (ctypes.c_double * 3)())
    assert lib.mg_create(ctypes.byref(good), None, None, None, ctypes.byref(bc), None, None,
                         ctypes.byref(ctx)) == mg.MG_ERR_INVALID_ARG
    badbc = mg.BC((ctypes.c_int * 6)(1, 1, 7, 1, 0, 0), (ctypes.c_double * 6)())
    good = mg.Grid(8, 8, 8, 0.1, (ctypes.c_double * 3)())
    assert lib.mg_create(ctypes.byref(good), None, None, None, ctypes.byref(badbc), None, None,
                         ctypes.byref(ctx)) == mg.MG_ERR_INVALID_ARG
    opt = mg.Options(2, 2, 10, 9, 1, 4, 0, 0)
    assert lib.mg_create(ctypes.byref(good), None, None, None, ctypes.byref(bc), ctypes.byref(opt),
                         None, ctypes.byref(ctx)) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_create(None, None, None, None, None, None, None, None) == mg.MG_ERR_INVALID_ARG


def test_solve_rejects_null_context(lib):
    from paper_1809_08857_gb300 import mg

    assert lib.mg_solve_poisson(None, None, None, 1e-10, None) == mg.MG_ERR_INVALID_ARG
    assert lib.mg_solve_helmholtz_batch(None, None, None, None, 1e-10, None) == mg.MG_ERR_INVALID_ARG
    lib.mg_destroy(None)
    assert lib.mg_error_string(mg.MG_ERR_NOT_CONVERGED) == b"not converged within max_cycles"


def test_default_options(lib):
    from paper_1809_08857_gb300 import mg

    o = mg.default_options()
    assert (o.nu1, o.nu2, o.max_cycles, o.precision, o.inner_cycles, o.concurrency,
            o.no_graphs) == (2, 2, 100, 0, 1, 4, 0)


@pytest.mark.parametrize("boxes,msg", [
    ([(1, (8, 8, 0), (8, 8, 8))], b"footprint"),       # touches the domain boundary
    ([(1, (8, 8, 8), (8, 8, 8)), (1, (8, 8, 16), (8, 8, 8))], b"apart"),  # siblings too close
    ([(1, (8, 8, 7), (8, 8, 8))], b"even"),            # odd corner
    ([(2, (20, 20, 20), (8, 8, 8))], b"footprint"),    # no level-1 parent
    ([(0, (8, 8, 8), (8, 8, 8))], b"level"),
])
def test_amr_create_rejects_bad_hierarchies_without_gpu(lib, boxes, msg):
    """The nesting rules of the composite hierarchy are checked on the host
    before any device work (corners and sizes here in x, y, z order)."""
    from paper_1809_08857_gb300 import mg

    g = mg.Grid(16, 16, 16, 1.0 / 16, (ctypes.c_double * 3)())
    bc = mg.BC((ctypes.c_int * 6)(1, 1, 1, 1, 0, 0), (ctypes.c_double * 6)(0, 0, 0, 0, 0, 1))
    arr = (mg.AmrBox * len(boxes))()
    for q, (lev, lo, n) in enumerate(boxes):
        arr[q] = mg.AmrBox(lev, (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*n))
    out = ctypes.c_void_p()
    st = lib.mg_amr_create(ctypes.byref(g), len(boxes), arr, None, None, None, ctypes.byref(bc),
                           None, None, ctypes.byref(out))
    assert st == mg.MG_ERR_INVALID_ARG
    assert msg in lib.mg_last_error()
    assert not out.value
    assert lib.mg_amr_solve(None, 0, 0.0, None, None, 1e-10, None) == mg.MG_ERR_INVALID_ARG
    lib.mg_amr_destroy(None)


def test_conv3d_rejects_bad_arguments_without_gpu(lib):
    """The network convolution checks channels and 16-byte alignment (its
    operands are read by tiled tensor copies) before touching any memory;
    the pointer values below are never dereferenced."""
    from paper_1809_08857_gb300 import mg

    P = ctypes.c_void_p
    good, odd = P(0x10000), P(0x10002)
    conv = lib.mg_nn_conv3d
    args = lambda x1, c1, x2, c2, w, cout: (x1, c1, x2, c2, w, None, 1, cout, 1, 8, 8, 8, good, None)
    assert conv(*args(odd, 16, None, 0, good, 16)) == mg.MG_ERR_INVALID_ARG
    assert b"aligned" in lib.mg_last_error()
    assert conv(*args(good, 16, odd, 16, good, 16)) == mg.MG_ERR_INVALID_ARG
    assert conv(*args(good, 16, None, 0, odd, 32)) == mg.MG_ERR_INVALID_ARG
    assert conv(*args(good, 24, None, 0, good, 16)) == mg.MG_ERR_UNSUPPORTED
    assert conv(*args(good, 0, good, 16, good, 16)) == mg.MG_ERR_UNSUPPORTED
    assert conv(*args(good, 16, None, 0, good, 80)) == mg.MG_ERR_UNSUPPORTED
    assert conv(*args(None, 16, None, 0, good, 16)) == mg.MG_ERR_INVALID_ARG
    # the wait self-check runs the same checks first
    stalled = lib.mg_nn_conv3d_stalled
    assert stalled(*args(odd, 16, None, 0, good, 16)) == mg.MG_ERR_INVALID_ARG
    assert stalled(*args(good, 24, None, 0, good, 16)) == mg.MG_ERR_UNSUPPORTED


def test_noalloc_binding_rejects_mismatched_shapes():
    """The binding of mg_residual_norm_noalloc checks shapes, rank and the
    output size before anything reaches the library (so a smaller rhs or mask
    can never be read past its end)."""
    torch = pytest.importorskip("torch")
    from paper_1809_08857_gb300 import mg

    u = torch.zeros((4, 5, 6), dtype=torch.float64)
    with pytest.raises(ValueError, match="rhs shape"):
        mg.residual_norm_noalloc(u, torch.zeros((4, 5, 5), dtype=torch.float64), 0.1)
    with pytest.raises(ValueError, match="mask shape"):
        mg.residual_norm_noalloc(u, u, 0.1, mask=torch.zeros((4, 5, 5), dtype=torch.uint8))
    with pytest.raises(ValueError, match="3-D"):
        mg.residual_norm_noalloc(u.view(-1), u.view(-1), 0.1)
    with pytest.raises(ValueError, match="at least one"):
        mg.residual_norm_noalloc(u, u, 0.1, out=torch.empty(0, dtype=torch.float64))


@pytest.mark.parametrize("field,value,msg", [
    ("sweep_zchunk", 7, b"sweep_zchunk"),
    ("sweep_zchunk", -2, b"sweep_zchunk"),
    ("coarse_visits", 3, b"coarse_visits"),
    ("fixed_cycles", 2, b"fixed_cycles"),
    ("stack", 2, b"stack"),
])
def test_create_rejects_bad_option_values(lib, field, value, msg):
    """Option values outside their documented sets are refused before any
    device work."""
    from paper_1809_08857_gb300 import mg

    ctx = ctypes.c_void_p()
    bc = mg.BC((ctypes.c_int * 6)(1, 1, 1, 1, 0, 0), (ctypes.c_double * 6)(0, 0, 0, 0, 0, 1))
    good = mg.Grid(8, 8, 8, 0.1, (ctypes.c_double * 3)())
    opt = mg.default_options()
    setattr(opt, field, value)
    assert lib.mg_create(ctypes.byref(good), None, None, None, ctypes.byref(bc), ctypes.byref(opt),
                         None, ctypes.byref(ctx)) == mg.MG_ERR_INVALID_ARG
    assert msg in lib.mg_last_error()
