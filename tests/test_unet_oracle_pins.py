"""Pins for the numpy U-Net oracle (oracle/unet.py): the convolution against
scipy.ndimage.correlate, the backward pass against central finite
differences in FP64, and the pooling / upsampling identities."""
import numpy as np
import pytest

from oracle import unet as U


def test_conv3d_matches_scipy_correlate():
    from scipy.ndimage import correlate

    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 7, 3))
    w = rng.standard_normal((4, 27, 3))
    b = rng.standard_normal(4)
    y = U.conv3d(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = np.full(x.shape[1:4], b[co])
            for ci in range(3):
                ker = w[co, :, ci].reshape(3, 3, 3)  # [kd, kh, kw]
                ref += correlate(x[n, ..., ci], ker, mode="constant", cval=0.0)
            np.testing.assert_allclose(y[n, ..., co], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_backward_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 4, 5, 3, 2))
    w = rng.standard_normal((3, 27, 2))
    gy = rng.standard_normal((1, 4, 5, 3, 3))
    f = lambda xx, ww: float(np.sum(U.conv3d(xx, ww) * gy))
    gx, gw, gb = U.conv3d_backward(x, w, gy)
    eps = 1e-6
    for idx in [(0, 0, 0, 0, 0), (0, 3, 4, 2, 1), (0, 2, 1, 1, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        assert abs((f(xp, w) - f(xm, w)) / (2 * eps) - gx[idx]) < 1e-6
    for idx in [(0, 0, 0), (2, 13, 1), (1, 26, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += eps
        wm[idx] -= eps
        assert abs((f(x, wp) - f(x, wm)) / (2 * eps) - gw[idx]) < 1e-6
    b = rng.standard_normal(3)
    fb = lambda bb: float(np.sum(U.conv3d(x, w, bb) * gy))
    for co in range(3):
        bp, bm = b.copy(), b.copy()
        bp[co] += eps
        bm[co] -= eps
        assert abs((fb(bp) - fb(bm)) / (2 * eps) - gb[co]) < 1e-6


def test_pool_up_identities():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 4, 6, 8, 3))
    np.testing.assert_allclose(U.pool(U.up(x)), x)
    g = rng.standard_normal((1, 8, 12, 16, 3))
    # adjoints: <pool(a), b> = <a, pool_backward(b)>, <up(a), g> = <a, up_backward(g)>
    a = rng.standard_normal((1, 8, 12, 16, 3))
    bb = rng.standard_normal((1, 4, 6, 8, 3))
    assert abs(np.sum(U.pool(a) * bb) - np.sum(a * U.pool_backward(bb))) < 1e-10
    assert abs(np.sum(U.up(bb) * g) - np.sum(bb * U.up_backward(g))) < 1e-10


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5, 1e-3])
    r = U.to_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0  # tie rounds to even
    assert r[2] == 1.0 + 2**-7
    assert r[3] == -2.5
    assert abs(r[4] - 1e-3) < 1e-3 * 2**-8


@pytest.mark.parametrize("part", ["w", "b"])
@pytest.mark.parametrize("layer", ["enc0a", "enc2b", "enc3a", "up1", "dec0a", "dec2b", "head"])
def test_network_gradient_finite_differences(layer, part):
    """Whole U-Net (FP64): analytic gradients of the MSE loss with respect to
    weights and biases (every sampled layer, the head included) agree with
    central differences."""
    rng = np.random.default_rng(3)
    shapes = U.layer_shapes()
    flat = []
    for name, co, ci in shapes:
        flat += [rng.standard_normal(co * 27 * ci) * np.sqrt(2.0 / (27 * ci)), 0.1 * rng.standard_normal(co)]
    flat += [0.3 * rng.standard_normal(16), [0.05]]
    p = U.unpack(np.concatenate(flat))
    rho = rng.standard_normal((1, 8, 8, 8))
    prev = rng.standard_normal((1, 8, 8, 8))
    phi = prev + 0.1 * rng.standard_normal((1, 8, 8, 8))
    sc = (0.7, 1.3, 5.0)
    loss, G = U.loss_and_grads(p, rho, prev, phi, sc)
    key = f"{layer}.{part}"
    eps = 1e-6
    flatk = p[key].reshape(-1)
    for q in rng.choice(flatk.size, size=min(3, flatk.size), replace=False):
        orig = flatk[q]
        flatk[q] = orig + eps
        lp, _ = U.loss_and_grads(p, rho, prev, phi, sc)
        flatk[q] = orig - eps
        lm, _ = U.loss_and_grads(p, rho, prev, phi, sc)
        flatk[q] = orig
        fd = (lp - lm) / (2 * eps)
        an = G[key].reshape(-1)[q]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (key, q, fd, an)
