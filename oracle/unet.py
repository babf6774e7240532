"""Plain numpy reference of the warm-start U-Net (TEST INFRASTRUCTURE ONLY).

Same architecture, parameter order and input packing as libmg's network:
4 levels with 16/32/48/64 channels, two 3x3x3 convolutions (zero padding,
ReLU) per level, 2x average pooling down, nearest 2x upsampling followed by a
3x3x3 convolution (ReLU) up, skip connections by channel concatenation
(upsampled branch first), and a 1x1x1 head to one channel.  Tensors are
channels-last (n, d, h, w, c); conv weights (cout, 27, cin) with tap
t = (kd*3 + kh)*3 + kw.

Arithmetic is FP64.  With ``bf16=True`` every stored activation and every
weight is rounded to bfloat16 (round to nearest even of the float32 bits), as
the GPU stores them, so that its gradients can be compared closely.

Pinned by tests/test_unet_oracle_pins.py: the convolution against
scipy.ndimage.correlate, the backward pass against central finite
differences, pooling/upsampling identities.
"""
import numpy as np

CHAN = (16, 32, 48, 64)


def to_bf16(a):
    """Round to bfloat16 (nearest, ties to even) and return float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _shift(x, kd, kh, kw):
    """x[.., d + kd - 1, h + kh - 1, w + kw - 1, :] with zeros outside."""
    n, d, h, w, c = x.shape
    p = np.zeros((n, d + 2, h + 2, w + 2, c))
    p[:, 1:-1, 1:-1, 1:-1] = x
    return p[:, kd:kd + d, kh:kh + h, kw:kw + w]


def conv3d(x, w, b=None):
    """Pre-activation 3x3x3 convolution: y[v, co] = sum_t,ci x[v + off(t), ci] w[co, t, ci] + b."""
    n, d, h, ww, c = x.shape
    cout = w.shape[0]
    y = np.zeros((n, d, h, ww, cout))
    for t in range(27):
        kd, kh, kw = t // 9, (t // 3) % 3, t % 3
        y += _shift(x, kd, kh, kw) @ w[:, t, :].T
    if b is not None:
        y += b
    return y


def conv3d_backward(x, w, gy):
    """Gradients of conv3d (pre-activation gy): returns (gx, gw, gb)."""
    n, d, h, ww, c = x.shape
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    gyf = gy.reshape(-1, gy.shape[-1])
    for t in range(27):
        kd, kh, kw = t // 9, (t // 3) % 3, t % 3
        xs = _shift(x, kd, kh, kw)
        gw[:, t, :] = gyf.T @ xs.reshape(-1, c)
        # y[v] takes x[v + off]; so x[u] receives gy[u - off]
        contrib = gy @ w[:, t, :]
        p = np.zeros((n, d + 2, h + 2, ww + 2, c))
        p[:, kd:kd + d, kh:kh + h, kw:kw + ww] = contrib
        gx += p[:, 1:-1, 1:-1, 1:-1]
    return gx, gw, gyf.sum(axis=0)


def pool(x):
    n, d, h, w, c = x.shape
    return x.reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4, 6))


def pool_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(gy):
    n, d, h, w, c = gy.shape
    return gy.reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4, 6))


def layer_shapes():
    """(name, cout, cin) of every conv in parameter order."""
    out = []
    for l in range(4):
        cin = 16 if l == 0 else CHAN[l - 1]
        out += [(f"enc{l}a", CHAN[l], cin), (f"enc{l}b", CHAN[l], CHAN[l])]
    for l in range(3):
        out += [(f"up{l}", CHAN[l], CHAN[l + 1]), (f"dec{l}a", CHAN[l], 2 * CHAN[l]),
                (f"dec{l}b", CHAN[l], CHAN[l])]
    return out


def unpack(flat):
    """Flat parameter vector (libmg order) -> dict of arrays."""
    p, off = {}, 0
    flat = np.asarray(flat, dtype=np.float64)
    for name, co, ci in layer_shapes():
        k = co * 27 * ci
        p[name + ".w"] = flat[off:off + k].reshape(co, 27, ci)
        off += k
        p[name + ".b"] = flat[off:off + co]
        off += co
    p["head.w"] = flat[off:off + 16]
    p["head.b"] = flat[off + 16:off + 17]
    assert off + 17 == flat.size
    return p


def pack(p):
    parts = []
    for name, co, ci in layer_shapes():
        parts += [p[name + ".w"].ravel(), p[name + ".b"].ravel()]
    parts += [p["head.w"].ravel(), p["head.b"].ravel()]
    return np.concatenate(parts)


def pack_input(rho, prev, s_rho, s_phi, bf16=False):
    """(n, d, h, w) fields -> (n, d, h, w, 16) input, channels 2..15 zero."""
    x = np.zeros(rho.shape + (16,))
    x[..., 0] = rho * s_rho
    x[..., 1] = prev * s_phi
    return to_bf16(x) if bf16 else x


def forward(p, x, bf16=False):
    """Returns (out (n, d, h, w), cache of activations)."""
    r = to_bf16 if bf16 else (lambda a: a)
    W = {k: (r(v) if k.endswith(".w") and not k.startswith("head") else v) for k, v in p.items()}
    cache = {"x": x}

    def cv(name, inp):
        y = r(np.maximum(conv3d(inp, W[name + ".w"], W[name + ".b"]), 0.0))
        cache[name] = y
        return y

    h = x
    for l in range(4):
        a = cv(f"enc{l}a", h)
        e = cv(f"enc{l}b", a)
        cache[f"e{l}"] = e
        if l < 3:
            h = r(pool(e))
            cache[f"p{l}"] = h
    below = cache["e3"]
    for l in (2, 1, 0):
        u = up(below)
        cache[f"u{l}"] = u
        uc = cv(f"up{l}", u)
        da = cv(f"dec{l}a", np.concatenate([uc, cache[f"e{l}"]], axis=-1))
        below = cv(f"dec{l}b", da)
    out = below @ p["head.w"] + p["head.b"][0]
    return out, cache


def loss_and_grads(p, rho, prev, phi, scales, bf16=False):
    """MSE loss of (out - (phi - prev) s_out) and gradients (dict like p)."""
    s_rho, s_phi, s_out = scales
    x = pack_input(rho, prev, s_rho, s_phi, bf16)
    out, c = forward(p, x, bf16)
    t = (phi - prev) * s_out
    nv = out.size
    loss = float(np.sum((out - t) ** 2) / nv)
    g_out = 2.0 * (out - t) / nv
    r = to_bf16 if bf16 else (lambda a: a)
    W = {k: (r(v) if k.endswith(".w") and not k.startswith("head") else v) for k, v in p.items()}
    G = {}
    d0 = c["dec0b"]
    G["head.w"] = (d0 * g_out[..., None]).reshape(-1, d0.shape[-1]).sum(axis=0)
    G["head.b"] = np.array([g_out.sum()])
    gy = r(g_out[..., None] * p["head.w"])

    def back(name, inp, gy):
        gpre = np.where(c[name] > 0, gy, 0.0)
        gx, gw, gb = conv3d_backward(inp, W[name + ".w"], gpre)
        G[name + ".w"], G[name + ".b"] = gw, gb
        return r(gx)

    ge = {}
    for l in (0, 1, 2):
        gda = back(f"dec{l}b", c[f"dec{l}a"], gy)
        cat = np.concatenate([c[f"up{l}"], c[f"e{l}"]], axis=-1)
        gcat = back(f"dec{l}a", cat, gda)
        guc, ge[l] = gcat[..., :CHAN[l]], gcat[..., CHAN[l]:]
        gu = back(f"up{l}", c[f"u{l}"], guc)
        gy = r(up_backward(gu))  # gradient of d_{l+1} (or e3)
    ge[3] = gy
    for l in (3, 2, 1, 0):
        ga = back(f"enc{l}b", c[f"enc{l}a"], ge[l])
        inp = c["x"] if l == 0 else c[f"p{l - 1}"]
        gin = back(f"enc{l}a", inp, ga)
        if l > 0:
            ge[l - 1] = r(ge[l - 1] + pool_backward(gin))
    return loss, G
