"""GPU tests of the warm-start U-Net kernels and network against the numpy
oracle (oracle/unet.py), which runs in FP64 on the same BF16 weights and,
for the whole network, rounds stored activations to BF16 as the GPU does."""
import numpy as np
import pytest

from oracle import unet as U

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


def bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("shape,c1,c2,cout,relu", [
    ((2, 3, 5, 19), 16, 0, 16, True),     # ragged against the 16 x 4 x 2 tile
    ((1, 4, 8, 16), 32, 0, 48, True),
    ((1, 5, 6, 7), 48, 48, 48, True),     # concatenated input
    ((1, 4, 4, 20), 16, 16, 96, False),   # widest output (input gradient of a concat layer)
    ((1, 2, 9, 33), 64, 0, 64, False),
])
def test_conv3d_matches_oracle(mg, shape, c1, c2, cout, relu):
    rng = np.random.default_rng(c1 + c2 + cout)
    n, d, h, w = shape
    x1 = U.to_bf16(rng.standard_normal((n, d, h, w, c1)))
    x2 = U.to_bf16(rng.standard_normal((n, d, h, w, c2))) if c2 else None
    wt = U.to_bf16(rng.standard_normal((cout, 27, c1 + c2)) * 0.1)
    b = rng.standard_normal(cout).astype(np.float32)
    y = mg.conv3d(bf(x1), bf(wt), torch.from_numpy(b).cuda(), None if x2 is None else bf(x2), relu)
    torch.cuda.synchronize()
    got = y.float().cpu().numpy().astype(np.float64)
    xin = x1 if x2 is None else np.concatenate([x1, x2], axis=-1)
    ref = U.conv3d(xin, wt, b.astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0.0)
    # output rounded to bfloat16 (relative 2^-8), FP32 accumulation
    assert np.all(np.abs(got - ref) <= 2.0**-8 * np.abs(ref) + 1e-4 * np.abs(ref).max())


def test_conv3d_bounded_wait_gives_up_and_context_stays_usable(mg):
    """The tensor-core kernels' waits are bounded: the self-check asks the
    first chunk's barrier for 16 bytes its copies never deliver, the wait
    gives up after 50 ms, the kernel drains and frees its tensor memory, the
    call reports MG_ERR_CUDA, and the next convolution is correct."""
    rng = np.random.default_rng(77)
    x = U.to_bf16(rng.standard_normal((1, 2, 16, 8, 16)))
    wt = U.to_bf16(rng.standard_normal((16, 27, 16)) * 0.1)
    b = rng.standard_normal(16).astype(np.float32)
    with pytest.raises(mg.MGError) as err:
        mg.conv3d(bf(x), bf(wt), torch.from_numpy(b).cuda(), relu=True, stalled=True)
    assert err.value.status == mg.MG_ERR_CUDA and "gave up" in str(err.value)
    y = mg.conv3d(bf(x), bf(wt), torch.from_numpy(b).cuda(), relu=True)
    torch.cuda.synchronize()
    got = y.float().cpu().numpy().astype(np.float64)
    ref = np.maximum(U.conv3d(x, wt, b.astype(np.float64)), 0.0)
    assert np.all(np.abs(got - ref) <= 2.0**-8 * np.abs(ref) + 1e-4 * np.abs(ref).max())


@pytest.mark.parametrize("c1,c2,cout,relu", [
    (16, 0, 16, True),     # resident weights, four stages
    (32, 32, 32, False),   # concatenated input, streamed weights
    (48, 0, 48, True),     # three stages
    (64, 0, 64, True),     # two stages
    (16, 0, 64, False),
])
def test_conv3d_persistent_matches_oracle(mg, c1, c2, cout, relu):
    """A volume large enough for the persistent kernel (540 tiles of 8 x 16 x
    2 voxels on at most one CTA per SM, so each CTA runs several tiles
    through both accumulators and around its stage ring), ragged in every
    direction against the tile."""
    rng = np.random.default_rng(100 + c1 + c2 + cout)
    n, d, h, w = 1, 40, 44, 70
    x1 = U.to_bf16(rng.standard_normal((n, d, h, w, c1)))
    x2 = U.to_bf16(rng.standard_normal((n, d, h, w, c2))) if c2 else None
    wt = U.to_bf16(rng.standard_normal((cout, 27, c1 + c2)) * 0.1)
    b = rng.standard_normal(cout).astype(np.float32)
    y = mg.conv3d(bf(x1), bf(wt), torch.from_numpy(b).cuda(), None if x2 is None else bf(x2), relu)
    torch.cuda.synchronize()
    got = y.float().cpu().numpy().astype(np.float64)
    xin = x1 if x2 is None else np.concatenate([x1, x2], axis=-1)
    ref = U.conv3d(xin, wt, b.astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0.0)
    assert np.all(np.abs(got - ref) <= 2.0**-8 * np.abs(ref) + 1e-4 * np.abs(ref).max())


@pytest.mark.parametrize("cout,c1,c2,shape", [
    (16, 16, 0, (2, 4, 6, 9)),      # ragged against the 8 x 4 x 4 voxel box
    (48, 48, 48, (2, 4, 6, 9)),     # concatenated input
    (64, 64, 0, (2, 4, 6, 9)),
    (32, 16, 0, (2, 4, 6, 9)),
    (96, 32, 16, (1, 5, 7, 10)),    # widest output
    (16, 16, 0, (2, 32, 32, 32)),   # several boxes per CTA: both stages reused
    (16, 128, 0, (1, 4, 5, 9)),     # 216 atoms fill the last M-tile: the ones get their own
])
def test_wgrad_matches_oracle(mg, cout, c1, c2, shape):
    """Weight and bias gradients on the tensor cores against the oracle's
    plain per-tap products (FP32 sums in a run-dependent order)."""
    rng = np.random.default_rng(cout * 7 + c1)
    n, d, h, w = shape
    x1 = U.to_bf16(rng.standard_normal((n, d, h, w, c1)))
    x2 = U.to_bf16(rng.standard_normal((n, d, h, w, c2))) if c2 else None
    dy = U.to_bf16(rng.standard_normal((n, d, h, w, cout)))
    dw, db = mg.conv3d_wgrad(bf(dy), bf(x1), None if x2 is None else bf(x2), bias=True)
    dw, db = dw.cpu().numpy(), db.cpu().numpy()
    xin = x1 if x2 is None else np.concatenate([x1, x2], axis=-1)
    _, ref, refb = U.conv3d_backward(xin, np.zeros((cout, 27, c1 + c2)), dy)
    assert np.abs(dw - ref).max() <= 1e-5 * np.abs(ref).max()
    # each |sum| is at most the sum of |dy|: FP32 rounding of that many terms
    bound = np.abs(dy).reshape(-1, cout).sum(axis=0)
    assert np.all(np.abs(db - refb) <= 1e-6 * bound + 1e-6)


def _batch(rng, n, s):
    rho = rng.standard_normal((n, s, s, s))
    prev = np.cumsum(rng.standard_normal((n, s, s, s)), axis=1) * 0.1
    phi = prev + 0.05 * rng.standard_normal((n, s, s, s)) + 0.02 * rho
    return rho, prev, phi


def _cuda64(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,s", [(2, 16), (1, 48)])
def test_network_gradients_match_oracle(mg, n, s):
    """Loss and every layer's weight gradient of the whole U-Net against the
    oracle with BF16 storage emulated; at 48^3 the level-0 convolutions and
    their input gradients (one of them split into two outputs) run on the
    persistent kernel."""
    rng = np.random.default_rng(5)
    net = mg.UNet(seed=3)
    params = net.get_params()
    params[-17:-1] = 0.3 * rng.standard_normal(16)  # non-zero head so every layer gets gradient
    params[-1] = 0.05
    net.set_params(params)
    net.set_scales(0.8, 1.2, 4.0)
    rho, prev, phi = _batch(rng, n, s)
    g, loss = net.grads(_cuda64(rho), _cuda64(prev), _cuda64(phi))
    p = U.unpack(params.astype(np.float64))
    ref_loss, G = U.loss_and_grads(p, rho, prev, phi, (0.8, 1.2, 4.0), bf16=True)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    gd = U.unpack(g.astype(np.float64))
    for name, co, ci in U.layer_shapes() + [("head", 1, 16)]:
        for part in (".w", ".b"):
            a, b = gd[name + part].ravel(), G[name + part].ravel()
            err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert err <= 0.05, (name + part, err)
    net.close()


def test_training_reduces_loss_and_save_load_roundtrip(mg, tmp_path):
    rng = np.random.default_rng(6)
    net = mg.UNet(seed=1)
    net.set_scales(1.0, 1.0, 5.0)
    rho_np, prev_np, _ = _batch(rng, 2, 16)
    phi_np = prev_np + 0.05 * rho_np  # a learnable change
    rho, prev, phi = _cuda64(rho_np), _cuda64(prev_np), _cuda64(phi_np)
    losses = [net.train_step(rho, prev, phi, lr=2e-3) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0]
    path = tmp_path / "w.bin"
    net.save(path)
    g1 = net.predict(rho, prev)
    net2 = mg.UNet(seed=99)
    net2.load_file(path)
    assert net2.scales() == (1.0, 1.0, 5.0)
    g2 = net2.predict(rho, prev)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    net.close()
    net2.close()


def test_untrained_network_predicts_previous_potential(mg):
    """The head starts at zero: the network's candidate is phi_prev exactly,
    so both candidates of the judged warm start are phi_prev after the same
    nu1 = 2 red-black sweeps, it accepts the network's (equal residual), and
    the guess equals the oracle's two sweeps of phi_prev."""
    import oracle

    n = 32
    rng = np.random.default_rng(7)
    from paper_1809_08857_gb300 import workloads as W

    rho_np, prev_np = W.gaussian_blobs(n, 1), rng.standard_normal((n, n, n))
    rho, prev = _cuda64(rho_np), _cuda64(prev_np)
    net = mg.UNet(seed=2)
    s = mg.Solver((n, n, n), 1.0 / n, precision=1, nu1=2)
    s.warmstart_attach(net)
    guess, used = s.warmstart_predict(rho, prev)
    torch.cuda.synchronize()
    assert used
    P = oracle.poisson((n, n, n), 1.0 / n)
    ref = prev_np
    for _ in range(2):
        ref = P.rbgs(rho_np / oracle.EPS0, P.rbgs(rho_np / oracle.EPS0, ref, 0), 1)
    assert oracle.rel_l2(guess.cpu().numpy(), ref) <= 1e-13
    s.close()
    net.close()
