"""The seeded synthetic inputs follow their stated recipe (CPU only): seeds
reproduce, the dielectric slab covers the cell layers whose centres lie below
z = 0.2, the streamer shell is the band of cells within h of the capsule
surface with lognormal amplitudes, the refined boxes nest as the composite
solver requires, sub-boxes stay inside [0.1, 0.9], the needle is the stated
hyperboloid, and the channel shells lie within h of the channel cylinders."""
import numpy as np

from paper_1809_08857_gb300 import workloads as W


def test_seeds_reproduce_and_differ():
    a, b, c = W.gaussian_blobs(16, 3), W.gaussian_blobs(16, 3), W.gaussian_blobs(16, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    s1, s2 = W.streamer_shell(32, 7), W.streamer_shell(32, 7)
    assert np.array_equal(s1, s2) and not np.array_equal(s1, W.streamer_shell(32, 8))


def test_dielectric_slab_layers():
    for n in (16, 64, 512):
        z = (np.arange(n) + 0.5) / n
        layers = int((z < 0.2).sum())
        eps = W.dielectric_slab_box((n, 2, 2), 1.0 / n, (0.0, 0.0, 0.0))
        assert np.all(eps[:layers] == 4.0) and np.all(eps[layers:] == 1.0)
    assert int(((np.arange(512) + 0.5) / 512 < 0.2).sum()) == 102   # layers 0..101 at 512^3


def test_streamer_shell_is_the_band_within_h_of_the_capsule():
    n = 64
    h = 1.0 / n
    rho = W.streamer_shell(n, 0) / W.EPS0
    k, j, i = np.nonzero(rho)
    x, y, z = (i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h
    r = np.hypot(x - 0.5, y - 0.5)
    d = np.where(z > 0.8, np.abs(np.hypot(r, z - 0.8) - 0.02),
                 np.where(z >= 0.4, np.abs(r - 0.02), np.hypot(r - 0.02, 0.4 - z)))
    assert len(d) > 100 and np.all(d <= h + 1e-15)
    amp = rho[k, j, i] * h * h / 1e-3          # exp(0.1 xi), xi ~ N(0, 1)
    assert np.all(amp > 0) and abs(np.log(amp).std() - 0.1) < 0.03
    assert np.all(W.ionization_source(32, 0) >= 0.0)


def test_streamer_amr_boxes_nest():
    for n0 in (64, 128, 256):
        boxes = W.streamer_amr_layout(n0)
        assert [b[0] for b in boxes] == [1, 2, 3]
        parent = (0, (0, 0, 0), (n0, n0, n0))
        for lev, lo, shape in boxes:
            assert all(v % 2 == 0 for v in lo + shape) and all(s > 0 for s in shape)
            g = 1 if parent[0] == 0 else 2    # parent cells of margin (2 inside a refined box)
            plo, pshape = parent[1], parent[2]
            for a in range(3):
                assert lo[a] >= 2 * (plo[a] + g)
                assert lo[a] + shape[a] <= 2 * (plo[a] + pshape[a] - g)
            parent = (lev, lo, shape)


def test_subboxes_stay_inside():
    n = 256
    for (o, dims) in W.subbox_layout(n, 16, 0):
        m = dims[0]
        assert dims == (m, m, m) and m in (32, 48, 64, 96, 128)
        for a in range(3):
            assert o[a] >= np.ceil(0.1 * n) and o[a] + m // 2 <= np.floor(0.9 * n)


def test_needle_is_the_hyperboloid():
    n = 64
    mask = W.needle_mask(n)
    z = (np.arange(n) + 0.5) / n
    assert not mask[z < 0.8].any() and mask[-1].any()   # nothing below the tip, up to the top
    R, t2 = 5.0 / n, np.tan(np.deg2rad(10.0)) ** 2
    x = (np.arange(n) + 0.5) / n
    r2 = (x[None, :] - 0.5) ** 2 + (x[:, None] - 0.5) ** 2
    for k in np.nonzero(z >= 0.8)[0]:
        d = z[k] - 0.8
        assert np.array_equal(mask[k].astype(bool), r2 <= 2 * R * d + d * d * t2)
    widths = mask.reshape(n, -1).sum(axis=1)
    assert np.all(np.diff(widths[z >= 0.8]) >= 0)       # the needle widens upwards


def test_channel_shells_lie_on_the_cylinders():
    n = 128
    h = 1.0 / n
    idx, val = W.channel_shell_cells(n, 0)
    assert len(idx) > 0 and np.all(np.diff(idx) > 0) and np.all(val > 0)
    k, rem = np.divmod(idx, n * n)
    j, i = np.divmod(rem, n)
    p = np.stack([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h], axis=1)
    best = np.full(len(idx), np.inf)
    for a, b in W.branching_channels(0):
        ab = b - a
        t = np.clip(((p - a) @ ab) / (ab @ ab), 0.0, 1.0)
        dist = np.linalg.norm(p - (a + t[:, None] * ab), axis=1)
        best = np.minimum(best, np.abs(dist - 0.01))
    assert np.all(best <= h + 1e-12)
