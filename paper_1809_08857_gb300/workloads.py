"""Seeded synthetic inputs for the elliptic solves (shared by the oracle tests
and the CUDA path).  This module holds no solver arithmetic: it only draws
charge densities, permittivities, sources and electrode masks, as numpy
arrays of shape (nz, ny, nx) on the unit cube with h = 1/n.

The shapes follow the paper's geometries (rod-plane and needle-plane gaps with
a live top face and a grounded bottom face, Secs. 3 and 4) and the charged
filaments of a propagating streamer; the kinetic data and Perlin table the
paper uses are not available, so these synthetic fields stand in for them.
"""
import numpy as np

EPS0 = 8.8541878128e-12  # F/m, CODATA 2018

# Boundary conditions of the gap: Neumann on the four sides, phi = 0 at z = 0
# (grounded plane) and phi = 1 at z = 1 (live face).  Faces -x,+x,-y,+y,-z,+z;
# kind 0 = Dirichlet, 1 = Neumann.
GAP_BC_KIND = (1, 1, 1, 1, 0, 0)
GAP_BC_VALUE = (0.0, 0.0, 0.0, 0.0, 0.0, 1.0)


def centres(n):
    """Cell-centre coordinates (i + 1/2) h of an n-cell axis on [0, 1]."""
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def gaussian_blobs(n, seed, nblobs=4, width=0.05):
    """Space charge rho (C/m^3) = eps0 * sum_k a_k exp(-|x - c_k|^2 / (2 w^2)),
    centres uniform in [0.2, 0.8]^3, amplitudes a_k ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.2, 0.8, size=(nblobs, 3))
    a = rng.standard_normal(nblobs)
    x = centres(n)
    rho = np.zeros((n, n, n))
    for k in range(nblobs):
        ex = np.exp(-((x - c[k, 0]) ** 2) / (2 * width**2))
        ey = np.exp(-((x - c[k, 1]) ** 2) / (2 * width**2))
        ez = np.exp(-((x - c[k, 2]) ** 2) / (2 * width**2))
        rho += a[k] * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return rho * EPS0


def dielectric_slab(n, z_top=0.2, eps_slab=4.0):
    """Relative permittivity eps_slab for cell centres with z < z_top, else 1."""
    return dielectric_slab_box((n, n, n), 1.0 / n, (0.0, 0.0, 0.0), z_top, eps_slab)


def dielectric_slab_box(shape, h, origin, z_top=0.2, eps_slab=4.0):
    """The dielectric slab sampled on a box (shape (nz, ny, nx), cell size h,
    lower corner origin (x, y, z))."""
    z = origin[2] + (np.arange(shape[0]) + 0.5) * h
    eps = np.ones(shape)
    eps[z < z_top] = eps_slab
    return eps


def _shell_distance_slab(x, y, z, axis_xy, z0, z1, radius):
    """Distance from points of one z plane to the open capsule surface: a
    cylinder of the given radius from z0 to z1 along z, closed by a
    hemispherical head at z1, open at z0."""
    r = np.sqrt((x[None, :] - axis_xy[0]) ** 2 + (y[:, None] - axis_xy[1]) ** 2)
    if z > z1:
        return np.abs(np.sqrt(r**2 + (z - z1) ** 2) - radius)
    if z >= z0:
        return np.abs(r - radius)
    return np.sqrt((r - radius) ** 2 + (z0 - z) ** 2)


def streamer_shell(n, seed, radius=0.02, z0=0.4, z1=0.8, axis_xy=(0.5, 0.5),
                   amplitude=1e-3, noise=0.1):
    """Charged shell of a streamer channel: cells within h of the surface of a
    cylinder (radius, from z0 to z1 on the axis) with a hemispherical head.
    Density amplitude * eps0 / h^2 times a lognormal factor exp(noise * xi),
    xi ~ N(0, 1) per shell cell (drawn in index order)."""
    return streamer_shell_box((n, n, n), 1.0 / n, (0.0, 0.0, 0.0), seed, radius, z0, z1,
                              axis_xy, amplitude, noise)


def streamer_shell_box(shape, h, origin, seed, radius=0.02, z0=0.4, z1=0.8, axis_xy=(0.5, 0.5),
                       amplitude=1e-3, noise=0.1, thickness=None):
    """The streamer shell sampled on a box of the given shape (nz, ny, nx),
    cell size h and lower corner origin (x, y, z): cells within t of the
    surface carry amplitude * eps0 / t^2 * exp(noise * xi), t = thickness
    (default h; a fixed t gives one shell sampled alike on every level of an
    AMR hierarchy)."""
    idx, val = streamer_shell_cells(shape, h, origin, seed, radius, z0, z1, axis_xy, amplitude,
                                    noise, thickness)
    rho = np.zeros(shape)
    rho.reshape(-1)[idx] = val
    return rho


def streamer_shell_cells(shape, h, origin, seed, radius=0.02, z0=0.4, z1=0.8,
                         axis_xy=(0.5, 0.5), amplitude=1e-3, noise=0.1, thickness=None):
    """The cells of streamer_shell_box as (flat indices in (k, j, i) order,
    values incl. eps0), without a dense array: only the columns within
    radius + t + h of the axis can hold shell cells, so the distance test
    runs on that window of every plane; xi ~ N(0, 1) is drawn per shell cell
    in index order."""
    t = h if thickness is None else float(thickness)
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    x = origin[0] + (np.arange(nx) + 0.5) * h
    y = origin[1] + (np.arange(ny) + 0.5) * h
    z = origin[2] + (np.arange(nz) + 0.5) * h
    reach = radius + t + h
    ix = np.nonzero(np.abs(x - axis_xy[0]) <= reach)[0]
    iy = np.nonzero(np.abs(y - axis_xy[1]) <= reach)[0]
    hit = []
    if len(ix) and len(iy):
        x0, y0 = int(ix[0]), int(iy[0])
        xs, ys = x[x0:ix[-1] + 1], y[y0:iy[-1] + 1]
        for k in range(nz):
            jj, ii = np.nonzero(_shell_distance_slab(xs, ys, z[k], axis_xy, z0, z1, radius) <= t)
            if len(jj):
                hit.append(((k * ny + (jj + y0)) * nx + (ii + x0)).astype(np.int64))
    idx = np.concatenate(hit) if hit else np.zeros(0, dtype=np.int64)
    val = amplitude / t**2 * np.exp(noise * rng.standard_normal(len(idx)))
    return idx, val * EPS0


def ionization_source(n, seed, sigma_cells=2.0):
    """Non-negative photo-emission source S for the radiative-transfer solves:
    the magnitude of the streamer-shell charge (in units of eps0), smoothed by
    a Gaussian of width sigma_cells cells."""
    from scipy.ndimage import gaussian_filter

    shell = np.abs(streamer_shell(n, seed)) / EPS0
    s = gaussian_filter(shell, sigma=sigma_cells, mode="constant", truncate=4.0)
    return np.maximum(s, 0.0)


def subbox_layout(n_parent, count, seed, sizes=(32, 48, 64, 96, 128), lo=0.1, hi=0.9):
    """Refined sub-boxes (ratio 2) of a parent grid of n_parent^3 cells on the
    unit cube: sizes (fine cells per side) drawn from `sizes`, lower corners
    uniform so that each box lies inside [lo, hi]^3, aligned to parent cells.
    Returns a list of (origin (x, y, z) in parent cells, dims (x, y, z) in fine
    cells)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(rng.choice(sizes))
        half = m // 2
        lo_c = int(np.ceil(lo * n_parent))
        hi_c = int(np.floor(hi * n_parent)) - half
        o = rng.integers(lo_c, hi_c + 1, size=3)
        out.append(((int(o[0]), int(o[1]), int(o[2])), (m, m, m)))
    return out


def streamer_amr_layout(n0):
    """Nested refined boxes (ratio 2) around the streamer channel and head of
    streamer_shell on a base grid of n0^3 cells (n0 a multiple of 64), as the
    refinement around streamer heads and space-charge layers of Sec. 4:
      level 1 (h0/2): x, y in 0.5 +- 1/16, z in [0.34375, 0.875];
      level 2 (h0/4): x, y in 0.5 +- 1/32, z in [0.703125, 0.859375];
      level 3 (h0/8): x, y in 0.5 +- 1/64, z in [0.765625, 0.8359375].
    Returns (level, lo, shape) per box, lo and shape in (z, y, x) cells of
    that level."""
    spec = ((1, 0.0625, 0.34375, 0.875), (2, 0.03125, 0.703125, 0.859375),
            (3, 0.015625, 0.765625, 0.8359375))
    boxes = []
    for lev, half, z0, z1 in spec:
        m = n0 * 2 ** lev
        lo_xy = int(round((0.5 - half) * m))
        n_xy = int(round(2 * half * m))
        lo_z = int(round(z0 * m)) // 2 * 2
        n_z = (int(round(z1 * m)) - lo_z) // 2 * 2
        boxes.append((lev, (lo_z, lo_xy, lo_xy), (n_z, n_xy, n_xy)))
    return boxes


def amr_box_origin(h0, box):
    """Lower corner (x, y, z) and cell size of a refined box (level, lo, shape)."""
    lev, lo, _ = box
    h = h0 / 2 ** lev
    return (lo[2] * h, lo[1] * h, lo[0] * h), h


def needle_mask(n, tip_z=0.8, tip_radius_cells=5.0, half_angle_deg=10.0, axis_xy=(0.5, 0.5)):
    """Electrode cells of a needle from the top face down to a hyperboloid tip:
    r^2 <= 2 R d + d^2 tan^2(theta), d = z - tip_z >= 0, R = tip radius."""
    h = 1.0 / n
    R = tip_radius_cells * h
    t2 = np.tan(np.deg2rad(half_angle_deg)) ** 2
    x = centres(n)
    r2 = (x[None, :] - axis_xy[0]) ** 2 + (x[:, None] - axis_xy[1]) ** 2
    mask = np.zeros((n, n, n), dtype=np.uint8)
    for k in range(n):
        d = x[k] - tip_z
        if d >= 0:
            mask[k] = r2 <= 2 * R * d + d * d * t2
    return mask


def branching_channels(seed, tip=(0.5, 0.5, 0.8), nchan=3):
    """Axis segments of streamer channels leaving a needle tip: nchan primary
    channels going down from the tip at tilt U[10, 30] degrees from -z and
    azimuth 2 pi c / nchan + U[-0.3, 0.3], length U[0.12, 0.2]; each splits at
    its end into two daughters of length U[0.08, 0.15], turned by +-U[10, 25]
    degrees in the azimuth.  Returns a list of (start, end) points (x, y, z)."""
    rng = np.random.default_rng(seed)
    segs = []

    def direction(tilt, az):
        return np.array([np.sin(tilt) * np.cos(az), np.sin(tilt) * np.sin(az), -np.cos(tilt)])

    p0 = np.asarray(tip, dtype=np.float64)
    for c in range(nchan):
        tilt = np.deg2rad(rng.uniform(10.0, 30.0))
        az = 2.0 * np.pi * c / nchan + rng.uniform(-0.3, 0.3)
        p1 = p0 + rng.uniform(0.12, 0.2) * direction(tilt, az)
        segs.append((p0, p1))
        for sgn in (-1.0, 1.0):
            daz = sgn * np.deg2rad(rng.uniform(10.0, 25.0))
            dtilt = np.deg2rad(rng.uniform(-5.0, 5.0))
            p2 = p1 + rng.uniform(0.08, 0.15) * direction(tilt + dtilt, az + daz)
            segs.append((p1, p2))
    return segs


def channel_shell_cells(n, seed, radius=0.01, amplitude=1e-3, noise=0.1):
    """Charged shells of the branching channels of branching_channels(seed) on
    an n^3 grid (h = 1/n): cells whose centre lies within h of the lateral
    surface of the cylinder of the given radius around any segment (distance
    to the segment's axis within radius +- h).  Returns (flat cell indices in
    (k, j, i) order, sorted, and the density amplitude * eps0 / h^2 *
    exp(noise * xi), xi ~ N(0, 1) drawn in index order), so that large grids
    need no dense array on the host."""
    h = 1.0 / n
    rng = np.random.default_rng(seed + 1000)
    hit = []
    for a, b in branching_channels(seed):
        lo = np.maximum(np.floor((np.minimum(a, b) - radius - 2 * h) * n).astype(int), 0)
        hi = np.minimum(np.ceil((np.maximum(a, b) + radius + 2 * h) * n).astype(int), n)
        x = (np.arange(lo[0], hi[0]) + 0.5) * h
        y = (np.arange(lo[1], hi[1]) + 0.5) * h
        ab = b - a
        L2 = float(ab @ ab)
        for k in range(lo[2], hi[2]):
            z = (k + 0.5) * h
            px = x[None, :] - a[0]
            py = y[:, None] - a[1]
            pz = z - a[2]
            t = np.clip((px * ab[0] + py * ab[1] + pz * ab[2]) / L2, 0.0, 1.0)
            dx = px - t * ab[0]
            dy = py - t * ab[1]
            dz = pz - t * ab[2]
            d = np.sqrt(dx * dx + dy * dy + dz * dz)
            jj, ii = np.nonzero(np.abs(d - radius) <= h)
            if len(jj):
                hit.append(((k * n + (jj + lo[1])) * n + (ii + lo[0])).astype(np.int64))
    idx = np.unique(np.concatenate(hit)) if hit else np.zeros(0, dtype=np.int64)
    val = amplitude / h**2 * np.exp(noise * rng.standard_normal(len(idx)))
    return idx, val * EPS0


def helmholtz_kappas():
    """Inverse absorption lengths of the three photon groups, kappa L = 10, 100, 1000."""
    return (10.0, 100.0, 1000.0)
