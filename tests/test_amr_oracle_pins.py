"""Pins of the composite AMR oracle (oracle/amr.py) against facts fixed by the
mathematics, independent of the oracle's own code: interpolation exactness on
monomials, exactness of the composite operator for quadratics (every valid
cell away from the domain boundary, three levels), discrete conservation of
the refluxed fluxes, the single-grid oracle when nothing is refined, and
second-order convergence of the composite solution."""
import numpy as np
import pytest

import oracle
from oracle import amr

NEUMANN = (1,) * 6


def test_normal_ghost_weights_are_the_lagrange_values():
    """The quadratic through (x = +h: coarse, -h/2: first fine, -3h/2: second
    fine) at x = +h/2 reproduces 1, x, x^2."""
    wc, w1, w2 = amr.ghost_normal_weights()
    np.testing.assert_allclose((wc, w1, w2), (8 / 15, 2 / 3, -1 / 5), rtol=0, atol=1e-15)
    for p in range(3):
        val = wc * 1.0 ** p + w1 * (-0.5) ** p + w2 * (-1.5) ** p
        assert abs(val - 0.5 ** p) < 1e-14


@pytest.mark.parametrize("s1,s2", [(0.25, 0.25), (-0.25, 0.25), (0.25, -0.25), (-0.25, -0.25)])
def test_tangential_weights_reproduce_quadratics(s1, s2):
    """Weighted sum over the 3 x 3 coarse cells of every monomial of degree
    <= 2 in the face plane equals the monomial at (s1, s2)."""
    for p1, p2 in [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1)]:
        val = sum(amr.tangential_weight(a, b, s1, s2) * a ** p1 * b ** p2
                  for a in (-1, 0, 1) for b in (-1, 0, 1))
        assert abs(val - s1 ** p1 * s2 ** p2) < 1e-15


def three_level(N=16, alpha=0.7, beta=None, bc_kind=NEUMANN, mask=None, mask_value=None):
    boxes = [(1, (8, 8, 8), (12, 16, 8)), (1, (6, 20, 18), (8, 6, 10)), (2, (20, 20, 20), (8, 8, 8))]
    return amr.Hierarchy((N, N, N), 1.0 / N, boxes, alpha=alpha, beta=beta, bc_kind=bc_kind,
                         mask=mask, mask_value=mask_value), boxes


def test_hierarchy_links():
    H, _ = three_level()
    assert [b.parent for b in H.boxes] == [None, 0, 0, 1]
    assert [b.level for b in H.boxes] == [0, 1, 1, 2]
    # cells of box 0 covered by the two level-1 footprints
    assert H.covered(0).sum() == 6 * 8 * 4 + 4 * 3 * 5
    assert H.covered(1).sum() == 4 ** 3


def test_quadratic_is_exact_on_every_level():
    """-div(beta grad q) = -2 beta (a + b + c) for a quadratic q with all six
    second-order terms: the composite rows (same-level, coarse-fine ghost and
    refluxed coarse rows) are exact for it away from the domain boundary."""
    N = 16
    beta_c = 2.5
    boxes_shapes = [(N, N, N), (12, 16, 8), (8, 6, 10), (8, 8, 8)]
    H, _ = three_level(N, beta=[np.full(s, beta_c) for s in boxes_shapes])
    a, b, c, d, e, f = 0.3, -0.7, 1.1, 0.5, -0.9, 0.4

    def q(z, y, x):
        return (a * x * x + b * y * y + c * z * z + d * x * y + e * y * z + f * x * z
                + 0.2 * x - 0.3 * y + 0.1 * z + 0.05)

    u = [q(*H.cell_centres(k)) for k in range(len(H.boxes))]
    Au = H.apply(u)
    checked = 0
    for k in range(len(H.boxes)):
        z, y, x = H.cell_centres(k)
        exact = 0.7 * q(z, y, x) - 2.0 * beta_c * (a + b + c)
        v = H.valid(k)
        if k == 0:
            inner = np.zeros_like(v)
            inner[1:-1, 1:-1, 1:-1] = True
            v &= inner
        scale = 2.0 * beta_c / H.boxes[k].h ** 2
        assert np.abs(Au[k][v] - exact[v]).max() <= 1e-12 * scale
        checked += v.sum()
    assert checked > 0.75 * H.n


def test_constant_is_a_null_vector_of_the_flux_part():
    """With Neumann faces and alpha = 0 every row sums to zero (a constant has
    zero flux everywhere, coarse-fine ghosts included)."""
    rng = np.random.default_rng(3)
    shapes = [(16, 16, 16), (12, 16, 8), (8, 6, 10), (8, 8, 8)]
    H, _ = three_level(alpha=0.0, beta=[np.exp(rng.standard_normal(s)) for s in shapes])
    A, lift, _ = H.assemble()
    assert np.abs(A @ np.ones(H.n)).max() <= 1e-12 * np.abs(A).max()
    assert not lift.any()


def test_refluxing_conserves_the_total_flux():
    """Neumann faces, alpha = 0, random beta on all levels, random u: the
    volume-weighted sum of A u over the valid cells vanishes (the flux out of
    every coarse cell enters the fine cells exactly)."""
    rng = np.random.default_rng(4)
    shapes = [(16, 16, 16), (12, 16, 8), (8, 6, 10), (8, 8, 8)]
    H, _ = three_level(alpha=0.0, beta=[np.exp(rng.standard_normal(s)) for s in shapes])
    u = [rng.standard_normal(s) for s in shapes]
    y = H.gather(H.apply(u)) * H.volumes()
    assert abs(y.sum()) <= 1e-13 * np.abs(y).sum()


def test_without_refined_boxes_it_is_the_single_grid_operator():
    """No refined boxes: residual, ||b||, homogeneous operator and solution
    equal those of the single-grid oracle (variable beta, electrodes,
    mixed Dirichlet/Neumann faces, alpha > 0)."""
    rng = np.random.default_rng(5)
    N = 16
    mask = np.zeros((N, N, N), np.uint8)
    mask[3:6, 4:9, 2:5] = 1
    mv = rng.standard_normal((N, N, N))
    beta = np.exp(rng.standard_normal((N, N, N)))
    bk = (0, 1, 1, 0, 0, 0)
    bv = (0.3, 0.0, 0.0, -0.2, 1.0, 0.5)
    H = amr.Hierarchy((N, N, N), 1.0 / N, [], alpha=2.0, beta=[beta], mask=mask,
                      mask_value=mv, bc_kind=bk, bc_value=bv)
    P = oracle.Problem((N, N, N), 1.0 / N, 2.0, beta, mask, bk, bv)
    u = rng.standard_normal((N, N, N))
    u[mask != 0] = mv[mask != 0]
    f = rng.standard_normal((N, N, N))
    r1, n1 = P.residual(f, u)
    r2, n2 = H.residual([f], [u])
    np.testing.assert_allclose(r2[0], r1, rtol=0, atol=1e-12 * np.abs(r1).max())
    assert abs(n1 - n2) <= 1e-12 * n1
    assert abs(P.rhs_norm(f, np.where(mask != 0, mv, 0.0)) - H.rhs_norm([f])) <= 1e-12 * n1
    a1 = P.apply(u, homog=True)
    np.testing.assert_allclose(H.apply([u])[0], a1, rtol=0, atol=1e-12 * np.abs(a1).max())
    ref, _, _, _ = P.solve(f, u0=np.where(mask != 0, mv, 0.0))
    assert oracle.rel_l2(H.solve([f])[0], ref, mask) <= 1e-11


def sine_error(N):
    h = 1.0 / N
    H = amr.Hierarchy((N, N, N), h, [(1, (N // 2, N // 2, N // 2), (N, N, N))],
                      bc_kind=(0,) * 6)
    ex, fs = [], []
    for q in range(len(H.boxes)):
        z, y, x = H.cell_centres(q)
        e = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        ex.append(e)
        fs.append(3.0 * np.pi ** 2 * e)
    d = H.gather(H.solve(fs)) - H.gather(ex)
    return np.abs(d).max(), np.sqrt(np.sum(H.volumes() * d * d))


def test_composite_solution_is_second_order():
    """-lap u = 3 pi^2 sin sin sin, u = 0 on the boundary, a refined central
    box: halving h divides the error by about 4 (max and L2 norms)."""
    e8, e16 = sine_error(8), sine_error(16)
    assert e16[0] < 0.3 * e8[0] and e16[1] < 0.3 * e8[1]
    assert e8[0] / e16[0] > 3.5 and e8[1] / e16[1] > 3.5


def test_average_down_of_a_linear_function_is_the_coarse_value():
    H, _ = three_level()

    def lin(z, y, x):
        return 1.5 * x - 0.25 * y + 2.0 * z - 0.3

    u = [lin(*H.cell_centres(k)) for k in range(len(H.boxes))]
    junk = [np.where(H.covered(k), 1e3, u[k]) for k in range(len(H.boxes))]
    back = H.average_down(junk)
    for k in range(len(H.boxes)):
        np.testing.assert_allclose(back[k], u[k], rtol=0, atol=1e-13)


@pytest.mark.parametrize("boxes", [
    [(1, (0, 8, 8), (8, 8, 8))],                              # touches the domain boundary
    [(1, (8, 8, 8), (8, 8, 8)), (1, (16, 8, 8), (8, 8, 8))],  # siblings too close
    [(1, (7, 8, 8), (8, 8, 8))],                              # odd corner
    [(2, (20, 20, 20), (8, 8, 8))],                           # no parent
    [(1, (8, 8, 8), (12, 16, 8)), (2, (18, 18, 18), (4, 4, 4))],  # one cell inside a refined parent
])
def test_bad_hierarchies_are_rejected(boxes):
    with pytest.raises(ValueError):
        amr.Hierarchy((16, 16, 16), 1.0 / 16, boxes)


def test_electrode_next_to_a_refined_box_is_rejected():
    mask = np.zeros((16, 16, 16), np.uint8)
    mask[8, 3, 8] = 1  # inside the grown footprint of the box below
    with pytest.raises(ValueError):
        amr.Hierarchy((16, 16, 16), 1.0 / 16, [(1, (8, 8, 8), (8, 8, 8))], mask=mask)
