"""Composite operator of a ratio-2 adaptive (AMR) hierarchy of cell-centred
boxes, and its exact discrete solution.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and never imports it.

The paper solves its elliptic equations (Eqs. 2-3) with second-order
cell-centred finite volumes on patch-based AMR grids (Sec. 2 items (ii)-(iii);
the grids of Secs. 3 and 4 are nested Cartesian patches made by the
Berger-Rigoutsos algorithm).  It does not print how a level meets the level
below it; the composite discretisation written here is the reading taken
(the standard one for cell-centred AMR: refluxing of Berger and Colella and
the quadratic coarse-fine interpolation of Martin and Cartwright):

* Hierarchy.  Level 0 is one box covering the domain, cells of size h.  A
  level-l box (l >= 1) has cells of size h / 2^l; it is given by its lower
  corner and shape in level-l cell indices counted from the domain's low
  corner (both even, so that it covers whole cells of level l - 1: its
  footprint).  Its footprint grown by one cell must lie inside one box of
  level l - 1 (the parent) -- grown by two cells when the parent is itself
  a refined box, whose own coarse-fine ghosts read its two outermost cell
  layers --, must not reach another box of level l, and on level 0 must
  hold no electrode cell.

* Unknowns.  The valid cells: cells of a box not covered by a box of the next
  level; electrode cells (level 0) are excluded and hold their given value.

* Rows.  Every valid free cell c of size h_c obeys the balance
      alpha u_c - (1/h_c) sum over its six faces of F = f_c,
  F = beta du/dn across the face (outward).
    - Two cells of one level: F = hmean(beta_c, beta_n) (u_n - u_c) / h_c
      (hmean the harmonic mean).  Electrode neighbour: beta_c, value at its
      centre.  Domain face: Dirichlet ghost 2 g - u_c, Neumann ghost u_c.
    - Fine cell f on the boundary of its box: the outside value is a ghost g
      (below), F = hmean(beta_f, beta_C) (g - u_f) / h_f, where C is the
      coarse valid cell that holds the ghost's centre.
    - Coarse valid cell C next to a covered cell: F on that face is the mean
      of the four fine fluxes through it (the fine side's F, sign reversed),
      so that what leaves C enters the fine cells exactly.

* Ghost g of the fine cell f across a coarse-fine face: a quadratic along the
  face normal through u_f (distance h_f/2 inside the face), the next fine
  cell inward u_f2 (3 h_f / 2 inside) and a coarse value cc on the normal
  line at the centre of C (h_f outside):
      g = (8/15) cc + (2/3) u_f - (1/5) u_f2,
  the Lagrange weights of the three points at the ghost centre (h_f/2
  outside).  cc is the two-dimensional quadratic through the 3 x 3 coarse
  cells around C in the face plane, with the mixed term, evaluated at the
  ghost's offset (s1, s2) = (+-1/4, +-1/4) coarse cells from C's centre:
      cc = u_C + s1 d1 + s2 d2 + s1^2/2 d11 + s2^2/2 d22 + s1 s2 d12,
  d1, d11 centred first and second differences, d12 the four-corner mixed
  difference.

Arrays are numpy of shape (nz, ny, nx) per box; corners and shapes are given
in (z, y, x) order.  Faces -x, +x, -y, +y, -z, +z; bc_kind 0 = Dirichlet
(value in bc_value), 1 = homogeneous Neumann.

Parity status: pinned by ``tests/test_amr_oracle_pins.py`` (exact for
quadratics away from the domain boundary, flux conservation, the single-grid
oracle when there are no patches, second-order convergence of the composite
solution).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

def hmean(a, b):
    return 2.0 * a * b / (a + b)


def ghost_normal_weights():
    """Lagrange weights (coarse value, first fine cell, second fine cell) of
    the quadratic through positions +h, -h/2, -3h/2 (fine cell size h,
    coarse-fine face at 0) evaluated at the ghost centre +h/2."""
    pts = (1.0, -0.5, -1.5)
    x = 0.5
    w = []
    for a in range(3):
        v = 1.0
        for b in range(3):
            if b != a:
                v *= (x - pts[b]) / (pts[a] - pts[b])
        w.append(v)
    return tuple(w)


def tangential_weight(a, b, s1, s2):
    """Weight of the coarse cell at offset (a, b) in {-1, 0, 1}^2 (face-plane
    axes) in the 2D quadratic with mixed term
        u_C + s1 d1 + s2 d2 + s1^2/2 d11 + s2^2/2 d22 + s1 s2 d12
    (d1 = (u_{+1,0} - u_{-1,0})/2, d11 = u_{+1,0} - 2 u_C + u_{-1,0},
    d12 = (u_{++} - u_{+-} - u_{-+} + u_{--})/4) at offset (s1, s2) coarse
    cells; s1, s2 may be arrays."""
    if a == 0 and b == 0:
        return 1.0 - s1 * s1 - s2 * s2
    if b == 0:
        return s1 * a / 2.0 + s1 * s1 / 2.0
    if a == 0:
        return s2 * b / 2.0 + s2 * s2 / 2.0
    return s1 * s2 * a * b / 4.0


class Box:
    def __init__(self, level, lo, shape, h):
        self.level = int(level)
        self.lo = tuple(int(v) for v in lo)
        self.shape = tuple(int(v) for v in shape)
        self.h = float(h)
        self.parent = None
        self.children = []

    @property
    def hi(self):
        return tuple(a + b for a, b in zip(self.lo, self.shape))

    def footprint(self):
        """(lo, hi) in the parent level's cell indices."""
        return tuple(v // 2 for v in self.lo), tuple(v // 2 for v in self.hi)


def _inside(lo, hi, olo, ohi):
    return all(olo[a] <= lo[a] and hi[a] <= ohi[a] for a in range(3))


def _overlap(lo, hi, olo, ohi):
    return all(lo[a] < ohi[a] and olo[a] < hi[a] for a in range(3))


class Hierarchy:
    """A composite problem alpha u - div(beta grad u) = f on an AMR hierarchy.

    base_shape, h: level-0 box (nz, ny, nx) and cell size.
    boxes: list of (level, lo, shape) of the refined boxes (level >= 1), lo
      and shape in (z, y, x) cell indices of that level.
    beta: None (1 everywhere) or a list with one array (or None) per box,
      level 0 first, then the refined boxes in the given order.
    mask, mask_value: electrode cells of level 0 and their values.
    """

    def __init__(self, base_shape, h, boxes=(), alpha=0.0, beta=None, mask=None,
                 mask_value=None, bc_kind=(0,) * 6, bc_value=(0.0,) * 6):
        self.alpha = float(alpha)
        self.bc_kind = tuple(int(v) for v in bc_kind)
        self.bc_value = tuple(float(v) for v in bc_value)
        self.boxes = [Box(0, (0, 0, 0), base_shape, h)]
        for lev, lo, shape in boxes:
            if lev < 1:
                raise ValueError("refined boxes have level >= 1")
            if any(v % 2 for v in tuple(lo) + tuple(shape)) or min(shape) < 2:
                raise ValueError("refined boxes need even corners and even sizes >= 2")
            self.boxes.append(Box(lev, lo, shape, h / 2 ** lev))
        nb = len(self.boxes)
        self.beta = [None] * nb
        if beta is not None:
            for q, b in enumerate(beta):
                if b is not None:
                    b = np.ascontiguousarray(b, dtype=np.float64)
                    if b.shape != self.boxes[q].shape:
                        raise ValueError("beta of box %d has the wrong shape" % q)
                    self.beta[q] = b
        self.mask = None if mask is None else np.asarray(mask) != 0
        self.mask_value = (np.zeros(base_shape) if mask_value is None
                           else np.asarray(mask_value, dtype=np.float64))
        self._link()
        self._index()

    # ---- structure --------------------------------------------------------
    def _link(self):
        for q, b in enumerate(self.boxes):
            if b.level == 0:
                continue
            flo, fhi = b.footprint()
            glo = tuple(v - 1 for v in flo)
            ghi = tuple(v + 1 for v in fhi)
            # a refined parent's ghosts read its two outermost layers
            g = 1 if b.level == 1 else 2
            par = [p for p, o in enumerate(self.boxes)
                   if o.level == b.level - 1
                   and _inside(tuple(v - g for v in flo), tuple(v + g for v in fhi), o.lo, o.hi)]
            if len(par) != 1:
                raise ValueError("box %d: grown footprint not inside one box of level %d"
                                 % (q, b.level - 1))
            b.parent = par[0]
            self.boxes[par[0]].children.append(q)
            for p, o in enumerate(self.boxes):
                if p != q and o.level == b.level:
                    olo, ohi = o.footprint()
                    if _overlap(glo, ghi, olo, ohi):
                        raise ValueError("boxes %d and %d of level %d are too close"
                                         % (q, p, b.level))
            if b.level == 1 and self.mask is not None:
                if self.mask[glo[0]:ghi[0], glo[1]:ghi[1], glo[2]:ghi[2]].any():
                    raise ValueError("electrode cell under or next to box %d" % q)

    def covered(self, q):
        """Boolean array of the cells of box q covered by its children."""
        b = self.boxes[q]
        cov = np.zeros(b.shape, dtype=bool)
        for c in b.children:
            flo, fhi = self.boxes[c].footprint()
            sl = tuple(slice(flo[a] - b.lo[a], fhi[a] - b.lo[a]) for a in range(3))
            cov[sl] = True
        return cov

    def valid(self, q):
        """Boolean array: valid free cells of box q (the unknowns)."""
        v = ~self.covered(q)
        if q == 0 and self.mask is not None:
            v &= ~self.mask
        return v

    def _index(self):
        self.uid = []
        n = 0
        for q in range(len(self.boxes)):
            v = self.valid(q)
            ids = np.full(v.shape, -1, dtype=np.int64)
            k = int(v.sum())
            ids[v] = np.arange(n, n + k)
            self.uid.append(ids)
            n += k
        self.n = n

    def _beta(self, q):
        b = self.beta[q]
        return np.ones(self.boxes[q].shape) if b is None else b

    # ---- assembly ---------------------------------------------------------
    def assemble(self):
        """(A, lift, E): the sparse matrix over the unknowns, the Dirichlet
        domain-face lift and the sparse coupling E (unknowns x level-0 cells)
        of free cells to electrode values, so that b = f + lift + E g for
        electrode values g, and the operator applied to u (electrode cells
        holding their values) is A u - E u_0."""
        rows, cols, vals = [], [], []
        erows, ecols, evals = [], [], []
        lift = np.zeros(self.n)
        n0 = int(np.prod(self.boxes[0].shape))

        def add(r, c, v):
            rows.append(np.asarray(r).ravel())
            cols.append(np.asarray(c).ravel())
            vals.append(np.broadcast_to(np.asarray(v, dtype=np.float64), np.shape(r)).ravel())

        for q, b in enumerate(self.boxes):
            ids = self.uid[q]
            beta = self._beta(q)
            ih2 = 1.0 / (b.h * b.h)
            cov = self.covered(q)
            cells = np.argwhere(ids >= 0)
            rid = ids[ids >= 0]
            add(rid, rid, self.alpha)
            for ax in range(3):
                for side in (-1, 1):
                    face = 2 * (2 - ax) + (0 if side < 0 else 1)
                    nb = cells.copy()
                    nb[:, ax] += side
                    ins = (nb[:, ax] >= 0) & (nb[:, ax] < b.shape[ax])
                    bc_ = beta[tuple(cells.T)]
                    # same-level neighbours
                    sel = np.where(ins)[0]
                    nidx = tuple(nb[sel].T)
                    ncov = cov[nidx]
                    nmask = (np.zeros(len(sel), bool) if (q > 0 or self.mask is None)
                             else self.mask[nidx])
                    free = ~ncov & ~nmask
                    s = sel[free]
                    w = hmean(bc_[s], beta[tuple(nb[s].T)]) * ih2
                    add(rid[s], rid[s], w)
                    add(rid[s], ids[tuple(nb[s].T)], -w)
                    s = sel[nmask]
                    if len(s):
                        w = bc_[s] * ih2
                        add(rid[s], rid[s], w)
                        erows.append(rid[s])
                        ecols.append(np.ravel_multi_index(tuple(nb[s].T), b.shape))
                        evals.append(w)
                    # covered neighbours are handled from the fine side
                    # outside the box
                    s = np.where(~ins)[0]
                    if len(s) and q == 0:
                        if self.bc_kind[face] == 0:
                            w = 2.0 * bc_[s] * ih2
                            add(rid[s], rid[s], w)
                            lift[rid[s]] += w * self.bc_value[face]
                        elif self.bc_kind[face] != 1:
                            raise ValueError("bc_kind must be 0 or 1")
            if q > 0:
                self._coarse_fine(q, add)
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n, self.n))
        A.sum_duplicates()
        if erows:
            E = sp.csr_matrix((np.concatenate(evals), (np.concatenate(erows),
                                                       np.concatenate(ecols))),
                              shape=(self.n, n0))
        else:
            E = sp.csr_matrix((self.n, n0))
        return A, lift, E

    def _coarse_fine(self, q, add):
        """Rows of the fine boundary cells of box q and the refluxed coarse
        rows of its parent."""
        b = self.boxes[q]
        p = self.boxes[b.parent]
        wc, w1, w2 = ghost_normal_weights()
        beta_f, beta_p = self._beta(q), self._beta(b.parent)
        ids, pids = self.uid[q], self.uid[b.parent]
        ih2f = 1.0 / (b.h * b.h)
        ih2c = 1.0 / (p.h * p.h)
        for ax in range(3):
            t1, t2 = [a for a in range(3) if a != ax]
            for side in (-1, 1):
                # fine boundary cells of this face
                grids = [np.arange(n) for n in b.shape]
                grids[ax] = np.array([0 if side < 0 else b.shape[ax] - 1])
                cells = np.stack(np.meshgrid(*grids, indexing="ij"), -1).reshape(-1, 3)
                f1 = ids[tuple(cells.T)]
                c2 = cells.copy()
                c2[:, ax] -= side
                f2 = ids[tuple(c2.T)]
                # global fine index of the ghost, its coarse cell in parent
                # local indices
                gfine = cells + np.array(b.lo)
                gfine[:, ax] += side
                C = gfine // 2 - np.array(p.lo)
                s1 = np.where(gfine[:, t1] % 2 == 1, 0.25, -0.25)
                s2 = np.where(gfine[:, t2] % 2 == 1, 0.25, -0.25)
                wface = hmean(beta_f[tuple(cells.T)], beta_p[tuple(C.T)])
                cid = pids[tuple(C.T)]
                if (f1 < 0).any() or (f2 < 0).any() or (cid < 0).any():
                    raise ValueError("coarse-fine stencil leaves the valid cells")
                # fine row: w ih2f (u_f - g)
                kf = wface * ih2f
                add(f1, f1, kf * (1.0 - w1))
                add(f1, f2, -kf * w2)
                # coarse row: (ih2c / 2) w (g - u_f) (the mean of the four
                # fine fluxes through C's face, divided by h_c)
                kc = 0.5 * ih2c * wface
                add(cid, f1, kc * (w1 - 1.0))
                add(cid, f2, kc * w2)
                for a in (-1, 0, 1):
                    for bb in (-1, 0, 1):
                        Cs = C.copy()
                        Cs[:, t1] += a
                        Cs[:, t2] += bb
                        sid = pids[tuple(Cs.T)]
                        if (sid < 0).any():
                            raise ValueError("coarse-fine stencil leaves the valid cells")
                        lam = tangential_weight(a, bb, s1, s2)
                        add(f1, sid, -kf * wc * lam)
                        add(cid, sid, kc * wc * lam)

    # ---- vectors ----------------------------------------------------------
    def gather(self, arrays):
        """Unknown vector from per-box arrays (valid free cells)."""
        x = np.empty(self.n)
        for q, a in enumerate(arrays):
            ids = self.uid[q]
            x[ids[ids >= 0]] = np.asarray(a, dtype=np.float64)[ids >= 0]
        return x

    def scatter(self, x, fill=0.0):
        """Per-box arrays from an unknown vector; other cells = fill."""
        out = []
        for q, b in enumerate(self.boxes):
            a = np.full(b.shape, fill, dtype=np.float64)
            ids = self.uid[q]
            a[ids >= 0] = x[ids[ids >= 0]]
            out.append(a)
        return out

    def average_down(self, arrays):
        """Covered cells := mean of their 8 children, finest level first."""
        arrays = [np.array(a, dtype=np.float64, copy=True) for a in arrays]
        for q in sorted(range(len(self.boxes)), key=lambda r: -self.boxes[r].level):
            b = self.boxes[q]
            if b.level == 0:
                continue
            p = self.boxes[b.parent]
            a = arrays[q]
            m = a.reshape(b.shape[0] // 2, 2, b.shape[1] // 2, 2, b.shape[2] // 2, 2)
            avg = m.mean(axis=(1, 3, 5))
            flo, fhi = b.footprint()
            sl = tuple(slice(flo[x] - p.lo[x], fhi[x] - p.lo[x]) for x in range(3))
            arrays[b.parent][sl] = avg
        return arrays

    def rhs(self, f):
        """b = f + lifts (domain faces and electrode values) on the unknowns."""
        _, lift, E = self.assemble()
        return self.gather(f) + lift + E @ self.mask_value.ravel()

    def apply(self, u):
        """Per-box operator applied to u on the valid free cells (0
        elsewhere); u[0] holds the electrode values on masked cells."""
        A, _, E = self.assemble()
        y = A @ self.gather(u) - E @ np.asarray(u[0], dtype=np.float64).ravel()
        return self.scatter(y)

    def residual(self, f, u):
        """Per-box r = f + domain lifts - (operator applied to u) on the
        unknowns (0 elsewhere) and ||r||_2; electrode values come from u[0]
        (with u[0] = mask_value there this is b - A u)."""
        _, lift, _ = self.assemble()
        r = self.gather(f) + lift - self.gather(self.apply(u))
        return self.scatter(r), float(np.linalg.norm(r))

    def rhs_norm(self, f):
        return float(np.linalg.norm(self.rhs(f)))

    def solve(self, f):
        """Exact solution of the composite system (sparse direct solve).
        Returns per-box arrays: valid cells the solution, electrode cells
        their value, covered cells the mean of their children."""
        A, _, _ = self.assemble()
        x = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A").solve(self.rhs(f))
        out = self.scatter(x)
        if self.mask is not None:
            out[0][self.mask] = self.mask_value[self.mask]
        return self.average_down(out)

    def rel_l2(self, u, ref):
        """Relative L2 difference over the unknowns."""
        a, r = self.gather(u), self.gather(ref)
        return float(np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-300))

    def cell_centres(self, q):
        """(z, y, x) coordinate arrays of the cell centres of box q."""
        b = self.boxes[q]
        return np.meshgrid(*[(b.lo[a] + np.arange(b.shape[a]) + 0.5) * b.h for a in range(3)],
                           indexing="ij")

    def volumes(self):
        """Unknown vector of cell volumes."""
        return self.gather([np.full(b.shape, b.h ** 3) for b in self.boxes])
