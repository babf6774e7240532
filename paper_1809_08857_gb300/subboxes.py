"""Refined sub-boxes under a parent grid: the one-way stand-in for the
patch-based refinement of the paper's streamer runs (Secs. 3-4).

One time step's elliptic solves on a parent n^3 grid (the Poisson problem
with the dielectric slab and the streamer-shell charge, the three
radiative-transfer problems with the smoothed ionisation source), then
`count` refined sub-boxes (ratio 2) of uneven sizes drawn from
{32, 48, 64, 96, 128}^3 (workloads.subbox_layout): each box gets the charge
and permittivity sampled on its own cells and Dirichlet data on its faces by
trilinear interpolation of the parent answers (mg_subbox_bc), and its
Poisson and three Helmholtz problems are solved together with those of all
other boxes in one mg_solve_batch call.  Every step runs through libmg.
"""
import numpy as np
import torch

from . import mg, workloads as W

KAPPAS = (10.0, 100.0, 1000.0)


def box_inputs(n, origin, dims, seed):
    """Charge (C/m^3), permittivity and Helmholtz source of a ratio-2 sub-box of
    an n^3 parent on the unit cube: the parent's shell (thickness and
    amplitude of the parent cell size) sampled on the fine cells, the slab
    permittivity, and the shell magnitude / eps0 smoothed by a Gaussian of two
    parent cells (four fine cells)."""
    from scipy.ndimage import gaussian_filter

    hp = 1.0 / n
    hf = hp / 2
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    o = tuple(v * hp for v in origin)
    rho = W.streamer_shell_box(shape, hf, o, seed, thickness=hp)
    eps = W.dielectric_slab_box(shape, hf, o)
    S = gaussian_filter(np.abs(rho) / W.EPS0, sigma=4.0, mode="constant", truncate=4.0)
    return rho, eps, np.maximum(S, 0.0)


class Config3:
    """The parent set and `count` sub-boxes, built once (contexts, inputs,
    face arrays); run() solves everything from zero."""

    def __init__(self, n=256, count=16, seed=0, dev="cuda", inner_cycles=3):
        self.n = n
        h = 1.0 / n
        self.rho = torch.from_numpy(W.streamer_shell(n, seed)).to(dev)
        self.eps = torch.from_numpy(W.dielectric_slab(n)).to(dev)
        self.S = torch.from_numpy(W.ionization_source(n, seed)).to(dev)
        self.parent = mg.Solver((n, n, n), h, eps_r=self.eps, precision=mg.MG_PREC_MIXED,
                                inner_cycles=inner_cycles)
        self.phi = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
        self.psi = [torch.zeros_like(self.phi) for _ in KAPPAS]
        self.layout = W.subbox_layout(n, count, seed)
        self.boxes = []
        for q, (origin, dims) in enumerate(self.layout):
            rho_b, eps_b, S_b = box_inputs(n, origin, dims, 100 + q)
            shape = rho_b.shape
            s = mg.Solver(shape, h / 2, eps_r=torch.from_numpy(eps_b).to(dev),
                          bc_kind=(0,) * 6, precision=mg.MG_PREC_MIXED, inner_cycles=inner_cycles)
            nf = mg.face_count(shape)
            self.boxes.append({
                "origin": origin, "dims": dims, "shape": shape, "solver": s,
                "rho": torch.from_numpy(rho_b).to(dev), "eps": eps_b,
                "S": torch.from_numpy(S_b).to(dev),
                "u": [torch.zeros(shape, dtype=torch.float64, device=dev) for _ in range(4)],
                "faces": [torch.empty(nf, dtype=torch.float64, device=dev) for _ in range(4)]})
        self.problems = []
        for b in self.boxes:
            self.problems.append({"solver": b["solver"], "kind": "poisson", "rhs": b["rho"],
                                  "u": b["u"][0], "faces": b["faces"][0]})
            for j, k in enumerate(KAPPAS):
                self.problems.append({"solver": b["solver"], "kind": "helmholtz", "kappa": k,
                                      "rhs": b["S"], "u": b["u"][1 + j],
                                      "faces": b["faces"][1 + j]})

    def run(self, tol=1e-10):
        """Parent set, face data, batched sub-box solves (all from zero).
        Returns (parent stats, sub-box stats)."""
        self.phi.zero_()
        for p in self.psi:
            p.zero_()
        st_parent = self.parent.solve_set(self.rho, self.phi, self.S, self.psi, KAPPAS, tol)
        parents = [self.phi] + self.psi
        for b in self.boxes:
            for u in b["u"]:
                u.zero_()
            for j in range(4):
                self.parent.subbox_bc(parents[j], b["origin"], b["dims"], out=b["faces"][j])
        st_boxes = mg.solve_batch(self.problems, tol)
        return st_parent, st_boxes

    def cells(self):
        return self.n ** 3, sum(int(np.prod(b["shape"])) for b in self.boxes)

    def close(self):
        for b in self.boxes:
            b["solver"].close()
        self.parent.close()
