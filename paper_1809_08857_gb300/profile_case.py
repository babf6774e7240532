"""Small, fixed workloads for profiling single kernels under ncu.

  python -m paper_1809_08857_gb300.profile_case --case solve256
      one mixed-precision Poisson + 3 Helmholtz set at 256^3 (arrays of
      128 MiB each, larger than the 129 MB L2), concurrency 1, no graphs, so
      kernel launches are individually visible;
  python -m paper_1809_08857_gb300.profile_case --case set512
      one solve set at 512^3 with the benchmark's options, one problem at a
      time, no graphs, after an untimed set; prints libmg's launch counts;
  python -m paper_1809_08857_gb300.profile_case --case unet64
      one U-Net training step on a batch of 2 crops of 64^3;
  python -m paper_1809_08857_gb300.profile_case --case amr256
      one composite AMR Poisson solve: base 256^3 with three nested refined
      levels around the streamer head (workloads.streamer_amr_layout), mixed
      precision, two inner V-cycles, from zero to 1e-10;
  python -m paper_1809_08857_gb300.profile_case --case conv128
      one 3x3x3 convolution, 32 -> 32 channels on a 128^3 BF16 volume (128 MiB
      in, 128 MiB out), three untimed launches, then 20 timed with CUDA events;
  python -m paper_1809_08857_gb300.profile_case --case conv_shapes
      the same timing for the convolution shapes of the U-Net levels (batch 2
      at 64^3 .. 8^3) and two 128^3 volumes.
"""
import argparse
import os
import sys

import numpy as np
import torch

from . import mg, workloads as W


def solve256():
    n = 256
    h = 1.0 / n
    rho = torch.from_numpy(W.streamer_shell(n, 0)).cuda()
    eps = torch.from_numpy(W.dielectric_slab(n)).cuda()
    S = torch.from_numpy(W.ionization_source(n, 0)).cuda()
    s = mg.Solver((n, n, n), h, eps_r=eps, precision=mg.MG_PREC_MIXED, inner_cycles=3,
                  concurrency=1, graphs=False)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    psi = [torch.zeros_like(phi) for _ in range(3)]
    st = s.solve_set(rho, phi, S, psi, W.helmholtz_kappas(), 1e-10)
    torch.cuda.synchronize()
    print("steps", [x["cycles"] for x in st])
    s.close()


def set512():
    """One solve set at 512^3 with the options the benchmark times (V(2,1),
    4 inner V-cycles with the last step trimmed, 128-plane refinement tile),
    one problem at a time and without graphs so that every launch is
    visible: a first set builds the coarse inverses, then the set to
    profile.  Prints libmg's launch counts before and during that set (the
    -s / -c of an ncu launch list filtered to libmg's kernels)."""
    n = 512
    h = 1.0 / n
    rho = torch.from_numpy(W.streamer_shell(n, 0)).cuda()
    eps = torch.from_numpy(W.dielectric_slab(n)).cuda()
    S = torch.from_numpy(W.ionization_source(n, 0)).cuda()
    s = mg.Solver((n, n, n), h, eps_r=eps, precision=mg.MG_PREC_MIXED, nu1=2, nu2=1,
                  inner_cycles=4, concurrency=1, graphs=False)
    s.set_options(ir_zchunk=128)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    psi = [torch.zeros_like(phi) for _ in range(3)]
    s.solve_set(rho, phi, S, psi, W.helmholtz_kappas(), 1e-10)
    torch.cuda.synchronize()
    l0 = mg.launch_count()
    phi.zero_()
    for p in psi:
        p.zero_()
    st = s.solve_set(rho, phi, S, psi, W.helmholtz_kappas(), 1e-10)
    torch.cuda.synchronize()
    print("launches_before", l0, "launches_set", mg.launch_count() - l0)
    print("steps", [x["cycles"] for x in st], "vcycles", [x["vcycles"] for x in st])
    s.close()


def unet64():
    rng = np.random.default_rng(0)
    net = mg.UNet(seed=0)
    shape = (2, 64, 64, 64)
    a = [torch.from_numpy(rng.standard_normal(shape)).cuda() for _ in range(3)]
    print("loss", net.train_step(a[0], a[1], a[2], lr=1e-4))
    torch.cuda.synchronize()
    net.close()


def amr256():
    n0 = 256
    h0 = 1.0 / n0
    boxes = W.streamer_amr_layout(n0)
    eps = [torch.from_numpy(W.dielectric_slab(n0)).cuda()] + [None] * len(boxes)
    rho = [W.streamer_shell_box((n0,) * 3, h0, (0, 0, 0), 0, thickness=h0)]
    for q, b in enumerate(boxes):
        o, h = W.amr_box_origin(h0, b)
        rho.append(W.streamer_shell_box(b[2], h, o, q + 1, thickness=h0))
    rho = [torch.from_numpy(r).cuda() for r in rho]
    a = mg.Amr((n0,) * 3, h0, boxes, eps_r=eps, bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE,
               precision=mg.MG_PREC_MIXED, inner_cycles=2)
    u = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in a.shapes]
    st = a.solve("poisson", rho, u, tol=1e-10)
    torch.cuda.synchronize()
    print("fac iterations", st["cycles"], "rel", st["rel_resid"])
    a.close()


def _time_conv(n, s, cin, cout, reps=20):
    g = torch.Generator(device="cpu").manual_seed(0)
    x = (torch.randn((n, s, s, s, cin), generator=g) * 0.5).to(torch.bfloat16).cuda()
    w = (torch.randn((cout, 27, cin), generator=g) * 0.1).to(torch.bfloat16).cuda()
    b = torch.randn(cout, generator=g).cuda()
    for _ in range(3):
        y = mg.conv3d(x, w, b, relu=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        y = mg.conv3d(x, w, b, relu=True)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / reps * 1e3
    flop = 2.0 * 27 * cin * cout * n * s ** 3
    print(f"conv {n} x {s}^3 {cin}->{cout}: {us:.1f} us per launch, "
          f"{flop / us * 1e-6:.1f} TFLOP/s, checksum {float(y.float().sum()):.6e}")


def conv128():
    _time_conv(1, 128, 32, 32)


def conv_shapes():
    for shape in [(2, 64, 16, 16), (2, 64, 32, 16), (2, 32, 16, 32), (2, 32, 32, 32),
                  (2, 32, 64, 32), (2, 16, 32, 48), (2, 16, 48, 48), (2, 16, 96, 48),
                  (2, 8, 48, 64), (2, 8, 64, 64), (1, 128, 16, 16), (1, 128, 32, 32)]:
        _time_conv(*shape)


def main():
    ap = argparse.ArgumentParser()
    cases = {"solve256": solve256, "set512": set512, "unet64": unet64, "amr256": amr256,
             "conv128": conv128,
             "conv_shapes": conv_shapes}
    ap.add_argument("--case", choices=sorted(cases), required=True)
    args = ap.parse_args()
    cases[args.case]()


if __name__ == "__main__":
    sys.exit(main())
