"""Learned warm start: data generation, training and evaluation.

The paper re-solves the elliptic equations only every coarse step while the
charge moves (Sec. 2.2), so consecutive Poisson solves see slowly varying
charge.  This module produces training sequences with the plain solver on a
streamer head that advances one cell per step (seeded radius, random lateral
drift), trains libmg's U-Net (every kernel is libmg's: mg_unet_train_step) to
predict phi_n - phi_{n-1} from (rho_n, phi_{n-1}), and measures what the
network saves: V-cycles (refinement steps) to 1e-10 and solves per second,
inference included, against the plain warm start phi_{n-1}.  Multigrid
corrects every guess to the same tolerance, so the answer does not change.
"""
import time

import numpy as np
import torch

from . import mg, workloads as W


def shell_on_device(n, seed, radius, z0, z1, axis):
    """workloads.streamer_shell_box on the n^3 unit cube as a CUDA float64
    tensor, scattered from its sparse shell cells (no dense host array)."""
    idx, val = W.streamer_shell_cells((n, n, n), 1.0 / n, (0.0, 0.0, 0.0), seed, radius=radius,
                                      z0=z0, z1=z1, axis_xy=tuple(axis))
    rho = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    rho[torch.from_numpy(idx).cuda()] = torch.from_numpy(val).cuda()
    return rho.view(n, n, n)


def episode(n, seed, steps, z_start=0.9, z_channel=0.1, eps_slab=True, tol=1e-10, solver=None):
    """Generate one advancing-head sequence on an n^3 gap (dielectric slab,
    phi = 0 / 1 on the bottom / top faces): a list of (rho_k, phi_k, r_k) as
    CUDA float64 tensors, phi_k solved from phi_{k-1} by the plain solver and
    r_k = b_k - A phi_{k-1} (the network's input; r_0 = b_0)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    radius = rng.uniform(0.015, 0.03)
    axis = np.array([0.5, 0.5])
    own = solver is None
    if own:
        eps = torch.from_numpy(W.dielectric_slab(n) if eps_slab else np.ones((n, n, n))).cuda()
        solver = mg.Solver((n, n, n), h, eps_r=eps, precision=mg.MG_PREC_MIXED, inner_cycles=3)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    out = []
    r = torch.empty_like(phi)
    for k in range(steps):
        axis = axis + rng.normal(0.0, 0.25 * h, size=2)
        z1 = z_start - k * h
        rho = shell_on_device(n, seed * 100003 + k, radius, z_channel, z1, axis)
        phi = phi.clone()
        r = solver.poisson_residual(rho, phi, torch.empty_like(phi))
        solver.solve_poisson(rho, phi, tol)
        out.append((rho, phi, r))
    if own:
        solver.close()
    return out


def scales(episodes):
    """Input/output scales: inverse RMS of the residual input, of phi and of
    the step change."""
    r = np.sqrt(np.mean([float((e[k][2] ** 2).mean()) for e in episodes for k in range(1, len(e))]))
    p = np.sqrt(np.mean([float((e[k][1] ** 2).mean()) for e in episodes for k in range(len(e))]))
    d = np.sqrt(np.mean([float(((e[k][1] - e[k - 1][1]) ** 2).mean())
                         for e in episodes for k in range(1, len(e))]))
    return 1.0 / max(r, 1e-300), 1.0 / max(p, 1e-300), 1.0 / max(d, 1e-300)


def train(net, episodes, iters, crop=32, batch=4, lr=1e-3, seed=0, log_every=0):
    """Adam on random crops (r_k, phi_{k-1}) -> phi_k; returns the loss history."""
    rng = np.random.default_rng(seed)
    n = episodes[0][0][0].shape[0]
    losses = []
    for it in range(iters):
        rs, ps, ts = [], [], []
        for _ in range(batch):
            e = episodes[rng.integers(len(episodes))]
            k = int(rng.integers(1, len(e)))
            o = rng.integers(0, n - crop + 1, size=3)
            sl = (slice(o[0], o[0] + crop), slice(o[1], o[1] + crop), slice(o[2], o[2] + crop))
            rs.append(e[k][2][sl])
            ps.append(e[k - 1][1][sl])
            ts.append(e[k][1][sl])
        rho = torch.stack(rs).contiguous()
        prev = torch.stack(ps).contiguous()
        tgt = torch.stack(ts).contiguous()
        losses.append(net.train_step(rho, prev, tgt, lr=lr))
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {losses[-1]:.4e}", flush=True)
    return losses


def evaluate(net, ep, n, tol=1e-10, eps_slab=True):
    """Solve every step of a held-out episode three ways: from phi_{k-1} (the
    plain warm start), from the raw network guess, and from the judged guess
    (mg_warmstart_predict: the network unless its FP64 residual is worse).
    Reports mean refinement steps, solves/s (network: inference included),
    the relative L2 error of each starting guess against the converged
    answer, and the largest relative difference between the answers."""
    h = 1.0 / n
    eps = torch.from_numpy(W.dielectric_slab(n) if eps_slab else np.ones((n, n, n))).cuda()
    s = mg.Solver((n, n, n), h, eps_r=eps, precision=mg.MG_PREC_MIXED, inner_cycles=3)
    s.warmstart_attach(net)
    acc = {k: [] for k in ("steps_plain", "steps_net", "steps_judged", "err_plain", "err_net")}
    t_plain = t_net = t_judged = 0.0
    used, diff = 0, 0.0
    for k in range(1, len(ep)):
        rho, prev = ep[k][0], ep[k - 1][1]
        sync = torch.cuda.synchronize
        a = prev.clone()
        sync()
        t0 = time.perf_counter()
        acc["steps_plain"].append(s.solve_poisson(rho, a, tol)["cycles"])
        sync()
        t_plain += time.perf_counter() - t0
        t0 = time.perf_counter()
        g = net.predict(ep[k][2], prev)
        g0 = g.clone()
        acc["steps_net"].append(s.solve_poisson(rho, g, tol)["cycles"])
        sync()
        t_net += time.perf_counter() - t0
        t0 = time.perf_counter()
        j, u = s.warmstart_predict(rho, prev)
        acc["steps_judged"].append(s.solve_poisson(rho, j, tol)["cycles"])
        sync()
        t_judged += time.perf_counter() - t0
        used += int(u)
        an = float(a.norm())
        acc["err_plain"].append(float((prev - a).norm()) / an)
        acc["err_net"].append(float((g0 - a).norm()) / an)
        diff = max(diff, float((g - a).norm()) / an, float((j - a).norm()) / an)
    s.close()
    m = len(ep) - 1
    out = {k: float(np.mean(v)) for k, v in acc.items()}
    out.update({"solves_per_s_plain": m / t_plain, "solves_per_s_net": m / t_net,
                "solves_per_s_judged": m / t_judged, "net_guess_used": used / m,
                "max_rel_diff": diff, "grid": n, "steps_evaluated": m})
    return out


def head_path(n, seed, steps, z_start=0.9, z_channel=0.1):
    """Charge of one advancing-head episode, step by step (no solve): a
    generator of rho_k as CUDA float64 tensors, with the seeded radius
    U[0.015, 0.03] and lateral Gaussian drift of 0.25 h per step of
    episode()."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    radius = rng.uniform(0.015, 0.03)
    axis = np.array([0.5, 0.5])
    for k in range(steps):
        axis = axis + rng.normal(0.0, 0.25 * h, size=2)
        z1 = z_start - k * h
        yield shell_on_device(n, seed * 100003 + k, radius, z_channel, z1, axis)


def train_online(net, n, seeds, steps, crop=64, batch=4, iters_per_step=1, buffer=192,
                 lr=1e-3, seed=0, tol=1e-10):
    """Training on sequences too large to keep: every episode (one per seed)
    is solved step by step with the plain solver from phi_{k-1}; each step
    adds `batch` random crops of (r_k, phi_{k-1}, phi_k) to a replay buffer
    of at most `buffer` crops (oldest dropped), then `iters_per_step` Adam
    steps train on random batches from the buffer.  The scales are set from
    the first episode's first steps.  Returns (losses, solver seconds)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    eps = torch.from_numpy(W.dielectric_slab(n)).cuda()
    solver = mg.Solver((n, n, n), h, eps_r=eps, precision=mg.MG_PREC_MIXED, inner_cycles=3)
    buf = []
    losses = []
    t_solve = 0.0
    scaled = False
    for sd in seeds:
        phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
        for k, rho in enumerate(head_path(n, sd, steps)):
            prev = phi
            phi = prev.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = solver.poisson_residual(rho, phi, torch.empty_like(phi))
            solver.solve_poisson(rho, phi, tol)
            torch.cuda.synchronize()
            t_solve += time.perf_counter() - t0
            if k == 0:
                continue  # a cold solve has no previous potential
            if not scaled:
                d = float((phi - prev).pow(2).mean().sqrt())
                net.set_scales(1.0 / max(float(r.pow(2).mean().sqrt()), 1e-300),
                               1.0 / max(float(phi.pow(2).mean().sqrt()), 1e-300),
                               1.0 / max(d, 1e-300))
                scaled = True
            for _ in range(batch):
                o = rng.integers(0, n - crop + 1, size=3)
                sl = (slice(o[0], o[0] + crop), slice(o[1], o[1] + crop),
                      slice(o[2], o[2] + crop))
                buf.append((r[sl].clone(), prev[sl].clone(), phi[sl].clone()))
            del buf[:max(0, len(buf) - buffer)]
            for _ in range(iters_per_step):
                pick = rng.integers(0, len(buf), size=batch)
                losses.append(net.train_step(torch.stack([buf[q][0] for q in pick]).contiguous(),
                                             torch.stack([buf[q][1] for q in pick]).contiguous(),
                                             torch.stack([buf[q][2] for q in pick]).contiguous(),
                                             lr=lr))
    solver.close()
    return losses, t_solve


def evaluate_stream(net, n, seed, steps, tol=1e-10):
    """evaluate() on a held-out episode generated step by step (only the
    previous potential is kept): step k is solved from phi_{k-1}, from the
    raw network guess and from the judged guess, and the plain answer
    becomes phi_k."""
    h = 1.0 / n
    eps = torch.from_numpy(W.dielectric_slab(n)).cuda()
    s = mg.Solver((n, n, n), h, eps_r=eps, precision=mg.MG_PREC_MIXED, inner_cycles=3)
    s.warmstart_attach(net)
    acc = {k: [] for k in ("steps_plain", "steps_net", "steps_judged", "err_plain", "err_net")}
    t_plain = t_net = t_judged = 0.0
    used, diff, m = 0, 0.0, 0
    sync = torch.cuda.synchronize
    phi = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    for k, rho in enumerate(head_path(n, seed, steps)):
        if k == 0:
            s.solve_poisson(rho, phi, tol)
            continue
        prev = phi
        r = s.poisson_residual(rho, prev.clone(), torch.empty_like(prev))
        a = prev.clone()
        sync()
        t0 = time.perf_counter()
        acc["steps_plain"].append(s.solve_poisson(rho, a, tol)["cycles"])
        sync()
        t_plain += time.perf_counter() - t0
        t0 = time.perf_counter()
        g = net.predict(r, prev)
        g0 = g.clone()
        acc["steps_net"].append(s.solve_poisson(rho, g, tol)["cycles"])
        sync()
        t_net += time.perf_counter() - t0
        t0 = time.perf_counter()
        j, u = s.warmstart_predict(rho, prev)
        acc["steps_judged"].append(s.solve_poisson(rho, j, tol)["cycles"])
        sync()
        t_judged += time.perf_counter() - t0
        used += int(u)
        an = float(a.norm())
        acc["err_plain"].append(float((prev - a).norm()) / an)
        acc["err_net"].append(float((g0 - a).norm()) / an)
        diff = max(diff, float((g - a).norm()) / an, float((j - a).norm()) / an)
        phi = a
        m += 1
    s.close()
    out = {k: float(np.mean(v)) for k, v in acc.items()}
    out.update({"solves_per_s_plain": m / t_plain, "solves_per_s_net": m / t_net,
                "solves_per_s_judged": m / t_judged, "net_guess_used": used / m,
                "max_rel_diff": diff, "grid": n, "steps_evaluated": m})
    return out


def config4(n=256, train_seeds=tuple(range(1000, 1010)), held_seeds=(4242, 4343), steps=200,
            held_steps=200, iters_per_step=1, crop=64, batch=4, lr=1e-3):
    """The warm-start experiment at 256^3: train on 10 episodes x 200 steps
    of the advancing head (2000 solves of the plain solver, online), then
    evaluate on held-out episodes (each step solved from phi_{k-1}, from the
    raw network guess and from the judged guess).  Returns the evaluation of
    each held-out episode plus training figures."""
    net = mg.UNet(seed=0)
    t0 = time.perf_counter()
    losses, t_solve = train_online(net, n, train_seeds, steps, crop=crop, batch=batch,
                                   iters_per_step=iters_per_step, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    evals = [evaluate_stream(net, n, sd, held_steps) for sd in held_seeds]
    net.close()
    return {"grid": n, "train_episodes": len(train_seeds), "steps_per_episode": steps,
            "train_iters": len(losses), "train_s": t_train, "solver_s_in_training": t_solve,
            "loss_first": float(np.mean(losses[:50])), "loss_last": float(np.mean(losses[-50:])),
            "held_out": evals}


def main():
    """Scaled config-4 experiment: python -m paper_1809_08857_gb300.warmstart
    [--n 128] [--episodes 6] [--steps 40] [--iters 1500] [--out file.json];
    with --config4 the 256^3 experiment of config4() (online training on
    10 x 200 steps, held-out evaluation), --steps and --held-steps its
    episode lengths."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--episodes", type=int, default=6)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--crop", type=int, default=64)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="")
    ap.add_argument("--config4", action="store_true")
    ap.add_argument("--held-steps", type=int, default=200)
    a = ap.parse_args()
    if a.config4:
        res = config4(n=a.n, steps=a.steps, held_steps=a.held_steps, crop=a.crop, batch=a.batch,
                      lr=a.lr)
        print(json.dumps(res))
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh, indent=1)
        return
    t0 = time.perf_counter()
    eps_train = [episode(a.n, 1000 + q, a.steps) for q in range(a.episodes)]
    held = episode(a.n, 4242, max(8, a.steps // 2))
    t_data = time.perf_counter() - t0
    net = mg.UNet(seed=0)
    net.set_scales(*scales(eps_train))
    t0 = time.perf_counter()
    losses = train(net, eps_train, a.iters, crop=a.crop, batch=a.batch, lr=a.lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = evaluate(net, held, a.n)
    res.update({"data_s": t_data, "train_s": t_train, "iters": a.iters,
                "loss_first": float(np.mean(losses[:50])), "loss_last": float(np.mean(losses[-50:]))})
    print(json.dumps(res))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
