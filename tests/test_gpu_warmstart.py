"""The learned warm start: train libmg's U-Net on advancing-head sequences
produced by the plain solver, then solve a held-out sequence from the plain
warm start (phi_{n-1}) and from the judged network guess.  The answers must
agree to the parity bar (multigrid corrects the guess to the same
tolerance); the refinement steps and solves/s of both are reported (what
they gain is measured, not asserted: the judge compares residuals, which
does not guarantee fewer steps).  The judge itself is pinned on the oracle:
its guess is the better of the two candidates after nu1 red-black sweeps."""
import json
import os

import numpy as np
import pytest

import oracle

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


def test_trained_warm_start_gain(mg):
    from paper_1809_08857_gb300 import warmstart as WS
    from paper_1809_08857_gb300 import workloads as W

    n = 64
    train_eps = [WS.episode(n, seed, 16) for seed in (11, 12, 13)]
    held = WS.episode(n, 99, 10)
    net = mg.UNet(seed=0)
    net.set_scales(*WS.scales(train_eps))
    # a fixed validation batch: the whole 64^3 field of every held-out step
    # (the mini-batch losses of training vary several-fold from crop to crop)
    val = [torch.stack([held[k][q] for k in range(1, len(held))]).contiguous() for q in (2,)]
    val_prev = torch.stack([held[k - 1][1] for k in range(1, len(held))]).contiguous()
    val_phi = torch.stack([held[k][1] for k in range(1, len(held))]).contiguous()
    _, loss_before = net.grads(val[0], val_prev, val_phi)
    losses = WS.train(net, train_eps, iters=300, crop=32, batch=4, lr=1e-3)
    _, loss_after = net.grads(val[0], val_prev, val_phi)
    assert loss_after < loss_before, (loss_before, loss_after)
    res = WS.evaluate(net, held, n)
    print("warm start:", json.dumps(res))
    report = os.environ.get("MG_WARMSTART_REPORT")  # optional JSON report path
    if report:
        with open(report, "w") as fh:
            json.dump(dict(res, loss_first=float(np.mean(losses[:30])),
                           loss_last=float(np.mean(losses[-30:])),
                           val_loss_before=loss_before, val_loss_after=loss_after), fh)
    assert res["max_rel_diff"] <= 1e-9
    # the trained network's guess is closer to the answer than phi_{n-1}
    assert res["err_net"] < res["err_plain"]
    # the held-out answer meets parity with the oracle on the last step
    rho, phi, _ = held[-1]
    ref, _, _, _ = oracle.poisson((n, n, n), 1.0 / n, eps_r=W.dielectric_slab(n)).solve(
        rho.cpu().numpy() / oracle.EPS0)
    assert oracle.rel_l2(phi.cpu().numpy(), ref) <= 1e-9
    net.close()


def test_judge_smooths_both_candidates_and_keeps_the_better(mg):
    """mg_warmstart_predict on a 32^3 gap with the dielectric slab: with a
    network of large random weights (a guess far off) the judge returns
    phi_prev after two red-black Gauss-Seidel sweeps, equal to the oracle's
    own two sweeps of phi_prev; with an untrained network (zero head, so the
    candidate is phi_prev itself) both candidates are the same and the
    network's is kept."""
    from paper_1809_08857_gb300 import workloads as W

    n = 32
    h = 1.0 / n
    eps = W.dielectric_slab(n)
    rho_prev, rho = W.streamer_shell(n, 1), W.streamer_shell(n, 2)
    P = oracle.poisson((n, n, n), h, eps_r=eps)
    prev, _, _, _ = P.solve(rho_prev / oracle.EPS0)
    f = rho / oracle.EPS0
    ref = prev
    for _ in range(2):  # nu1 = 2 sweeps, red then black
        ref = P.rbgs(f, ref, 0)
        ref = P.rbgs(f, ref, 1)
    s = mg.Solver((n, n, n), h, eps_r=torch.from_numpy(eps).cuda(), precision=1, nu1=2)
    rho_t, prev_t = torch.from_numpy(rho).cuda(), torch.from_numpy(prev).cuda()
    bad = mg.UNet(seed=3)
    bad.set_scales(1.0, 1.0, 1.0)
    bad.set_params(np.random.default_rng(4).standard_normal(bad.num_params()).astype(np.float32)
                   * 10.0)
    s.warmstart_attach(bad)
    guess, used = s.warmstart_predict(rho_t, prev_t)
    assert not used
    assert oracle.rel_l2(guess.cpu().numpy(), ref) <= 1e-13
    zero = mg.UNet(seed=5)
    zero.set_scales(1.0, 1.0, 1.0)
    s.warmstart_attach(zero)
    guess, used = s.warmstart_predict(rho_t, prev_t)
    assert used
    assert oracle.rel_l2(guess.cpu().numpy(), ref) <= 1e-13
    s.close()
    bad.close()
    zero.close()
