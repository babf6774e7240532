"""What the trained warm-start network gains: train libmg's U-Net on
advancing-head sequences produced by the plain solver, then solve a held-out
sequence from the plain warm start (phi_{n-1}) and from the judged network
guess.  The answers must agree to the parity bar (multigrid corrects the
guess to the same tolerance); the refinement steps and solves/s of both are
reported, and the judged guess is never worse than the plain one."""
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
    losses = WS.train(net, train_eps, iters=300, crop=32, batch=4, lr=1e-3)
    assert np.mean(losses[-30:]) < np.mean(losses[:30])
    res = WS.evaluate(net, held, n)
    print("warm start:", json.dumps(res))
    report = os.environ.get("MG_WARMSTART_REPORT")  # optional JSON report path
    if report:
        with open(report, "w") as fh:
            json.dump(dict(res, loss_first=float(np.mean(losses[:30])),
                           loss_last=float(np.mean(losses[-30:]))), fh)
    assert res["max_rel_diff"] <= 1e-9
    assert res["steps_judged"] <= res["steps_plain"] + 1e-9
    # the trained network's guess is closer to the answer than phi_{n-1}
    assert res["err_net"] < res["err_plain"]
    # the held-out answer meets parity with the oracle on the last step
    rho, phi, _ = held[-1]
    ref, _, _, _ = oracle.poisson((n, n, n), 1.0 / n, eps_r=W.dielectric_slab(n)).solve(
        rho.cpu().numpy() / oracle.EPS0)
    assert oracle.rel_l2(phi.cpu().numpy(), ref) <= 1e-9
    net.close()
