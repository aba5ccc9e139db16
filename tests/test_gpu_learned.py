"""Row a6 with the trained weights the package ships: the learned modes
reach the oracle's solution, and the trained network's warm start is closer
to it, in the energy norm, than an untrained network's."""
import os

import numpy as np
import pytest

from oracle import poisson as P
from oracle import unet as U
from paper_1112_3507_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_1112_3507_gb300", "weights", "unet_16_32_48_64.bin")
CH = (16, 32, 48, 64)
HELD_OUT = (30000, 30002, 30005, 30007)


@pytest.fixture(scope="module")
def lm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_3507_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()
    from paper_1112_3507_gb300 import lowmach
    return lowmach


@pytest.fixture(scope="module")
def untrained(lm, tmp_path_factory):
    """He-normal weights, zero biases: the same network before training."""
    P0 = U.init_params(np.random.default_rng(0), cin=3, ch=CH)
    net = lm.Net(CH)
    net.set_params(U.flat_params(P0, cin=3, ch=CH))
    path = str(tmp_path_factory.mktemp("net") / "untrained.bin")
    net.save(path)
    net.close()
    return path


def _problem(seed):
    p = I.config_training_2d(seed, n=256)
    op = P.operator_from_problem(p)
    return p, op, P.solve_direct(op, p.f).ravel()


@pytest.mark.parametrize("seed", HELD_OUT[:2])
@pytest.mark.parametrize("net_precond", [0, 1])
def test_learned_mode_reaches_the_oracle_solution(lm, seed, net_precond):
    p, op, xs = _problem(seed)
    with lm.Grid.for_problem(p) as g:
        g.set_problem(p)
        g.load_network(WEIGHTS)
        r = g.solve(mode="learned", rtol=1e-12, net_precond=net_precond, max_outer=30)
        x = g.solution()
        hist = g.residual_history()
    assert r["status"] == 0 and r["rel_residual"] <= 1e-12
    assert np.isfinite(hist[0])
    assert P.rel_residual(op, x, p.f) <= 1.001e-12
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


def _energy_error_of_guess(lm, g, net_path, p, op, xs):
    """||x* - a n||_A / ||x*||_A for the network guess n = s NN(features(f))
    at its energy-optimal scale a = f.n / n^T A n."""
    f = torch.as_tensor(p.f.ravel(), device="cuda")
    feat = torch.empty(3 * p.size, dtype=torch.float32, device="cuda")
    s = g.features(f, feat)
    net = lm.Net.load(net_path)
    y = torch.empty(p.size, dtype=torch.float32, device="cuda")
    net.forward(feat, y, 1, p.n[2], p.n[0])
    net.close()
    n = y.cpu().numpy().astype(np.float64) * s
    An = op.apply(n).ravel()
    a = max(float(p.f.ravel() @ n) / float(n @ An), 0.0)
    e = xs - a * n
    return float(np.sqrt((e @ op.apply(e).ravel()) / (xs @ p.f.ravel())))


def test_training_gains_over_the_untrained_network(lm, untrained):
    """What training buys: the energy-norm error of the warm start (1 would
    be no better than x0 = 0)."""
    got = []
    for seed in HELD_OUT:
        p, op, xs = _problem(seed)
        with lm.Grid.for_problem(p) as g:
            g.set_problem(p)
            et = _energy_error_of_guess(lm, g, WEIGHTS, p, op, xs)
            eu = _energy_error_of_guess(lm, g, untrained, p, op, xs)
        got.append((seed, et, eu))
    print("energy-norm warm-start error (seed, trained, untrained):", got)
    assert all(et < eu for _, et, eu in got), got
    assert np.mean([et for _, et, _ in got]) < 0.9, got
