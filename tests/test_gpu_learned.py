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


@pytest.mark.parametrize("make", [lambda: I.config_semiconvection_3d(32),
                                  lambda: I.config_convection_3d(32, seed=3)])
@pytest.mark.parametrize("net_precond", [0, 1])
def test_learned_mixed_3d_matches_oracle(lm, make, net_precond):
    """The learned mode on 3D grids (the two-component semiconvection recipe
    of the 512^3 workload, downsized, and the convection recipe): the 2D
    network runs on every x-z slice, its warm start enters the refinement
    (the initial residual is that of the warm start, not of x = 0), and the
    solution matches the oracle's to 1e-8."""
    p = make()
    op = P.operator_from_problem(p)
    xs = P.solve_direct(op, p.f).ravel()
    with lm.Grid.for_problem(p) as g:
        g.set_problem(p)
        g.load_network(WEIGHTS)
        r = g.solve(mode="learned", rtol=1e-12, net_precond=net_precond, max_outer=30)
        x = g.solution()
        hist = g.residual_history()
    assert r["status"] == 0 and r["rel_residual"] <= 1e-12
    assert hist[0] != 1.0
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_network_input_of_a_3d_grid_is_its_slices(lm):
    """A 3D grid is ny images of its x-z slices: with two identical slices the
    network input of each equals that of the 2D grid of one slice."""
    import dataclasses
    p2 = I.config_training_2d(30001, n=64)
    rep = lambda a: np.repeat(a, 2, axis=1)                  # (nz, 1, nx) -> (nz, 2, nx)
    p3 = dataclasses.replace(p2, n=(p2.n[0], 2, p2.n[2]), ndim=3, rho_old=rep(p2.rho_old), rho_new=rep(p2.rho_new),
                             cs2=rep(p2.cs2), f=rep(p2.f))
    out = {}
    for p in (p2, p3):
        with lm.Grid.for_problem(p) as g:
            g.set_problem(p)
            v = torch.as_tensor(p.f.ravel(), device="cuda")
            feat = torch.empty(3 * p.size, dtype=torch.float32, device="cuda")
            out[p.ndim] = (g.features(v, feat), feat.cpu().numpy())
    s2, f2 = out[2]
    s3, f3 = out[3]
    assert s3 == pytest.approx(s2, rel=1e-12)
    f3 = f3.reshape(2, p2.n[2], p2.n[0], 3)
    np.testing.assert_allclose(f3[0], f2.reshape(p2.n[2], p2.n[0], 3), rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(f3[0], f3[1])
