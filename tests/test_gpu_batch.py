"""Row a8: the batched, graph-captured solve of uneven 2D grids vs the
oracle's direct solves and vs the one-grid path (needs a GB300)."""
import json
import os

import numpy as np
import pytest

from oracle import poisson as P
from paper_1112_3507_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_3507_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()
    from paper_1112_3507_gb300 import lowmach
    return lowmach


def _batch(lm, problems):
    grids = []
    for p in problems:
        g = lm.Grid.for_problem(p)
        g.set_problem(p)
        grids.append(g)
    return grids


def test_batch_matches_oracle_and_single_path(lm, tmp_path):
    """Uneven sizes (the sides of the 64-solve workload divided by 8), Ma and
    density contrast drawn per solve: every solution agrees with the direct
    solve to 1e-8 and with the one-grid mixed solve."""
    cache = tmp_path / "tune.json"
    lm.autotune_set_cache(str(cache))
    problems = I.config_batch(count=6, seed=42, scale=8)
    assert len({p.n for p in problems}) > 2
    grids = _batch(lm, problems)
    try:
        res = lm.batch_solve(grids, rtol=1e-12, max_outer=12, inner_max_iter=10)
        for p, g, r in zip(problems, grids, res):
            assert r["status"] == 0 and r["rel_residual"] <= 1e-12, r
            x = g.solution()
            op = P.operator_from_problem(p)
            xs = P.solve_direct(op, p.f).ravel()
            assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs), p.name
            assert P.rel_residual(op, x, p.f) <= 2e-12
        # second call reuses the captured plan and gives the same bits
        x1 = [g.solution() for g in grids]
        res2 = lm.batch_solve(grids, rtol=1e-12, max_outer=12, inner_max_iter=10)
        for g, a, r1, r2 in zip(grids, x1, res, res2):
            assert np.array_equal(g.solution(), a) and r1["iters"] == r2["iters"]
        # the one-grid path solves each to the same tolerance
        for p, g in zip(problems, grids):
            r = g.solve(mode="mixed", rtol=1e-12, max_outer=12)
            assert r["status"] == 0
    finally:
        for g in grids:
            g.close()
    tuned = json.loads(cache.read_text())
    assert any("|rbgs2d-zm|" in k for k in tuned) and all(v in (4, 8, 16, 32, 64) for v in tuned.values())


def test_batch_whole_row_grids_match_oracle(lm, tmp_path):
    """Sides 64..512 (the workload's divided by 2): the whole-row 2D sweep and
    the per-grid one-block coarse cycles inside the batched graph."""
    lm.autotune_set_cache(str(tmp_path / "tune.json"))
    problems = I.config_batch(count=4, seed=5, scale=2)
    assert any(p.n[0] % 256 == 0 for p in problems)
    grids = _batch(lm, problems)
    try:
        res = lm.batch_solve(grids, rtol=1e-11, max_outer=12, inner_max_iter=12)
        for p, g, r in zip(problems, grids, res):
            assert r["status"] == 0 and r["rel_residual"] <= 1e-11, r
            op = P.operator_from_problem(p)
            xs = P.solve_direct(op, p.f).ravel()
            x = g.solution()
            assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs), p.name
    finally:
        for g in grids:
            g.close()


def test_batch_uneven_convergence_and_tolerance(lm, tmp_path):
    """Grids converge at different steps; each stops at its own tolerance."""
    lm.autotune_set_cache(str(tmp_path / "t.json"))
    problems = [I.make_problem(32, 64, ma=0.1, contrast=5.0, seed=1, rtol=1e-8),
                I.make_problem(64, 32, ma=0.001, contrast=30.0, noise=0.01, seed=2, rtol=1e-8),
                I.make_problem(16, 16, ma=0.01, contrast=10.0, seed=3, rtol=1e-8)]
    grids = _batch(lm, problems)
    try:
        res = lm.batch_solve(grids, rtol=1e-8)
        for p, g, r in zip(problems, grids, res):
            assert r["status"] == 0 and r["rel_residual"] <= 1e-8
            assert P.rel_residual(P.operator_from_problem(p), g.solution(), p.f) <= 1.001e-8
    finally:
        for g in grids:
            g.close()


def test_batch_rejects_bad_inputs(lm):
    p2 = I.config_plain_2d(16)
    p3 = I.config_convection_3d(8)
    g2, g3 = _batch(lm, [p2, p3])
    try:
        with pytest.raises(lm.LowMachError) as e:
            lm.batch_solve([g2, g3])
        assert e.value.code == lm.LM_ERR_INVALID_ARG
        with pytest.raises(lm.LowMachError) as e:
            lm.batch_solve([g2, g2])
        assert e.value.code == lm.LM_ERR_INVALID_ARG
        with pytest.raises(lm.LowMachError):
            lm.batch_solve([g2], nu1=2, nu2=2)
    finally:
        g2.close()
        g3.close()
