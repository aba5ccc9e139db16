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
    assert any("|rbgs2d-zrow|" in k for k in tuned) and any("|rbgs2d-batch-zrow|" in k for k in tuned)
    assert all(v in (8, 16, 32, 64, 128, 256) for v in tuned.values())


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
            lm.batch_solve([g2], nu1=0, nu2=2)
        with pytest.raises(lm.LowMachError):
            lm.batch_solve([g2], nu1=2, nu2=9)
    finally:
        g2.close()
        g3.close()


@pytest.mark.parametrize("nu", [(2, 3), (1, 2), (3, 1)])
def test_batch_any_smoothing_counts(lm, tmp_path, nu):
    """The library's default smoothing (nu1 = 2, nu2 = 3) and other counts in
    the batched V-cycle: solutions match the direct solves; the one-block
    coarse cycles and the whole-row sweeps take the same counts."""
    lm.autotune_set_cache(str(tmp_path / "t.json"))
    problems = I.config_batch(count=5, seed=7, scale=4)
    grids = _batch(lm, problems)
    try:
        res = lm.batch_solve(grids, rtol=1e-11, max_outer=12, inner_max_iter=12, nu1=nu[0], nu2=nu[1])
        for p, g, r in zip(problems, grids, res):
            assert r["status"] == 0 and r["rel_residual"] <= 1e-11, r
            op = P.operator_from_problem(p)
            xs = P.solve_direct(op, p.f).ravel()
            assert np.linalg.norm(g.solution() - xs) <= 1e-8 * np.linalg.norm(xs), p.name
    finally:
        for g in grids:
            g.close()


def test_batch_set_coefficients_matches_per_grid(lm):
    """lm_batch_set_coefficients (one launch for all grids) leaves every grid
    with the coefficients lm_set_coefficients gives, bit for bit; a grid with
    a non-positive density is reported and left without coefficients."""
    problems = I.config_batch(count=6, seed=11, scale=8)
    ga, gb = _batch(lm, problems), [lm.Grid.for_problem(p) for p in problems]
    try:
        tens = [[torch.as_tensor(a.ravel(), device="cuda") for a in (p.rho_old, p.rho_new, p.cs2)] for p in problems]
        lm.batch_set_coefficients(gb, [t[0] for t in tens], [t[1] for t in tens], [t[2] for t in tens],
                                  [p.dt for p in problems])
        for a, b in zip(ga, gb):
            for x, y in zip(a.coefficients(), b.coefficients()):
                assert torch.equal(x, y)
        bad = [t[1].clone() for t in tens]
        bad[2][5] = -1.0
        with pytest.raises(lm.LowMachError) as e:
            lm.batch_set_coefficients(gb, [t[0] for t in tens], bad, [t[2] for t in tens], [p.dt for p in problems])
        assert e.value.code == lm.LM_ERR_NOT_POSITIVE
        with pytest.raises(lm.LowMachError) as e:
            gb[2].coefficients()
        assert e.value.code == lm.LM_ERR_STATE
        gb[0].coefficients()                       # the other grids were assembled
    finally:
        for g in ga + gb:
            g.close()


def test_batch_refresh_after_new_coefficients(lm, tmp_path):
    """Solve, assemble new coefficients for every grid in one launch, solve
    again: the hierarchies are refreshed level by level over all grids and
    the coarsest inverses one block per grid; both solves match the oracle."""
    lm.autotune_set_cache(str(tmp_path / "t.json"))
    first = I.config_batch(count=5, seed=13, scale=8)
    second = I.config_batch(count=5, seed=14, scale=8)
    shapes = [p.n for p in first]
    second = [I.make_problem(p.n[0], p.n[2], ma=q.ma if q.ma else 0.01, contrast=12.0, noise=0.01, seed=60 + i)
              for i, (p, q) in enumerate(zip(first, second))]
    assert [p.n for p in second] == shapes
    grids = _batch(lm, first)
    try:
        for probs in (first, second):
            tens = [[torch.as_tensor(a.ravel(), device="cuda") for a in (p.rho_old, p.rho_new, p.cs2, p.f)]
                    for p in probs]
            lm.batch_set_coefficients(grids, [t[0] for t in tens], [t[1] for t in tens], [t[2] for t in tens],
                                      [p.dt for p in probs])
            for g, t in zip(grids, tens):
                g.set_rhs(t[3])
            res = lm.batch_solve(grids, rtol=1e-11, max_outer=12, inner_max_iter=12)
            for p, g, r in zip(probs, grids, res):
                assert r["status"] == 0, r
                xs = P.solve_direct(P.operator_from_problem(p), p.f).ravel()
                assert np.linalg.norm(g.solution() - xs) <= 1e-8 * np.linalg.norm(xs)
    finally:
        for g in grids:
            g.close()


def test_batch_full_size_1024_grid_matches_oracle(lm, tmp_path):
    """A 1024 x 1024 grid of the 64-solve workload's largest size class,
    batched with smaller ones, against the oracle's direct solve."""
    lm.autotune_set_cache(str(tmp_path / "t.json"))
    problems = [I.make_problem(1024, 1024, ma=0.003, contrast=20.0, noise=0.01, seed=71, rtol=1e-8),
                I.make_problem(256, 512, ma=0.05, contrast=8.0, noise=0.01, seed=72, rtol=1e-8),
                I.make_problem(128, 128, ma=0.001, contrast=30.0, noise=0.01, seed=73, rtol=1e-8)]
    grids = _batch(lm, problems)
    try:
        res = lm.batch_solve(grids, rtol=1e-11, max_outer=12, inner_max_iter=15)
        for p, g, r in zip(problems, grids, res):
            assert r["status"] == 0 and r["rel_residual"] <= 1e-11, r
            xs = P.solve_direct(P.operator_from_problem(p), p.f).ravel()
            assert np.linalg.norm(g.solution() - xs) <= 1e-8 * np.linalg.norm(xs), p.name
    finally:
        for g in grids:
            g.close()
