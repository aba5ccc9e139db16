"""The Q1 finite-element operator on the GPU (lm_fe_*, Sec. 2.5) against
oracle.fem: the float64 and float32 apply element by element, the lumped
mass, Jacobi-PCG and the mixed solve against the oracle's direct solve, the
paper's e^x error table (Sec. 2.5.2, Table perturbtest) reproduced through
the C ABI, and the positivity check (needs a GB300)."""
import os
from pathlib import Path

import numpy as np
import pytest

from oracle import fem as F
from oracle.poisson import NEUMANN, PERIODIC
from paper_1112_3507_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = Path(__file__).parent / "golden" / "perturbtest_table.txt"


@pytest.fixture(scope="module")
def lm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_3507_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()
    from paper_1112_3507_gb300 import lowmach
    return lowmach


# (points per axis, spacings, boundary conditions): 2D and 3D, partial
# 32 x 8 column tiles, cubic (face weights zero) and stretched elements
CASES = [((17, 1, 20), (0.1, 1.0, 0.08), (NEUMANN, PERIODIC, PERIODIC)),
         ((64, 1, 65), (1 / 64, 1.0, 1 / 64), (PERIODIC, PERIODIC, NEUMANN)),
         ((40, 12, 17), (0.1, 0.1, 0.1), (PERIODIC, PERIODIC, NEUMANN)),
         ((33, 9, 10), (0.2, 0.3, 0.25), (NEUMANN, PERIODIC, NEUMANN)),
         ((8, 8, 8), (0.5, 0.5, 0.5), (NEUMANN, NEUMANN, NEUMANN)),
         ((70, 20, 6), (0.05, 0.05, 0.05), (PERIODIC, PERIODIC, PERIODIC))]


def _coefs(n, seed, spread=2.0):
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    rho = np.exp(rng.uniform(-spread, spread, shape))
    ct = np.exp(rng.uniform(-1.0, 1.0, shape))
    return ct, rho, rng


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=dtype, device="cuda")


@pytest.mark.parametrize("n,h,bc", CASES)
def test_apply_fp64_matches_oracle(lm, n, h, bc):
    """y = B x and x^T B x in float64, element by element against the oracle."""
    ct, rho, rng = _coefs(n, sum(n))
    op = F.FEOperator(ct, rho, h, bc)
    x = rng.standard_normal(ct.shape)
    ref = op.apply(x).ravel()
    # rounding scale of each row: |V c~ x| + sum over the element terms
    scale = np.abs(op.volume * ct * x).ravel() + (np.abs(op.assemble()) @ np.abs(x.ravel()))
    with lm.FEGrid(n, h, bc) as g:
        g.set_coefficients(ct, rho)
        xd = _dev(x)
        y = torch.empty_like(xd)
        dot = g.apply(xd, y, prec=lm.PREC_FP64, with_dot=True)
        got = y.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-14 * scale)
    assert dot == pytest.approx(float(x.ravel() @ ref), rel=1e-12)


@pytest.mark.parametrize("n,h,bc", CASES)
def test_apply_fp32_matches_oracle(lm, n, h, bc):
    """y = B x in float32 (column-marching kernel in 3D) against the oracle on
    the same float32-rounded input, relative to each row's magnitude."""
    ct, rho, rng = _coefs(n, 7 + sum(n))
    op = F.FEOperator(ct, rho, h, bc)
    x = rng.standard_normal(ct.shape).astype(np.float32).astype(np.float64)
    ref = op.apply(x).ravel()
    scale = np.abs(op.volume * ct * x).ravel() + (np.abs(op.assemble()) @ np.abs(x.ravel()))
    with lm.FEGrid(n, h, bc) as g:
        g.set_coefficients(ct, rho)
        xd = _dev(x, torch.float32)
        y = torch.empty_like(xd)
        dot = g.apply(xd, y, prec=lm.PREC_FP32, with_dot=True)
        got = y.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2e-6 * scale)
    assert dot == pytest.approx(float(x.ravel() @ ref), rel=1e-5)


@pytest.mark.parametrize("n,h,bc", CASES[:4])
def test_lumped_mass(lm, n, h, bc):
    ct, rho, _ = _coefs(n, 3)
    op = F.FEOperator(ct, rho, h, bc)
    with lm.FEGrid(n, h, bc) as g:
        v = g.lumped_mass()
    np.testing.assert_allclose(v, op.volume.ravel(), rtol=1e-15)


SOLVE_CASES = [CASES[0], CASES[2], ((33, 10, 10), (0.2, 0.3, 0.25), (NEUMANN, PERIODIC, NEUMANN))]


@pytest.mark.parametrize("mode,rtol,tol", [("jacobi", 1e-12, 1e-9), ("mixed", 1e-12, 1e-9)])
@pytest.mark.parametrize("n,h,bc", SOLVE_CASES)
def test_solve_matches_direct(lm, mode, rtol, tol, n, h, bc):
    """Both solvers reach the oracle's sparse direct solution (condition
    numbers below 1e3 here, so a 1e-12 residual bounds the error by 1e-9)."""
    ct, rho, rng = _coefs(n, 11 + sum(n), spread=1.5)
    op = F.FEOperator(ct, rho, h, bc)
    b = op.volume * rng.standard_normal(ct.shape)
    ref = F.solve(op, b).ravel()
    x = np.zeros(op.size)
    with lm.FEGrid(n, h, bc) as g:
        g.set_coefficients(ct, rho)
        r = g.solve(b.ravel(), x, mode=mode, rtol=rtol, max_iter=20000)
    assert r["rel_residual"] <= rtol
    assert np.linalg.norm(x - ref) <= tol * np.linalg.norm(ref)
    # the reported residual is the oracle's
    res = np.linalg.norm(b.ravel() - op.apply(x).ravel()) / np.linalg.norm(b)
    assert res == pytest.approx(r["rel_residual"], rel=1e-3, abs=1e-15)


def test_mixed_needs_even_periodic_counts(lm):
    """The mixed solve's preconditioner is the red-black cell-centred V-cycle,
    which needs an even number of points on every periodic axis: an odd one
    is refused (LM_ERR_INVALID_ARG), and Jacobi-PCG still solves it."""
    n, h, bc = CASES[3]
    ct, rho, rng = _coefs(n, 4, spread=1.0)
    op = F.FEOperator(ct, rho, h, bc)
    b = op.volume * rng.standard_normal(ct.shape)
    x = np.zeros(op.size)
    with lm.FEGrid(n, h, bc) as g:
        g.set_coefficients(ct, rho)
        with pytest.raises(lm.LowMachError) as e:
            g.solve(b.ravel(), x, mode="mixed", rtol=1e-10)
        assert e.value.code == lm.LM_ERR_INVALID_ARG
        r = g.solve(b.ravel(), x, mode="jacobi", rtol=1e-12)
    assert r["rel_residual"] <= 1e-12


def test_mixed_solve_device_buffers_and_initial_guess(lm):
    """Device-resident b and x, and a warm start from the solution of a
    neighbouring right-hand side, through the same entry point."""
    n, h, bc = (48, 16, 33), (1 / 47, 1 / 47, 1 / 32), (NEUMANN, PERIODIC, NEUMANN)
    ct, rho, rng = _coefs(n, 5, spread=1.0)
    op = F.FEOperator(ct, rho, h, bc)
    b = op.volume * rng.standard_normal(ct.shape)
    ref = F.solve(op, b).ravel()
    with lm.FEGrid(n, h, bc) as g:
        g.set_coefficients(_dev(ct), _dev(rho))
        bd, xd = _dev(b), torch.zeros(op.size, dtype=torch.float64, device="cuda")
        r1 = g.solve(bd, xd, mode="mixed", rtol=1e-9)
        bd2 = _dev(b * 1.001)
        r2 = g.solve(bd2, xd, mode="mixed", rtol=1e-9, use_x0=1)
        got = xd.cpu().numpy()
    assert r1["rel_residual"] <= 1e-9 and r2["rel_residual"] <= 1e-9
    assert r2["iters"] < r1["iters"]
    assert np.linalg.norm(got - 1.001 * ref) <= 1e-7 * np.linalg.norm(ref)


def _golden():
    rows = {}
    for line in GOLDEN.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows[name] = [float(v) for v in vals]
    return rows


@pytest.mark.parametrize("mode", ["jacobi", "mixed"])
def test_exp_test_reproduces_the_papers_table(lm, mode):
    """Sec. 2.5.2: -Lap(phi) + phi = 0 with phi = e^x, 100 intervals per
    direction, solved on the GPU: the L1, L2 and Linf errors against e^x are
    the paper's unperturbed row (Table perturbtest) within 0.5 %."""
    t = I.analytic_exp_problem_nodes(101)
    op = F.FEOperator(t["ctilde"], 1.0 / t["kappa"], t["h"], t["bc"])
    b = op.volume * t["f"]
    b[:, :, 0] += t["g_low"] * t["h"][2]
    b[:, :, -1] += t["g_high"] * t["h"][2]
    x = np.zeros(op.size)
    with lm.FEGrid(t["n"], t["h"], t["bc"]) as g:
        g.set_coefficients(t["ctilde"], 1.0 / t["kappa"])
        r = g.solve(b.ravel(), x, mode=mode, rtol=1e-12, max_iter=50000, inner_max_iter=200)
    assert r["rel_residual"] <= 1e-12
    err = np.abs(x.reshape(op.shape) - t["exact"])
    got = (err.mean(), np.sqrt(np.mean(err ** 2)), err.max())
    for gv, wv in zip(got, _golden()["unperturbed_1core"]):
        assert gv == pytest.approx(wv, rel=5e-3), got


def test_not_positive_and_state(lm):
    n, h, bc = (8, 1, 9), (0.1, 1.0, 0.1), (NEUMANN, PERIODIC, PERIODIC)
    ct, rho, _ = _coefs(n, 1)
    with lm.FEGrid(n, h, bc) as g:
        x = torch.zeros(g.N, dtype=torch.float64, device="cuda")
        with pytest.raises(lm.LowMachError) as e:
            g.apply(x, torch.empty_like(x))
        assert e.value.code == lm.LM_ERR_STATE
        bad = rho.copy()
        bad[3, 0, 4] = 0.0
        with pytest.raises(lm.LowMachError) as e:
            g.set_coefficients(ct, bad)
        assert e.value.code == lm.LM_ERR_NOT_POSITIVE
        g.set_coefficients(ct, rho)
        g.apply(x, torch.empty_like(x))
    with pytest.raises(lm.LowMachError) as e:
        lm.FEGrid((8, 1, 1), h, bc, ndim=2)
    assert e.value.code == lm.LM_ERR_INVALID_ARG


def test_full_size_apply_sampled_and_solve(lm):
    """256^3 points, the convection recipe's coefficients: float64 and float32
    B x checked on sampled rows computed by the oracle's element sums one by
    one, and the mixed solve's float64 residual recomputed by the oracle."""
    p = I.config_convection_3d(256, seed=1)
    ct = 1.0 / ((p.dt * p.dt) * p.rho_old * p.cs2)
    n, h = p.n, (1 / 256, 1 / 256, 1 / 255)
    bc = p.bc
    rng = np.random.default_rng(9)
    x = rng.standard_normal(ct.shape)
    with lm.FEGrid(n, h, bc) as g:
        g.set_coefficients(_dev(ct), _dev(p.rho_new))
        xd = _dev(x)
        y = torch.empty_like(xd)
        g.apply(xd, y)
        y64 = y.cpu().numpy().reshape(ct.shape)
        x32 = xd.float()
        y32 = torch.empty_like(x32)
        g.apply(x32, y32, prec=lm.PREC_FP32)
        y32 = y32.cpu().numpy().astype(np.float64).reshape(ct.shape)
        v = g.lumped_mass().reshape(ct.shape)
        b = v * p.f
        sol = torch.zeros(g.N, dtype=torch.float64, device="cuda")
        r = g.solve(_dev(b), sol, mode="mixed", rtol=1e-8)
        sol = sol.cpu().numpy().reshape(ct.shape)
    # sampled rows: a 6 x 6 x 6 sub-box around each sample, the oracle on it
    # with the sub-box's own elements only at its interior point
    nz, ny, nx = ct.shape
    x32r = x.astype(np.float32).astype(np.float64)
    for s in range(24):
        k, j, i = (int(rng.integers(0, m)) for m in (nz, ny, nx))
        zi = [(k + d) % nz for d in (-1, 0, 1)]
        yi = [(j + d) % ny for d in (-1, 0, 1)]
        xi = [(i + d) % nx for d in (-1, 0, 1)]
        want64 = _row(ct, p.rho_new, x, h, bc, zi, yi, xi, (k, j, i))
        want32 = _row(ct, p.rho_new, x32r, h, bc, zi, yi, xi, (k, j, i))
        assert abs(y64[k, j, i] - want64[0]) <= 1e-13 * want64[1]
        assert abs(y32[k, j, i] - want32[0]) <= 3e-6 * want32[1]
    assert r["rel_residual"] <= 1e-8
    op = F.FEOperator(ct, p.rho_new, h, bc)
    res = np.linalg.norm(b - op.apply(sol)) / np.linalg.norm(b)
    assert res <= 1.01e-8


def _row(ct, rho, x, h, bc, zi, yi, xi, kji):
    """(B x) at one point from the element definitions: the 8 elements around
    it, each kappa_e K_ref applied to its corner values (oracle.fem's
    reference element), plus the lumped c~ term; returns (value, magnitude)."""
    import itertools
    nz, ny, nx = ct.shape
    k, j, i = kji
    full = (nx, ny, nz)
    ref = F.FEOperator(np.ones((2, 2, 2)), np.ones((2, 2, 2)), h, (NEUMANN,) * 3).kref
    corners = list(itertools.product((0, 1), repeat=3))
    val, mag = 0.0, 0.0
    for d in corners:                          # element whose corner d is our point
        low = [(i - d[0]), (j - d[1]), (k - d[2])]
        if any(bc[a] == NEUMANN and not (0 <= low[a] <= full[a] - 2) for a in range(3)):
            continue
        pts = [((low[2] + c[2]) % nz, (low[1] + c[1]) % ny, (low[0] + c[0]) % nx) for c in corners]
        kap = 8.0 / sum(rho[q] for q in pts)
        p = corners.index((d[0], d[1], d[2]))
        for q, pt in enumerate(pts):
            val += kap * ref[p, q] * x[pt]
            mag += abs(kap * ref[p, q] * x[pt])
    vol = 1.0
    for a, c in enumerate((i, j, k)):
        vol *= 0.5 * h[a] if (bc[a] == NEUMANN and c in (0, full[a] - 1)) else h[a]
    val += vol * ct[k, j, i] * x[k, j, i]
    mag += abs(vol * ct[k, j, i] * x[k, j, i])
    return val, mag
