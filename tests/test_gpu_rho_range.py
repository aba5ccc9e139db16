"""Density ranges far from 1, through the C ABI (needs a GB300).

The operator is homogeneous in rho: with c_s^2 and dt fixed, scaling rho^n
and rho^{n+1} by s scales c~ and every face conductance by 1/s (Eqs.
cpoiss, kappapoiss), so A x = f has the solution s x*.  The float32 kernels
keep rho in float32 and form face weights from sums and products of rho;
the library rescales its float32 copy of rho by a power of two when rho
leaves the band those formulas are safe in, and refuses the float32 modes
when no scaling fits.  Each case is checked against the float64 oracle."""
import dataclasses

import numpy as np
import pytest

from oracle import multigrid as OM
from oracle import poisson as P
from paper_1112_3507_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_3507_gb300 import build as B
    import os
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()


def lm():
    from paper_1112_3507_gb300 import lowmach
    return lowmach


NEU = I.BC_NEUMANN
BASE = {
    # whole 256-cell rows with walls: the whole-row sweep's wall product
    "rows3d-walls-256x16x8": lambda: I.make_problem(256, 8, 16, ma=0.02, contrast=10.0, noise=0.01, seed=13,
                                                    bc=(NEU, NEU, NEU)),
    "conv3d-16": lambda: I.config_convection_3d(16, seed=2),
    "plain2d-64": lambda: I.config_plain_2d(64, seed=1),
}


def scaled(p, s):
    return dataclasses.replace(p, rho_old=p.rho_old * s, rho_new=p.rho_new * s)


@pytest.mark.parametrize("name", list(BASE))
@pytest.mark.parametrize("s", [1e15, 1e-15])
def test_sweep_with_scaled_density(name, s):
    """One float32 red-black sweep on rho scaled by 1e+-15, vs the oracle's
    sweep on the float32-rounded scaled coefficients."""
    p = scaled(BASE[name](), s)
    op = P.operator_from_problem(p)
    ct32 = op.ct.astype(np.float32).astype(np.float64)
    rho32 = p.rho_new.astype(np.float32).astype(np.float64)
    level = OM.build_hierarchy(ct32, rho32, p.h, p.bc)[0]
    rng = np.random.default_rng(21)
    f = (rng.standard_normal(p.size) / s).astype(np.float32)        # keeps x of order 1
    x0 = rng.standard_normal(p.size).astype(np.float32)
    with lm().Grid.for_problem(p) as g:
        g.set_problem(p)
        fd = torch.as_tensor(f, device="cuda")
        out = torch.empty(p.size, dtype=torch.float32, device="cuda")
        ref = OM.sweep(level, x0.astype(np.float64).reshape(p.shape3), f.astype(np.float64).reshape(p.shape3),
                       "RB").ravel()
        g.mg_sweep(torch.as_tensor(x0, device="cuda"), fd, out, 0)
        got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", list(BASE))
@pytest.mark.parametrize("s", [1e15, 1e-15])
@pytest.mark.parametrize("mode,bar", [("mixed", 1e-8), ("fp64-mg", 1e-10)])
def test_solve_with_scaled_density(name, s, mode, bar):
    """The multigrid modes reach x* = s x*(rho) to the parity bars."""
    p0 = BASE[name]()
    p = scaled(p0, s)
    op = P.operator_from_problem(p)
    xs = P.solve_direct(op, p.f).ravel()
    with lm().Grid.for_problem(p) as g:
        g.set_problem(p)
        r = g.solve(mode=mode, rtol=1e-13, max_iter=2000, max_outer=30)
        x = g.solution()
    assert r["status"] == 0 and r["iters"] <= 60
    assert np.linalg.norm(x - xs) <= bar * np.linalg.norm(xs)


def test_density_range_beyond_float32_is_refused_by_multigrid():
    """rho spanning 1e-30 .. 1e30 fits no power-of-two scaling of a float32
    copy: the multigrid modes return LM_ERR_INVALID_ARG, while the float64
    Jacobi-PCG still solves the system (a checkerboard, so that every face
    joins a light and a heavy cell and A stays well conditioned)."""
    p = I.config_plain_2d(16, seed=4)
    k, _, i = np.indices(p.shape3)
    rho = np.where((i + k) % 2 == 0, 1e-30, 1e30)
    p = dataclasses.replace(p, rho_old=np.ones(p.shape3), rho_new=rho, cs2=p.cs2)
    op = P.operator_from_problem(p)
    xs = P.solve_direct(op, p.f).ravel()
    L = lm()
    with L.Grid.for_problem(p) as g:
        g.set_problem(p)
        for mode in ("mixed", "fp64-mg"):
            with pytest.raises(L.LowMachError) as e:
                g.solve(mode=mode, rtol=1e-10)
            assert e.value.code == L.LM_ERR_INVALID_ARG
        r = g.solve(mode="jacobi", rtol=1e-12, max_iter=100000)
        x = g.solution()
    assert r["status"] == 0
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
