"""Pins of oracle.fractional (one fractional step around the solve, Sec. 2.4
steps (i)-(ix), on the Gresho vortex of Sec. 5.5.2): the limiter and the
MUSCL states, conservation, exactness on uniform states, second-order
advection, the equation-of-state round trip, the vortex's pressure balance,
and the paper's finding that the semi-implicit step's dissipation does not
depend on the Mach number."""
import numpy as np
import pytest

from oracle import fractional as FR
from oracle.poisson import NEUMANN, PERIODIC
from paper_1112_3507_gb300 import inputs as I


def test_minmod():
    a = np.array([1.0, -2.0, 3.0, 0.0, -1.0])
    b = np.array([2.0, -1.0, -3.0, 5.0, -4.0])
    np.testing.assert_array_equal(FR.minmod(a, b), [1.0, -1.0, 0.0, 0.0, -1.0])


def test_muscl_states_exact_on_linear_data_and_no_new_extrema():
    """Linear data: both states equal the face value; a step: the states stay
    within the neighbouring cell values (the TVD property)."""
    q = (2.0 + 0.5 * np.arange(12.0))[None, None, :]
    left, right = FR.muscl_states(q, 2, NEUMANN)
    face = 2.0 + 0.5 * (np.arange(12.0) + 0.5)
    np.testing.assert_allclose(left[0, 0, 1:-2], face[1:-2], rtol=1e-15)
    np.testing.assert_allclose(right[0, 0, 1:-2], face[1:-2], rtol=1e-15)
    step = np.where(np.arange(16) < 8, 1.0, 3.0)[None, None, :]
    left, right = FR.muscl_states(step, 2, PERIODIC)
    assert left.min() >= 1.0 and left.max() <= 3.0 and right.min() >= 1.0 and right.max() <= 3.0


@pytest.mark.parametrize("bc", [(PERIODIC, PERIODIC, PERIODIC), (PERIODIC, PERIODIC, NEUMANN),
                                (NEUMANN, PERIODIC, NEUMANN)])
@pytest.mark.parametrize("shape", [(12, 1, 16), (6, 5, 8)])
def test_advection_conserves(bc, shape):
    """The flux form telescopes: the totals of rho, rho u, e and rho c are
    unchanged (no flux through walls, periodic axes wrap)."""
    rng = np.random.default_rng(3)
    rho = 1.0 + 0.3 * rng.random(shape)
    mom = [rng.standard_normal(shape) * (0.0 if shape[2 - a] == 1 else 1.0) for a in range(3)]
    e = 5.0 + rng.random(shape)
    rc = rho * rng.random(shape)
    h = (0.1, 0.2, 0.15)
    r1, m1, e1, c1 = FR.advect(rho, mom, e, 0.01, h, bc, rho_c=rc)
    for a0, a1 in [(rho, r1), (e, e1), (rc, c1)] + list(zip(mom, m1)):
        assert a1.sum() == pytest.approx(a0.sum(), rel=1e-13, abs=1e-12)


def test_uniform_flow_stays_uniform():
    shape = (8, 1, 10)
    rho = np.full(shape, 1.3)
    mom = [np.full(shape, 0.4), np.zeros(shape), np.full(shape, -0.2)]
    e = np.full(shape, 7.0)
    r1, m1, e1, _ = FR.advect(rho, mom, e, 0.05, (0.1, 1.0, 0.1), (PERIODIC,) * 3)
    np.testing.assert_allclose(r1, rho, rtol=1e-15)
    np.testing.assert_allclose(e1, e, rtol=1e-15)
    for a in range(3):
        np.testing.assert_allclose(m1[a], mom[a], rtol=1e-15, atol=1e-15)


def test_advection_tendency_is_second_order():
    """rho u = rho u0 with u0 constant makes every face velocity u0 (Eq.
    step1), so one step's tendency (rho^{n+1} - rho^n) / dt is the MUSCL
    flux divergence of rho u0; on a smooth monotone profile it approaches
    -u0 d(rho)/dx with an error falling about 4x per halving of h (cells
    next to the walls excluded)."""
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        rho = (1.0 + 0.3 * np.tanh(3.0 * (x - 0.5)))[None, None, :]
        drho = 0.9 / np.cosh(3.0 * (x - 0.5)) ** 2
        u0, dt = 0.7, 1e-3
        mom = [rho * u0, np.zeros_like(rho), np.zeros_like(rho)]
        r1, _, _, _ = FR.advect(rho, mom, np.ones_like(rho), dt, (h, 1.0, 1.0), (NEUMANN, PERIODIC, PERIODIC))
        tend = ((r1 - rho) / dt)[0, 0, 3:-3]
        errs.append(np.abs(tend + u0 * drho[3:-3]).max())
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_eos_round_trip():
    rng = np.random.default_rng(1)
    shape = (4, 3, 5)
    rho = 1 + rng.random(shape)
    mom = [rng.standard_normal(shape) for _ in range(3)]
    p = 2 + rng.random(shape)
    gamma = 5.0 / 3.0
    e = p / (gamma - 1) + 0.5 * sum(m * m for m in mom) / rho
    p1, cs2 = FR.eos_ideal(rho, mom, e, gamma)
    np.testing.assert_allclose(p1, p, rtol=1e-13)
    np.testing.assert_allclose(cs2, gamma * p / rho, rtol=1e-13)


def test_gresho_initial_condition_is_in_radial_balance():
    """Sec. 5.5.2: the printed P(r) balances the centrifugal force,
    dP/dr = rho u_phi^2 / r, checked by central differences along the row
    next to the centre (away from the kinks at r = 0.2, 0.4), and the
    velocity is a rotation (no radial component; the printed components
    (sin t, cos t) u_phi are read as (-sin t, cos t) u_phi, since the
    printed pair points radially outward at t = pi/4)."""
    n = 400
    g = I.gresho_vortex(n, 0.1)
    h = 1.0 / n
    k = n // 2
    P = g["P"][k, 0, :]
    x = (np.arange(n) + 0.5) * h
    z = (k + 0.5) * h
    r = np.sqrt((x - 0.5) ** 2 + (z - 0.5) ** 2)
    uphi = np.sqrt(g["mom"][0][k, 0, :] ** 2 + g["mom"][2][k, 0, :] ** 2)
    dPdx = np.gradient(P, h)             # along the row: dP/dr times (x - 1/2) / r
    ok = (np.abs(r - 0.2) > 3 * h) & (np.abs(r - 0.4) > 3 * h) & (r > 3 * h) & (r < 0.45)
    np.testing.assert_allclose(dPdx[ok], (uphi ** 2 / r * (x - 0.5) / r)[ok], rtol=2e-3, atol=1e-3)
    zz, xx = np.meshgrid((np.arange(n) + 0.5) * h - 0.5, (np.arange(n) + 0.5) * h - 0.5, indexing="ij")
    radial = g["mom"][0][:, 0, :] * xx + g["mom"][2][:, 0, :] * zz
    assert np.abs(radial).max() < 1e-12


def test_one_step_keeps_the_vortex_and_the_pressure_evolution():
    """One full step (i)-(ix) at Ma = 0.01: density stays within 1e-3 of 1,
    kinetic energy changes by less than 1e-3 of itself, and the predicted
    pressure stays within a few units of the background P0 = 1/(gamma Ma^2)
    (the pressure variation is O(1), not O(1/Ma^2))."""
    g = I.gresho_vortex(32, 0.01)
    rho1, mom1, e1, p1, pp = FR.step(g["rho"], g["mom"], g["e"], g["P"], g["dt"], g["h"], g["bc"], g["gamma"])
    ke0 = FR.kinetic_energy(g["rho"], g["mom"], g["h"])
    ke1 = FR.kinetic_energy(rho1, mom1, g["h"])
    assert np.abs(rho1 - 1).max() < 1e-3
    assert abs(ke1 / ke0 - 1) < 1e-3
    p0 = 1.0 / (g["gamma"] * 0.01 ** 2)
    assert np.abs(pp - p0).max() < 5.0 and np.abs(p1 - p0).max() < 5.0


def test_dissipation_does_not_depend_on_the_mach_number():
    """Sec. 5.5.2 (Fig. dissipation1): the semi-implicit step's loss of
    kinetic energy over the same physical time is the same at Ma = 0.1 and
    Ma = 0.01 (here to 5 % of the loss; each Mach number uses its own
    sound-speed-induced step)."""
    losses = []
    for ma in (0.1, 0.01):
        g = I.gresho_vortex(32, ma)
        rho, mom, e, p = g["rho"], g["mom"], g["e"], g["P"]
        ke0 = FR.kinetic_energy(rho, mom, g["h"])
        for _ in range(int(round(0.02 / g["dt"]))):
            rho, mom, e, p, _ = FR.step(rho, mom, e, p, g["dt"], g["h"], g["bc"], g["gamma"])
        losses.append(1 - FR.kinetic_energy(rho, mom, g["h"]) / ke0)
    assert 0 < losses[0] < 0.01
    assert losses[1] == pytest.approx(losses[0], rel=0.05), losses
