"""Pins of oracle.projection (the steps either side of the solve, Sec. 2,
steps (iv)-(viii)): the interpolation and difference formulas on cases with
known answers, conservation, and the discrete pressure-evolution identity
that ties the right-hand side, the operator and the face update together."""
import numpy as np
import pytest

from oracle import poisson as P
from oracle import projection as J
from oracle.poisson import NEUMANN, PERIODIC


def _state(shape, bc, seed=1):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = (np.arange(nz) + 0.5) / nz
    rho_o = (1.0 - 0.8 * z)[:, None, None] * (1.0 + 0.05 * rng.uniform(-1, 1, shape))
    rho_n = rho_o * (1.0 + 0.02 * rng.uniform(-1, 1, shape))
    p_o = (1.0 - 0.8 * z)[:, None, None] ** 1.6 * (1.0 + 0.01 * rng.uniform(-1, 1, shape))
    cs2 = 5.0 / 3.0 * p_o / rho_o
    m_o = [0.1 * rng.standard_normal(shape) * rho_o for _ in range(3)]
    m_s = [mc + 0.01 * rng.standard_normal(shape) for mc in m_o]
    if ny == 1:
        m_o[1][:] = 0.0
        m_s[1][:] = 0.0
    return rho_o, rho_n, p_o, cs2, m_o, m_s


def test_face_pressure_is_eq_pbnd():
    P0 = np.array([[[1.0, 3.0]]])
    rho = np.array([[[2.0, 6.0]]])
    pf = J.face_pressure(P0, rho, 0, (PERIODIC, PERIODIC, PERIODIC))
    # face between cell 0 and 1: (P_1 rho_0 + P_0 rho_1) / (rho_0 + rho_1) = (3*2 + 1*6) / 8
    assert pf[0, 0, 1] == pytest.approx(12.0 / 8.0)
    assert pf[0, 0, 0] == pytest.approx(12.0 / 8.0)           # periodic: the same face seen from cell 0
    c = np.full((4, 3, 5), 2.5)
    r = np.random.default_rng(0).uniform(0.5, 2.0, c.shape)
    for a in range(3):
        np.testing.assert_allclose(J.face_pressure(c, r, a, (NEUMANN,) * 3), 2.5)


def test_gradient_of_linear_pressure():
    """Constant density: the face value is the midpoint, so interior cells
    see the exact slope (a central difference)."""
    nx = 12
    x = np.arange(nx, dtype=float)
    Pl = np.broadcast_to(3.0 * x * 0.1, (4, 2, nx)).copy()
    rho = np.full(Pl.shape, 1.7)
    g = J.grad_p(Pl, rho, (0.1, 1.0, 1.0), (NEUMANN, PERIODIC, PERIODIC))
    np.testing.assert_allclose(g[0][:, :, 1:-1], 3.0, rtol=1e-12)
    np.testing.assert_allclose(g[1], 0.0, atol=1e-12)
    np.testing.assert_allclose(g[2], 0.0, atol=1e-12)
    # next to the wall the mirror ghost halves the one-sided slope
    np.testing.assert_allclose(g[0][:, :, 0], 1.5, rtol=1e-12)


@pytest.mark.parametrize("bc", [(PERIODIC, PERIODIC, NEUMANN), (PERIODIC, PERIODIC, PERIODIC),
                                (NEUMANN, NEUMANN, NEUMANN)])
def test_divergence_telescopes(bc):
    rho_o, rho_n, p_o, cs2, m_o, m_s = _state((6, 5, 8), bc)
    uf = J.face_velocity(m_s, rho_n, bc)
    assert abs(J.divergence(uf, (0.1, 0.2, 0.3), bc).sum()) <= 1e-12 * sum(np.abs(u).sum() for u in uf) * 30


@pytest.mark.parametrize("shape,bc", [((8, 6, 10), (PERIODIC, PERIODIC, NEUMANN)),
                                      ((12, 1, 16), (PERIODIC, PERIODIC, NEUMANN)),
                                      ((6, 6, 6), (NEUMANN, NEUMANN, NEUMANN))])
@pytest.mark.parametrize("with_source", [False, True])
def test_pressure_evolution_identity(shape, bc, with_source):
    """After solving A P = f (Eq. Poiss with f from Eq. fpoiss) and updating
    the face velocities (step (vii)), their divergence is the discrete
    pressure evolution: div u^{n+1} = (P^n - dt u^n.grad P^n - P) / (dt rho^n c^2) - dt S.
    A sign or index slip in f, in the face update or in the operator breaks it."""
    nz, ny, nx = shape
    h = (1.0 / nz,) * 3
    rho_o, rho_n, p_o, cs2, m_o, m_s = _state(shape, bc, seed=3)
    dt = 0.5 * h[2] / (0.01 * np.sqrt(cs2.max()))
    S = 0.1 * np.random.default_rng(4).standard_normal(shape) if with_source else None
    f, uf = J.rhs(p_o, rho_o, cs2, m_o, m_s, rho_n, dt, h, bc, S)
    op = P.operator_from_state(rho_o, rho_n, cs2, dt, h, bc)
    Pp = P.solve_direct(op, f)
    e_s = np.random.default_rng(5).uniform(1.0, 2.0, shape)
    m_new, uf_new, e_new = J.update(Pp, rho_n, m_s, uf, e_s, dt, h, bc)
    u_o = [mc / rho_o for mc in m_o]
    gp = J.grad_p(p_o, rho_o, h, bc)
    want = (p_o - dt * sum(u_o[a] * gp[a] for a in range(3)) - Pp) / (dt * rho_o * cs2)
    if S is not None:
        want = want - dt * S
    got = J.divergence(uf_new, h, bc)
    scale = np.abs(J.divergence(uf, h, bc)).max()
    assert np.max(np.abs(got - want)) <= 1e-8 * scale


def test_momentum_and_energy_on_linear_pressure():
    """P_pred linear in x, uniform density and momentum: the momentum loses
    dt * slope, the face velocities dt * slope / rho, and the interior
    energy changes by -dt u^{n+1} * slope (div u^{n+1} = 0 there)."""
    nx, ny, nz = 16, 2, 4
    h = (0.1, 1.0, 1.0)
    bc = (NEUMANN, PERIODIC, PERIODIC)
    x = np.arange(nx, dtype=float) * h[0]
    Pp = np.broadcast_to(2.0 * x, (nz, ny, nx)).copy()
    rho = np.full(Pp.shape, 1.25)
    m_s = [np.full(Pp.shape, 0.5), np.zeros(Pp.shape), np.zeros(Pp.shape)]
    uf = J.face_velocity(m_s, rho, bc)
    e_s = np.full(Pp.shape, 3.0)
    dt = 0.01
    m_new, uf_new, e_new = J.update(Pp, rho, m_s, uf, e_s, dt, h, bc)
    np.testing.assert_allclose(m_new[0][:, :, 1:-1], 0.5 - dt * 2.0, rtol=1e-12)
    np.testing.assert_allclose(uf_new[0][:, :, 1:], 0.5 / 1.25 - dt * 2.0 / 1.25, rtol=1e-12)
    assert np.all(uf_new[0][:, :, 0] == 0.0)
    u_new = (0.5 - dt * 2.0) / 1.25
    np.testing.assert_allclose(e_new[:, :, 2:-2], 3.0 - dt * u_new * 2.0, rtol=1e-12)
