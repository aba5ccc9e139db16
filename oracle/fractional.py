"""One fractional step of the semi-implicit method around the pressure
solve, in float64: the explicit advection of steps (i)-(iii), the solve of
step (vi), the projection steps (iv)-(v), (vii)-(viii) (oracle.projection)
and the equation-of-state reset of step (ix) (Sec. 2.4).

Step (i): face velocities u_{i+1/2} = ((rho u)_i + (rho u)_{i+1}) /
(rho_i + rho_{i+1}) (Eq. step1) and the modified flux F~ = (rho, rho c,
rho u, e)_j u_{i+1/2}.  Steps (ii)-(iii): q^{new} = q^n - dt d(F~)/dx, summed
over the axes.  The paper evaluates F~ with its CPM/MENO reconstruction,
which it does not reproduce in the text; reading: the advected quantities
at the face are the upwind side's MUSCL values (van Leer 1979) with the
minmod-limited slope, q_{i+1/2} = q_i + minmod(q_i - q_{i-1}, q_{i+1} - q_i)/2
for u_{i+1/2} > 0 and the mirror image otherwise -- a second-order TVD
reading of "upwinded flux".  On a wall axis the wall face carries no flux
and the slope of a wall cell is zero (its outer neighbour does not exist);
a periodic axis wraps.  The flow is inviscid (F_vis = 0), as in the
paper's Gresho-vortex test.

Step (ix): ideal gas, P = (gamma - 1) (e - |rho u|^2 / (2 rho)), and
c_s^2 = gamma P / rho for the next step's c~ (Eq. cpoiss).

Arrays are numpy (nz, ny, nx); vector fields are lists of three arrays.
Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import poisson as P
from . import projection as PR
from .poisson import NEUMANN, _np_axis


def minmod(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """0 where a and b differ in sign, else the one of smaller magnitude."""
    return np.where(a * b > 0.0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


def _wall_index(a: np.ndarray, ax: int, pos: int) -> tuple:
    idx = [slice(None)] * a.ndim
    idx[ax] = pos
    return tuple(idx)


def muscl_states(q: np.ndarray, ax: int, bc: int):
    """Left and right states at each cell's plus face along numpy axis ax:
    (q_i + s_i / 2, q_{i+1} - s_{i+1} / 2), s the minmod slope (0 in the
    cells next to a wall)."""
    dm = q - np.roll(q, 1, axis=ax)
    dp = np.roll(q, -1, axis=ax) - q
    s = minmod(dm, dp)
    if bc == NEUMANN:
        s[_wall_index(s, ax, 0)] = 0.0
        s[_wall_index(s, ax, -1)] = 0.0
    left = q + 0.5 * s
    right = np.roll(q - 0.5 * s, -1, axis=ax)
    return left, right


def advect(rho, mom, e, dt, h, bc, rho_c=None):
    """Steps (i)-(iii): returns (rho^{n+1}, (rho u)*, e*, (rho c)^{n+1} or None)."""
    qs = [rho, mom[0], mom[1], mom[2], e] + ([rho_c] if rho_c is not None else [])
    out = [np.array(q, dtype=np.float64, copy=True) for q in qs]
    for a in range(3):
        ax = _np_axis(a)
        if rho.shape[ax] == 1:
            continue
        m = mom[a]
        u = (m + np.roll(m, -1, axis=ax)) / (rho + np.roll(rho, -1, axis=ax))   # plus face, Eq. step1
        if bc[a] == NEUMANN:
            u[_wall_index(u, ax, -1)] = 0.0
        for q, o in zip(qs, out):
            left, right = muscl_states(q, ax, bc[a])
            flux = np.where(u > 0.0, left, right) * u
            o -= dt * (flux - np.roll(flux, 1, axis=ax)) / h[a]
    rho1, m1x, m1y, m1z, e1 = out[:5]
    return rho1, [m1x, m1y, m1z], e1, (out[5] if rho_c is not None else None)


def eos_ideal(rho, mom, e, gamma: float):
    """Step (ix): P = (gamma - 1)(e - |rho u|^2 / (2 rho)), c_s^2 = gamma P / rho."""
    kin = 0.5 * (mom[0] ** 2 + mom[1] ** 2 + mom[2] ** 2) / rho
    p = (gamma - 1.0) * (e - kin)
    return p, gamma * p / rho


def step(rho, mom, e, p, dt, h, bc, gamma, solve=None):
    """One fractional step (i)-(ix) with the pressure solve of step (vi)
    done by `solve(op, f)` (default: sparse direct).  Returns
    (rho, mom, e, P, P_pred)."""
    if solve is None:
        solve = P.solve_direct
    cs2 = gamma * p / rho
    rho1, mom_s, e_s, _ = advect(rho, mom, e, dt, h, bc)
    f, uf_s = PR.rhs(p, rho, cs2, mom, mom_s, rho1, dt, h, bc)
    op = P.operator_from_state(rho, rho1, cs2, dt, h, bc)
    p_pred = solve(op, f).reshape(rho.shape)
    mom1, _, e1 = PR.update(p_pred, rho1, mom_s, uf_s, e_s, dt, h, bc)
    p1, _ = eos_ideal(rho1, mom1, e1, gamma)
    return rho1, mom1, e1, p1, p_pred


def kinetic_energy(rho, mom, h) -> float:
    """sum over cells of |rho u|^2 / (2 rho) times the cell volume."""
    vol = float(np.prod([v for v in h]))
    return float(np.sum(0.5 * (mom[0] ** 2 + mom[1] ** 2 + mom[2] ** 2) / rho) * vol)
