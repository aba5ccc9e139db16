"""The steps either side of the pressure solve, in float64: the right-hand
side assembly and the projection update of one fractional step.

Sec. 2 of the paper (the Kwatra-type algorithm, steps (iv)-(viii)):

  pressure at faces   P_{i+1/2} = (P_{i+1} rho_i + P_i rho_{i+1}) / (rho_i + rho_{i+1})   (Eq. pbnd)
  cell gradient       (grad P)_i = (P_{i+1/2} - P_{i-1/2}) / dx                           (Eq. nablaP)
  face velocity       u_{i+1/2} = ((rho u)_i + (rho u)_{i+1}) / (rho_i + rho_{i+1})       (the MAC value, Sec. 2.3)
  divergence          (div u)_i = sum over axes (u_{i+1/2} - u_{i-1/2}) / dx
  right-hand side     f = (P^n - dt u^n . grad P^n) / (dt^2 rho^n c^2) - (div u*) / dt - S (Eq. fpoiss)
  momentum            (rho u)^{n+1} = (rho u)* - dt grad P_pred                          (Eq. momupdate)
  face velocity       u^{n+1}_{i+1/2} = u*_{i+1/2} - dt (P_{i+1} - P_i)/dx * 2/(rho_{i+1} + rho_i)   (step (vii))
  energy              e^{n+1} = e* - dt (P_pred div u^{n+1} + u^{n+1} . grad P_pred)       (step (viii))

S stands for the viscous and conductive part of Eq. fpoiss (the terms in
tau and K), which the caller supplies already divided as printed (0 for
the inviscid case).  The paper leaves the boundaries of these steps to its
walls (Eq. vonNeumannBC) and periodic axes (Sec. 3.2); reading: on a wall
axis the face at the wall carries no velocity (u = 0 there) and its
pressure is the wall cell's (zero normal gradient, a mirror ghost with the
same density); a periodic axis wraps.  Cell velocities are momentum over
density: u^n = (rho u)^n / rho^n, u^{n+1} = (rho u)^{n+1} / rho^{n+1}; the
pressure interpolation uses the density of the pressure's own time level
(rho^n for P^n, rho^{n+1} for P_pred).

Arrays are numpy (nz, ny, nx); vector fields are lists of three arrays
(x, y, z components); face arrays hold, per axis, each cell's MINUS face
(the face between cell i-1 and i), as the operator's conductances do.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .poisson import NEUMANN, PERIODIC, _np_axis


def _wall_first(a: np.ndarray, ax: int) -> tuple:
    idx = [slice(None)] * a.ndim
    idx[ax] = 0
    return tuple(idx)


def face_pressure(P: np.ndarray, rho: np.ndarray, a: int, bc) -> np.ndarray:
    """Eq. pbnd on every cell's minus face along grid axis a (the wall face
    of a Neumann axis takes the wall cell's pressure)."""
    ax = _np_axis(a)
    Pm, rm = np.roll(P, 1, axis=ax), np.roll(rho, 1, axis=ax)
    pf = (P * rm + Pm * rho) / (rm + rho)
    if bc[a] == NEUMANN:
        pf[_wall_first(pf, ax)] = P[_wall_first(P, ax)]
    return pf


def _plus(face_minus: np.ndarray, a: int, bc, wall_value: np.ndarray | None = None) -> np.ndarray:
    """Each cell's plus face from the minus faces: the next cell's minus face;
    on a wall axis the last cell's plus face is the wall (wall_value there)."""
    ax = _np_axis(a)
    fp = np.roll(face_minus, -1, axis=ax)
    if bc[a] == NEUMANN:
        idx = [slice(None)] * fp.ndim
        idx[ax] = -1
        fp[tuple(idx)] = 0.0 if wall_value is None else wall_value[tuple(idx)]
    return fp


def grad_p(P: np.ndarray, rho: np.ndarray, h, bc) -> list:
    """Eq. nablaP per axis (zero along axes with one cell)."""
    out = []
    for a in range(3):
        if P.shape[_np_axis(a)] == 1:
            out.append(np.zeros_like(P))
            continue
        pm = face_pressure(P, rho, a, bc)
        pp = _plus(pm, a, bc, wall_value=P)
        out.append((pp - pm) / h[a])
    return out


def face_velocity(m: list, rho: np.ndarray, bc) -> list:
    """u on every cell's minus face per axis: ((rho u)_{i-1} + (rho u)_i) /
    (rho_{i-1} + rho_i); 0 at walls and along axes with one cell."""
    out = []
    for a in range(3):
        ax = _np_axis(a)
        if rho.shape[ax] == 1:
            out.append(np.zeros_like(rho))
            continue
        u = (np.roll(m[a], 1, axis=ax) + m[a]) / (np.roll(rho, 1, axis=ax) + rho)
        if bc[a] == NEUMANN:
            u[_wall_first(u, ax)] = 0.0
        out.append(u)
    return out


def divergence(uf: list, h, bc) -> np.ndarray:
    """sum over axes of (u_{i+1/2} - u_{i-1/2}) / dx from minus-face values."""
    d = np.zeros_like(uf[0])
    for a in range(3):
        if uf[a].shape[_np_axis(a)] == 1:
            continue
        d = d + (_plus(uf[a], a, bc) - uf[a]) / h[a]
    return d


def rhs(P_old, rho_old, cs2_old, m_old, m_star, rho_new, dt, h, bc, S=None):
    """Eq. fpoiss: returns (f, u*_faces)."""
    u_old = [mc / rho_old for mc in m_old]
    gp = grad_p(P_old, rho_old, h, bc)
    adv = sum(u_old[a] * gp[a] for a in range(3))
    uf = face_velocity(m_star, rho_new, bc)
    f = (P_old - dt * adv) / (dt * dt * rho_old * cs2_old) - divergence(uf, h, bc) / dt
    if S is not None:
        f = f - S
    return f, uf


def update(P_pred, rho_new, m_star, uf_star, e_star, dt, h, bc):
    """Steps (vi)-(viii): returns (momentum^{n+1}, face velocities^{n+1}, e^{n+1})."""
    gp = grad_p(P_pred, rho_new, h, bc)
    m_new = [m_star[a] - dt * gp[a] for a in range(3)]
    uf_new = []
    for a in range(3):
        ax = _np_axis(a)
        if P_pred.shape[ax] == 1:
            uf_new.append(np.zeros_like(P_pred))
            continue
        dP = (P_pred - np.roll(P_pred, 1, axis=ax)) / h[a]
        u = uf_star[a] - dt * dP * 2.0 / (rho_new + np.roll(rho_new, 1, axis=ax))
        if bc[a] == NEUMANN:
            u[_wall_first(u, ax)] = 0.0
        uf_new.append(u)
    u_cell = [mc / rho_new for mc in m_new]
    e_new = e_star - dt * (P_pred * divergence(uf_new, h, bc) + sum(u_cell[a] * gp[a] for a in range(3)))
    return m_new, uf_new, e_new
