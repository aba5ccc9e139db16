"""The dissipative fourth-order second-derivative stencil, in float64.

Sec. 4 of the paper (Eqs. fv-approach, fv-approach2, dissipativestencil4)
derives the viscous second derivative from the finite-volume picture: the
derivative at a face from a centred 4-point polynomial of the cell averages,

    p_{i+1/2} = (U_{i-1} - 15 U_i + 15 U_{i+1} - U_{i+2}) / (12 h),

and the second derivative as the difference of the two face values,

    (U_xx)_i = (p_{i+1/2} - p_{i-1/2}) / h
             = (-U_{i-2} + 16 U_{i-1} - 30 U_i + 16 U_{i+1} - U_{i+2}) / (12 h^2).

In several dimensions the operator is the sum over axes (directional
splitting, Sec. 4).  Boundaries (the paper gives none for this stencil;
reading): a periodic axis wraps; on a Neumann (wall) axis the face at the
wall carries no flux and the face values next to it take mirror ghosts
U_{-1-k} = U_k, so the scheme stays conservative.  Arrays are numpy
(nz, ny, nx), x fastest, as in poisson.py.

Also here, for the dissipativity comparison of Sec. 4: the earlier
nine-point fourth-order stencil (Eq. nondissipativestencil), whose Fourier
symbol vanishes at the highest grid frequency.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .poisson import NEUMANN, PERIODIC, _np_axis


def _shift(u: np.ndarray, k: int, ax: int, bc: int) -> np.ndarray:
    """u shifted so that entry i holds U_{i+k} along axis ax: wrapped on a
    periodic axis, mirrored about the walls on a Neumann axis."""
    n = u.shape[ax]
    idx = np.arange(n) + k
    if bc == PERIODIC:
        idx = idx % n
    else:
        idx = np.where(idx < 0, -1 - idx, idx)
        idx = np.where(idx >= n, 2 * n - 1 - idx, idx)
    return np.take(u, idx, axis=ax)


def face_derivative(u: np.ndarray, h: float, ax: int, bc: int) -> np.ndarray:
    """p_{i+1/2} for every i along numpy axis ax (Eq. fv-approach2); on a
    Neumann axis the last face (the wall) is set to 0."""
    p = (_shift(u, -1, ax, bc) - 15.0 * u + 15.0 * _shift(u, 1, ax, bc) - _shift(u, 2, ax, bc)) / (12.0 * h)
    if bc == NEUMANN:
        sl = [slice(None)] * u.ndim
        sl[ax] = -1
        p[tuple(sl)] = 0.0
    return p


def second_derivative(u: np.ndarray, h: float, ax: int, bc: int) -> np.ndarray:
    """(U_xx)_i = (p_{i+1/2} - p_{i-1/2}) / h along numpy axis ax; the wall
    face below the first cell of a Neumann axis carries no flux."""
    p = face_derivative(u, h, ax, bc)
    pm = np.roll(p, 1, axis=ax)
    if bc == NEUMANN:
        sl = [slice(None)] * u.ndim
        sl[ax] = 0
        pm[tuple(sl)] = 0.0
    return (p - pm) / h


def laplacian4(u: np.ndarray, h, bc) -> np.ndarray:
    """Sum over the grid axes with more than one cell of the fourth-order
    dissipative second derivative; h, bc per grid axis (x, y, z)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    for a in range(3):
        ax = _np_axis(a)
        if u.shape[ax] > 1:
            out = out + second_derivative(u, float(h[a]), ax, int(bc[a]))
    return out


def explicit_diffusion_step(u: np.ndarray, nu: float, dt: float, h, bc) -> np.ndarray:
    """One forward-Euler step of u_t = nu (sum of u_xx): u + dt nu lap4(u)."""
    return np.asarray(u, dtype=np.float64) + dt * nu * laplacian4(u, h, bc)


def symbol_dissipative(theta) -> np.ndarray:
    """h^2 times the Fourier symbol of the five-point stencil:
    (32 cos t - 2 cos 2t - 30) / 12."""
    t = np.asarray(theta, dtype=np.float64)
    return (32.0 * np.cos(t) - 2.0 * np.cos(2.0 * t) - 30.0) / 12.0


def nondissipative_1d(u: np.ndarray, h: float) -> np.ndarray:
    """The nine-point stencil of Eq. nondissipativestencil on a periodic 1D
    array, read as (U_{i+4} - 18 U_{i+3} + 80 U_{i+2} + 18 U_{i+1} - 162 U_i
    + 18 U_{i-1} + 80 U_{i-2} - 18 U_{i-3} + U_{i-4}) / (192 h^2).  The text
    prints the U_{i+4} term with a minus sign, which leaves the weights
    summing to -2 (a constant would not be annihilated); the symmetric
    reading sums to zero, has second moment 2 * 192 and a symbol that
    vanishes at the grid frequency, the lack of dissipativity the section
    describes."""
    c = {4: 1.0, 3: -18.0, 2: 80.0, 1: 18.0, 0: -162.0, -1: 18.0, -2: 80.0, -3: -18.0, -4: 1.0}
    return sum(w * np.roll(u, -k) for k, w in c.items()) / (192.0 * h * h)
