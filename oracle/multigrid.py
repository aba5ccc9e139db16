"""Geometric-multigrid V-cycle for the generalized-Poisson operator, in float64.

The paper solves its pressure equation with incomplete-Cholesky PCG
(Sec. 2.5) and says nothing about multigrid; this V-cycle is the
preconditioner the GPU path uses in its place.  It is written here level by
level, with no fusion, so that each GPU kernel can be compared with it:

  hierarchy   an axis is halved while its cell count is even (a periodic axis
              additionally keeps an even count, or one cell, so that the
              red-black colouring stays a 2-colouring); coarsening stops once
              a level has at most COARSE_MAX cells or no axis can be halved.
              Coarse coefficients: c~ and rho are the means over the 2^d'
              children (d' = number of halved axes); faces are then formed
              from the coarse rho exactly as on the finest level, so the
              coarse face kappa is the harmonic mean of the coarse cells'
              kappa = 1/rho.
  restriction mean over the children (R = 2^-d' P^T).
  prolongation piecewise-constant injection of the parent's value (P).
  smoother    red-black Gauss-Seidel, colour (i + j + k) mod 2, red = 0.
              Pre-smoothing sweeps red then black; post-smoothing black then
              red (the adjoint order), so the cycle is symmetric for nu1 = nu2.
  coarsest    exact dense solve when the level has <= COARSE_MAX cells, else
              `coarse_sweeps` pairs of (red-black, black-red) sweeps.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .poisson import NEUMANN, PERIODIC, Operator, _np_axis

COARSE_MAX = 64


def _halvable(n: int, bc: int) -> bool:
    if n < 2 or n % 2:
        return False
    if bc == PERIODIC:
        return (n // 2) % 2 == 0 or n // 2 == 1
    return True


class Level:
    def __init__(self, ct, rho, h, bc):
        self.ct = np.asarray(ct, dtype=np.float64)
        self.rho = np.asarray(rho, dtype=np.float64)
        self.h = tuple(h)
        self.bc = tuple(bc)
        self.op = Operator(self.ct, self.rho, self.h, self.bc)
        self.shape = self.ct.shape
        self.halved = None          # axes halved to reach the next level

    @property
    def size(self):
        return int(np.prod(self.shape))


def _block_mean(a: np.ndarray, halved) -> np.ndarray:
    """Mean over the 2^d' children of each coarse cell."""
    nz, ny, nx = a.shape
    fz, fy, fx = (2 if halved[2] else 1), (2 if halved[1] else 1), (2 if halved[0] else 1)
    b = a.reshape(nz // fz, fz, ny // fy, fy, nx // fx, fx)
    return b.mean(axis=(1, 3, 5))


def _inject(ac: np.ndarray, halved) -> np.ndarray:
    """Piecewise-constant prolongation: every child takes its parent's value."""
    out = ac
    for a in range(3):
        if halved[a]:
            out = np.repeat(out, 2, axis=_np_axis(a))
    return out


def build_hierarchy(ct, rho, h, bc, coarse_max: int = COARSE_MAX):
    """Levels from fine to coarse."""
    ct = np.asarray(ct, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    if ct.ndim == 2:
        ct, rho = ct[:, None, :], rho[:, None, :]
    levels = [Level(ct, rho, h, bc)]
    while levels[-1].size > coarse_max:
        L = levels[-1]
        nz, ny, nx = L.shape
        halved = tuple(_halvable(n, L.bc[a]) for a, n in enumerate((nx, ny, nz)))
        if not any(halved):
            break
        L.halved = halved
        hc = tuple(L.h[a] * (2.0 if halved[a] else 1.0) for a in range(3))
        levels.append(Level(_block_mean(L.ct, halved), _block_mean(L.rho, halved), hc, L.bc))
    return levels


def restrict(r: np.ndarray, halved) -> np.ndarray:
    return _block_mean(r, halved)


def prolong(e: np.ndarray, halved) -> np.ndarray:
    return _inject(e, halved)


def colour(shape) -> np.ndarray:
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (i + j + k) % 2


def gs_colour_update(level: Level, x: np.ndarray, f: np.ndarray, c: int) -> np.ndarray:
    """Gauss-Seidel update of every cell of colour c: the cell's row of
    A x = f solved for x_i with the neighbours' current values,
    x_i = (f_i + sum_f g_f x_nb) / (c~_i + sum_f g_f)."""
    op = level.op
    num = np.array(f, dtype=np.float64)
    for a in range(3):
        ax = _np_axis(a)
        num = num + op.g_minus[a] * np.roll(x, 1, axis=ax) + op.g_plus(a) * np.roll(x, -1, axis=ax)
    new = num / op.diagonal()
    mask = colour(level.shape) == c
    out = x.copy()
    out[mask] = new[mask]
    return out


def sweep(level: Level, x, f, order: str):
    """One red-black sweep: order 'RB' (red then black) or 'BR'."""
    first, second = (0, 1) if order == "RB" else (1, 0)
    x = gs_colour_update(level, x, f, first)
    return gs_colour_update(level, x, f, second)


def coarse_solve(level: Level, f: np.ndarray, coarse_max: int = COARSE_MAX, coarse_sweeps: int = 32):
    if level.size <= coarse_max:
        A = level.op.assemble().toarray()
        return np.linalg.solve(A, f.ravel()).reshape(level.shape)
    x = np.zeros(level.shape)
    for _ in range(coarse_sweeps):
        x = sweep(level, x, f, "RB")
        x = sweep(level, x, f, "BR")
    return x


def vcycle(levels, f: np.ndarray, l: int = 0, nu1: int = 1, nu2: int = 1,
           coarse_max: int = COARSE_MAX, coarse_sweeps: int = 32) -> np.ndarray:
    """One V-cycle from a zero initial guess: returns z ~ A_l^{-1} f."""
    L = levels[l]
    f = np.asarray(f, dtype=np.float64).reshape(L.shape)
    if l == len(levels) - 1:
        return coarse_solve(L, f, coarse_max, coarse_sweeps)
    x = np.zeros(L.shape)
    for _ in range(nu1):
        x = sweep(L, x, f, "RB")
    r = f - L.op.apply(x)
    ec = vcycle(levels, restrict(r, L.halved), l + 1, nu1, nu2, coarse_max, coarse_sweeps)
    x = x + prolong(ec, L.halved)
    for _ in range(nu2):
        x = sweep(L, x, f, "BR")
    return x


def mg_pcg(levels, f, rtol=1e-12, maxiter=500, nu1=1, nu2=1):
    """Conjugate gradients preconditioned by one V-cycle per iteration."""
    op = levels[0].op
    f = np.asarray(f, dtype=np.float64).reshape(op.shape)
    fn = np.linalg.norm(f)
    x = np.zeros(op.shape)
    r = f.copy()
    z = vcycle(levels, r, nu1=nu1, nu2=nu2)
    p = z.copy()
    rz = float(np.vdot(r, z))
    hist = [1.0]
    it = 0
    while it < maxiter and hist[-1] > rtol:
        q = op.apply(p)
        alpha = rz / float(np.vdot(p, q))
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(float(np.linalg.norm(r) / fn))
        z = vcycle(levels, r, nu1=nu1, nu2=nu2)
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist
