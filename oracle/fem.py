"""The generalized Poisson operator in a Q1 finite-element discretization, in
float64.

The paper discretizes Eq. GeneralizedPoisson with finite elements because
they give a symmetric positive-definite system (Sec. 2.5; the element
details are in a reference the text does not reproduce).  Reading (the
variant of the operator next to the cell-centred finite volumes of
poisson.py): multilinear (Q1) elements on the grid of points

    x_i = i h  (i = 0 .. n-1 on every axis),

the same array layout as the cell grid, x fastest.  A periodic axis closes
into a ring of n elements; a wall axis (Neumann) has n - 1 elements and its
end points lie on the walls, where the homogeneous Neumann condition is the
natural one of the weak form.  An axis with one point carries no elements
(a 2D grid).  Per element e:

    kappa_e = (number of corners) / sum over corners of rho,
              the harmonic mean of kappa = 1/rho over its corners;
    K_e     = kappa_e * sum over axes a of (S_a x prod_{b != a} M_b),
              S = [[1, -1], [-1, 1]] / h and M = [[2, 1], [1, 2]] h / 6 the
              1D element stiffness and mass (tensor products);

and the c~ term is mass-lumped: V_i c~_i with V_i = prod over axes of the
point's share of its elements (h, or h/2 at a wall end).  The system is

    B x = V f,   B = diag(V c~) + sum_e K_e,

symmetric positive definite for rho > 0, c~ > 0 (Sec. 2.5, the Lax-Milgram
conditions).  Inhomogeneous Neumann data g enter as b_i += g_i times the
boundary measure of point i (the caller's).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse

from .poisson import NEUMANN, PERIODIC, _np_axis

S1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0


class FEOperator:
    """B = diag(V c~) + sum_e K_e on a grid of points (nz, ny, nx)."""

    def __init__(self, ct, rho, h, bc):
        ct = np.asarray(ct, dtype=np.float64)
        rho = np.asarray(rho, dtype=np.float64)
        if ct.ndim == 2:
            ct, rho = ct[:, None, :], rho[:, None, :]
        self.ct, self.rho = ct, rho
        self.h = tuple(float(v) for v in h)
        self.bc = tuple(int(b) for b in bc)
        self.shape = ct.shape
        n = (self.shape[2], self.shape[1], self.shape[0])
        self.axes = [a for a in range(3) if n[a] > 1]             # axes carrying elements
        # each point's share of its elements (lumped mass)
        V = np.ones(self.shape)
        for a in self.axes:
            ax = _np_axis(a)
            w = np.full(n[a], self.h[a])
            if self.bc[a] == NEUMANN:
                w[0] = w[-1] = 0.5 * self.h[a]
            shp = [1, 1, 1]
            shp[ax] = n[a]
            V = V * w.reshape(shp)
        self.volume = V
        # elements: indexed by their lowest corner; on a wall axis the last point starts none
        mask = np.ones(self.shape, dtype=bool)
        for a in self.axes:
            if self.bc[a] == NEUMANN:
                idx = [slice(None)] * 3
                idx[_np_axis(a)] = -1
                mask[tuple(idx)] = False
        self.mask = mask
        self.corners = list(itertools.product((0, 1), repeat=len(self.axes)))
        rsum = sum(self._corner(rho, c) for c in self.corners)
        self.kappa_e = np.where(mask, len(self.corners) / rsum, 0.0)
        self.kref = np.zeros((len(self.corners), len(self.corners)))
        for p, cp in enumerate(self.corners):
            for q, cq in enumerate(self.corners):
                v = 0.0
                for ia, a in enumerate(self.axes):
                    t = S1[cp[ia], cq[ia]] / self.h[a]
                    for ib, b in enumerate(self.axes):
                        if ib != ia:
                            t *= M1[cp[ib], cq[ib]] * self.h[b]
                    v += t
                self.kref[p, q] = v

    def _corner(self, u: np.ndarray, c) -> np.ndarray:
        """u at corner c of every element (element index = its lowest corner)."""
        for ia, a in enumerate(self.axes):
            if c[ia]:
                u = np.roll(u, -1, axis=_np_axis(a))
        return u

    def _back(self, y: np.ndarray, c) -> np.ndarray:
        """Element values moved to the point that is corner c of the element."""
        for ia, a in enumerate(self.axes):
            if c[ia]:
                y = np.roll(y, 1, axis=_np_axis(a))
        return y

    @property
    def size(self) -> int:
        return int(np.prod(self.shape))

    def apply(self, x: np.ndarray) -> np.ndarray:
        """B x: lumped c~ term plus each element's K_e times its corner values."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        y = self.volume * self.ct * x
        xc = [self._corner(x, c) for c in self.corners]
        for p, cp in enumerate(self.corners):
            ye = self.kappa_e * sum(self.kref[p, q] * xc[q] for q in range(len(self.corners)))
            y = y + self._back(ye, cp)
        return y

    def assemble(self) -> scipy.sparse.csr_matrix:
        """B as a sparse matrix, element by element."""
        N = self.size
        idx = np.arange(N).reshape(self.shape)
        rows, cols, vals = [idx.ravel()], [idx.ravel()], [(self.volume * self.ct).ravel()]
        ci = [self._corner(idx, c) for c in self.corners]
        m = self.mask.ravel()
        ke = self.kappa_e.ravel()
        for p in range(len(self.corners)):
            for q in range(len(self.corners)):
                rows.append(ci[p].ravel()[m])
                cols.append(ci[q].ravel()[m])
                vals.append((ke * self.kref[p, q])[m])
        return scipy.sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                       shape=(N, N)).tocsr()

    def diagonal(self) -> np.ndarray:
        return self.assemble().diagonal().reshape(self.shape)


def fe_from_state(rho_old, rho_new, cs2, dt, h, bc) -> FEOperator:
    """c~ from rho^n, c_s^2, dt (Eq. cpoiss); element kappa from rho^{n+1} (Eq. kappapoiss)."""
    return FEOperator(1.0 / ((dt * dt) * rho_old * cs2), rho_new, h, bc)


def solve(op: FEOperator, b: np.ndarray) -> np.ndarray:
    """Sparse direct solve of B x = b."""
    import scipy.sparse.linalg
    x = scipy.sparse.linalg.spsolve(op.assemble().tocsc(), np.asarray(b, dtype=np.float64).ravel())
    return np.asarray(x).reshape(op.shape)


def symbol(theta, h, kappa0: float, c0: float) -> float:
    """B v = V lambda v for the periodic mode of angles theta (per axis with
    elements; constant kappa0, c0): lambda = c0 + kappa0 sum_a
    2 (1 - cos t_a) / h_a^2 prod_{b != a} (2 + cos t_b) / 3."""
    lam = c0
    for ia, t in enumerate(theta):
        term = 2.0 * (1.0 - np.cos(t)) / h[ia] ** 2
        for ib, u in enumerate(theta):
            if ib != ia:
                term *= (2.0 + np.cos(u)) / 3.0
        lam += kappa0 * term
    return lam
