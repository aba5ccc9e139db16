"""The discrete generalized-Poisson operator and reference solves, in float64.

Continuous problem (Sec. 2, Eq. Poiss; Sec. 2.5, Eq. GeneralizedPoisson):

    c~ P - div(kappa grad P) = f,   c~ = 1/(dt^2 rho^n c_s^2)   (Eq. cpoiss)
                                    kappa = 1/rho^{n+1}          (Eq. kappapoiss)

with homogeneous Neumann walls dP/dn = 0 (Eq. vonNeumannBC) and, as in the
paper's simulations (Sec. 3.2) and its solver test (Sec. 2.5.2), optionally
periodic axes.

Discretization (the paper's own is a finite-element scheme whose details are
not given in the text; this is the cell-centred finite-volume reading, which
is symmetric positive definite like the paper's):

    (A x)_i = c~_i x_i + sum over faces f of cell i of  g_f (x_i - x_nb(f)),
    g_f = kappa_f / h_axis^2,   kappa_f = 2 / (rho_L + rho_R),

where kappa_f is the harmonic mean of kappa = 1/rho on the two cells sharing
the face -- the same factor 2/(rho_{i+1} + rho_i) the face-velocity update of
the fractional-step algorithm, step (viii), uses.  A wall face carries no
flux; a periodic axis wraps.  Arrays are numpy shape (nz, ny, nx), x fastest.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

PERIODIC = 0
NEUMANN = 1


def ctilde(rho_old: np.ndarray, cs2: np.ndarray, dt: float) -> np.ndarray:
    """c~ = 1 / (dt^2 rho^n c_s^2), Eq. cpoiss, evaluated as 1/(((dt*dt)*rho)*cs2)."""
    return 1.0 / ((dt * dt) * rho_old * cs2)


def face_kappa(rho_a: np.ndarray, rho_b: np.ndarray) -> np.ndarray:
    """kappa on the face between two cells: 2/(rho_a + rho_b), the harmonic
    mean of kappa = 1/rho (Eq. kappapoiss; factor of step (viii))."""
    return 2.0 / (rho_a + rho_b)


def _np_axis(a: int) -> int:
    """numpy axis of grid axis a (0 = x, 1 = y, 2 = z) in a (nz, ny, nx) array."""
    return 2 - a


def _first(arr: np.ndarray, ax: int):
    idx = [slice(None)] * arr.ndim
    idx[ax] = 0
    return tuple(idx)


class Operator:
    """A = diag(c~) + sum_faces g_f (e_L - e_R)(e_L - e_R)^T on one grid.

    g_minus[a] holds, for every cell, the conductance g = kappa_f / h_a^2 of
    the face it shares with its minus-neighbour along axis a (0 on a wall
    face, and 0 when the axis has a single cell, whose periodic face would
    join the cell to itself)."""

    def __init__(self, ct: np.ndarray, rho: np.ndarray, h, bc):
        ct = np.asarray(ct, dtype=np.float64)
        rho = np.asarray(rho, dtype=np.float64)
        if ct.ndim == 2:
            ct = ct[:, None, :]
            rho = rho[:, None, :]
        self.ct = ct
        self.h = tuple(float(v) for v in h)
        self.bc = tuple(int(b) for b in bc)
        self.shape = ct.shape
        self.g_minus = []
        for a in range(3):
            ax = _np_axis(a)
            n = ct.shape[ax]
            rho_minus = np.roll(rho, 1, axis=ax)          # rho of cell i-1 (wraps)
            g = face_kappa(rho, rho_minus) / (self.h[a] * self.h[a])
            if n == 1:
                g = np.zeros_like(g)
            elif self.bc[a] == NEUMANN:
                g[_first(g, ax)] = 0.0                     # wall at the low end
            self.g_minus.append(g)

    @property
    def size(self) -> int:
        return int(np.prod(self.shape))

    def g_plus(self, a: int) -> np.ndarray:
        """Conductance of each cell's face with its plus-neighbour: the
        minus-face of cell i+1; on a Neumann axis the last cell's plus-face
        is the wall, which the roll maps onto the (zero) wall face of cell 0."""
        return np.roll(self.g_minus[a], -1, axis=_np_axis(a))

    def apply(self, x: np.ndarray) -> np.ndarray:
        """y = A x, cell by cell from the flux definition."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        y = self.ct * x
        for a in range(3):
            ax = _np_axis(a)
            y = y + self.g_minus[a] * (x - np.roll(x, 1, axis=ax))
            y = y + self.g_plus(a) * (x - np.roll(x, -1, axis=ax))
        return y

    def diagonal(self) -> np.ndarray:
        """D_i = c~_i + sum of the conductances of cell i's faces (Jacobi)."""
        d = self.ct.copy()
        for a in range(3):
            d = d + self.g_minus[a] + self.g_plus(a)
        return d

    def assemble(self) -> scipy.sparse.csr_matrix:
        """Sparse matrix built face by face: each face (L, R) with conductance
        g adds g to A[L,L] and A[R,R] and -g to A[L,R] and A[R,L]."""
        N = self.size
        idx = np.arange(N).reshape(self.shape)
        rows = [idx.ravel()]
        cols = [idx.ravel()]
        vals = [self.ct.ravel()]
        for a in range(3):
            ax = _np_axis(a)
            g = self.g_minus[a].ravel()
            L = np.roll(idx, 1, axis=ax).ravel()      # minus-neighbour
            R = idx.ravel()
            keep = g != 0.0
            L, R, g = L[keep], R[keep], g[keep]
            rows += [L, R, L, R]
            cols += [L, R, R, L]
            vals += [g, g, -g, -g]
        A = scipy.sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                    shape=(N, N))
        return A.tocsr()


def operator_from_state(rho_old, rho_new, cs2, dt, h, bc) -> Operator:
    """Coefficient assembly (step (v)): c~ from rho^n, c_s^2, dt; faces from rho^{n+1}."""
    return Operator(ctilde(rho_old, cs2, dt), rho_new, h, bc)


def operator_from_problem(p) -> Operator:
    return operator_from_state(p.rho_old, p.rho_new, p.cs2, p.dt, p.h, p.bc)


def rel_residual(op: Operator, x: np.ndarray, f: np.ndarray) -> float:
    """||f - A x||_2 / ||f||_2, unweighted over cells."""
    f = np.asarray(f, dtype=np.float64).reshape(op.shape)
    r = f - op.apply(x)
    return float(np.linalg.norm(r) / np.linalg.norm(f))


def solve_cholesky(op: Operator, f: np.ndarray) -> np.ndarray:
    """Dense Cholesky solve (small grids).  Raises numpy.linalg.LinAlgError
    if A is not positive definite."""
    A = op.assemble().toarray()
    L = np.linalg.cholesky(A)
    y = scipy.linalg.solve_triangular(L, np.asarray(f, dtype=np.float64).ravel(), lower=True)
    x = scipy.linalg.solve_triangular(L.T, y, lower=False)
    return x.reshape(op.shape)


def solve_direct(op: Operator, f: np.ndarray) -> np.ndarray:
    """Sparse LU solve (SuperLU) of A x = f."""
    A = op.assemble().tocsc()
    x = scipy.sparse.linalg.spsolve(A, np.asarray(f, dtype=np.float64).ravel())
    return np.asarray(x).reshape(op.shape)


def solve_pcg_jacobi(op: Operator, f: np.ndarray, rtol: float = 1e-14, maxiter: int = 100000,
                     x0: np.ndarray | None = None, max_seconds: float | None = None):
    """Preconditioned conjugate gradients (the paper's solver family, Sec. 2.5)
    with the Jacobi preconditioner diag(A) in place of incomplete Cholesky.

    Stops when the recursive residual reaches rtol * ||f||, confirms with the
    true residual, and returns (x, iterations, history of relative residuals).
    `max_seconds` bounds the run (for timing samples): it then returns early."""
    import time
    t0 = time.perf_counter()
    f = np.asarray(f, dtype=np.float64).reshape(op.shape)
    x = np.zeros(op.shape) if x0 is None else np.array(x0, dtype=np.float64).reshape(op.shape)
    dinv = 1.0 / op.diagonal()
    fnorm = float(np.linalg.norm(f))
    if fnorm == 0.0:
        return np.zeros(op.shape), 0, [0.0]
    r = f - op.apply(x)
    z = dinv * r
    p = z.copy()
    rz = float(np.vdot(r, z))
    hist = [float(np.linalg.norm(r)) / fnorm]
    it = 0
    while it < maxiter and hist[-1] > rtol:
        q = op.apply(p)
        alpha = rz / float(np.vdot(p, q))
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(float(np.linalg.norm(r)) / fnorm)
        if hist[-1] <= rtol:
            r = f - op.apply(x)                     # confirm with the true residual
            hist[-1] = float(np.linalg.norm(r)) / fnorm
            if hist[-1] <= rtol:
                break
        if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
            break
        z = dinv * r
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def fourier_mode(shape, h, bc, modes, kappa0: float, c0: float):
    """Discrete eigenpair of A for constant kappa0 (rho = 1/kappa0) and c~ = c0.

    Per axis of n cells: periodic -> cos(2 pi k j / n) with eigenvalue
    (4 kappa0/h^2) sin^2(pi k / n); Neumann -> cos(pi m (j + 1/2)/n) with
    eigenvalue (4 kappa0/h^2) sin^2(pi m/(2n)).
    The eigenvector is the tensor product; its eigenvalue is c0 + the sum over axes.
    Returns (v, lambda).  `modes` = (kx, ky, kz)."""
    nz, ny, nx = shape
    ns = (nx, ny, nz)
    v = np.ones(shape)
    lam = c0
    for a in range(3):
        n = ns[a]
        k = modes[a]
        j = np.arange(n, dtype=np.float64)
        if n == 1:
            vec = np.ones(1)
            la = 0.0
        elif bc[a] == PERIODIC:
            vec = np.cos(2.0 * np.pi * k * j / n)
            la = 4.0 * kappa0 / h[a] ** 2 * np.sin(np.pi * k / n) ** 2
        else:
            vec = np.cos(np.pi * k * (j + 0.5) / n)
            la = 4.0 * kappa0 / h[a] ** 2 * np.sin(np.pi * k / (2.0 * n)) ** 2
        shp = [1, 1, 1]
        shp[_np_axis(a)] = n
        v = v * vec.reshape(shp)
        lam += la
    return v, lam


def solve_fft_periodic(c0: float, kappa0: float, h, f: np.ndarray) -> np.ndarray:
    """Direct solve of the constant-coefficient operator on an all-periodic box
    by diagonalisation with the discrete Fourier transform."""
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    lam = np.full(f.shape, c0)
    for n, hh, ax in ((nx, h[0], 2), (ny, h[1], 1), (nz, h[2], 0)):
        k = np.arange(n)
        la = 4.0 * kappa0 / hh ** 2 * np.sin(np.pi * k / n) ** 2
        shp = [1, 1, 1]
        shp[ax] = n
        lam = lam + la.reshape(shp)
    return np.real(np.fft.ifftn(np.fft.fftn(f) / lam))
