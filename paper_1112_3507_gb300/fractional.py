"""Time stepping with the fractional-step method on one GPU (Sec. 2.4).

Host-side sequencing only: every step on grid data is one call of the C ABI
(liblowmach.so) on device tensors, in the order of the paper's algorithm:

  (i)-(iii)  lm_advect             rho^{n+1}, (rho u)*, e* (explicit, inviscid)
  (iv)-(v)   lm_projection_rhs     f of Eq. fpoiss and the face velocities u*
             lm_set_coefficients   c~ from rho^n, c_s^2, dt; kappa from rho^{n+1}
  (vi)       lm_solve              the generalized Poisson solve, warm-started
                                   from P^n (the pressure changes little per step)
  (vii)-(viii) lm_projection_update momentum, face velocities, energy
  (ix)       lm_eos_ideal          P^{n+1} and c_s^2 from the ideal-gas law

The state (rho, rho u, e, P, c_s^2) stays resident on the device between
steps; one step costs one host synchronisation (the solve's convergence
test).
"""
from __future__ import annotations

import numpy as np

from . import lowmach as lm


class FractionalStep:
    """Steps (i)-(ix) of Sec. 2.4 on an (nx, ny, nz) grid of cells."""

    def __init__(self, n, h, bc, gamma: float, mode: str = "mixed", rtol: float = 1e-11, device="cuda"):
        import torch
        self.torch = torch
        self.n, self.h, self.bc = tuple(int(v) for v in n), tuple(float(v) for v in h), tuple(int(b) for b in bc)
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.gamma, self.mode, self.rtol = float(gamma), mode, float(rtol)
        self.grid = lm.Grid(self.n, self.h, self.bc)

        def z(k=1):
            return torch.zeros(k * self.N, dtype=torch.float64, device=device)

        self.rho, self.mom, self.e, self.p, self.cs2 = z(), z(3), z(), z(), z()
        self.rho1, self.mom_s, self.e_s = z(), z(3), z()
        self.f, self.uf_s, self.uf1, self.p_pred = z(), z(3), z(3), z()
        self.mom1, self.e1 = z(3), z()
        self.last = None

    def close(self):
        if self.grid is not None:
            self.grid.close()
            self.grid = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, rho, mom, e, stream=None):
        """rho, e: N values; mom: three arrays or one of 3N (host or device);
        P and c_s^2 follow from the equation of state (step (ix))."""
        torch = self.torch
        self.rho.copy_(torch.as_tensor(np.asarray(rho).ravel() if not torch.is_tensor(rho) else rho.ravel()))
        m = mom if torch.is_tensor(mom) else torch.as_tensor(np.concatenate([np.asarray(a).ravel() for a in mom]))
        self.mom.copy_(m.ravel())
        self.e.copy_(torch.as_tensor(np.asarray(e).ravel() if not torch.is_tensor(e) else e.ravel()))
        lm.eos_ideal(self.gamma, self.rho, self.mom, self.e, self.p, self.cs2, stream=stream)

    def step(self, dt: float, stream=None) -> dict:
        """One fractional step; returns the solve's result."""
        g = self.grid
        lm.advect(self.n, self.h, self.bc, dt, self.rho, self.mom, self.e, self.rho1, self.mom_s, self.e_s,
                  stream=stream)
        lm.projection_rhs(self.n, self.h, self.bc, dt, self.p, self.rho, self.cs2, self.mom, self.mom_s, self.rho1,
                          self.f, self.uf_s, stream=stream)
        g.set_coefficients(self.rho, self.rho1, self.cs2, dt, stream)
        g.set_rhs(self.f, stream)
        g.set_initial_guess(self.p, stream)
        res = g.solve(mode=self.mode, rtol=self.rtol, stream=stream, use_x0=1)
        g.solution(self.p_pred, stream)
        lm.projection_update(self.n, self.h, self.bc, dt, self.p_pred, self.rho1, self.mom_s, self.uf_s, self.e_s,
                             self.mom1, self.uf1, self.e1, stream=stream)
        lm.eos_ideal(self.gamma, self.rho1, self.mom1, self.e1, self.p, self.cs2, stream=stream)
        # the new state becomes the current one (buffers swap, nothing is copied)
        self.rho, self.rho1 = self.rho1, self.rho
        self.mom, self.mom1 = self.mom1, self.mom
        self.e, self.e1 = self.e1, self.e
        self.last = res
        return res

    def state(self):
        """(rho, [m_x, m_y, m_z], e, P) as numpy arrays in (nz, ny, nx) layout."""
        shape = (self.n[2], self.n[1], self.n[0])
        m = self.mom.cpu().numpy().reshape(3, *shape)
        return (self.rho.cpu().numpy().reshape(shape), [m[0], m[1], m[2]], self.e.cpu().numpy().reshape(shape),
                self.p.cpu().numpy().reshape(shape))
