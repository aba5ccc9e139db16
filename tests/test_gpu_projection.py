"""The steps either side of the solve on the GPU (lm_projection_rhs /
lm_projection_update, Sec. 2 steps (iv)-(viii)) against oracle.projection,
and one whole fractional-step projection through the library: right-hand
side, solve, update -- whose face velocities then satisfy the discrete
pressure-evolution identity (needs a GB300)."""
import os

import numpy as np
import pytest

from oracle import projection as J
from oracle.poisson import NEUMANN, PERIODIC

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_3507_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()
    from paper_1112_3507_gb300 import lowmach
    return lowmach


def _state(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = (np.arange(nz) + 0.5) / nz
    rho_o = (1.0 - 0.8 * z)[:, None, None] * (1.0 + 0.05 * rng.uniform(-1, 1, shape))
    rho_n = rho_o * (1.0 + 0.02 * rng.uniform(-1, 1, shape))
    p_o = (1.0 - 0.8 * z)[:, None, None] ** 1.6 * (1.0 + 0.01 * rng.uniform(-1, 1, shape))
    cs2 = 5.0 / 3.0 * p_o / rho_o
    m_o = [0.1 * rng.standard_normal(shape) * rho_o for _ in range(3)]
    m_s = [mc + 0.01 * rng.standard_normal(shape) for mc in m_o]
    e_s = rng.uniform(1.0, 2.0, shape)
    S = 0.05 * rng.standard_normal(shape)
    return rho_o, rho_n, p_o, cs2, m_o, m_s, e_s, S


def _d(a):
    return torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


def _v(comps):
    return _d(np.concatenate([c.ravel() for c in comps]))


CASES = [((10, 6, 12), (PERIODIC, PERIODIC, NEUMANN)), ((16, 1, 24), (PERIODIC, PERIODIC, NEUMANN)),
         ((6, 8, 5), (NEUMANN, NEUMANN, NEUMANN)), ((4, 4, 8), (PERIODIC, PERIODIC, PERIODIC))]


@pytest.mark.parametrize("shape,bc", CASES)
def test_projection_kernels_match_oracle(lm, shape, bc):
    nz, ny, nx = shape
    n = (nx, ny, nz)
    h = (1.0 / nz, 0.7 / nz, 1.0 / nz)
    rho_o, rho_n, p_o, cs2, m_o, m_s, e_s, S = _state(shape, seed=sum(shape))
    if ny == 1:
        m_o[1][:] = 0.0
        m_s[1][:] = 0.0
    dt = 1e-3
    N = nx * ny * nz
    f = torch.empty(N, dtype=torch.float64, device="cuda")
    uf = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    lm.projection_rhs(n, h, bc, dt, _d(p_o), _d(rho_o), _d(cs2), _v(m_o), _v(m_s), _d(rho_n), f, uf, source=_d(S))
    f_ref, uf_ref = J.rhs(p_o, rho_o, cs2, m_o, m_s, rho_n, dt, h, bc, S)
    np.testing.assert_allclose(f.cpu().numpy(), f_ref.ravel(), rtol=1e-12, atol=1e-12 * np.abs(f_ref).max())
    np.testing.assert_allclose(uf.cpu().numpy(), np.concatenate([u.ravel() for u in uf_ref]), rtol=1e-12,
                               atol=1e-14)
    Pp = p_o * (1.0 + 0.01 * np.random.default_rng(3).standard_normal(shape))
    m_new, uf_new, e_new = (torch.empty(3 * N, dtype=torch.float64, device="cuda"),
                            torch.empty(3 * N, dtype=torch.float64, device="cuda"),
                            torch.empty(N, dtype=torch.float64, device="cuda"))
    lm.projection_update(n, h, bc, dt, _d(Pp), _d(rho_n), _v(m_s), uf, _d(e_s), m_new, uf_new, e_new)
    mr, ufr, er = J.update(Pp, rho_n, m_s, uf_ref, e_s, dt, h, bc)
    np.testing.assert_allclose(m_new.cpu().numpy(), np.concatenate([m.ravel() for m in mr]), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(uf_new.cpu().numpy(), np.concatenate([u.ravel() for u in ufr]), rtol=1e-12,
                               atol=1e-13)
    np.testing.assert_allclose(e_new.cpu().numpy(), er.ravel(), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("shape,bc", [((32, 16, 32), (PERIODIC, PERIODIC, NEUMANN)),
                                      ((64, 1, 64), (PERIODIC, PERIODIC, NEUMANN))])
def test_fractional_step_projection_on_gpu(lm, shape, bc):
    """rhs -> lm_set_coefficients / lm_set_rhs -> lm_solve (mixed, to 1e-12)
    -> update, all on the GPU: div u^{n+1} equals the discrete pressure
    evolution (P^n - dt u^n.grad P^n - P) / (dt rho^n c^2) - dt S to the
    solve's tolerance."""
    nz, ny, nx = shape
    n = (nx, ny, nz)
    h = (1.0 / nz,) * 3
    rho_o, rho_n, p_o, cs2, m_o, m_s, e_s, S = _state(shape, seed=7)
    if ny == 1:
        m_o[1][:] = 0.0
        m_s[1][:] = 0.0
    dt = 0.5 * h[2] / (0.01 * np.sqrt(cs2.max()))
    N = nx * ny * nz
    f = torch.empty(N, dtype=torch.float64, device="cuda")
    uf = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    dS = _d(S)
    lm.projection_rhs(n, h, bc, dt, _d(p_o), _d(rho_o), _d(cs2), _v(m_o), _v(m_s), _d(rho_n), f, uf, source=dS)
    with lm.Grid(n, h, bc) as g:
        g.set_coefficients(_d(rho_o), _d(rho_n), _d(cs2), dt)
        g.set_rhs(f)
        r = g.solve(mode="mixed", rtol=1e-12, max_outer=20)
        assert r["status"] == 0
        Pp = torch.empty(N, dtype=torch.float64, device="cuda")
        g.solution(Pp)
    m_new, uf_new, e_new = (torch.empty(3 * N, dtype=torch.float64, device="cuda"),
                            torch.empty(3 * N, dtype=torch.float64, device="cuda"),
                            torch.empty(N, dtype=torch.float64, device="cuda"))
    lm.projection_update(n, h, bc, dt, Pp, _d(rho_n), _v(m_s), uf, _d(e_s), m_new, uf_new, e_new)
    P_h = Pp.cpu().numpy().reshape(shape)
    ufn = [a.reshape(shape) for a in np.split(uf_new.cpu().numpy(), 3)]
    div = J.divergence(ufn, h, bc)
    u_o = [mc / rho_o for mc in m_o]
    gp = J.grad_p(p_o, rho_o, h, bc)
    want = (p_o - dt * sum(u_o[a] * gp[a] for a in range(3)) - P_h) / (dt * rho_o * cs2) - dt * S
    ufs = [a.reshape(shape) for a in np.split(uf.cpu().numpy(), 3)]
    scale = np.abs(J.divergence(ufs, h, bc)).max()
    assert np.max(np.abs(div - want)) <= 1e-7 * scale
