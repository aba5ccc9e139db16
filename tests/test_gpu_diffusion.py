"""The dissipative fourth-order stencil kernel (lm_diffusion4, Sec. 4)
against oracle.diffusion, float64 and float32, periodic and wall axes,
2D and 3D, through the C ABI (needs a GB300)."""
import os

import numpy as np
import pytest

from oracle import diffusion as D
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


CASES = [((37, 1, 50), (0.02, 1.0, 0.02), (PERIODIC, PERIODIC, NEUMANN)),
         ((64, 1, 64), (1 / 64, 1.0, 1 / 64), (NEUMANN, PERIODIC, NEUMANN)),
         ((40, 24, 33), (0.1, 0.2, 0.15), (PERIODIC, PERIODIC, NEUMANN)),
         ((16, 8, 12), (0.3, 0.3, 0.3), (NEUMANN, NEUMANN, NEUMANN)),
         ((256, 16, 8), (1 / 256, 1 / 256, 1 / 256), (PERIODIC, PERIODIC, PERIODIC)),
         ((3, 2, 5), (1.0, 0.5, 0.25), (NEUMANN, PERIODIC, NEUMANN))]


@pytest.mark.parametrize("n,h,bc", CASES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_diffusion4_matches_oracle(lm, n, h, bc, dtype):
    rng = np.random.default_rng(sum(n))
    u = rng.standard_normal((n[2], n[1], n[0]))
    if dtype == torch.float32:
        u = u.astype(np.float32).astype(np.float64)
    alpha, beta = 0.37, 0.8
    ref = beta * u + alpha * D.laplacian4(u, h, bc)
    # the scale of the rounding error: alpha * sum over axes of (|16 (u_{-1} + u_{+1})| + ...) / (12 h^2)
    mag = beta * np.abs(u) + alpha * sum(
        64.0 * np.abs(u).max() / (12 * h[a] ** 2) for a in range(3) if n[a] > 1)
    ud = torch.as_tensor(u.ravel(), dtype=dtype, device="cuda")
    out = torch.empty_like(ud)
    lm.diffusion4(ud, out, n, h, bc, alpha=alpha, beta=beta)
    got = out.cpu().numpy().astype(np.float64).reshape(u.shape)
    tol = 1e-14 if dtype == torch.float64 else 2e-6
    assert np.all(np.abs(got - ref) <= tol * mag)


def test_diffusion4_explicit_steps_decay_and_conserve(lm):
    """Twenty explicit steps at nu dt / h^2 = 0.12 (inside 3/(8 d) = 0.125 in
    3D) on a wall-bounded box: every step agrees with the oracle's step,
    the total stays constant (no flux through the walls), and the grid-scale
    content decays."""
    n, hh = (24, 16, 20), 0.05
    h, bc = (hh, hh, hh), (PERIODIC, PERIODIC, NEUMANN)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((n[2], n[1], n[0]))
    dt = 0.12 * hh * hh
    a = torch.as_tensor(u.ravel(), device="cuda")
    b = torch.empty_like(a)
    ref = u.copy()
    for _ in range(20):
        lm.diffusion4(a, b, n, h, bc, alpha=dt, beta=1.0)
        a, b = b, a
        ref = D.explicit_diffusion_step(ref, 1.0, dt, h, bc)
    got = a.cpu().numpy().reshape(u.shape)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    assert got.sum() == pytest.approx(u.sum(), abs=1e-9)
    assert np.abs(got).max() < np.abs(u).max()


def test_diffusion4_rejects_aliasing_and_bad_sizes(lm):
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    L = lm
    with pytest.raises(L.LowMachError):
        L.diffusion4(t, t, (8, 1, 1), (1, 1, 1), (0, 0, 1))
    with pytest.raises(L.LowMachError):
        L.diffusion4(t, torch.empty_like(t), (8, 1, 1), (0.0, 1, 1), (0, 0, 1))
