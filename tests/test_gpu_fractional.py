"""The fractional step on the GPU (Sec. 2.4 steps (i)-(ix)) against
oracle.fractional: the advection kernel element by element (2D and 3D,
periodic and wall axes, with the two-component rho c), the equation of
state, one whole step of the Gresho vortex (Sec. 5.5.2), and fifty steps'
kinetic energy (needs a GB300)."""
import os

import numpy as np
import pytest

from oracle import fractional as FR
from oracle.poisson import NEUMANN, PERIODIC
from paper_1112_3507_gb300 import inputs as I

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


def _d(a):
    return torch.as_tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("shape,bc", [((16, 1, 24), (PERIODIC, PERIODIC, PERIODIC)),
                                      ((16, 1, 24), (NEUMANN, PERIODIC, NEUMANN)),
                                      ((6, 5, 9), (PERIODIC, PERIODIC, NEUMANN)),
                                      ((4, 3, 2), (NEUMANN, NEUMANN, PERIODIC))])
@pytest.mark.parametrize("with_c", [False, True])
def test_advect_matches_oracle(lm, shape, bc, with_c):
    rng = np.random.default_rng(sum(shape))
    n = (shape[2], shape[1], shape[0])
    h = (0.1, 0.2, 0.15)
    rho = 1.0 + 0.5 * rng.random(shape)
    mom = [rng.standard_normal(shape) for _ in range(3)]
    e = 4.0 + rng.random(shape)
    rc = rho * rng.random(shape) if with_c else None
    dt = 0.01
    r1, m1, e1, c1 = FR.advect(rho, mom, e, dt, h, bc, rho_c=rc)
    N = rho.size
    rho_d, mom_d, e_d = _d(rho), _d(np.concatenate([m.ravel() for m in mom])), _d(e)
    out = [torch.empty(N, dtype=torch.float64, device="cuda"), torch.empty(3 * N, dtype=torch.float64, device="cuda"),
           torch.empty(N, dtype=torch.float64, device="cuda")]
    rc_d = _d(rc) if with_c else None
    rc1 = torch.empty(N, dtype=torch.float64, device="cuda") if with_c else None
    lm.advect(n, h, bc, dt, rho_d, mom_d, e_d, out[0], out[1], out[2], rho_c=rc_d, rho_c_new=rc1)
    got_m = out[1].cpu().numpy().reshape(3, *shape)
    # rounding scale: dt / h times the flux magnitudes
    for ref, got, q0 in [(r1, out[0].cpu().numpy(), rho), (e1, out[2].cpu().numpy(), e)] + \
            [(m1[a], got_m[a], mom[a]) for a in range(3)] + \
            ([(c1, rc1.cpu().numpy(), rc)] if with_c else []):
        scale = np.abs(q0).max() * (1 + dt * 20.0 / min(h))
        np.testing.assert_allclose(got.reshape(shape), ref, rtol=0, atol=1e-14 * scale)


def test_advect_rejects_overlap(lm):
    n = (8, 1, 8)
    t = torch.ones(8 * 8, dtype=torch.float64, device="cuda")
    m = torch.zeros(3 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(lm.LowMachError):
        lm.advect(n, (0.1, 1.0, 0.1), (PERIODIC,) * 3, 0.01, t, m, t.clone(), t, m.clone(), t.clone())


def test_eos_matches_oracle(lm):
    rng = np.random.default_rng(2)
    shape = (5, 4, 6)
    rho = 1 + rng.random(shape)
    mom = [rng.standard_normal(shape) for _ in range(3)]
    e = 10 + rng.random(shape)
    p_ref, c_ref = FR.eos_ideal(rho, mom, e, 1.4)
    p = torch.empty(rho.size, dtype=torch.float64, device="cuda")
    c = torch.empty_like(p)
    lm.eos_ideal(1.4, _d(rho), _d(np.concatenate([m.ravel() for m in mom])), _d(e), p, c)
    np.testing.assert_allclose(p.cpu().numpy().reshape(shape), p_ref, rtol=1e-14)
    np.testing.assert_allclose(c.cpu().numpy().reshape(shape), c_ref, rtol=1e-14)


@pytest.mark.parametrize("ma", [0.1, 0.01])
def test_one_gresho_step_matches_oracle(lm, ma):
    """One whole step (i)-(ix) on the GPU (mixed solve to 1e-12, warm start
    from P^n) against the oracle's step with a direct solve."""
    from paper_1112_3507_gb300.fractional import FractionalStep
    g = I.gresho_vortex(32, ma)
    ref = FR.step(g["rho"], g["mom"], g["e"], g["P"], g["dt"], g["h"], g["bc"], g["gamma"])
    with FractionalStep(g["n"], g["h"], g["bc"], g["gamma"], rtol=1e-12) as fs:
        fs.set_state(g["rho"], g["mom"], g["e"])
        res = fs.step(g["dt"])
        rho, mom, e, p = fs.state()
    assert res["rel_residual"] <= 1e-12
    np.testing.assert_allclose(rho, ref[0], rtol=1e-13)
    for a in (0, 2):
        np.testing.assert_allclose(mom[a], ref[1][a], rtol=0, atol=1e-9)
    np.testing.assert_allclose(e, ref[2], rtol=1e-12)
    # the pressure: the solve's tolerance times |P| bounds the difference
    np.testing.assert_allclose(p, ref[3], rtol=0, atol=1e-12 * np.abs(ref[3]).max() * 50)


def test_fifty_steps_kinetic_energy(lm):
    """Fifty steps at Ma = 0.01: the GPU's kinetic energy history follows the
    oracle's (1e-9 relative) and decays slowly (the vortex is stationary)."""
    from paper_1112_3507_gb300.fractional import FractionalStep
    g = I.gresho_vortex(32, 0.01)
    rho, mom, e, p = g["rho"], g["mom"], g["e"], g["P"]
    ke0 = FR.kinetic_energy(rho, mom, g["h"])
    ke_ref = []
    for _ in range(50):
        rho, mom, e, p, _ = FR.step(rho, mom, e, p, g["dt"], g["h"], g["bc"], g["gamma"])
        ke_ref.append(FR.kinetic_energy(rho, mom, g["h"]) / ke0)
    ke_gpu = []
    with FractionalStep(g["n"], g["h"], g["bc"], g["gamma"], rtol=1e-12) as fs:
        fs.set_state(g["rho"], g["mom"], g["e"])
        iters = []
        for _ in range(50):
            iters.append(fs.step(g["dt"])["iters"])
            r, m, _, _ = fs.state()
            ke_gpu.append(FR.kinetic_energy(r, m, g["h"]) / ke0)
    np.testing.assert_allclose(ke_gpu, ke_ref, rtol=1e-9)
    assert 0.99 < ke_gpu[-1] < 1.0
    assert max(iters[5:]) <= max(iters[:2])       # warm starts do not need more iterations
