"""Host-side input recipe: the seeded generators and the stratifications
(no solver arithmetic; CPU only)."""
import math

import numpy as np

from paper_1112_3507_gb300 import inputs as I


def test_counter_generator_is_reproducible_and_offsettable():
    a = I.splitmix64(12345, 10)
    assert np.array_equal(a, I.splitmix64(12345, 10))
    assert np.array_equal(a[4:], I.splitmix64(12345, 6, offset=4))
    # first output of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    assert int(I.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    u = I.uniform01(7, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3
    z = I.normal(7, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1.0) < 1e-2


def test_smoothed_noise_properties():
    for sigma in (0.0, 2.0):
        f = I.smoothed_noise((16, 1, 32), (I.BC_PERIODIC, I.BC_PERIODIC, I.BC_NEUMANN), 3, sigma=sigma)
        assert abs(f.sum()) < 1e-12 and abs(np.linalg.norm(f) - 1.0) < 1e-12
    white = I.smoothed_noise((64, 1, 64), (0, 0, 1), 4, sigma=0.0)
    smooth = I.smoothed_noise((64, 1, 64), (0, 0, 1), 4, sigma=2.0)
    # smoothing removes roughness: the mean squared x-difference drops
    rough = lambda a: np.mean(np.diff(a[:, 0, :], axis=1) ** 2)
    assert rough(smooth) < 0.1 * rough(white)


def test_polytrope_and_mach_timestep():
    rho, P = I.polytrope(4, 1, 64, contrast=20.0)
    assert 15.0 < rho[0, 0, 0] / rho[-1, 0, 0] < 20.0          # cell centres sit inside the ends
    assert np.allclose(P, rho ** (5.0 / 3.0))                    # polytrope of index 3/2
    p = I.config_convection_3d(16)
    assert p.dt == I.CFL_ADV * p.h[2] / (0.01 * math.sqrt(p.cs2.max()))


def test_semiconvection_profile():
    """Two-component stratification: hydrostatic to the RK4 accuracy, the
    stabilising mu-gradient held at R_rho times the superadiabatic gradient,
    helium rising downward from c_top."""
    nz = 128
    T, mu, P = I.semiconvection_profile(nz)
    z = (np.arange(nz) + 0.5) / nz
    lnP = np.log(P)
    # central differences of ln P against -g mu / (R T) at interior centres (second order)
    d = (lnP[2:] - lnP[:-2]) / (2.0 / nz)
    assert np.max(np.abs(d + mu[1:-1] / T[1:-1]) / (mu[1:-1] / T[1:-1])) < 1e-3
    nabla = ((np.log(T[2:]) - np.log(T[:-2])) / (lnP[2:] - lnP[:-2]))
    nabla_mu = ((np.log(mu[2:]) - np.log(mu[:-2])) / (lnP[2:] - lnP[:-2]))
    assert np.all(nabla > 1.0 - 1.0 / I.GAMMA)                    # superadiabatic
    assert np.allclose(nabla_mu / (nabla - (1.0 - 1.0 / I.GAMMA)), 1.1, rtol=2e-3)
    c = (1.0 - 1.0 / mu) / 0.75
    assert abs(c[-1] - 0.2) < 0.01 and np.all(np.diff(c) < 0)      # helium increases downward
    p = I.config_semiconvection_3d(16)
    assert p.rho_old.shape == (16, 16, 16) and np.all(p.rho_old > 0) and np.all(p.cs2 > 0)
    assert p.ma == 0.001 and p.rtol == 1e-8 and p.bc == (0, 0, 1)


def test_training_family_and_batch_specs():
    names = {I.config_training_2d(i, n=16).name.split("sigma")[1] for i in range(10000, 10040)}
    assert names == {str(s) for s in I.TRAIN_SIGMAS}
    p = I.config_training_2d(10003, n=16)
    assert 1e-3 <= p.ma <= 1e-1
    specs = I.batch_specs(64)
    assert len(specs) == 64 and specs == I.batch_specs(64)
