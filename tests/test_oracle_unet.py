"""Pins of the network oracle: closed-form special cases of the layers and
central finite differences of the whole network's hand-derived gradients."""
import numpy as np
import pytest

from oracle import unet as U


def test_conv3_center_tap_is_channel_matmul_and_delta_gives_flipped_kernel():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 5, 6, 3))
    W = np.zeros((3, 3, 3, 4))
    W[1, 1] = rng.standard_normal((3, 4))
    b = rng.standard_normal(4)
    assert np.allclose(U.conv3_fwd(x, W, b), x @ W[1, 1] + b)
    # a unit impulse at (2, 2) reproduces the kernel, flipped (cross-correlation)
    d = np.zeros((1, 5, 5, 1))
    d[0, 2, 2, 0] = 1.0
    K = rng.standard_normal((3, 3, 1, 1))
    out = U.conv3_fwd(d, K, np.zeros(1))
    assert np.allclose(out[0, 1:4, 1:4, 0], K[::-1, ::-1, 0, 0])
    # zero padding: a constant image loses the outside taps at the border
    one = np.ones((1, 4, 4, 1))
    Ks = np.ones((3, 3, 1, 1))
    o = U.conv3_fwd(one, Ks, np.zeros(1))[0, :, :, 0]
    assert o[0, 0] == 4 and o[0, 1] == 6 and o[1, 1] == 9


def test_pool_up_adjoint_and_constant():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 8, 6, 3))
    y = rng.standard_normal((2, 4, 3, 3))
    assert np.allclose(U.pool_fwd(np.full((1, 4, 4, 2), 3.0)), 3.0)
    # <pool x, y> = <x, pool_bwd y>;  <up y, x> = <y, up_bwd x>
    assert np.vdot(U.pool_fwd(x), y) == pytest.approx(np.vdot(x, U.pool_bwd(y)))
    assert np.vdot(U.up_fwd(y), x) == pytest.approx(np.vdot(y, U.up_bwd(x)))


def _fd_check(f, P, G, names, rng, n=6, eps=1e-6):
    for name in names:
        A = P[name]
        for _ in range(n):
            idx = tuple(rng.integers(0, s) for s in A.shape)
            old = A[idx]
            A[idx] = old + eps
            fp = f()
            A[idx] = old - eps
            fm = f()
            A[idx] = old
            num = (fp - fm) / (2 * eps)
            assert num == pytest.approx(G[name][idx], rel=1e-5, abs=1e-8), (name, idx)


def test_network_gradients_match_finite_differences():
    """Tiny instance (channels 2, 3, 3, 4; 8x8 images): every parameter
    tensor and the input, against central differences of the scalar loss."""
    rng = np.random.default_rng(3)
    ch = (2, 3, 3, 4)
    P = U.init_params(rng, cin=3, ch=ch)
    for k in P:
        if k.islower():
            P[k] = rng.standard_normal(P[k].shape) * 0.1
    x = rng.standard_normal((2, 8, 8, 3))
    t = rng.standard_normal((2, 8, 8, 1))

    def loss():
        y, _ = U.forward(P, x, ch)
        return U.mse_loss(y, t)[0]

    y, cache = U.forward(P, x, ch)
    L, gy = U.mse_loss(y, t)
    G, gx = U.backward(P, cache, gy, ch)
    assert set(G) == {n for n, _ in U.param_shapes(3, ch)}
    _fd_check(loss, P, G, [n for n, _ in U.param_shapes(3, ch)], rng)
    # input gradient
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        old = x[idx]
        x[idx] = old + 1e-6
        fp = loss()
        x[idx] = old - 1e-6
        fm = loss()
        x[idx] = old
        assert (fp - fm) / 2e-6 == pytest.approx(gx[idx], rel=1e-5, abs=1e-8)


def test_param_count_of_the_default_network():
    n = sum(int(np.prod(s)) for _, s in U.param_shapes())
    assert 200_000 < n < 260_000


def test_features_invariances():
    """The network input is invariant to the scale of v (ch0 and s scale
    out), the log-density channel vanishes for constant rho, and s is
    linear in rms(v)."""
    rng = np.random.default_rng(5)
    H, W = 8, 12
    v = rng.standard_normal((H, W))
    rho = 1.0 + rng.random((H, W))
    ct = 0.1 + rng.random((H, W))
    x1, s1 = U.features(v, rho, ct, 0.125)
    x2, s2 = U.features(3.0 * v, rho, ct, 0.125)
    assert np.allclose(x1, x2) and s2 == pytest.approx(3.0 * s1)
    assert np.sqrt(np.mean(x1[0, :, :, 0] ** 2)) == pytest.approx(1.0)
    x3, _ = U.features(v, np.full((H, W), 2.5), ct, 0.125)
    assert np.all(x3[0, :, :, 1] == 0.0)
    # constant c~ rho h^2 = 1 gives a zero third channel
    x4, s4 = U.features(v, np.full((H, W), 2.0), np.full((H, W), 0.5 * 64.0), 0.125)
    assert np.allclose(x4[0, :, :, 2], 0.0)
    assert s4 == pytest.approx(np.sqrt(np.mean(v * v)) / (32.0 + np.pi ** 2 / 2.0))
