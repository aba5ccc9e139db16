"""Pins of oracle.diffusion (the dissipative fourth-order stencil, Sec. 4):
the paper's printed weights, the Fourier symbol, fourth-order convergence,
conservation, dissipativity against the nine-point stencil, and the
stability limit of an explicit step."""
import numpy as np
import pytest

from oracle import diffusion as D
from oracle.poisson import NEUMANN, PERIODIC


def test_interior_weights_are_the_papers():
    """Eq. dissipativestencil4: (-1, 16, -30, 16, -1) / (12 h^2) away from walls."""
    n, h = 16, 0.25
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        col = D.second_derivative(e, h, 0, PERIODIC)
        want = np.zeros(n)
        for off, w in ((-2, -1.0), (-1, 16.0), (0, -30.0), (1, 16.0), (2, -1.0)):
            want[(k + off) % n] = w / (12 * h * h)
        np.testing.assert_allclose(col, want, atol=1e-13)
    # the flux form's face value is Eq. fv-approach2's
    u = np.random.default_rng(1).standard_normal(n)
    p = D.face_derivative(u, h, 0, PERIODIC)
    i = 5
    assert p[i] == pytest.approx((u[i - 1] - 15 * u[i] + 15 * u[i + 1] - u[i + 2]) / (12 * h), rel=1e-14)


@pytest.mark.parametrize("k", [1, 3, 7, 16])
def test_fourier_symbol_periodic(k):
    """A periodic mode exp(i t j) is an eigenvector with eigenvalue
    (32 cos t - 2 cos 2t - 30) / (12 h^2); in 3D the symbols add."""
    n, h = 32, 0.1
    t = 2 * np.pi * k / n
    j = np.arange(n)
    v = np.cos(t * j)
    np.testing.assert_allclose(D.second_derivative(v, h, 0, PERIODIC), D.symbol_dissipative(t) / h ** 2 * v,
                               atol=1e-10)
    z, y, x = np.meshgrid(np.arange(8), np.arange(4), np.arange(16), indexing="ij")
    tx, ty, tz = 2 * np.pi * 3 / 16, 2 * np.pi * 1 / 4, 2 * np.pi * 2 / 8
    w = np.cos(tx * x + ty * y + tz * z)
    hs = (0.1, 0.2, 0.3)
    lam = sum(D.symbol_dissipative(tt) / hh ** 2 for tt, hh in ((tx, hs[0]), (ty, hs[1]), (tz, hs[2])))
    np.testing.assert_allclose(D.laplacian4(w, hs, (PERIODIC,) * 3), lam * w, atol=1e-9)


def test_fourth_order_convergence():
    """On sin(2 pi x) sampled at cell centres the error of u_xx falls 16x per
    halving of h (to the rounding floor)."""
    errs = []
    for n in (16, 32, 64, 128):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        u = np.sin(2 * np.pi * x)
        err = np.max(np.abs(D.second_derivative(u, h, 0, PERIODIC) + (2 * np.pi) ** 2 * u))
        errs.append(err)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(15.0 < r < 17.0 for r in ratios), ratios


@pytest.mark.parametrize("bc", [PERIODIC, NEUMANN])
def test_conservative(bc):
    """Flux form: the sum of the second derivative over all cells vanishes
    (periodic wrap, or no flux through the walls)."""
    u = np.random.default_rng(2).standard_normal((6, 5, 12))
    out = D.laplacian4(u, (0.1, 0.2, 0.3), (PERIODIC, PERIODIC, bc))
    assert abs(out.sum()) <= 1e-10 * np.abs(out).sum()


def test_neumann_exact_on_even_extension():
    """On a wall axis the operator equals the periodic one applied to the
    even (mirror) extension of u, except at the two cells next to each wall,
    whose wall face carries no flux by construction."""
    n, h = 12, 0.5
    u = np.random.default_rng(3).standard_normal(n)
    ext = np.concatenate([u, u[::-1]])
    per = D.second_derivative(ext, h, 0, PERIODIC)[:n]
    neu = D.second_derivative(u, h, 0, NEUMANN)
    np.testing.assert_allclose(neu[2:n - 2], per[2:n - 2], rtol=1e-13, atol=1e-13)
    # the mirror extension makes the wall face's derivative vanish by symmetry,
    # so the two forms agree next to the walls too
    np.testing.assert_allclose(neu, per, rtol=1e-12, atol=1e-12)


def test_dissipative_unlike_the_nine_point_stencil():
    """Sec. 4: the five-point symbol is negative for every non-zero
    frequency (-16/3 at the grid frequency); the nine-point stencil's symbol
    vanishes there, so a forward step leaves that mode undamped."""
    t = np.linspace(1e-3, np.pi, 400)
    s5 = D.symbol_dissipative(t)
    assert np.all(s5 < 0) and D.symbol_dissipative(np.pi) == pytest.approx(-16.0 / 3.0)
    n, h = 32, 1.0
    v = np.cos(np.pi * np.arange(n))
    assert np.allclose(D.nondissipative_1d(v, h), 0.0, atol=1e-12)
    # the nine-point weights annihilate constants and approximate u_xx
    x = np.arange(n, dtype=float)
    assert np.allclose(D.nondissipative_1d(np.ones(n), h), 0.0)
    c = np.cos(2 * np.pi * x / n)
    approx = D.nondissipative_1d(c, h)
    assert np.max(np.abs(approx + (2 * np.pi / n) ** 2 * c)) < 1e-3


def test_explicit_step_stability_limit():
    """Forward Euler damps every mode while nu dt / h^2 <= 3 / (8 d) (the
    grid-frequency amplification 1 - (16/3) d lambda reaches -1 there) and
    the grid-frequency mode grows beyond it."""
    h = 0.1
    z, y, x = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    v = np.cos(np.pi * (x + y + z))                  # the grid-frequency mode in 3D
    for lam, grows in ((0.99 * 3 / 24, False), (1.01 * 3 / 24, True)):
        dt = lam * h * h
        w = D.explicit_diffusion_step(v, 1.0, dt, (h, h, h), (PERIODIC,) * 3)
        amp = np.abs(w).max() / np.abs(v).max()
        assert (amp > 1.0) == grows, (lam, amp)
