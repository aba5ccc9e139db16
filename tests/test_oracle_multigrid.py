"""Pins of the oracle's multigrid pieces: transfer identities, an independent
cell-by-cell Gauss-Seidel loop, fixed points, symmetry of the V-cycle and
convergence to the direct solve (no GPU)."""
import numpy as np
import pytest

from oracle import multigrid as M
from oracle import poisson as P

PER, NEU = P.PERIODIC, P.NEUMANN


def _coefs(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.05, 1.0, shape), rng.uniform(0.5, 3.0, shape)


def test_hierarchy_shapes():
    lv = M.build_hierarchy(np.ones((64, 1, 64)), np.ones((64, 1, 64)), (1, 1, 1), (PER, PER, NEU))
    assert [L.shape for L in lv] == [(64, 1, 64), (32, 1, 32), (16, 1, 16), (8, 1, 8)]
    lv = M.build_hierarchy(np.ones((32, 32, 32)), np.ones((32, 32, 32)), (1, 1, 1), (PER, PER, NEU))
    assert lv[-1].shape == (4, 4, 4) and len(lv) == 4
    # a periodic axis never reaches an odd count > 1 (red-black stays a 2-colouring)
    lv = M.build_hierarchy(np.ones((100, 1, 100)), np.ones((100, 1, 100)), (1, 1, 1), (NEU, PER, PER))
    for L in lv:
        assert L.shape[0] % 2 == 0 or L.shape[0] == 1


@pytest.mark.parametrize("halved", [(True, False, True), (True, True, True), (False, False, True)])
def test_transfer_identities(halved):
    """Restriction and prolongation are exact on constants, and
    <R r, e> * 2^d' = <r, P e>  (R = 2^-d' P^T)."""
    shape = (8, 4 if halved[1] else 3, 6)
    rng = np.random.default_rng(1)
    c = np.full(shape, 2.5)
    assert np.allclose(M.restrict(c, halved), 2.5)
    cshape = M.restrict(c, halved).shape
    assert np.allclose(M.prolong(np.full(cshape, -1.5), halved), -1.5)
    r = rng.standard_normal(shape)
    e = rng.standard_normal(cshape)
    dprime = sum(halved)
    assert np.vdot(M.restrict(r, halved), e) * 2 ** dprime == pytest.approx(np.vdot(r, M.prolong(e, halved)), rel=1e-13)


def test_coarse_coefficients_are_child_means():
    shape = (4, 1, 4)
    ct, rho = _coefs(shape, 2)
    lv = M.build_hierarchy(ct, rho, (0.25, 1.0, 0.25), (PER, PER, NEU), coarse_max=1)
    c1 = lv[1]
    assert c1.shape == (2, 1, 2)
    assert c1.ct[0, 0, 1] == pytest.approx(ct[0:2, 0, 2:4].mean(), rel=1e-15)
    assert c1.rho[1, 0, 0] == pytest.approx(rho[2:4, 0, 0:2].mean(), rel=1e-15)
    assert c1.h == (0.5, 1.0, 0.5)


def _loop_gs(level, x, f, colour_first):
    """Independent reference: Gauss-Seidel visiting the cells one at a time
    in lexicographic order, first all cells of one colour, then the other,
    solving each cell's row of the assembled matrix."""
    A = level.op.assemble().toarray()
    x = x.ravel().copy()
    f = f.ravel()
    nz, ny, nx = level.shape
    for c in (colour_first, 1 - colour_first):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    if (i + j + k) % 2 != c:
                        continue
                    r = i + nx * (j + ny * k)
                    s = f[r] - A[r] @ x + A[r, r] * x[r]
                    x[r] = s / A[r, r]
    return x.reshape(level.shape)


@pytest.mark.parametrize("shape,bc", [((6, 1, 8), (PER, PER, NEU)), ((4, 4, 6), (PER, PER, NEU)),
                                      ((5, 1, 7), (NEU, PER, NEU))])
def test_redblack_sweep_matches_cellwise_loop(shape, bc):
    ct, rho = _coefs(shape, 3)
    lv = M.Level(ct, rho, (0.2, 0.3, 0.25), bc)
    rng = np.random.default_rng(4)
    x0, f = rng.standard_normal(shape), rng.standard_normal(shape)
    for order, first in (("RB", 0), ("BR", 1)):
        assert np.allclose(M.sweep(lv, x0, f, order), _loop_gs(lv, x0, f, first), rtol=1e-13, atol=1e-13)


def test_sweep_fixed_point_and_contraction():
    shape = (8, 1, 8)
    ct, rho = _coefs(shape, 5)
    lv = M.Level(ct, rho, (1 / 8, 1.0, 1 / 8), (PER, PER, NEU))
    f = np.random.default_rng(6).standard_normal(shape)
    xs = P.solve_direct(lv.op, f)
    assert np.allclose(M.sweep(lv, xs, f, "RB"), xs, rtol=1e-12, atol=1e-12)
    x = np.zeros(shape)
    e_prev = xs
    for _ in range(3):
        x = M.sweep(lv, x, f, "RB")
        e = x - xs
        # Gauss-Seidel is a contraction in the A-norm
        assert np.vdot(e, lv.op.apply(e)) < np.vdot(e_prev, lv.op.apply(e_prev))
        e_prev = e


@pytest.mark.parametrize("shape,bc", [((16, 1, 16), (PER, PER, NEU)), ((8, 8, 8), (PER, PER, NEU)),
                                      ((8, 1, 32), (PER, PER, NEU))])
def test_vcycle_symmetric_positive(shape, bc):
    ct, rho = _coefs(shape, 7)
    lv = M.build_hierarchy(ct, rho, (0.1, 0.1, 0.1), bc, coarse_max=8)
    assert len(lv) >= 3
    rng = np.random.default_rng(8)
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    Mu, Mv = M.vcycle(lv, u), M.vcycle(lv, v)
    assert np.vdot(v, Mu) == pytest.approx(np.vdot(u, Mv), rel=1e-12)
    assert np.vdot(u, Mu) > 0
    # linear: M(2u + v) = 2 M u + M v
    assert np.allclose(M.vcycle(lv, 2 * u + v), 2 * Mu + Mv, rtol=1e-12, atol=1e-12)


def test_mg_pcg_converges_to_direct_solution():
    shape = (32, 1, 32)
    ct, rho = _coefs(shape, 9)
    ct *= 1e-3      # near-singular regime: small c~ relative to the flux part
    lv = M.build_hierarchy(ct, rho, (1 / 32, 1.0, 1 / 32), (PER, PER, NEU))
    f = np.random.default_rng(10).standard_normal(shape)
    x, it, hist = M.mg_pcg(lv, f, rtol=1e-12)
    xs = P.solve_direct(lv[0].op, f)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert it < 40, it
