"""Pins of oracle.fem (the Q1 finite-element operator of Sec. 2.5): the
element matrices against Gauss quadrature of the bilinear / trilinear basis,
the lumped mass against the basis integrals, the Fourier symbol, the null
space of the stiffness part, symmetry and definiteness, second-order
convergence, and the paper's printed errors for the e^x test (Sec. 2.5.2,
Table perturbtest)."""
import itertools
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import fem as F
from oracle.poisson import NEUMANN, PERIODIC
from paper_1112_3507_gb300 import inputs as I

GOLDEN = Path(__file__).parent / "golden" / "perturbtest_table.txt"


def _basis(c, xi):
    """1D linear basis function of corner c (0 or 1) at xi in [0, 1], and its derivative."""
    return (1.0 - xi, -1.0) if c == 0 else (xi, 1.0)


def _element_by_quadrature(h):
    """Stiffness and consistent mass of one box element of sides h by two-point
    Gauss-Legendre quadrature per axis (exact for these polynomial products)."""
    d = len(h)
    g = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))
    corners = list(itertools.product((0, 1), repeat=d))
    K = np.zeros((len(corners), len(corners)))
    M = np.zeros_like(K)
    for pt in itertools.product(g, repeat=d):
        w = np.prod(h) / 2 ** d                          # each Gauss weight is 1/2 on [0,1]
        for p, cp in enumerate(corners):
            vp = [_basis(cp[a], pt[a]) for a in range(d)]
            for q, cq in enumerate(corners):
                vq = [_basis(cq[a], pt[a]) for a in range(d)]
                M[p, q] += w * np.prod([vp[a][0] * vq[a][0] for a in range(d)])
                for a in range(d):
                    gp = vp[a][1] / h[a] * np.prod([vp[b][0] for b in range(d) if b != a])
                    gq = vq[a][1] / h[a] * np.prod([vq[b][0] for b in range(d) if b != a])
                    K[p, q] += w * gp * gq
    return corners, K, M


def _brute_matrix(ct, rho, h, bc):
    """Global matrix element by element: a point of grid index (i, j, k) is
    corner c of the element whose lowest corner is index - c (wrapped on a
    periodic axis; an element past a wall does not exist)."""
    ct3 = ct if ct.ndim == 3 else ct[:, None, :]
    rho3 = rho if rho.ndim == 3 else rho[:, None, :]
    nz, ny, nx = ct3.shape
    n = (nx, ny, nz)
    axes = [a for a in range(3) if n[a] > 1]
    corners, Kref, Mref = _element_by_quadrature([h[a] for a in axes])
    N = nx * ny * nz
    B = np.zeros((N, N))
    Mc = np.zeros((N, N))

    def flat(c3):
        return c3[0] + nx * (c3[1] + ny * c3[2])

    for low in itertools.product(range(nx), range(ny), range(nz)):
        ok = all(not (bc[a] == NEUMANN and low[a] == n[a] - 1) for a in axes)
        if not ok:
            continue
        pts = []
        for c in corners:
            p = list(low)
            for ia, a in enumerate(axes):
                p[a] = (p[a] + c[ia]) % n[a]
            pts.append(flat(p))
        rvals = [rho3.reshape(-1)[p] for p in pts]
        kappa = len(pts) / sum(rvals)
        for p in range(len(pts)):
            for q in range(len(pts)):
                B[pts[p], pts[q]] += kappa * Kref[p, q]
                Mc[pts[p], pts[q]] += Mref[p, q]
    V = Mc.sum(axis=1)                                     # lumped mass: row sums
    B += np.diag(V * ct3.reshape(-1))
    return B, V


CASES = [
    ((5, 1, 6), (0.3, 1.0, 0.2), (NEUMANN, PERIODIC, PERIODIC)),
    ((4, 1, 5), (0.25, 1.0, 0.25), (PERIODIC, PERIODIC, NEUMANN)),
    ((4, 3, 5), (0.2, 0.3, 0.25), (NEUMANN, PERIODIC, NEUMANN)),
    ((3, 4, 4), (0.5, 0.4, 0.3), (PERIODIC, NEUMANN, PERIODIC)),
    ((3, 3, 3), (0.1, 0.1, 0.1), (NEUMANN, NEUMANN, NEUMANN)),
]


@pytest.mark.parametrize("n,h,bc", CASES)
def test_matrix_matches_quadrature_assembly(n, h, bc):
    """B assembled from element matrices integrated by Gauss quadrature, with
    the harmonic-mean element kappa and the lumped c~ term, equals the
    oracle's matrix, its matrix-free apply and its diagonal."""
    rng = np.random.default_rng(sum(n))
    shape = (n[2], n[1], n[0])
    rho = np.exp(rng.uniform(-2, 2, shape))
    ct = rng.uniform(0.5, 3.0, shape)
    op = F.FEOperator(ct, rho, h, bc)
    B, V = _brute_matrix(ct, rho, h, bc)
    np.testing.assert_allclose(op.volume.ravel(), V, rtol=1e-13)
    np.testing.assert_allclose(op.assemble().toarray(), B, rtol=1e-12, atol=1e-12 * np.abs(B).max())
    x = rng.standard_normal(shape)
    np.testing.assert_allclose(op.apply(x).ravel(), B @ x.ravel(), rtol=1e-12, atol=1e-12 * np.abs(B).max())
    np.testing.assert_allclose(op.diagonal().ravel(), np.diag(B), rtol=1e-12)


def test_two_dimensional_input_is_the_xz_plane():
    """A (nz, nx) array is the grid with one point along y."""
    rng = np.random.default_rng(3)
    rho, ct = np.exp(rng.uniform(-1, 1, (6, 7))), rng.uniform(1, 2, (6, 7))
    h, bc = (0.2, 1.0, 0.3), (NEUMANN, PERIODIC, PERIODIC)
    x = rng.standard_normal((6, 7))
    a = F.FEOperator(ct, rho, h, bc).apply(x)
    b = F.FEOperator(ct[:, None, :], rho[:, None, :], h, bc).apply(x[:, None, :])
    np.testing.assert_allclose(a, b, rtol=1e-15)


@pytest.mark.parametrize("shape,modes", [((8, 1, 12), (3, 0, 2)), ((6, 8, 10), (1, 2, 5)), ((4, 4, 4), (2, 2, 2))])
def test_fourier_symbol(shape, modes):
    """On a periodic grid with constant kappa and c~ the mode cos(t . i) is an
    eigenvector of B / V with the Q1 symbol (stiffness symbol 2 (1 - cos t) / h
    per axis times the mass symbol h (2 + cos t) / 3 of the others)."""
    nz, ny, nx = shape
    h = (0.1, 0.2, 0.15)
    kappa0, c0 = 2.5, 0.7
    op = F.FEOperator(np.full(shape, c0), np.full(shape, 1.0 / kappa0), h, (PERIODIC,) * 3)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    n = (nx, ny, nz)
    t = [2 * np.pi * modes[a] / n[a] for a in range(3)]
    v = np.cos(t[0] * i + t[1] * j + t[2] * k)
    th = [t[a] for a in range(3) if n[a] > 1]
    hh = [h[a] for a in range(3) if n[a] > 1]
    lam = F.symbol(th, hh, kappa0, c0)
    # the symbol written out independently for the check
    want = c0
    for ia in range(len(th)):
        term = (2 - 2 * np.cos(th[ia])) / hh[ia] ** 2
        for ib in range(len(th)):
            if ib != ia:
                term *= (2 + np.cos(th[ib])) / 3
        want += kappa0 * term
    assert lam == pytest.approx(want, rel=1e-14)
    np.testing.assert_allclose(op.apply(v), op.volume * lam * v, atol=1e-10 * np.abs(op.volume * lam).max())


@pytest.mark.parametrize("n,h,bc", CASES)
def test_constants_and_definiteness(n, h, bc):
    """The stiffness part annihilates constants (B 1 = V c~); B is symmetric
    with positive eigenvalues for rho > 0 and c~ > 0 (Sec. 2.5)."""
    rng = np.random.default_rng(11)
    shape = (n[2], n[1], n[0])
    rho = np.exp(rng.uniform(-4, 4, shape))
    ct = np.exp(rng.uniform(-3, 1, shape))
    op = F.FEOperator(ct, rho, h, bc)
    np.testing.assert_allclose(op.apply(np.ones(shape)), op.volume * ct, rtol=1e-10)
    B = op.assemble().toarray()
    np.testing.assert_allclose(B, B.T, rtol=0, atol=1e-14 * np.abs(B).max())
    assert np.linalg.eigvalsh(B).min() > 0


def test_volumes_sum_to_the_domain():
    """The lumped masses tile the domain: sum V = prod over axes of the extent
    (n h periodic, (n - 1) h between walls)."""
    op = F.FEOperator(np.ones((5, 4, 6)), np.ones((5, 4, 6)), (0.1, 0.2, 0.3), (NEUMANN, PERIODIC, NEUMANN))
    assert op.volume.sum() == pytest.approx((5 * 0.1) * (4 * 0.2) * (4 * 0.3), rel=1e-14)


def test_second_order_variable_kappa():
    """-div(kappa grad u) + u = f with u = cos(pi x) cos(pi y) cos(pi z) on the
    unit cube (zero normal derivative at the walls), kappa = 1 + x / 2: the
    nodal error falls by about 4 per halving of h."""
    errs = []
    for n in (9, 17, 33):
        h = 1.0 / (n - 1)
        z, y, x = np.meshgrid(*(np.arange(n) * h,) * 3, indexing="ij")
        u = np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        kap = 1.0 + 0.5 * x
        ux = -np.pi * np.sin(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        f = kap * 3 * np.pi ** 2 * u - 0.5 * ux + u
        op = F.FEOperator(np.ones_like(u), 1.0 / kap, (h, h, h), (NEUMANN,) * 3)
        sol = F.solve(op, op.volume * f)
        errs.append(np.abs(sol - u).max())
    r = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(3.5 < v < 4.5 for v in r), (errs, r)


def _exp_errors(n, perturb=None):
    t = I.analytic_exp_problem_nodes(n, perturb=perturb)
    op = F.FEOperator(t["ctilde"], 1.0 / t["kappa"], t["h"], t["bc"])
    b = op.volume * t["f"]
    # the Neumann data enter the weak form as boundary integrals: g times the
    # wall share (the periodic spacing) of each wall point
    hz = t["h"][2]
    b[:, :, 0] += t["g_low"] * hz
    b[:, :, -1] += t["g_high"] * hz
    err = np.abs(F.solve(op, b) - t["exact"])
    return float(err.mean()), float(np.sqrt(np.mean(err ** 2))), float(err.max())


def _golden():
    rows = {}
    for line in GOLDEN.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows[name] = [float(v) for v in vals]
    return rows


def test_exp_test_reproduces_the_papers_table():
    """Sec. 2.5.2, Table perturbtest: with Q1 elements, the lumped c~ term and
    100 intervals per direction, the errors against e^x (L1, L2 as means over
    the points, Linf) are the paper's unperturbed ones to within 0.5 % (the
    two printed rows differ by up to 0.1 % between solver runs)."""
    got = _exp_errors(101)
    want = _golden()["unperturbed_1core"]
    for g, w in zip(got, want):
        assert g == pytest.approx(w, rel=5e-3), (got, want)


def test_exp_test_perturbations():
    """Same table, perturbed rows.  The noise draws are not the paper's, so
    only magnitudes are pinned: each perturbation of size 1e-2 raises the
    error, perturbing kappa raises the maximum error most (paper: Linf 2.3e-4
    against 3.0e-5 unperturbed), and every error stays at the magnitude of
    the paper's perturbed rows (below 3e-4)."""
    e0 = _exp_errors(101)
    ef = _exp_errors(101, "f")
    ek = _exp_errors(101, "kappa")
    ec = _exp_errors(101, "c")
    for e in (ef, ek, ec):
        assert all(a > b for a, b in zip(e, e0)), (e, e0)
        assert e[2] < 3e-4
    assert ek[2] > max(ef[2], ec[2])
    assert 4.0 < ek[2] / e0[2] < 16.0
