"""The schedule of the whole-row red-black sweep, checked on the CPU.

The 3D sweep kernel for levels with whole rows (k_rbgs_row) gives each block
the rows j0 .. j0 + TY - 1 of a chunk of planes k0 .. k1 - 1 and marches up z:
at step p it updates the first colour of plane p on its rows and one halo row
each side, and the second colour of plane p - 2 on its rows, both from the
values staged at the start of the step (one barrier per step); plane p - 3 is
then final.  Halo rows, halo planes and rows past a periodic edge come from
the sweep's input.  This test replays that schedule with numpy on small grids
(several row tiles and z chunks, walls and periodic axes) and checks that it
reproduces the oracle's sequential red-black sweep: the reading that the
lag-two schedule needs no second barrier and no cross-block communication.
The arithmetic of each update uses the oracle's face conductances; only the
order of the updates is under test.  The segmented kernels (512-cell rows as
two segments; the 2D sweep's 128-cell warp segments) are replayed the same
way: the segment schedule of the sweep, and the row-end staging of the
apply and residual kernels, whose end slots hold the neighbouring segment's
cells.
"""
import numpy as np
import pytest

from oracle import multigrid as OM
from oracle import poisson as P

PER, NEU = P.PERIODIC, P.NEUMANN


def _faces(level):
    """Per-cell conductances of the six faces, indexed [face][k, j, i]."""
    op = level.op
    gs = []
    for a in range(3):
        gs += [op.g_minus[a], op.g_plus(a)]
    return gs


def _row_schedule_sweep(level, x_in, f, first, TY, KZ, lag=2):
    nz, ny, nx = level.shape
    bcx, bcy, bcz = level.bc
    g = _faces(level)
    ct = level.ct
    out = np.full_like(x_in, np.nan)

    def wrap(n, c, bc):
        if 0 <= c < n:
            return c
        return c % n if bc == PER else None

    for j0 in range(0, ny, TY):
        for k0 in range(0, nz, KZ):
            k1 = min(k0 + KZ, nz)
            rows = [wrap(ny, j0 - 2 + r, bcy) for r in range(TY + 4)]

            def stage(p):
                kw = wrap(nz, p, bcz)
                a = np.zeros((TY + 4, nx))
                if kw is not None:
                    for r, jw in enumerate(rows):
                        if jw is not None:
                            a[r] = x_in[kw, jw]
                return a

            ring = {p: stage(p) for p in (k0 - 2, k0 - 1, k0)}

            def update(snap, p, r, colour):
                """New values of the colour-`colour` cells of staged row r on plane p."""
                kw, jw = wrap(nz, p, bcz), rows[r]
                i = np.arange(nx)
                xc = snap[p]
                xm, xp = np.roll(xc[r], 1), np.roll(xc[r], -1)     # x walls: face weight 0
                num = f[kw, jw] + g[0][kw, jw] * xm + g[1][kw, jw] * xp
                num = num + g[2][kw, jw] * xc[r - 1] + g[3][kw, jw] * xc[r + 1]
                num = num + g[4][kw, jw] * snap[p - 1][r] + g[5][kw, jw] * snap[p + 1][r]
                d = ct[kw, jw] + sum(g[q][kw, jw] for q in range(6))
                sel = ((i + jw + kw) & 1) == colour
                return sel, num / d

            for p in range(k0 - 1, k1 + lag + 1):
                snap = {q: a.copy() for q, a in ring.items()}      # the state at the barrier
                writes = []
                if p <= k1 and wrap(nz, p, bcz) is not None:
                    for r in range(1, TY + 3):                    # the block's rows and one halo row each side
                        if rows[r] is not None:
                            writes.append((p, r) + update(snap, p, r, first))
                q = p - lag
                if k0 <= q < k1:
                    for r in range(2, TY + 2):
                        writes.append((q, r) + update(snap, q, r, 1 - first))
                for pl, r, sel, v in writes:
                    ring[pl][r][sel] = v[sel]
                w = p - lag - 1                                   # final since the last step
                if k0 <= w < k1:
                    out[w, j0:j0 + TY] = ring[w][2:TY + 2]
                    del ring[w]
                if p + 2 <= k1 + 1:
                    ring[p + 2] = stage(p + 2)
    return out


@pytest.mark.parametrize("shape,bc,TY,KZ", [
    ((7, 32, 16), (PER, PER, NEU), 16, 3),       # (nz, ny, nx); bc per axis x, y, z
    ((6, 16, 8), (NEU, NEU, PER), 8, 2),
    ((8, 16, 12), (PER, NEU, PER), 16, 8),
    ((5, 24, 10), (NEU, PER, NEU), 8, 1),
])
@pytest.mark.parametrize("order", ["RB", "BR"])
def test_row_schedule_equals_sequential_sweep(shape, bc, TY, KZ, order):
    rng = np.random.default_rng(sum(shape) + KZ)
    ct = rng.uniform(0.05, 1.0, shape)
    rho = rng.uniform(1.0, 20.0, shape)
    level = OM.Level(ct, rho, (0.3, 0.5, 0.7), bc)
    x = rng.standard_normal(shape)
    f = rng.standard_normal(shape)
    ref = OM.sweep(level, x, f, order)
    got = _row_schedule_sweep(level, x, f, 0 if order == "RB" else 1, TY, KZ)
    assert not np.isnan(got).any()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_row_schedule_catches_a_one_plane_lag():
    """Planted mistake: the second colour only one plane behind the first,
    still with one barrier per step, reads plane q + 1's first colour before
    that step's update is visible; the replay then differs from the sweep."""
    shape, bc = (6, 16, 8), (PER, PER, NEU)
    rng = np.random.default_rng(5)
    level = OM.Level(rng.uniform(0.05, 1.0, shape), rng.uniform(1.0, 20.0, shape), (0.3, 0.5, 0.7), bc)
    x, f = rng.standard_normal(shape), rng.standard_normal(shape)
    ref = OM.sweep(level, x, f, "RB")
    good = _row_schedule_sweep(level, x, f, 0, 16, 3, lag=2)
    np.testing.assert_allclose(good, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    bad = _row_schedule_sweep(level, x, f, 0, 16, 3, lag=1)
    assert not np.allclose(bad, ref, rtol=1e-6, atol=1e-6)


def _segment_schedule_sweep(level, x_in, f, first, NX, KZ, halo_update=True):
    """The schedule of the segmented sweeps (the 2D sweep's warp per 128-cell
    segment and half chunk, and the 3D sweep's 512-cell rows in two
    segments), replayed on a 2D grid: a segment stages its NX cells plus two
    cells each side (wrapped, or absent past a wall), updates at step p the
    first colour of row p on its cells and on the one outside cell of that
    colour, and the second colour of row p - 2 on its cells; row p - 3 is
    then final.  halo_update=False plants the mistake of leaving the outside
    cell at its input value."""
    nz, _, nx = level.shape
    bcx, _, bcz = level.bc
    g = _faces(level)
    ct = level.ct
    out = np.full_like(x_in, np.nan)

    def wrap(n, c, bc):
        if 0 <= c < n:
            return c
        return c % n if bc == PER else None

    for c0 in range(0, nx, NX):
        cols = [wrap(nx, c0 - 2 + t, bcx) for t in range(NX + 4)]
        for k0 in range(0, nz, KZ):
            k1 = min(k0 + KZ, nz)

            def stage(p):
                kw = wrap(nz, p, bcz)
                a = np.zeros(NX + 4)
                if kw is not None:
                    for t, cw in enumerate(cols):
                        if cw is not None:
                            a[t] = x_in[kw, 0, cw]
                return a

            ring = {p: stage(p) for p in (k0 - 2, k0 - 1, k0)}

            def value(snap, p, t):
                """Gauss-Seidel value of staged position t of row p."""
                kw, cw = wrap(nz, p, bcz), cols[t]
                xc = snap[p]
                num = f[kw, 0, cw] + g[0][kw, 0, cw] * xc[t - 1] + g[1][kw, 0, cw] * xc[t + 1]
                num = num + g[4][kw, 0, cw] * snap[p - 1][t] + g[5][kw, 0, cw] * snap[p + 1][t]
                d = ct[kw, 0, cw] + sum(g[q][kw, 0, cw] for q in (0, 1, 4, 5))
                return num / d

            for p in range(k0 - 1, k1 + 3):
                snap = {q: a.copy() for q, a in ring.items()}
                writes = []
                if p <= k1 and wrap(nz, p, bcz) is not None:
                    kw = wrap(nz, p, bcz)
                    for t in range(2, NX + 2):
                        if ((cols[t] + kw) & 1) == first:
                            writes.append((p, t, value(snap, p, t)))
                    if halo_update:
                        for t in (1, NX + 2):                # the outside cell of the first colour
                            if cols[t] is not None and ((cols[t] + kw) & 1) == first:
                                writes.append((p, t, value(snap, p, t)))
                q = p - 2
                if k0 <= q < k1:
                    kw = wrap(nz, q, bcz)
                    for t in range(2, NX + 2):
                        if ((cols[t] + kw) & 1) == 1 - first:
                            writes.append((q, t, value(snap, q, t)))
                for pl, t, v in writes:
                    ring[pl][t] = v
                w = p - 3
                if k0 <= w < k1:
                    out[w, 0, c0:c0 + NX] = ring[w][2:NX + 2]
                    del ring[w]
                if p + 2 <= k1 + 1:
                    ring[p + 2] = stage(p + 2)
    return out


@pytest.mark.parametrize("shape,bc,NX,KZ", [
    ((9, 1, 16), (PER, PER, NEU), 8, 3),         # (nz, 1, nx); bc per axis x, y, z
    ((8, 1, 24), (NEU, PER, PER), 8, 4),
    ((7, 1, 16), (NEU, PER, NEU), 4, 2),
    ((6, 1, 8), (PER, PER, PER), 8, 6),          # one segment: its outside cells wrap onto itself
])
@pytest.mark.parametrize("order", ["RB", "BR"])
def test_segment_schedule_equals_sequential_sweep(shape, bc, NX, KZ, order):
    rng = np.random.default_rng(sum(shape) + NX)
    level = OM.Level(rng.uniform(0.05, 1.0, shape), rng.uniform(1.0, 20.0, shape), (0.3, 1.0, 0.7), bc)
    x, f = rng.standard_normal(shape), rng.standard_normal(shape)
    ref = OM.sweep(level, x, f, order)
    got = _segment_schedule_sweep(level, x, f, 0 if order == "RB" else 1, NX, KZ)
    assert not np.isnan(got).any()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_segment_schedule_needs_the_outside_update():
    """Planted mistake: without the first-colour update of the outside cell,
    the second colour at a segment's end reads a stale neighbour."""
    shape, bc = (8, 1, 24), (NEU, PER, PER)
    rng = np.random.default_rng(7)
    level = OM.Level(rng.uniform(0.05, 1.0, shape), rng.uniform(1.0, 20.0, shape), (0.3, 1.0, 0.7), bc)
    x, f = rng.standard_normal(shape), rng.standard_normal(shape)
    ref = OM.sweep(level, x, f, "RB")
    bad = _segment_schedule_sweep(level, x, f, 0, 8, 4, halo_update=False)
    assert not np.allclose(bad, ref, rtol=1e-6, atol=1e-6)


def _segmented_apply(level, x, NX, whole_row_wrap=False):
    """A x by the segmented row kernels' staging, replayed with numpy: the
    grid's rows are cut into segments of NX cells; a segment's staged row
    holds its cells plus one row-end slot each side, filled with the cell
    just outside the segment (wrapped on a periodic x axis, a wall -- no
    face -- past a wall), and the x faces at the segment's ends read those
    slots; y and z neighbours come from the grid.  whole_row_wrap plants
    the mistake of wrapping inside the segment, as a whole-row kernel does."""
    nz, ny, nx = level.shape
    bcx = level.bc[0]
    op = level.op
    g = _faces(level)
    y = op.ct * x
    for a in (1, 2):                                     # y and z faces from the grid
        xm = np.roll(x, 1, axis=2 - a)
        xp = np.roll(x, -1, axis=2 - a)
        y = y + g[2 * a] * (x - xm) + g[2 * a + 1] * (x - xp)
    for c0 in range(0, nx, NX):
        cols = np.arange(c0, c0 + NX)
        left = c0 - 1 if not whole_row_wrap else c0 + NX - 1
        right = c0 + NX if not whole_row_wrap else c0
        xl = np.empty_like(x[..., cols])
        xr = np.empty_like(x[..., cols])
        xl[..., 1:] = x[..., cols[:-1]]
        xr[..., :-1] = x[..., cols[1:]]
        okl = left >= 0 or bcx == PER or whole_row_wrap
        okr = right < nx or bcx == PER or whole_row_wrap
        xl[..., 0] = x[..., left % nx] if okl else 0.0
        xr[..., -1] = x[..., right % nx] if okr else 0.0
        wl = g[0][..., cols].copy()
        wr = g[1][..., cols].copy()
        if not okl:
            wl[..., 0] = 0.0
        if not okr:
            wr[..., -1] = 0.0
        y[..., cols] += wl * (x[..., cols] - xl) + wr * (x[..., cols] - xr)
    return y


@pytest.mark.parametrize("shape,bc,NX", [
    ((4, 6, 16), (PER, PER, NEU), 8),        # (nz, ny, nx); bc per axis x, y, z
    ((3, 4, 24), (NEU, PER, NEU), 8),
    ((5, 2, 12), (PER, NEU, PER), 4),
    ((2, 3, 8), (NEU, NEU, NEU), 8),         # one segment: both ends are walls
])
def test_segmented_apply_equals_operator(shape, bc, NX):
    rng = np.random.default_rng(sum(shape) + NX)
    level = OM.Level(rng.uniform(0.05, 1.0, shape), rng.uniform(1.0, 20.0, shape), (0.3, 0.5, 0.7), bc)
    x = rng.standard_normal(shape)
    ref = level.op.apply(x)
    got = _segmented_apply(level, x, NX)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_segmented_apply_needs_the_outside_cells():
    """Planted mistake: a segment of a periodic row wrapping onto itself (the
    whole-row rule) instead of reading the neighbouring segment's cell."""
    shape, bc = (4, 6, 16), (PER, PER, NEU)
    rng = np.random.default_rng(3)
    level = OM.Level(rng.uniform(0.05, 1.0, shape), rng.uniform(1.0, 20.0, shape), (0.3, 0.5, 0.7), bc)
    x = rng.standard_normal(shape)
    ref = level.op.apply(x)
    np.testing.assert_allclose(_segmented_apply(level, x, 16), ref, rtol=1e-12, atol=1e-12)   # one segment: fine
    bad = _segmented_apply(level, x, 8, whole_row_wrap=True)
    assert not np.allclose(bad, ref, rtol=1e-6, atol=1e-6)
