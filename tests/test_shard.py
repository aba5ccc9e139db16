"""The z-slab decomposed solve (paper_1112_3507_gb300.shard) on CPU ranks.

The decomposition logic -- slab bounds, ghost planes, halo exchanges, the
all-reduce points of the Krylov loops, the gather/scatter of the level-1
vectors to rank 0 -- is product code; the per-rank stencil work here is a
float64 numpy stand-in built from the oracle's operator and multigrid
functions.  Ranks are threads (ThreadComm) or gloo processes (TorchComm,
world size 2); results are compared with the single-domain oracle."""
import dataclasses
import os
import sys

import numpy as np
import pytest
import torch

from oracle import multigrid as OM
from oracle import poisson as P
from paper_1112_3507_gb300 import inputs as I
from paper_1112_3507_gb300 import shard as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NEU, PER = I.BC_NEUMANN, I.BC_PERIODIC


class NumpySlab:
    """The per-rank backend interface of shard.py in float64 numpy (a host
    stand-in for the GPU kernels): vectors are torch CPU tensors of the
    extended local size."""

    def __init__(self, geo, p):
        self.geo = geo
        g = geo
        self.shape = (g.nz_ext, g.n[1], g.n[0])
        ct = P.ctilde(p.rho_old, p.cs2, p.dt)
        self.ct, self.rho = g.extract(ct).reshape(self.shape), g.extract(p.rho_new).reshape(self.shape)
        self.op = P.Operator(self.ct, self.rho, g.h, g.bc_ext)
        self.levels = OM.build_hierarchy(self.ct, self.rho, g.h, g.bc_ext)
        self.f = g.extract(p.f).reshape(-1)
        self.N = self.f.size
        self.v = {}
        self.o0, self.o1 = g.glo * g.plane, (g.glo + g.nz_loc) * g.plane

    def like(self):
        return torch.zeros(1, dtype=torch.float64)

    def zeros(self, name, prec):
        self.v[name] = torch.zeros(self.N, dtype=torch.float64)

    def buf_f32(self, n):
        return torch.zeros(n, dtype=torch.float64)

    buf_f64 = buf_f32

    def empty_like_buf(self, b):
        return torch.zeros_like(b)

    def _a(self, name):
        return self.v[name].numpy()

    def set_rhs(self, name):
        a = self._a(name)
        a[:] = 0.0
        a[self.o0:self.o1] = self.f[self.o0:self.o1]

    def axpby(self, a, x, b, y, out):
        s = slice(self.o0, self.o1)
        val = a * self._a(x)[s] + (b * self._a(y)[s] if y is not None else 0.0)
        self._a(out)[s] = val

    def mul(self, d, r, z):
        s = slice(self.o0, self.o1)
        self._a(z)[s] = self._a(d)[s] * self._a(r)[s]

    def dot(self, a, b):
        s = slice(self.o0, self.o1)
        return float(np.dot(self._a(a)[s], self._a(b)[s]))

    def jacobi_dinv(self, name):
        self._a(name)[:] = (1.0 / self.op.diagonal()).ravel()

    def apply64(self, x, y):
        self._a(y)[:] = self.op.apply(self._a(x).reshape(self.shape)).ravel()

    def sweep(self, x_in, f, x_out, order):
        x = np.zeros(self.shape) if x_in is None else self._a(x_in).reshape(self.shape)
        self._a(x_out)[:] = OM.sweep(self.levels[0], x, self._a(f).reshape(self.shape), "RB" if order == 0 else
                                     "BR").ravel()

    def pack(self, name, nplanes):
        g, a = self.geo, self._a(name)
        buf = np.zeros(2 * nplanes * g.plane)
        h = nplanes * g.plane
        if g.lo_rank is not None:
            buf[:h] = a[g.glo * g.plane:(g.glo + nplanes) * g.plane]
        if g.hi_rank is not None:
            buf[h:] = a[(g.glo + g.nz_loc - nplanes) * g.plane:(g.glo + g.nz_loc) * g.plane]
        return torch.from_numpy(buf)

    def unpack(self, name, buf, nplanes):
        g, a, b = self.geo, self._a(name), buf.numpy()
        h = nplanes * g.plane
        if g.lo_rank is not None:
            a[(g.glo - nplanes) * g.plane:g.glo * g.plane] = b[:h]
        if g.hi_rank is not None:
            a[(g.glo + g.nz_loc) * g.plane:(g.glo + g.nz_loc + nplanes) * g.plane] = b[h:]

    def coarse_shape(self):
        L1 = self.levels[1]
        return (L1.shape[2], L1.shape[1], L1.shape[0])

    def _own_coarse(self, a1):
        g = self.geo
        c0 = g.glo // 2
        return torch.from_numpy(np.ascontiguousarray(a1[c0:c0 + g.nz_loc // 2]).ravel())

    def coarse_coefficients(self):
        L1 = self.levels[1]
        return self._own_coarse(L1.ct), self._own_coarse(L1.rho)

    def restrict_residual(self, x, f):
        L0 = self.levels[0]
        r = self._a(f).reshape(self.shape) - L0.op.apply(self._a(x).reshape(self.shape))
        return self._own_coarse(OM.restrict(r, L0.halved))

    def prolong_add(self, ec_mine, x):
        L0, L1 = self.levels[0], self.levels[1]
        ec = ec_mine.numpy().reshape(L1.shape)
        self._a(x)[:] += OM.prolong(ec, L0.halved).ravel()

    def take_planes(self, flat, planes, plane_size):
        return flat.reshape(-1, plane_size)[list(planes)].reshape(-1).clone()

    def coarse_solver(self, n, h, bc, ct_parts, rho_parts):
        shape = (n[2], n[1], n[0])
        ct = torch.cat(ct_parts).numpy().reshape(shape)
        rho = torch.cat(rho_parts).numpy().reshape(shape)
        levels = OM.build_hierarchy(ct, rho, h, bc)

        class C:
            def vcycle(self, parts, nu1, nu2):
                r = torch.cat(parts).numpy().reshape(shape)
                return torch.from_numpy(OM.vcycle(levels, r, nu1=nu1, nu2=nu2).ravel())
        return C()

    def solution(self):
        return self._a("x")[self.o0:self.o1]


PROBLEMS = {
    "conv3d-8x8x16-zwall": lambda: I.make_problem(8, 16, 8, ma=0.05, contrast=10.0, noise=0.01, seed=31),
    "conv3d-8x4x24-zper": lambda: I.make_problem(8, 24, 4, ma=0.05, contrast=6.0, noise=0.01, seed=32,
                                                 bc=(PER, PER, PER)),
    "plain2d-16x32": lambda: I.make_problem(16, 32, ma=0.1, contrast=8.0, noise=0.01, seed=33),
}


def run_threads(world, fn):
    """Run fn(rank, comm) on `world` threads; return their results by rank."""
    import threading
    comms = S.ThreadComm.group(world)
    out, err = [None] * world, []

    def body(r):
        try:
            out[r] = fn(r, comms[r])
        except BaseException as e:          # noqa: BLE001 - reported below
            err.append(e)
            comms[r].s["barrier"].abort()
    ts = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if err:
        raise err[0]
    return out


def gather_owned(results, geos):
    return np.concatenate([results[r] for r in range(len(geos))])


# ------------------------------------------------------------------ pure logic
def test_slab_bounds():
    assert S.slab_bounds(16, 2) == [(0, 8), (8, 16)]
    b = S.slab_bounds(30, 4)
    assert b[0][0] == 0 and b[-1][1] == 30 and all(z0 % 2 == 0 and z1 % 2 == 0 for z0, z1 in b)
    assert all(b[i][1] == b[i + 1][0] for i in range(3))
    assert max(z1 - z0 for z0, z1 in b) - min(z1 - z0 for z0, z1 in b) <= 2
    with pytest.raises(ValueError):
        S.slab_bounds(15, 2)
    with pytest.raises(ValueError):
        S.slab_bounds(8, 8)


def test_geometry_ghosts_and_neighbours():
    wall = [S.SlabGeometry((8, 8, 24), (1, 1, 1), (PER, PER, NEU), r, 3) for r in range(3)]
    assert [(g.lo_rank, g.hi_rank) for g in wall] == [(None, 1), (0, 2), (1, None)]
    assert [(g.glo, g.ghi) for g in wall] == [(0, 2), (2, 2), (2, 0)]
    per = [S.SlabGeometry((8, 8, 24), (1, 1, 1), (PER, PER, PER), r, 2) for r in range(2)]
    assert [(g.lo_rank, g.hi_rank) for g in per] == [(1, 1), (0, 0)]
    assert per[0].ext_planes()[:2] == [22, 23] and per[0].ext_planes()[-2:] == [12, 13]
    one = S.SlabGeometry((4, 4, 8), (1, 1, 1), (PER, PER, PER), 0, 1)
    assert (one.lo_rank, one.hi_rank, one.nz_ext) == (0, 0, 12)


# ------------------------------------------------------------------ threads
@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("world", [1, 2, 3])
def test_distributed_apply_and_sweep_match_single_domain(name, world):
    """One exchange then the float64 apply, and two-plane exchanges around a
    red-black sweep pair: the owned planes equal the single-domain oracle's."""
    p = PROBLEMS[name]()
    if p.n[2] // world < 2 * S.GHOST // 2 or p.n[2] % 2:
        pytest.skip("too few planes")
    op = P.operator_from_problem(p)
    L0 = OM.build_hierarchy(op.ct, p.rho_new, p.h, p.bc)[0]
    rng = np.random.default_rng(5)
    x = rng.standard_normal(p.shape3)
    y_ref = op.apply(x).ravel()
    s_ref = OM.sweep(L0, OM.sweep(L0, x, p.f.reshape(p.shape3), "RB"), p.f.reshape(p.shape3), "BR").ravel()

    def rank(r, comm):
        geo = S.SlabGeometry(p.n, p.h, p.bc, r, world)
        ops = NumpySlab(geo, p)
        ops.zeros("x", "f64"), ops.zeros("y", "f64"), ops.zeros("f", "f64"), ops.zeros("a", "f64")
        ops.v["x"][ops.o0:ops.o1] = torch.from_numpy(geo.extract(x).ravel()[ops.o0:ops.o1])
        ops.set_rhs("f")
        S.exchange(ops, comm, "x", 1)
        ops.apply64("x", "y")
        y = ops.v["y"][ops.o0:ops.o1].numpy().copy()
        S.exchange(ops, comm, "f", S.GHOST)
        S.exchange(ops, comm, "x", S.GHOST)
        ops.sweep("x", "f", "a", 0)
        S.exchange(ops, comm, "a", S.GHOST)
        ops.sweep("a", "f", "y", 1)
        return y, ops.v["y"][ops.o0:ops.o1].numpy().copy()

    res = run_threads(world, rank)
    y = np.concatenate([r[0] for r in res])
    sw = np.concatenate([r[1] for r in res])
    assert np.allclose(y, y_ref, rtol=0, atol=1e-13 * np.abs(y_ref).max())
    assert np.allclose(sw, s_ref, rtol=0, atol=1e-13 * np.abs(s_ref).max())


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("world", [1, 2, 3])
def test_distributed_vcycle_matches_single_domain(name, world):
    """The distributed V-cycle (levels >= 1 agglomerated on rank 0) equals
    the oracle's single-domain V-cycle."""
    p = PROBLEMS[name]()
    op = P.operator_from_problem(p)
    levels = OM.build_hierarchy(op.ct, p.rho_new, p.h, p.bc)
    rng = np.random.default_rng(6)
    r0 = rng.standard_normal(p.shape3)
    z_ref = OM.vcycle(levels, r0, nu1=2, nu2=2).ravel()

    def rank(r, comm):
        geo = S.SlabGeometry(p.n, p.h, p.bc, r, world)
        q = dataclasses.replace(p, f=r0)
        ops = NumpySlab(geo, q)
        for v in ("r32", "z32", "xa", "xb"):
            ops.zeros(v, "f32")
        ops.set_rhs("r32")
        coarse = S.CoarseLevel(ops, comm)
        S.vcycle(ops, comm, coarse, "r32", "z32", 2, 2)
        return ops.v["z32"][ops.o0:ops.o1].numpy().copy()

    z = np.concatenate(run_threads(world, rank))
    assert np.allclose(z, z_ref, rtol=0, atol=1e-12 * np.abs(z_ref).max())


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("world", [2, 3])
def test_distributed_solvers_match_direct_solve(name, world):
    """Jacobi-PCG and multigrid-preconditioned flexible CG, distributed, reach
    the oracle's direct solution to 1e-10 (the float64 bar); PCG's residual
    history follows the single-domain oracle's for its first iterations."""
    p = PROBLEMS[name]()
    op = P.operator_from_problem(p)
    xs = P.solve_direct(op, p.f).ravel()
    _, _, h_ref = P.solve_pcg_jacobi(op, p.f, rtol=1e-14, maxiter=20000)

    def rank(r, comm):
        geo = S.SlabGeometry(p.n, p.h, p.bc, r, world)
        ops = NumpySlab(geo, p)
        k, hist = S.pcg_jacobi(ops, comm, rtol=1e-13, max_iter=20000)
        x1 = ops.solution().copy()
        rel1 = S.true_residual(ops, comm)
        k2, hist2 = S.mg_fcg(ops, comm, rtol=1e-13, max_iter=200)
        x2 = ops.solution().copy()
        rel2 = S.true_residual(ops, comm)
        return x1, hist, rel1, x2, k2, rel2

    res = run_threads(world, rank)
    x1 = np.concatenate([r[0] for r in res])
    x2 = np.concatenate([r[3] for r in res])
    hist = res[0][1]
    m = min(20, len(hist), len(h_ref))
    np.testing.assert_allclose(hist[:m], h_ref[:m], rtol=1e-8)
    for x, rel in ((x1, res[0][2]), (x2, res[0][5])):
        assert rel <= 2e-13
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    assert res[0][4] <= 30


# ------------------------------------------------------------------ gloo processes
def _gloo_rank(rank, world, port, name, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = PROBLEMS[name]()
        comm = S.TorchComm()
        geo = S.SlabGeometry(p.n, p.h, p.bc, rank, world)
        ops = NumpySlab(geo, p)
        k, hist = S.pcg_jacobi(ops, comm, rtol=1e-13, max_iter=20000)
        x1 = ops.solution().copy()
        k2, _ = S.mg_fcg(ops, comm, rtol=1e-13, max_iter=200)
        x2 = ops.solution().copy()
        rel2 = S.true_residual(ops, comm)
        q.put((rank, x1, x2, k2, rel2, hist[:20]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["conv3d-8x8x16-zwall", "conv3d-8x4x24-zper"])
def test_gloo_two_ranks(name):
    """Two gloo processes (TorchComm): distributed PCG and MG-FCG vs the oracle."""
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, name, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = sorted([q.get(timeout=300) for _ in range(2)], key=lambda t: t[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = PROBLEMS[name]()
    op = P.operator_from_problem(p)
    xs = P.solve_direct(op, p.f).ravel()
    _, _, h_ref = P.solve_pcg_jacobi(op, p.f, rtol=1e-14, maxiter=20000)
    x1 = np.concatenate([g[1] for g in got])
    x2 = np.concatenate([g[2] for g in got])
    np.testing.assert_allclose(got[0][5], h_ref[:len(got[0][5])], rtol=1e-8)
    assert np.linalg.norm(x1 - xs) <= 1e-10 * np.linalg.norm(xs)
    assert np.linalg.norm(x2 - xs) <= 1e-10 * np.linalg.norm(xs)
    assert got[0][4] <= 2e-13
