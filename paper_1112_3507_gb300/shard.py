"""The pressure solve decomposed into z slabs, one rank per GPU.

The paper solves its generalized Poisson equation in parallel on a CPU
cluster (Sec. 2.5, the parallel solver and its strong-scaling table).  Here
the same equation is split along z across ranks (one process per GPU):

  slabs      rank r of W owns the planes [z0, z1) of the global grid
             (slab_bounds: even boundaries, sizes as equal as they can be),
             stored as an extended local grid with GHOST planes on every
             side that has a neighbour (periodic z: both sides; a Neumann
             wall: none past it).  The local grid has a wall in z, and its
             wall faces touch ghost planes only.
  apply      y = A x on the owned planes needs one ghost plane of x from each
             neighbour: one halo exchange per operator application.
  sweep      a red-black Gauss-Seidel sweep on the extended grid gives the
             right owned values when two ghost planes of x are current: the
             first-colour values of the inner ghost plane are recomputed
             locally from the outer one (the neighbour computes the same
             values for its own cells).  One exchange of two planes per
             sweep.
  Krylov     float64 dot products are summed over the owned planes and then
             over ranks: an all-reduce of two or three scalars per
             iteration.
  multigrid  levels 0 -> 1 of the V-cycle run distributed (pre-sweeps,
             residual + restriction); the level-1 right-hand side (1/8 of
             the cells in 3D) is gathered to rank 0, which runs the rest of
             the V-cycle on the whole level-1 grid, and scatters the
             correction back (each rank gets its coarse planes plus one
             coarse ghost plane per neighbour) for the prolongation and the
             post-sweeps.  The arithmetic is that of the single-domain
             V-cycle; only the order of the cross-rank sums differs.

The driver below is host logic only: it sequences a per-rank backend (the
GPU one, GpuSlab, calls the library's C ABI on device tensors) and a
communicator (TorchComm over torch.distributed -- NCCL between GPUs, gloo
between CPU processes -- or ThreadComm for ranks that are threads of one
process).  Every arithmetic step on grid data runs in the backend.
"""
from __future__ import annotations

import math
import threading

import numpy as np

GHOST = 2
PERIODIC, NEUMANN = 0, 1


# ------------------------------------------------------------------ geometry
def slab_bounds(nz: int, world: int, align: int = 2):
    """[(z0, z1)] of each rank: boundaries multiples of `align` (so that the
    red-black colouring and the level-1 halving agree across ranks), slab
    sizes differing by at most `align` planes.  Every slab must hold at
    least GHOST planes."""
    if nz % align:
        raise ValueError(f"nz = {nz} is not a multiple of {align}")
    units = nz // align
    if units < world or (nz // world) < GHOST:
        raise ValueError(f"{nz} planes cannot be split over {world} ranks")
    out, z = [], 0
    for r in range(world):
        u = units // world + (1 if r < units % world else 0)
        out.append((z, z + u * align))
        z += u * align
    return out


class SlabGeometry:
    """The global grid (n = (nx, ny, nz), spacings h, boundary conditions bc)
    and rank `rank`'s slab of it."""

    def __init__(self, n, h, bc, rank: int, world: int):
        self.n, self.h, self.bc = tuple(int(v) for v in n), tuple(float(v) for v in h), tuple(int(b) for b in bc)
        self.rank, self.world = rank, world
        self.bounds = slab_bounds(self.n[2], world)
        self.z0, self.z1 = self.bounds[rank]
        self.nz_loc = self.z1 - self.z0
        per = self.bc[2] == PERIODIC
        self.lo_rank = (rank - 1) % world if (rank > 0 or per) else None
        self.hi_rank = (rank + 1) % world if (rank < world - 1 or per) else None
        self.glo = GHOST if self.lo_rank is not None else 0
        self.ghi = GHOST if self.hi_rank is not None else 0
        self.nz_ext = self.nz_loc + self.glo + self.ghi
        self.plane = self.n[0] * self.n[1]
        self.n_ext = (self.n[0], self.n[1], self.nz_ext)
        self.bc_ext = (self.bc[0], self.bc[1], NEUMANN)

    @property
    def owned_cells(self) -> int:
        return self.plane * self.nz_loc

    def ext_planes(self):
        """Global plane index of every local plane (wrapped on a periodic z)."""
        return [(self.z0 - self.glo + k) % self.n[2] for k in range(self.nz_ext)]

    def extract(self, a):
        """The extended local part of a global (nz, ny, nx) array."""
        return np.ascontiguousarray(np.asarray(a)[self.ext_planes()])


# ------------------------------------------------------------------ communicators
class TorchComm:
    """Halo exchange, all-reduce, gather and scatter over torch.distributed
    (an initialised process group; NCCL with device tensors, gloo with host
    tensors -- device tensors are staged through host memory for gloo)."""

    TAG_DOWN, TAG_UP, TAG_GATHER, TAG_SCATTER = 1, 2, 3, 4

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.host = dist.get_backend() == "gloo"

    def _wire(self, t):
        return t.cpu() if (self.host and t.is_cuda) else t

    def exchange(self, geo: SlabGeometry, send_lo, send_hi, recv_lo, recv_hi):
        """send_lo (my bottom owned planes) goes to my lower neighbour's top
        ghost, send_hi to my upper neighbour's bottom ghost; recv_lo / recv_hi
        receive my bottom / top ghosts (in place).  Sends to one peer are
        posted [down, up] and receives from one peer [from above, from
        below], so that the two lists match in order even when both
        neighbours are the same rank."""
        if self.world == 1:
            if geo.lo_rank is not None:
                recv_lo.copy_(send_hi)
                recv_hi.copy_(send_lo)
            return
        P = self.dist.P2POp
        sl, sh = self._wire(send_lo), self._wire(send_hi)
        rl = self._wire(recv_lo) if geo.lo_rank is not None else None
        rh = self._wire(recv_hi) if geo.hi_rank is not None else None
        ops = []
        if geo.lo_rank is not None:
            ops.append(P(self.dist.isend, sl, geo.lo_rank, tag=self.TAG_DOWN))
        if geo.hi_rank is not None:
            ops.append(P(self.dist.isend, sh, geo.hi_rank, tag=self.TAG_UP))
        if geo.hi_rank is not None:
            ops.append(P(self.dist.irecv, rh, geo.hi_rank, tag=self.TAG_DOWN))
        if geo.lo_rank is not None:
            ops.append(P(self.dist.irecv, rl, geo.lo_rank, tag=self.TAG_UP))
        for w in self.dist.batch_isend_irecv(ops):
            w.wait()
        if rl is not None and rl is not recv_lo:
            recv_lo.copy_(rl)
        if rh is not None and rh is not recv_hi:
            recv_hi.copy_(rh)

    def allreduce(self, values, like):
        """Sum over ranks of a few float64 scalars (a tensor on `like`'s device, or host for gloo)."""
        import torch
        dev = "cpu" if (self.host or not like.is_cuda) else like.device
        t = torch.tensor(values, dtype=torch.float64, device=dev)
        self.dist.all_reduce(t)
        return [float(v) for v in t.tolist()]

    def gather0(self, geo: SlabGeometry, part, parts_out):
        """Rank 0 receives every rank's `part` into parts_out[r] (rank 0's own copied)."""
        if self.rank == 0:
            parts_out[0].copy_(part)
            for r in range(1, self.world):
                buf = self._wire(parts_out[r])
                self.dist.recv(buf, r, tag=self.TAG_GATHER)
                if buf is not parts_out[r]:
                    parts_out[r].copy_(buf)
        else:
            self.dist.send(self._wire(part), 0, tag=self.TAG_GATHER)

    def scatter0(self, geo: SlabGeometry, parts_in, mine):
        """Rank r receives parts_in[r] from rank 0 into `mine`."""
        if self.rank == 0:
            for r in range(1, self.world):
                self.dist.send(self._wire(parts_in[r]), r, tag=self.TAG_SCATTER)
            mine.copy_(parts_in[0])
        else:
            buf = self._wire(mine)
            self.dist.recv(buf, 0, tag=self.TAG_SCATTER)
            if buf is not mine:
                mine.copy_(buf)


class ThreadComm:
    """The same operations for ranks that are threads of one process (one
    ThreadComm per rank, built by ThreadComm.group): buffers are handed over
    through shared slots between barriers; sums run in rank order."""

    def __init__(self, rank, world, shared):
        self.rank, self.world, self.s = rank, world, shared

    @classmethod
    def group(cls, world: int):
        shared = {"barrier": threading.Barrier(world), "slots": [None] * world}
        return [cls(r, world, shared) for r in range(world)]

    def _sync(self):
        self.s["barrier"].wait(timeout=120)

    def exchange(self, geo, send_lo, send_hi, recv_lo, recv_hi):
        self.s["slots"][self.rank] = (send_lo, send_hi)
        self._sync()
        if geo.lo_rank is not None:
            recv_lo.copy_(self.s["slots"][geo.lo_rank][1])       # lower neighbour's top owned planes
        if geo.hi_rank is not None:
            recv_hi.copy_(self.s["slots"][geo.hi_rank][0])       # upper neighbour's bottom owned planes
        self._sync()

    def allreduce(self, values, like=None):
        self.s["slots"][self.rank] = list(values)
        self._sync()
        tot = [0.0] * len(values)
        for r in range(self.world):
            tot = [a + b for a, b in zip(tot, self.s["slots"][r])]
        self._sync()
        return tot

    def gather0(self, geo, part, parts_out):
        self.s["slots"][self.rank] = part
        self._sync()
        if self.rank == 0:
            for r in range(self.world):
                parts_out[r].copy_(self.s["slots"][r])
        self._sync()

    def scatter0(self, geo, parts_in, mine):
        if self.rank == 0:
            self.s["slots"][0] = parts_in
        self._sync()
        mine.copy_(self.s["slots"][0][self.rank])
        self._sync()


# ------------------------------------------------------------------ halo exchange
def exchange(ops, comm, name: str, nplanes: int):
    """Refresh `nplanes` ghost planes of vector `name` on every side with a neighbour."""
    g = ops.geo
    if g.lo_rank is None and g.hi_rank is None:
        return
    buf = ops.pack(name, nplanes)                  # [bottom owned planes | top owned planes]
    recv = ops.empty_like_buf(buf)
    half = buf.numel() // 2
    comm.exchange(g, buf[:half], buf[half:], recv[:half], recv[half:])
    ops.unpack(name, recv, nplanes)


# ------------------------------------------------------------------ solvers
def pcg_jacobi(ops, comm, rtol: float = 1e-8, max_iter: int = 10000):
    """Float64 conjugate gradients with the Jacobi preconditioner (the plain
    PCG of Sec. 2.5 with diag(A) for incomplete Cholesky), distributed: one
    one-plane exchange and two all-reduces per iteration.  Returns
    (iterations, relative residual history); the solution is ops' "x"."""
    for v in ("x", "r", "p", "q", "z", "dinv"):
        ops.zeros(v, "f64")
    ops.set_rhs("r")
    ops.jacobi_dinv("dinv")
    ops.mul("dinv", "r", "z")
    ops.axpby(1.0, "z", 0.0, None, "p")
    rr, rz, ff = comm.allreduce([ops.dot("r", "r"), ops.dot("r", "z"), ops.dot("r", "r")], ops.like())
    fnorm = math.sqrt(ff)
    hist = [math.sqrt(rr) / fnorm if fnorm > 0 else 0.0]
    k = 0
    while hist[-1] > rtol and k < max_iter:
        exchange(ops, comm, "p", 1)
        ops.apply64("p", "q")
        (pq,) = comm.allreduce([ops.dot("p", "q")], ops.like())
        if not (pq > 0.0) or not math.isfinite(pq):
            raise FloatingPointError("Krylov breakdown: p^T A p <= 0")
        alpha = rz / pq
        ops.axpby(alpha, "p", 1.0, "x", "x")
        ops.axpby(-alpha, "q", 1.0, "r", "r")
        ops.mul("dinv", "r", "z")
        rr, rz_new = comm.allreduce([ops.dot("r", "r"), ops.dot("r", "z")], ops.like())
        k += 1
        hist.append(math.sqrt(rr) / fnorm)
        ops.axpby(1.0, "z", rz_new / rz, "p", "p")
        rz = rz_new
    return k, hist


def _pow2_near_inv(v: float) -> float:
    if not (v > 0.0) or not math.isfinite(v):
        return 1.0
    return 2.0 ** max(-100, min(100, -round(math.log2(v))))


class CoarseLevel:
    """The level-1 grid of the global hierarchy, agglomerated on rank 0:
    shapes of every rank's owned coarse planes, and rank 0's solver."""

    def __init__(self, ops, comm):
        g = ops.geo
        self.per = g.bc[2] == PERIODIC
        nc = ops.coarse_shape()                       # level 1 of the extended local grid
        if nc[2] * 2 != g.nz_ext:
            raise ValueError("the level-1 hierarchy does not halve z: no slab multigrid")
        self.n = (nc[0], nc[1], g.n[2] // 2)
        self.h = tuple(g.h[a] * (g.n[a] // self.n[a]) for a in range(3))
        self.cplane = nc[0] * nc[1]
        self.bounds = [(z0 // 2, z1 // 2) for z0, z1 in g.bounds]
        c0, c1 = self.bounds[g.rank]
        self.own = (c0, c1)
        self.glo_c, self.ghi_c = g.glo // 2, g.ghi // 2      # coarse ghost planes (1 where a neighbour exists)
        ct, rho = ops.coarse_coefficients()
        parts = [ops.buf_f64(self.cplane * (b1 - b0)) for b0, b1 in self.bounds] if g.rank == 0 else None
        parts_r = [ops.buf_f64(self.cplane * (b1 - b0)) for b0, b1 in self.bounds] if g.rank == 0 else None
        comm.gather0(g, ct, parts)
        comm.gather0(g, rho, parts_r)
        self.solver = ops.coarse_solver(self.n, self.h, g.bc, parts, parts_r) if g.rank == 0 else None

    def ext_planes(self, r):
        """Global coarse planes rank r receives: its own plus one ghost plane per neighbour side."""
        (c0, c1) = self.bounds[r]
        nzc = self.n[2]
        lo = 1 if (r > 0 or self.per) else 0
        hi = 1 if (r < len(self.bounds) - 1 or self.per) else 0
        return [(c0 - lo + k) % nzc for k in range(c1 - c0 + lo + hi)]


def vcycle(ops, comm, coarse: CoarseLevel, f: str, out: str, nu1: int, nu2: int):
    """z = M f for the float32 vector `f`, written to `out`: the single-domain
    V-cycle's arithmetic with the halo exchanges of the slab layout and the
    levels below 0 agglomerated on rank 0."""
    g = ops.geo
    exchange(ops, comm, f, GHOST)                    # f on the inner ghost plane (first-colour updates there)
    cur, other = "xa", "xb"
    ops.sweep(None, f, cur, 0)
    for _ in range(nu1 - 1):
        exchange(ops, comm, cur, GHOST)
        ops.sweep(cur, f, other, 0)
        cur, other = other, cur
    exchange(ops, comm, cur, GHOST)                  # x ghosts for the residual and the prolonged sweeps
    fc = ops.restrict_residual(cur, f)               # owned coarse planes
    world = g.world
    if g.rank == 0:
        parts = [ops.buf_f32(coarse.cplane * (b1 - b0)) for b0, b1 in coarse.bounds]
    else:
        parts = None
    comm.gather0(g, fc, parts)
    mine = ops.buf_f32(coarse.cplane * len(coarse.ext_planes(g.rank)))
    if g.rank == 0:
        zc = coarse.solver.vcycle(parts, nu1, nu2)   # the global level-1 correction (flat, float32)
        sends = [ops.take_planes(zc, coarse.ext_planes(r), coarse.cplane) for r in range(world)]
    else:
        sends = None
    comm.scatter0(g, sends, mine)
    ops.prolong_add(mine, cur)                       # x += P ec on every local plane, ghosts included
    for it in range(nu2):
        dst = out if it == nu2 - 1 else other
        ops.sweep(cur, f, dst, 1)
        if it < nu2 - 1:
            exchange(ops, comm, dst, GHOST)
            cur, other = dst, cur


def mg_fcg(ops, comm, rtol: float = 1e-8, max_iter: int = 500, nu1: int = 2, nu2: int = 2):
    """Float64 flexible conjugate gradients preconditioned by the float32
    V-cycle (the library's LM_FP64_MG_PCG mode), distributed: per iteration
    one V-cycle (its exchanges, one gather and one scatter of the level-1
    vectors), one one-plane exchange of p for A p, and three all-reduces
    (z.q_old; p.q and p.r; r.r).  Returns (iterations, history); solution in
    ops' "x"."""
    g = ops.geo
    for v in ("x", "r", "p", "q"):
        ops.zeros(v, "f64")
    for v in ("r32", "z32", "xa", "xb"):
        ops.zeros(v, "f32")
    ops.set_rhs("r")
    coarse = CoarseLevel(ops, comm)
    (ff,) = comm.allreduce([ops.dot("r", "r")], ops.like())
    fnorm = math.sqrt(ff)
    hist = [1.0 if fnorm > 0 else 0.0]
    N = g.n[0] * g.n[1] * g.n[2]
    rs = _pow2_near_inv(fnorm / math.sqrt(N))
    ops.axpby(rs, "r", 0.0, None, "r32")
    pq_old, k = 0.0, 0
    while hist[-1] > rtol and k < max_iter:
        vcycle(ops, comm, coarse, "r32", "z32", nu1, nu2)
        if k == 0:
            ops.axpby(1.0, "z32", 0.0, None, "p")
        else:
            (zq,) = comm.allreduce([ops.dot("z32", "q")], ops.like())
            ops.axpby(1.0, "z32", -zq / pq_old, "p", "p")
        exchange(ops, comm, "p", 1)
        ops.apply64("p", "q")
        pq, pr = comm.allreduce([ops.dot("p", "q"), ops.dot("p", "r")], ops.like())
        if not (pq > 0.0) or not math.isfinite(pq):
            raise FloatingPointError("Krylov breakdown: p^T A p <= 0")
        alpha = pr / pq
        ops.axpby(alpha, "p", 1.0, "x", "x")
        ops.axpby(-alpha, "q", 1.0, "r", "r")
        (rr,) = comm.allreduce([ops.dot("r", "r")], ops.like())
        k += 1
        hist.append(math.sqrt(rr) / fnorm)
        rs = _pow2_near_inv(math.sqrt(rr / N))
        ops.axpby(rs, "r", 0.0, None, "r32")
        pq_old = pq
    return k, hist


def true_residual(ops, comm) -> float:
    """||f - A x|| / ||f|| of ops' "x", recomputed (one exchange, one all-reduce)."""
    ops.zeros("t", "f64")
    ops.zeros("fr", "f64")
    ops.set_rhs("fr")
    exchange(ops, comm, "x", 1)
    ops.apply64("x", "t")
    ops.axpby(1.0, "fr", -1.0, "t", "t")
    rr, ff = comm.allreduce([ops.dot("t", "t"), ops.dot("fr", "fr")], ops.like())
    return math.sqrt(rr / ff) if ff > 0 else 0.0


# ------------------------------------------------------------------ GPU backend
class GpuSlab:
    """The per-rank backend on this process's GPU: the extended local grid
    as an lm_grid, vectors as device tensors of the extended size, every
    step one call of the library's C ABI on the given stream."""

    def __init__(self, geo: SlabGeometry, rho_old, rho_new, cs2, dt, f, device=None, stream=None):
        import torch

        from . import lowmach as lm
        self.torch, self.lm, self.geo = torch, lm, geo
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        self.N = geo.plane * geo.nz_ext
        self.grid = lm.Grid(geo.n_ext, geo.h, geo.bc_ext, ndim=3 if geo.n[1] > 1 else 2)
        ext = [torch.as_tensor(geo.extract(a).ravel(), dtype=torch.float64, device=self.dev)
               for a in (rho_old, rho_new, cs2)]
        self.grid.set_coefficients(ext[0], ext[1], ext[2], dt, self._s())
        self.f_ext = torch.as_tensor(geo.extract(f).ravel(), dtype=torch.float64, device=self.dev)
        self.v = {}
        self.scratch = torch.empty(1025, dtype=torch.float64, device=self.dev)
        self.o0, self.o1 = geo.glo * geo.plane, (geo.glo + geo.nz_loc) * geo.plane

    def _s(self):
        return self.stream

    def _sp(self):
        return self.lm._stream_ptr(self.stream)

    def _ptr(self, t, offset=0):
        import ctypes
        return ctypes.c_void_p(t.data_ptr() + offset * t.element_size())

    def _prec(self, t):
        return self.lm.PREC_FP64 if t.dtype == self.torch.float64 else self.lm.PREC_FP32

    def like(self):
        return self.f_ext

    def zeros(self, name, prec):
        dt = self.torch.float64 if prec == "f64" else self.torch.float32
        self.v[name] = self.torch.zeros(self.N, dtype=dt, device=self.dev)

    def buf_f32(self, n):
        return self.torch.zeros(n, dtype=self.torch.float32, device=self.dev)

    def buf_f64(self, n):
        return self.torch.zeros(n, dtype=self.torch.float64, device=self.dev)

    def empty_like_buf(self, b):
        return self.torch.zeros_like(b)

    def set_rhs(self, name):
        t = self.v[name]
        t.zero_()
        self._axpby_range(1.0, self.f_ext, 0.0, None, t)

    def _axpby_range(self, a, x, b, y, out):
        n = self.o1 - self.o0
        L = self.lm
        L._check(L.lib().lm_vec_axpby(n, a, self._ptr(x, self.o0), self._prec(x), b,
                                      self._ptr(y, self.o0) if y is not None else None,
                                      self._prec(y) if y is not None else 0, self._ptr(out, self.o0),
                                      self._prec(out), self._sp()), "lm_vec_axpby")

    def axpby(self, a, x, b, y, out):
        self._axpby_range(a, self.v[x], b, self.v[y] if y is not None else None, self.v[out])

    def mul(self, d, r, z):
        n = self.o1 - self.o0
        L = self.lm
        L._check(L.lib().lm_vec_mul(n, self._ptr(self.v[d], self.o0), self._ptr(self.v[r], self.o0),
                                    self._ptr(self.v[z], self.o0), self._sp()), "lm_vec_mul")

    def dot(self, a, b):
        import ctypes
        ta, tb = self.v[a], self.v[b]
        out = ctypes.c_double(0.0)
        L = self.lm
        L._check(L.lib().lm_vec_dot(self.o1 - self.o0, self._ptr(ta, self.o0), self._prec(ta), self._ptr(tb, self.o0),
                                    self._prec(tb), self._ptr(self.scratch), ctypes.byref(out), self._sp()),
                 "lm_vec_dot")
        return out.value

    def jacobi_dinv(self, name):
        L = self.lm
        L._check(L.lib().lm_jacobi_inverse_diagonal(self.grid._g, self._ptr(self.v[name]), self._sp()),
                 "lm_jacobi_inverse_diagonal")

    def apply64(self, x, y):
        self.grid.apply(self.v[x], self.v[y], prec=self.lm.PREC_FP64, stream=self.stream)

    def sweep(self, x_in, f, x_out, order):
        self.grid.mg_sweep(self.v[x_in] if x_in is not None else None, self.v[f], self.v[x_out], order,
                           stream=self.stream)

    def pack(self, name, nplanes):
        g, t = self.geo, self.v[name]
        buf = self.torch.zeros(2 * nplanes * g.plane, dtype=t.dtype, device=self.dev)
        lo = g.glo if g.lo_rank is not None else -1
        hi = g.glo + g.nz_loc - nplanes if g.hi_rank is not None else -1
        L = self.lm
        L._check(L.lib().lm_halo_pack(self._ptr(t), t.element_size(), g.plane, lo, hi, nplanes, self._ptr(buf), 0,
                                      self._sp()), "lm_halo_pack")
        return buf

    def unpack(self, name, buf, nplanes):
        g, t = self.geo, self.v[name]
        lo = g.glo - nplanes if g.lo_rank is not None else -1
        hi = g.glo + g.nz_loc if g.hi_rank is not None else -1
        L = self.lm
        L._check(L.lib().lm_halo_pack(self._ptr(t), t.element_size(), g.plane, lo, hi, nplanes, self._ptr(buf), 1,
                                      self._sp()), "lm_halo_pack")

    def coarse_shape(self):
        return self.grid.mg_levels()[1]

    def _coarse_ext_sizes(self):
        nc = self.coarse_shape()
        return nc[0] * nc[1], nc[0] * nc[1] * nc[2]

    def coarse_coefficients(self):
        """This rank's owned coarse planes of level-1 c~ and rho (float64, true rho)."""
        import ctypes
        cplane, ncell = self._coarse_ext_sizes()
        ct = self.torch.empty(ncell, dtype=self.torch.float32, device=self.dev)
        rho = self.torch.empty_like(ct)
        scale = ctypes.c_double(1.0)
        L = self.lm
        L._check(L.lib().lm_mg_level_coefficients(self.grid._g, 1, self._ptr(ct), self._ptr(rho),
                                                  ctypes.byref(scale), self._sp()), "lm_mg_level_coefficients")
        a, b = (self.geo.glo // 2) * cplane, (self.geo.glo // 2 + self.geo.nz_loc // 2) * cplane
        return ct[a:b].double(), rho[a:b].double() * scale.value

    def restrict_residual(self, x, f):
        cplane, ncell = self._coarse_ext_sizes()
        fc = self.torch.empty(ncell, dtype=self.torch.float32, device=self.dev)
        L = self.lm
        L._check(L.lib().lm_mg_restrict_residual(self.grid._g, self._ptr(self.v[x]), self._ptr(self.v[f]),
                                                 self._ptr(fc), self._sp()), "lm_mg_restrict_residual")
        a = (self.geo.glo // 2) * cplane
        return fc[a:a + (self.geo.nz_loc // 2) * cplane].contiguous()

    def prolong_add(self, ec_mine, x):
        """ec_mine: this rank's coarse planes plus its coarse ghost planes;
        laid into a level-1 vector of the extended grid, then x += P ec."""
        cplane, ncell = self._coarse_ext_sizes()
        ec = self.torch.zeros(ncell, dtype=self.torch.float32, device=self.dev)
        ec[: ec_mine.numel()].copy_(ec_mine)
        L = self.lm
        L._check(L.lib().lm_mg_prolong_add(self.grid._g, self._ptr(ec), self._ptr(self.v[x]), self._sp()),
                 "lm_mg_prolong_add")

    def take_planes(self, flat, planes, plane_size):
        idx = self.torch.as_tensor(planes, device=flat.device)
        return flat.view(-1, plane_size)[idx].reshape(-1).contiguous()

    def coarse_solver(self, n, h, bc, ct_parts, rho_parts):
        return _GpuCoarse(self, n, h, bc, self.torch.cat(ct_parts), self.torch.cat(rho_parts))

    def solution(self):
        return self.v["x"][self.o0:self.o1]

    def close(self):
        self.grid.close()


class _GpuCoarse:
    """Rank 0's level-1 grid: an lm_grid with the gathered float32
    coefficients (as float64, exactly) and its own V-cycle."""

    def __init__(self, ops, n, h, bc, ct, rho):
        lm, torch = ops.lm, ops.torch
        self.ops = ops
        self.grid = lm.Grid(n, h, bc, ndim=3 if n[1] > 1 else 2)
        self.grid.set_coefficients_raw(ct.contiguous(), rho.contiguous(), ops.stream)
        self.N = n[0] * n[1] * n[2]
        self.z = torch.empty(self.N, dtype=torch.float32, device=ops.dev)

    def vcycle(self, parts, nu1, nu2):
        r = self.ops.torch.cat(parts).contiguous()
        self.grid.mg_vcycle(r, self.z, nu1, nu2, stream=self.ops.stream)
        return self.z
