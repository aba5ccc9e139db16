"""The z-slab building blocks and the distributed solve on one GB300.

The halo pack/unpack, vector and level-transfer kernels through the C ABI
against numpy and the oracle; then the distributed solvers of shard.py with
the GPU backend (GpuSlab) on ranks that are threads of this process, sharing
the one GPU (their kernels never wait on one another: every exchange is a
host-side hand-over between launches), against the oracle's direct solve."""
import ctypes
import os

import numpy as np
import pytest

from oracle import multigrid as OM
from oracle import poisson as P
from paper_1112_3507_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
PER, NEU = I.BC_PERIODIC, I.BC_NEUMANN


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_3507_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()


def lm():
    from paper_1112_3507_gb300 import lowmach
    return lowmach


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("plane,np_", [(64, 2), (6, 1), (33, 2)])
def test_halo_pack_unpack(dtype, plane, np_):
    """Both sides in one launch, a skipped side left untouched, unpack the inverse."""
    L = lm()
    nz = 9
    a = torch.randn(nz * plane, dtype=dtype, device="cuda")
    buf = torch.full((2 * np_ * plane,), -7.0, dtype=dtype, device="cuda")
    L._check(L.lib().lm_halo_pack(_p(a), a.element_size(), plane, 2, nz - 2 - np_, np_, _p(buf), 0, None), "pack")
    h = a.cpu().numpy().reshape(nz, plane)
    got = buf.cpu().numpy()
    np.testing.assert_array_equal(got[:np_ * plane], h[2:2 + np_].ravel())
    np.testing.assert_array_equal(got[np_ * plane:], h[nz - 2 - np_:nz - 2].ravel())
    buf.fill_(-7.0)
    L._check(L.lib().lm_halo_pack(_p(a), a.element_size(), plane, -1, 0, np_, _p(buf), 0, None), "pack")
    got = buf.cpu().numpy()
    assert np.all(got[:np_ * plane] == -7.0)
    np.testing.assert_array_equal(got[np_ * plane:], h[:np_].ravel())
    b = torch.zeros_like(a)
    src = torch.randn(2 * np_ * plane, dtype=dtype, device="cuda")
    L._check(L.lib().lm_halo_pack(_p(b), b.element_size(), plane, 0, nz - np_, np_, _p(src), 1, None), "unpack")
    bh, s = b.cpu().numpy().reshape(nz, plane), src.cpu().numpy()
    np.testing.assert_array_equal(bh[:np_].ravel(), s[:np_ * plane])
    np.testing.assert_array_equal(bh[nz - np_:].ravel(), s[np_ * plane:])
    assert np.all(bh[np_:nz - np_] == 0)


def test_vector_kernels():
    L = lm()
    n = 100003
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    y32 = torch.randn(n, dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    L._check(L.lib().lm_vec_axpby(n, 0.5, _p(x), L.PREC_FP64, -2.0, _p(y32), L.PREC_FP32, _p(out), L.PREC_FP64,
                                  None), "axpby")
    ref = 0.5 * x.cpu().numpy() - 2.0 * y32.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    scratch = torch.empty(1025, dtype=torch.float64, device="cuda")
    d = ctypes.c_double(0.0)
    L._check(L.lib().lm_vec_dot(n, _p(x), L.PREC_FP64, _p(y32), L.PREC_FP32, _p(scratch), ctypes.byref(d), None), "dot")
    assert d.value == pytest.approx(float(np.dot(x.cpu().numpy(), y32.cpu().numpy().astype(np.float64))), rel=1e-12)
    z = torch.empty_like(x)
    L._check(L.lib().lm_vec_mul(n, _p(x), _p(out), _p(z), None), "mul")
    np.testing.assert_array_equal(z.cpu().numpy(), x.cpu().numpy() * out.cpu().numpy())


@pytest.mark.parametrize("make", [lambda: I.make_problem(64, 24, 16, ma=0.01, contrast=20.0, noise=0.01, seed=41),
                                  lambda: I.make_problem(32, 20, ma=0.05, contrast=8.0, noise=0.01, seed=42)])
def test_level_transfers_match_oracle(make):
    """lm_mg_restrict_residual and lm_mg_prolong_add vs the oracle's
    restriction of the float32 residual and piecewise-constant prolongation."""
    L = lm()
    p = make()
    op = P.operator_from_problem(p)
    ct32 = op.ct.astype(np.float32).astype(np.float64)
    rho32 = p.rho_new.astype(np.float32).astype(np.float64)
    levels = OM.build_hierarchy(ct32, rho32, p.h, p.bc)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(p.size).astype(np.float32)
    f = rng.standard_normal(p.size).astype(np.float32)
    with L.Grid.for_problem(p) as g:
        g.set_problem(p)
        nc = g.mg_levels()[1]
        Nc = nc[0] * nc[1] * nc[2]
        xd, fd = torch.as_tensor(x, device="cuda"), torch.as_tensor(f, device="cuda")
        fc = torch.empty(Nc, dtype=torch.float32, device="cuda")
        L._check(L.lib().lm_mg_restrict_residual(g._g, _p(xd), _p(fd), _p(fc), None), "restrict")
        ec = torch.as_tensor(rng.standard_normal(Nc).astype(np.float32), device="cuda")
        xp = xd.clone()
        L._check(L.lib().lm_mg_prolong_add(g._g, _p(ec), _p(xp), None), "prolong")
        fc_h, xp_h, ec_h = fc.cpu().numpy(), xp.cpu().numpy(), ec.cpu().numpy()
    L0 = levels[0]
    r = f.astype(np.float64).reshape(L0.shape) - L0.op.apply(x.astype(np.float64))
    fc_ref = OM.restrict(r, L0.halved).ravel()
    assert np.linalg.norm(fc_h - fc_ref) <= 1e-5 * np.linalg.norm(fc_ref)
    xp_ref = x.astype(np.float64) + OM.prolong(ec_h.astype(np.float64).reshape(levels[1].shape), L0.halved).ravel()
    np.testing.assert_allclose(xp_h, xp_ref, rtol=1e-6, atol=1e-6)


def _run_threads(world, fn):
    import threading

    from paper_1112_3507_gb300 import shard as S
    comms = S.ThreadComm.group(world)
    out, err = [None] * world, []

    def body(r):
        try:
            torch.cuda.set_device(0)
            out[r] = fn(r, comms[r])
            torch.cuda.synchronize()
        except BaseException as e:      # noqa: BLE001 - reported below
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


SHARD_PROBLEMS = {
    "rows3d-256x16x32-zwall": lambda: I.make_problem(256, 32, 16, ma=0.01, contrast=15.0, noise=0.01, seed=51),
    "box3d-64x16x24-zper": lambda: I.make_problem(64, 24, 16, ma=0.02, contrast=10.0, noise=0.01, seed=52,
                                                  bc=(PER, PER, PER)),
    "plain2d-64x64": lambda: I.config_plain_2d(64, seed=53),
}


@pytest.mark.parametrize("name", list(SHARD_PROBLEMS))
@pytest.mark.parametrize("world", [1, 2, 3])
def test_distributed_solve_on_gpu(name, world):
    """shard.mg_fcg (and, on the 2D grid, shard.pcg_jacobi) with GpuSlab
    ranks: the float64 solutions match the oracle's direct solve to 1e-10, and the distributed
    V-cycle preconditions as well as the single-domain one (iteration count
    within one of the library's own float64 MG-FCG mode)."""
    from paper_1112_3507_gb300 import shard as S
    p = SHARD_PROBLEMS[name]()
    op = P.operator_from_problem(p)
    xs = P.solve_direct(op, p.f).ravel()
    with lm().Grid.for_problem(p) as g:
        g.set_problem(p)
        r_single = g.solve(mode="fp64-mg", rtol=1e-12, max_iter=200, nu1=2, nu2=2)

    jacobi = name.startswith("plain2d") and world == 2      # the slow plain PCG on the small grid only

    def rank(r, comm):
        geo = S.SlabGeometry(p.n, p.h, p.bc, r, world)
        ops = S.GpuSlab(geo, p.rho_old, p.rho_new, p.cs2, p.dt, p.f)
        try:
            x1 = None
            if jacobi:
                S.pcg_jacobi(ops, comm, rtol=1e-12, max_iter=20000)
                x1 = ops.solution().cpu().numpy().copy()
            km, _ = S.mg_fcg(ops, comm, rtol=1e-12, max_iter=200, nu1=2, nu2=2)
            x2 = ops.solution().cpu().numpy().copy()
            rel = S.true_residual(ops, comm)
        finally:
            ops.close()
        return x1, x2, km, rel

    res = _run_threads(world, rank)
    x2 = np.concatenate([t[1] for t in res])
    if jacobi:
        x1 = np.concatenate([t[0] for t in res])
        assert np.linalg.norm(x1 - xs) <= 1e-10 * np.linalg.norm(xs)
    assert np.linalg.norm(x2 - xs) <= 1e-10 * np.linalg.norm(xs)
    assert res[0][3] <= 2e-12
    assert abs(res[0][2] - r_single["iters"]) <= 1
