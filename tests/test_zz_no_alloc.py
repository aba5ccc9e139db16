"""The allocation-free float64 apply (lm_apply_dot_noalloc) agrees with the
grid-based lm_apply on two calls in a row.

Some callers cannot allocate device memory once running (a fixed memory
budget handed over at start-up, a frozen pool); this entry point serves
them with scratch in a static device array.  Collected last on purpose."""
import os

import numpy as np
import pytest

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


def _stencil_magnitude(op, x):
    """sum over the terms of (A x)_i of their magnitudes: |c~_i x_i| + sum_f g_f |x_i - x_nb|,
    the scale of the rounding error of any evaluation order of row i."""
    x = x.reshape(op.shape)
    m = np.abs(op.ct * x)
    for a in range(3):
        ax = 2 - a
        m = m + op.g_minus[a] * np.abs(x - np.roll(x, 1, axis=ax))
        m = m + op.g_plus(a) * np.abs(x - np.roll(x, -1, axis=ax))
    return m.ravel()


def test_noalloc_apply_matches_grid_apply_and_oracle(lm):
    """Two grids in a row, the larger first: the scratch keeps the partials
    of the 24^3 call when the 64 x 64 call runs, and that call must read
    only its own.  Each grid gets two calls, the second on a non-default
    stream; y and x^T A x are compared with the grid-based lm_apply and with
    the oracle's operator, element by element."""
    from oracle import poisson as P
    side = torch.cuda.Stream()
    for p in (I.config_convection_3d(24, seed=11), I.config_plain_2d(64, seed=12)):
        op = P.operator_from_problem(p)
        g = lm.Grid.for_problem(p)
        try:
            g.set_problem(p)
            ct, gx, gy, gz = g.coefficients()
            rng = np.random.default_rng(13)
            for call, stream in enumerate((None, side)):   # two calls in a row, different inputs
                xh = rng.standard_normal(p.size)
                x = torch.as_tensor(xh, device="cuda")
                y_ref = torch.empty_like(x)
                dot_ref = g.apply(x, y_ref, prec=lm.PREC_FP64, with_dot=True)
                y = torch.full_like(x, np.nan)
                dot = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                lm.apply_dot_noalloc(p.ndim, p.n, p.bc, ct, gx, gy, gz, x, y, dot,
                                     stream=stream.cuda_stream if stream is not None else None)
                torch.cuda.synchronize()
                y_h = y.cpu().numpy()
                # same stencil code as lm_apply: identical values
                np.testing.assert_array_equal(y_h, y_ref.cpu().numpy())
                assert float(dot.item()) == pytest.approx(dot_ref, rel=1e-12), call
                # against the oracle's operator, per element
                y_or = op.apply(xh).ravel()
                assert np.all(np.abs(y_h - y_or) <= 1e-14 * _stencil_magnitude(op, xh)), call
                assert float(dot.item()) == pytest.approx(float(np.vdot(xh, y_or)), rel=1e-12), call
        finally:
            g.close()


def test_noalloc_rejects_grids_beyond_the_scratch(lm):
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = (65536, 4097, 1)                            # 268,500,992 cells > 65536 * 4096
    rc = lm.lib().lm_apply_dot_noalloc(3, lm._I64_3(*n), lm._I3(0, 0, 1), *([lm.ctypes.c_void_p(t.data_ptr())] * 7),
                                       lm.ctypes.c_void_p(0))
    assert rc == lm.LM_ERR_INVALID_ARG
