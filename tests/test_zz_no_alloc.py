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


@pytest.mark.parametrize("make", [lambda: I.config_convection_3d(24, seed=11),
                                  lambda: I.config_plain_2d(64, seed=12)])
def test_noalloc_apply_matches_grid_apply(lm, make):
    p = make()
    g = lm.Grid.for_problem(p)
    try:
        g.set_problem(p)
        ct, gx, gy, gz = g.coefficients()
        rng = np.random.default_rng(13)
        for call in range(2):                       # two calls in a row, different inputs
            x = torch.as_tensor(rng.standard_normal(p.size), device="cuda")
            y_ref = torch.empty_like(x)
            dot_ref = g.apply(x, y_ref, prec=lm.PREC_FP64, with_dot=True)
            y = torch.full_like(x, np.nan)
            dot = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            lm.apply_dot_noalloc(p.ndim, p.n, p.bc, ct, gx, gy, gz, x, y, dot)
            torch.cuda.synchronize()
            y_ref_h, y_h = y_ref.cpu().numpy(), y.cpu().numpy()
            assert np.linalg.norm(y_h - y_ref_h) <= 1e-14 * np.linalg.norm(y_ref_h), call
            assert float(dot.item()) == pytest.approx(dot_ref, rel=1e-12), call
    finally:
        g.close()


def test_noalloc_rejects_grids_beyond_the_scratch(lm):
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = (65536, 4097, 1)                            # 268,500,992 cells > 65536 * 4096
    rc = lm.lib().lm_apply_dot_noalloc(3, lm._I64_3(*n), lm._I3(0, 0, 1), *([lm.ctypes.c_void_p(t.data_ptr())] * 7),
                                       lm.ctypes.c_void_p(0))
    assert rc == lm.LM_ERR_INVALID_ARG
