"""The C-ABI library builds, loads and exports every function that
include/*.h declares (no GPU: no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1112_3507_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_api():
    names = _declared()
    for must in ("lm_grid_create", "lm_set_coefficients", "lm_set_rhs", "lm_solve", "lm_get_solution",
                 "lm_get_residual_history", "lm_grid_destroy", "lm_apply", "lm_mg_vcycle"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_matches_header():
    from paper_1112_3507_gb300 import lowmach
    assert set(lowmach.declared_symbols()) <= _declared()
    assert _declared() <= set(lowmach.declared_symbols())


def test_status_strings_and_defaults(lib):
    from paper_1112_3507_gb300 import lowmach as lm
    assert lm.status_string(lm.LM_ERR_NOT_POSITIVE).startswith("coefficients")
    o = lm.SolveOpts()
    lm.lib().lm_default_opts(ctypes.byref(o))
    assert o.mode == lm.MIXED_MG_IR and o.rtol == 1e-8 and o.nu1 == 2 and o.nu2 == 3 and o.inner_rtol == 1e-4 and o.net_precond == 0


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1112_3507_gb300 import lowmach as lm
    monkeypatch.setattr(lm, "_lib", None)
    monkeypatch.setattr(lm, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lm.lib()
