"""The C-ABI library loads and exports every symbol include/fe.h declares;
argument validation that needs no GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fe():
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe as fe_mod
    return fe_mod


def _header_functions():
    src = open(os.path.join(ROOT, "include", "fe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(fe):
    declared = _header_functions()
    assert len(declared) >= 18
    assert sorted(fe.EXPORTS) == declared
    for name in declared:
        assert hasattr(fe.lib, name), name


def test_abi_version_and_strings(fe):
    import re
    hdr = open(os.path.join(ROOT, "include", "fe.h")).read()
    assert fe.lib.fe_abi_version() == int(re.search(r"#define FE_ABI_VERSION (\d+)", hdr).group(1)) == 2
    assert fe.lib.fe_status_string(0) == b"ok"
    assert fe.lib.fe_status_string(5) == b"backtracking limit reached"


def test_default_params(fe):
    p = fe.default_params()
    assert (p.ksize, p.lambda_, p.beta, p.L0, p.eta, p.c2, p.max_backtrack, p.prec) == \
        (7, 5.0, 0.8, 1.0, 2.0, 1e-6, 30, 0)
    assert (p.tile, p.model, p.lambda1) == (0, 0, 0.0)


def _init(fe, **over):
    k = np.zeros((48, 7, 7), np.float32)
    th = np.full(48, 0.1, np.float32)
    p = fe.default_params()
    p.nf, p.ksize = 48, 7
    p.filters = k.ctypes.data_as(C.POINTER(C.c_float))
    p.theta = th.ctypes.data_as(C.POINTER(C.c_float))
    H = over.pop("H", 16)
    W = over.pop("W", 16)
    for a, v in over.items():
        setattr(p, a, v)
    f = np.ones((max(H, 1), max(W, 1)), np.float32)
    ctx = C.c_void_p()
    st = fe.lib.fe_init(C.byref(ctx), C.byref(p), H, W, f.ctypes.data, None, None)
    return st, ctx, (k, th, f)


@pytest.mark.parametrize("over", [dict(nf=0), dict(nf=65), dict(ksize=5), dict(lambda_=0.0),
                                  dict(beta=1.0), dict(beta=-0.1), dict(L0=0.0), dict(eta=1.0),
                                  dict(c2=-1.0), dict(max_backtrack=-1), dict(prec=7),
                                  dict(H=7), dict(W=4), dict(H=0)])
def test_invalid_arguments_rejected_before_any_device_work(fe, over):
    st, ctx, _ = _init(fe, **over)
    assert st == fe.FE_EINVAL
    assert ctx.value is None
    assert len(fe.lib.fe_last_error(None)) > 0


def test_null_context_calls(fe):
    assert fe.lib.fe_step(None, 1, None) == fe.FE_EINVAL
    assert fe.lib.fe_solve(None, 1, 0.0) == fe.FE_EINVAL
    assert fe.lib.fe_num_images(None) == 0
    fe.lib.fe_destroy(None)
