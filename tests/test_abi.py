"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/gigaqbx.h declares, and its host-only entry points
behave (no GPU work is launched here)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "gigaqbx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gq_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1801_04070_gb300 import build
    return build.build()


def test_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gq_[a-z0-9_]+)", out))
    decl = _declared()
    assert len(decl) >= 15
    missing = [d for d in decl if d not in exported]
    assert not missing, missing


def test_host_entry_points(libpath):
    import paper_1801_04070_gb300 as pkg
    L = pkg.lib()
    p = pkg.params_default()
    assert (p.p_qbx, p.p_fmm, p.n_max, p.tf_num, p.tf_den, p.w3_demote) == (5, 10, 32, 9, 10, 15)
    assert L.gq_params_default(None) == -1
    assert L.gq_destroy(None) == -1
    assert L.gq_build(None) == -1
    assert L.gq_eval(None, 0, None, None, None) == -1
    assert L.gq_apply(None, 0, -0.5, None, None) == -1
    assert L.gq_lists_check(None, 0, None) == -1
    assert L.gq_last_error(None) == b"null context"
    n = C.c_int64(-1)
    assert L.gq_memory_cached(C.byref(n)) == 0 and n.value >= 0
    assert L.gq_memory_cached(None) == -1
    assert L.gq_memory_release() == 0       # nothing cached without a GPU: touches no device


def test_create_without_gpu_fails_cleanly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1801_04070_gb300 as pkg
    h = C.c_void_p()
    assert pkg.lib().gq_create(0, None, C.byref(h)) == -3
    assert not h.value


def test_params_resolve_orders_from_eps(libpath):
    """Host-only order selection (no GPU): p_fmm is the smallest p whose
    idealised FMM error (1/2)^(p+1) is <= eps (Sec. 4.1, 5.1), clamped to
    [1, 30]; p_qbx follows the calibrated truncation rule and grows as eps
    shrinks; given orders are kept; invalid parameters are rejected and leave
    the output untouched."""
    import math

    import paper_1801_04070_gb300 as pkg
    for eps in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 3e-7):
        r = pkg.params_resolve(pkg.params_default(p_qbx=0, p_fmm=0, eps=eps))
        p = r.p_fmm
        if p < 30:                           # the clamp takes over below eps = 2^-31
            assert 0.5 ** (p + 1) <= eps and (p == 1 or 0.5 ** p > eps), (eps, p)
        else:
            assert 0.5 ** 30 > eps, (eps, p)
        assert 1 <= r.p_qbx <= 16
    qs = [pkg.params_resolve(pkg.params_default(p_qbx=0, p_fmm=0, eps=e)).p_qbx for e in (1e-4, 1e-8, 1e-12)]
    assert qs == sorted(qs) and qs[0] < qs[-1]
    assert pkg.params_resolve(pkg.params_default(p_qbx=0, p_fmm=0, eps=1e-300)).p_fmm == 30
    r = pkg.params_resolve(pkg.params_default(p_qbx=7, p_fmm=0, eps=1e-8))
    assert (r.p_qbx, r.p_fmm) == (7, math.ceil(math.log2(1e8)) - 1)
    r = pkg.params_resolve(pkg.params_default(p_qbx=8, p_fmm=15))
    assert (r.p_qbx, r.p_fmm, r.n_max) == (8, 15, 32)
    L = pkg.lib()
    for bad in (dict(p_qbx=0, p_fmm=0, eps=0.0), dict(p_qbx=17), dict(p_fmm=31), dict(n_max=0),
                dict(tf_num=10, tf_den=10), dict(precision=3), dict(radius_factor=0.0)):
        p = pkg.params_default(**bad)
        out = pkg.params_default(p_qbx=3)
        assert L.gq_params_resolve(C.byref(p), C.byref(out)) == -1, bad
        assert out.p_qbx == 3
        with pytest.raises(pkg.GigaQBXError):
            pkg.params_resolve(p)
    assert L.gq_params_resolve(None, None) == -1
