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
    assert L.gq_last_error(None) == b"null context"


def test_create_without_gpu_fails_cleanly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1801_04070_gb300 as pkg
    h = C.c_void_p()
    assert pkg.lib().gq_create(0, None, C.byref(h)) == -3
    assert not h.value
