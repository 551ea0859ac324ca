"""gq_eval_noalloc, the evaluation entry point for callers that cannot
allocate device memory while running (graph replays, services that reserve
all memory at start-up).  It must give the results of gq_eval, call after
call, from its fixed device array; problems too large for the array and
host pointers must be refused with an error, not served."""
import ctypes as C

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the FP64 parity bar used by the other GPU tests


def _setup(g):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Geometry, lib, params_default
    geo = Geometry(g, params_default(p_qbx=int(g["p_qbx"]), p_fmm=int(g["p_fmm"]), n_max=int(g["n_max"])))
    geo.build()
    return torch, lib(), geo


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def _two_calls(torch, L, geo, g, kernels):
    nt = len(g["tgt_xy"])
    rng = np.random.default_rng(5)
    dens = [torch.tensor(g["density"], dtype=torch.float64, device="cuda"),
            torch.tensor(rng.normal(size=len(g["density"])), dtype=torch.float64, device="cuda")]
    for kern in kernels:
        for call in range(2):                      # two calls in a row
            out = torch.full((nt,), float("nan"), dtype=torch.float64, device="cuda")
            assert L.gq_eval_noalloc(geo._geom, kern, dens[call].data_ptr(), out.data_ptr()) == 0, \
                L.gq_last_error(geo._ctx)
            ref = torch.empty(nt, dtype=torch.float64, device="cuda")
            geo.eval(kern, dens[call], ref)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert _rel(out, ref) <= TOL, (kern, call)


@pytest.mark.parametrize("which", ["c1", "grid"])
def test_noalloc_matches_eval_on_two_calls(which):
    """S and D (and S' on c1, whose targets are the base nodes, on-surface)."""
    g = workloads.starfish_c1() if which == "c1" else workloads.small_grid(3, 2, 24, 5000, seed=11)
    torch, L, geo = _setup(g)
    _two_calls(torch, L, geo, g, (0, 1, 2) if which == "c1" else (0, 1))
    geo.close()


def test_noalloc_per_centre_orders():
    """Per-centre QBX orders (gq_set_centre_orders) are honoured as in gq_eval."""
    g = workloads.starfish_c1()
    torch, L, geo = _setup(g)
    q = np.random.default_rng(9).integers(2, int(g["p_qbx"]) + 1, size=2 * len(g["base_xy"])).astype(np.int32)
    geo.set_centre_orders(q)
    _two_calls(torch, L, geo, g, (0, 1, 2))
    geo.close()


_FRESH = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import workloads
from paper_1801_04070_gb300 import Geometry, lib, params_default
g = workloads.starfish_c1()
geo = Geometry(g, params_default(p_qbx=5, p_fmm=10, n_max=32))
geo.build()
L = lib()
d = torch.tensor(g["density"], dtype=torch.float64, device="cuda")
a = torch.full((len(g["tgt_xy"]),), float("nan"), dtype=torch.float64, device="cuda")
assert L.gq_eval_noalloc(geo._geom, 0, d.data_ptr(), a.data_ptr()) == 0, L.gq_last_error(geo._ctx)
torch.cuda.synchronize()
b = torch.empty_like(a)
geo.eval("S", d, b)
torch.cuda.synchronize()
err = float((a - b).abs().max() / b.abs().max())
assert err <= 1e-12, err
print("fresh ok", err)
"""


def test_noalloc_first_call_in_fresh_process():
    """The set-up on a device that no gq_eval has touched yet (its own table
    writes only), in a fresh process: the first call already matches gq_eval."""
    import os
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH % root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


def test_noalloc_refuses_oversize_and_host_pointers():
    g = workloads.starfish_grid(8, 8, 64, n_off=1 << 16, seed=3)
    torch, L, geo = _setup(g)
    nt = len(g["tgt_xy"])
    dens = torch.tensor(g["density"], dtype=torch.float64, device="cuda")
    out = torch.empty(nt, dtype=torch.float64, device="cuda")
    assert L.gq_eval_noalloc(geo._geom, 0, dens.data_ptr(), out.data_ptr()) == -5   # GQ_ERR_UNSUPPORTED
    assert b"scratch" in L.gq_last_error(geo._ctx)
    geo.close()
    g = workloads.starfish_c1()
    torch, L, geo = _setup(g)
    host = np.ascontiguousarray(g["density"])
    out = torch.empty(len(g["tgt_xy"]), dtype=torch.float64, device="cuda")
    assert L.gq_eval_noalloc(geo._geom, 0, C.c_void_p(host.ctypes.data), out.data_ptr()) == -1   # GQ_ERR_INVALID
    geo.close()
