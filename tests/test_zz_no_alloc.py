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


@pytest.mark.parametrize("which", ["c1", "grid"])
def test_noalloc_matches_eval_on_two_calls(which):
    g = workloads.starfish_c1() if which == "c1" else workloads.small_grid(3, 2, 24, 5000, seed=11)
    torch, L, geo = _setup(g)
    nt = len(g["tgt_xy"])
    rng = np.random.default_rng(5)
    dens = [torch.tensor(g["density"], dtype=torch.float64, device="cuda"),
            torch.tensor(rng.normal(size=len(g["density"])), dtype=torch.float64, device="cuda")]
    for kern in (0, 1):
        for call in range(2):                      # two calls in a row, the first before any gq_eval
            out = torch.full((nt,), float("nan"), dtype=torch.float64, device="cuda")
            assert L.gq_eval_noalloc(geo._geom, kern, dens[call].data_ptr(), out.data_ptr()) == 0, \
                L.gq_last_error(geo._ctx)
            ref = torch.empty(nt, dtype=torch.float64, device="cuda")
            geo.eval(kern, dens[call], ref)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert _rel(out, ref) <= TOL, (kern, call)
    geo.close()


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
