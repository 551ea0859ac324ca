"""The caching device allocator: buffers freed by the build go to the cache,
gq_memory_release hands them back to the driver, and the library keeps
working afterwards (no error left behind for the next launch check), with
the same results bit for bit."""
import ctypes as C

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_release_cache_then_evaluate():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_04070_gb300 as pkg
    L = pkg.lib()
    g = workloads.small_grid(2, 2, 16, 3000, seed=7)
    geo = pkg.Geometry(g, pkg.params_default(p_qbx=5, p_fmm=10, n_max=32))
    geo.build()
    v0 = geo.eval("S", g["density"])
    torch.cuda.synchronize()
    cached = C.c_int64(-1)
    assert L.gq_memory_cached(C.byref(cached)) == 0 and cached.value > 0   # build temporaries
    assert L.gq_memory_release() == 0
    assert L.gq_memory_cached(C.byref(cached)) == 0 and cached.value == 0
    v1 = geo.eval("S", g["density"])
    geo.build()                                                            # allocates again
    v2 = geo.eval("S", g["density"])
    assert np.array_equal(v0, v1) and np.array_equal(v0, v2)
