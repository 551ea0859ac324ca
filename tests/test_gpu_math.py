"""The FP64 logarithm (Tang's table-driven method) and reciprocal (FP32 seed +
two Newton steps) used by the direct-interaction kernels, and their
double-FP32 counterparts in the split-precision kernels, checked against
CUDA's log and IEEE division over the ranges the kernels meet and beyond."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(fn, x):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_04070_gb300 as pkg
    import workloads
    geo = pkg.Geometry(workloads.starfish_c1())
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    assert pkg.lib().gq_probe_math(geo._ctx, fn, len(x), xd.data_ptr(), yd.data_ptr()) == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _inputs():
    rng = np.random.default_rng(0)
    return np.concatenate([10.0 ** rng.uniform(-12, 12, 200000), 1.0 + rng.uniform(-1e-3, 1e-3, 20000),
                           np.array([1.0, 2.0, 0.5, 1e-300, 1e300, 0.0, np.inf, 7.0 / 3.0])])


def test_log_matches_cuda_log():
    x = _inputs()
    mine, ref = _run(0, x), _run(1, x)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(mine), fin)
    err = np.abs(mine[fin] - ref[fin])
    print(f"FP64 log: max error {(err / np.spacing(np.maximum(np.abs(ref[fin]), 1.0))).max():.2f} ulp of max(|log x|, 1)")
    # absolute error within a few ulp of max(|log x|, 1), i.e. of the terms it multiplies
    assert (err <= 4 * np.spacing(np.maximum(np.abs(ref[fin]), 1.0))).all(), err.max()


def test_reciprocal_matches_division():
    x = _inputs()
    x = x[(x > 0) & np.isfinite(x)]
    x = np.concatenate([x, -x])
    mine, ref = _run(2, x), _run(3, x)
    ulps = np.abs(mine - ref) / np.spacing(np.abs(ref))
    print(f"FP64 reciprocal: max error {ulps.max():.2f} ulp, {np.mean(ulps > 0):.2e} of results not the IEEE quotient")
    assert (ulps <= 2).all()


def _split_inputs():
    rng = np.random.default_rng(2)
    return np.concatenate([10.0 ** rng.uniform(-30, 30, 200000), 1.0 + rng.uniform(-1e-3, 1e-3, 20000),
                           1.0 + rng.uniform(0, 64, 20000), np.array([1.0, 2.0, 0.5, 7.0 / 3.0, 2.0 ** 126])])


def test_split_log_matches_cuda_log():
    """Pair logarithm: absolute error about 2^-47 max(|log x|, 1) (48-bit pairs)."""
    x = _split_inputs()
    mine, ref = _run(4, x), _run(1, x)
    err = np.abs(mine - ref) / np.maximum(np.abs(ref), 1.0)
    print(f"double-FP32 log: max error {err.max():.2e} (2^{np.log2(err.max()):.1f})")
    assert err.max() <= 2.0 ** -45


def test_split_reciprocal_matches_division():
    x = _split_inputs()
    x = np.concatenate([x, -x])
    mine, ref = _run(5, x), _run(3, x)
    err = np.abs(mine - ref) / np.abs(ref)
    print(f"double-FP32 reciprocal: max relative error {err.max():.2e} (2^{np.log2(err.max()):.1f})")
    assert err.max() <= 2.0 ** -44


def test_fma_probe_rates():
    """The throughput probe behind the ALU roofline: every variant returns a
    positive rate, FP32 beats FP64, the combined FP64 FMA + MMA run is at least
    the slower of the two, and an unknown variant is rejected."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes as C

    import paper_1801_04070_gb300 as pkg
    import workloads
    geo = pkg.Geometry(workloads.starfish_c1())
    L = pkg.lib()
    rates = []
    for what in range(4):
        v = C.c_double()
        assert L.gq_probe_fma_peak(geo._ctx, what, C.byref(v)) == 0
        assert v.value > 0
        rates.append(v.value)
    assert rates[1] > rates[0]
    assert rates[3] >= 0.9 * min(rates[0], rates[2])
    v = C.c_double()
    assert L.gq_probe_fma_peak(geo._ctx, 4, C.byref(v)) != 0
    print("probe TFLOP/s fp64 fma, fp32 fma, fp64 mma, fp64 fma+mma:", [round(r, 3) for r in rates])
