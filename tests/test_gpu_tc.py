"""The tensor-core building blocks the tensor-core M2L uses (tcgen05.mma with
BF16 inputs and FP32 accumulation in tensor memory, K-major operands in
shared memory without swizzling): a 128 x 32 x K product of integer-valued
BF16 matrices must equal the exact integer product, including sums close to
2^24, where every partial sum is still an exactly representable FP32
integer.  The FP64 emulation by digit splitting relies on exactly that."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import lib
    L = lib()
    ctx = C.c_void_p()
    assert L.gq_create(0, None, C.byref(ctx)) == 0
    return L, ctx


def _bf16_bits(x):
    """BF16 bit patterns of small integers (exact: |x| <= 256)."""
    return (np.asarray(x, np.float32).view(np.uint32) >> 16).astype(np.uint16)


def _run(L, ctx, A, B, swap=0):
    K = A.shape[1]
    a = np.ascontiguousarray(_bf16_bits(A))
    b = np.ascontiguousarray(_bf16_bits(B))
    d = np.zeros((128, 32), np.float32)
    st = L.gq_probe_umma(ctx, K, a.ctypes.data, b.ctypes.data, swap, d.ctypes.data)
    assert st == 0, L.gq_last_error(ctx)
    return d


@pytest.mark.parametrize("K", [16, 64, 256])
def test_umma_exact_integer_products(K):
    L, ctx = _ctx()
    rng = np.random.default_rng(K)
    A = rng.integers(-16, 17, size=(128, K))
    B = rng.integers(-16, 17, size=(32, K))
    d = _run(L, ctx, A, B)
    ref = A.astype(np.int64) @ B.astype(np.int64).T
    assert np.array_equal(d.astype(np.int64), ref)
    L.gq_destroy(ctx)


def test_umma_sums_near_2_24_are_exact():
    """|a|, |b| <= 255 and K = 256: sums up to 255^2 * 256 < 2^24 stay exact."""
    L, ctx = _ctx()
    rng = np.random.default_rng(7)
    A = rng.integers(-255, 256, size=(128, 256))
    B = rng.integers(-255, 256, size=(32, 256))
    A[:4] = 255
    B[:4] = 255                               # rows reaching 255^2 * 256 = 16,646,400
    B[4:8] = -255
    d = _run(L, ctx, A, B)
    ref = A.astype(np.int64) @ B.astype(np.int64).T
    assert np.abs(ref).max() > 2 ** 23
    assert np.array_equal(d.astype(np.int64), ref)
    L.gq_destroy(ctx)


def test_descriptor_offsets_are_not_interchangeable():
    """The layout check behind the descriptor encoding: with the leading and
    stride byte offsets exchanged, the product is wrong (so the passing
    assignment above is the one the hardware reads)."""
    L, ctx = _ctx()
    rng = np.random.default_rng(3)
    A = rng.integers(-16, 17, size=(128, 64))
    B = rng.integers(-16, 17, size=(32, 64))
    ref = A.astype(np.int64) @ B.astype(np.int64).T
    d = _run(L, ctx, A, B, swap=1)
    assert not np.array_equal(d.astype(np.int64), ref)
    L.gq_destroy(ctx)
