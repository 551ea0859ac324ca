"""The List 2 translations (Stage 4, Sec. 3.1 eq. m2l) and the List 3 far
multipole-to-QBX translations (Stage 5b) on the BF16 tensor cores with FP64
accuracy (digit splitting, GQ_M2L_AUTO) against the FP64 FMA kernels
(GQ_M2L_FP64) and the FP64 oracle: the potentials of the two modes agree to
1e-13 relative and both to the oracle within the 1e-12 parity bar; p_fmm =
16 isolates the second (the List 2 kernel takes p_fmm <= 15), p_fmm > 16
falls back to the FP64 kernels; repeated evaluations give the same bits."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _geo(g, **kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Geometry, params_default
    geo = Geometry(g, params_default(**kw))
    geo.build()
    return geo


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("case", ["c1", "grid4", "grid8"])
def test_tensor_m2l_matches_fp64_and_oracle(case):
    if case == "c1":
        g, p, q = workloads.starfish_c1(), 10, 5
    elif case == "grid4":
        g, p, q = workloads.starfish_grid(4, 4, 64, n_off=1 << 16, on_surface="up", seed=1), 15, 8
    else:
        g, p, q = workloads.starfish_grid(8, 8, 64, n_off=1 << 18, seed=2), 15, 8
    tc = _geo(g, p_qbx=q, p_fmm=p, n_max=32, m2l=0)
    f64 = _geo(g, p_qbx=q, p_fmm=p, n_max=32, m2l=1)
    o = oracle.Oracle(g, oracle.default_params(g, p_qbx=q, p_fmm=p))
    kind, _ = o.association()
    rng = np.random.default_rng(4)
    mask = np.zeros(len(kind), np.int32)
    for k in (0, 1, 2):
        ids = np.nonzero(kind == k)[0]
        mask[rng.choice(ids, min(400, len(ids)), replace=False)] = 1
    sel = mask.astype(bool)
    for kern in ("S", "D"):
        a = tc.eval(kern, g["density"])
        b = f64.eval(kern, g["density"])
        assert _rel(a, b) <= 1e-13, (case, kern, _rel(a, b))
        ref = o.eval(kern, g["density"], target_mask=mask)
        assert _rel(a[sel], ref[sel]) <= 1e-12, (case, kern)
        assert np.array_equal(a, tc.eval(kern, g["density"]))
    tc.close()
    f64.close()


@pytest.mark.parametrize("p,q", [(16, 8), (12, 12), (10, 15)])
def test_tensor_m2qbxl_alone(p, q):
    """M2QBXL on the tensor cores with the FP64 List 2 kernel (p_fmm = 16) or
    at QBX orders up to 15 (the binomial table's largest entry C(q+p-1, p-1)
    stays below 2^24)."""
    g = workloads.starfish_grid(4, 4, 64, n_off=1 << 16, on_surface="up", seed=3)
    tc = _geo(g, p_qbx=q, p_fmm=p, n_max=32, m2l=0)
    f64 = _geo(g, p_qbx=q, p_fmm=p, n_max=32, m2l=1)
    o = oracle.Oracle(g, oracle.default_params(g, p_qbx=q, p_fmm=p))
    kind, _ = o.association()
    rng = np.random.default_rng(6)
    mask = np.zeros(len(kind), np.int32)
    for k in (0, 1, 2):
        ids = np.nonzero(kind == k)[0]
        mask[rng.choice(ids, min(300, len(ids)), replace=False)] = 1
    sel = mask.astype(bool)
    for kern in ("S", "D"):
        a = tc.eval(kern, g["density"])
        b = f64.eval(kern, g["density"])
        assert _rel(a, b) <= 1e-13, (p, q, kern, _rel(a, b))
        ref = o.eval(kern, g["density"], target_mask=mask)
        assert _rel(a[sel], ref[sel]) <= 1e-12, (p, q, kern)
        assert np.array_equal(a, tc.eval(kern, g["density"]))
    tc.close()
    f64.close()


def test_high_order_falls_back_to_fp64():
    g = workloads.small_grid(2, 2, 16, 3000, seed=7)
    a = _geo(g, p_qbx=5, p_fmm=20, n_max=32, m2l=0)
    b = _geo(g, p_qbx=5, p_fmm=20, n_max=32, m2l=1)
    for kern in ("S", "D"):
        assert np.array_equal(a.eval(kern, g["density"]), b.eval(kern, g["density"]))


def test_unknown_m2l_mode_rejected():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import GigaQBXError, Geometry, params_default
    g = workloads.starfish_c1()
    with pytest.raises(GigaQBXError):
        Geometry(g, params_default(m2l=2))


def test_tensor_paths_are_taken():
    """gq_tensor_paths: both translations run on the tensor cores at the
    benchmark orders (the occupancy-checked launch did not fall back), the List
    2 kernel stops at p_fmm 15, both stop past p_fmm 16 and with
    GQ_M2L_FP64, and the mixed tier's pair kernel takes List 3 far."""
    g = workloads.small_grid(2, 2, 16, 3000, seed=7)
    cases = [(dict(p_qbx=8, p_fmm=15), (True, True)), (dict(p_qbx=8, p_fmm=16), (False, True)),
             (dict(p_qbx=5, p_fmm=20), (False, False)), (dict(p_qbx=8, p_fmm=15, m2l=1), (False, False)),
             (dict(p_qbx=8, p_fmm=15, eps=1e-8, precision=1), (True, False))]
    for kw, want in cases:
        geo = _geo(g, n_max=32, **kw)
        assert geo.tensor_paths() == want, kw
        geo.close()
