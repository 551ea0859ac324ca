"""Precision modes (MIXED: FP32 direct sums when eps >= 5e-6, double-FP32
power sums when 1e-12 <= eps < 5e-6, FP64 translations; MIXED_FMM: the
translations in double-FP32 pairs as well) and the accuracy
sweep with orders chosen from the requested accuracy, checked against the
FP64 oracle: O2 at the same orders (rounding of the mixed path) and O1,
unaccelerated QBX at the same p_qbx (FMM + rounding error, the quantity the
Theorem of Sec. 4.5 bounds)."""
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


@pytest.mark.parametrize("kern", ["S", "D"])
def test_mixed_fp32_tier_matches_oracle(kern):
    g = workloads.small_grid(3, 2, 24, 5000, seed=11, on_surface="up", p_qbx=8, p_fmm=15)
    geo = _geo(g, p_qbx=8, p_fmm=15, n_max=32, eps=5e-6, precision=1)
    v = geo.eval(kern, g["density"])
    ref = oracle.Oracle(g, oracle.default_params(g)).eval(kern, g["density"])
    err = np.abs(v - ref).max() / np.abs(ref).max()
    print(f"MIXED (FP32 direct) {kern}: rel err vs FP64 oracle {err:.2e}")
    assert err <= 1e-6          # <= eps/5 at the FP32 tier threshold eps = 5e-6


@pytest.mark.parametrize("kern", ["S", "D"])
@pytest.mark.parametrize("eps,bound", [(1e-8, 2e-11), (1e-12, 2e-13)])
def test_mixed_split_tier_matches_oracle(kern, eps, bound):
    """1e-12 <= eps < 5e-6: power recurrences in double-FP32 pairs (about 48
    significant bits).  Pairs with sources near a centre amplify the rounding
    by |r/w|^m: those inside the disk are taken in FP64, and below eps = 1e-10
    also the point-target pairs closer than 1/8 of the box half-width.  M2L
    runs in pairs at eps = 1e-8 and in FP64 at 1e-12.  Bound: eps/5 at the
    smallest eps of each range (1e-10 and 1e-12)."""
    g = workloads.small_grid(3, 2, 24, 5000, seed=11, on_surface="up", p_qbx=8, p_fmm=15)
    geo = _geo(g, p_qbx=8, p_fmm=15, n_max=32, eps=eps, precision=1)
    v = geo.eval(kern, g["density"])
    f = _geo(g, p_qbx=8, p_fmm=15, n_max=32, eps=eps, precision=0).eval(kern, g["density"])
    ref = oracle.Oracle(g, oracle.default_params(g)).eval(kern, g["density"])
    err = np.abs(v - ref).max() / np.abs(ref).max()
    added = np.abs(v - f).max() / np.abs(f).max()
    print(f"MIXED (double-FP32 power sums, eps {eps:.0e}) {kern}: rel err vs FP64 oracle {err:.2e}, "
          f"vs the FP64 path {added:.2e}")
    assert added <= bound                 # the rounding the tier adds
    assert err <= max(bound, 1e-12)       # and the FP64 parity bound against the oracle


@pytest.mark.parametrize("kern", ["S", "D"])
def test_mixed_split_tier_sampled_at_eps_orders(kern):
    """The double-FP32 tier on a 4x4 starfish grid at the orders eps = 1e-10
    selects (p_qbx 7, p_fmm 30), where the List 3 far translations (M2QBXL,
    M2P) and the point-target direct sums also run in pairs: sampled targets
    of every kind against the FP64 oracle at the same orders."""
    g = workloads.starfish_grid(4, 4, 64, n_off=1 << 16, on_surface="up", seed=1)
    geo = _geo(g, p_qbx=0, p_fmm=0, n_max=32, eps=1e-10, precision=1)
    prm = geo.params
    v = geo.eval(kern, g["density"])
    o = oracle.Oracle(g, oracle.default_params(g, p_qbx=prm.p_qbx, p_fmm=prm.p_fmm))
    kind, _ = o.association()
    rng = np.random.default_rng(3)
    mask = np.zeros(len(kind), np.int32)
    for k in (0, 1, 2):
        ids = np.nonzero(kind == k)[0]
        mask[rng.choice(ids, min(300, len(ids)), replace=False)] = 1
    sel = mask.astype(bool)
    ref = o.eval(kern, g["density"], target_mask=mask)
    err = np.abs(v[sel] - ref[sel]).max() / np.abs(ref[sel]).max()
    print(f"MIXED double-FP32 {kern} at p_qbx {prm.p_qbx} p_fmm {prm.p_fmm}: rel err vs FP64 oracle {err:.2e}")
    assert err <= 2e-11


@pytest.mark.parametrize("kern", ["S", "D"])
@pytest.mark.parametrize("eps,p_fmm", [(1e-5, 16), (1e-6, 19), (1e-10, 30)])
def test_pair_fmm_passes_rounding(kern, eps, p_fmm):
    """GQ_PREC_MIXED_FMM: P2M, M2M, M2L, L2L and L2QBXL in FP32 pairs on top
    of either mixed tier (eps >= 1e-10): on a 4x4 starfish grid, whose far field runs through several hundred thousand
    List 2 translations, the mixed evaluation at p_fmm up to 30 stays within eps/5 of
    the FP64 path at the same orders; in the pair tier the QBX coefficients
    (which carry the translated local expansions) also stay within eps/5 of the
    FP64 ones, order by order."""
    g = workloads.starfish_grid(4, 4, 64, n_off=1 << 16, on_surface="up", seed=1)
    mixed = _geo(g, p_qbx=7, p_fmm=p_fmm, n_max=32, eps=eps, precision=2)
    fp64 = _geo(g, p_qbx=7, p_fmm=p_fmm, n_max=32, eps=eps, precision=0)
    v = mixed.eval(kern, g["density"])
    qm = mixed.qbx_coefficients()
    f = fp64.eval(kern, g["density"])
    qf = fp64.qbx_coefficients()
    added = np.abs(v - f).max() / np.abs(f).max()
    qerr = max(np.abs(qm[:, m] - qf[:, m]).max() / np.abs(qf[:, m]).max() for m in range(qf.shape[1]))
    print(f"pair FMM passes, eps {eps:.0e}, p_fmm {p_fmm}, {kern}: potential {added:.2e}, QBX coefficients {qerr:.2e} "
          f"relative to the FP64 path")
    assert added <= eps / 5
    if eps < 5e-6:
        assert qerr <= eps / 5


def test_mixed_below_threshold_is_fp64():
    g = workloads.small_grid(2, 2, 16, 3000, seed=7)
    geo = _geo(g, p_qbx=5, p_fmm=10, n_max=32, eps=1e-13, precision=1)
    v = geo.eval("S", g["density"])
    ref = oracle.Oracle(g, oracle.default_params(g)).eval("S", g["density"])
    assert np.abs(v - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8, 1e-10, 1e-12])
def test_accuracy_sweep(eps):
    g = workloads.starfish_grid(4, 4, 64, n_off=1 << 16, on_surface="up", seed=1)
    from paper_1801_04070_gb300 import params_default
    geo = _geo(g, p_qbx=0, p_fmm=0, n_max=32, eps=eps, precision=1)
    prm = geo.params
    v = geo.eval("S", g["density"])
    o = oracle.Oracle(g, oracle.default_params(g, p_qbx=prm.p_qbx, p_fmm=prm.p_fmm))
    kind, _ = o.association()
    rng = np.random.default_rng(1)
    mask = np.zeros(len(kind), np.int32)
    for k in (1, 2):
        ids = np.nonzero(kind == k)[0]
        mask[rng.choice(ids, min(150, len(ids)), replace=False)] = 1
    sel = mask.astype(bool)
    o1 = o.direct("S", g["density"], target_mask=mask)
    err = np.abs(v[sel] - o1[sel]).max() / np.abs(o1[sel]).max()
    print(f"eps {eps:.0e}: p_qbx {prm.p_qbx} p_fmm {prm.p_fmm}: rel err vs unaccelerated QBX {err:.2e}")
    assert err <= max(eps, 1e-11)


def test_unknown_precision_rejected():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Geometry, params_default
    from paper_1801_04070_gb300._lib import GigaQBXError
    g = workloads.starfish_c1()
    with pytest.raises(GigaQBXError):
        Geometry(g, params_default(p_qbx=5, p_fmm=10, n_max=32, precision=3))
