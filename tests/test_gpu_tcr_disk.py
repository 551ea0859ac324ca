"""The disk-shaped target confinement region (tcr_shape 1, the variant of
the paper's appendix corrigendum) on the GPU against the oracle: centres and
their levels, the tree, owners and all six interaction lists bit for bit,
the potentials within the 1e-12 parity bar; single-curve and grid
geometries, and sampled targets of every kind on an 8 x 8 grid."""
import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import check_build

pytestmark = pytest.mark.gpu


def _pair(g, **kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Geometry, params_default
    p = oracle.default_params(g, tcr_shape=1, **kw)
    geo = Geometry(g, params_default(p_qbx=p["p_qbx"], p_fmm=p["p_fmm"], n_max=p["n_max"], tcr_shape=1))
    geo.build()
    return geo, oracle.Oracle(g, p)


@pytest.mark.parametrize("case", ["c1", "grid32", "grid44"])
def test_disk_tcr_tree_lists_and_values_match_oracle(case):
    g = {"c1": workloads.starfish_c1(),
         "grid32": workloads.small_grid(3, 2, 24, 5000, seed=11),
         "grid44": workloads.starfish_grid(4, 4, 32, n_off=4000, seed=5)}[case]
    geo, orc = _pair(g)
    check_build(geo, orc)
    _, _, lc_sq = oracle.Oracle(g, oracle.default_params(g)).centres()
    _, _, lc = orc.centres()
    assert (lc <= lc_sq).all() and (lc < lc_sq).any()   # the disk TCR changes the tree
    for kern in ("S", "D"):
        v, ref = geo.eval(kern, g["density"]), orc.eval(kern, g["density"])
        assert np.abs(v - ref).max() <= 1e-12 * np.abs(ref).max(), (case, kern)
    geo.close()


def test_disk_tcr_sampled_at_scale():
    g = workloads.starfish_grid(8, 8, 64, n_off=1 << 18, seed=2)
    geo, orc = _pair(g, p_qbx=8, p_fmm=15)
    check_build(geo, orc)
    kind, _ = orc.association()
    rng = np.random.default_rng(8)
    mask = np.zeros(len(kind), np.int32)
    for k in (0, 1, 2):
        ids = np.nonzero(kind == k)[0]
        mask[rng.choice(ids, min(500, len(ids)), replace=False)] = 1
    sel = mask.astype(bool)
    for kern in ("S", "D"):
        v = geo.eval(kern, g["density"])
        ref = orc.eval(kern, g["density"], target_mask=mask)
        assert np.abs(v[sel] - ref[sel]).max() <= 1e-12 * np.abs(ref[sel]).max(), kern
    geo.close()


def test_tcr_shape_is_validated():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import GigaQBXError, Geometry, params_default
    g = workloads.starfish_c1()
    with pytest.raises(GigaQBXError):
        Geometry(g, params_default(tcr_shape=2))
