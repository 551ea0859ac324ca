"""The level-restricted tree (Sec. 4.6, remark on level-restricted
quadtrees) on the GPU against the oracle: the balanced tree, owners and all
six interaction lists bit for bit, and the potentials within the 1e-12
parity bar, on single-curve and grid geometries."""
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
    p = oracle.default_params(g, level_restrict=1, **kw)
    geo = Geometry(g, params_default(p_qbx=p["p_qbx"], p_fmm=p["p_fmm"], n_max=p["n_max"], level_restrict=1))
    geo.build()
    return geo, oracle.Oracle(g, p)


@pytest.mark.parametrize("case", ["c1", "grid32", "grid44"])
def test_restricted_tree_and_values_match_oracle(case):
    g = {"c1": workloads.starfish_c1(),
         "grid32": workloads.small_grid(3, 2, 24, 5000, seed=11),
         "grid44": workloads.starfish_grid(4, 4, 32, n_off=4000, seed=5)}[case]
    geo, orc = _pair(g)
    plain = oracle.Oracle(g, oracle.default_params(g))
    assert orc.nbox > plain.nbox
    check_build(geo, orc)
    for kern in ("S", "D"):
        v, ref = geo.eval(kern, g["density"]), orc.eval(kern, g["density"])
        assert np.abs(v - ref).max() <= 1e-12 * np.abs(ref).max(), (case, kern)
    geo.close()


def test_restricted_tree_sampled_at_scale():
    """An 8 x 8 starfish grid (256 k off-surface targets): tree and lists bit
    for bit, sampled targets of every kind within 1e-12."""
    g = workloads.starfish_grid(8, 8, 64, n_off=1 << 18, seed=2)
    geo, orc = _pair(g, p_qbx=8, p_fmm=15)
    check_build(geo, orc)
    kind, _ = orc.association()
    rng = np.random.default_rng(6)
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
