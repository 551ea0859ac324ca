"""gq_apply: the operator identity * mu + K mu at the base nodes (K = S, D,
S'), as the second-kind equation of Sec. 1 applies it, compared with the
FP64 oracle's Stages 1-8 (O2) at the base nodes as two-sided targets within
1e-12 relative, with host and device arrays, on geometries whose own target
set is the base nodes or a different one (off-surface point targets)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _with_base_targets(g):
    """The workload's targets followed by the base nodes as on-surface
    targets.  On-surface (QBX) targets are not tree particles, so the oracle
    builds the same tree as the geometry with the workload's targets alone."""
    g2 = dict(g)
    nb = len(g["base_xy"])
    g2["tgt_xy"] = np.ascontiguousarray(np.concatenate([g["tgt_xy"], g["base_xy"]]))
    g2["tgt_onsurf"] = np.ascontiguousarray(np.concatenate([g["tgt_onsurf"], np.arange(nb, dtype=np.int32)]))
    return g2, len(g["tgt_xy"])


@pytest.mark.parametrize("case", ["c1", "grid_points"])
def test_apply_matches_oracle(case):
    torch = _torch()
    from paper_1801_04070_gb300 import Geometry, params_default
    g = workloads.starfish_c1() if case == "c1" else workloads.small_grid(3, 2, 24, 8000, seed=11)
    prm = dict(p_qbx=6, p_fmm=12, n_max=32)
    geo = Geometry(g, params_default(**prm))
    geo.build()
    assert case == "c1" or geo.npt > 0
    g2, off = _with_base_targets(g)
    o = oracle.Oracle(g2, oracle.default_params(**prm))
    rng = np.random.default_rng(3)
    mu = rng.normal(size=len(g["base_xy"]))
    for kern in ("S", "D", "SP"):
        ref = o.eval(kern, mu)[off:]
        scale = np.abs(ref).max()
        for ident in (0.0, -0.5):
            want = ident * mu + ref
            v = geo.apply(kern, mu, identity=ident)                      # host arrays
            assert np.abs(v - want).max() <= 1e-12 * scale, (kern, ident)
            dm = torch.tensor(mu, dtype=torch.float64, device="cuda")
            dv = torch.full_like(dm, float("nan"))
            geo.apply(kern, dm, dv, identity=ident)                     # device arrays
            torch.cuda.synchronize()
            assert np.abs(dv.cpu().numpy() - want).max() <= 1e-12 * scale, (kern, ident)
    geo.close()


def test_apply_equals_eval_at_base_targets():
    """With the base nodes as the geometry's targets, gq_apply(K, 0) and
    gq_eval(K) run the same kernels on the same tree: equal bit for bit."""
    _torch()
    from paper_1801_04070_gb300 import Geometry, params_default
    g = workloads.starfish_c1()
    geo = Geometry(g, params_default(p_qbx=5, p_fmm=10, n_max=32))
    geo.set_targets(g["base_xy"], np.arange(len(g["base_xy"]), dtype=np.int32))
    geo.build()
    mu = np.cos(3 * g["base_theta"]) + 0.1
    for kern in ("S", "D", "SP"):
        assert np.array_equal(geo.apply(kern, mu), geo.eval(kern, mu)), kern
    geo.close()


def test_apply_rejects_bad_calls():
    _torch()
    from paper_1801_04070_gb300 import GigaQBXError, Geometry, params_default
    g = workloads.starfish_c1()
    geo = Geometry(g, params_default())
    with pytest.raises(GigaQBXError):
        geo.apply("S", np.ones(len(g["base_xy"])))     # before gq_build
    geo.build()
    with pytest.raises(GigaQBXError):
        geo.apply(7, np.ones(len(g["base_xy"])))
    geo.close()
