"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer results (centre levels, association, tree, owners, all six
interaction lists) must be bit-exact; FP64 values must agree to 1e-12
relative to the oracle's max-norm per output array (the plain-FP64 bar)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Geometry, params_default
    return torch, Geometry, params_default


def _make(g, **kw):
    torch, Geometry, params_default = _gpu()
    p = oracle.default_params(g, **kw)
    geo = Geometry(g, params_default(p_qbx=p["p_qbx"], p_fmm=p["p_fmm"], n_max=p["n_max"],
                                     tf_num=p["tf_num"], tf_den=p["tf_den"], w3_demote=p["w3_demote"],
                                     max_level=p["max_level"], radius_factor=p["radius_factor"],
                                     assoc_slack=p["assoc_slack"]))
    geo.build()
    return geo, oracle.Oracle(g, p)


def _box_keys(bx):
    return list(zip(bx["level"].tolist(), bx["ix"].tolist(), bx["iy"].tolist()))


def check_build(geo, orc):
    """Bit-exact comparison of everything gq_build produces."""
    assert geo.root() == orc.root()
    xg, rg, lg = geo.centres()
    xo, ro, lo = orc.centres()
    assert np.array_equal(xg, xo) and np.array_equal(rg, ro) and np.array_equal(lg, lo)
    kg, cg = geo.association()
    ko, co = orc.association()
    assert np.array_equal(kg, ko) and np.array_equal(cg[kg > 0], co[ko > 0])
    bg, bo = geo.boxes(), orc.boxes()
    kg_, ko_ = _box_keys(bg), _box_keys(bo)
    assert kg_ == ko_, "box sets / numbering differ"
    for k in ("parent", "nsrc", "nctr", "ntgt", "sub_src", "sub_tgt"):
        assert np.array_equal(bg[k], bo[k]), k
    og, oo = geo.owners(), orc.owners()
    for a, b in zip(og, oo):
        assert np.array_equal(a, b)
    Lg, Lo = geo.lists(), orc.lists()
    for name in oracle.LISTS:
        assert np.array_equal(canonical_pairs(*Lg[name]), canonical_pairs(*Lo[name])), name


def canonical_pairs(off, idx):
    """(box, entry) pairs of a CSR list, sorted: equal iff the lists are equal as sets per box."""
    box = np.repeat(np.arange(len(off) - 1), np.diff(off))
    o = np.lexsort((idx, box))
    return np.stack([box[o], idx[o]])


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def c1_pair():
    g = workloads.starfish_c1()
    geo, orc = _make(g)
    return g, geo, orc


def test_c1_build_bit_exact(c1_pair):
    g, geo, orc = c1_pair
    check_build(geo, orc)


@pytest.mark.parametrize("kern", ["S", "D", "SP"])
def test_c1_values(c1_pair, kern):
    g, geo, orc = c1_pair
    v = geo.eval(kern, g["density"])
    ref = orc.eval(kern, g["density"])
    assert rel(v, ref) <= TOL


def test_c1_device_pointers_and_coefficients(c1_pair):
    torch, _, _ = _gpu()
    g, geo, orc = c1_pair
    dens = torch.tensor(g["density"], dtype=torch.float64, device="cuda")
    out = torch.empty(len(g["tgt_xy"]), dtype=torch.float64, device="cuda")
    geo.eval("D", dens, out)
    torch.cuda.synchronize()
    ref, qref = orc.eval("D", g["density"], want_qbx=True)
    assert rel(out.cpu().numpy(), ref) <= TOL
    q = geo.qbx_coefficients()
    assert np.abs(q - qref).max() <= TOL * np.abs(qref).max()
    geo.eval("S", dens, out)
    torch.cuda.synchronize()
    ref, qref = orc.eval("S", g["density"], want_qbx=True)
    q = geo.qbx_coefficients()
    assert np.abs(q[:, 1:] - qref[:, 1:]).max() <= TOL * np.abs(qref[:, 1:]).max()
    assert np.abs(q[:, 0].real - qref[:, 0].real).max() <= TOL * np.abs(qref[:, 0].real).max()


@pytest.mark.parametrize("case", [
    dict(nx=2, ny=2, n_panels=16, n_off=3000, seed=7),
    dict(nx=3, ny=2, n_panels=24, n_off=5000, seed=11, on_surface="up"),
    dict(nx=4, ny=3, n_panels=20, n_off=20000, seed=13, p_qbx=8, p_fmm=15),
])
def test_small_grids(case):
    g = workloads.small_grid(**case)
    geo, orc = _make(g)
    check_build(geo, orc)
    for kern in ("S", "D"):
        v = geo.eval(kern, g["density"])
        ref = orc.eval(kern, g["density"])
        assert rel(v, ref) <= TOL, kern


@pytest.mark.parametrize("kw", [dict(p_qbx=1, p_fmm=1), dict(p_qbx=16, p_fmm=30), dict(n_max=1),
                                dict(n_max=4000), dict(tf_num=0, tf_den=1), dict(w3_demote=1),
                                dict(p_qbx=3, p_fmm=20, n_max=8)])
def test_parameter_edges(kw):
    g = workloads.small_grid(2, 1, 12, 800, seed=21)
    geo, orc = _make(g, **kw)
    check_build(geo, orc)
    for kern in ("S", "D"):
        v = geo.eval(kern, g["density"])
        ref = orc.eval(kern, g["density"])
        assert rel(v, ref) <= TOL, (kern, kw)


def test_no_targets():
    torch, Geometry, params_default = _gpu()
    g = workloads.small_grid(1, 1, 8, 0, seed=3)
    g["tgt_xy"] = np.zeros((0, 2))
    g["tgt_onsurf"] = np.zeros(0, np.int32)
    geo = Geometry(g)
    geo.build()
    out = geo.eval("S", g["density"])
    assert out.shape == (0,)


def test_unit_circle_closed_form_gpu():
    _gpu()
    g = workloads.unit_circle(32, n_off=50, off_radii=[0.5, 0.95, 1.05, 2.0])
    geo, orc = _make(g, p_qbx=8, p_fmm=15)
    t = g["tgt_xy"]
    rho = np.hypot(t[:, 0], t[:, 1])
    th = np.arctan2(t[:, 1], t[:, 0])
    on = g["tgt_onsurf"] >= 0
    rho = np.where(on, 1.0, rho)
    S = np.where(rho <= 1.0, rho ** 3, rho ** -3.0) * np.cos(3 * th) / 6
    v = geo.eval("S", np.cos(3 * g["base_theta"]))
    assert np.abs(v - S).max() < 2e-8


@pytest.mark.parametrize("seed", [0, 1])
def test_repeat_and_alternate(c1_pair, seed):
    """Evaluations reuse the build; results do not depend on earlier calls."""
    g, geo, orc = c1_pair
    rng = np.random.default_rng(seed)
    mu = rng.normal(size=len(g["density"]))
    a = geo.eval("S", mu)
    geo.eval("D", g["density"])
    b = geo.eval("S", mu)
    assert np.array_equal(a, b)
    assert rel(a, orc.eval("S", mu)) <= TOL


def test_invalid_on_surface_index_leaves_no_targets():
    """An on-surface index outside [-1, nbase) is refused, the geometry then has
    no targets (build refused) until a valid set is given."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Geometry, GigaQBXError, params_default
    g = workloads.starfish_c1()
    geo = Geometry(g, params_default(p_qbx=5, p_fmm=10, n_max=32))
    on = np.arange(len(g["base_xy"]), dtype=np.int32)
    bad = on.copy()
    bad[7] = len(on)
    with pytest.raises(GigaQBXError):
        geo.set_targets(g["base_xy"], bad)
    with pytest.raises(GigaQBXError):
        geo.build()
    geo.set_targets(g["base_xy"], on)
    geo.build()
    v = geo.eval("S", g["density"])
    assert np.isfinite(v).all() and len(v) == len(on)
    geo.close()


@pytest.mark.parametrize("scale_exp", [-100, 0, 100])
def test_density_scaling_is_exact(scale_exp):
    """The potentials are linear in the density.  A power-of-two scale 2^k
    scales every FP64 operation exactly, and the direct kernels' FP32 copies
    of the strengths are rebased to the largest strength of the call.  So
    S and D of 2^k mu are 2^k times those of mu, bit for bit, even where
    2^k takes the strengths far outside FP32's range.  The oracle agrees at
    1e-12."""
    g = workloads.small_grid(2, 2, 16, 3000, seed=7)
    geo, orc = _make(g, p_qbx=5, p_fmm=10)
    mu = g["density"]
    for kern in ("S", "D"):
        base = geo.eval(kern, mu)
        v = geo.eval(kern, np.ldexp(mu, scale_exp))
        assert np.array_equal(v, np.ldexp(base, scale_exp)), kern
        ref = orc.eval(kern, mu)
        assert np.abs(base - ref).max() <= TOL * np.abs(ref).max(), kern
