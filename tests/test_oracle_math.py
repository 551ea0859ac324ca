"""Pins of the oracle's arithmetic against mathematics that does not come
from the oracle itself: exact expansions of single sources, the error bounds
of Lemmas 1-3 (Sec. 3.2), closed forms on the unit circle, Green's identity
(Sec. 5.1) and the accuracy Theorem (Sec. 4.5)."""
import numpy as np
import pytest

import oracle
import workloads

RNG = np.random.default_rng(1234)


def _phi_S(z, y):              # complex potential of a unit S source at y
    return np.log(z - y)


# ------------------------------------------------------------------ single operators
@pytest.mark.parametrize("kernel", ["S", "D"])
def test_p2m_matches_direct_far_field(kernel):
    c = 0.3 + 0.1j
    ys = c + 0.1 * (RNG.random(20) - 0.5 + 1j * (RNG.random(20) - 0.5))
    st = RNG.normal(size=20) + (1j * RNG.normal(size=20) if kernel == "D" else 0)
    p = 30
    a = oracle.op_p2m(kernel, p, c, ys, st)
    ts = c + 2.0 * np.exp(2j * np.pi * RNG.random(7))
    got = oracle.op_eval_mpole(p, c, a, ts)
    if kernel == "S":
        ref = (st[None, :] * np.log(ts[:, None] - ys[None, :])).sum(1)
    else:
        ref = (st[None, :] / (ys[None, :] - ts[:, None])).sum(1)
    assert np.abs(got.real - ref.real).max() < 1e-13 * np.abs(st).sum()


@pytest.mark.parametrize("kernel", ["S", "D"])
def test_m2m_exact(kernel):
    """M2M keeps the retained coefficients exact (Sec. 3.2: the FMM forgets
    intermediate translations): shifting a P2M expansion equals P2M about
    the new centre, coefficient by coefficient."""
    c_old, c_new = 0.25 + 0.25j, 0.5 + 0.5j
    ys = c_old + 0.2 * (RNG.random(15) - 0.5 + 1j * (RNG.random(15) - 0.5))
    st = RNG.normal(size=15) * (1 + (1j if kernel == "D" else 0))
    p = 12
    shifted = oracle.op_m2m(p, c_old, c_new, oracle.op_p2m(kernel, p, c_old, ys, st))
    direct = oracle.op_p2m(kernel, p, c_new, ys, st)
    scale = np.abs(direct).max()
    assert np.abs(shifted - direct).max() <= 1e-13 * scale


def test_l2l_is_exact_recentering():
    c_old, c_new = 0.0, 0.11 - 0.07j
    b = RNG.normal(size=11) + 1j * RNG.normal(size=11)
    shifted = oracle.op_l2l(10, 10, c_old, c_new, b)
    ts = c_new + 0.2 * np.exp(2j * np.pi * RNG.random(9))
    v1 = oracle.op_eval_local(10, c_old, b, ts)
    v2 = oracle.op_eval_local(10, c_new, shifted, ts)
    assert np.abs(v1 - v2).max() < 1e-14 * np.abs(v1).max()


def test_p2l_local_is_taylor_of_potential():
    c = 0.0
    y = 1.0 + 0.5j
    b = oracle.op_p2l("S", 40, c, [y], [1.0])
    ts = 0.3 * np.exp(2j * np.pi * RNG.random(8))
    got = oracle.op_eval_local(40, c, b, ts)
    assert np.abs(got.real - np.log(np.abs(ts - y))).max() < 1e-13
    bd = oracle.op_p2l("D", 40, c, [y], [0.3 + 0.4j])
    gd = oracle.op_eval_local(40, c, bd, ts)
    assert np.abs(gd - (0.3 + 0.4j) / (y - ts)).max() < 1e-13


def _lemma_geometry(lam, cc, r=1.0):
    """A unit source in B(z0, lam r) with |z0| = (cc + 1 + lam) r, an inner
    point z with |z| < r and y with |y - z| <= r - |z| (Lemma 1 setup)."""
    ang = 2 * np.pi * RNG.random()
    z0 = (cc + 1 + lam) * r * np.exp(1j * ang)
    src = z0 + lam * r * np.sqrt(RNG.random()) * np.exp(2j * np.pi * RNG.random())
    z = 0.6 * r * np.sqrt(RNG.random()) * np.exp(2j * np.pi * RNG.random())
    y = z + (r - abs(z)) * np.exp(2j * np.pi * RNG.random())
    return z0, src, z, y


@pytest.mark.parametrize("p,q", [(3, 3), (6, 5), (10, 8), (15, 8)])
def test_lemma1_m2qbxl_bound(p, q):
    lam, cc = 1.0, 2.0
    omega = 1.0 / (1.0 + cc / lam)
    bound = (q + 1) / (p + 1) * omega ** (p + 1) / (1 - omega)
    worst = 0.0
    for _ in range(40):
        z0, src, z, y = _lemma_geometry(lam, cc)
        a = oracle.op_p2m("S", p, z0, [src], [1.0])
        bt = oracle.op_m2l(p, q, z0, z, a)                   # truncated multipole -> local at z
        be = oracle.op_p2l("S", q, z, [src], [1.0])          # exact local at z
        err = abs((oracle.op_eval_local(q, z, bt, [y]) - oracle.op_eval_local(q, z, be, [y]))[0].real)
        worst = max(worst, err)
    assert worst <= bound
    assert worst > 1e-3 * bound * omega      # the bound is not vacuous for this test


@pytest.mark.parametrize("p,q", [(3, 3), (8, 5), (15, 8)])
def test_lemma2_l2qbxl_bound(p, q):
    cc = 2.0
    alpha = 1.0 / (1.0 + cc)
    bound = (q + 1) / (p + 1) * alpha ** (p + 1) / (1 - alpha)
    for _ in range(40):
        z0 = (cc + 1) * np.exp(2j * np.pi * RNG.random())
        z = 0.6 * np.sqrt(RNG.random()) * np.exp(2j * np.pi * RNG.random())
        y = z + (1 - abs(z)) * np.exp(2j * np.pi * RNG.random())
        b0 = oracle.op_p2l("S", p, 0.0, [z0], [1.0])
        bt = oracle.op_l2l(p, q, 0.0, z, b0)
        be = oracle.op_p2l("S", q, z, [z0], [1.0])
        err = abs((oracle.op_eval_local(q, z, bt, [y]) - oracle.op_eval_local(q, z, be, [y]))[0].real)
        assert err <= bound


@pytest.mark.parametrize("p,q", [(4, 3), (10, 5), (15, 8)])
def test_lemma3_m2l2qbxl_bound(p, q):
    lam, cc = 1.0, 3.0
    alpha, omega = 1.0 / (1.0 + cc), 1.0 / (1.0 + cc / lam)
    bound = (q + 1) * omega ** (p + 1) / (1 - omega) + (q + 1) / (p + 1) * alpha ** (p + 1) / (1 - alpha)
    for _ in range(40):
        z0, src, z, y = _lemma_geometry(lam, cc)
        a = oracle.op_p2m("S", p, z0, [src], [1.0])
        l0 = oracle.op_m2l(p, p, z0, 0.0, a)
        bt = oracle.op_l2l(p, q, 0.0, z, l0)
        be = oracle.op_p2l("S", q, z, [src], [1.0])
        err = abs((oracle.op_eval_local(q, z, bt, [y]) - oracle.op_eval_local(q, z, be, [y]))[0].real)
        assert err <= bound


def test_m2l_sign_of_log_term():
    """The a_0 term of M2L: log(z) about y has Taylor coefficients
    (-1)^(m+1) / (m y^m).  A pure a_0 = 1 multipole must reproduce log(z)."""
    p = 20
    a = np.zeros(p + 1, complex)
    a[0] = 1.0
    b = oracle.op_m2l(p, p, 0.0, 3.0 + 1.0j, a)
    ts = 3.0 + 1.0j + 0.5 * np.exp(2j * np.pi * RNG.random(5))
    v = oracle.op_eval_local(p, 3.0 + 1.0j, b, ts)
    assert np.abs(v.real - np.log(np.abs(ts))).max() < 1e-9


# ------------------------------------------------------------------ upsampling
def test_upsample_exact_for_polynomials(c1_oracle, c1):
    o = c1_oracle
    nb, nu = c1["nb"], c1["nu"]
    rb, ru = c1["ref_b"], c1["ref_u"]
    coef = RNG.normal(size=nb)
    mu_b = np.tile(np.polynomial.legendre.legval(rb, coef), c1["npanels"])
    mu_u = o.upsample(mu_b)
    ref = np.tile(np.polynomial.legendre.legval(ru, coef), c1["npanels"])
    assert np.abs(mu_u - ref).max() < 1e-11 * np.abs(ref).max()


# ------------------------------------------------------------------ closed forms
@pytest.fixture(scope="module")
def circle():
    g = workloads.unit_circle(32, n_off=40, off_radii=[0.5, 0.93, 1.07, 1.6])
    o = oracle.Oracle(g, oracle.default_params(p_qbx=8, p_fmm=15))
    return g, o


def _closed_forms(g, k):
    t = g["tgt_xy"]
    rho = np.hypot(t[:, 0], t[:, 1])
    th = np.arctan2(t[:, 1], t[:, 0])
    on = g["tgt_onsurf"] >= 0
    rho = np.where(on, 1.0, rho)
    inside = rho < 1.0
    S = np.where(inside | on, rho ** k, rho ** -k) * np.cos(k * th) / (2 * k)
    D = np.where(on, 0.0, np.where(inside, -0.5 * rho ** k, 0.5 * rho ** -k)) * np.cos(k * th)
    D1 = np.where(on, -0.5, np.where(inside, -1.0, 0.0))
    S1 = np.where(inside | on, 0.0, -np.log(rho))
    return S, D, D1, S1


@pytest.mark.parametrize("which", ["direct", "eval"])
def test_unit_circle_closed_forms(circle, which):
    g, o = circle
    k = 3
    mu_k = np.cos(k * g["base_theta"])
    one = np.ones_like(mu_k)
    S, D, D1, S1 = _closed_forms(g, k)
    f = o.direct if which == "direct" else o.eval
    for kern, mu, ref in (("S", mu_k, S), ("D", mu_k, D), ("D", one, D1), ("S", one, S1)):
        v = f(kern, mu)
        assert np.abs(v - ref).max() < 2e-8, (kern, np.abs(v - ref).max())


@pytest.mark.parametrize("n_panels", [16, 32, 48])
def test_unit_circle_centres(n_panels):
    """Centre placement (Sec. 2.2.2) on the unit circle, where every panel of
    n equal panels has arc length 2 pi / n: with centres half a panel length
    off the curve (the workload's radius), centre 2i lies on the ray of base
    node i at distance 1 - pi/n (interior) and centre 2i+1 at 1 + pi/n
    (exterior), both with radius pi/n.  Fixes the reading of the expansion
    radius (full arc length times 1/2, not half of the half-length h_k)."""
    g = workloads.unit_circle(n_panels)
    o = oracle.Oracle(g, oracle.default_params(p_qbx=4, p_fmm=8))
    xy, r, _ = o.centres()
    nb = len(g["base_xy"])
    assert len(r) == 2 * nb
    h = np.pi / n_panels
    assert np.abs(r - h).max() < 1e-13
    th = np.arctan2(g["base_xy"][:, 1], g["base_xy"][:, 0])
    for side, rad in ((0, 1.0 - h), (1, 1.0 + h)):
        c = xy[side::2]
        assert np.abs(np.hypot(c[:, 0], c[:, 1]) - rad).max() < 1e-13, side
        ang = np.angle(np.exp(1j * (np.arctan2(c[:, 1], c[:, 0]) - th)))
        assert np.abs(ang).max() < 1e-12, side


def test_unit_circle_qbx_order_convergence():
    """Error of on/near-surface values drops with the QBX order (truncation
    error, eq. qbx-truncation-estimate)."""
    g = workloads.unit_circle(32, n_off=40, off_radii=[1.07])
    errs = []
    for q in (2, 4, 8):
        o = oracle.Oracle(g, oracle.default_params(p_qbx=q, p_fmm=20))
        S = _closed_forms(g, 5)[0]
        errs.append(np.abs(o.eval("S", np.cos(5 * g["base_theta"])) - S).max())
    assert errs[0] > 10 * errs[1] > 100 * errs[2]


# ------------------------------------------------------------------ Green's identity
def test_green_identity_starfish(c1_oracle, c1):
    """S(d_n u) - D(u) = u/2 on the curve for u harmonic inside (Sec. 5.1)."""
    o = c1_oracle
    x = c1["base_xy"]
    n = c1["base_n"]
    x0 = np.array([2.0, 1.0])
    d = x - x0
    u = 0.5 * np.log((d ** 2).sum(1))
    dn_u = (n * d).sum(1) / (d ** 2).sum(1)
    res = o.eval("S", dn_u) - o.eval("D", u) - 0.5 * u
    rel = np.abs(res).max() / np.abs(u).max()
    assert rel < 1e-6, rel
    # and the unaccelerated QBX residual is of the same size
    res1 = o.direct("S", dn_u) - o.direct("D", u) - 0.5 * u
    assert np.abs(res1).max() / np.abs(u).max() < 1e-6


# ------------------------------------------------------------------ Theorem
def _theorem_bound(A, p, q, tf=0.9):
    alpha = (tf + np.sqrt(2)) / (6 - np.sqrt(2))
    w3 = 3 * A / (3 - np.sqrt(2)) * (q + 1) / (p + 1) * (np.sqrt(2) / 3) ** (p + 1)
    v2 = A / (1 - alpha) * (q + 1) * (1 + 1 / (p + 1)) * alpha ** (p + 1)
    return (2 * w3 + v2) / (2 * np.pi)


@pytest.mark.parametrize("fix,geom", [("c1_oracle", "c1"), ("small_oracle", "small")])
def test_fmm_within_theorem_bound(fix, geom, request):
    o, g = request.getfixturevalue(fix), request.getfixturevalue(geom)
    mu = g["density"]
    A = np.abs(g["up_w"] * o.upsample(mu)).sum()
    v2 = o.eval("S", mu)
    v1 = o.direct("S", mu)
    kind, _ = o.association()
    qbx = kind > 0
    bound = _theorem_bound(A, o.params["p_fmm"], o.params["p_qbx"])
    assert np.abs(v2 - v1)[qbx].max() <= bound
    # point targets: a (loose) FMM bound for point potentials
    if (~qbx).any():
        assert np.abs(v2 - v1)[~qbx].max() <= bound


def test_fmm_converges_to_direct_qbx(c1):
    """With a high FMM order the accelerated result reaches unaccelerated
    QBX to near rounding: any dropped or doubled interaction would show."""
    o = oracle.Oracle(c1, oracle.default_params(c1, p_fmm=40))
    for kern in ("S", "D"):
        v2, q2 = o.eval(kern, c1["density"], want_qbx=True)
        v1, q1 = o.direct(kern, c1["density"], want_qbx=True)
        assert np.abs(v2 - v1).max() < 1e-11 * np.abs(v1).max(), kern
        # coefficients m >= 1 agree too (constant term: only its real part is defined)
        assert np.abs(q2[:, 1:] - q1[:, 1:]).max() < 1e-10 * np.abs(q1[:, 1:]).max()
        assert np.abs(q2[:, 0].real - q1[:, 0].real).max() < 1e-10 * np.abs(q1[:, 0].real).max()


def test_threads_do_not_change_results(c1):
    """The OpenMP evaluation loops sum every output in the serial order: O1
    and O2 values and QBX coefficients are the same bits for 1 and 4 threads."""
    g = workloads.small_grid(2, 2, 16, 3000, seed=7)
    o = oracle.Oracle(g, oracle.default_params(p_qbx=5, p_fmm=10))
    mu = np.random.default_rng(2).normal(size=len(g["density"]))
    res = {}
    for nt in (1, 4):
        oracle.set_threads(nt)
        try:
            res[nt] = [o.eval(k, mu, want_qbx=True) for k in ("S", "D")] + [o.direct("S", mu)]
        finally:
            oracle.set_threads(1)
    for a, b in zip(res[1], res[4]):
        for x, y in zip(a if isinstance(a, tuple) else (a,), b if isinstance(b, tuple) else (b,)):
            assert np.array_equal(x, y)
