"""Pins of the oracle's disk-shaped target confinement region (the l2 TCR of
the appendix corrigendum; reading: TCR(b) is the closed l2 disk of radius
|b|(1 + t_f) about b's centre, and every definition of Sec. 4.3 -- a centre
stays where its disk fits the TCR, adequate separation as an l-inf distance
between sets -- is kept).

The separation relations are checked against the geometry itself (the
l-inf distance between a square and a disk, minimised over a fine sampling
of the circle), not against their own algebra; the centre levels against
brute-force containment; the lists on the disk tree against the brute-force
lists and the partition of interactions; the FMM on it against direct QBX."""
import numpy as np
import pytest

import oracle
import workloads

KEYBITS = 30
TN, TD = 9, 10
TF = TN / TD


def _centre(level, ix, iy):
    h = float(1 << (KEYBITS - level))
    return np.array([(2 * ix + 1) * h, (2 * iy + 1) * h]), h


def _linf_square_disk(cs, hs, cd, rho, n=400_000):
    """l-inf distance between the closed square S(cs, hs) and the closed disk
    D(cd, rho): the smallest l-inf distance from cs to a point of D, less hs
    (0 when they meet).  The distance from cs is convex, so outside the disk
    its minimum lies on the circle, sampled at n angles."""
    if np.hypot(*(cs - cd)) <= rho:
        return 0.0
    th = np.linspace(0.0, 2 * np.pi, n, endpoint=False)
    y = cd[:, None] + rho * np.stack([np.cos(th), np.sin(th)])
    m = np.abs(y - cs[:, None]).max(0).min()
    return max(0.0, m - hs)


def _pairs(rng, n):
    out = []
    while len(out) < n:
        la = int(rng.integers(3, 9))
        lb = int(rng.integers(max(2, la - 3), min(10, la + 3)))
        ca = rng.integers(8, 40, size=2) << 3
        # b near a: within a few boxes of the coarser size
        hb = 1 << (KEYBITS - lb)
        ha = 1 << (KEYBITS - la)
        span = 12 * max(ha, hb)
        cx, cy = (2 * ca + 1) * ha
        bx = (cx + rng.integers(-span, span)) // (2 * hb)
        by = (cy + rng.integers(-span, span)) // (2 * hb)
        out.append(((la, int(ca[0]), int(ca[1])), (lb, int(bx), int(by))))
    return out


@pytest.mark.parametrize("which", [0, 1])
def test_disk_separation_is_the_geometric_relation(which):
    """which 0: a |> TCR(b) iff dist_inf(a, disk TCR(b)) >= 2|a| (Def. 5 with
    the disk); which 1: TCR(a) |> b iff dist_inf(disk TCR(a), b) >= 2|a|(1+t_f)
    (Def. 8 with the disk).  Pairs within 1e-4 of a tie are skipped (the
    sampling's resolution); both outcomes must occur."""
    rng = np.random.default_rng(20 + which)
    seen = {True: 0, False: 0}
    for a, b in _pairs(rng, 400):
        ca, ha = _centre(*a)
        cb, hb = _centre(*b)
        if which == 0:
            dist, need, scale = _linf_square_disk(ca, ha, cb, hb * (1 + TF)), 2 * ha, ha
        else:
            dist, need, scale = _linf_square_disk(cb, hb, ca, ha * (1 + TF)), 2 * ha * (1 + TF), ha
        if abs(dist - need) <= 1e-4 * scale:
            continue
        want = dist >= need
        assert oracle.sep_test(1, TN, TD, which, a, b) == want, (a, b, dist, need)
        seen[want] += 1
    assert seen[True] > 20 and seen[False] > 20, seen


def test_square_separation_is_the_geometric_relation():
    """The same check for the square TCR (the paper's Def. 5 and Def. 8):
    the l-inf distance between squares is the centre distance less both
    half-widths."""
    rng = np.random.default_rng(7)
    for a, b in _pairs(rng, 300):
        ca, ha = _centre(*a)
        cb, hb = _centre(*b)
        d = np.abs(ca - cb).max()
        assert oracle.sep_test(0, TN, TD, 0, a, b) == (d - ha - hb * (1 + TF) >= 2 * ha)
        assert oracle.sep_test(0, TN, TD, 1, a, b) == (d - ha * (1 + TF) - hb >= 2 * ha * (1 + TF))


def test_disk_relations_are_monotone():
    """Sec. 4.3's monotonicity, which the list construction relies on, holds
    for the disk TCR (t_f = 0.9 >= sqrt 2 - 1, so a child's disk lies in its
    parent's): a separated box's children are separated, for both relations."""
    rng = np.random.default_rng(5)
    n = 0
    for a, b in _pairs(rng, 300):
        for which in (0, 1):
            if not oracle.sep_test(1, TN, TD, which, a, b):
                continue
            for q in range(4):
                ch = (a[0] + 1, 2 * a[1] + (q & 1), 2 * a[2] + (q >> 1))
                assert oracle.sep_test(1, TN, TD, which, ch, b), (which, a, b, ch)
                n += 1
    assert n > 100


@pytest.fixture(scope="module", params=["c1", "grid32"])
def disk(request):
    g = {"c1": workloads.starfish_c1(), "grid32": workloads.small_grid(3, 2, 24, 5000, seed=11)}[request.param]
    return (request.param, g, oracle.Oracle(g, oracle.default_params(g, tcr_shape=1)),
            oracle.Oracle(g, oracle.default_params(g)))


def test_centre_disks_fit_their_disk_tcr(disk):
    """Every centre's disk lies in the disk TCR of the level-L_c box on its
    key path and not in the next level's (unless L_c is the deepest level);
    the disk TCR lies in the square one, so no centre sits deeper than with
    the square TCR.  Cases within 1e-9 of a tie are skipped."""
    name, g, od, osq = disk
    xy, r, lc = od.centres()
    _, _, lc_sq = osq.centres()
    rt = od.root()
    lo = np.array([rt["lo_x"], rt["lo_y"]])

    def slack(c, level):
        hb = rt["H"] / 2 ** level
        k = np.floor((xy[c] - lo) / (2 * hb))
        cb = lo + (2 * k + 1) * hb
        return hb * (1 + TF) - (np.hypot(*(xy[c] - cb)) + r[c]), hb

    checked = 0
    for c in range(len(r)):
        s, hb = slack(c, lc[c])
        if abs(s) > 1e-9 * hb:
            assert s >= 0, (name, c)
            checked += 1
        if lc[c] < 30:
            s, hb = slack(c, lc[c] + 1)
            if abs(s) > 1e-9 * hb:
                assert s < 0, (name, c)
    assert checked > 0.9 * len(r)
    assert (lc <= lc_sq).all() and (lc < lc_sq).any(), name


def test_disk_lists_equal_bruteforce(disk):
    name, g, od, _ = disk
    od.brute_force_lists()
    A, B = od.lists(), od.lists(brute=True)
    for lst in oracle.LISTS:
        oa, ia = A[lst]
        ob, ib = B[lst]
        for b in range(od.nbox):
            assert sorted(ia[oa[b]:oa[b + 1]]) == sorted(ib[ob[b]:ob[b + 1]]), (name, lst, b)


def test_disk_partition_of_interactions(disk):
    """Every (target box, source) pair is conveyed exactly once by the lists of
    the box and its ancestors (the case split of the Theorem's proof)."""
    name, g, od, _ = disk
    bx = od.boxes()
    so, co, to = od.owners()
    lev = bx["level"]
    anc = np.full((od.nsrc, lev.max() + 1), -1, np.int64)
    for s in range(od.nsrc):
        b = so[s]
        while b >= 0:
            anc[s, lev[b]] = b
            b = bx["parent"][b]
    L = od.lists()
    rows = lambda lst, b: lst[1][lst[0][b]:lst[0][b + 1]]  # noqa: E731
    for b in sorted(set(co.tolist()) | set(int(t) for t in to if t >= 0)):
        cnt = np.zeros(od.nsrc, np.int64)
        for nm in ("U", "WC", "XC"):
            for d in rows(L[nm], b):
                cnt += (so == d)
        for d in rows(L["WF"], b):
            cnt += (anc[:, lev[d]] == d)
        w = b
        while w >= 0:
            for d in rows(L["V"], w):
                cnt += (anc[:, lev[d]] == d)
            for d in rows(L["XF"], w):
                cnt += (so == d)
            w = bx["parent"][w]
        assert (cnt == 1).all(), (name, b)


def test_disk_fmm_converges_to_direct_qbx():
    """p_fmm = 40 on the disk tree reproduces direct QBX (a dropped or doubled
    interaction, or an expansion used outside its disk of convergence, would
    show)."""
    g = workloads.small_grid(3, 2, 24, 5000, seed=11)
    o = oracle.Oracle(g, oracle.default_params(g, p_qbx=5, p_fmm=40, tcr_shape=1))
    for kern in ("S", "D"):
        a, b = o.eval(kern, g["density"]), o.direct(kern, g["density"])
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max(), kern


def test_disk_fmm_error_decays_with_order():
    """At moderate orders the acceleration error on the disk tree falls with
    p_fmm like the square one's and stays within a factor of it."""
    g = workloads.small_grid(3, 2, 24, 5000, seed=11)
    errs = {}
    for shape in (0, 1):
        for p in (6, 12):
            o = oracle.Oracle(g, oracle.default_params(g, p_qbx=5, p_fmm=p, tcr_shape=shape))
            a, b = o.eval("S", g["density"]), o.direct("S", g["density"])
            errs[shape, p] = np.abs(a - b).max() / np.abs(b).max()
    print(errs)
    for shape in (0, 1):
        assert errs[shape, 12] < errs[shape, 6] / 10
    assert errs[1, 12] <= 100 * errs[0, 12] and errs[0, 12] <= 100 * errs[1, 12]
