"""Pins of the oracle's level-restricted tree (Sec. 4.6, remark on
level-restricted quadtrees: adjacent leaves' levels differ by at most one),
checked against brute force over all box pairs rather than the oracle's own
candidate search, plus the tree and list invariants of the unrestricted tree
on the restricted one and the accuracy of the FMM built on it."""
import numpy as np
import pytest

import oracle
import workloads

KEYBITS = 30


def _geoms():
    return {"c1": workloads.starfish_c1(),
            "grid32": workloads.small_grid(3, 2, 24, 5000, seed=11),
            "grid44": workloads.starfish_grid(4, 4, 32, n_off=4000, seed=5)}


@pytest.fixture(scope="module", params=["c1", "grid32", "grid44"])
def pair(request):
    g = _geoms()[request.param]
    plain = oracle.Oracle(g, oracle.default_params(g))
    bal = oracle.Oracle(g, oracle.default_params(g, level_restrict=1))
    return request.param, g, plain, bal


def _geometry(o):
    bx = o.boxes()
    lev = bx["level"].astype(np.int64)
    h = np.left_shift(np.int64(1), KEYBITS - lev)
    cx = (2 * bx["ix"] + 1) * h
    cy = (2 * bx["iy"] + 1) * h
    has_child = np.zeros(o.nbox, bool)
    has_child[bx["parent"][bx["parent"] >= 0]] = True
    return bx, lev, h, cx, cy, has_child


def _eligible_own(o, bx):
    """Particles a box owns that are eligible for its children: sources, point
    targets, and centres whose level L_c exceeds the box's level."""
    _, _, lc = o.centres()
    _, co, _ = o.owners()
    el = bx["nsrc"].astype(np.int64) + bx["ntgt"]
    np.add.at(el, co, (lc > bx["level"][co]).astype(np.int64))
    return el


def _eligible_subtree(o, bx):
    """Particles in a box's subtree eligible at the box's level."""
    so, co, to = o.owners()
    _, _, lc = o.centres()
    el = np.zeros(o.nbox, np.int64)
    par = bx["parent"]
    lev = bx["level"]

    def up(b, ok):
        while b >= 0:
            if ok(lev[b]):
                el[b] += 1
            b = par[b]
    for b in so:
        up(b, lambda l: True)
    for b in to:
        if b >= 0:
            up(b, lambda l: True)
    for c, b in enumerate(co):
        up(b, lambda l, L=lc[c]: L > l)
    return el


def test_restriction_changes_the_tree(pair):
    name, g, plain, bal = pair
    assert bal.nbox > plain.nbox, name


def test_balanced_tree_has_no_violation(pair):
    """No leaf that owns a particle eligible for children (and lies above
    level 30) touches a box two or more levels deeper (closed squares)."""
    name, g, plain, bal = pair
    bx, lev, h, cx, cy, has_child = _geometry(bal)
    el = _eligible_own(bal, bx)
    leaves = np.nonzero(~has_child & (el > 0) & (lev < KEYBITS))[0]
    for a in leaves:
        deep = lev >= lev[a] + 2
        d = np.maximum(np.abs(cx[deep] - cx[a]), np.abs(cy[deep] - cy[a]))
        assert not (d <= h[a] + h[deep]).any(), (name, a)


def test_plain_tree_has_violations(pair):
    """The same check fails on the unrestricted tree (so it has teeth here)."""
    name, g, plain, bal = pair
    bx, lev, h, cx, cy, has_child = _geometry(plain)
    el = _eligible_own(plain, bx)
    bad = 0
    for a in np.nonzero(~has_child & (el > 0))[0]:
        deep = lev >= lev[a] + 2
        d = np.maximum(np.abs(cx[deep] - cx[a]), np.abs(cy[deep] - cy[a]))
        bad += int((d <= h[a] + h[deep]).any())
    assert bad > 0, name


def test_balanced_refines_plain(pair):
    name, g, plain, bal = pair
    bp, bb = plain.boxes(), bal.boxes()
    kp = set(zip(bp["level"].tolist(), bp["ix"].tolist(), bp["iy"].tolist()))
    kb = set(zip(bb["level"].tolist(), bb["ix"].tolist(), bb["iy"].tolist()))
    assert kp <= kb, name


def test_every_extra_subdivision_is_justified(pair):
    """Minimality: a box subdivided although its count does not ask for it
    (at most n_max eligible particles) touches, from outside its own
    subtree, a box two or more levels deeper."""
    name, g, plain, bal = pair
    bx, lev, h, cx, cy, has_child = _geometry(bal)
    el = _eligible_subtree(bal, bx)
    nmax = int(g["n_max"])
    par = bx["parent"]
    forced = np.nonzero(has_child & (el <= nmax))[0]
    assert len(forced) > 0, name

    def descendant(d, b):
        while d >= 0:
            if d == b:
                return True
            d = par[d]
        return False
    for b in forced:
        cand = np.nonzero(lev >= lev[b] + 2)[0]
        d = np.maximum(np.abs(cx[cand] - cx[b]), np.abs(cy[cand] - cy[b]))
        touching = cand[d <= h[b] + h[cand]]
        assert any(not descendant(t, b) for t in touching), (name, b)


def test_balanced_lists_equal_bruteforce(pair):
    name, g, plain, bal = pair
    if name == "grid44":
        pytest.skip("brute-force lists are O(nbox^2); two geometries suffice")
    bal.brute_force_lists()
    A, B = bal.lists(), bal.lists(brute=True)
    for lst in oracle.LISTS:
        for b in range(bal.nbox):
            oa, ia = A[lst]
            ob, ib = B[lst]
            assert sorted(ia[oa[b]:oa[b + 1]]) == sorted(ib[ob[b]:ob[b + 1]]), (lst, b)


def test_balanced_partition_of_interactions(pair):
    """Every (target, source) pair is still conveyed exactly once (case split
    of the Theorem's proof) on the restricted tree."""
    name, g, plain, bal = pair
    if name == "grid44":
        pytest.skip("quadratic check; two geometries suffice")
    bx = bal.boxes()
    so, co, to = bal.owners()
    lev = bx["level"]
    anc = np.full((bal.nsrc, lev.max() + 1), -1, np.int64)
    for s in range(bal.nsrc):
        b = so[s]
        while b >= 0:
            anc[s, lev[b]] = b
            b = bx["parent"][b]
    L = bal.lists()
    rows = lambda lst, b: lst[1][lst[0][b]:lst[0][b + 1]]  # noqa: E731
    for b in sorted(set(co.tolist()) | set(int(t) for t in to if t >= 0)):
        cnt = np.zeros(bal.nsrc, np.int64)
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


def test_balanced_fmm_converges_to_direct_qbx():
    """With p_fmm = 40 the FMM on the restricted tree reproduces direct QBX
    (any dropped or doubled interaction would show)."""
    g = workloads.small_grid(3, 2, 24, 5000, seed=11)
    o = oracle.Oracle(g, oracle.default_params(g, p_qbx=5, p_fmm=40, level_restrict=1))
    for kern in ("S", "D"):
        a, b = o.eval(kern, g["density"]), o.direct(kern, g["density"])
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max(), kern


def test_list3_bounded_on_restricted_tree(pair):
    """Remark: on a level-restricted tree List 3 (close and far) of a leaf
    holds a bounded number of boxes.  Its boxes touch neither the leaf nor
    each other's interiors and lie in the leaf's 3 x 3 neighbourhood at one or
    two levels deeper, so at most 12 x 12 - 6 x 6 = 108 of them."""
    name, g, plain, bal = pair
    bx, lev, h, cx, cy, has_child = _geometry(bal)
    L = bal.lists()
    for b in np.nonzero(~has_child)[0]:
        n = (L["WC"][0][b + 1] - L["WC"][0][b]) + (L["WF"][0][b + 1] - L["WF"][0][b])
        assert n <= 108, (name, b, n)
