"""Pins of the oracle's tree and interaction lists (Sec. 4.3) against
brute force, the paper's printed bounds and the interaction partition that
the accuracy proof relies on (Sec. 4.5, proof of the Theorem)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _rows(lst, b):
    off, idx = lst
    return idx[off[b]:off[b + 1]]


@pytest.mark.parametrize("fix", ["c1_oracle", "small_oracle"])
def test_o2_lists_equal_bruteforce(fix, request):
    o = request.getfixturevalue(fix)
    A, B = o.lists(), o.lists(brute=True)
    for name in oracle.LISTS:
        for b in range(o.nbox):
            ra, rb = sorted(_rows(A[name], b)), sorted(_rows(B[name], b))
            assert ra == rb, (name, b)
            assert len(set(ra)) == len(ra), ("duplicate entry", name, b)


def test_o2_lists_equal_bruteforce_onsurface_up():
    g = workloads.small_grid(3, 2, 24, 4000, seed=11, on_surface="up")
    o = oracle.Oracle(g)
    o.brute_force_lists()
    A, B = o.lists(), o.lists(brute=True)
    for name in oracle.LISTS:
        for b in range(o.nbox):
            assert sorted(_rows(A[name], b)) == sorted(_rows(B[name], b)), (name, b)


@pytest.mark.parametrize("fix", ["c1_oracle", "small_oracle"])
def test_touching_same_level_leaves_in_list1(fix, request):
    """Def. 1 from box indices alone: a same-level leaf with sources whose
    square shares an edge or a corner with a target-owning box b (index
    offsets within one) belongs to List 1 of b.  This pins the adjacency
    reading (closed squares that touch are adjacent) independently of the
    distance test the list code uses."""
    o = request.getfixturevalue(fix)
    bx = o.boxes()
    lists = o.lists()
    n = o.nbox
    has_child = np.zeros(n, bool)
    has_child[bx["parent"][bx["parent"] >= 0]] = True
    key = {(int(bx["level"][d]), int(bx["ix"][d]), int(bx["iy"][d])): d for d in range(n)}
    checked = 0
    for b in range(n):
        if bx["nctr"][b] + bx["ntgt"][b] == 0:
            continue
        u = set(_rows(lists["U"], b).tolist())
        l, x, y = int(bx["level"][b]), int(bx["ix"][b]), int(bx["iy"][b])
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                d = key.get((l, x + dx, y + dy))
                if d is None or d == b or has_child[d] or bx["sub_src"][d] == 0:
                    continue
                assert d in u, (b, d)
                checked += 1
    assert checked > 0


def _ancestor_table(o):
    bx = o.boxes()
    so, co, to = o.owners()
    nlev = bx["level"].max() + 1
    anc = np.full((o.nsrc, nlev), -1, np.int64)
    for s in range(o.nsrc):
        b = so[s]
        while b >= 0:
            anc[s, bx["level"][b]] = b
            b = bx["parent"][b]
    return bx, so, co, to, anc


@pytest.mark.parametrize("fix", ["c1_oracle", "small_oracle"])
def test_partition_of_interactions(fix, request):
    """Every (target, source) pair is conveyed exactly once: directly
    (List 1, 3 close, 4 close), through a List 3 far multipole, or through
    the box local expansion fed by List 2 / List 4 far of the target box and
    its ancestors (case split of the Theorem's proof)."""
    o = request.getfixturevalue(fix)
    bx, so, co, to, anc = _ancestor_table(o)
    L = o.lists()
    lev = bx["level"]
    tboxes = sorted(set(co.tolist()) | set(int(t) for t in to if t >= 0))
    for b in tboxes:
        cnt = np.zeros(o.nsrc, np.int64)
        for name in ("U", "WC", "XC"):
            for d in _rows(L[name], b):
                cnt += (so == d)
        for d in _rows(L["WF"], b):
            cnt += (anc[:, lev[d]] == d)
        w = b
        while w >= 0:
            for d in _rows(L["V"], w):
                cnt += (anc[:, lev[d]] == d)
            for d in _rows(L["XF"], w):
                cnt += (so == d)
            w = bx["parent"][w]
        assert (cnt == 1).all(), (b, np.unique(cnt))


@pytest.mark.parametrize("fix", ["c1_oracle", "small_oracle"])
def test_list_bounds_and_separation(fix, request):
    o = request.getfixturevalue(fix)
    bx = o.boxes()
    L = o.lists()
    H = o.root()["H"]
    tf = 0.9
    h = H * 2.0 ** -bx["level"].astype(float)
    cx = (2 * bx["ix"] + 1) * h
    cy = (2 * bx["iy"] + 1) * h
    dist = lambda a, b: max(abs(cx[a] - cx[b]), abs(cy[a] - cy[b]))  # noqa: E731
    for b in range(o.nbox):
        assert len(_rows(L["V"], b)) <= GOLD["list2_max"]["value"]
        assert len(_rows(L["XC"], b)) <= GOLD["list4close_max"]["value"]
        assert len(_rows(L["XF"], b)) <= GOLD["list4far_max"]["value"]
        for d in _rows(L["V"], b):          # 2-well-separated, same level
            assert bx["level"][d] == bx["level"][b] and dist(b, d) >= 6 * h[b] - 1e-12 * H
        for d in _rows(L["WF"], b):         # d < TCR(b)
            assert dist(b, d) >= 3 * h[d] + h[b] * (1 + tf) - 1e-12 * H
        for d in _rows(L["XF"], b):         # TCR(b) < d
            assert dist(b, d) >= 3 * h[b] * (1 + tf) + h[d] - 1e-12 * H


def test_tree_invariants(small_oracle):
    o = small_oracle
    bx = o.boxes()
    so, co, to = o.owners()
    xy, r, lc = o.centres()
    rt = o.root()
    H, lo_x, lo_y = rt["H"], rt["lo_x"], rt["lo_y"]
    lev = bx["level"]
    h = H * 2.0 ** -lev.astype(float)
    bcx = lo_x + (2 * bx["ix"] + 1) * h
    bcy = lo_y + (2 * bx["iy"] + 1) * h
    # root is a power of two and covers every disk
    assert np.log2(H) == np.round(np.log2(H))
    assert (xy[:, 0] - r >= lo_x).all() and (xy[:, 0] + r <= lo_x + 2 * H).all()
    # centre disks fit the TCR of their owner box
    b = co
    fit = np.maximum(abs(xy[:, 0] - bcx[b]), abs(xy[:, 1] - bcy[b])) + r
    assert (fit <= h[b] * 1.9 * (1 + 1e-15)).all()
    # suspended centres (owned by non-leaf boxes) have r > t_f |b| / 2
    has_child = np.zeros(o.nbox, bool)
    has_child[bx["parent"][bx["parent"] >= 0]] = True
    susp = has_child[co]
    assert (r[susp] > GOLD["suspended_radius_factor"]["value"] * 0.9 * h[co[susp]] * (1 - 1e-14)).all()
    # sources and point targets live in leaves, inside their box
    up = o.g["up_xy"]
    assert not has_child[so].any()
    assert (abs(up[:, 0] - bcx[so]) <= h[so] * (1 + 1e-12)).all()
    # subdivided boxes owned more than n_max eligible particles
    for bb in np.nonzero(has_child)[0]:
        assert bx["sub_src"][bb] + bx["sub_tgt"][bb] > o.params["n_max"]
    # leaves own at most n_max particles eligible for children (no level cap reached here)
    leaf = ~has_child
    elig_ctr = np.bincount(co[lc > lev[co]], minlength=o.nbox)
    assert (bx["nsrc"][leaf] + elig_ctr[leaf] + bx["ntgt"][leaf] <= o.params["n_max"]).all()


def test_association_bruteforce(small_oracle, small):
    o = small_oracle
    kind, ctr = o.association()
    xy, r, _ = o.centres()
    t = small["tgt_xy"]
    on = small["tgt_onsurf"]
    for i in range(len(t)):
        if on[i] >= 0:
            assert kind[i] == 2 and ctr[i] == 2 * on[i]
            continue
        key = ((t[i, 0] - xy[:, 0]) ** 2 + (t[i, 1] - xy[:, 1]) ** 2) / r ** 2
        j = int(np.argmin(key))
        if key[j] <= 1.44:
            assert kind[i] == 1 and ctr[i] == j
        else:
            assert kind[i] == 0
    assert (kind == 0).sum() == o.npt and (kind == 1).sum() > 0


def test_golden_idealized_factor():
    g = GOLD["green_table_idealized"]
    for p, v in zip(g["p_fmm"], g["value"]):
        assert abs(0.5 ** (p + 1) - v) <= 1e-6 * v
    tf = GOLD["tf_clean_bound"]["value"]
    alpha = (tf + np.sqrt(2)) / (6 - np.sqrt(2))
    assert abs(max(np.sqrt(2) / 3, alpha) - 0.5) < 1e-12
    assert abs(GOLD["list3far_factor"]["value"] - np.sqrt(2) / 3) < 1e-15
