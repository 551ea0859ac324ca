"""Host checks of the two rounding arguments the build kernels rest on,
replayed with numpy's IEEE FP32/FP64 operations in the kernels' order (the
tree file is compiled without FMA contraction, so every operation rounds on
its own, as numpy's do).

1. Target association (k_associate): for each candidate centre the FP32
   distance d_f gives rho = |t - c| / r in [lo, hi]; the exact minimiser of
   the FP64 key, and every candidate tied with it, must survive the filter
   "lo <= min hi", so that the two-scan search returns the brute-force
   argmin (lowest id on ties) bit for bit.
2. Centre levels (k_keys): the levels skipped before the scan, those below
   ilogb(kappa H / r), must all pass the FP64 fit test that the scan from the
   root would apply, so that the deepest admissible level is unchanged.
"""
import math

import numpy as np
import pytest

F = np.float32
KEYBITS = 30


# ------------------------------------------------------------------ association
def _assoc_floats(cx, cy, r, slack, delta):
    """The per-centre FP32 table of the kernel: x, y, slack threshold, 1/r."""
    lim = slack * r * 1.001 + delta
    v = lim * lim * 1.001
    z = F(v)
    if float(z) < v:                                      # FP32 rounded upwards
        z = np.nextafter(z, F(np.inf))
    return F(cx), F(cy), z, F(1.0 / r)


def _bounds(tx, ty, fx_c, fy_c, fz, fw, delta_f):
    """(passes the slack prefilter, lo, hi) exactly as the kernel forms them."""
    txf, tyf = F(tx), F(ty)
    fx = F(txf - fx_c)
    fy = F(tyf - fy_c)
    d2f = F(F(fx * fx) + F(fy * fy))
    df = np.sqrt(d2f)                                     # IEEE sqrtf
    hi = F(F(F(df + delta_f) * fw) * F(1.00001))
    lo = F(F(F(df - delta_f) * fw) * F(0.99999))
    return d2f <= fz, lo, hi


def _delta(X, cell):
    return 16.0 * (X + 2.0 * cell) * 2.0 ** -24


@pytest.mark.parametrize("scale", [1.0, 40.0, 3000.0])
def test_float_interval_holds_the_exact_ratio(scale):
    rng = np.random.default_rng(int(scale))
    n = 20000
    r = rng.uniform(0.002, 0.08, n) * scale / 40.0
    cell = 1.25 * 1.2 * r.max()
    X = scale
    delta = _delta(X, cell)
    delta_f = F(delta * 1.001)
    cx = rng.uniform(-X, X, n)
    cy = rng.uniform(-X, X, n)
    ang = rng.uniform(0, 2 * np.pi, n)
    dist = r * rng.uniform(0.0, 1.6, n)
    tx, ty = cx + dist * np.cos(ang), cy + dist * np.sin(ang)
    for i in range(n):
        fx_c, fy_c, fz, fw = _assoc_floats(cx[i], cy[i], r[i], 1.2, delta)
        ok, lo, hi = _bounds(tx[i], ty[i], fx_c, fy_c, fz, fw, delta_f)
        rho = math.hypot(tx[i] - cx[i], ty[i] - cy[i]) / r[i]
        assert float(lo) <= rho * (1 + 1e-12) and rho * (1 - 1e-12) <= float(hi), (i, lo, rho, hi)
        if rho <= 1.2:
            assert ok, i                                   # the prefilter keeps every acceptable centre


def _two_scan(tx, ty, C, delta):
    """The kernel's search over one candidate set: FP32 minimum of hi, then
    exact FP64 keys for the survivors (lowest id on ties)."""
    delta_f = F(delta * 1.001)
    tabs = [_assoc_floats(cx, cy, r, 1.2, delta) for (cx, cy, r) in C]
    hmin = F(np.inf)
    for tab in tabs:
        ok, lo, hi = _bounds(tx, ty, *tab, delta_f)
        if ok:
            hmin = min(hmin, hi)
    best, bestk, nexact = -1, np.inf, 0
    for cid, ((cx, cy, r), tab) in enumerate(zip(C, tabs)):
        ok, lo, hi = _bounds(tx, ty, *tab, delta_f)
        if not ok or lo > hmin:
            continue
        nexact += 1
        dx, dy = tx - cx, ty - cy
        key = (dx * dx + dy * dy) / (r * r)
        if key < bestk or (key == bestk and cid < best):
            best, bestk = cid, key
    return (best if best >= 0 and bestk <= 1.2 * 1.2 else -1), nexact


def _brute(tx, ty, C):
    best, bestk = -1, np.inf
    for cid, (cx, cy, r) in enumerate(C):
        dx, dy = tx - cx, ty - cy
        key = (dx * dx + dy * dy) / (r * r)
        if key < bestk or (key == bestk and cid < best):
            best, bestk = cid, key
    return best if best >= 0 and bestk <= 1.2 * 1.2 else -1


def test_two_scan_search_equals_brute_force_argmin():
    """Centres along a curve in curve order (the case that made every
    candidate improve the running minimum), plus exact ties: mirrored centre
    pairs and duplicated centres."""
    rng = np.random.default_rng(3)
    total_exact = 0
    ntest = 0
    for trial in range(300):
        X = rng.choice([1.0, 25.0, 500.0])
        h = rng.uniform(0.01, 0.1)
        s = np.linspace(0, 1.5, 48)
        base = np.stack([X * 0.5 + s, X * 0.3 + 0.2 * np.sin(3 * s)], 1)
        C = [(x, y + h / 2, h / 2) for x, y in base] + [(x, y - h / 2, h / 2) for x, y in base]
        if trial % 3 == 0:                      # exact duplicates: the lower id must win
            C = C + C[:10]
        delta = _delta(X + 2, 1.5 * h)
        for _ in range(20):
            t = base[rng.integers(len(base))] + rng.normal(0, h, 2)
            if trial % 5 == 0:                  # on the mirror line of a centre pair: exact ties
                t = base[rng.integers(len(base))].copy()
            got, nexact = _two_scan(t[0], t[1], C, delta)
            assert got == _brute(t[0], t[1], C)
            total_exact += nexact
            ntest += 1
    assert total_exact / ntest < 4.0            # about one exact key per target, not one per candidate


# ------------------------------------------------------------------ centre levels
def _key1(v, lo, inv_u):
    f = math.floor((v - lo) * inv_u)
    return int(min(max(f, 0), (1 << KEYBITS) - 1))


def _fits(x, y, r, kx, ky, l, lo_x, lo_y, H, scale, shape):
    ix, iy = kx >> (KEYBITS - l), ky >> (KEYBITS - l)
    hb = math.ldexp(H, -l)
    bx = lo_x + float(2 * ix + 1) * hb
    by = lo_y + float(2 * iy + 1) * hb
    dx, dy = x - bx, y - by
    d = math.sqrt(dx * dx + dy * dy) if shape == 1 else max(abs(dx), abs(dy))
    d += r
    return d <= hb * scale


def _level_scan(x, y, r, kx, ky, lo_x, lo_y, H, scale, shape, max_level, l0):
    lc = l0 - 1
    for l in range(l0, max_level + 1):
        if _fits(x, y, r, kx, ky, l, lo_x, lo_y, H, scale, shape):
            lc = l
        else:
            break
    return max(lc, 0)


@pytest.mark.parametrize("shape", [0, 1])
@pytest.mark.parametrize("tf", [(9, 10), (1, 10), (1, 1)])
def test_skipped_levels_all_fit(shape, tf):
    """Every level below the kernel's starting level passes the fit, and the
    scan from there gives the level the scan from the root gives."""
    tn, td = tf
    scale = (td + tn) / td
    c0 = 1.4143 if shape == 1 else 1.0
    kappa = 0.8 * (scale - c0 - 1.0 / 32.0)
    rng = np.random.default_rng(11 + shape + tn)
    for trial in range(40):
        H = math.ldexp(1.0, int(rng.integers(-3, 8)))
        u = math.ldexp(H, 1 - KEYBITS)
        lo_x = math.floor(rng.uniform(-50, 50) / u) * u
        lo_y = math.floor(rng.uniform(-50, 50) / u) * u
        inv_u = 1.0 / u
        kappa_H = kappa * H if kappa > 0 else 0.0
        max_level = int(rng.choice([30, 12]))
        for _ in range(200):
            x = lo_x + rng.uniform(0, 2 * H)
            y = lo_y + rng.uniform(0, 2 * H)
            r = H * math.exp(rng.uniform(math.log(1e-7), math.log(0.5)))
            kx, ky = _key1(x, lo_x, inv_u), _key1(y, lo_y, inv_u)
            l0 = 0
            if kappa_H > 0 and r > 0:
                l0 = max(min(math.frexp(kappa_H / r)[1] - 1, max_level, KEYBITS - 7), 0)   # ilogb
            for l in range(l0):
                assert _fits(x, y, r, kx, ky, l, lo_x, lo_y, H, scale, shape), (trial, l, l0)
            full = _level_scan(x, y, r, kx, ky, lo_x, lo_y, H, scale, shape, max_level, 0)
            fast = _level_scan(x, y, r, kx, ky, lo_x, lo_y, H, scale, shape, max_level, l0)
            assert full == fast
