"""CPU FP64 oracle for GIGAQBX -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_1801_04070_gb300``)
never does.  The C library (``gq_oracle.c``) is compiled with gcc on first
use (or by ``__graft_entry__.build()``), with ``-ffp-contract=off`` so every
floating-point operation that decides an integer result rounds separately.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libgq_oracle.so")
# a deliberately broken build of the oracle, for the mutation test only
_LIB_OVERRIDE = os.environ.get("GQ_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

LISTS = ("U", "V", "WC", "WF", "XC", "XF")
KERNELS = {"S": 0, "D": 1, "SP": 2}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "gq_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Geom(C.Structure):
    _fields_ = [("npanels", C.c_int), ("nb", C.c_int), ("nu", C.c_int),
                ("ref_b", C.c_void_p), ("ref_u", C.c_void_p),
                ("base_xy", C.c_void_p), ("base_n", C.c_void_p),
                ("up_xy", C.c_void_p), ("up_n", C.c_void_p), ("up_w", C.c_void_p),
                ("panel_len", C.c_void_p), ("ntargets", C.c_int),
                ("tgt_xy", C.c_void_p), ("tgt_onsurf", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("p_qbx", C.c_int), ("p_fmm", C.c_int), ("n_max", C.c_int),
                ("tf_num", C.c_int), ("tf_den", C.c_int), ("w3_demote", C.c_int),
                ("max_level", C.c_int), ("radius_factor", C.c_double),
                ("assoc_slack", C.c_double), ("level_restrict", C.c_int), ("tcr_shape", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_LIB_OVERRIDE or build())
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(_Geom), C.POINTER(_Params)]
            L.orc_destroy.argtypes = [C.c_void_p]
            for f in ("orc_build", "orc_lists_bruteforce", "orc_nbox", "orc_ncentres",
                      "orc_npoint_targets"):
                getattr(L, f).argtypes = [C.c_void_p]
                getattr(L, f).restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            L.orc_max_threads.argtypes = []
            L.orc_max_threads.restype = C.c_int
            L.orc_list_size.restype = C.c_int64
            L.orc_list_size.argtypes = [C.c_void_p, C.c_int, C.c_int]
            L.orc_list.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_root.argtypes = [C.c_void_p, C.c_void_p]
            L.orc_boxes.argtypes = [C.c_void_p] + [C.c_void_p] * 9
            L.orc_centres.argtypes = [C.c_void_p] * 4
            L.orc_assoc.argtypes = [C.c_void_p] * 3
            L.orc_owners.argtypes = [C.c_void_p] * 4
            L.orc_upsample.argtypes = [C.c_void_p] * 3
            for f in ("orc_eval", "orc_direct"):
                getattr(L, f).argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]
                getattr(L, f).restype = C.c_int
            L.orc_sep_test.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64,
                                       C.c_int, C.c_int64, C.c_int64]
            L.orc_sep_test.restype = C.c_int
            L.orc_op_p2m.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_op_p2l.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_op_m2m.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_op_m2l.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_op_l2l.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_op_eval_local.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_op_eval_mpole.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def sep_test(shape, tn, td, which, a, b) -> bool:
    """The oracle's adequate-separation relation (Sec. 4.3) for boxes a, b
    given as (level, ix, iy): which 0 tests a |> TCR(b), 1 tests TCR(a) |> b;
    shape 0 the square TCR, 1 the disk-shaped one."""
    return bool(lib().orc_sep_test(int(shape), int(tn), int(td), int(which), int(a[0]), int(a[1]), int(a[2]),
                                   int(b[0]), int(b[1]), int(b[2])))


def set_threads(n: int) -> int:
    """Threads of the oracle's evaluation loops (1 = serial, the default).
    Every output is summed by one thread in the serial order, so the results
    are the same bits for any count.  Returns the count in effect."""
    return int(lib().orc_set_threads(int(n)))


def max_threads() -> int:
    """Processors the oracle's OpenMP runtime sees."""
    return int(lib().orc_max_threads())


def _p(a):
    return a.ctypes.data if a is not None else None


def default_params(g: dict | None = None, **kw) -> dict:
    p = dict(p_qbx=5, p_fmm=10, n_max=32, tf_num=9, tf_den=10, w3_demote=15,
             max_level=30, radius_factor=0.5, assoc_slack=1.2, level_restrict=0, tcr_shape=0)
    if g is not None:
        for k in ("p_qbx", "p_fmm", "n_max"):
            if k in g:
                p[k] = int(g[k])
    p.update(kw)
    return p


class Oracle:
    """O1/O2/O3 on one geometry + target set."""

    def __init__(self, g: dict, params: dict | None = None, build_now: bool = True):
        self.L = lib()
        self.params = params or default_params(g)
        self.g = g
        # keep references to the arrays handed to C (it copies them on create)
        self._arr = {k: np.ascontiguousarray(g[k], dtype=np.float64)
                     for k in ("ref_b", "ref_u", "base_xy", "base_n", "up_xy", "up_n",
                               "up_w", "panel_len", "tgt_xy")}
        self._arr["tgt_onsurf"] = np.ascontiguousarray(g["tgt_onsurf"], dtype=np.int32)
        a = self._arr
        geom = _Geom(int(g["npanels"]), int(g["nb"]), int(g["nu"]), _p(a["ref_b"]), _p(a["ref_u"]),
                     _p(a["base_xy"]), _p(a["base_n"]), _p(a["up_xy"]), _p(a["up_n"]),
                     _p(a["up_w"]), _p(a["panel_len"]), int(len(a["tgt_xy"])),
                     _p(a["tgt_xy"]), _p(a["tgt_onsurf"]))
        pr = self.params
        prm = _Params(pr["p_qbx"], pr["p_fmm"], pr["n_max"], pr["tf_num"], pr["tf_den"],
                      pr["w3_demote"], pr["max_level"], pr["radius_factor"], pr["assoc_slack"],
                      int(pr.get("level_restrict", 0)), int(pr.get("tcr_shape", 0)))
        self.h = self.L.orc_create(C.byref(geom), C.byref(prm))
        self.nt = len(a["tgt_xy"])
        self.nsrc = int(g["npanels"]) * int(g["nu"])
        if build_now:
            self.build()

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def build(self):
        self.L.orc_build(self.h)
        self.nbox = self.L.orc_nbox(self.h)
        self.nc = self.L.orc_ncentres(self.h)
        self.npt = self.L.orc_npoint_targets(self.h)

    def brute_force_lists(self):
        self.L.orc_lists_bruteforce(self.h)

    def root(self):
        out = np.zeros(4)
        self.L.orc_root(self.h, _p(out))
        return dict(lo_x=out[0], lo_y=out[1], H=out[2], u=out[3])

    def boxes(self):
        n = self.nbox
        i32 = lambda: np.zeros(n, np.int32)  # noqa: E731
        d = dict(level=i32(), ix=np.zeros(n, np.int64), iy=np.zeros(n, np.int64), parent=i32(),
                 nsrc=i32(), nctr=i32(), ntgt=i32(), sub_src=i32(), sub_tgt=i32())
        self.L.orc_boxes(self.h, *[_p(d[k]) for k in ("level", "ix", "iy", "parent", "nsrc",
                                                       "nctr", "ntgt", "sub_src", "sub_tgt")])
        return d

    def centres(self):
        xy = np.zeros((self.nc, 2)); r = np.zeros(self.nc); lc = np.zeros(self.nc, np.int32)
        self.L.orc_centres(self.h, _p(xy), _p(r), _p(lc))
        return xy, r, lc

    def association(self):
        kind = np.zeros(self.nt, np.int32); ctr = np.zeros(self.nt, np.int32)
        self.L.orc_assoc(self.h, _p(kind), _p(ctr))
        return kind, ctr

    def owners(self):
        so = np.zeros(self.nsrc, np.int32); co = np.zeros(self.nc, np.int32); to = np.zeros(self.nt, np.int32)
        self.L.orc_owners(self.h, _p(so), _p(co), _p(to))
        return so, co, to

    def lists(self, brute: bool = False):
        out = {}
        for i, name in enumerate(LISTS):
            n = self.L.orc_list_size(self.h, i, int(brute))
            off = np.zeros(self.nbox + 1, np.int32); idx = np.zeros(max(n, 1), np.int32)
            self.L.orc_list(self.h, i, int(brute), _p(off), _p(idx))
            out[name] = (off, idx[:n])
        return out

    def upsample(self, mu_base):
        mu_base = np.ascontiguousarray(mu_base, np.float64)
        out = np.zeros(self.nsrc)
        self.L.orc_upsample(self.h, _p(mu_base), _p(out))
        return out

    def _run(self, fn, kernel, mu, target_mask, want_qbx):
        mu = np.ascontiguousarray(mu, np.float64)
        val = np.full(self.nt, np.nan)
        mask = None if target_mask is None else np.ascontiguousarray(target_mask, np.int32)
        qbx = np.zeros((self.nc, self.params["p_qbx"] + 1, 2)) if want_qbx else None
        fn(self.h, KERNELS[kernel], _p(mu), _p(mask), _p(val), _p(qbx))
        if want_qbx:
            return val, qbx[..., 0] + 1j * qbx[..., 1]
        return val

    def eval(self, kernel, mu, target_mask=None, want_qbx=False):
        """O2: the GIGAQBX FMM."""
        return self._run(self.L.orc_eval, kernel, mu, target_mask, want_qbx)

    def direct(self, kernel, mu, target_mask=None, want_qbx=False):
        """O1: unaccelerated QBX."""
        return self._run(self.L.orc_direct, kernel, mu, target_mask, want_qbx)


# ---------------------------------------------------------------- single operators
def _c(z):
    return np.array([complex(z).real, complex(z).imag])


def _cv(v):
    v = np.asarray(v, np.complex128)
    return np.ascontiguousarray(np.stack([v.real, v.imag], -1).ravel())


def _uncv(a):
    return a[0::2] + 1j * a[1::2]


def op_p2m(kernel, p, c, ys, strengths):
    out = np.zeros(2 * (p + 1))
    cc, yy, ss = _c(c), _cv(ys), _cv(strengths)
    lib().orc_op_p2m(KERNELS[kernel], p, _p(cc), len(ys), _p(yy), _p(ss), _p(out))
    return _uncv(out)


def op_p2l(kernel, p, c, ys, strengths):
    out = np.zeros(2 * (p + 1))
    cc, yy, ss = _c(c), _cv(ys), _cv(strengths)
    lib().orc_op_p2l(KERNELS[kernel], p, _p(cc), len(ys), _p(yy), _p(ss), _p(out))
    return _uncv(out)


def op_m2m(p, c_old, c_new, a):
    out = np.zeros(2 * (p + 1))
    c0, c1, aa = _c(c_old), _c(c_new), _cv(a)
    lib().orc_op_m2m(p, _p(c0), _p(c1), _p(aa), _p(out))
    return _uncv(out)


def op_m2l(p_in, p_out, c_m, c_l, a):
    out = np.zeros(2 * (p_out + 1))
    c0, c1, aa = _c(c_m), _c(c_l), _cv(a)
    lib().orc_op_m2l(p_in, p_out, _p(c0), _p(c1), _p(aa), _p(out))
    return _uncv(out)


def op_l2l(p_in, p_out, c_old, c_new, b):
    out = np.zeros(2 * (p_out + 1))
    c0, c1, bb = _c(c_old), _c(c_new), _cv(b)
    lib().orc_op_l2l(p_in, p_out, _p(c0), _p(c1), _p(bb), _p(out))
    return _uncv(out)


def op_eval_local(p, c, b, ts):
    out = np.zeros(2 * len(ts))
    cc, bb, tt = _c(c), _cv(b), _cv(ts)
    lib().orc_op_eval_local(p, _p(cc), _p(bb), len(ts), _p(tt), _p(out))
    return _uncv(out)


def op_eval_mpole(p, c, a, ts):
    out = np.zeros(2 * len(ts))
    cc, aa, tt = _c(c), _cv(a), _cv(ts)
    lib().orc_op_eval_mpole(p, _p(cc), _p(aa), len(ts), _p(tt), _p(out))
    return _uncv(out)
