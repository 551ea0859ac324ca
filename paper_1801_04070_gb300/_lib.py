"""ctypes binding of include/gigaqbx.h (same function names)."""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libgigaqbx.so")
_lock = threading.Lock()
_lib = None

GQ_S, GQ_D, GQ_SP = 0, 1, 2
GQ_PREC_FP64, GQ_PREC_MIXED, GQ_PREC_MIXED_FMM = 0, 1, 2
KERNELS = {"S": GQ_S, "D": GQ_D, "SP": GQ_SP}
LISTS = ("U", "V", "WC", "WF", "XC", "XF")


class GigaQBXError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gigaqbx error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("p_qbx", C.c_int), ("p_fmm", C.c_int), ("n_max", C.c_int),
                ("tf_num", C.c_int), ("tf_den", C.c_int), ("w3_demote", C.c_int),
                ("max_level", C.c_int), ("radius_factor", C.c_double),
                ("assoc_slack", C.c_double), ("eps", C.c_double), ("precision", C.c_int), ("m2l", C.c_int),
                ("level_restrict", C.c_int), ("tcr_shape", C.c_int)]


class GeometryDesc(C.Structure):
    _fields_ = [("npanels", C.c_int), ("nb", C.c_int), ("nu", C.c_int),
                ("ref_b", C.c_void_p), ("ref_u", C.c_void_p), ("base_xy", C.c_void_p),
                ("base_n", C.c_void_p), ("up_xy", C.c_void_p), ("up_n", C.c_void_p),
                ("up_w", C.c_void_p), ("panel_len", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("ms_total", C.c_double),
                ("ms_stage", C.c_double * 12)]


class TreeInfo(C.Structure):
    _fields_ = [("nbox", C.c_int), ("nlevels", C.c_int), ("ncentres", C.c_int),
                ("npoint_targets", C.c_int), ("ntargets", C.c_int), ("nsources", C.c_int),
                ("list_size", C.c_int64 * 6)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libgigaqbx.so; raises if it was not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: run __graft_entry__.build() "
                              "(or python -m paper_1801_04070_gb300.build)")
        L = C.CDLL(_LIB_PATH)
        vp, i32, st = C.c_void_p, C.c_int, C.c_int
        sig = {
            "gq_params_default": (st, [C.POINTER(Params)]),
            "gq_params_resolve": (st, [C.POINTER(Params), C.POINTER(Params)]),
            "gq_create": (st, [i32, vp, C.POINTER(vp)]),
            "gq_destroy": (st, [vp]),
            "gq_last_error": (C.c_char_p, [vp]),
            "gq_set_stream": (st, [vp, vp]),
            "gq_geometry_create": (st, [vp, C.POINTER(GeometryDesc), C.POINTER(Params), C.POINTER(vp)]),
            "gq_geometry_destroy": (st, [vp]),
            "gq_geometry_params": (st, [vp, C.POINTER(Params)]),
            "gq_targets_set": (st, [vp, i32, vp, vp]),
            "gq_build": (st, [vp]),
            "gq_eval": (st, [vp, i32, vp, vp, C.POINTER(Stats)]),
            "gq_eval_noalloc": (st, [vp, i32, vp, vp]),
            "gq_apply": (st, [vp, i32, C.c_double, vp, vp]),
            "gq_gmres": (st, [vp, vp, C.c_double, i32, i32, vp, C.POINTER(i32), C.POINTER(C.c_double)]),
            "gq_context_launches": (st, [vp, C.POINTER(C.c_int64)]),
            "gq_probe_fma_peak": (st, [vp, i32, C.POINTER(C.c_double)]),
            "gq_probe_math": (st, [vp, i32, i32, vp, vp]),
            "gq_probe_umma": (st, [vp, i32, vp, vp, i32, vp]),
            "gq_tensor_paths": (st, [vp, C.POINTER(i32), C.POINTER(i32)]),
            "gq_lists_check": (st, [vp, i32, C.POINTER(i32)]),
            "gq_memory_cached": (st, [C.POINTER(C.c_int64)]),
            "gq_memory_release": (st, []),
            "gq_tree_info_get": (st, [vp, C.POINTER(TreeInfo)]),
            "gq_centre_features": (st, [vp, vp]),
            "gq_mlp_create": (st, [vp, C.c_uint64, C.POINTER(vp)]),
            "gq_mlp_destroy": (st, [vp]),
            "gq_mlp_weights": (st, [vp, vp, vp, C.POINTER(i32)]),
            "gq_mlp_loss_grad": (st, [vp, vp, vp, i32, C.POINTER(C.c_float), vp]),
            "gq_mlp_train": (st, [vp, vp, vp, i32, i32, i32, C.c_float, C.c_uint64, C.POINTER(C.c_float)]),
            "gq_mlp_predict": (st, [vp, vp, i32, vp]),
            "gq_learned_orders": (st, [vp, vp, C.c_double, C.c_double, C.c_double, i32, i32, i32, C.POINTER(i32),
                                      C.POINTER(i32)]),
            "gq_set_orders": (st, [vp, i32, i32]),
            "gq_set_centre_orders": (st, [vp, vp]),
            "gq_batch_create": (st, [vp, i32, C.POINTER(vp), C.POINTER(vp)]),
            "gq_batch_destroy": (st, [vp]),
            "gq_batch_eval": (st, [vp, i32, i32, C.POINTER(vp), C.POINTER(vp)]),
            "gq_batch_streams": (st, [vp, C.POINTER(i32)]),
            "gq_batch_mode": (st, [vp, i32]),
            "gq_batch_persistent": (st, [vp, C.POINTER(i32)]),
            "gq_batch_persistent_ctas": (st, [vp, C.POINTER(i32)]),
            "gq_batch_wait_test": (st, [vp, C.c_int64, i32]),
            "gq_batch_gmres": (st, [vp, C.POINTER(vp), C.c_double, i32, i32, C.POINTER(vp), C.POINTER(i32),
                                    C.POINTER(C.c_double)]),
            "gq_export_root": (st, [vp, vp]),
            "gq_export_boxes": (st, [vp] + [vp] * 9),
            "gq_export_list": (st, [vp, i32, vp, vp]),
            "gq_export_centres": (st, [vp, vp, vp, vp]),
            "gq_export_assoc": (st, [vp, vp, vp]),
            "gq_export_owners": (st, [vp, vp, vp, vp]),
            "gq_export_qbx": (st, [vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def params_default(**kw) -> Params:
    p = Params()
    lib().gq_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def params_resolve(p: Params) -> Params:
    """The parameters a geometry built with `p` uses (orders from eps when
    given as 0); raises GigaQBXError for parameters the library rejects."""
    out = Params()
    st = lib().gq_params_resolve(C.byref(p), C.byref(out))
    if st != 0:
        raise GigaQBXError(st, "invalid parameters")
    return out


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None stays None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _current_stream(device):
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except Exception:
        pass
    return None


class Geometry:
    """One context + discretised curve + targets, built once, evaluated many times."""

    def __init__(self, g: dict, params: Params | None = None, device: int = 0, stream=None):
        self.L = lib()
        self._ctx = C.c_void_p()
        s = stream if stream is not None else _current_stream(device)
        self._check(self.L.gq_create(device, s, C.byref(self._ctx)), ctx=False)
        self.params = params or params_default(p_qbx=int(g.get("p_qbx", 5)), p_fmm=int(g.get("p_fmm", 10)),
                                                n_max=int(g.get("n_max", 32)))
        keep = {k: np.ascontiguousarray(g[k], np.float64)
                for k in ("ref_b", "ref_u", "base_xy", "base_n", "up_xy", "up_n", "up_w", "panel_len")}
        d = GeometryDesc(int(g["npanels"]), int(g["nb"]), int(g["nu"]), _ptr(keep["ref_b"]),
                         _ptr(keep["ref_u"]), _ptr(keep["base_xy"]), _ptr(keep["base_n"]),
                         _ptr(keep["up_xy"]), _ptr(keep["up_n"]), _ptr(keep["up_w"]),
                         _ptr(keep["panel_len"]))
        self._geom = C.c_void_p()
        self._check(self.L.gq_geometry_create(self._ctx, C.byref(d), C.byref(self.params), C.byref(self._geom)))
        resolved = Params()
        self._check(self.L.gq_geometry_params(self._geom, C.byref(resolved)))
        self.params = resolved
        self.nbase = int(g["npanels"]) * int(g["nb"])
        self.nsrc = int(g["npanels"]) * int(g["nu"])
        self.nt = 0
        if "tgt_xy" in g:
            self.set_targets(g["tgt_xy"], g["tgt_onsurf"])

    # -------------------------------------------------------------- plumbing
    def _check(self, status, ctx=True):
        if status != 0:
            msg = self.L.gq_last_error(self._ctx).decode() if ctx else "context creation failed"
            raise GigaQBXError(status, msg)

    def close(self):
        if getattr(self, "_geom", None):
            self.L.gq_geometry_destroy(self._geom)
            self._geom = None
        if getattr(self, "_ctx", None):
            self.L.gq_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(self.L.gq_set_stream(self._ctx, stream))

    # -------------------------------------------------------------- API
    def set_targets(self, xy, on_surface_node):
        xy_a = xy if not isinstance(xy, np.ndarray) else np.ascontiguousarray(xy, np.float64)
        on_a = on_surface_node if not isinstance(on_surface_node, np.ndarray) else \
            np.ascontiguousarray(on_surface_node, np.int32)
        self.nt = int(len(on_a))
        self._check(self.L.gq_targets_set(self._geom, self.nt, _ptr(xy_a), _ptr(on_a)))

    def build(self):
        self._check(self.L.gq_build(self._geom))
        info = TreeInfo()
        self._check(self.L.gq_tree_info_get(self._geom, C.byref(info)))
        self.info = info
        self.nbox = info.nbox
        self.nc = info.ncentres
        self.npt = info.npoint_targets
        return self

    def eval(self, kernel, density, out=None, stats: bool = False):
        """Evaluate S, D or SP at the targets.  density / out: numpy (host) or
        torch CUDA tensors (device).  Returns out (allocated on the host when
        not given) and optionally the library's statistics."""
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        if isinstance(density, np.ndarray):
            density = np.ascontiguousarray(density, np.float64)
        if out is None:
            out = np.empty(self.nt, np.float64)
        st = Stats()
        self._check(self.L.gq_eval(self._geom, k, _ptr(density), _ptr(out), C.byref(st)))
        return (out, st) if stats else out

    def apply(self, kernel, mu, out=None, identity=0.0):
        """identity * mu + K mu at the base nodes (gq_apply), K = S, D or SP
        evaluated two-sided.  mu / out: numpy (host) or torch CUDA tensors."""
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        if isinstance(mu, np.ndarray):
            mu = np.ascontiguousarray(mu, np.float64)
        if out is None:
            out = np.empty(self.nbase, np.float64)
        self._check(self.L.gq_apply(self._geom, k, float(identity), _ptr(mu), _ptr(out)))
        return out

    def gmres(self, rhs, tol=1e-10, maxit=500, restart=50, mu=None):
        """Solve -mu/2 + S' mu = rhs at the base nodes (the operator is
        gq_apply).  Returns (mu, iterations, relative residual)."""
        if isinstance(rhs, np.ndarray):
            rhs = np.ascontiguousarray(rhs, np.float64)
        if mu is None:
            mu = np.empty(self.nbase, np.float64)
        it = C.c_int()
        res = C.c_double()
        self._check(self.L.gq_gmres(self._geom, _ptr(rhs), tol, maxit, restart, _ptr(mu), C.byref(it), C.byref(res)))
        return mu, it.value, res.value

    def tensor_paths(self):
        """(List 2 on the tensor cores, List 3 far to centres on the tensor
        cores) for the next evaluation (gq_tensor_paths)."""
        a, b = C.c_int(), C.c_int()
        self._check(self.L.gq_tensor_paths(self._geom, C.byref(a), C.byref(b)))
        return bool(a.value), bool(b.value)

    def lists_check(self, row_cap=-1):
        """Enumeration passes of the last list construction (gq_lists_check);
        row_cap >= 0 sets the scratch row capacity of the next builds (0: the
        default capacities)."""
        n = C.c_int()
        self._check(self.L.gq_lists_check(self._geom, int(row_cap), C.byref(n)))
        return n.value

    def features(self):
        """[ncentres, 32] FP32 per-centre features (gq_centre_features)."""
        f = np.zeros((self.nc, 32), np.float32)
        self._check(self.L.gq_centre_features(self._geom, _ptr(f)))
        return f

    def learned_orders(self, mlp, eps, margin_qbx=1.0, margin_fmm=1.0, q_ref=4, p_ref=8, p_bound=30):
        p = C.c_int()
        q = C.c_int()
        self._check(self.L.gq_learned_orders(self._geom, mlp._m, eps, margin_qbx, margin_fmm, q_ref, p_ref, p_bound,
                                             C.byref(p), C.byref(q)))
        return p.value, q.value

    def set_orders(self, p_qbx, p_fmm):
        self._check(self.L.gq_set_orders(self._geom, p_qbx, p_fmm))

    def set_centre_orders(self, q):
        q = np.ascontiguousarray(q, np.int32)
        self._check(self.L.gq_set_centre_orders(self._geom, _ptr(q)))

    # -------------------------------------------------------------- exports
    def root(self):
        o = np.zeros(4)
        self._check(self.L.gq_export_root(self._geom, _ptr(o)))
        return dict(lo_x=o[0], lo_y=o[1], H=o[2], u=o[3])

    def boxes(self):
        n = self.nbox
        d = dict(level=np.zeros(n, np.int32), ix=np.zeros(n, np.int64), iy=np.zeros(n, np.int64),
                 parent=np.zeros(n, np.int32), nsrc=np.zeros(n, np.int32), nctr=np.zeros(n, np.int32),
                 ntgt=np.zeros(n, np.int32), sub_src=np.zeros(n, np.int32), sub_tgt=np.zeros(n, np.int32))
        self._check(self.L.gq_export_boxes(self._geom, *[_ptr(d[k]) for k in
                                                        ("level", "ix", "iy", "parent", "nsrc", "nctr",
                                                         "ntgt", "sub_src", "sub_tgt")]))
        return d

    def lists(self):
        out = {}
        for i, name in enumerate(LISTS):
            n = int(self.info.list_size[i])
            off = np.zeros(self.nbox + 1, np.int32)
            idx = np.zeros(max(n, 1), np.int32)
            self._check(self.L.gq_export_list(self._geom, i, _ptr(off), _ptr(idx)))
            out[name] = (off, idx[:n])
        return out

    def centres(self):
        xy = np.zeros((self.nc, 2)); r = np.zeros(self.nc); lc = np.zeros(self.nc, np.int32)
        self._check(self.L.gq_export_centres(self._geom, _ptr(xy), _ptr(r), _ptr(lc)))
        return xy, r, lc

    def association(self):
        kind = np.zeros(self.nt, np.int32); ctr = np.zeros(self.nt, np.int32)
        self._check(self.L.gq_export_assoc(self._geom, _ptr(kind), _ptr(ctr)))
        return kind, ctr

    def owners(self):
        so = np.zeros(self.nsrc, np.int32); co = np.zeros(self.nc, np.int32); to = np.zeros(self.nt, np.int32)
        self._check(self.L.gq_export_owners(self._geom, _ptr(so), _ptr(co), _ptr(to)))
        return so, co, to

    def qbx_coefficients(self):
        q = np.zeros((self.nc, self.params.p_qbx + 1, 2))
        self._check(self.L.gq_export_qbx(self._geom, _ptr(q)))
        return q[..., 0] + 1j * q[..., 1]


class Batch:
    """Independent built geometries evaluated together by one CUDA-graph launch
    (gq_batch_*).  Densities and outputs are torch CUDA tensors of shape
    [ndens, n] per geometry."""

    def __init__(self, geoms):
        self.L = lib()
        self.geoms = list(geoms)
        self._ctx = self.geoms[0]._ctx
        arr = (C.c_void_p * len(self.geoms))(*[g._geom.value for g in self.geoms])
        self._b = C.c_void_p()
        st = self.L.gq_batch_create(self._ctx, len(self.geoms), arr, C.byref(self._b))
        if st != 0:
            raise GigaQBXError(st, self.L.gq_last_error(self._ctx).decode())

    def eval(self, kernel, dens, outs):
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        nd = int(dens[0].shape[0])
        dp = (C.c_void_p * len(dens))(*[d.data_ptr() for d in dens])
        op = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        st = self.L.gq_batch_eval(self._b, k, nd, dp, op)
        if st != 0:
            raise GigaQBXError(st, self.L.gq_last_error(self._ctx).decode())
        return outs

    def mode(self, mode):
        """0: persistent launch where supported, 1: graph branches only,
        2 (default): whichever of the two the autotuner measures faster."""
        st = self.L.gq_batch_mode(self._b, int(mode))
        if st != 0:
            raise GigaQBXError(st, self.L.gq_last_error(self._ctx).decode())

    def persistent_tile(self):
        t = C.c_int()
        self.L.gq_batch_persistent(self._b, C.byref(t))
        return t.value

    def persistent_ctas(self):
        """CTAs of the persistent launch in use (0 when the graph branches run)."""
        t = C.c_int()
        self.L.gq_batch_persistent_ctas(self._b, C.byref(t))
        return t.value

    def wait_test(self, wait_ns, stall_geom):
        st = self.L.gq_batch_wait_test(self._b, int(wait_ns), int(stall_geom))
        if st != 0:
            raise GigaQBXError(st, self.L.gq_last_error(self._ctx).decode())

    def streams(self):
        s = C.c_int()
        self.L.gq_batch_streams(self._b, C.byref(s))
        return s.value

    def gmres(self, rhs, mus, tol=1e-10, maxit=500, restart=50):
        """Exterior Neumann solves for all geometries at once (gq_batch_gmres):
        rhs and mus are lists of torch CUDA tensors [npanels*nb].  Returns
        (iterations, relative residuals) per geometry."""
        n = len(self.geoms)
        rp = (C.c_void_p * n)(*[r.data_ptr() for r in rhs])
        mp = (C.c_void_p * n)(*[m.data_ptr() for m in mus])
        it = (C.c_int * n)()
        res = (C.c_double * n)()
        st = self.L.gq_batch_gmres(self._b, rp, tol, maxit, restart, mp, it, res)
        if st != 0:
            raise GigaQBXError(st, self.L.gq_last_error(self._ctx).decode())
        return list(it), list(res)

    def close(self):
        if getattr(self, "_b", None):
            self.L.gq_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The order-selection network (gq_mlp_*): FP32 training, BF16 inference."""

    def __init__(self, geo_or_ctx, seed=0):
        self.L = lib()
        self._ctx = geo_or_ctx._ctx if hasattr(geo_or_ctx, "_ctx") else geo_or_ctx
        self._m = C.c_void_p()
        self._check(self.L.gq_mlp_create(self._ctx, seed, C.byref(self._m)))
        n = C.c_int()
        self._check(self.L.gq_mlp_weights(self._m, None, None, C.byref(n)))
        self.nparams = n.value

    def _check(self, st):
        if st != 0:
            raise GigaQBXError(st, self.L.gq_last_error(self._ctx).decode())

    def weights(self, set=None):
        w = np.zeros(self.nparams, np.float32)
        s = None if set is None else np.ascontiguousarray(set, np.float32)
        self._check(self.L.gq_mlp_weights(self._m, _ptr(w), _ptr(s), None))
        return w

    def loss_grad(self, X, Y):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        loss = C.c_float()
        grad = np.zeros(self.nparams, np.float32)
        self._check(self.L.gq_mlp_loss_grad(self._m, _ptr(X), _ptr(Y), len(X), C.byref(loss), _ptr(grad)))
        return loss.value, grad

    def train(self, X, Y, epochs=50, batch=512, lr=1e-3, seed=0):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        loss = C.c_float()
        self._check(self.L.gq_mlp_train(self._m, _ptr(X), _ptr(Y), len(X), epochs, batch, lr, seed, C.byref(loss)))
        return loss.value

    def predict(self, X):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.zeros((len(X), 2), np.float32)
        self._check(self.L.gq_mlp_predict(self._m, _ptr(X), len(X), _ptr(Y)))
        return Y

    def close(self):
        if getattr(self, "_m", None):
            self.L.gq_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

