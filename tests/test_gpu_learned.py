"""Learned order selection on the GPU: gradients of the training kernels
against the FP64 reference network, BF16 inference against FP32, and the
full loop -- features on the GPU, labels from the oracle on random star-
shaped curves, training by the CUDA kernels, deployment on starfish curves at
a requested accuracy of 1e-8 -- compared with the bound-driven orders: both
must meet the accuracy against converged unaccelerated QBX (the oracle), and
the learned orders must evaluate faster, and faster still with the
mixed-precision tier of the same accuracy."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import mlp as ref_mlp

pytestmark = pytest.mark.gpu

Q_REF, P_REF, Q_HI = 4, 8, 12


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_04070_gb300 as pkg
    return torch, pkg


def _mlp(pkg, seed=0):
    g = workloads.starfish_c1()
    geo = pkg.Geometry(g)
    return geo, pkg.MLP(geo, seed=seed)


def test_gradients_match_fp64_reference():
    torch, pkg = _gpu()
    geo, m = _mlp(pkg)
    rng = np.random.default_rng(0)
    w = rng.normal(0, 0.2, m.nparams).astype(np.float32)
    m.weights(set=w)
    X = rng.normal(size=(300, 32)).astype(np.float32)
    Y = rng.normal(size=(300, 2)).astype(np.float32)
    loss, g = m.loss_grad(X, Y)
    rloss, rg = ref_mlp.loss_grad(w.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - rloss) <= 1e-5 * abs(rloss)
    assert np.abs(g - rg).max() <= 1e-5 * np.abs(rg).max()


def test_bf16_inference_close_to_fp32():
    torch, pkg = _gpu()
    geo, m = _mlp(pkg, seed=3)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(1000, 32)).astype(np.float32)
    w = m.weights()
    y = m.predict(X)
    yr = ref_mlp.forward(w.astype(np.float64), X.astype(np.float64))[0]
    assert np.abs(y - yr).max() <= 3e-2 * np.abs(yr).max()


def _bf16(x):
    """Round float32 values to BF16 (nearest, ties to even), returned as float64."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_tensor_core_inference_matches_bf16_network():
    """The mma.sync inference equals the network with BF16 weights, biases,
    inputs and hidden activations and exact sums, up to FP32 summation (a
    different FP32 sum can move a hidden activation by one BF16 step), on a
    sample count that is not a multiple of the 16 rows of a warp's tile."""
    torch, pkg = _gpu()
    geo, m = _mlp(pkg, seed=5)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(1003, 32)).astype(np.float32)
    y = m.predict(X)
    w = _bf16(m.weights())
    dims = [32, 64, 32, 32, 2]
    a, o = _bf16(X), 0
    for l in range(4):
        W = w[o:o + dims[l] * dims[l + 1]].reshape(dims[l + 1], dims[l])
        o += dims[l] * dims[l + 1]
        b = w[o:o + dims[l + 1]]
        o += dims[l + 1]
        z = a @ W.T + b
        a = _bf16(np.maximum(z, 0).astype(np.float32)) if l < 3 else z
    d = np.abs(y - a)
    assert d.max() <= 5e-3 * np.abs(a).max()
    assert np.median(d) <= 1e-5 * np.abs(a).max()


def _label_module():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_order_labels.py")
    spec = importlib.util.spec_from_file_location("make_order_labels", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _stored_set(pkg, lo, hi):
    """Features (GPU) and stored oracle labels of training curves lo ... hi-1,
    one array pair per curve."""
    y, meta = _label_module().load()
    per = meta["centres_per_curve"]
    curves = workloads.order_training_curves(meta["n_curves"], meta["curve_seed"])
    X, Y = [], []
    for i in range(lo, hi):
        geo = pkg.Geometry(workloads.order_training_problem(curves[i], i),
                           pkg.params_default(p_qbx=Q_REF, p_fmm=P_REF, n_max=32))
        geo.build()
        X.append(geo.features().astype(np.float32))
        geo.close()
        Y.append(y[i * per:(i + 1) * per])
    return X, Y


def test_train_and_deploy_beats_bound_driven_orders():
    """Trained on 400 curves of the stored oracle labels (409,600 centres),
    deployed on a 4 x 4 starfish grid at eps = 1e-8: one learned FMM order
    with the QBX order fixed, against unaccelerated QBX of that order (the
    Theorem's quantity): within eps and faster than the bound-driven order,
    and faster again with the mixed-precision tier."""
    torch, pkg = _gpu()
    Xs_tr, Ys_tr = _stored_set(pkg, 0, 400)
    Xs, Ys = _stored_set(pkg, 400, 420)
    X, Y = np.concatenate(Xs_tr), np.concatenate(Ys_tr)
    Xv, Yv = np.concatenate(Xs), np.concatenate(Ys)
    geo0, m = _mlp(pkg, seed=7)
    loss = m.train(X, Y, epochs=20, batch=1024, lr=1e-3, seed=0)
    pv = m.predict(Xv)
    r2 = [1 - ((pv[:, k] - Yv[:, k]) ** 2).mean() / Yv[:, k].var() for k in (0, 1)]
    # deployment margins from held-out curves: per centre for the QBX order (upper tail
    # of the residuals); per geometry for the one FMM order of the tree (largest excess
    # of a curve's worst measured error over its worst prediction)
    margin_q = float(np.quantile(Yv[:, 0] - pv[:, 0], 0.995)) + 0.25
    margin_f = max(float(y[:, 1].max() - m.predict(x)[:, 1].max()) for x, y in zip(Xs, Ys)) + 0.5
    print(f"training loss {loss:.3f}; held-out R^2 QBX {r2[0]:.3f} FMM {r2[1]:.3f}; "
          f"margins {margin_q:.2f} {margin_f:.2f}")
    assert r2[0] > 0.2          # better than the mean; the density, unseen by the features, drives the rest

    eps = 1e-8
    g = workloads.starfish_grid(4, 4, 64, n_off=1 << 16, on_surface="up", seed=1)
    q_fixed = 5
    results = {}
    for mode in ("bound", "learned", "learned+mixed"):
        prec = 1 if mode == "learned+mixed" else 0
        geo = pkg.Geometry(g, pkg.params_default(p_qbx=q_fixed, p_fmm=0, n_max=32, eps=eps, precision=prec))
        geo.build()
        pb = geo.params.p_fmm
        if mode != "bound":
            p, q = geo.learned_orders(m, eps, margin_qbx=margin_q, margin_fmm=margin_f, q_ref=0, p_ref=P_REF,
                                      p_bound=pb)
        else:
            p, q = pb, q_fixed
        v = geo.eval("S", g["density"])
        ms = []
        for _ in range(3):
            _, st = geo.eval("S", g["density"], stats=True)
            ms.append(st.ms_total)
        results[mode] = (v, min(ms), p, q)
        geo.close()
    o = oracle.Oracle(g, oracle.default_params(g, p_qbx=q_fixed, p_fmm=P_REF))
    kind, _ = o.association()
    rng = np.random.default_rng(9)
    mask = np.zeros(len(kind), np.int32)
    for k in (0, 1, 2):
        ids = np.nonzero(kind == k)[0]
        mask[rng.choice(ids, min(200, len(ids)), replace=False)] = 1
    sel = mask.astype(bool)
    # the acceleration error against unaccelerated QBX of the same order
    ref = o.direct("S", g["density"], target_mask=mask)
    scale = np.abs(ref[sel]).max()
    for mode in ("bound", "learned", "learned+mixed"):
        v, ms, p, q = results[mode]
        err = np.abs(v[sel] - ref[sel]).max() / scale
        print(f"{mode}: p_fmm {p} p_qbx {q} eval {ms:.2f} ms, error vs unaccelerated QBX {err:.2e}")
        assert err <= eps, mode
    assert results["learned"][2] < results["bound"][2]
    assert results["learned"][1] < results["bound"][1]
    assert results["learned+mixed"][1] < results["learned"][1]


def test_centre_orders_truncate_each_expansion():
    """Per-centre orders: all centres at q equal the global order q; mixed
    orders give, at each target, the value of its centre's own order."""
    torch, pkg = _gpu()
    g = workloads.small_grid(2, 2, 16, 2000, seed=7, p_qbx=8, p_fmm=15)
    vals = {}
    for q in (3, 8):
        geo = pkg.Geometry(g, pkg.params_default(p_qbx=q, p_fmm=15, n_max=32))
        geo.build()
        vals[q] = geo.eval("S", g["density"])
        nc = geo.nc
        geo.close()
    geo = pkg.Geometry(g, pkg.params_default(p_qbx=8, p_fmm=15, n_max=32))
    geo.build()
    geo.set_centre_orders(np.full(nc, 3, np.int32))
    v3 = geo.eval("S", g["density"])
    assert np.abs(v3 - vals[3]).max() <= 1e-12 * np.abs(vals[3]).max()
    kind, ctr = geo.association()
    qs = np.where(np.arange(nc) % 4 == 0, 3, 8).astype(np.int32)
    geo.set_centre_orders(qs)
    vm = geo.eval("S", g["density"])
    one = kind == 1
    want = np.where(qs[ctr[one]] == 3, vals[3][one], vals[8][one])
    assert np.abs(vm[one] - want).max() <= 1e-12 * np.abs(want).max()
    geo.close()
