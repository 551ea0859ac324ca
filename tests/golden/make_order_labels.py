"""Writes order_labels.npz: oracle labels of the order-selection training set.

For curve i of workloads.order_training_curves() (the problem is
workloads.order_training_problem(curve, i)) and each of its 1,024 centres,
two numbers, measured at the centre's own base node (an on-surface target
of that centre):
  0: log10 of the QBX truncation error at order Q_REF: the terms Q_REF+1 ...
     Q_HI of the direct (unaccelerated) QBX expansion of order Q_HI (Sec. 2.2,
     eq. qbx; the oracle's O1),
  1: log10 of the acceleration error at FMM order P_REF: the difference of
     the first Q_REF+1 QBX coefficients formed by the oracle's GIGAQBX Stages
     1-8 (Sec. 4.4 Algorithm) at p_fmm = P_REF from the direct ones,
each relative to the largest |value| on the curve (+1e-16 inside the log).
Stored as uint8 in steps of 1/16 decade: label = -code / 16.

Only the oracle computes labels; the curves and densities come from the
seeded generators in workloads/.  Run from the repository root:
    python tests/golden/make_order_labels.py [n_curves]
"""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

import oracle  # noqa: E402
import workloads  # noqa: E402

Q_REF, P_REF, Q_HI = 4, 8, 12
STEP = 16          # codes per decade
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "order_labels.npz")


def labels(g):
    """Per centre (centre-id order): [log10 QBX truncation error at Q_REF,
    log10 acceleration error at P_REF], as described above."""
    o_hi = oracle.Oracle(g, oracle.default_params(p_qbx=Q_HI, p_fmm=P_REF))
    o_ref = oracle.Oracle(g, oracle.default_params(p_qbx=Q_REF, p_fmm=P_REF))
    _, b_hi = o_hi.direct("S", g["density"], want_qbx=True)
    _, b_ref = o_ref.eval("S", g["density"], want_qbx=True)
    xy, _, _ = o_hi.centres()
    node = np.arange(len(xy)) // 2
    t = g["base_xy"][node, 0] + 1j * g["base_xy"][node, 1]
    z = t - (xy[:, 0] + 1j * xy[:, 1])
    pw = z[:, None] ** np.arange(Q_HI + 1)[None, :]
    full = (b_hi * pw).sum(1).real
    scale = np.abs(full).max()
    tail = (b_hi[:, Q_REF + 1:] * pw[:, Q_REF + 1:]).sum(1).real
    fmm = ((b_ref - b_hi[:, :Q_REF + 1]) * pw[:, :Q_REF + 1]).sum(1).real
    return np.stack([np.log10(np.abs(tail) / scale + 1e-16), np.log10(np.abs(fmm) / scale + 1e-16)], 1)


def encode(y):
    return np.clip(np.rint(-y * STEP), 0, 255).astype(np.uint8)


def decode(code):
    return -code.astype(np.float32) / STEP


def load(path=OUT):
    """(labels [n_centres, 2] float32, metadata dict)."""
    with np.load(path) as f:
        return decode(f["codes"]), json.loads(str(f["meta"]))


def main(n_curves=2000):
    oracle.set_threads(oracle.max_threads())
    curves = workloads.order_training_curves(n_curves)
    codes, per = [], []
    t0 = time.time()
    for i, cv in enumerate(curves):
        y = labels(workloads.order_training_problem(cv, i))
        codes.append(encode(y))
        per.append(len(y))
        if (i + 1) % 200 == 0:
            print(f"{i + 1} curves, {time.time() - t0:.0f} s", flush=True)
    meta = {"n_curves": n_curves, "curve_seed": 5, "centres_per_curve": per[0] if len(set(per)) == 1 else per,
            "q_ref": Q_REF, "p_ref": P_REF, "q_hi": Q_HI, "codes_per_decade": STEP,
            "generator": "tests/golden/make_order_labels.py"}
    np.savez_compressed(OUT, codes=np.concatenate(codes), meta=json.dumps(meta))
    print(f"wrote {OUT}: {sum(per)} centres")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2000)
