"""The stored order-selection labels (tests/golden/order_labels.npz) are the
oracle's: recomputed for a few curves spread over the set, they give the
stored codes exactly, and the file holds what its metadata says.  The labels
themselves rest on O1 and O2, whose pins are in the other oracle tests."""
import importlib.util
import os

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _mod():
    spec = importlib.util.spec_from_file_location("make_order_labels", os.path.join(HERE, "golden", "make_order_labels.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def stored():
    mod = _mod()
    if not os.path.exists(mod.OUT):
        pytest.skip("labels not generated")
    y, meta = mod.load()
    return mod, y, meta


def test_metadata(stored):
    mod, y, meta = stored
    assert meta["n_curves"] * meta["centres_per_curve"] == len(y)
    assert (meta["q_ref"], meta["p_ref"], meta["q_hi"]) == (mod.Q_REF, mod.P_REF, mod.Q_HI)
    assert y.shape[1] == 2 and (y <= 0).all() and (y >= -16).all()


@pytest.mark.parametrize("i", [0, 777, 1999])
def test_codes_are_the_oracle_labels(stored, i):
    mod, y, meta = stored
    if i >= meta["n_curves"]:
        pytest.skip("fewer curves stored")
    per = meta["centres_per_curve"]
    curves = workloads.order_training_curves(meta["n_curves"], meta["curve_seed"])
    lab = mod.labels(workloads.order_training_problem(curves[i], i))
    assert np.array_equal(mod.decode(mod.encode(lab)), y[i * per:(i + 1) * per])


def test_labels_vary_over_the_set(stored):
    """Both labels spread over more than a decade and a half (what the
    network learns from), and at these orders (QBX 4, FMM 8) the
    acceleration error lies below the truncation error on average."""
    mod, y, meta = stored
    for k in (0, 1):
        assert np.percentile(y[:, k], 95) - np.percentile(y[:, k], 5) > 1.5, k
    assert y[:, 1].mean() < y[:, 0].mean()
