"""Pin of the FP64 reference network: its analytic gradient against central
finite differences of its loss (no shared code with the CUDA kernels)."""
import numpy as np

from oracle import mlp


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    n = sum(a * b + b for a, b in zip(mlp.DIMS[:-1], mlp.DIMS[1:]))
    w = rng.normal(0, 0.3, n)
    X = rng.normal(size=(7, 32))
    Y = rng.normal(size=(7, 2))
    loss, g = mlp.loss_grad(w, X, Y)
    idx = rng.choice(n, 60, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_grad(wp, X, Y)[0] - mlp.loss_grad(wm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i
    assert loss > 0
