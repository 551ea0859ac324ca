"""Pin of the oracle's S' (normal derivative of S, two-sided = principal value)
through the exterior Neumann equation -mu/2 + S' mu = g (Sec. 1): on the unit
circle u = Re(1/z) = cos(theta)/r is S[2 cos theta] outside, so g = -cos(theta)
and the solution is mu = 2 cos(theta)."""
import numpy as np
import pytest

import oracle
import workloads


def _solve(q, p_fmm):
    spla = pytest.importorskip("scipy.sparse.linalg")
    g = workloads.unit_circle(24)
    o = oracle.Oracle(g, oracle.default_params(p_qbx=q, p_fmm=p_fmm))
    th = g["base_theta"]
    n = len(th)
    A = spla.LinearOperator((n, n), matvec=lambda v: -0.5 * v + o.eval("SP", np.asarray(v).ravel()))
    mu, info = spla.gmres(A, -np.cos(th), rtol=1e-13, atol=0.0, restart=50, maxiter=200)
    assert info == 0
    return o, th, np.abs(mu - 2 * np.cos(th)).max()


def test_unit_circle_neumann_closed_form():
    o8, th, e8 = _solve(8, 15)
    o12, th, e12 = _solve(12, 20)
    # the error is the QBX truncation error of the derivative: it drops with the order
    assert e8 < 1e-6 and e12 < 1e-8 and e12 < e8 / 50
    # S' of cos(k theta) has principal value 0 on the unit circle, of 1 it is -1/2
    assert np.abs(o12.eval("SP", np.cos(3 * th))).max() < 1e-8
    assert np.abs(o12.eval("SP", np.ones(len(th))) + 0.5).max() < 1e-9
