"""GMRES for the exterior Neumann equation -mu/2 + S' mu = g (Sec. 1) on the
GPU: closed form on the unit circle, a known exterior harmonic function on
the starfish, and parity with GMRES driven by the oracle's S'."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _geo(g, **kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Geometry, params_default
    p = oracle.default_params(g, **kw)
    geo = Geometry(g, params_default(p_qbx=p["p_qbx"], p_fmm=p["p_fmm"], n_max=p["n_max"]))
    geo.set_targets(g["base_xy"], np.arange(len(g["base_xy"]), dtype=np.int32))
    geo.build()
    return geo, p


def _exterior_check(g, p, mu, z0, radius):
    from paper_1801_04070_gb300 import Geometry, params_default
    th = np.linspace(0, 2 * np.pi, 200, endpoint=False)
    t = np.stack([radius * np.cos(th), radius * np.sin(th)], 1)
    geo = Geometry(g, params_default(p_qbx=p["p_qbx"], p_fmm=p["p_fmm"], n_max=p["n_max"]))
    geo.set_targets(t, -np.ones(len(t), np.int32))
    geo.build()
    u = geo.eval("S", mu)
    z = t[:, 0] + 1j * t[:, 1]
    return np.abs(u - (1.0 / (z - z0)).real).max()


def test_unit_circle_closed_form():
    g = workloads.unit_circle(24)
    geo, p = _geo(g, p_qbx=12, p_fmm=20)
    th = g["base_theta"]
    mu, it, res = geo.gmres(-np.cos(th), tol=1e-12, maxit=100, restart=30)
    assert res < 1e-11 and it < 20
    assert np.abs(mu - 2 * np.cos(th)).max() < 1e-8
    assert _exterior_check(g, p, mu, 0.0, 2.0) < 1e-8


def test_starfish_known_solution_and_oracle_parity():
    spla = pytest.importorskip("scipy.sparse.linalg")
    g = workloads.starfish_c1()
    geo, p = _geo(g, p_qbx=10, p_fmm=20)
    z0 = 0.1 + 0.2j
    x = g["base_xy"][:, 0] + 1j * g["base_xy"][:, 1]
    nrm = g["base_n"][:, 0] + 1j * g["base_n"][:, 1]
    rhs = (nrm * (-1.0 / (x - z0) ** 2)).real          # d/dn Re(1/(z - z0))
    mu, it, res = geo.gmres(rhs, tol=1e-12, maxit=300, restart=60)
    assert res < 1e-11
    assert _exterior_check(g, p, mu, z0, 2.5) < 2e-5     # QBX truncation of S' at 64 panels
    # parity with GMRES on the oracle's operator
    g2 = dict(g)
    g2["tgt_xy"] = g["base_xy"]
    g2["tgt_onsurf"] = np.arange(len(x), dtype=np.int32)
    o = oracle.Oracle(g2, p)
    n = len(x)
    A = spla.LinearOperator((n, n), matvec=lambda v: -0.5 * v + o.eval("SP", np.asarray(v).ravel()))
    mu_o, info = spla.gmres(A, rhs, rtol=1e-13, atol=0.0, restart=60, maxiter=300)
    assert info == 0
    assert np.abs(mu - mu_o).max() <= 1e-9 * np.abs(mu_o).max()


def test_any_target_set():
    """The GMRES operator is gq_apply at the base nodes, so the solve does not
    depend on the targets the geometry was built with: with off-surface point
    targets (a deeper tree) the solution agrees with the base-node build to
    the FMM accuracy, and gq_apply(SP, -1/2) of it reproduces rhs."""
    g = workloads.starfish_c1()
    geo, p = _geo(g, p_qbx=8, p_fmm=20)
    x = g["base_xy"][:, 0] + 1j * g["base_xy"][:, 1]
    nrm = g["base_n"][:, 0] + 1j * g["base_n"][:, 1]
    rhs = (nrm * (-1.0 / (x - 0.1 - 0.2j) ** 2)).real
    mu0, _, res0 = geo.gmres(rhs, tol=1e-12, maxit=300, restart=60)
    rng = np.random.default_rng(5)
    t = rng.uniform(-1.5, 1.5, size=(3000, 2))
    geo.set_targets(t, -np.ones(len(t), np.int32))
    geo.build()
    mu1, _, res1 = geo.gmres(rhs, tol=1e-12, maxit=300, restart=60)
    assert res0 < 1e-11 and res1 < 1e-11
    assert np.abs(mu1 - mu0).max() <= 1e-9 * np.abs(mu0).max()
    r = geo.apply("SP", mu1, identity=-0.5)
    assert np.abs(r - rhs).max() <= 1e-10 * np.abs(rhs).max()


def test_batched_gmres_equals_individual_solves():
    """gq_batch_gmres: four single-curve geometries of different sizes solved
    in lockstep (each Arnoldi step one graph replay of S' over all of them)
    give the solutions and iteration counts of one gq_gmres after another."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Batch, Geometry, params_default
    curves = workloads.random_fourier_curves(2, seed=11)
    gs = [workloads.starfish_c1(), workloads.unit_circle(24), workloads.discretize([curves[0]], 32),
          workloads.discretize([curves[1]], 48)]
    z0 = 0.1 + 0.1j
    geos, rhs = [], []
    for g in gs:
        geo = Geometry(g, params_default(p_qbx=8, p_fmm=20, n_max=32))
        geo.set_targets(g["base_xy"], np.arange(len(g["base_xy"]), dtype=np.int32))
        geo.build()
        geos.append(geo)
        x = g["base_xy"][:, 0] + 1j * g["base_xy"][:, 1]
        nrm = g["base_n"][:, 0] + 1j * g["base_n"][:, 1]
        rhs.append(torch.tensor((nrm * (-1.0 / (x - z0) ** 2)).real, dtype=torch.float64, device="cuda"))
    mus = [torch.zeros_like(r) for r in rhs]
    b = Batch(geos)
    its, res = b.gmres(rhs, mus, tol=1e-10, maxit=200, restart=20)
    torch.cuda.synchronize()
    for geo, r, mu, it, rr in zip(geos, rhs, mus, its, res):
        ref = torch.empty_like(r)
        _, it1, rr1 = geo.gmres(r, tol=1e-10, maxit=200, restart=20, mu=ref)
        torch.cuda.synchronize()
        assert rr <= 2e-10 and it == it1
        assert torch.abs(mu - ref).max().item() <= 1e-13 * torch.abs(ref).max().item()
    b.close()
