"""Batched evaluation and batched GMRES against the FP64 oracle directly
(not against one-at-a-time gq_eval).

gq_batch_eval has its own near-field kernel in FP64 mode: the direct part of
the QBX coefficients (Sec. 4.4, Stages 3, 5a and 6a) is formed for up to four
densities of a geometry at once.  Seven densities per geometry run it with 4,
2 and 1 densities per launch.  Every output of every geometry and density is
compared with the oracle's Stages 1-8 (O2) at the same orders: FP64 within
1e-12 relative; the mixed tiers within eps/5 of the oracle.  Densities are
random Fourier series per curve, as in the batched workload.  gq_batch_gmres is
compared with GMRES driven by the oracle's S' (exterior Neumann equation,
Sec. 1)."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

ND = 7          # 4 + 2 + 1 densities per multi-density launch


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _geometries():
    return [workloads.starfish_c1(),
            workloads.small_grid(2, 2, 16, 3000, seed=7),
            workloads.small_grid(3, 2, 24, 5000, seed=11, on_surface="up"),
            workloads.small_grid(1, 1, 8, 200, seed=3)]


def _rel(a, ref):
    return float(np.abs(a - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def batch_case():
    torch = _torch()
    gs = _geometries()
    rng = np.random.default_rng(21)
    # random-Fourier densities, the batched workload's recipe
    dens = [np.stack([workloads.starfish.fourier_density(g, rng) for _ in range(ND)]) for g in gs]
    refs = {}
    for i, (g, d) in enumerate(zip(gs, dens)):
        o = oracle.Oracle(g, oracle.default_params(p_qbx=5, p_fmm=10, n_max=32))
        for kern in ("S", "D"):
            refs[i, kern] = np.stack([o.eval(kern, d[j]) for j in range(ND)])
    return torch, gs, dens, refs


@pytest.mark.parametrize("prec,eps,tol", [(0, 1e-12, 1e-12), (1, 5e-6, 1e-6), (1, 1e-8, 2e-9), (2, 1e-8, 2e-9)])
def test_batch_eval_matches_oracle(batch_case, prec, eps, tol):
    torch, gs, dens, refs = batch_case
    from paper_1801_04070_gb300 import Batch, Geometry, params_default
    geos = []
    for g in gs:
        geo = Geometry(g, params_default(p_qbx=5, p_fmm=10, n_max=32, eps=eps, precision=prec))
        geo.build()
        geos.append(geo)
    dd = [torch.tensor(d, dtype=torch.float64, device="cuda") for d in dens]
    outs = [torch.full((ND, len(g["tgt_xy"])), float("nan"), dtype=torch.float64, device="cuda") for g in gs]
    b = Batch(geos)
    for kern in ("S", "D"):
        for rep in range(2):            # the eager pass, then a graph replay
            for o in outs:
                o.fill_(float("nan"))
            b.eval(kern, dd, outs)
            torch.cuda.synchronize()
            for i, o in enumerate(outs):
                v = o.cpu().numpy()
                assert np.isfinite(v).all(), (i, kern, rep)
                for j in range(ND):
                    err = _rel(v[j], refs[i, kern][j])
                    assert err <= tol, (prec, eps, kern, rep, i, j, err)
    b.close()
    for geo in geos:
        geo.close()


def test_batch_gmres_matches_oracle_gmres():
    """Solutions of gq_batch_gmres on two geometries of different size equal
    those of GMRES on the oracle's -mu/2 + S' mu to 1e-9 relative."""
    torch = _torch()
    spla = pytest.importorskip("scipy.sparse.linalg")
    from paper_1801_04070_gb300 import Batch, Geometry, params_default
    curve = workloads.random_fourier_curves(1, seed=13)[0]
    gs = [workloads.starfish_c1(), workloads.discretize([curve], 32)]
    z0 = 0.05 + 0.1j
    geos, rhs, rhs_np = [], [], []
    for g in gs:
        geo = Geometry(g, params_default(p_qbx=8, p_fmm=20, n_max=32))
        geo.set_targets(g["base_xy"], np.arange(len(g["base_xy"]), dtype=np.int32))
        geo.build()
        geos.append(geo)
        x = g["base_xy"][:, 0] + 1j * g["base_xy"][:, 1]
        nrm = g["base_n"][:, 0] + 1j * g["base_n"][:, 1]
        r = (nrm * (-1.0 / (x - z0) ** 2)).real
        rhs_np.append(r)
        rhs.append(torch.tensor(r, dtype=torch.float64, device="cuda"))
    mus = [torch.zeros_like(r) for r in rhs]
    b = Batch(geos)
    its, res = b.gmres(rhs, mus, tol=1e-12, maxit=300, restart=60)
    torch.cuda.synchronize()
    for g, r, mu, rr in zip(gs, rhs_np, mus, res):
        assert rr <= 2e-12
        g2 = dict(g)
        g2["tgt_xy"] = g["base_xy"]
        g2["tgt_onsurf"] = np.arange(len(g["base_xy"]), dtype=np.int32)
        o = oracle.Oracle(g2, oracle.default_params(p_qbx=8, p_fmm=20, n_max=32))
        n = len(r)
        A = spla.LinearOperator((n, n), matvec=lambda v: -0.5 * v + o.eval("SP", np.asarray(v).ravel()))
        mu_o, info = spla.gmres(A, r, rtol=1e-13, atol=0.0, restart=60, maxiter=300)
        assert info == 0
        assert _rel(mu.cpu().numpy(), mu_o) <= 1e-9
    b.close()
    for geo in geos:
        geo.close()
