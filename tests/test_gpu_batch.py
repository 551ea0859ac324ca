"""Batched evaluation (gq_batch_*): several independent geometries of uneven
size, several densities each, one CUDA-graph launch.  The direct part of the
QBX coefficients is formed for several densities of a geometry at once (the
per-pair geometry and powers shared), which rounds differently from one
gq_eval per density: results must agree with the one-at-a-time gq_eval results
to 1e-13 relative, on the first call and on graph replays with new density
values, and repeated batched calls must agree bit for bit."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_batch_equals_individual_evaluations():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Batch, Geometry, params_default
    gs = [workloads.starfish_c1(), workloads.small_grid(2, 2, 16, 3000, seed=7),
          workloads.small_grid(3, 2, 24, 5000, seed=11, on_surface="up"),
          workloads.small_grid(1, 1, 8, 200, seed=3), workloads.starfish_grid(4, 3, 64, n_off=20000, seed=2)]
    geos = []
    for g in gs:
        geo = Geometry(g, params_default(p_qbx=5, p_fmm=10, n_max=32))
        geo.build()
        geos.append(geo)
    rng = np.random.default_rng(0)
    nd = 3
    dens = [torch.tensor(rng.normal(size=(nd, len(g["density"]))), dtype=torch.float64, device="cuda") for g in gs]
    outs = [torch.zeros((nd, len(g["tgt_xy"])), dtype=torch.float64, device="cuda") for g in gs]
    b = Batch(geos)
    for kern in ("S", "D"):
        for rep in range(2):
            if rep:
                for d in dens:
                    d.copy_(torch.tensor(rng.normal(size=tuple(d.shape)), dtype=torch.float64))
            b.eval(kern, dens, outs)
            torch.cuda.synchronize()
            for geo, d, o in zip(geos, dens, outs):
                for j in range(nd):
                    ref = torch.empty(o.shape[1], dtype=torch.float64, device="cuda")
                    geo.eval(kern, d[j], ref)
                    torch.cuda.synchronize()
                    err = (o[j] - ref).abs().max().item() / max(ref.abs().max().item(), 1e-300)
                    assert err <= 1e-13, (kern, rep, j, err)
    # repeated batched calls (graph replays) give the same bits
    b.eval("S", dens, outs)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    b.eval("S", dens, outs)
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(first, outs))
    assert b.streams() >= 1
    b.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_mixed_modes_equal_individual_evaluations(prec):
    """The batch in the mixed modes (MIXED at eps 1e-8, the pair tier, and
    MIXED_FMM with the FMM passes in pairs too): each density runs through the
    same kernels as one gq_eval, so the graph replays give the one-at-a-time
    results bit for bit, for geometries of uneven size."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Batch, Geometry, params_default
    gs = [workloads.starfish_c1(), workloads.small_grid(3, 2, 24, 5000, seed=11, on_surface="up"),
          workloads.starfish_grid(4, 3, 64, n_off=20000, seed=2)]
    geos = []
    for g in gs:
        geo = Geometry(g, params_default(p_qbx=5, p_fmm=20, n_max=32, eps=1e-8, precision=prec))
        geo.build()
        geos.append(geo)
    rng = np.random.default_rng(1)
    nd = 2
    dens = [torch.tensor(rng.normal(size=(nd, len(g["density"]))), dtype=torch.float64, device="cuda") for g in gs]
    outs = [torch.zeros((nd, len(g["tgt_xy"])), dtype=torch.float64, device="cuda") for g in gs]
    b = Batch(geos)
    for kern in ("S", "D"):
        b.eval(kern, dens, outs)
        b.eval(kern, dens, outs)     # a graph replay
        torch.cuda.synchronize()
        for geo, d, o in zip(geos, dens, outs):
            for j in range(nd):
                ref = torch.empty(o.shape[1], dtype=torch.float64, device="cuda")
                geo.eval(kern, d[j], ref)
                torch.cuda.synchronize()
                assert torch.equal(o[j], ref), (prec, kern, j)
    b.close()
