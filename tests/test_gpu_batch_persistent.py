"""The persistent batched launch (gq_batch_mode 0): the per-geometry branches
run only the strengths and FMM passes, one persistent kernel takes the direct
parts and final sums of all geometries and densities as work items, with
bounded waits on per-geometry counters.  Replays give the same bits; the
results agree with the graph-branch evaluation (mode 1) and with one-at-a-time
gq_eval to 1e-12 relative (FP64 sums of the same terms; the device bodies
inlined into the persistent kernel round a few ulps apart from their
stand-alone kernels, and the multi-density grouping from gq_eval, amplified
by the order-8 expansion at on-surface targets to a few 1e-13); a wait that
cannot be satisfied runs out into GQ_ERR_TIMEOUT without stopping the other
work."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _setup(q, nd, seed=0):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_04070_gb300 import Batch, Geometry, params_default
    gs = [workloads.starfish_c1(), workloads.small_grid(2, 2, 16, 3000, seed=7),
          workloads.small_grid(3, 2, 24, 5000, seed=11, on_surface="up"), workloads.small_grid(1, 1, 8, 200, seed=3)]
    geos = []
    for g in gs:
        geo = Geometry(g, params_default(p_qbx=q, p_fmm=12, n_max=32))
        geo.build()
        geos.append(geo)
    rng = np.random.default_rng(seed)
    dens = [torch.tensor(np.stack([workloads.starfish.fourier_density(g, rng) for _ in range(nd)]),
                         dtype=torch.float64, device="cuda") for g in gs]
    outs = [torch.full((nd, len(g["tgt_xy"])), float("nan"), dtype=torch.float64, device="cuda") for g in gs]
    return torch, Batch, gs, geos, dens, outs


@pytest.mark.parametrize("q,nd", [(5, 7), (8, 3)])
def test_persistent_equals_graph_and_eval(q, nd):
    torch, Batch, gs, geos, dens, outs = _setup(q, nd)
    b = Batch(geos)
    for kern in ("S", "D"):
        b.mode(0)
        b.eval(kern, dens, outs)
        torch.cuda.synchronize()
        first = [o.clone() for o in outs]
        b.eval(kern, dens, outs)           # a replay
        torch.cuda.synchronize()
        assert b.persistent_tile() in (1, 2, 4)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert b.persistent_ctas() in (sms, sms * 3 // 4, sms // 2)
        assert all(torch.equal(a, c) for a, c in zip(first, outs)), kern
        pers = [o.clone() for o in outs]
        b.mode(1)
        b.eval(kern, dens, outs)
        torch.cuda.synchronize()
        assert b.persistent_tile() == 0 and b.persistent_ctas() == 0
        for a, c in zip(pers, outs):
            assert (a - c).abs().max().item() <= 1e-12 * c.abs().max().item(), kern
        for geo, d, o in zip(geos, dens, pers):
            for j in range(nd):
                ref = torch.empty(o.shape[1], dtype=torch.float64, device="cuda")
                geo.eval(kern, d[j], ref)
                torch.cuda.synchronize()
                assert (o[j] - ref).abs().max().item() <= 1e-12 * ref.abs().max().item(), (kern, j)
    b.close()


def test_stalled_wait_times_out_and_recovers():
    """Geometry 1's final items wait for a count nothing reaches: the waits run
    out after 2 ms, the call reports GQ_ERR_TIMEOUT, every other geometry's
    outputs are complete; with the hook cleared the next call succeeds."""
    torch, Batch, gs, geos, dens, outs = _setup(5, 2, seed=3)
    from paper_1801_04070_gb300 import GigaQBXError
    b = Batch(geos)
    b.mode(0)
    b.eval("S", dens, outs)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    b.wait_test(2_000_000, 1)
    with pytest.raises(GigaQBXError) as e:
        b.eval("S", dens, outs)
    assert e.value.code == -4
    torch.cuda.synchronize()
    for i, (a, c) in enumerate(zip(outs, ref)):
        if i != 1:
            assert torch.equal(a, c), i
    b.wait_test(1_000_000_000, -1)
    b.eval("S", dens, outs)
    torch.cuda.synchronize()
    for a, c in zip(outs, ref):
        assert torch.equal(a, c)
    b.close()


def test_default_mode_takes_the_faster_path():
    """The default mode times the persistent launch and the graph branches and
    keeps one of them; its results agree with both to 1e-12."""
    torch, Batch, gs, geos, dens, outs = _setup(8, 2, seed=5)
    b = Batch(geos)
    b.eval("D", dens, outs)
    torch.cuda.synchronize()
    auto = [o.clone() for o in outs]
    assert b.persistent_tile() in (0, 1, 2, 4)
    for m in (0, 1):
        b.mode(m)
        b.eval("D", dens, outs)
        torch.cuda.synchronize()
        for a, c in zip(auto, outs):
            assert (a - c).abs().max().item() <= 1e-12 * c.abs().max().item(), m
    b.close()
