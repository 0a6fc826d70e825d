"""Batched tracing of several scenes of uneven size (one persistent SBR launch
over all of them) against the per-scene path and against the oracle, plus the
tracing autotuner."""
import numpy as np
import pytest
import torch

import scenegen
from gpu_helpers import assert_same_paths, oracle_trace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def _split(ex, p, s):
    """Paths of scene s out of a batch export, with scene-local triangle ids and receivers."""
    r0, r1 = p.scene_rx_offsets[s], p.scene_rx_offsets[s + 1]
    offs = ex["rx_offsets"]
    a, b = offs[r0], offs[r1]
    seq = ex["seq"][a:b].copy()
    seq[seq >= 0] -= p.scene_tri_offsets[s]
    return dict(rx=ex["rx"][a:b] - r0, depth=ex["depth"][a:b], seq=seq, tau=ex["tau"][a:b], pts=ex["pts"][a:b],
                rx_offsets=offs[r0:r1 + 1] - a)


def test_batch_equals_per_scene_and_fields(rt, ctx):
    cities = scenegen.city_batch()
    pick = [2, 7, 10, 4]                     # 2978, 890, 950, 1154 triangles: uneven
    n_rays, depth = 200_000, 4
    scenes = [rt.Scene.from_synthetic(ctx, cities[i]) for i in pick]
    rxs = [cities[i].rx[: 40 + 13 * j] for j, i in enumerate(pick)]
    p = rt.trace_batch(ctx, scenes, [cities[i].tx for i in pick], rxs, n_rays, depth)
    ex = {k: v.cpu().numpy() for k, v in p.export().items()}
    eps = torch.tensor(cities[pick[0]].eps_r, device="cuda")
    sig = torch.tensor(cities[pick[0]].sigma, device="cuda")
    a_batch = rt.eval_fields(ctx, p, eps, sig, 3.5e9).cpu().numpy()
    total = 0
    for s, i in enumerate(pick):
        q = rt.trace_paths(ctx, scenes[s], cities[i].tx, torch.tensor(rxs[s], device="cuda"), n_rays, depth)
        exq = {k: v.cpu().numpy() for k, v in q.export().items()}
        exb = _split(ex, p, s)
        for k in ("rx", "depth", "seq", "rx_offsets"):
            assert np.array_equal(exb[k], exq[k]), (s, k)
        np.testing.assert_allclose(exb["tau"], exq["tau"], rtol=1e-15)
        aq = rt.eval_fields(ctx, q, eps, sig, 3.5e9).cpu().numpy()
        a0, a1 = ex["rx_offsets"][p.scene_rx_offsets[s]], ex["rx_offsets"][p.scene_rx_offsets[s + 1]]
        np.testing.assert_allclose(a_batch[a0:a1], aq, rtol=1e-6, atol=1e-12)
        total += len(exq["tau"])
    assert total == p.n_paths and total > 100
    assert ctx.status_word() == 0


def test_batch_matches_oracle(rt, ctx):
    cities = scenegen.city_batch()
    pick = [7, 10]
    n_rays, depth = 100_000, 3
    scenes = [rt.Scene.from_synthetic(ctx, cities[i]) for i in pick]
    rxs = [cities[i].rx[:48] for i in pick]
    p = rt.trace_batch(ctx, scenes, [cities[i].tx for i in pick], rxs, n_rays, depth)
    ex = {k: v.cpu().numpy() for k, v in p.export().items()}
    for s, i in enumerate(pick):
        o, tr = oracle_trace(cities[i], n_rays=n_rays, depth=depth, rx=rxs[s])
        assert_same_paths(_split(ex, p, s), tr, o.diag)


def test_autotuner(rt, ctx):
    sc = scenegen.street_canyon()
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx = torch.tensor(sc.rx[::4], device="cuda")
    ref = {k: v.cpu().numpy() for k, v in rt.trace_paths(ctx, scene, sc.tx, rx, 300_000, 3).export().items()}
    chosen, ms = rt.autotune_trace(ctx, scene, sc.tx, rx, 300_000, 3)
    assert all(1 <= c <= 64 for c in chosen) and ms > 0
    chosen2, ms2 = rt.autotune_trace(ctx, scene, sc.tx, rx, 300_000, 3)   # cached
    assert chosen2 == chosen and ms2 == 0.0
    got = {k: v.cpu().numpy() for k, v in rt.trace_paths(ctx, scene, sc.tx, rx, 300_000, 3).export().items()}
    for k in ("rx", "depth", "seq", "rx_offsets"):
        assert np.array_equal(got[k], ref[k])
    rt.set_tuning(ctx, 8, 16, 8)
    with pytest.raises(rt.RtError):
        rt.set_tuning(ctx, 0, 16, 8)


def test_batch_and_calibration_in_one_cuda_graph(rt):
    # the batched trace (which waits for nothing inside a capture) and the
    # calibration step (fields, fused CFR + loss + adjoint, fields adjoint) of the
    # small cities captured in one CUDA graph; every replay gives the results of
    # the same calls made outside the graph
    ctx = rt.Context(0)
    cities = scenegen.city_batch()
    pick = [i for i, c in enumerate(cities) if c.n_tris < 3500]
    n_rays, depth, N = 100_000, 4, 256
    small = [cities[i] for i in pick]
    scenes = [rt.Scene.from_synthetic(ctx, c) for c in small]
    rxs = [torch.tensor(c.rx, dtype=torch.float64, device="cuda") for c in small]
    txs = [c.tx for c in small]
    sc0 = small[0]
    fc, df, f = sc0.f_center_hz, 50e6 / N, sc0.freq_hz
    eps = torch.tensor(sc0.eps_r * 1.2, device="cuda")
    sig = torch.tensor(sc0.sigma * 0.7, device="cuda")
    p0 = rt.trace_batch(ctx, scenes, txs, rxs, n_rays, depth)       # learns the capacities
    a0 = rt.eval_fields(ctx, p0, torch.tensor(sc0.eps_r, device="cuda"), torch.tensor(sc0.sigma, device="cuda"), f)
    T = (rt.cfr(ctx, p0.rx_offsets, a0, p0.tau, fc, df, N).abs() ** 2).float().contiguous()
    w = (1.0 / T.mean(1).clamp_min(1e-30)).float().contiguous()

    def step():
        p = rt.trace_batch(ctx, scenes, txs, rxs, n_rays, depth)
        a = rt.eval_fields(ctx, p, eps, sig, f)
        loss, ga, _ = rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, fc, df, N, T, w)
        ge, gs, gg = rt.eval_fields_backward(ctx, p, eps, sig, f, ga)
        return p, loss, ge, gs

    _, L_ref, ge_ref, gs_ref = step()
    L_ref, ge_ref, gs_ref = L_ref.item(), ge_ref.cpu().numpy(), gs_ref.cpu().numpy()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()                                  # sizes every scratch buffer on this stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p, loss, ge, gs = step()
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        assert loss.item() == pytest.approx(L_ref, rel=1e-6)
        np.testing.assert_allclose(ge.cpu().numpy(), ge_ref, rtol=1e-5, atol=1e-12)
        np.testing.assert_allclose(gs.cpu().numpy(), gs_ref, rtol=1e-5, atol=1e-12)
        assert torch.equal(p.rx_offsets, p0.rx_offsets)
    assert ctx.status_word() == 0
    p.resolve()
    assert p.n_paths == p0.n_paths
