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
