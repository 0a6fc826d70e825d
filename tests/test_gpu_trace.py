"""GPU path tracing vs the FP64 oracle: exact path sets (Sec. II-F)."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from gpu_helpers import assert_same_paths, gpu_trace, oracle_trace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def test_tiny_box_exact(rt, ctx):
    sc = scenegen.tiny_box()
    scene, p, ex = gpu_trace(rt, ctx, sc)
    o, tr = oracle_trace(sc)
    cand = p.candidates().cpu().numpy()
    assert np.array_equal(cand, tr["candidates"])
    assert_same_paths(ex, tr, o.diag)
    assert ctx.status_word() == 0


def test_street_canyon_full_size(rt, ctx):
    # the full street-canyon workload: 1e6 rays, depth 3, 4096 receivers
    sc = scenegen.street_canyon()
    scene, p, ex = gpu_trace(rt, ctx, sc)
    o, tr = oracle_trace(sc)
    assert np.array_equal(p.candidates().cpu().numpy(), tr["candidates"])
    assert_same_paths(ex, tr, o.diag)
    # receivers inside buildings get no path
    counts = np.diff(ex["rx_offsets"])
    assert (counts == 0).sum() > 0 and (counts > 0).sum() > 1000
    assert ctx.status_word() == 0


def test_indoor_subset(rt, ctx):
    sc = scenegen.indoor_diff()
    rx = sc.rx[::8]
    scene, p, ex = gpu_trace(rt, ctx, sc, n_rays=200_000, rx=rx)
    o, tr = oracle_trace(sc, n_rays=200_000, rx=rx)
    assert np.array_equal(p.candidates().cpu().numpy(), tr["candidates"])
    assert_same_paths(ex, tr, o.diag)
    assert ctx.status_word() == 0


def test_room_corridor_subset(rt, ctx):
    sc = scenegen.room_corridor(n_rx=64)
    scene, p, ex = gpu_trace(rt, ctx, sc, n_rays=100_000)
    o, tr = oracle_trace(sc, n_rays=100_000)
    assert np.array_equal(p.candidates().cpu().numpy(), tr["candidates"])
    assert_same_paths(ex, tr, o.diag)


def test_depth4_city(rt, ctx):
    sc = scenegen.city_batch()[7]
    rx = sc.rx[:96]
    scene, p, ex = gpu_trace(rt, ctx, sc, n_rays=100_000, depth=4, rx=rx)
    o, tr = oracle_trace(sc, n_rays=100_000, depth=4, rx=rx)
    assert np.array_equal(p.candidates().cpu().numpy(), tr["candidates"])
    assert_same_paths(ex, tr, o.diag)


def test_ragged_ray_counts(rt, ctx):
    # ray counts that are not multiples of the warp / block size, and one receiver
    sc = scenegen.tiny_box()
    for n in (1, 33, 1001):
        scene, p, ex = gpu_trace(rt, ctx, sc, n_rays=n, rx=sc.rx[5:6])
        o, tr = oracle_trace(sc, n_rays=n, rx=sc.rx[5:6])
        assert_same_paths(ex, tr, o.diag)


def test_trace_rejects_bad_arguments(rt, ctx):
    sc = scenegen.tiny_box()
    scene = rt.Scene.from_synthetic(ctx, sc)
    rxt = torch.tensor(sc.rx, dtype=torch.float64, device="cuda")
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.trace_paths(ctx, scene, sc.tx, rxt, 1000, 5)
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.trace_paths(ctx, scene, sc.tx, rxt, 0, 2)
    with pytest.raises(rt.RtError, match="NUMERIC"):
        rt.trace_paths(ctx, scene, (float("nan"), 0, 0), rxt, 10, 2)
    bad = sc.tris.copy()
    bad[0, 0] = 10_000
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.Scene(ctx, sc.verts, bad, sc.tri_material, sc.is_pec)
