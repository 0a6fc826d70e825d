"""Instrumentation of the trace (rt_set_profiling / rt_profile_read): the stage
events are recorded on the stream and read out by rt_profile_read, and profiling
changes neither the paths nor the traversal they come from."""
import numpy as np
import pytest
import torch

import scenegen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


def _trace(rt, ctx, scene, sc, rx):
    p = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
    ex = p.export()
    return p, {k: v.cpu().numpy() for k, v in ex.items()}


def test_stage_times_read_after_the_trace(rt):
    ctx = rt.Context(0)
    sc = scenegen.street_canyon()
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda")
    _, ref = _trace(rt, ctx, scene, sc, rx)
    ctx.set_profiling(1)
    n0, ms0, _ = ctx.profile()
    assert ms0 == [0.0] * 8                       # nothing traced since the reset
    p, ex = _trace(rt, ctx, scene, sc, rx)
    n1, ms, _ = ctx.profile()
    assert n1 > n0
    assert all(np.isfinite(ms)) and min(ms) >= 0.0
    assert ms[5] > 0.0
    # the total is the sum of the five consecutive stages (same events)
    assert abs(sum(ms[:5]) - ms[5]) <= 1e-3 * ms[5] + 5e-3   # event resolution ~0.5 us
    # the SBR kernel and its FP64 re-trace lie inside the SBR stage
    assert ms[6] + ms[7] <= ms[0] * (1 + 1e-3) + 5e-3
    # a second read returns the same times (nothing pending)
    assert ctx.profile()[1] == ms
    # two traces, one read: the times of the later one
    _trace(rt, ctx, scene, sc, rx)
    _, ex2 = _trace(rt, ctx, scene, sc, rx)
    ms2 = ctx.profile()[1]
    assert ms2[5] > 0.0 and abs(sum(ms2[:5]) - ms2[5]) <= 1e-3 * ms2[5] + 5e-3
    for k in ("rx", "depth", "seq", "tau", "rx_offsets"):
        assert np.array_equal(ex[k], ref[k]) and np.array_equal(ex2[k], ref[k])
    ctx.set_profiling(0)
    assert ctx.profile()[1] == [0.0] * 8
    assert ctx.status_word() == 0


def test_traversal_counters(rt):
    ctx = rt.Context(0)
    sc = scenegen.street_canyon()
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda")
    _, ref = _trace(rt, ctx, scene, sc, rx)
    ctx.set_profiling(2)
    _, ex = _trace(rt, ctx, scene, sc, rx)
    _, ms, c = ctx.profile()
    assert ms == [0.0] * 8                        # bit 0 off: no stage times
    # node visits, triangle tests, closest-hit queries (at most n_rays x depth),
    # visibility work and (candidate, receiver) pairs are all counted
    assert c[0] > 0 and c[1] > 0 and 0 < c[2] <= sc.n_rays * sc.max_depth
    assert c[4] > 0 and c[6] > 0 and c[7] > 0
    assert 0 <= c[3] <= c[2]
    for k in ("rx", "depth", "seq", "tau"):
        assert np.array_equal(ex[k], ref[k])
    ctx.set_profiling(0)
    assert ctx.status_word() == 0
