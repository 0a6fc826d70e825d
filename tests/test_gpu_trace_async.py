"""The trace without host waits (rt_set_trace_async): the same paths and the same
calibration results as the trace that waits, on unresolved paths (counted on the
device), and a capacity that overflows is reported, not used."""
import numpy as np
import pytest
import torch

import scenegen

pytestmark = pytest.mark.gpu

RT_ERR_CAPACITY = 4


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


def _step(rt, ctx, p, sc, eps, sig, T, w, N):
    a = rt.eval_fields(ctx, p, eps, sig, sc.freq_hz)
    loss, ga, _ = rt.cfr_power_mse_fused(ctx, p.rx_offsets, a, p.tau, sc.f_center_hz, sc.delta_f_hz, N, T, w)
    ge, gs, gg = rt.eval_fields_backward(ctx, p, eps, sig, sc.freq_hz, ga)
    return loss.item(), ge.cpu().numpy(), gs.cpu().numpy(), gg.cpu().numpy()


def test_async_trace_matches_waiting_trace(rt):
    ctx = rt.Context(0)
    sc = scenegen.street_canyon()
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda")
    N = 1024
    p0 = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
    eps = torch.tensor(sc.eps_r * 1.2, device="cuda")
    sig = torch.tensor(sc.sigma * 0.7, device="cuda")
    a0 = rt.eval_fields(ctx, p0, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
                        sc.freq_hz)
    T = (rt.cfr(ctx, p0.rx_offsets, a0, p0.tau, sc.f_center_hz, sc.delta_f_hz, N).abs() ** 2).float().contiguous()
    w = (1.0 / T.mean(1).clamp_min(1e-30)).float().contiguous()
    ref = _step(rt, ctx, p0, sc, eps, sig, T, w, N)
    ex0 = {k: v.cpu().numpy() for k, v in p0.export().items()}
    rt.set_trace_async(ctx, True)
    try:
        for _ in range(2):
            p1 = rt.trace_paths(ctx, scene, sc.tx, rx, sc.n_rays, sc.max_depth)
            assert p1.n_paths >= p0.n_paths           # slots
            got = _step(rt, ctx, p1, sc, eps, sig, T, w, N)   # on unresolved paths
            assert got[0] == ref[0]
            # the gradients are sums over all paths with float atomics, whose order
            # varies from run to run; the gain gradient sums terms of both signs, so
            # its rounding is relative to the largest terms, not to the sum
            for x, y in zip(got[1:], ref[1:]):
                np.testing.assert_allclose(x, y, rtol=1e-5, atol=0)
            assert torch.equal(p1.rx_offsets, p0.rx_offsets)
            p1.resolve()
            assert p1.n_paths == p0.n_paths
            ex1 = {k: v.cpu().numpy() for k, v in p1.export().items()}
            for k in ("seq", "depth", "rx", "tau", "pts"):
                np.testing.assert_array_equal(ex1[k], ex0[k])
    finally:
        rt.set_trace_async(ctx, False)
    assert ctx.status_word() == 0


def test_async_overflow_is_reported(rt):
    # capacities learned on 64 receivers, then 4096 receivers without waiting: the
    # path capacity overflows; the status word says so, the receivers are emptied
    # (nothing reads past the slots) and resolve() refuses the paths
    ctx = rt.Context(0)
    sc = scenegen.street_canyon()
    scene = rt.Scene.from_synthetic(ctx, sc)
    small = torch.tensor(sc.rx[::64], dtype=torch.float64, device="cuda")
    full = torch.tensor(sc.rx, dtype=torch.float64, device="cuda")
    rt.trace_paths(ctx, scene, sc.tx, small, 200_000, 3)
    rt.set_trace_async(ctx, True)
    try:
        p = rt.trace_paths(ctx, scene, sc.tx, full, 200_000, 3)
        a = rt.eval_fields(ctx, p, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
                           sc.freq_hz)
        H = rt.cfr(ctx, p.rx_offsets, a, p.tau, sc.f_center_hz, sc.delta_f_hz, 256)
        torch.cuda.synchronize()
        assert ctx.status_word() == RT_ERR_CAPACITY
        assert int(p.rx_offsets[-1]) == 0 and torch.all(H == 0)
        with pytest.raises(rt.RtError):
            p.resolve()
    finally:
        rt.set_trace_async(ctx, False)
    # a waiting trace afterwards learns the larger capacities and is complete
    p2 = rt.trace_paths(ctx, scene, sc.tx, full, 200_000, 3)
    assert p2.n_paths > 1000
    assert ctx.status_word() == 0
