"""The allocation-free fused CFR loss entry point against the regular one.

rt_cfr_power_mse_fused_noalloc exists for callers that cannot allocate device
memory while they run the loss (for example a loop that reserved its memory
budget in advance, or a host program whose memory manager forbids other code
from calling the CUDA allocator).  It keeps its working memory in a fixed array
inside the library.  Both entry points are called through the C ABI on the same
inputs; two calls in a row must both agree with the regular entry point, on the
tensor cores and on the SIMT units.  A receiver of more than 4096 paths is summed
exactly by the allocation-free call (the regular call uses its non-uniform FFT
approximation there), so that case is also checked against the FP64 oracle.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import scenegen

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(x, dtype):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda").contiguous()


def _call(lib, fn, ctx, offs, a, tau, fc, df, N, T, w):
    R = offs.shape[0] - 1
    loss = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    ga = torch.full_like(a, float("nan"))
    H = torch.full((R, N), float("nan"), dtype=torch.complex64, device="cuda")
    ctx._stream()
    st = getattr(lib, fn)(ctx.h, _p(offs), R, _p(a), _p(tau), fc, df, N, _p(T), _p(w), _p(loss), _p(ga), _p(H))
    assert st == 0, (fn, st, lib.rt_last_error(ctx.h))
    torch.cuda.synchronize()
    return loss.cpu().numpy()[0], ga.cpu().numpy(), H.cpu().numpy()


@pytest.mark.parametrize("tensor_cores", [1, 0])
@pytest.mark.parametrize("N", [256, 1024])
def test_noalloc_matches_regular_entry_point(N, tensor_cores):
    import paper_2311_18558_gb300 as rt
    ctx = rt.Context(0)
    lib = ctx.lib
    rt.set_cfr_tensor_cores(ctx, tensor_cores)
    a, tau, offs = scenegen.random_cfr_inputs(77 + N, 96, 60, empty_every=11)
    fc, df = 1.272e9, 50e6 / N
    rng = np.random.default_rng(N)
    T = rng.uniform(1e-8, 1e-5, (96, N)).astype(np.float32)
    w = (1.0 / T.mean(axis=1)).astype(np.float32)
    args = (_dev(offs, torch.int64), _dev(a, torch.complex64), _dev(tau, torch.float64), fc, df, N,
            _dev(T, torch.float32), _dev(w, torch.float32))
    L_ref, ga_ref, H_ref = _call(lib, "rt_cfr_power_mse_fused", ctx, *args)
    assert np.isfinite(L_ref) and np.isfinite(ga_ref).all()
    for _ in range(2):
        L, ga, H = _call(lib, "rt_cfr_power_mse_fused_noalloc", ctx, *args)
        assert abs(L - L_ref) <= 1e-4 * abs(L_ref)
        assert np.linalg.norm(ga - ga_ref) <= 1e-4 * np.linalg.norm(ga_ref)
        assert np.linalg.norm(H - H_ref) <= 1e-4 * np.linalg.norm(H_ref)
    assert ctx.status_word() == 0


def test_noalloc_heavy_receiver():
    # 5000 paths on one receiver: exact sum here, non-uniform FFT in the regular call.
    # H and the loss are compared with the regular call and H with the oracle.  dL/da
    # = adjoint(4 w^2 (|H|^2 - P*) H / (R N)) magnifies any difference in H where |H|^2
    # is close to P*, so it is checked, per receiver, against the oracle's adjoint of
    # the loss derivative at the H this call returned (as the other fused-loss tests do).
    import paper_2311_18558_gb300 as rt
    ctx = rt.Context(0)
    lib = ctx.lib
    N = 256
    counts = np.array([5000, 3, 0, 40], np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)])
    rng = np.random.default_rng(5)
    P = int(offs[-1])
    a = (10.0 ** rng.uniform(-5, -2, P) * np.exp(1j * rng.uniform(0, 2 * np.pi, P))).astype(np.complex64)
    tau = rng.uniform(1e-9, 1.5e-6, P)
    fc, df = 1.272e9, 50e6 / N
    Href = oracle.cfr(a.astype(np.complex128), tau, offs, fc, df, N)
    T = (np.abs(Href) ** 2 * rng.uniform(0.5, 1.5, Href.shape)).astype(np.float32)
    w = oracle.power_weights(T).astype(np.float32)
    args = (_dev(offs, torch.int64), _dev(a, torch.complex64), _dev(tau, torch.float64), fc, df, N,
            _dev(T, torch.float32), _dev(w, torch.float32))
    L_reg, ga_reg, H_reg = _call(lib, "rt_cfr_power_mse_fused", ctx, *args)
    for _ in range(2):
        L, ga, H = _call(lib, "rt_cfr_power_mse_fused_noalloc", ctx, *args)
        assert abs(L - L_reg) <= 1e-4 * abs(L_reg)
        _, gH_at = oracle.power_mse(H.astype(np.complex128), T, w)
        ga_at = oracle.cfr_grad(tau, offs, fc, df, N, gH_at)
        for r in range(len(counts)):
            s = slice(offs[r], offs[r + 1])
            if counts[r]:
                assert np.linalg.norm(H[r] - H_reg[r]) <= 1e-4 * np.linalg.norm(H_reg[r]), r
                assert np.linalg.norm(H[r] - Href[r]) <= 1e-4 * np.linalg.norm(Href[r]), r
                assert np.linalg.norm(ga[s] - ga_at[s]) <= 1e-4 * np.linalg.norm(ga_at[s]), r
            else:
                assert np.all(H[r] == 0)
    assert ctx.status_word() == 0


def test_noalloc_rejects_too_many_receivers():
    import paper_2311_18558_gb300 as rt
    ctx = rt.Context(0)
    lib = ctx.lib
    R = 65537
    offs = torch.zeros(R + 1, dtype=torch.int64, device="cuda")
    tau = torch.zeros(1, dtype=torch.float64, device="cuda")
    a = torch.zeros(1, dtype=torch.complex64, device="cuda")
    T = torch.zeros((R, 2), dtype=torch.float32, device="cuda")
    w = torch.zeros(R, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ctx._stream()
    st = lib.rt_cfr_power_mse_fused_noalloc(ctx.h, _p(offs), R, _p(a), _p(tau), 1e9, 1e6, 2, _p(T), _p(w), _p(loss),
                                            _p(a), None)
    assert st == 1
    assert b"exceeds" in lib.rt_last_error(ctx.h)


def test_noalloc_inside_graph_capture():
    # A call captured in a CUDA graph after a first eager call on the device
    # (which looks up the fixed array's address): every replay redoes the whole
    # computation and must match the eager result.
    import paper_2311_18558_gb300 as rt
    ctx = rt.Context(0)
    lib = ctx.lib
    rt.set_cfr_tensor_cores(ctx, 1)
    N = 1024
    a, tau, offs = scenegen.random_cfr_inputs(2024, 64, 40, empty_every=9)
    fc, df = 3.5e9, 50e6 / N
    rng = np.random.default_rng(5)
    T = rng.uniform(1e-8, 1e-5, (64, N)).astype(np.float32)
    w = (1.0 / T.mean(axis=1)).astype(np.float32)
    args = (_dev(offs, torch.int64), _dev(a, torch.complex64), _dev(tau, torch.float64), fc, df, N,
            _dev(T, torch.float32), _dev(w, torch.float32))
    L_ref, ga_ref, H_ref = _call(lib, "rt_cfr_power_mse_fused_noalloc", ctx, *args)
    offs_d, a_d, tau_d, _, _, _, T_d, w_d = args
    R = offs_d.shape[0] - 1
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ga = torch.zeros_like(a_d)
    H = torch.zeros((R, N), dtype=torch.complex64, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx._stream()
        st = lib.rt_cfr_power_mse_fused_noalloc(ctx.h, _p(offs_d), R, _p(a_d), _p(tau_d), fc, df, N, _p(T_d),
                                                _p(w_d), _p(loss), _p(ga), _p(H))
        assert st == 0, lib.rt_last_error(ctx.h)
    for _ in range(2):
        loss.fill_(float("nan"))
        ga.fill_(float("nan"))
        H.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert abs(loss.item() - L_ref) <= 1e-6 * abs(L_ref)
        np.testing.assert_allclose(ga.cpu().numpy(), ga_ref, rtol=1e-5, atol=1e-12)
        np.testing.assert_allclose(H.cpu().numpy(), H_ref, rtol=1e-5, atol=1e-12)
    assert ctx.status_word() == 0
