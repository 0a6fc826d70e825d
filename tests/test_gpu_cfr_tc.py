"""Tensor-core CFR (tcgen05, 3xTF32) vs the FP64 oracle and vs the SIMT path.

Receivers carry path counts at the chunk edges of the tensor-core kernel (32
paths per chunk): 0, 1, 31, 32, 33, 64, 65 and 100.  Tolerances as for the SIMT
path: CFR normwise per receiver <= 1e-4, gradients normwise <= 1e-4, loss
relative <= 1e-4 (FP32 GPU vs FP64 oracle).

The fused gradient is dL/da for dL/dH = 4 w^2 (|H|^2 - P*) H / (R N) at the
kernel's own H.  Where |H|^2 is close to P* that derivative magnifies any
rounding of H (by ~2 |H|^2 / | |H|^2 - P* |), so the fused gradient is checked
against the oracle's adjoint applied to the loss derivative at the H the kernel
returned, and that H against the oracle's CFR; both at 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import normwise_rows

pytestmark = pytest.mark.gpu

COUNTS = np.array([0, 1, 31, 32, 33, 64, 65, 100, 7, 0, 2, 40], np.int64)


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def _dev(x, dtype):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda").contiguous()


def _inputs(seed):
    rng = np.random.default_rng(seed)
    offs = np.zeros(len(COUNTS) + 1, np.int64)
    offs[1:] = np.cumsum(COUNTS)
    P = int(offs[-1])
    a = (10.0 ** rng.uniform(-5, -2, P) * np.exp(1j * rng.uniform(0, 2 * np.pi, P))).astype(np.complex64)
    tau = rng.uniform(1e-9, 1.5e-6, P)
    return a, tau, offs


def _run(rt, ctx, tensor_cores, a, tau, offs, fc, df, N, gH, T, w):
    rt.set_cfr_tensor_cores(ctx, tensor_cores)
    try:
        o, ad, td = _dev(offs, torch.int64), _dev(a, torch.complex64), _dev(tau, torch.float64)
        H = rt.cfr(ctx, o, ad, td, fc, df, N).cpu().numpy()
        ga = rt.cfr_backward(ctx, o, td, fc, df, N, _dev(gH, torch.complex64)).cpu().numpy()
        Hf = torch.empty((len(offs) - 1, N), dtype=torch.complex64, device="cuda")
        out = []
        for _ in range(2):   # twice: the kernel's counters must reset themselves
            loss, gaf, _ = rt.cfr_power_mse_fused(ctx, o, ad, td, fc, df, N, _dev(T, torch.float32),
                                                  _dev(w, torch.float32), H=Hf)
            out.append((loss.item(), gaf.cpu().numpy(), Hf.cpu().numpy()))
        assert ctx.status_word() == 0
        return H, ga, out
    finally:
        rt.set_cfr_tensor_cores(ctx, True)


@pytest.mark.parametrize("n_sub", [256, 512, 1024, 2048, 4096])
def test_cfr_tensor_cores(rt, ctx, n_sub):
    a, tau, offs = _inputs(100 + n_sub)
    fc, df = 1.272e9, 50e6 / n_sub
    rng = np.random.default_rng(n_sub)
    Href = oracle.cfr(a.astype(np.complex128), tau, offs, fc, df, n_sub)
    gH = (rng.normal(size=Href.shape) + 1j * rng.normal(size=Href.shape)).astype(np.complex64)
    ga_ref = oracle.cfr_grad(tau, offs, fc, df, n_sub, gH.astype(np.complex128))
    T = (np.abs(Href) ** 2 * rng.uniform(0.5, 1.5, Href.shape)).astype(np.float32)
    w = oracle.power_weights(T).astype(np.float32)
    L_ref, _ = oracle.power_mse(Href, T, w)

    results = {}
    for tc in (True, False):
        H, ga, fused = _run(rt, ctx, tc, a, tau, offs, fc, df, n_sub, gH, T, w)
        num, den = normwise_rows(H, Href)
        nz = den > 0
        assert (num[nz] / den[nz]).max() <= 1e-4, (tc, (num[nz] / den[nz]).max())
        assert np.all(H[~nz] == 0)
        assert np.linalg.norm(ga - ga_ref) <= 1e-4 * np.linalg.norm(ga_ref), tc
        for loss, gaf, Hf in fused:
            assert abs(loss - L_ref) <= 1e-4 * abs(L_ref), (tc, loss, L_ref)
            num, den = normwise_rows(Hf, Href)
            assert (num[den > 0] / den[den > 0]).max() <= 1e-4
            _, gH_at = oracle.power_mse(Hf.astype(np.complex128), T, w)
            ga_at = oracle.cfr_grad(tau, offs, fc, df, n_sub, gH_at)
            assert np.linalg.norm(gaf - ga_at) <= 1e-4 * np.linalg.norm(ga_at), tc
        results[tc] = (H, ga, fused[0][0])
    # the two arithmetic paths agree with each other as closely as each with the oracle
    num, den = normwise_rows(results[True][0], results[False][0])
    nz = den > 0
    assert (num[nz] / den[nz]).max() <= 2e-4
    assert abs(results[True][2] - results[False][2]) <= 2e-4 * abs(L_ref)


# receivers above 4096 paths are split over CTAs (segments of 1024 paths) and
# evaluated by a non-uniform FFT, in the fused loss, the plain CFR and its
# adjoint; 4096 itself stays whole
SPLIT_COUNTS = np.array([3, 4096, 4097, 9000, 0, 40000, 17, 5000], np.int64)


@pytest.mark.parametrize("n_sub", [256, 1024])
def test_fused_split_receivers(rt, ctx, n_sub):
    rng = np.random.default_rng(7 + n_sub)
    offs = np.zeros(len(SPLIT_COUNTS) + 1, np.int64)
    offs[1:] = np.cumsum(SPLIT_COUNTS)
    P = int(offs[-1])
    a = (10.0 ** rng.uniform(-5, -2, P) * np.exp(1j * rng.uniform(0, 2 * np.pi, P))).astype(np.complex64)
    tau = rng.uniform(1e-9, 1.5e-6, P)
    fc, df = 1.272e9, 50e6 / n_sub
    Href = oracle.cfr(a.astype(np.complex128), tau, offs, fc, df, n_sub)
    T = (np.abs(Href) ** 2 * rng.uniform(0.5, 1.5, Href.shape)).astype(np.float32)
    w = oracle.power_weights(T).astype(np.float32)
    L_ref, _ = oracle.power_mse(Href, T, w)
    o, ad, td = _dev(offs, torch.int64), _dev(a, torch.complex64), _dev(tau, torch.float64)
    # the plain CFR and its adjoint split the same receivers
    gH = (rng.normal(size=Href.shape) + 1j * rng.normal(size=Href.shape)).astype(np.complex64)
    ga_ref = oracle.cfr_grad(tau, offs, fc, df, n_sub, gH.astype(np.complex128))
    for _ in range(2):
        Hc = rt.cfr(ctx, o, ad, td, fc, df, n_sub).cpu().numpy()
        num, den = normwise_rows(Hc, Href)
        assert (num[den > 0] / den[den > 0]).max() <= 1e-4
        assert np.all(Hc[SPLIT_COUNTS == 0] == 0)
        gab = rt.cfr_backward(ctx, o, td, fc, df, n_sub, _dev(gH, torch.complex64)).cpu().numpy()
        for r in range(len(SPLIT_COUNTS)):
            s = slice(offs[r], offs[r + 1])
            if offs[r + 1] > offs[r]:
                assert np.linalg.norm(gab[s] - ga_ref[s]) <= 1e-4 * np.linalg.norm(ga_ref[s]), r
    Hf = torch.empty((len(offs) - 1, n_sub), dtype=torch.complex64, device="cuda")
    for _ in range(2):   # twice: counters, flags and rows must be reset by each call
        loss, gaf, _ = rt.cfr_power_mse_fused(ctx, o, ad, td, fc, df, n_sub, _dev(T, torch.float32),
                                              _dev(w, torch.float32), H=Hf)
        loss, gaf, H = loss.item(), gaf.cpu().numpy(), Hf.cpu().numpy()
        assert abs(loss - L_ref) <= 1e-4 * abs(L_ref), (loss, L_ref)
        num, den = normwise_rows(H, Href)
        assert (num[den > 0] / den[den > 0]).max() <= 1e-4
        assert np.all(H[SPLIT_COUNTS == 0] == 0)
        _, gH_at = oracle.power_mse(H.astype(np.complex128), T, w)
        ga_at = oracle.cfr_grad(tau, offs, fc, df, n_sub, gH_at)
        for r in range(len(SPLIT_COUNTS)):   # per receiver, so a split one cannot hide behind the others
            s = slice(offs[r], offs[r + 1])
            if offs[r + 1] > offs[r]:
                assert np.linalg.norm(gaf[s] - ga_at[s]) <= 1e-4 * np.linalg.norm(ga_at[s]), r
    assert ctx.status_word() == 0


RT_ERR_TIMEOUT = 7


def test_wait_timeout_sets_status(rt, ctx):
    # With a limit of one poll, a CTA that has to move from the forward segments of
    # the split receivers to their adjoint segments (which takes one poll of its
    # own) runs out: every call of this shape sets RT_ERR_TIMEOUT.  The kernel must
    # return, the status word must say so, and the next call with the default limit
    # must be correct (nothing left behind by the cut-short call).
    counts = np.array([5000, 3, 9000, 0, 60], np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)])
    rng = np.random.default_rng(21)
    P = int(offs[-1])
    a = (10.0 ** rng.uniform(-5, -2, P) * np.exp(1j * rng.uniform(0, 2 * np.pi, P))).astype(np.complex64)
    tau = rng.uniform(1e-9, 1.5e-6, P)
    n_sub = 256
    fc, df = 1.272e9, 50e6 / n_sub
    Href = oracle.cfr(a.astype(np.complex128), tau, offs, fc, df, n_sub)
    T = (np.abs(Href) ** 2 * rng.uniform(0.5, 1.5, Href.shape)).astype(np.float32)
    w = oracle.power_weights(T).astype(np.float32)
    L_ref, _ = oracle.power_mse(Href, T, w)
    args = (_dev(offs, torch.int64), _dev(a, torch.complex64), _dev(tau, torch.float64), fc, df, n_sub,
            _dev(T, torch.float32), _dev(w, torch.float32))
    assert ctx.status_word() == 0
    with pytest.raises(Exception):
        rt.set_wait_limit(ctx, -1)
    rt.set_wait_limit(ctx, 1)
    try:
        rt.cfr_power_mse_fused(ctx, *args)
        torch.cuda.synchronize()
        assert ctx.status_word() == RT_ERR_TIMEOUT
    finally:
        rt.set_wait_limit(ctx, 0)
    for _ in range(2):
        loss, ga, _ = rt.cfr_power_mse_fused(ctx, *args)
        assert abs(loss.item() - L_ref) <= 1e-4 * abs(L_ref)
    assert ctx.status_word() == 0


def test_fused_split_beyond_heavy_cap(rt, ctx):
    # 4100 receivers of 4097 paths: the first 4096 are split, the rest stay whole.
    # Receivers on both sides of the cap are checked against the FP64 oracle one
    # by one (a receiver's H and dL/da depend only on its own paths and target,
    # with the loss normalised by R N of the whole call)
    R, n_sub, Pr = 4100, 256, 4097
    rng = np.random.default_rng(11)
    P = R * Pr
    a_h = (10.0 ** rng.uniform(-5, -2, P) * np.exp(1j * rng.uniform(0, 2 * np.pi, P))).astype(np.complex64)
    tau_h = rng.uniform(1e-9, 1.5e-6, P)
    offs = torch.arange(R + 1, dtype=torch.int64, device="cuda") * Pr
    a, tau = _dev(a_h, torch.complex64), _dev(tau_h, torch.float64)
    fc, df = 1.272e9, 50e6 / n_sub
    T = (rt.cfr(ctx, offs, a, tau, fc, df, n_sub).abs() ** 2 * 1.3).float().contiguous()
    w = torch.ones(R, device="cuda")
    H = torch.empty((R, n_sub), dtype=torch.complex64, device="cuda")
    loss, ga, _ = rt.cfr_power_mse_fused(ctx, offs, a, tau, fc, df, n_sub, T, w, H=H)
    H, ga, T = H.cpu().numpy(), ga.cpu().numpy(), T.cpu().numpy()
    one = np.array([0, Pr], np.int64)
    for r in (0, 4095, 4096, 4099):
        s = slice(r * Pr, (r + 1) * Pr)
        Href = oracle.cfr(a_h[s].astype(np.complex128), tau_h[s], one, fc, df, n_sub)
        assert np.linalg.norm(H[r] - Href[0]) <= 1e-4 * np.linalg.norm(Href[0]), r
        _, gH_at = oracle.power_mse(H[r:r + 1].astype(np.complex128), T[r:r + 1], np.ones(1))
        ga_at = oracle.cfr_grad(tau_h[s], one, fc, df, n_sub, gH_at / R)
        err = np.linalg.norm(ga[s] - ga_at) / np.linalg.norm(ga_at)
        assert err <= 1e-4, (r, err)
    assert ctx.status_word() == 0
