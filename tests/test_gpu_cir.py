"""GPU CIR, delay spread, the paper's SMAPE loss, power scaling and metrics vs
the FP64 oracle (oracle/cir.py).

Tolerances: h normwise per receiver <= 1e-5 (FP32 FFT, log2 N stages); P and
tau_RMS relative <= 1e-4; loss relative <= 1e-4; dL/dH normwise <= 1e-4.  The
end-to-end gradient w.r.t. eps_r and sigma is compared with the oracle's FP64
chain applied at the CFR the GPU computed (the loss is a nonlinear function of
H, so the FP32 rounding of H is taken out of the comparison), at 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from gpu_helpers import assert_grad_close, gpu_trace, normwise_rows, oracle_trace
from oracle import cir as oc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def _dev(x, dtype):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda").contiguous()


def _random_H(seed, R, N, scale=1e-3):
    rng = np.random.default_rng(seed)
    return ((rng.normal(size=(R, N)) + 1j * rng.normal(size=(R, N))) * scale).astype(np.complex64)


@pytest.mark.parametrize("N", [2, 8, 64, 1024, 4096])
def test_cir_and_stats(rt, ctx, N):
    H = _random_H(N, 17, N)
    H[3] = 0   # a receiver without paths
    Hd = _dev(H, torch.complex64)
    h = rt.cir(ctx, Hd).cpu().numpy()
    href = oc.cir(H.astype(np.complex128))
    num, den = normwise_rows(h, href)
    nz = den > 0
    assert (num[nz] / den[nz]).max() <= 1e-5
    assert np.all(h[3] == 0)
    df = 50e6 / N
    P, t = rt.cir_stats(ctx, Hd, df)
    Pr, _, tr = oc.stats(H.astype(np.complex128), df)
    np.testing.assert_allclose(P.cpu().numpy()[nz], Pr[nz], rtol=1e-4)
    np.testing.assert_allclose(t.cpu().numpy()[nz], tr[nz], rtol=1e-4)
    assert P[3].item() == 0 and t[3].item() == 0


def test_stats_of_traced_cfr(rt, ctx):
    # the CIR statistics of a CFR from traced paths (indoor, 1024 subcarriers)
    sc = scenegen.indoor_diff()
    rx = sc.rx[::64]
    scene, p, ex = gpu_trace(rt, ctx, sc, n_rays=200_000, rx=rx)
    a = rt.eval_fields(ctx, p, _dev(sc.eps_r, torch.float32), _dev(sc.sigma, torch.float32), sc.freq_hz)
    H = rt.cfr(ctx, p.rx_offsets, a, p.tau, sc.f_center_hz, sc.delta_f_hz, sc.n_sub)
    P, t = rt.cir_stats(ctx, H, sc.delta_f_hz)
    Pr, _, tr = oc.stats(H.cpu().numpy().astype(np.complex128), sc.delta_f_hz)
    ok = Pr > 0
    np.testing.assert_allclose(P.cpu().numpy()[ok], Pr[ok], rtol=1e-4)
    np.testing.assert_allclose(t.cpu().numpy()[ok], tr[ok], rtol=1e-4)
    assert 1e-10 < np.median(tr[ok]) < 1e-6   # tens of ns in a 20 m room


@pytest.mark.parametrize("N", [64, 1024])
def test_loss_and_gradient(rt, ctx, N):
    rng = np.random.default_rng(N + 1)
    R = 40
    H = _random_H(N + 2, R, N)
    H[5] = 0
    df = 50e6 / N
    Pr, _, tr = oc.stats(H.astype(np.complex128), df)
    Pm = (Pr * rng.uniform(0.3, 3.0, R) + 1e-9).astype(np.float32)
    tm = (np.where(tr > 0, tr, 1e-8) * rng.uniform(0.5, 2.0, R)).astype(np.float32)
    state = torch.tensor([1.7, 1.0], device="cuda")
    Hd = _dev(H, torch.complex64)
    Pp = torch.empty(R, device="cuda")
    tp = torch.empty(R, device="cuda")
    for _ in range(2):   # twice: the completion counter resets itself
        loss, gH = rt.delay_spread_power_loss(ctx, Hd, df, _dev(Pm, torch.float32), _dev(tm, torch.float32), state,
                                              P_pred=Pp, tau_pred=tp)
        L_ref, gH_ref = oc.loss(H.astype(np.complex128), Pm, tm, df, 1.7)
        assert abs(loss.item() - L_ref) <= 1e-4 * abs(L_ref)
        g = gH.cpu().numpy()
        assert np.linalg.norm(g - gH_ref) <= 1e-4 * np.linalg.norm(gH_ref)
    np.testing.assert_allclose(Pp.cpu().numpy(), Pr, rtol=1e-4, atol=1e-30)
    assert ctx.status_word() == 0


def test_power_scale_ema_and_metrics(rt, ctx):
    rng = np.random.default_rng(7)
    Pm = rng.uniform(1e-9, 1e-6, 300).astype(np.float32)
    P1 = (Pm * 2.5 * rng.uniform(0.9, 1.1, 300)).astype(np.float32)
    P2 = (Pm * 3.5 * rng.uniform(0.9, 1.1, 300)).astype(np.float32)
    state = torch.zeros(2, device="cuda")
    rt.power_scale_ema(ctx, _dev(Pm, torch.float32), _dev(P1, torch.float32), 0.9, state)
    a1 = oc.alpha_ema(None, oc.alpha_hat(Pm, P1), 0.9, first=True)
    np.testing.assert_allclose(state[0].item(), a1, rtol=1e-5)
    rt.power_scale_ema(ctx, _dev(Pm, torch.float32), _dev(P2, torch.float32), 0.9, state)
    a2 = oc.alpha_ema(a1, oc.alpha_hat(Pm, P2), 0.9, first=False)
    np.testing.assert_allclose(state[0].item(), a2, rtol=1e-5)
    tm = rng.uniform(1e-8, 5e-8, 300).astype(np.float32)
    tp = (tm * rng.uniform(0.5, 1.5, 300)).astype(np.float32)
    ale, rae = rt.cir_metrics(ctx, _dev(Pm, torch.float32), _dev(tm, torch.float32), _dev(P1, torch.float32),
                              _dev(tp, torch.float32), state)
    np.testing.assert_allclose(ale.cpu().numpy(), oc.ale_db(a2 * Pm.astype(np.float64), P1), rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(rae.cpu().numpy(), oc.rae(tm, tp), rtol=1e-5, atol=1e-7)


def test_paper_loss_gradient_end_to_end(rt, ctx):
    # autograd through eval_fields -> CFR -> the paper's loss, against the oracle's FP64
    # adjoint chain applied at the CFR the GPU computed
    sc = scenegen.indoor_diff()
    rx = sc.rx[::16]
    scene, p, ex = gpu_trace(rt, ctx, sc, n_rays=200_000, rx=rx)
    o, tr = oracle_trace(sc, n_rays=200_000, rx=rx)
    fc, df, N = sc.f_center_hz, sc.delta_f_hz, sc.n_sub
    sc2 = sc.subset_rx(np.arange(0, sc.n_rx, 16))
    ors = oracle.OracleScene(sc2)
    H_gt = oracle.cfr(ors.fields(tr), tr["tau"], tr["rx_offsets"], fc, df, N)
    Pm, _, tm = oc.stats(H_gt, df)
    keep = Pm > 0
    Pm = np.where(keep, Pm, 1e-30).astype(np.float32)
    tm = np.where(keep, tm, 1e-9).astype(np.float32)
    eps0 = np.full(8, 4.0, np.float32)
    sig0 = np.full(8, 0.05, np.float32)
    params = rt.LogMaterials(eps0, sig0).cuda()
    eps, sig = params()
    state = torch.tensor([1.0, 1.0], device="cuda")
    loss = rt.paper_calibration_loss(ctx, p, eps, sig, _dev(Pm, torch.float32), _dev(tm, torch.float32), state,
                                     sc.freq_hz, fc, df, N, update_scale=False)
    loss.backward()
    a_gpu = rt.eval_fields(ctx, p, torch.tensor(eps0, device="cuda"), torch.tensor(sig0, device="cuda"), sc.freq_hz)
    H_gpu = rt.cfr(ctx, p.rx_offsets, a_gpu, p.tau, fc, df, N).cpu().numpy().astype(np.complex128)
    L_ref, gH = oc.loss(H_gpu, Pm, tm, df, 1.0)
    ga = oracle.cfr_grad(tr["tau"], tr["rx_offsets"], fc, df, N, gH)
    ge, gs, _ = ors.fields_grad(tr, ga, eps_r=eps0, sigma=sig0)
    assert abs(loss.item() - L_ref) <= 1e-4 * L_ref
    got_e = params.w_eps.grad.cpu().numpy()
    got_s = params.w_sigma.grad.cpu().numpy()
    g_weps = ge * (eps0 - 1.0)
    g_wsig = gs * sig0
    assert_grad_close(got_e, g_weps, what="eps_r")
    assert_grad_close(got_s, g_wsig, what="sigma")


@pytest.mark.parametrize("param", ["log", "embeddings"])
def test_paper_loss_calibration_descends(rt, ctx, param):
    # Algorithm 1 with the paper's loss and the moving-average power scale on the
    # indoor scene: the loss on the training receivers falls by half within 60 steps,
    # with per-material log parameters or with L = 30 material embeddings
    # (Eq. trainable_materials_1/2; Adam's per-element step moves v . w by about
    # lr sqrt(L), hence the smaller rate)
    sc = scenegen.indoor_diff()
    dev = "cuda"
    scene = rt.Scene.from_synthetic(ctx, sc)
    rx = torch.tensor(sc.rx, device=dev)
    p = rt.trace_paths(ctx, scene, sc.tx, rx, 300_000, sc.max_depth)
    fc, df, N = sc.f_center_hz, sc.delta_f_hz, sc.n_sub
    a = rt.eval_fields(ctx, p, torch.tensor(sc.eps_r, device=dev), torch.tensor(sc.sigma, device=dev), sc.freq_hz)
    H = rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N)
    Pm, tm = rt.cir_stats(ctx, H, df)
    Pm = Pm * 0.25                     # measurements known up to a common scale
    keep = Pm > 0
    Pm = torch.where(keep, Pm, torch.full_like(Pm, 1e-30)).contiguous()
    tm = torch.where(keep, tm, torch.full_like(tm, 1e-9)).contiguous()
    if param == "log":
        params = rt.LogMaterials(np.full(8, 4.0), np.full(8, 0.05)).cuda()
        lr = 0.05
    else:
        params = rt.MaterialEmbeddings(np.full(8, 4.0), np.full(8, 0.05), L=30, seed=2).cuda()
        lr = 0.01
    opt = torch.optim.Adam(params.parameters(), lr=lr)
    state = torch.zeros(2, device=dev)
    losses = []
    for _ in range(60):
        eps, sig = params()
        L = rt.paper_calibration_loss(ctx, p, eps.contiguous(), sig.contiguous(), Pm, tm, state, sc.freq_hz, fc, df,
                                      N, decay=0.9)
        opt.zero_grad()
        L.backward()
        opt.step()
        losses.append(L.item())
    assert losses[-1] < 0.5 * losses[0], losses[::10]
    assert abs(state[0].item() - 4.0) < 2.0   # the scale settles near 1 / 0.25
    assert ctx.status_word() == 0
