"""Trainable antenna patterns on the GPU (rt_antenna_apply and its adjoint) vs
the FP64 oracle (oracle/antenna.py), and their recovery by gradient descent.

Tolerances: per-path coefficients and gains within 1e-5 relative (FP32
directions and exponentials); pattern gradients within 1e-4 normwise."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from gpu_helpers import assert_grad_close, assert_same_paths, gpu_trace, oracle_trace
from oracle import antenna as oa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


@pytest.fixture(scope="module")
def indoor(rt, ctx):
    sc = scenegen.indoor_diff()
    rx = sc.rx[::32]
    scene, p, ex = gpu_trace(rt, ctx, sc, n_rays=200_000, rx=rx)
    o, tr = oracle_trace(sc, n_rays=200_000, rx=rx)
    assert_same_paths(ex, tr, o.diag)
    return sc.subset_rx(np.arange(0, sc.n_rx, 32)), p, tr


def _pack(eta, w, lam, mu):
    return np.concatenate([[eta], np.concatenate([np.asarray(w)[:, None], np.asarray(lam)[:, None],
                                                  np.asarray(mu)], 1).reshape(-1)]).astype(np.float32)


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


TX = (0.9, np.array([0.6, 0.4]), np.array([3.0, 15.0]), _unit([[0.3, 0.1, -0.9], [1.0, 0.5, 0.2]]))
RX = (0.8, np.array([1.0]), np.array([1.5]), _unit([[0.0, 0.2, 1.0]]))


def _fp32(pat):
    """The pattern as the GPU sees it (FP32 values), for the oracle."""
    p = _pack(*pat).astype(np.float64)
    M = (len(p) - 1) // 5
    lob = p[1:].reshape(M, 5)
    return lob[:, 0], lob[:, 1], lob[:, 2:5], p[0]


def test_apply_matches_oracle(rt, ctx, indoor):
    sc, p, tr = indoor
    a = rt.eval_fields(ctx, p, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
                       sc.freq_hz)
    txd = torch.tensor(_pack(*TX), device="cuda")
    rxd = torch.tensor(_pack(*RX), device="cuda")
    a_out, gt, gr = rt.antenna_apply(ctx, p, a, txd, rxd)
    aod, aoa = oa.directions(tr["pts"], tr["depth"])
    w, lam, mu, eta = _fp32(TX)
    gt_ref = oa.gain(aod, w, lam, mu, eta)
    w2, lam2, mu2, eta2 = _fp32(RX)
    gr_ref = oa.gain(aoa, w2, lam2, mu2, eta2)
    np.testing.assert_allclose(gt.cpu().numpy(), gt_ref, rtol=1e-5)
    np.testing.assert_allclose(gr.cpu().numpy(), gr_ref, rtol=1e-5)
    a_gpu = a.cpu().numpy()
    np.testing.assert_allclose(a_out.cpu().numpy(), a_gpu * np.sqrt(gt_ref * gr_ref), rtol=1e-5, atol=0)
    # no pattern on either side: the coefficients pass unchanged
    a_id, _, _ = rt.antenna_apply(ctx, p, a)
    assert torch.equal(a_id, a)
    assert ctx.status_word() == 0


def test_backward_matches_oracle(rt, ctx, indoor):
    sc, p, tr = indoor
    rng = np.random.default_rng(5)
    a = rt.eval_fields(ctx, p, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
                       sc.freq_hz)
    txd = torch.tensor(_pack(*TX), device="cuda")
    rxd = torch.tensor(_pack(*RX), device="cuda")
    a_out, gt, gr = rt.antenna_apply(ctx, p, a, txd, rxd)
    P = p.n_paths
    g = (rng.normal(size=P) + 1j * rng.normal(size=P)).astype(np.complex64) * 1e3
    ga, gtx, grx = rt.antenna_apply_backward(ctx, p, a_out, gt, gr, torch.tensor(g, device="cuda"), txd, rxd)
    aod, aoa = oa.directions(tr["pts"], tr["depth"])
    a_out_h = a_out.cpu().numpy().astype(np.complex128)
    gt_h, gr_h = gt.cpu().numpy().astype(np.float64), gr.cpu().numpy().astype(np.float64)
    da, dgt, dgr = oa.apply_grad(a_out_h, gt_h, gr_h, g.astype(np.complex128))
    np.testing.assert_allclose(ga.cpu().numpy(), da, rtol=1e-5, atol=1e-30)
    for pat, d, dirs, got in ((TX, dgt, aod, gtx), (RX, dgr, aoa, grx)):
        w, lam, mu, eta = _fp32(pat)
        dw, dlam, dmu = oa.gain_grad(dirs, w, lam, mu, eta, d)
        deta = float((d * oa.gain(dirs, w, lam, mu, eta)).sum() / eta)
        ref = np.concatenate([[deta], np.concatenate([dw[:, None], dlam[:, None], dmu], 1).reshape(-1)])
        assert_grad_close(got.cpu().numpy(), ref)


def test_pattern_recovery(rt, ctx, indoor):
    # a hidden one-lobe transmit pattern is recovered from CFR powers through the
    # calibration chain: eval_fields -> pattern -> CFR + power MSE
    sc, p, tr = indoor
    dev = "cuda"
    fc, df, N = sc.f_center_hz, sc.delta_f_hz, 256
    eps = torch.tensor(sc.eps_r, device=dev)
    sig = torch.tensor(sc.sigma, device=dev)
    a0 = rt.eval_fields(ctx, p, eps, sig, sc.freq_hz)
    mu_true = _unit([0.5, -0.6, -0.3])
    hidden = torch.tensor(_pack(1.0, [1.0], [4.0], mu_true[None, :]), device=dev)
    a_t, _, _ = rt.antenna_apply(ctx, p, a0, hidden)
    T = (rt.cfr(ctx, p.rx_offsets, a_t, p.tau, fc, df, N).abs() ** 2).float().contiguous()
    m = T.mean(1)
    w = torch.where(m > 0, 1 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).contiguous()
    pat = rt.AntennaPattern(n_lobes=1, lam_init=1.0, eta_init=0.9, seed=3).to(dev)
    opt = torch.optim.Adam(pat.parameters(), lr=0.05)
    losses = []
    for _ in range(200):
        a = rt.AntennaApply.apply(a0, pat(), None, ctx, p)
        L = rt.CfrPowerMSE.apply(a, p.tau, p.rx_offsets, T, w, ctx, fc, df, N)
        opt.zero_grad()
        L.backward()
        opt.step()
        losses.append(L.item())
    mu = torch.nn.functional.normalize(pat.mu_raw.detach(), dim=1)[0].cpu().numpy()
    assert losses[-1] < 0.1 * losses[0], losses[::20]
    assert float(mu @ mu_true) > 0.9, (mu, mu_true)
    assert ctx.status_word() == 0
