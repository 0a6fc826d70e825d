"""Pins of the FP64 oracle of the CIR, delay spread, SMAPE loss and power scaling
(oracle/cir.py) to closed forms and to numerical differentiation."""
import numpy as np

import oracle
from oracle import cir as oc


def _cfr_of_taps(N, df, taps, fc=1.272e9):
    """CFR of paths at integer multiples k/W of the delay resolution: H[n] = sum a_k e^{-j 2 pi (fc + n df) tau_k}."""
    n = np.arange(N) - N // 2
    W = N * df
    H = np.zeros(N, np.complex128)
    for k, a in taps:
        tau = k / W
        H += a * np.exp(-2j * np.pi * (fc + n * df) * tau)
    return H


def test_cir_matches_numpy_ifft():
    # h is the centred IDFT: ifftshift / ifft / fftshift with sqrt(N) scaling
    rng = np.random.default_rng(0)
    H = rng.normal(size=(3, 64)) + 1j * rng.normal(size=(3, 64))
    ref = np.fft.fftshift(np.fft.ifft(np.fft.ifftshift(H, axes=-1), axis=-1), axes=-1) * np.sqrt(64)
    np.testing.assert_allclose(oc.cir(H), ref, rtol=0, atol=1e-12)


def test_parseval_and_adjoint():
    rng = np.random.default_rng(1)
    H = rng.normal(size=(2, 32)) + 1j * rng.normal(size=(2, 32))
    h = oc.cir(H)
    np.testing.assert_allclose((np.abs(h) ** 2).sum(-1), (np.abs(H) ** 2).sum(-1), rtol=1e-12)
    g = rng.normal(size=h.shape) + 1j * rng.normal(size=h.shape)
    # <cir(H), g> = <H, cir_adjoint(g)>
    np.testing.assert_allclose(np.vdot(g, oc.cir(H)), np.vdot(oc.cir_adjoint(g), H), rtol=1e-12)


def test_single_tap_closed_form():
    # one path at delay k/W: all power on tap k, tau_bar = k, tau_RMS = 0, P = N |a|^2
    N, df = 256, 50e6 / 256
    H = _cfr_of_taps(N, df, [(7, 0.3 - 0.1j)])[None, :]
    h = oc.cir(H)[0]
    p = np.abs(h) ** 2
    assert np.argmax(p) == 7 + N // 2
    P, tbar, trms = oc.stats(H, df)
    np.testing.assert_allclose(P, N * abs(0.3 - 0.1j) ** 2, rtol=1e-12)
    np.testing.assert_allclose(tbar, 7.0, atol=1e-9)
    assert trms[0] < 1e-12


def test_two_taps_closed_form():
    # taps k1, k2 with powers p1, p2: tau_RMS = |k1 - k2| sqrt(p1 p2) / (p1 + p2) / W
    N, df = 512, 50e6 / 512
    W = N * df
    a1, a2 = 0.5, 0.2 + 0.1j
    H = _cfr_of_taps(N, df, [(3, a1), (40, a2)])[None, :]
    p1, p2 = abs(a1) ** 2, abs(a2) ** 2
    P, tbar, trms = oc.stats(H, df)
    np.testing.assert_allclose(tbar, (3 * p1 + 40 * p2) / (p1 + p2), rtol=1e-10)
    np.testing.assert_allclose(trms, 37 * np.sqrt(p1 * p2) / (p1 + p2) / W, rtol=1e-10)


def test_smape_properties():
    x = np.array([1.0, 2.0, 0.0, 5.0])
    y = np.array([1.0, 1.0, 0.0, 0.0])
    s = oc.smape(x, y)
    np.testing.assert_allclose(s, [0.0, 1.0 / 3.0, 0.0, 1.0])
    np.testing.assert_allclose(oc.smape(y, x), s)   # symmetric
    # derivative against central differences
    for xv, yv in [(2.0, 1.0), (1.0, 3.0)]:
        e = 1e-6
        fd = (oc.smape(xv, yv + e) - oc.smape(xv, yv - e)) / (2 * e)
        np.testing.assert_allclose(oc.smape_dy(xv, yv), fd, rtol=1e-6)


def test_alpha_closed_form_and_ema():
    rng = np.random.default_rng(3)
    Pm = rng.uniform(1e-9, 1e-6, 50)
    assert abs(oc.alpha_hat(Pm, 3.5 * Pm) - 3.5) < 1e-12
    a = oc.alpha_ema(None, 2.0, 0.9, first=True)
    assert a == 2.0                               # alpha_0 = alpha^_1
    a = oc.alpha_ema(a, 4.0, 0.9, first=False)
    np.testing.assert_allclose(a, 0.9 * 2.0 + 0.1 * 4.0)


def test_metrics():
    np.testing.assert_allclose(oc.ale_db([1.0, 1e-3], [10.0, 1e-3]), [10.0, 0.0])
    np.testing.assert_allclose(oc.rae([2e-8, 1e-8], [1e-8, 1e-8]), [0.5, 0.0])


def test_loss_gradient_finite_differences():
    # the analytic gradient of Eq. loss against central differences of the loss
    rng = np.random.default_rng(4)
    N, df = 32, 50e6 / 32
    R = 3
    H = (rng.normal(size=(R, N)) + 1j * rng.normal(size=(R, N))) * 1e-3
    Pm = rng.uniform(0.5, 2.0, R) * (np.abs(H) ** 2).sum(-1)
    tm = rng.uniform(0.5, 2.0, R) * oc.stats(H, df)[2]
    alpha = 1.3
    L, g = oc.loss(H, Pm, tm, df, alpha)
    e = 1e-9
    for (r, n) in [(0, 0), (1, 5), (2, 31)]:
        for part in (1.0, 1j):
            Hp, Hm = H.copy(), H.copy()
            Hp[r, n] += e * part
            Hm[r, n] -= e * part
            fd = (oc.loss(Hp, Pm, tm, df, alpha)[0] - oc.loss(Hm, Pm, tm, df, alpha)[0]) / (2 * e)
            got = g[r, n].real if part == 1.0 else g[r, n].imag
            np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-9 * abs(fd) + 1e-12)


def test_loss_on_traced_cfr_is_zero_at_truth():
    # the loss of a CFR against its own statistics (alpha = 1) is exactly 0
    sc_H = oracle.cfr(np.array([1e-3 + 0j, 2e-4j]), np.array([1e-7, 3e-7]), np.array([0, 2]), 1.272e9, 50e6 / 64, 64)
    P, _, t = oc.stats(sc_H, 50e6 / 64)
    L, g = oc.loss(sc_H, P, t, 50e6 / 64, 1.0)
    assert L == 0.0
