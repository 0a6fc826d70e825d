"""FP64 oracle of the paper's calibration loss and metrics (arXiv 2311.18558):
the CIR by N-point IDFT (Sec. II-A), total channel gain (Eq. channel_gain), RMS
delay spread (Eq. delay_spread), the SMAPE loss (Eq. smape, Eq. loss), the
power scaling by an exponential moving average (Eq. scaling_param, alpha_hat),
and the evaluation metrics ALE and RAE (Sec. IV-C).

Test infrastructure only: tests, the smoke check and the benchmark's CPU
baseline may call it; the library never does.

Readings (where the paper is silent):
  - H is stored as the library stores it: row r, column n + N/2 for
    n = -N/2 .. N/2-1; h likewise, column l + N/2 for l = -N/2 .. N/2-1.
  - A CIR with P = 0 (a receiver without paths) has tau_RMS = 0 and passes no
    gradient through its delay statistics; SMAPE(0, 0) = 0.
  - alpha scales the measured powers only (Algorithm 1 scales h_b by sqrt(alpha),
    so P_b -> alpha P_b and tau_RMS,b is unchanged) and carries no gradient.
"""
import numpy as np


def cir(H):
    """h[l] = N^-1/2 sum_n H[n] exp(+j 2 pi n l / N), n, l = -N/2 .. N/2-1 (Sec. II-A),
    written as the direct sum."""
    H = np.asarray(H, np.complex128)
    N = H.shape[-1]
    k = np.arange(N) - N // 2
    E = np.exp(2j * np.pi * np.outer(k, k) / N) / np.sqrt(N)   # E[n, l]
    return H @ E


def cir_adjoint(g_h):
    """Adjoint of cir() (the map is linear and unitary): g_H = E^H g_h."""
    g_h = np.asarray(g_h, np.complex128)
    N = g_h.shape[-1]
    k = np.arange(N) - N // 2
    E = np.exp(2j * np.pi * np.outer(k, k) / N) / np.sqrt(N)
    return g_h @ E.conj().T


def stats(H, delta_f):
    """Per receiver: P = sum_l p_l (Eq. channel_gain), tau_bar = sum_l l p_l / P and
    tau_RMS = sqrt(sum_l ((l - tau_bar) / W)^2 p_l / P) (Eq. delay_spread) with
    p_l = |h[l]|^2 and W = N delta_f; tau_RMS = 0 where P = 0."""
    h = cir(H)
    N = h.shape[-1]
    W = N * float(delta_f)
    p = np.abs(h) ** 2
    ell = np.arange(N) - N // 2
    P = p.sum(-1)
    safe = np.where(P > 0, P, 1.0)
    tbar = (p * ell).sum(-1) / safe
    var = (((ell[None, :] - tbar[:, None]) / W) ** 2 * p).sum(-1) / safe
    trms = np.where(P > 0, np.sqrt(np.maximum(var, 0.0)), 0.0)
    return P, np.where(P > 0, tbar, 0.0), trms


def smape(x, y):
    """Eq. smape: |x - y| / (x + y), with SMAPE(0, 0) = 0."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    s = x + y
    return np.where(s > 0, np.abs(x - y) / np.where(s > 0, s, 1.0), 0.0)


def smape_dy(x, y):
    """d SMAPE(x, y) / dy = 2 x sign(y - x) / (x + y)^2 (0 where x + y = 0)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    s = x + y
    return np.where(s > 0, 2.0 * x * np.sign(y - x) / np.where(s > 0, s, 1.0) ** 2, 0.0)


def alpha_hat(P_meas, P_pred):
    """Eq. alpha_hat: argmin_alpha mean_b (alpha P_b - P^_b)^2 = sum P P^ / sum P^2."""
    P_meas = np.asarray(P_meas, np.float64)
    P_pred = np.asarray(P_pred, np.float64)
    return float((P_meas * P_pred).sum() / (P_meas ** 2).sum())


def alpha_ema(alpha_prev, a_hat, decay, first):
    """Eq. scaling_param: alpha_i = delta alpha_{i-1} + (1 - delta) alpha^_i with alpha_0 = alpha^_1."""
    prev = a_hat if first else alpha_prev
    return decay * prev + (1.0 - decay) * a_hat


def loss(H, P_meas, tau_meas, delta_f, alpha):
    """Mean over the batch of Eq. loss, SMAPE(tau_RMS, tau^_RMS) + SMAPE(alpha P, P^),
    and its gradient g_H = dL/dRe H + j dL/dIm H.

    Chain: p_l = |h_l|^2, dP/dp_l = 1, d tau_RMS / d p_l = ((l - tau_bar)^2 / W^2
    - tau_RMS^2) / (2 tau_RMS P); g_h = 2 (dL/dp_l) h_l; g_H = cir_adjoint(g_h)."""
    H = np.asarray(H, np.complex128)
    R, N = H.shape
    W = N * float(delta_f)
    h = cir(H)
    p = np.abs(h) ** 2
    ell = np.arange(N) - N // 2
    P, tbar, trms = stats(H, delta_f)
    Pm = alpha * np.asarray(P_meas, np.float64)
    tm = np.asarray(tau_meas, np.float64)
    L_b = smape(tm, trms) + smape(Pm, P)
    L = float(L_b.mean())
    dL_dtrms = smape_dy(tm, trms) / R
    dL_dP = smape_dy(Pm, P) / R
    ok = (P > 0) & (trms > 0)
    safe_P = np.where(P > 0, P, 1.0)
    safe_t = np.where(trms > 0, trms, 1.0)
    dtrms_dp = (((ell[None, :] - tbar[:, None]) / W) ** 2 - trms[:, None] ** 2) / (2.0 * safe_t[:, None] * safe_P[:, None])
    dL_dp = dL_dP[:, None] + np.where(ok[:, None], dL_dtrms[:, None] * dtrms_dp, 0.0)
    g_h = 2.0 * dL_dp * h
    return L, cir_adjoint(g_h)


def ale_db(P_meas, P_pred):
    """Absolute logarithmic error of the channel gain |P_dB - P^_dB| (Sec. IV-C)."""
    return np.abs(10.0 * np.log10(np.asarray(P_meas, np.float64)) - 10.0 * np.log10(np.asarray(P_pred, np.float64)))


def rae(tau_meas, tau_pred):
    """Relative absolute error of the delay spread |tau - tau^| / tau (Sec. IV-C)."""
    tm = np.asarray(tau_meas, np.float64)
    return np.abs(tm - np.asarray(tau_pred, np.float64)) / tm
