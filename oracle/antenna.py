"""FP64 oracle of the trainable antenna pattern (arXiv 2311.18558, Sec. III-B):
a directional gain made of M spherical Gaussians (von Mises-Fisher lobes),

    G(r) = 4 pi eta_rad sum_i w_i / a_i exp(lambda_i mu_i . r),
    a_i = (2 pi / lambda_i) (exp(lambda_i) - exp(-lambda_i)),

applied to a path through the vertical polarization model (Eq. polarization_model,
zeta = 0): C = [sqrt(G), 0], so a path coefficient scales by
sqrt(G_T(k_1) G_R(-k_{q+1})) with k_1 the departure direction and -k_{q+1} the
arrival direction seen from the receiver.

Reading: each lobe w_i / a_i exp(lambda_i mu_i . r) integrates to w_i over the
sphere, so without the factor 4 pi the gain would integrate to eta_rad, whereas
Eq. atenna_normalization asks for 4 pi eta_rad; the factor 4 pi makes the two
agree (and a nearly flat pattern gives G = eta_rad, the isotropic unit gain).

Test infrastructure only (tests, the smoke check and the benchmark's CPU
baseline); the library never calls it.
"""
import numpy as np


def directions(pts, depth):
    """Departure k_1 and arrival -k_{q+1} unit vectors of paths given by their
    points (P, D+2, 3) = Tx, s_1..s_q, Rx and depths."""
    pts = np.asarray(pts, np.float64)
    P = pts.shape[0]
    aod = np.zeros((P, 3))
    aoa = np.zeros((P, 3))
    for i in range(P):
        q = int(depth[i])
        d1 = pts[i, 1] - pts[i, 0]
        aod[i] = d1 / np.linalg.norm(d1)
        dl = pts[i, q] - pts[i, q + 1]          # from the receiver towards the last point
        aoa[i] = dl / np.linalg.norm(dl)
    return aod, aoa


def lobe_scale(lam):
    """1 / a(lambda) = lambda / (2 pi (e^lambda - e^-lambda))."""
    lam = np.asarray(lam, np.float64)
    return lam / (2.0 * np.pi * (np.exp(lam) - np.exp(-lam)))


def gain(r, w, lam, mu, eta=1.0):
    """G(r) for unit directions r (P, 3); w, lam (M,), mu (M, 3) unit."""
    r = np.asarray(r, np.float64)
    c = r @ np.asarray(mu, np.float64).T                        # (P, M)
    lam = np.asarray(lam, np.float64)
    return 4.0 * np.pi * eta * (np.exp(lam[None, :] * c) * (np.asarray(w) * lobe_scale(lam))[None, :]).sum(1)


def gain_grad(r, w, lam, mu, eta, g_G):
    """Given dL/dG per direction, returns dL/dw (M,), dL/dlambda (M,), dL/dmu (M, 3):
    dG/dw_i = 4 pi eta e_i / a_i,
    dG/dlambda_i = 4 pi eta w_i e_i / a_i (mu_i . r - coth(lambda_i) + 1 / lambda_i),
    dG/dmu_i = 4 pi eta w_i e_i / a_i lambda_i r,  with e_i = exp(lambda_i mu_i . r)."""
    r = np.asarray(r, np.float64)
    w = np.asarray(w, np.float64)
    lam = np.asarray(lam, np.float64)
    mu = np.asarray(mu, np.float64)
    g_G = np.asarray(g_G, np.float64)
    c = r @ mu.T
    base = 4.0 * np.pi * eta * np.exp(lam[None, :] * c) * lobe_scale(lam)[None, :]     # (P, M)
    dw = (g_G[:, None] * base).sum(0)
    dlam = (g_G[:, None] * base * w[None, :] * (c - 1.0 / np.tanh(lam)[None, :] + 1.0 / lam[None, :])).sum(0)
    dmu = ((g_G[:, None] * base * w[None, :] * lam[None, :])[:, :, None] * r[:, None, :]).sum(0)
    return dw, dlam, dmu


def apply(a, aod, aoa, tx, rx):
    """a_i sqrt(G_T(aod_i) G_R(aoa_i)); tx, rx = (w, lam, mu, eta) or None (unit gain).
    Returns (a_out, G_T, G_R)."""
    gt = gain(aod, *tx) if tx is not None else np.ones(len(a))
    gr = gain(aoa, *rx) if rx is not None else np.ones(len(a))
    return np.asarray(a, np.complex128) * np.sqrt(gt * gr), gt, gr


def apply_grad(a_out, gt, gr, g_out):
    """Adjoint of apply(): dL/da_in = sqrt(G_T G_R) g_out, dL/dG_T = Re(conj(g) a_out) / (2 G_T),
    dL/dG_R = Re(conj(g) a_out) / (2 G_R)."""
    g_out = np.asarray(g_out, np.complex128)
    a_out = np.asarray(a_out, np.complex128)
    s = np.real(np.conj(g_out) * a_out)
    return np.sqrt(gt * gr) * g_out, s / (2.0 * gt), s / (2.0 * gr)
