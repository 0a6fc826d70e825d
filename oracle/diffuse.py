"""FP64 oracle of diffuse reflection with the trainable scattering pattern
(arXiv 2311.18558, Sec. II-D "Diffuse reflection", Sec. III-C, Sec. II-F).
TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use it; the library never calls it.

Written in plain PyTorch CPU float64 so that the gradients with respect to every
material and pattern parameter are the exact derivatives of this forward model
(autograd); the pins in tests/test_oracle_diffuse.py check them against central
differences and check the forward against quadratures and closed forms.

Model of one diffuse path Tx -> s_1 .. s_{j-1} (specular) -> s_j (diffuse) -> Rx:

* Transmit field C_T = [sqrt(g_T), 0] (Eq. polarization_model, zeta = 0) in the
  theta/phi basis of the departure direction k_1.
* Specular bounces b < j: basis change D_b into the incidence basis
  (e_perp = k_b x n / |k_b x n|, e_par = e_perp x k_b, n facing the wave), then
  diag(R r_perp, R r_par) (Eq. specular_reflection) with R = sqrt(1 - S^2) of
  the bounce's material (Sec. II-D).
* Diffuse bounce j (Eq. scattered_field): v = D_j E is the incident field at s_j
  in the incidence basis, |E_in| = |v| / l_j with l_j = d_1 + .. + d_j (the wave
  stays spherical about the image source for planar facets), and
  Gamma |E_in| = |diag(r_perp, r_par) v| / l_j.
  Reading of dA (not specified in the paper): each of N launch rays carries the
  solid angle 4 pi / N, so the surface element it samples at s_j is
  dA = 4 pi l_j^2 / (N cos theta_i) and cos(theta_i) dA = 4 pi l_j^2 / N.  Hence
  |E_s| = sqrt(4 pi / N) S sqrt(f_s) |diag(r_perp, r_par) v|.
  Reading of the polarisation vector: [sqrt(1 - K_x) e^{j chi_1}, sqrt(K_x) e^{j chi_2}]
  is expressed in the basis of the scattered direction k_s and the normal:
  e_perp,s = k_s x n / |k_s x n|, e_par,s = e_perp,s x k_s.  The random phases
  chi are inputs (per path); without them chi_1 = chi_2 = 0, as the paper's
  synthetic data.
* Propagation to Rx: 1 / d_{j+1}, basis change D_{j+1} into the theta/phi basis
  of the arrival direction -k_s, projection on C_R = [sqrt(g_R), 0], times
  lambda / (4 pi).  The propagation phase is left to the CFR through
  tau = (l_j + d_{j+1}) / c, as for specular paths.

Scattering pattern (Eq. trainable_scattering_pattern), per material:
  f_s = w_1 / pi (k_s . n) + w_2 g(lambda_2, -k_i . k_s) + w_3 g(lambda_3, k_r . k_s),
  g(lambda, c) = exp(lambda c) / a(lambda, cos theta_i).
  Readings: the backscattering lobe's axis is -k_i (towards the source; with k_i
  the propagation direction of Sec. II-D, the literal k_i axis would point into
  the surface); the normaliser a(lambda, cos beta) is the hemispherical integral
  of exp(lambda mu . k_s) over the upper hemisphere, with cos beta = mu . n the
  angle between the lobe axis and the normal (for both lobes cos beta = cos theta_i;
  the printed cos beta = k_s . mu would make the normaliser depend on the
  evaluation direction).  It is approximated as the paper does, by a smooth step
  s(t, cos beta) between the exact integrals for the axis on the normal,
  U = 2 pi / lambda (e^lambda - 1), and opposite it, L = 2 pi / lambda (1 - e^-lambda):
  a = s U + (1 - s) L with the printed s and t(lambda) (the printed closed form of
  a changes sign and vanishes at cos beta = 0, so it cannot be used literally).
"""
from __future__ import annotations

import math

import numpy as np
import torch

C0 = 299792458.0
EPS0 = 8.8541878128e-12
DT = torch.float64


def _t(x):
    return x if torch.is_tensor(x) else torch.as_tensor(np.asarray(x), dtype=DT)


# ----------------------------------------------------------------------------- pattern

def lobe_t(lam):
    """t(lambda) of the hemispherical normaliser (Sec. III-C)."""
    lam = _t(lam)
    return torch.sqrt(lam) * (1.6988 * lam ** 2 + 10.8438 * lam) / (lam ** 2 + 6.2201 * lam + 10.2415)


def lobe_norm(lam, cos_beta):
    """a(lambda, cos beta): approximate integral of exp(lambda mu . k) over the
    hemisphere k . n > 0, mu . n = cos beta (Sec. III-C, reading above)."""
    lam, cb = _t(lam), _t(cos_beta)
    t = lobe_t(lam)
    s = torch.expm1(t * (1.0 + cb)) / (torch.expm1(t) * (torch.exp(t * cb) + 1.0))
    U = 2.0 * math.pi / lam * torch.expm1(lam)
    L = 2.0 * math.pi / lam * (-torch.expm1(-lam))
    return s * U + (1.0 - s) * L


def pattern(w, lam2, lam3, cos_n, cos_back, cos_spec, cos_i):
    """f_s of Eq. trainable_scattering_pattern for directions given by their
    cosines: cos_n = k_s . n, cos_back = -k_i . k_s, cos_spec = k_r . k_s,
    cos_i = cos(theta_i); w = (w_1, w_2, w_3) (last axis)."""
    w = _t(w)
    g2 = torch.exp(lam2 * _t(cos_back)) / lobe_norm(lam2, cos_i)
    g3 = torch.exp(lam3 * _t(cos_spec)) / lobe_norm(lam3, cos_i)
    return w[..., 0] / math.pi * _t(cos_n) + w[..., 1] * g2 + w[..., 2] * g3


# ----------------------------------------------------------------------------- geometry helpers

def _unit(v):
    return v / torch.linalg.norm(v, dim=-1, keepdim=True)


def _sph_basis(k):
    """theta_hat, phi_hat of direction k (phi = 0 for a vertical direction)."""
    theta = torch.acos(torch.clamp(k[..., 2], -1.0, 1.0))
    vertical = (k[..., 0] == 0) & (k[..., 1] == 0)
    phi = torch.where(vertical, torch.zeros_like(theta), torch.atan2(k[..., 1], k[..., 0]))
    th = torch.stack([torch.cos(theta) * torch.cos(phi), torch.cos(theta) * torch.sin(phi), -torch.sin(theta)], -1)
    ph = torch.stack([-torch.sin(phi), torch.cos(phi), torch.zeros_like(phi)], -1)
    return th, ph


def _dot(a, b):
    return (a * b).sum(-1)


def _basis_change(p_in, q_in, p_out, q_out):
    """2x2 real matrix [[p_in.p_out, p_in.q_out], [q_in.p_out, q_in.q_out]]."""
    return torch.stack([torch.stack([_dot(p_in, p_out), _dot(p_in, q_out)], -1),
                        torch.stack([_dot(q_in, p_out), _dot(q_in, q_out)], -1)], -2)


def _perp(k, n, fallback):
    """unit(k x n), or, where k is (numerically) along n, `fallback` made
    orthogonal to k (the normal-incidence reading of the specular chain)."""
    c = torch.cross(k, n, dim=-1)
    nc = torch.linalg.norm(c, dim=-1, keepdim=True)
    fb = fallback - _dot(fallback, k)[..., None] * k
    fb = _unit(fb)
    return torch.where(nc > 1e-12, c / torch.where(nc > 0, nc, torch.ones_like(nc)), fb)


def _fresnel(eta, cos_i):
    sin2 = 1.0 - cos_i ** 2
    s = torch.sqrt(eta - sin2)
    return (cos_i - s) / (cos_i + s), (eta * cos_i - s) / (eta * cos_i + s)


def _tri_normals(scene):
    v = torch.as_tensor(np.asarray(scene.verts, np.float64))
    t = torch.as_tensor(np.asarray(scene.tris, np.int64))
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return _unit(torch.cross(b - a, c - a, dim=-1))


# ----------------------------------------------------------------------------- fields

def fields(scene, paths, eps_r, sigma, scat, freq, n_rays, gain_tx=1.0, gain_rx=1.0, chi=None):
    """Coefficients a_i (complex128 tensor) of the diffuse paths from
    OracleScene.diffuse_paths.  eps_r, sigma: per material; scat: per material
    [S, K_x, w_1, w_2, w_3, lambda_2, lambda_3] (M x 7 or more columns); chi:
    optional per-path phases (P x 2, radians) of Eq. scattered_field.  Any of them
    may be tensors with requires_grad."""
    eps_r, sigma, scat = _t(eps_r), _t(sigma), _t(scat)
    lam_w = C0 / freq
    omega = 2.0 * math.pi * freq
    nrm = _tri_normals(scene)
    tri_mat = torch.as_tensor(np.asarray(scene.tri_material, np.int64))
    pec = torch.as_tensor(np.asarray(scene.is_pec, bool))
    P = int(paths["depth"].shape[0])
    a = torch.zeros(P, dtype=torch.complex128)
    dep = np.asarray(paths["depth"])
    for j in range(1, int(paths["seq"].shape[1]) + 1):
        idx = np.nonzero(dep == j)[0]
        if idx.size == 0:
            continue
        pts = torch.as_tensor(np.asarray(paths["pts"])[idx, : j + 2], dtype=DT)
        seq = torch.as_tensor(np.asarray(paths["seq"])[idx, :j], dtype=torch.int64)
        k = _unit(pts[:, 1:] - pts[:, :-1])                    # k_1 .. k_{j+1}
        seg = torch.linalg.norm(pts[:, 1:] - pts[:, :-1], dim=-1)
        out_p, out_q = _sph_basis(k[:, 0])
        E = torch.stack([torch.full((idx.size,), math.sqrt(gain_tx), dtype=DT),
                         torch.zeros(idx.size, dtype=DT)], -1).to(torch.complex128)
        for b in range(1, j + 1):
            kb = k[:, b - 1]
            n = nrm[seq[:, b - 1]]
            n = torch.where((_dot(kb, n) > 0)[:, None], -n, n)      # facing the incident wave
            cos_i = -_dot(kb, n)
            e_perp = _perp(kb, n, out_p)
            in_q = torch.cross(e_perp, kb, dim=-1)
            Dm = _basis_change(e_perp, in_q, out_p, out_q).to(torch.complex128)
            v = (Dm @ E[..., None])[..., 0]
            m = tri_mat[seq[:, b - 1]]
            eta = torch.complex(eps_r[m].to(DT), -sigma[m].to(DT) / (EPS0 * omega))
            rp, rl = _fresnel(eta, cos_i.to(torch.complex128))
            is_pec = pec[m]
            rp = torch.where(is_pec, torch.full_like(rp, -1.0), rp)
            rl = torch.where(is_pec, torch.full_like(rl, 1.0), rl)
            u = torch.stack([rp * v[:, 0], rl * v[:, 1]], -1)
            S = scat[m, 0].to(DT)
            if b < j:
                E = torch.sqrt(1.0 - S ** 2)[:, None] * u
                out_p = e_perp
                out_q = torch.cross(e_perp, k[:, b], dim=-1)
                continue
            # diffuse bounce (Eq. scattered_field) with the pattern of Eq. trainable_scattering_pattern
            ks = k[:, j]
            kr = kb - 2.0 * _dot(kb, n)[:, None] * n
            f = pattern(scat[m, 2:5].to(DT), scat[m, 5].to(DT), scat[m, 6].to(DT),
                        _dot(ks, n), -_dot(kb, ks), _dot(kr, ks), cos_i)
            nu = torch.sqrt((u.real ** 2 + u.imag ** 2).sum(-1))
            amp = math.sqrt(4.0 * math.pi / n_rays) * S * torch.sqrt(f) * nu / seg[:, j]
            Kx = scat[m, 1].to(DT)
            pol = torch.stack([torch.sqrt(1.0 - Kx), torch.sqrt(Kx)], -1).to(torch.complex128)
            if chi is not None:
                ch = torch.as_tensor(np.asarray(chi, np.float64)[idx])
                pol = pol * torch.exp(1j * ch)
            sp = _perp(ks, n, e_perp)
            sq = torch.cross(sp, ks, dim=-1)
            th, ph = _sph_basis(-ks)
            Dl = _basis_change(th, ph, sp, sq)
            er = Dl[:, 0, 0].to(torch.complex128) * pol[:, 0] + Dl[:, 0, 1].to(torch.complex128) * pol[:, 1]
            a_j = lam_w / (4.0 * math.pi) * math.sqrt(gain_rx) * amp * er
            a = a.index_put((torch.as_tensor(idx),), a_j.to(torch.complex128))
    return a


def specular_reduction(scene, paths, scat, a):
    """a_i prod_b R_b, R_b = sqrt(1 - S_b^2) of the material of each specular
    bounce (Sec. II-D, Eq. specular_reflection): the specular paths' share of the
    reflected energy when part of it is scattered diffusely."""
    scat = _t(scat)
    tri_mat = torch.as_tensor(np.asarray(scene.tri_material, np.int64))
    seq = torch.as_tensor(np.asarray(paths["seq"], np.int64))
    dep = torch.as_tensor(np.asarray(paths["depth"], np.int64))
    fac = torch.ones(seq.shape[0], dtype=DT)
    for b in range(seq.shape[1]):
        on = dep > b
        m = tri_mat[torch.clamp(seq[:, b], min=0)]
        R = torch.sqrt(1.0 - scat[m, 0].to(DT) ** 2)
        fac = fac * torch.where(on, R, torch.ones_like(R))
    a = a if torch.is_tensor(a) else torch.as_tensor(np.asarray(a, np.complex128))
    return a.to(torch.complex128) * fac


def tau(paths):
    return np.asarray(paths["tau"], np.float64)
