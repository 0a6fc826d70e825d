"""FP64 oracle of first-order diffraction (arXiv 2311.18558, Sec. II-D Eq. diffraction,
Sec. II-F).  TEST INFRASTRUCTURE: only the tests, the smoke check and the
benchmark's CPU baseline use it; the library never calls it.

The geometry (wedges of the mesh, candidate wedges from the first hits of the
launch rays, Keller's point of diffraction, exterior and visibility checks) is in
``rt_oracle.cpp`` (``orc_wedges``, ``orc_diffraction_paths``); its readings are
stated there.  This module computes the field of each path in plain PyTorch CPU
float64, so that the gradients with respect to the materials of both faces are
the exact derivatives of this forward model (autograd).

The paper gives the form of the field transformation, F(E) = Q E A^d e^{-j k d},
and names its ingredients: the uniform theory of diffraction of Kouyoumjian and
Pathak (Proc. IEEE 62(11), 1974) with Luebbers' heuristic extension to wedges of
finite conductivity (IEEE Trans. AP-32(1), 1984), in an edge-fixed frame.  It
does not print Q.  Written here from those publications:

* Edge-fixed frame.  e is the edge direction, t0 the unit vector from the edge
  into the incidence face ("face 0"), n0 = e x t0 its outward normal; the
  exterior angle of the wedge is n pi.  phi' and phi are the angles about e,
  measured from face 0 into the exterior, of the directions from the point of
  diffraction Q to the transmitter and to the receiver; beta_0 is the angle
  between e and the incident direction s' (the diffracted direction s has the
  same angle, Keller's cone).
* Bases: phi'_hat = e x s' / |e x s'|, beta'_hat = s' x phi'_hat for the incident
  field, phi_hat = e x s / |e x s|, beta_hat = s x phi_hat for the diffracted
  one.  Q = diag(D_s, D_h) from (beta', phi') to (beta, phi).
* D_{s,h} = -e^{-j pi/4} / (2 n sqrt(2 pi k) sin beta_0) *
        [ T(pi + (phi - phi')) + T(pi - (phi - phi'))
          + R_0^{s,h} T(pi - (phi + phi')) + R_n^{s,h} T(pi + (phi + phi')) ],
  T(y) = cot(eps / (2n)) F(2 k L sin^2(eps / 2)),
  eps = y - 2 pi n N with N the integer nearest to y / (2 pi n), which is the
  Kouyoumjian-Pathak term cot((pi +- beta) / 2n) F(k L a^+-(beta)) with
  a^+-(beta) = 2 cos^2((2 n pi N^+- - beta) / 2).  At |eps| < 1e-12 the term takes
  its limit n sqrt(2 pi k L) sgn(eps) e^{j pi/4} (sgn(0) = +1).
* Transition function F(X) = 2 j sqrt(X) e^{jX} int_{sqrt X}^inf e^{-j t^2} dt,
  with the Fresnel integral from scipy.special.fresnel.
* Distance parameter and spreading for a spherical incident wave (a point
  transmitter): L = s s' sin^2 beta_0 / (s + s'), A^d = sqrt(s' / (s (s + s'))).
* Luebbers: R_0 is the reflection coefficient of face 0 at the incidence angle
  with cos theta = |sin beta_0 sin phi'|, R_n that of the other face with
  cos theta = |sin beta_0 sin(n pi - phi)|; the soft coefficient (field along
  the edge at normal incidence) takes r_perp, the hard one r_par (Eq. fresnel-1,
  fresnel-2); a perfectly conducting face gives r_perp = -1, r_par = +1, which is
  the Kouyoumjian-Pathak wedge.  Readings: the oblique-incidence angle
  sin beta_0 sin(.) (Luebbers states normal incidence), and the incidence face is
  the face on the transmitter's side (phi' <= n pi / 2), since the heuristic is
  not symmetric in the two faces.
* Path coefficient: a = lambda / (4 pi) sqrt(g_R) theta_hat(-s) . E_d with
  E_d = [D_s (E_i . beta') beta + D_h (E_i . phi') phi] A^d / s',
  E_i = sqrt(g_T) theta_hat(s') (Eq. polarization_model, zeta = 0); the
  propagation phase goes to the CFR through tau = (s' + s) / c.
"""
from __future__ import annotations

import math

import numpy as np
import torch
from scipy.special import fresnel as _fresnel

from . import _c, _load, _p, OracleScene  # noqa: F401

C0 = 299792458.0
EPS0 = 8.8541878128e-12


# ----------------------------------------------------------------------------- geometry (rt_oracle.cpp)

def wedges(o: OracleScene):
    """Wedges of the mesh in canonical form: faces (W, 2) with f0 < fn, start vertex,
    edge direction e, t0, n0 (W, 3 each), length (W,), n (W,)."""
    lib = _load()
    import ctypes
    lib.orc_wedges.restype = ctypes.c_void_p
    lib.orc_wedges.argtypes = [ctypes.c_void_p]
    lib.orc_wedges_count.restype = ctypes.c_int64
    lib.orc_wedges_count.argtypes = [ctypes.c_void_p]
    lib.orc_wedges_get.restype = None
    lib.orc_wedges_get.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_wedges_free.restype = None
    lib.orc_wedges_free.argtypes = [ctypes.c_void_p]
    h = lib.orc_wedges(o.h)
    W = lib.orc_wedges_count(h)
    faces = np.empty((W, 2), np.int32)
    geo = np.empty((W, 14), np.float64)
    lib.orc_wedges_get(h, _p(faces), _p(geo))
    lib.orc_wedges_free(h)
    return dict(faces=faces, start=geo[:, 0:3], e=geo[:, 3:6], t0=geo[:, 6:9], n0=geo[:, 9:12],
                length=geo[:, 12], n=geo[:, 13])


def paths(o: OracleScene, n_rays=None, tx=None, rx=None):
    """Diffraction paths of every candidate wedge and receiver (see rt_oracle.cpp).

    Returns rx (P,), wedge (P,), faces (P, 2) = (incidence face, other face),
    pts (P, 3, 3) = Tx, Q, Rx, tau (P,), rx_offsets (R+1,), and the wedge table."""
    import ctypes
    lib = _load()
    sc = o.scene
    n_rays = sc.n_rays if n_rays is None else n_rays
    tx = _c(sc.tx if tx is None else tx, np.float64)
    rx = _c(sc.rx if rx is None else rx, np.float64).reshape(-1, 3)
    lib.orc_diffraction_paths.restype = ctypes.c_void_p
    lib.orc_diffraction_paths.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_void_p]
    lib.orc_wedges.restype = ctypes.c_void_p
    lib.orc_wedges.argtypes = [ctypes.c_void_p]
    lib.orc_wedges_free.argtypes = [ctypes.c_void_p]
    ch = lib.orc_candidates(o.h, _p(tx), int(n_rays), 1)
    wt = lib.orc_wedges(o.h)
    ph = lib.orc_diffraction_paths(o.h, wt, _p(tx), _p(rx), rx.shape[0], ch)
    lib.orc_candidates_free(ch)
    lib.orc_wedges_free(wt)
    P = lib.orc_paths_count(ph)
    out = dict(rx=np.empty(P, np.int32), depth=np.empty(P, np.int32), faces=np.empty((P, 2), np.int32),
               pts=np.empty((P, 4, 3), np.float64), tau=np.empty(P, np.float64), wedge=np.empty(P, np.int32))
    lib.orc_paths_get(ph, _p(out["rx"]), _p(out["depth"]), _p(out["faces"]), _p(out["pts"]), _p(out["tau"]))
    lib.orc_paths_rays(ph, _p(out["wedge"]))
    lib.orc_paths_free(ph)
    out["pts"] = out["pts"][:, :3]
    del out["depth"]
    offs = np.zeros(rx.shape[0] + 1, np.int64)
    np.add.at(offs, out["rx"] + 1, 1)
    out["rx_offsets"] = np.cumsum(offs)
    out["wedges"] = wedges(o)
    return out


# ----------------------------------------------------------------------------- UTD coefficients

def transition(X):
    """F(X) = 2 j sqrt(X) e^{jX} int_{sqrt X}^inf e^{-j t^2} dt (Kouyoumjian-Pathak), X >= 0."""
    X = np.asarray(X, np.float64)
    u = np.sqrt(X)
    S, C = _fresnel(u * math.sqrt(2.0 / math.pi))
    tail = math.sqrt(math.pi / 2.0) * ((0.5 - C) - 1j * (0.5 - S))
    return 2j * u * np.exp(1j * X) * tail


def term(y, n, k, L):
    """T(y) = cot(eps / 2n) F(2 k L sin^2(eps / 2)), eps = y reduced to [-n pi, n pi]."""
    y = np.asarray(y, np.float64)
    n = np.asarray(n, np.float64)
    eps = y - 2.0 * math.pi * n * np.round(y / (2.0 * math.pi * n))
    small = np.abs(eps) < 1e-12
    e_safe = np.where(small, 1.0, eps)
    X = 2.0 * k * L * np.sin(e_safe / 2.0) ** 2
    val = transition(X) / np.tan(e_safe / (2.0 * n))
    lim = n * np.sqrt(2.0 * math.pi * k * L) * np.where(eps < 0, -1.0, 1.0) * np.exp(1j * math.pi / 4)
    return np.where(small, lim, val)


def utd_terms(n, phi, php, k, L):
    """The four terms (T1, T2, T3, T4) multiplying 1, 1, R_0, R_n."""
    d, s = phi - php, phi + php
    return (term(math.pi + d, n, k, L), term(math.pi - d, n, k, L),
            term(math.pi - s, n, k, L), term(math.pi + s, n, k, L))


def coefficients(n, phi, php, sinb, k, L, R0s, R0h, Rns, Rnh):
    """(D_s, D_h) of Kouyoumjian-Pathak with Luebbers' face coefficients; works on
    numpy arrays or torch tensors for the R's (autograd through them)."""
    T1, T2, T3, T4 = (torch.as_tensor(t, dtype=torch.complex128) for t in utd_terms(n, phi, php, k, L))
    n = torch.as_tensor(n, dtype=torch.float64)
    sinb = torch.as_tensor(sinb, dtype=torch.float64)
    pre = -complex(math.cos(-math.pi / 4), math.sin(-math.pi / 4)) / (2.0 * n * math.sqrt(2.0 * math.pi * k) * sinb)
    Ds = pre * (T1 + T2 + R0s * T3 + Rns * T4)
    Dh = pre * (T1 + T2 + R0h * T3 + Rnh * T4)
    return Ds, Dh


def _fresnel_rc(eta, cos_i):
    s = torch.sqrt(eta - (1.0 - cos_i * cos_i))
    return (cos_i - s) / (cos_i + s), (eta * cos_i - s) / (eta * cos_i + s)


def _theta_hat(k):
    th = np.arccos(np.clip(k[:, 2], -1.0, 1.0))
    ph = np.where((k[:, 0] == 0) & (k[:, 1] == 0), 0.0, np.arctan2(k[:, 1], k[:, 0]))
    return np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def geometry(dp):
    """Per-path quantities that do not depend on materials or frequency:
    n, phi, phi' (in the incidence face's frame), sin beta_0, s', s, the four
    projections of the incident and diffracted bases, and the face materials' slots."""
    W = dp["wedges"]
    w = dp["wedge"]
    T, Q, R = dp["pts"][:, 0], dp["pts"][:, 1], dp["pts"][:, 2]
    e, t0, n0, n = W["e"][w], W["t0"][w], W["n0"][w], W["n"][w]

    def ang(d):
        p = d - np.sum(d * e, 1, keepdims=True) * e
        a = np.arctan2(np.sum(p * n0, 1), np.sum(p * t0, 1))
        return np.where(a < 0, a + 2 * math.pi, a)
    php, phi = ang(T - Q), ang(R - Q)
    swap = dp["faces"][:, 0] != W["faces"][w, 0]
    php = np.where(swap, n * math.pi - php, php)
    phi = np.where(swap, n * math.pi - phi, phi)
    sp = np.linalg.norm(Q - T, axis=1)
    sd = np.linalg.norm(R - Q, axis=1)
    s_in = (Q - T) / sp[:, None]
    s_out = (R - Q) / sd[:, None]
    sinb = np.linalg.norm(np.cross(e, s_in), axis=1)
    ph_in = _unit(np.cross(e, s_in))
    be_in = np.cross(s_in, ph_in)
    ph_out = _unit(np.cross(e, s_out))
    be_out = np.cross(s_out, ph_out)
    Ei = _theta_hat(s_in)
    Er = _theta_hat(-s_out)
    return dict(n=n, phi=phi, php=php, sinb=sinb, sp=sp, sd=sd,
                in_b=np.sum(Ei * be_in, 1), in_p=np.sum(Ei * ph_in, 1),
                out_b=np.sum(Er * be_out, 1), out_p=np.sum(Er * ph_out, 1))


def fields(sc, dp, eps_r, sigma, freq=None, gain_tx=1.0, gain_rx=1.0):
    """Coefficients a_i (complex128 torch tensor) of the diffraction paths `dp`.

    eps_r, sigma: per material (torch float64 tensors may require grad), indexed by
    the faces' material ids, or per triangle when the scene is per-triangle."""
    freq = sc.freq_hz if freq is None else freq
    g = geometry(dp)
    k = 2.0 * math.pi * freq / C0
    lam = C0 / freq
    L = g["sd"] * g["sp"] * g["sinb"] ** 2 / (g["sd"] + g["sp"])
    eps_r = torch.as_tensor(eps_r, dtype=torch.float64)
    sigma = torch.as_tensor(sigma, dtype=torch.float64)
    f0, fn = dp["faces"][:, 0], dp["faces"][:, 1]
    m0 = f0 if sc.per_triangle else sc.tri_material[f0]
    mn = fn if sc.per_triangle else sc.tri_material[fn]
    # perfect conductors are flagged per material id of the triangle, in both modes
    pec = np.asarray(sc.is_pec).astype(bool)
    pec0, pecn = pec[sc.tri_material[f0]], pec[sc.tri_material[fn]]
    w = 2.0 * math.pi * freq
    eta0 = eps_r[m0] - 1j * sigma[m0] / (EPS0 * w)
    etan = eps_r[mn] - 1j * sigma[mn] / (EPS0 * w)
    c0 = torch.as_tensor(np.abs(g["sinb"] * np.sin(g["php"])))
    cn = torch.as_tensor(np.abs(g["sinb"] * np.sin(g["n"] * math.pi - g["phi"])))
    R0s, R0h = _fresnel_rc(eta0, c0)
    Rns, Rnh = _fresnel_rc(etan, cn)
    one = torch.ones_like(R0s)
    p0, pn = torch.as_tensor(pec0), torch.as_tensor(pecn)
    R0s, R0h = torch.where(p0, -one, R0s), torch.where(p0, one, R0h)
    Rns, Rnh = torch.where(pn, -one, Rns), torch.where(pn, one, Rnh)
    Ds, Dh = coefficients(g["n"], g["phi"], g["php"], g["sinb"], k, L, R0s, R0h, Rns, Rnh)
    spread = np.sqrt(g["sp"] / (g["sd"] * (g["sd"] + g["sp"]))) / g["sp"]
    t = lambda x: torch.as_tensor(x, dtype=torch.float64)   # noqa: E731
    a = (lam / (4.0 * math.pi)) * math.sqrt(gain_tx * gain_rx) * t(spread) * (
        Ds * t(g["in_b"]) * t(g["out_b"]) + Dh * t(g["in_p"]) * t(g["out_p"]))
    return a
