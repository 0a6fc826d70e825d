"""Pins of the FP64 diffuse-reflection oracle (oracle/diffuse.py and the
next-event estimation in oracle/rt_oracle.cpp) to quadratures, closed forms,
brute force and numerical differentiation (Sec. II-D diffuse reflection,
Sec. II-F, Sec. III-C)."""
import math

import numpy as np
import pytest
import torch

import oracle
import scenegen
from oracle import diffuse as od


def _hemisphere(n_theta=200, n_phi=400):
    """Gauss-Legendre in cos(theta) on (0, 1) x uniform phi: directions about +z and weights."""
    x, wx = np.polynomial.legendre.leggauss(n_theta)
    c = 0.5 * (x + 1.0)
    wc = 0.5 * wx
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    C, PH = np.meshgrid(c, phi, indexing="ij")
    S = np.sqrt(1 - C ** 2)
    k = np.stack([S * np.cos(PH), S * np.sin(PH), C], -1).reshape(-1, 3)
    w = (wc[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).reshape(-1)
    return k, w


def test_lambert_term_integrates_to_one():
    k, w = _hemisphere()
    f = od.pattern([1.0, 0.0, 0.0], 1.0, 1.0, k[:, 2], 0.0, 0.0, 0.7)
    np.testing.assert_allclose(float((f.numpy() * w).sum()), 1.0, rtol=1e-10)


def test_lobe_normaliser_against_quadrature():
    # a(lambda, cos beta) is within 1.2 % of the exact hemispherical integral of
    # exp(lambda mu . k) for axes on or above the surface, and exact where the
    # smooth step reaches its end points (axis on the normal, axis in the plane)
    k, w = _hemisphere(300, 600)
    worst = 0.0
    for lam in (0.5, 2.0, 5.0, 15.0, 40.0):
        for cb in (0.0, 0.2, 0.5, 0.8, 1.0):
            mu = np.array([math.sqrt(1 - cb * cb), 0.0, cb])
            exact = float((np.exp(lam * (k @ mu)) * w).sum())
            approx = float(od.lobe_norm(lam, cb))
            err = abs(approx / exact - 1.0)
            worst = max(worst, err)
            if cb in (0.0, 1.0):
                assert err < 1e-9, (lam, cb, err)
    assert worst < 0.012, worst


def test_pattern_integrates_to_about_one():
    # f_s with both lobes integrates to ~1 over the hemisphere (the lobe axes are
    # -k_i and k_r, both at cos beta = cos theta_i above the surface)
    k, wq = _hemisphere(300, 600)
    rng = np.random.default_rng(0)
    for _ in range(6):
        th = rng.uniform(0.05, 1.4)
        ki = np.array([math.sin(th), 0.0, -math.cos(th)])     # propagating down onto n = +z
        kr = ki * np.array([1, 1, -1])
        wts = rng.dirichlet([1, 1, 1])
        lam2, lam3 = rng.uniform(1, 30, 2)
        f = od.pattern(wts, lam2, lam3, k[:, 2], -(k @ ki), k @ kr, math.cos(th)).numpy()
        assert abs(float((f * wq).sum()) - 1.0) < 0.012


def test_flat_lobe_limit():
    g = od.pattern([0.0, 1.0, 0.0], 1e-7, 1.0, 0.3, 0.5, 0.1, 0.6)
    np.testing.assert_allclose(float(g), 1.0 / (2 * np.pi), rtol=1e-6)


def test_closed_box_every_hit_sees_every_receiver():
    # in a closed convex room every ray hits D times and every receiver inside
    # sees every hit point from the incidence side: P = R N D, and the triangle
    # sequences are those of the plain SBR
    sc = scenegen.tiny_box()
    o = oracle.OracleScene(sc)
    N, D = 500, 2
    d = o.diffuse_paths(N, D)
    assert len(d["rx"]) == sc.n_rx * N * D
    seqs = o.sbr_rays(N, D)
    for i in range(0, len(d["rx"]), 97):
        j = d["depth"][i]
        np.testing.assert_array_equal(d["seq"][i, :j], seqs[d["ray"][i], :j])
        L = np.linalg.norm(np.diff(d["pts"][i, : j + 2], axis=0), axis=1).sum()
        np.testing.assert_allclose(d["tau"][i], L / oracle.C0, rtol=1e-14)
    assert np.all(np.diff(d["rx"]) >= 0)


def _mt_hits(o, d, tri_v):
    """Moller-Trumbore ray parameters of a segment o + t d against every triangle (nan = miss)."""
    v0, v1, v2 = tri_v[:, 0], tri_v[:, 1], tri_v[:, 2]
    e1, e2 = v1 - v0, v2 - v0
    p = np.cross(d, e2)
    det = (e1 * p).sum(1)
    inv = 1.0 / np.where(det == 0, 1.0, det)
    s = o - v0
    u = (s * p).sum(1) * inv
    q = np.cross(s, e1)
    v = (d * q).sum(1) * inv
    t = (e2 * q).sum(1) * inv
    return t, u, v, det


def test_visibility_and_sides_against_brute_force():
    # every (ray, hit, receiver) triple: the oracle keeps it iff the receiver is on the
    # incidence side and no other triangle crosses the segment (brute force, Moller-Trumbore);
    # triples within 1e-7 of a decision boundary are not compared
    sc = scenegen.indoor_diff().subset_rx(np.arange(0, 1024, 128))
    o = oracle.OracleScene(sc)
    N, D = 400, 2
    d = o.diffuse_paths(N, D)
    kept = set(zip(d["rx"].tolist(), d["ray"].tolist(), d["depth"].tolist()))
    tri_v = sc.verts[sc.tris].astype(np.float64)
    nrm = np.cross(tri_v[:, 1] - tri_v[:, 0], tri_v[:, 2] - tri_v[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    # the ray hit points from the diffuse paths of the first receiver are enough only if it sees
    # them all, so trace the hit points independently with the oracle's closest hit
    dirs = oracle.fibonacci(N).astype(np.float64)
    eps = 1e-6 * o.diag
    n_cmp = n_amb = 0
    for i in range(N):
        org, dr, prev, prev_pt = sc.tx.astype(np.float64), dirs[i], None, sc.tx.astype(np.float64)
        for j in range(1, D + 1):
            tri, th = o.closest_hit(org, dr, skip=None if prev is None else [prev])
            t = int(tri[0])
            if t < 0:
                break
            p = org + th[0] * dr
            for r in range(sc.n_rx):
                rxp = sc.rx[r]
                s_in, s_rx = np.dot(prev_pt - p, nrm[t]), np.dot(rxp - p, nrm[t])
                seg = rxp - p
                ln = np.linalg.norm(seg)
                tt, u, v, det = _mt_hits(p, seg, tri_v)
                tt[t] = np.nan
                lo, hi = eps / ln, 1 - eps / ln
                inside = (u >= 0) & (v >= 0) & (u + v <= 1) & (det != 0)
                block = inside & (tt > lo) & (tt < hi)
                margin = np.minimum.reduce([np.abs(u), np.abs(v), np.abs(1 - u - v)])
                amb = (np.abs(s_rx) < 1e-7 * o.diag or
                       np.any(((margin < 1e-7) & (tt > lo - 1e-7) & (tt < hi + 1e-7)) |
                              (inside & ((np.abs(tt - lo) < 1e-7) | (np.abs(tt - hi) < 1e-7)))))
                if amb:
                    n_amb += 1
                    continue
                expect = (s_in * s_rx > 0) and ln > eps and not np.any(block)
                assert ((r, i, j) in kept) == expect, (r, i, j)
                n_cmp += 1
            dr = dr - 2 * np.dot(dr, nrm[t]) * nrm[t]
            org, prev, prev_pt = p, t, p
    assert n_cmp > 5000 and n_amb < 0.01 * n_cmp


def test_ray_density_matches_the_area_element():
    # reading of dA: a ray sampling s_j stands for cos(theta_i) dA = 4 pi l^2 / N, so the
    # sum of |a|^2 over the traced diffuse paths equals the integral over the plane of
    # |a(p)|^2 N cos(theta_i) / (4 pi l(p)^2) dA, computed by quadrature on the plane
    sc = scenegen.ground_plane(half=200.0)
    o = oracle.OracleScene(sc)
    N = 400_000
    scat = np.array([[0.6, 0.3, 0.5, 0.2, 0.3, 4.0, 8.0, 0.0]])
    d = o.diffuse_paths(N, 1)
    a = od.fields(sc, d, sc.eps_r, sc.sigma, scat, sc.freq_hz, N)
    lhs = float((a.abs() ** 2).sum())

    def panels(foot):
        e = [foot + s * 0.25 * 1.6 ** k for s in (-1, 1) for k in range(20)]
        e = [x for x in e if -200 < x < 200] + [-200.0, 200.0]
        return np.unique(np.array(e))

    def gl(edges, n=16):
        x, w = np.polynomial.legendre.leggauss(n)
        a_, b_ = edges[:-1, None], edges[1:, None]
        return ((a_ + b_) / 2 + (b_ - a_) / 2 * x).ravel(), ((b_ - a_) / 2 * w).ravel()

    ex = np.unique(np.concatenate([panels(sc.tx[0]), panels(sc.rx[0, 0])]))
    ey = np.unique(np.concatenate([panels(sc.tx[1]), panels(sc.rx[0, 1])]))
    xs, wxs = gl(ex)
    ys, wys = gl(ey)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    W = (wxs[:, None] * wys[None, :]).ravel()
    npt = X.size
    pts = np.zeros((npt, 3, 3))
    pts[:, 0] = sc.tx
    pts[:, 1, 0], pts[:, 1, 1] = X.ravel(), Y.ravel()
    pts[:, 2] = sc.rx[0]
    fab = dict(depth=np.ones(npt, np.int32), seq=np.zeros((npt, 1), np.int32), pts=pts)
    af = od.fields(sc, fab, sc.eps_r, sc.sigma, scat, sc.freq_hz, N).abs().numpy() ** 2
    ell = np.linalg.norm(pts[:, 1] - pts[:, 0], axis=1)
    cos_i = sc.tx[2] / ell
    rhs = float((af * N * cos_i / (4 * np.pi * ell ** 2) * W).sum())
    np.testing.assert_allclose(lhs, rhs, rtol=5e-3)


def test_gradients_against_central_differences():
    sc = scenegen.indoor_diff().subset_rx(np.arange(0, 1024, 256))
    o = oracle.OracleScene(sc)
    N = 300
    d = o.diffuse_paths(N, 2)
    rng = np.random.default_rng(3)
    g = torch.as_tensor(rng.normal(size=len(d["rx"])) + 1j * rng.normal(size=len(d["rx"])))
    scat0 = scenegen.random_scattering(1, 8).astype(np.float64)[:, :7]
    eps0, sig0 = sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64)

    def L(e, s, c):
        a = od.fields(sc, d, e, s, c, sc.freq_hz, N)
        return (g.conj() * a).real.sum()
    e = torch.tensor(eps0, requires_grad=True)
    s = torch.tensor(sig0, requires_grad=True)
    c = torch.tensor(scat0, requires_grad=True)
    L(e, s, c).backward()
    used = np.unique(np.asarray(sc.tri_material)[d["seq"][d["seq"] >= 0]])
    for m in used[:4]:
        for arr, grad, nm in ((eps0, e.grad, "eps"), (sig0, s.grad, "sigma")):
            h = 1e-6 * arr[m]
            ap, am = arr.copy(), arr.copy()
            ap[m] += h
            am[m] -= h
            args_p = (ap, sig0, scat0) if nm == "eps" else (eps0, ap, scat0)
            args_m = (am, sig0, scat0) if nm == "eps" else (eps0, am, scat0)
            fd = (float(L(*args_p)) - float(L(*args_m))) / (2 * h)
            np.testing.assert_allclose(float(grad[m]), fd, rtol=1e-5, atol=1e-9 * abs(fd) + 1e-30)
        for col in range(7):
            h = 1e-6 * max(abs(scat0[m, col]), 1e-3)
            cp, cm = scat0.copy(), scat0.copy()
            cp[m, col] += h
            cm[m, col] -= h
            fd = (float(L(eps0, sig0, cp)) - float(L(eps0, sig0, cm))) / (2 * h)
            scale = float(c.grad[m].abs().max())
            np.testing.assert_allclose(float(c.grad[m, col]), fd, rtol=1e-5, atol=1e-7 * scale)


def test_specular_reduction():
    sc = scenegen.tiny_box()
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=2000, depth=2)
    a = o.fields(tr)
    scat = np.zeros((1, 7))
    np.testing.assert_allclose(od.specular_reduction(sc, tr, scat, a).numpy(), a, rtol=0, atol=0)
    scat[0, 0] = 0.6
    out = od.specular_reduction(sc, tr, scat, a).numpy()
    np.testing.assert_allclose(np.abs(out) ** 2, np.abs(a) ** 2 * 0.64 ** tr["depth"], rtol=1e-13)


def test_random_phases_rotate_each_polarisation():
    # K_x = 0 keeps only the first polarisation component: the phases turn a by
    # exp(j chi_1) and leave |a|; K_x = 1 keeps only the second: exp(j chi_2)
    sc = scenegen.tiny_box()
    o = oracle.OracleScene(sc)
    d = o.diffuse_paths(200, 2)
    rng = np.random.default_rng(9)
    chi = rng.uniform(0, 2 * np.pi, (len(d["rx"]), 2))
    for kx, col in ((0.0, 0), (1.0, 1)):
        scat = np.array([[0.5, kx, 0.4, 0.3, 0.3, 3.0, 6.0]])
        a0 = od.fields(sc, d, sc.eps_r, sc.sigma, scat, sc.freq_hz, 200).numpy()
        a1 = od.fields(sc, d, sc.eps_r, sc.sigma, scat, sc.freq_hz, 200, chi=chi).numpy()
        np.testing.assert_allclose(a1, a0 * np.exp(1j * chi[:, col]), rtol=1e-12, atol=1e-25)
