"""Pins of the FP64 oracle against closed forms, special cases and brute force.

Each test fixes one part of the oracle with something other than the oracle's own
code: textbook closed forms, geometric facts of the image method, brute force, or
invariants the mathematics guarantees.  Paper: arXiv 2311.18558.
"""
import cmath
import math

import numpy as np
import pytest

import oracle
import scenegen
from scenegen import Scene

C0 = 299792458.0
EPS0 = 8.8541878128e-12


def plane_scene(eps_r=5.24, sigma=0.0462, pec=False, half=50.0):
    """A single ground plane z = 0 (two triangles, normal +z)."""
    v = np.array([[-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return Scene(name="plane", verts=v, tris=t, tri_material=np.zeros(2, np.int32),
                 eps_r=np.array([eps_r], np.float32), sigma=np.array([sigma], np.float32),
                 is_pec=np.array([1 if pec else 0], np.uint8), tx=np.array([0.0, 0.0, 10.0]),
                 rx=np.array([[20.0, 5.0, 2.0]]), n_rays=20000, max_depth=1, freq_hz=3.5e9,
                 f_center_hz=3.5e9, delta_f_hz=1e6, n_sub=16)


# ----------------------------------------------------------------------------- permittivity / Fresnel

def test_permittivity_concrete():
    # eta = eps_r - j sigma / (eps0 * 2 pi f)  (Sec. II-D, ITU-R P.2040 Eq. 9b)
    eta = oracle.permittivity(5.24, 0.0462, 3.5e9)
    assert abs(eta.real - 5.24) < 1e-15
    assert abs(eta.imag - (-0.237271367)) < 1e-8


@pytest.mark.parametrize("eps_r,sigma,ref", [
    (5.24, 0.0462, complex(-0.392191, 0.009573)),
    (6.31, 0.0036, complex(-0.430520, 0.000597)),
    (15.0, 0.035, complex(-0.589589, 0.001954)),
])
def test_fresnel_normal_incidence(eps_r, sigma, ref):
    # At normal incidence both coefficients reduce to the textbook
    # r = (1 - sqrt(eta)) / (1 + sqrt(eta)) and r_par = -r_perp.
    eta = complex(eps_r, -sigma / (EPS0 * 2 * math.pi * 3.5e9))
    closed = (1 - cmath.sqrt(eta)) / (1 + cmath.sqrt(eta))
    rp, rl, _, _ = oracle.fresnel(eps_r, sigma, 3.5e9, 1.0)
    assert abs(rp - closed) < 1e-14
    assert abs(rl + closed) < 1e-14
    assert abs(rp - ref) < 1e-6


def test_fresnel_brewster():
    # Lossless dielectric: r_par vanishes at the Brewster angle tan(theta) = sqrt(eps_r).
    for eps_r in (2.0, 5.24, 15.0):
        th = math.atan(math.sqrt(eps_r))
        _, rl, _, _ = oracle.fresnel(eps_r, 0.0, 3.5e9, math.cos(th))
        assert abs(rl) < 1e-12
        _, rl2, _, _ = oracle.fresnel(eps_r, 0.0, 3.5e9, math.cos(th + 0.05))
        assert abs(rl2) > 1e-3


def test_fresnel_grazing():
    # Both coefficients tend to -1 at grazing incidence.
    rp, rl, _, _ = oracle.fresnel(5.24, 0.0462, 3.5e9, 1e-9)
    assert abs(rp + 1) < 1e-8 and abs(rl + 1) < 1e-8


def test_fresnel_passive():
    # Invariant I2: a lossy dielectric never reflects more than it receives.
    rng = np.random.default_rng(0)
    for _ in range(500):
        eps_r = rng.uniform(1.0, 20.0)
        sigma = 10 ** rng.uniform(-4, 1)
        c = rng.uniform(0, 1)
        rp, rl, _, _ = oracle.fresnel(eps_r, sigma, 1e9 * rng.uniform(0.5, 30), c)
        assert abs(rp) <= 1 + 1e-12 and abs(rl) <= 1 + 1e-12


def test_fresnel_derivative_fd():
    # d r / d eta against a central difference along the real eps_r axis and along
    # sigma (eta is holomorphic: d/dsigma = -j/(eps0 omega) d/deta).
    f = 2.0e9
    w = 2 * math.pi * f
    for eps_r, sigma, c in [(5.24, 0.0462, 0.7), (3.0, 0.5, 0.2), (12.0, 0.001, 0.95)]:
        rp, rl, dp, dl = oracle.fresnel(eps_r, sigma, f, c)
        h = 1e-6
        rp1, rl1, _, _ = oracle.fresnel(eps_r + h, sigma, f, c)
        rp0, rl0, _, _ = oracle.fresnel(eps_r - h, sigma, f, c)
        assert abs((rp1 - rp0) / (2 * h) - dp) < 1e-7 * max(1, abs(dp))
        assert abs((rl1 - rl0) / (2 * h) - dl) < 1e-7 * max(1, abs(dl))
        hs = 1e-6 * sigma
        rp1, rl1, _, _ = oracle.fresnel(eps_r, sigma + hs, f, c)
        rp0, rl0, _, _ = oracle.fresnel(eps_r, sigma - hs, f, c)
        assert abs((rp1 - rp0) / (2 * hs) - dp * (-1j / (EPS0 * w))) < 1e-6 * abs(dp / (EPS0 * w))


# ----------------------------------------------------------------------------- LoS, image method

def test_los_friis():
    # Free space: |a| = lambda / (4 pi d), a real positive for co-polarised vertical
    # antennas, tau = d / c  (Eq. cfr_cont with F_0 of Eq. init).
    sc = plane_scene()
    sc.tx = np.array([0.0, 0.0, 10.0])
    sc.rx = np.array([[1.0, 0.0, 10.0], [3.0, 4.0, 12.0], [-7.0, 2.0, 20.0]])
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=1000, depth=1)
    a = o.fields(tr)
    los = tr["depth"] == 0
    assert los.sum() == 3
    lam = C0 / 3.5e9
    for i in np.where(los)[0]:
        d = np.linalg.norm(tr["pts"][i, 1] - tr["pts"][i, 0])
        assert abs(abs(a[i]) - lam / (4 * math.pi * d)) < 1e-15
        assert abs(a[i].imag) < 1e-15 and a[i].real > 0
        assert abs(tr["tau"][i] - d / C0) < 1e-22
    assert abs(lam / (4 * math.pi * 1.0) - 6.81621e-3) < 1e-8


def _ref_specular_coefficient(tx, rx, s, n, r_perp, r_par, lam):
    """Independent 3-vector form of one specular reflection (no 2x2 basis changes).

    E_r = r_perp (E.e_perp) e_perp + r_par (E.e_par_in) e_par_out, with the
    incident field along theta_hat of the departure direction and the result
    projected on theta_hat of the arrival direction, times lambda/(4 pi L).
    """
    def th(k):
        t = math.acos(max(-1.0, min(1.0, k[2])))
        p = math.atan2(k[1], k[0])
        return np.array([math.cos(t) * math.cos(p), math.cos(t) * math.sin(p), -math.sin(t)])
    k1 = (s - tx) / np.linalg.norm(s - tx)
    k2 = (rx - s) / np.linalg.norm(rx - s)
    E = th(k1)
    nn = n if np.dot(k1, n) < 0 else -n
    ep = np.cross(k1, nn)
    ep /= np.linalg.norm(ep)
    Er = r_perp * np.dot(E, ep) * ep + r_par * np.dot(E, np.cross(ep, k1)) * np.cross(ep, k2)
    L = np.linalg.norm(s - tx) + np.linalg.norm(rx - s)
    return lam / (4 * math.pi * L) * np.dot(Er, th(-k2)), L


@pytest.mark.parametrize("pec", [False, True])
def test_single_plane_image_method(pec):
    # Two-ray geometry: the reflection point lies at fraction h1/(h1+h2) of the
    # horizontal distance, L = sqrt(rho^2 + (h1+h2)^2); the coefficient equals the
    # independent 3-vector computation.  For PEC, r_perp = -1 and r_par = +1, i.e.
    # E_r = 2 (E.n) n - E (tangential field flipped, normal field kept).
    sc = plane_scene(pec=pec)
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=20000, depth=1)
    a = o.fields(tr)
    assert tr["depth"].tolist() == [0, 1]
    tx, rx = sc.tx, sc.rx[0]
    h1, h2 = tx[2], rx[2]
    rho = np.linalg.norm(rx[:2] - tx[:2])
    s = tr["pts"][1, 1]
    frac = np.linalg.norm(s[:2] - tx[:2]) / rho
    assert abs(frac - h1 / (h1 + h2)) < 1e-14
    assert abs(s[2]) < 1e-14
    L = math.sqrt(rho ** 2 + (h1 + h2) ** 2)
    assert abs(tr["tau"][1] * C0 - L) < 1e-12
    lam = C0 / 3.5e9
    if pec:
        rp, rl = -1.0, 1.0
    else:
        c = abs(np.dot((s - tx) / np.linalg.norm(s - tx), [0, 0, 1.0]))
        rp, rl, _, _ = oracle.fresnel(float(np.float32(5.24)), float(np.float32(0.0462)), 3.5e9, c)
    ref, Lref = _ref_specular_coefficient(tx, rx, s, np.array([0, 0, 1.0]), rp, rl, lam)
    assert abs(a[1] - ref) < 1e-12 * abs(ref)
    if pec:
        # direct PEC mirror rule: E_r = 2(E.n)n - E with E = theta_hat(k1)
        k1 = (s - tx) / np.linalg.norm(s - tx)
        k2 = (rx - s) / np.linalg.norm(rx - s)
        E = np.array([k1[2] * k1[0], k1[2] * k1[1], -(k1[0] ** 2 + k1[1] ** 2)]) / math.hypot(k1[0], k1[1])
        n = np.array([0, 0, 1.0])
        Er = 2 * np.dot(E, n) * n - E
        thr = np.array([-k2[2] * -k2[0], -k2[2] * -k2[1], -(k2[0] ** 2 + k2[1] ** 2)]) / math.hypot(k2[0], k2[1])
        ref2 = lam / (4 * math.pi * L) * np.dot(Er, thr)
        assert abs(a[1] - ref2) < 1e-12 * abs(ref2)
        # vertical dipole over PEC ground: in-phase image (same sign as LoS)
        assert a[1].real > 0 and a[0].real > 0


def test_shoebox_images():
    # Rectangular room: the paths of order <= 2 are exactly the image sources of
    # order <= 2 (Allen & Berkley 1979), i.e. 1 + 6 + 18 per receiver, except images
    # whose line to the receiver crosses two walls at the same point (an edge of
    # the room): such a path degenerates and is rejected.  Compared by path length.
    sc = scenegen.tiny_box()
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=200000, depth=2)
    Lr = np.array([10.0, 8.0, 3.0])
    tx = sc.tx

    def mirror(p, ax, side):
        q = p.copy()
        q[ax] = -q[ax] if side == 0 else 2 * Lr[ax] - q[ax]
        return q

    walls = [(ax, sd) for ax in range(3) for sd in range(2)]
    for r in range(sc.n_rx):
        rx = sc.rx[r]
        expect = [np.linalg.norm(rx - tx)]
        images = {}
        for w1 in walls:
            i1 = mirror(tx, *w1)
            images[(w1,)] = i1
            for w2 in walls:
                if w2 == w1:
                    continue
                images[(w1, w2)] = mirror(i1, *w2)
        seen = set()
        for seqw, img in images.items():
            key = tuple(np.round(img, 9))
            if key in seen:
                continue
            # Unfolded straight line rx -> img: its crossings of the lattice planes
            # x = m Lx, y = m Ly, z = m Lz are the reflections of the path.
            us = []
            for ax in range(3):
                lo, hi = sorted((rx[ax], img[ax]))
                m0, m1 = math.floor(lo / Lr[ax]) + 1, math.ceil(hi / Lr[ax]) - 1
                for m in range(m0, m1 + 1):
                    us.append((m * Lr[ax] - rx[ax]) / (img[ax] - rx[ax]))
            if len(us) != len(seqw):
                continue   # this image belongs to a lower order
            seen.add(key)
            us = np.sort(us)
            if len(us) == 2 and abs(us[1] - us[0]) < 1e-12:
                continue   # passes through a room edge: degenerate
            expect.append(np.linalg.norm(rx - img))
        got = np.sort(tr["tau"][tr["rx"] == r] * C0)
        assert len(got) == len(expect), (r, len(got), len(expect))
        np.testing.assert_allclose(got, np.sort(expect), rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------- BVH, SBR, dedup

def test_bvh_equals_brute_force():
    sc = scenegen.street_canyon()
    o = oracle.OracleScene(sc)
    rng = np.random.default_rng(1)
    n = 20000
    orig = np.column_stack([rng.uniform(-260, 260, n), rng.uniform(-260, 260, n), rng.uniform(0.5, 45, n)])
    d = rng.normal(size=(n, 3))
    # rays aimed exactly at vertices and at edge midpoints
    V = sc.verts.astype(np.float64)
    T = sc.tris
    tv = V[T[:2000, 0]]
    te = 0.5 * (V[T[2000 % len(T):, 0]] + V[T[2000 % len(T):, 1]]) if len(T) > 2000 else 0.5 * (V[T[:, 0]] + V[T[:, 1]])
    tgt = np.concatenate([tv, te])
    o2 = np.column_stack([rng.uniform(-260, 260, len(tgt)), rng.uniform(-260, 260, len(tgt)), rng.uniform(0.5, 45, len(tgt))])
    orig = np.concatenate([orig, o2])
    d = np.concatenate([d, tgt - o2])
    t1, h1 = o.closest_hit(orig, d, use_bvh=True)
    t0, h0 = o.closest_hit(orig, d, use_bvh=False)
    assert np.array_equal(t1, t0)
    assert np.array_equal(h1, h0)
    assert (t1 >= 0).mean() > 0.3


def test_sbr_bvh_equals_brute_force_and_dedup():
    sc = scenegen.street_canyon()
    o = oracle.OracleScene(sc)
    s1 = o.sbr_rays(3000, 3, use_bvh=True)
    s0 = o.sbr_rays(3000, 3, use_bvh=False)
    assert np.array_equal(s1, s0)
    cands = o.candidates(3000, 3)
    ref = {()}
    for row in s1:
        pre = []
        for t in row:
            if t < 0:
                break
            pre.append(int(t))
            ref.add(tuple(pre))
    got = [tuple(int(x) for x in c if x >= 0) for c in cands]
    assert len(got) == len(set(got))
    assert set(got) == ref
    assert got == sorted(got, key=lambda s: (len(s), s))


def test_fibonacci_lattice_properties():
    # Fibonacci lattice: equally spaced z, consecutive azimuths differ by the golden
    # angle 2 pi (1 - g) (mod 2 pi), unit vectors up to FP32 rounding.
    n = 4097
    d = oracle.fibonacci(n).astype(np.float64)
    z = d[:, 2]
    np.testing.assert_allclose(np.diff(z), -2.0 / n, atol=2e-7)
    assert np.all(np.abs(np.linalg.norm(d, axis=1) - 1) < 3e-7)
    phi = np.arctan2(d[:, 1], d[:, 0])
    g = (math.sqrt(5) - 1) / 2
    dphi = np.mod(np.diff(phi) - 2 * math.pi * g, 2 * math.pi)
    dphi = np.minimum(dphi, 2 * math.pi - dphi)
    inner = slice(10, n - 11)          # azimuth is ill-conditioned at the poles
    assert np.all(dphi[inner] < 1e-4)
    assert abs(d.mean(axis=0)).max() < 1e-3
    # against the closed form of the lattice in FP64 (the 32-bit Weyl fraction
    # drifts from i*g by i * 1.2e-10 turns, and the FP32 sine/cosine by ~1e-7)
    i = np.arange(n)
    zz = 1 - (2 * i + 1) / n
    ph = 2 * np.pi * np.mod(i * g, 1.0)
    ref = np.stack([np.sqrt(1 - zz * zz) * np.cos(ph), np.sqrt(1 - zz * zz) * np.sin(ph), zz], 1)
    assert np.abs(d - ref).max() < 3e-6


# ----------------------------------------------------------------------------- fields invariants

def test_normal_incidence_basis_invariance():
    # Invariant I3: at normal incidence the perpendicular direction is arbitrary;
    # the coefficient must not depend on it.  Tx and Rx share y and z, so the
    # reflections off the walls x = 0 and x = 10 are at normal incidence.
    sc = scenegen.tiny_box()
    sc.rx = np.array([[6.0, 2.0, 2.0]])
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=20000, depth=2)
    a0 = o.fields(tr, ni_mode=0)
    a1 = o.fields(tr, ni_mode=1)
    assert len(a0) > 10
    np.testing.assert_allclose(a1, a0, rtol=1e-12, atol=1e-18)


def test_lossless_pec_room_energy_bound():
    # With PEC walls every reflection keeps |E| (|r| = 1), so each path's |a| is at
    # most lambda / (4 pi L): basis changes are orthogonal.
    sc = scenegen.tiny_box()
    sc.is_pec = np.array([1], np.uint8)
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=20000, depth=2)
    a = o.fields(tr)
    lam = C0 / sc.freq_hz
    bound = lam / (4 * math.pi * tr["tau"] * C0)
    assert np.all(np.abs(a) <= bound * (1 + 1e-12))


# ----------------------------------------------------------------------------- CFR

def test_cfr_single_path():
    # One path: |H[n]| = |a| for every n and the phase decreases linearly with
    # slope 2 pi df tau per subcarrier (Sec. II-A).
    a = np.array([0.3 - 0.4j])
    tau = np.array([1.234567e-7])
    H = oracle.cfr(a, tau, np.array([0, 1]), 2.0e9, 1.0e5, 64)[0]
    np.testing.assert_allclose(np.abs(H), 0.5, rtol=1e-14)
    ratio = H[1:] / H[:-1]
    np.testing.assert_allclose(ratio, np.exp(-2j * math.pi * 1.0e5 * tau[0]), rtol=1e-12)
    n0 = 32   # column of n = 0, i.e. the centre frequency
    np.testing.assert_allclose(H[n0], a[0] * np.exp(-2j * math.pi * 2.0e9 * tau[0]), rtol=1e-12)


def test_cfr_grad_is_adjoint():
    # <g_H, J a'> = <J^H g_H, a'> for the linear map a -> H (real inner product).
    a, tau, offs = scenegen.random_cfr_inputs(5, 4, 6)
    rng = np.random.default_rng(0)
    da = rng.normal(size=a.shape) + 1j * rng.normal(size=a.shape)
    gH = rng.normal(size=(4, 32)) + 1j * rng.normal(size=(4, 32))
    JH = oracle.cfr(da, tau, offs, 1e9, 1e6, 32)
    ga = oracle.cfr_grad(tau, offs, 1e9, 1e6, 32, gH)
    lhs = np.sum((np.conj(gH) * JH).real)
    rhs = np.sum((np.conj(ga) * da).real)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_power_mse_grad_fd():
    rng = np.random.default_rng(3)
    H = rng.normal(size=(3, 8)) + 1j * rng.normal(size=(3, 8))
    T = np.abs(rng.normal(size=(3, 8))) ** 2
    w = oracle.power_weights(T)
    L, gH = oracle.power_mse(H, T, w)
    h = 1e-7
    for (r, n) in [(0, 0), (1, 5), (2, 7)]:
        for unit in (1, 1j):
            Hp, Hm = H.copy(), H.copy()
            Hp[r, n] += h * unit
            Hm[r, n] -= h * unit
            fd = (oracle.power_mse(Hp, T, w)[0] - oracle.power_mse(Hm, T, w)[0]) / (2 * h)
            an = gH[r, n].real if unit == 1 else gH[r, n].imag
            assert abs(fd - an) < 1e-6 * max(1, abs(an))


# ----------------------------------------------------------------------------- gradients end to end

def _loss_pipeline(o, tr, eps, sig, gains, T, w, fc, df, N):
    a = o.fields(tr, eps_r=eps, sigma=sig, gain_tx=gains[0], gain_rx=gains[1])
    H = oracle.cfr(a, tr["tau"], tr["rx_offsets"], fc, df, N)
    return oracle.power_mse(H, T, w), a, H


def test_fields_grad_fd_and_holomorphy():
    # Analytic FP64 adjoint of the whole step (fields -> CFR -> power MSE) against
    # central finite differences; invariant I1: for single-material chains
    # dL/dsigma = Re(conj(g) (-j/(eps0 omega)) da/deta) follows from the same da/deta.
    sc = scenegen.indoor_diff()
    sc = sc.subset_rx(np.arange(6))
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=20000, depth=2)
    fc, df, N = sc.f_center_hz, sc.delta_f_hz * 16, 64
    eps = sc.eps_r.astype(np.float64)
    sig = sc.sigma.astype(np.float64)
    gains = (1.3, 0.8)
    # target: the same pipeline at perturbed materials
    (L0, _), a, H = _loss_pipeline(o, tr, eps, sig, gains, np.zeros((sc.n_rx, N)), np.ones(sc.n_rx), fc, df, N)
    Tt = np.abs(oracle.cfr(o.fields(tr, eps_r=eps * 1.1, sigma=sig * 0.7), tr["tau"], tr["rx_offsets"], fc, df, N)) ** 2
    w = oracle.power_weights(Tt)
    (L, gH), a, H = _loss_pipeline(o, tr, eps, sig, gains, Tt, w, fc, df, N)
    ga = oracle.cfr_grad(tr["tau"], tr["rx_offsets"], fc, df, N, gH)
    ge, gs, gg = o.fields_grad(tr, ga, eps_r=eps, sigma=sig, gain_tx=gains[0], gain_rx=gains[1])
    # eps/sigma are passed to the oracle as float32: perturb by exactly representable steps
    for m in range(len(eps)):
        for arr, g in ((eps, ge), (sig, gs)):
            h = 2.0 ** (math.floor(math.log2(abs(arr[m]))) - 10)
            ap, am = arr.copy(), arr.copy()
            ap[m] += h
            am[m] -= h
            if arr is eps:
                Lp = _loss_pipeline(o, tr, ap, sig, gains, Tt, w, fc, df, N)[0][0]
                Lm = _loss_pipeline(o, tr, am, sig, gains, Tt, w, fc, df, N)[0][0]
            else:
                Lp = _loss_pipeline(o, tr, eps, ap, gains, Tt, w, fc, df, N)[0][0]
                Lm = _loss_pipeline(o, tr, eps, am, gains, Tt, w, fc, df, N)[0][0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[m]) <= 2e-5 * max(abs(g).max(), 1e-30), (m, fd, g[m])
    for k in range(2):
        h = 1e-6
        gp, gm = list(gains), list(gains)
        gp[k] += h
        gm[k] -= h
        fd = (_loss_pipeline(o, tr, eps, sig, gp, Tt, w, fc, df, N)[0][0]
              - _loss_pipeline(o, tr, eps, sig, gm, Tt, w, fc, df, N)[0][0]) / (2 * h)
        assert abs(fd - gg[k]) <= 1e-6 * abs(gg[k])
    # holomorphy (I1): a unit cotangent g = 1 gives Re(da/deta); g = j gives Im(da/deta)
    one = np.zeros(len(a), complex)
    one[:] = 1.0
    e1, s1, _ = o.fields_grad(tr, one, eps_r=eps, sigma=sig)
    ej, sj, _ = o.fields_grad(tr, 1j * one, eps_r=eps, sigma=sig)
    deta = e1 + 1j * ej                       # sum of da/deta (conj(g) * x, real part)
    dsig = s1 + 1j * sj
    k = -1j / (EPS0 * 2 * math.pi * sc.freq_hz)
    np.testing.assert_allclose(dsig, k * deta, rtol=1e-10, atol=1e-30)
