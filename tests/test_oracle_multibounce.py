"""Pins of the oracle's multi-bounce path coefficient (paths of two and three bounces).

The oracle carries a path's field through 2x2 basis changes D_j and reflection
matrices diag(r_perp, r_par) (Eq. rel1, basis_transform, specular_reflection).
These tests fix that chain for q >= 2 with two computations that share none of
its structure:

* image theory for a vertically polarised source in a scene of perfectly
  conducting horizontal and vertical planes: every path's coefficient is
  s * lambda / (4 pi L) * sqrt(g_T g_R), with s = -1 per bounce on a vertical
  plane and +1 per bounce on a horizontal one (the image of a vertical dipole is
  in phase under a horizontal PEC plane and in antiphase behind a vertical one);
* a three-vector field update per bounce, E <- r_perp (E.e_perp) e_perp +
  r_par (E.e_par_in) e_par_out, started along theta_hat of the departure
  direction and projected on theta_hat of the arrival direction, times
  lambda / (4 pi L) (Sec. II-C/D with the McNamara reflection basis, reading R6).
  In the shoebox the directions and incidence angles come from the image
  sources in closed form (Allen & Berkley 1979), not from the oracle's points.

A final test checks that the comparison is sharp: a reference with one sign
convention changed disagrees with the oracle on most paths.  Paper: arXiv 2311.18558.
"""
import cmath
import math

import numpy as np
import pytest

import oracle
import scenegen

C0 = 299792458.0
EPS0 = 8.8541878128e-12


# ----------------------------------------------------------------------------- helpers

def theta_hat(k):
    """theta_hat of direction k (phi = 0 for a vertical direction)."""
    t = math.acos(max(-1.0, min(1.0, k[2])))
    p = math.atan2(k[1], k[0]) if (k[0] != 0.0 or k[1] != 0.0) else 0.0
    return np.array([math.cos(t) * math.cos(p), math.cos(t) * math.sin(p), -math.sin(t)])


def fresnel_pair(eta, cos_i):
    """Textbook Fresnel reflection coefficients (TE, TM) for relative permittivity eta."""
    s = cmath.sqrt(eta - (1.0 - cos_i * cos_i))
    return (cos_i - s) / (cos_i + s), (eta * cos_i - s) / (eta * cos_i + s)


def eta_of(eps_r, sigma, freq):
    return complex(eps_r, -sigma / (EPS0 * 2.0 * math.pi * freq))


def field_three_vector(ks, normals, coeffs, lam, L, gain_tx=1.0, gain_rx=1.0,
                       flip_par_out=False, swap_te_tm=False):
    """Coefficient of one path from its segment directions k_1..k_{q+1}, the unit
    normals of its q reflecting planes and the (r_perp, r_par) of each bounce."""
    E = math.sqrt(gain_tx) * theta_hat(ks[0]).astype(complex)
    for j, n in enumerate(normals):
        ki, kr = ks[j], ks[j + 1]
        nn = n if np.dot(ki, n) < 0 else -n
        ep = np.cross(ki, nn)
        ep /= np.linalg.norm(ep)
        e_in = np.cross(ep, ki)
        e_out = np.cross(ep, kr)
        if flip_par_out:
            e_out = -e_out
        rp, rl = coeffs[j]
        if swap_te_tm:
            rp, rl = rl, rp
        E = rp * np.dot(E, ep) * ep + rl * np.dot(E, e_in) * e_out
    return lam / (4.0 * math.pi * L) * math.sqrt(gain_rx) * np.dot(E, theta_hat(-ks[-1]))


def path_geometry(pts, q):
    seg = [pts[j + 1] - pts[j] for j in range(q + 1)]
    d = [np.linalg.norm(v) for v in seg]
    return [v / dv for v, dv in zip(seg, d)], float(sum(d))


def tri_normals(sc):
    V = sc.verts.astype(np.float64)
    T = sc.tris
    n = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def wall_of(sc):
    """(axis, coordinate) of the plane of each triangle of an axis-aligned mesh."""
    V = sc.verts.astype(np.float64)
    out = []
    for t in sc.tris:
        p = V[t]
        ax = [a for a in range(3) if p[0, a] == p[1, a] == p[2, a]]
        assert len(ax) == 1
        out.append((ax[0], float(p[0, ax[0]])))
    return out


def tol(L, lam):
    """Relative tolerance: 1e-12, plus the FP64 rounding of the carrier phases.

    The oracle multiplies a unit phasor per segment and removes exp(-j 2 pi f tau)
    at the end; each phase argument of magnitude 2 pi L / lambda carries an absolute
    rounding of a few units of 2^-53 times itself (about 3e-12 rad at 500 m, 3.5 GHz).
    """
    return 1e-12 + 1e-15 * 2.0 * math.pi * L / lam


def _near_vertical(ks):
    return any(math.hypot(k[0], k[1]) < 1e-6 for k in ks)


# ----------------------------------------------------------------------------- PEC image theory

def _pec(sc):
    sc.is_pec = np.ones_like(sc.is_pec)
    return sc


@pytest.mark.parametrize("scene", ["tiny_box", "street_canyon"])
def test_pec_image_theory_all_depths(scene):
    """PEC planes, vertical polarisation: a = s lambda sqrt(g_T g_R) / (4 pi L), any depth."""
    if scene == "tiny_box":
        sc = _pec(scenegen.tiny_box())
        n_rays, depth = 200_000, 3
    else:
        sc = _pec(scenegen.street_canyon())
        sc = sc.subset_rx(np.arange(0, 4096, 61))
        n_rays, depth = 200_000, 3
    walls = wall_of(sc)
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=n_rays, depth=depth)
    gt, gr = 1.3, 0.8
    a = o.fields(tr, gain_tx=gt, gain_rx=gr)
    lam = C0 / sc.freq_hz
    counts = {0: 0, 1: 0, 2: 0, 3: 0}
    mixed_q2 = 0
    checked = 0
    for i in range(len(a)):
        q = int(tr["depth"][i])
        ks, L = path_geometry(tr["pts"][i], q)
        if _near_vertical(ks):
            continue
        axes = [walls[t][0] for t in tr["seq"][i, :q]]
        s = (-1.0) ** sum(1 for ax in axes if ax != 2)
        ref = s * lam / (4 * math.pi * L) * math.sqrt(gt * gr)
        assert abs(a[i] - ref) <= tol(L, lam) * abs(ref), (i, q, axes, a[i], ref)
        assert abs(tr["tau"][i] * C0 - L) <= 1e-12 * L
        counts[q] += 1
        checked += 1
        if q == 2 and (2 in axes) and any(ax != 2 for ax in axes):
            mixed_q2 += 1
            assert ref.real < 0   # ground (or floor) + one wall: antiphase image
    assert checked >= 0.99 * len(a)
    assert counts[2] >= 20 and counts[3] >= 20, counts
    assert mixed_q2 >= 4


# ----------------------------------------------------------------------------- shoebox, analytic angles

def _shoebox_analytic(sc, rx, seq_walls, dims):
    """Directions, per-bounce cos(theta) and length of the path of a wall sequence, from
    its image source: the last segment runs along the unfolded line image -> rx, and
    each reflection, walked backwards, flips the direction's component along its wall."""
    img = sc.tx.astype(np.float64).copy()
    for ax, c in seq_walls:
        img[ax] = 2.0 * c - img[ax]
    L = float(np.linalg.norm(rx - img))
    k = (rx - img) / L
    ks = [k]
    for ax, _ in reversed(seq_walls):
        k = k.copy()
        k[ax] = -k[ax]
        ks.append(k)
    ks = ks[::-1]
    cos = [abs(ks[j][ax]) for j, (ax, _) in enumerate(seq_walls)]
    normals = []
    for ax, _ in seq_walls:
        n = np.zeros(3)
        n[ax] = 1.0
        normals.append(n)
    return ks, cos, normals, L


@pytest.mark.parametrize("material", ["concrete", "pec"])
def test_shoebox_coefficients_at_image_angles(material):
    """Every path of order <= 3 in the closed box against the three-vector reference at
    the analytic image-source angles (relative 1e-12)."""
    sc = scenegen.tiny_box()
    if material == "pec":
        sc = _pec(sc)
    walls = wall_of(sc)
    dims = np.array([10.0, 8.0, 3.0])
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=200_000, depth=3)
    a = o.fields(tr)
    lam = C0 / sc.freq_hz
    eta = eta_of(float(sc.eps_r[0]), float(sc.sigma[0]), sc.freq_hz)
    n_by_q = {1: 0, 2: 0, 3: 0}
    for i in range(len(a)):
        q = int(tr["depth"][i])
        if q == 0:
            continue
        r = int(tr["rx"][i])
        seq_walls = [walls[t] for t in tr["seq"][i, :q]]
        ks, cos, normals, L = _shoebox_analytic(sc, sc.rx[r], seq_walls, dims)
        # the oracle's reflection points lie on the unfolded line's crossings
        kk, Lo = path_geometry(tr["pts"][i], q)
        assert abs(Lo - L) <= 1e-12 * L
        for j in range(q + 1):
            assert np.abs(kk[j] - ks[j]).max() < 1e-12
        if material == "pec":
            coeffs = [(-1.0, 1.0)] * q
        else:
            coeffs = [fresnel_pair(eta, c) for c in cos]
        ref = field_three_vector(ks, normals, coeffs, lam, L)
        assert abs(a[i] - ref) <= tol(L, lam) * abs(ref), (i, q, seq_walls, a[i], ref)
        n_by_q[q] += 1
    assert n_by_q[2] >= 16 * 10 and n_by_q[3] >= 16 * 20, n_by_q


# ----------------------------------------------------------------------------- street canyon, mixed materials

def _mixed_street():
    sc = scenegen.street_canyon().subset_rx(np.arange(5, 4096, 29))
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=300_000, depth=3)
    return sc, o, tr


def _reference_from_points(sc, tr, i, normals, lam, gt=1.0, gr=1.0, **mut):
    q = int(tr["depth"][i])
    ks, L = path_geometry(tr["pts"][i], q)
    coeffs, ns = [], []
    for t in tr["seq"][i, :q]:
        m = int(sc.tri_material[t])
        n = normals[t]
        ns.append(n)
    for j, t in enumerate(tr["seq"][i, :q]):
        m = int(sc.tri_material[t])
        if sc.is_pec[m]:
            coeffs.append((-1.0, 1.0))
        else:
            c = abs(float(np.dot(ks[j], ns[j])))
            coeffs.append(fresnel_pair(eta_of(float(sc.eps_r[m]), float(sc.sigma[m]), sc.freq_hz), c))
    return field_three_vector(ks, ns, coeffs, lam, L, gt, gr, **mut), ks


def test_street_canyon_mixed_materials_three_vector():
    """Concrete, glass, PEC and ground in one path set: every path of depth 2 and 3
    against the three-vector reference on the oracle's points (relative 1e-12)."""
    sc, o, tr = _mixed_street()
    gt, gr = 1.7, 0.6
    a = o.fields(tr, gain_tx=gt, gain_rx=gr)
    normals = tri_normals(sc)
    lam = C0 / sc.freq_hz
    n = {2: 0, 3: 0}
    mats_seen = set()
    for i in range(len(a)):
        q = int(tr["depth"][i])
        if q < 2:
            continue
        ref, ks = _reference_from_points(sc, tr, i, normals, lam, gt, gr)
        if _near_vertical(ks):
            continue
        L = tr["tau"][i] * C0
        assert abs(a[i] - ref) <= tol(L, lam) * abs(ref), (i, q, a[i], ref)
        n[q] += 1
        mats_seen.update(int(sc.tri_material[t]) for t in tr["seq"][i, :q])
    assert n[2] >= 100 and n[3] >= 100, n
    assert mats_seen == {0, 1, 2, 3}, mats_seen


@pytest.mark.parametrize("mutation", ["flip_par_out", "swap_te_tm"])
def test_multibounce_reference_is_sharp(mutation):
    """The comparison above discriminates: changing one convention of the reference
    (the sign of e_par_out, or TE/TM swapped) breaks agreement on most q >= 2 paths."""
    sc, o, tr = _mixed_street()
    a = o.fields(tr)
    normals = tri_normals(sc)
    lam = C0 / sc.freq_hz
    bad = tot = 0
    for i in range(len(a)):
        if int(tr["depth"][i]) < 2:
            continue
        ref, ks = _reference_from_points(sc, tr, i, normals, lam, **{mutation: True})
        if _near_vertical(ks):
            continue
        tot += 1
        bad += abs(a[i] - ref) > 1e-6 * abs(a[i])
    assert tot > 0 and bad >= 0.5 * tot, (bad, tot)
