"""Pins of the diffraction oracle (Sec. II-D Eq. diffraction, Sec. II-F).

* The transition function against a quadrature of its definition (mpmath).
* The half-plane: the uniform theory of diffraction with the transition function
  reproduces Sommerfeld's exact solution for a plane wave on a perfectly
  conducting half-plane (both polarisations, every angle, near the edge too);
  the exact solution is written here with mpmath's Fresnel integrals.
* Keller's point: the oracle's point of diffraction minimises the path length
  over the edge (brute force) and puts both rays on one cone about the edge.
* Continuity of the total field (line of sight + reflections + diffraction) across
  the shadow and reflection boundaries of a wedge, which is what the uniform
  theory is built to achieve: a jump of the geometric-optics field there must be
  matched by the diffracted field, in amplitude, phase and polarisation.  This
  pins the vector form (bases, signs, spreading) against the separately pinned
  reflection chain.  Exact for perfectly conducting faces at oblique incidence,
  and for lossy faces (Luebbers) at normal incidence on the edge.
* Reciprocity for perfectly conducting wedges; the material gradient against
  central differences; the wedge table on closed and open shapes.
"""
import math

import mpmath
import numpy as np
import pytest
import torch

import oracle
import scenegen
from oracle import diffraction as od
from scenegen import Scene

C0 = 299792458.0


# ----------------------------------------------------------------------------- transition function

@pytest.mark.parametrize("X", [1e-4, 0.05, 0.7, 2.0, 5.5, 20.0, 300.0])
def test_transition_function_against_quadrature(X):
    with mpmath.workdps(40):
        u = mpmath.sqrt(X)
        # int_u^inf e^{-j t^2} dt = int_0^inf - int_0^u, the oscillating integrand
        # integrated piecewise at 40 digits
        tail = mpmath.sqrt(mpmath.pi) / 2 * mpmath.exp(-1j * mpmath.pi / 4) - mpmath.quad(
            lambda t: mpmath.exp(-1j * t * t), mpmath.linspace(0, u, 64))
        ref = complex(2j * u * mpmath.exp(1j * X) * tail)
    got = complex(od.transition(X))
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_transition_function_limits():
    assert abs(od.transition(1e6) - 1) < 1e-6
    X = 1e-10   # F(X) ~ sqrt(pi X) e^{j pi/4} for small X
    assert abs(od.transition(X) / (math.sqrt(math.pi * X) * np.exp(1j * math.pi / 4)) - 1) < 1e-4


# ----------------------------------------------------------------------------- half-plane, exact

def _G(x):
    """(e^{j pi/4} / sqrt(pi)) int_{-inf}^x e^{-j t^2} dt, via mpmath's Fresnel integrals."""
    v = x * mpmath.sqrt(2 / mpmath.pi)
    half = mpmath.sqrt(mpmath.pi / 2)
    i0x = half * (mpmath.fresnelc(v) - 1j * mpmath.fresnels(v))
    return complex(mpmath.exp(1j * mpmath.pi / 4) / mpmath.sqrt(mpmath.pi)
                   * (mpmath.sqrt(mpmath.pi) / 2 * mpmath.exp(-1j * mpmath.pi / 4) + i0x))


def _sommerfeld(k, rho, phi, php, hard):
    """Exact total field of a unit plane wave exp(j k rho cos(phi - phi')) on a perfectly
    conducting half-plane (Dirichlet: soft, Neumann: hard), e^{+j omega t} convention."""
    sgn = 1 if hard else -1
    return (np.exp(1j * k * rho * math.cos(phi - php)) * _G(math.sqrt(2 * k * rho) * math.cos((phi - php) / 2))
            + sgn * np.exp(1j * k * rho * math.cos(phi + php)) * _G(math.sqrt(2 * k * rho) * math.cos((phi + php) / 2)))


@pytest.mark.parametrize("hard", [False, True])
@pytest.mark.parametrize("krho", [2.0, 30.0, 900.0])
def test_half_plane_equals_sommerfeld(hard, krho):
    k = 2 * math.pi
    rho = krho / k
    R = 1.0 if hard else -1.0
    worst = 0.0
    for php in (0.4, 1.3, 2.9):
        for phi in np.linspace(0.03, 2 * math.pi - 0.03, 29):
            Ds, Dh = od.coefficients(2.0, phi, php, 1.0, k, rho, R, R, R, R)
            D = (Dh if hard else Ds).item()
            go = 0j
            if phi - php < math.pi:
                go += np.exp(1j * k * rho * math.cos(phi - php))
            if phi + php < math.pi:
                go += R * np.exp(1j * k * rho * math.cos(phi + php))
            utd = go + D * np.exp(-1j * k * rho) / math.sqrt(rho)
            worst = max(worst, abs(utd - _sommerfeld(k, rho, phi, php, hard)))
    assert worst < 1e-12, worst


# ----------------------------------------------------------------------------- scenes for the geometric pins

def _box_scene(eps=(5.24, 3.0), sig=(0.0462, 0.2), pec=(0, 0), tx=(-20.0, 4.0, 6.0), freq=0.3e9):
    """One 10 x 10 x 10 m box (outward normals), faces split in two materials:
    the x-faces and z-faces material 0, the y-faces material 1."""
    v, t, fid = scenegen.box_faces((0, 0, 0), (10, 10, 10), (1, 1, 1))
    mat = np.where((fid == 2) | (fid == 3), 1, 0).astype(np.int32)
    return Scene(name="box", verts=v, tris=t, tri_material=mat, eps_r=np.array(eps, np.float32),
                 sigma=np.array(sig, np.float32), is_pec=np.array(pec, np.uint8),
                 tx=np.array(tx, np.float64), rx=np.zeros((1, 3)), n_rays=100_000, max_depth=1,
                 freq_hz=freq, f_center_hz=freq, delta_f_hz=1e6, n_sub=16)


def _total_field(sc, rx):
    """H = sum_i a_i exp(-j 2 pi f tau_i) over line of sight, single reflections and
    diffraction, at receivers rx (R, 3)."""
    sc.rx = np.asarray(rx, np.float64)
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=sc.n_rays, depth=1)
    a = o.fields(tr)
    H = np.zeros(len(rx), complex)
    np.add.at(H, tr["rx"], a * np.exp(-2j * math.pi * sc.freq_hz * tr["tau"]))
    dp = od.paths(o, n_rays=sc.n_rays)
    ad = od.fields(sc, dp, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64)).numpy()
    np.add.at(H, dp["rx"], ad * np.exp(-2j * math.pi * sc.freq_hz * dp["tau"]))
    return H, tr, dp


def _boundary_pair(tx, through, beyond, off, delta):
    """Two receivers at distance `beyond` past `through` on the ray tx -> through,
    displaced by +-delta along `off`."""
    d = (through - tx) / np.linalg.norm(through - tx)
    c = through + beyond * d
    return np.stack([c + delta * off, c - delta * off])


def _assert_continuous(H, tr, scale, tol=2e-4):
    assert abs(H[0] - H[1]) <= tol * scale, (abs(H[0] - H[1]) / scale)


@pytest.mark.parametrize("case", ["pec_oblique", "lossy_normal"])
def test_total_field_continuous_across_shadow_boundary(case):
    # the top edge x = 0, z = 10 (along y) of the box; Tx to its left, below the roof
    if case == "pec_oblique":
        sc = _box_scene(pec=(1, 1), tx=(-20.0, 1.0, 6.0))
        edge_pt = np.array([0.0, 6.5, 10.0])
    else:
        sc = _box_scene(tx=(-20.0, 5.0, 6.0))
        edge_pt = np.array([0.0, 5.0, 10.0])
    tx = sc.tx
    d = (edge_pt - tx) / np.linalg.norm(edge_pt - tx)
    off = np.cross(d, [0, 1.0, 0])
    off /= np.linalg.norm(off)
    rx = _boundary_pair(tx, edge_pt, 4.0, off, 2e-6)
    H, tr, dp = _total_field(sc, rx)
    los = [(tr["rx"] == r) & (tr["depth"] == 0) for r in range(2)]
    assert los[0].sum() + los[1].sum() == 1          # the line of sight exists on one side only
    a_los = abs(oracle.OracleScene(sc).fields(tr)[los[0] | los[1]][0])
    assert a_los > 0
    _assert_continuous(H, tr, a_los)


@pytest.mark.parametrize("case", ["pec_oblique", "lossy_normal"])
def test_total_field_continuous_across_reflection_boundary(case):
    # reflection off the roof (z = 10) near its edge x = 0: Tx above the roof level
    if case == "pec_oblique":
        sc = _box_scene(pec=(1, 1), tx=(-12.0, 2.0, 14.0))
        edge_pt = np.array([0.0, 6.0, 10.0])
    else:
        sc = _box_scene(tx=(-12.0, 5.0, 14.0))
        edge_pt = np.array([0.0, 5.0, 10.0])
    tx = sc.tx
    d = (edge_pt - tx) / np.linalg.norm(edge_pt - tx)
    dr = d * np.array([1.0, 1.0, -1.0])            # reflected in the roof plane
    img = tx * np.array([1.0, 1.0, -1.0]) + np.array([0, 0, 20.0])   # Tx mirrored in z = 10
    off = np.cross(dr, [0, 1.0, 0])
    off /= np.linalg.norm(off)
    rx = _boundary_pair(img, edge_pt, 6.0, off, 2e-6)
    H, tr, dp = _total_field(sc, rx)
    refl = [(tr["rx"] == r) & (tr["depth"] == 1) for r in range(2)]
    roof = [t for t in range(len(sc.tris)) if np.all(sc.verts[sc.tris[t]][:, 2] == 10.0)]
    n_roof = [int(np.isin(tr["seq"][refl[r], 0], roof).sum()) for r in range(2)]
    assert sorted(n_roof) == [0, 1], n_roof        # the roof reflection exists on one side only
    a = oracle.OracleScene(sc).fields(tr)
    los = (tr["depth"] == 0)
    _assert_continuous(H, tr, float(np.abs(a[los]).max()))


def test_uniform_theory_is_needed_for_continuity():
    # without the diffracted field the total jumps at the shadow boundary: the
    # continuity checks above are sharp
    sc = _box_scene(pec=(1, 1), tx=(-20.0, 1.0, 6.0))
    edge_pt = np.array([0.0, 6.5, 10.0])
    d = (edge_pt - sc.tx) / np.linalg.norm(edge_pt - sc.tx)
    off = np.cross(d, [0, 1.0, 0])
    off /= np.linalg.norm(off)
    rx = _boundary_pair(sc.tx, edge_pt, 4.0, off, 2e-6)
    H, tr, dp = _total_field(sc, rx)
    ad = od.fields(sc, dp, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64)).numpy()
    Hd = np.zeros(2, complex)
    np.add.at(Hd, dp["rx"], ad * np.exp(-2j * math.pi * sc.freq_hz * dp["tau"]))
    go = H - Hd
    a_los = np.abs(oracle.OracleScene(sc).fields(tr)[tr["depth"] == 0]).max()
    assert abs(go[0] - go[1]) > 0.3 * a_los


# ----------------------------------------------------------------------------- Keller point, reciprocity, gradients

def test_keller_point_is_shortest_and_on_the_cone():
    sc = scenegen.street_canyon().subset_rx(np.arange(0, 4096, 211))
    o = oracle.OracleScene(sc)
    dp = od.paths(o, n_rays=100_000)
    W = dp["wedges"]
    assert len(dp["tau"]) > 20
    for i in range(0, len(dp["tau"]), max(1, len(dp["tau"]) // 25)):
        w = dp["wedge"][i]
        T, Q, R = dp["pts"][i]
        e, s0, ln = W["e"][w], W["start"][w], W["length"][w]
        x = np.linspace(0.0, ln, 20001)
        P = s0[None, :] + x[:, None] * e[None, :]
        Lb = np.linalg.norm(P - T, axis=1) + np.linalg.norm(R - P, axis=1)
        Lq = np.linalg.norm(Q - T) + np.linalg.norm(R - Q)
        assert Lq <= Lb.min() + 1e-9
        assert abs(Lq - dp["tau"][i] * C0) < 1e-9 * Lq
        ci = np.dot((Q - T) / np.linalg.norm(Q - T), e)
        co = np.dot((R - Q) / np.linalg.norm(R - Q), e)
        assert abs(ci - co) < 1e-9


def test_reciprocity_pec_wedge():
    sc = _box_scene(pec=(1, 1))
    A, B = np.array([-20.0, 2.0, 6.0]), np.array([14.0, 7.0, 16.0])
    res = []
    for tx, rx in ((A, B), (B, A)):
        sc.tx = tx.copy()
        sc.rx = rx[None, :].copy()
        o = oracle.OracleScene(sc)
        dp = od.paths(o, n_rays=sc.n_rays)
        a = od.fields(sc, dp, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64)).numpy()
        res.append({tuple(sorted(f)): v for f, v in zip(dp["faces"], a)})
    assert set(res[0]) == set(res[1]) and len(res[0]) >= 1
    for key in res[0]:
        assert abs(res[0][key] - res[1][key]) <= 1e-12 * abs(res[0][key])


def test_material_gradient_fd():
    sc = _box_scene(tx=(-20.0, 3.0, 6.0), freq=1.0e9)
    sc.rx = np.array([[14.0, 7.0, 16.0], [5.0, 16.0, 3.0], [-3.0, 12.0, 14.0]])
    o = oracle.OracleScene(sc)
    dp = od.paths(o, n_rays=sc.n_rays)
    assert len(dp["tau"]) >= 3
    mats = sc.tri_material[dp["faces"]]
    assert np.any(mats[:, 0] != mats[:, 1])         # wedges with different face materials
    rng = np.random.default_rng(0)
    g = rng.normal(size=len(dp["tau"])) + 1j * rng.normal(size=len(dp["tau"]))
    eps = torch.tensor(sc.eps_r.astype(np.float64), requires_grad=True)
    sig = torch.tensor(sc.sigma.astype(np.float64), requires_grad=True)
    a = od.fields(sc, dp, eps, sig)
    (torch.as_tensor(g).conj() * a).real.sum().backward()

    def loss(e, s):
        return float((np.conj(g) * od.fields(sc, dp, e, s).numpy()).real.sum())
    for arr, grad in ((sc.eps_r, eps.grad), (sc.sigma, sig.grad)):
        for m in range(2):
            h = 1e-6 * max(abs(float(arr[m])), 1e-3)
            p, q = arr.astype(np.float64), arr.astype(np.float64)
            p[m] += h
            q[m] -= h
            if arr is sc.eps_r:
                fd = (loss(p, sc.sigma.astype(np.float64)) - loss(q, sc.sigma.astype(np.float64))) / (2 * h)
            else:
                fd = (loss(sc.eps_r.astype(np.float64), p) - loss(sc.eps_r.astype(np.float64), q)) / (2 * h)
            assert abs(fd - grad[m].item()) <= 1e-6 * max(abs(grad[m].item()), 1e-30) + 1e-18, (m, fd, grad[m])


# ----------------------------------------------------------------------------- wedge table

def test_wedge_table_shapes():
    # a closed box: 12 convex edges (n = 3/2); its quad diagonals are flat (n = 1)
    o = oracle.OracleScene(_box_scene())
    W = od.wedges(o)
    assert len(W["n"]) == 12 and np.allclose(W["n"], 1.5)
    # the inside of a room (inward normals): every edge is concave, none is a wedge
    assert len(od.wedges(oracle.OracleScene(scenegen.tiny_box()))["n"]) == 0
    # a screen: two coincident triangles back to back give a half-plane (n = 2)
    v = np.array([[0, 0, 0], [4, 0, 0], [0, 0, 3]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 1]], np.int32)
    sc = Scene(name="screen", verts=v, tris=t, tri_material=np.zeros(2, np.int32), eps_r=np.ones(1, np.float32),
               sigma=np.zeros(1, np.float32), is_pec=np.ones(1, np.uint8), tx=np.zeros(3), rx=np.zeros((1, 3)),
               n_rays=10, max_depth=1, freq_hz=1e9, f_center_hz=1e9, delta_f_hz=1e6, n_sub=8)
    W = od.wedges(oracle.OracleScene(sc))
    assert len(W["n"]) == 3 and np.allclose(W["n"], 2.0)
