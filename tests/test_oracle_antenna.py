"""Pins of the FP64 oracle of the trainable antenna pattern (oracle/antenna.py)
to the normalisation of Eq. atenna_normalization, closed forms of a single lobe,
and numerical differentiation."""
import numpy as np

from oracle import antenna as oa


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _sphere_grid(n_theta=400, n_phi=400):
    """Gauss-Legendre in cos(theta) x uniform phi: directions and solid-angle weights."""
    x, wx = np.polynomial.legendre.leggauss(n_theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    c, p = np.meshgrid(x, phi, indexing="ij")
    s = np.sqrt(1 - c ** 2)
    r = np.stack([s * np.cos(p), s * np.sin(p), c], -1).reshape(-1, 3)
    wts = (wx[:, None] * np.full(n_phi, 2 * np.pi / n_phi)[None, :]).reshape(-1)
    return r, wts


def _params():
    w = np.array([0.5, 0.3, 0.2])
    lam = np.array([0.7, 5.0, 30.0])
    mu = _unit([[0.0, 0.0, 1.0], [1.0, 1.0, 0.0], [-0.3, 0.2, -0.9]])
    return w, lam, mu


def test_normalisation_4pi_eta():
    # the integral of G over the sphere equals 4 pi eta_rad (Eq. atenna_normalization)
    r, wts = _sphere_grid()
    w, lam, mu = _params()
    for eta in (1.0, 0.7):
        integral = (oa.gain(r, w, lam, mu, eta) * wts).sum()
        np.testing.assert_allclose(integral, 4 * np.pi * eta, rtol=1e-6)


def test_flat_limit_is_isotropic():
    r = _unit(np.random.default_rng(0).normal(size=(50, 3)))
    g = oa.gain(r, [1.0], [1e-5], [[0.0, 0.0, 1.0]], 0.9)
    np.testing.assert_allclose(g, 0.9, rtol=2e-5)


def test_single_lobe_closed_forms():
    mu = _unit([[0.2, -0.5, 0.8]])
    lam = 10.0
    # peak directivity 2 lambda / (1 - exp(-2 lambda)) along mu, ratio exp(2 lambda) to the opposite direction
    g_peak = oa.gain(mu, [1.0], [lam], mu)[0]
    np.testing.assert_allclose(g_peak, 2 * lam / (1 - np.exp(-2 * lam)), rtol=1e-12)
    g_back = oa.gain(-mu, [1.0], [lam], mu)[0]
    np.testing.assert_allclose(g_peak / g_back, np.exp(2 * lam), rtol=1e-10)
    # rotational symmetry about mu
    perp = _unit(np.cross(mu[0], [1.0, 0.0, 0.0]))
    perp2 = _unit(np.cross(mu[0], perp))
    c = 0.3
    s = np.sqrt(1 - c * c)
    r = np.stack([c * mu[0] + s * perp, c * mu[0] + s * perp2])
    g = oa.gain(r, [1.0], [lam], mu)
    np.testing.assert_allclose(g[0], g[1], rtol=1e-12)


def test_gain_gradient_finite_differences():
    rng = np.random.default_rng(1)
    r = _unit(rng.normal(size=(40, 3)))
    w, lam, mu = _params()
    eta = 0.8
    gG = rng.normal(size=40)
    dw, dlam, dmu = oa.gain_grad(r, w, lam, mu, eta, gG)

    def L(w_, lam_, mu_):
        return float((gG * oa.gain(r, w_, lam_, mu_, eta)).sum())
    e = 1e-6
    for i in range(3):
        d = np.zeros(3)
        d[i] = e
        np.testing.assert_allclose(dw[i], (L(w + d, lam, mu) - L(w - d, lam, mu)) / (2 * e), rtol=1e-6)
        np.testing.assert_allclose(dlam[i], (L(w, lam + d * lam[i], mu) - L(w, lam - d * lam[i], mu))
                                   / (2 * e * lam[i]), rtol=1e-5)
        for k in range(3):
            dm = np.zeros((3, 3))
            dm[i, k] = e
            np.testing.assert_allclose(dmu[i, k], (L(w, lam, mu + dm) - L(w, lam, mu - dm)) / (2 * e),
                                       rtol=1e-5, atol=1e-9)


def test_apply_and_adjoint():
    rng = np.random.default_rng(2)
    P = 30
    a = rng.normal(size=P) + 1j * rng.normal(size=P)
    aod = _unit(rng.normal(size=(P, 3)))
    aoa = _unit(rng.normal(size=(P, 3)))
    tx = (*_params(), 1.0)
    rx = (np.array([1.0]), np.array([3.0]), _unit([[0.0, 1.0, 0.0]]), 0.9)
    out, gt, gr = oa.apply(a, aod, aoa, tx, rx)
    np.testing.assert_allclose(np.abs(out) ** 2, np.abs(a) ** 2 * gt * gr, rtol=1e-12)
    # no pattern: the coefficient is unchanged
    np.testing.assert_allclose(oa.apply(a, aod, aoa, None, None)[0], a)
    g = rng.normal(size=P) + 1j * rng.normal(size=P)
    da, dgt, dgr = oa.apply_grad(out, gt, gr, g)

    def L(a_, gt_, gr_):
        return float(np.real(np.conj(g) * a_ * np.sqrt(gt_ * gr_)).sum())
    e = 1e-7
    for i in (0, 7):
        d = np.zeros(P)
        d[i] = e
        np.testing.assert_allclose(dgt[i], (L(a, gt + d, gr) - L(a, gt - d, gr)) / (2 * e), rtol=1e-6)
        np.testing.assert_allclose(dgr[i], (L(a, gt, gr + d) - L(a, gt, gr - d)) / (2 * e), rtol=1e-6)
        np.testing.assert_allclose(da[i].real, (L(a + d, gt, gr) - L(a - d, gt, gr)) / (2 * e), rtol=1e-6)


def test_directions_of_a_path():
    # Tx at the origin, one bounce at (3, 4, 0), Rx at (3, 4, 5)
    pts = np.zeros((1, 4, 3))
    pts[0, 1] = [3, 4, 0]
    pts[0, 2] = [3, 4, 5]
    aod, aoa = oa.directions(pts, [1])
    np.testing.assert_allclose(aod[0], [0.6, 0.8, 0.0])
    np.testing.assert_allclose(aoa[0], [0.0, 0.0, -1.0])
