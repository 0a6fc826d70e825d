"""Pins of the neural-material oracle (Sec. III-D): BF16 rounding from its
definition, the positional encoding at special points, the material transforms,
and the backward pass against central finite differences."""
import math

import numpy as np

from oracle import mlp
import scenegen


def test_bf16_round_to_nearest_even():
    # BF16 spacing at 1 is 2^-7; halfway cases go to the even mantissa
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20, 1 + 3 * 2.0 ** -8, -2.5, 3.0e-3, 0.0])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0
    assert r[2] == 1 + 2.0 ** -7
    assert r[3] == 1 + 2.0 ** -6
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 2.0 ** -8 * 3.0e-3 and r[6] == 0.0   # half a BF16 ulp
    # every BF16 value is a fixed point
    y = mlp.bf16_round(np.random.default_rng(0).normal(size=1000))
    assert np.array_equal(mlp.bf16_round(y), y)


def test_positional_encoding_special_points():
    # p = 0: sines 0, cosines 1; p = 1/8 along x: sin(2^k pi / 8) for k = 1..6
    g0 = mlp.encode(np.zeros((1, 3)))
    assert g0.shape == (1, 39)
    assert np.allclose(g0[0, :3], 0) and np.allclose(g0[0, 3::6], 0) and np.allclose(g0[0, 6::6], 1)
    g = mlp.encode(np.array([[0.125, 0.0, 0.0]]))
    for k in range(1, 7):
        assert abs(g[0, 3 + 6 * (k - 1)] - math.sin(2 ** k * math.pi / 8)) < 1e-15
        assert abs(g[0, 6 + 6 * (k - 1)] - math.cos(2 ** k * math.pi / 8)) < 1e-15


def test_normalisation_unit_cube():
    lo, hi = np.array([0.0, -2.0, 0.0]), np.array([24.0, 10.0, 3.5])
    p = mlp.normalize(np.array([[0.0, -2.0, 0.0], [24.0, 10.0, 3.5], [12.0, 4.0, 1.75]]), lo, hi)
    assert np.allclose(p[0], [-0.5, -0.25, -3.5 / 48]) and np.allclose(p[1], [0.5, 0.25, 3.5 / 48])
    assert np.allclose(p[2], 0.0)


def test_material_transforms():
    out = np.array([[math.log(0.05), math.log(3.0)]])
    eps, sig = mlp.materials(out)
    assert abs(sig[0] - 0.05) < 1e-15 and abs(eps[0] - 4.0) < 1e-14


def test_backward_matches_finite_differences():
    Ws, bs = scenegen.random_mlp_params(3, width=16)
    rng = np.random.default_rng(1)
    x = mlp.encode(rng.uniform(-0.5, 0.5, (20, 3)))
    ge, gs = rng.normal(size=20), rng.normal(size=20)

    def L(Ws_, bs_):
        out, _, _ = mlp.forward(x, Ws_, bs_, bf16=False)
        eps, sig = mlp.materials(out)
        return float(np.sum(ge * eps + gs * sig))

    gW, gb = mlp.backward(x, Ws, bs, ge, gs, bf16=False)
    h = 1e-6
    for li, (i, j) in [(0, (5, 3)), (1, (2, 7)), (2, (11, 0)), (3, (4, 1))]:
        Wp = [w.astype(np.float64).copy() for w in Ws]
        Wm = [w.astype(np.float64).copy() for w in Ws]
        Wp[li][i, j] += h
        Wm[li][i, j] -= h
        fd = (L(Wp, bs) - L(Wm, bs)) / (2 * h)
        assert abs(fd - gW[li][i, j]) <= 1e-6 * max(1.0, abs(fd))
    for li, j in [(0, 2), (3, 1)]:
        bp = [b.astype(np.float64).copy() for b in bs]
        bm = [b.astype(np.float64).copy() for b in bs]
        bp[li][j] += h
        bm[li][j] -= h
        fd = (L(Ws, bp) - L(Ws, bm)) / (2 * h)
        assert abs(fd - gb[li][j]) <= 1e-6 * max(1.0, abs(fd))
