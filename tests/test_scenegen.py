"""The seeded synthetic workloads: the sizes, seeds and structure that stand in for
the paper's scenes (the input recipe), determinism under a seed, and the
properties both the CUDA path and the oracle rely on (FP32-exact coordinates,
valid triangle and material indices)."""
import numpy as np
import pytest

import scenegen


def _valid(sc):
    assert sc.verts.dtype == np.float32 and sc.verts.ndim == 2 and sc.verts.shape[1] == 3
    assert sc.tris.dtype == np.int32 and sc.tris.shape[1] == 3
    assert sc.tris.min() >= 0 and sc.tris.max() < sc.verts.shape[0]
    assert sc.tri_material.shape == (sc.n_tris,)
    if sc.per_triangle:
        assert sc.eps_r.shape[0] == sc.n_tris
    else:
        assert sc.tri_material.min() >= 0 and sc.tri_material.max() < sc.n_materials
    assert sc.eps_r.shape == sc.sigma.shape == sc.is_pec.shape
    assert np.all(sc.eps_r >= 1.0) and np.all(sc.sigma >= 0.0)
    # transmitter and receivers are exactly representable in FP32
    assert np.array_equal(sc.tx, sc.tx.astype(np.float32).astype(np.float64))
    assert np.array_equal(sc.rx, sc.rx.astype(np.float32).astype(np.float64))
    # no degenerate triangle
    v = sc.verts.astype(np.float64)
    n = np.cross(v[sc.tris[:, 1]] - v[sc.tris[:, 0]], v[sc.tris[:, 2]] - v[sc.tris[:, 0]])
    assert np.all(np.linalg.norm(n, axis=1) > 0.0)


def _same(a, b):
    for f in ("verts", "tris", "tri_material", "eps_r", "sigma", "is_pec", "tx", "rx"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_tiny_box():
    sc = scenegen.tiny_box()
    _valid(sc)
    assert (sc.n_tris, sc.n_rx, sc.n_rays, sc.max_depth) == (12, 16, 10_000, 2)


def test_street_canyon_recipe():
    sc = scenegen.street_canyon()
    _valid(sc)
    assert (sc.n_tris, sc.n_rx, sc.n_rays, sc.max_depth) == (770, 4096, 1_000_000, 3)
    assert (sc.n_sub, sc.delta_f_hz, sc.freq_hz) == (1024, 48828.125, 3.5e9)
    assert sc.n_sub * sc.delta_f_hz == 50e6            # 1024 subcarriers over 50 MHz
    assert np.any(sc.is_pec == 1)                       # metal
    assert np.allclose(sc.rx[:, 2], 1.5)                # receivers at 1.5 m
    _same(sc, scenegen.street_canyon())
    assert not np.array_equal(scenegen.street_canyon(seed=5).verts, sc.verts)   # the seed places the boxes


def test_indoor_recipe():
    sc = scenegen.indoor_diff()
    _valid(sc)
    assert (sc.n_tris, sc.n_rx, sc.n_rays, sc.max_depth, sc.n_materials) == (5088, 1024, 1_000_000, 3, 8)
    assert (sc.n_sub, sc.delta_f_hz, sc.f_center_hz) == (1024, 48828.125, 1.272e9)
    assert np.all((sc.eps_r >= 2.0) & (sc.eps_r <= 10.0))
    assert np.all((sc.sigma >= 1e-3) & (sc.sigma <= 1.0))
    # receivers on a walk of 0.1 m steps at 1.5 m
    steps = np.linalg.norm(np.diff(sc.rx, axis=0), axis=1)
    assert np.allclose(steps, 0.1, atol=1e-5) and np.allclose(sc.rx[:, 2], 1.5)
    _same(sc, scenegen.indoor_diff())


def test_room_corridor_recipe():
    sc = scenegen.room_corridor(n_rx=2000)
    _valid(sc)
    assert sc.per_triangle and sc.n_tris == 19_626 and sc.n_rx == 2000
    assert (sc.n_sub, sc.delta_f_hz) == (256, 195312.5)
    assert np.all((sc.eps_r >= 2.0) & (sc.eps_r <= 10.0))
    assert np.all((sc.sigma >= 1e-3) & (sc.sigma <= 1.0))


def test_city_batch_recipe():
    cities = scenegen.city_batch()
    assert len(cities) == 16
    assert sum(c.n_rx for c in cities) == 65_536 and min(c.n_rx for c in cities) >= 256
    t = np.array([c.n_tris for c in cities])
    assert t.min() >= 500 and t.max() <= 60_000 and t.max() / t.min() > 10   # uneven sizes
    for c in cities:
        _valid(c)
        assert (c.n_rays, c.max_depth, c.n_sub) == (10_000_000, 4, 256)


@pytest.mark.parametrize("seed", [0, 7])
def test_random_cfr_inputs_recipe(seed):
    a, tau, offs = scenegen.random_cfr_inputs(seed, 64, 5, empty_every=7)
    a2, tau2, offs2 = scenegen.random_cfr_inputs(seed, 64, 5, empty_every=7)
    assert np.array_equal(a, a2) and np.array_equal(tau, tau2) and np.array_equal(offs, offs2)
    counts = np.diff(offs)
    assert offs[0] == 0 and offs[-1] == len(a) == len(tau)
    assert np.all(counts[::7] == 0) and len(set(counts[1::7].tolist() + counts[2::7].tolist())) > 1   # ragged
    mag = np.abs(a.astype(np.complex128))
    assert mag.min() >= 1e-5 * (1 - 1e-6) and mag.max() <= 1e-2 * (1 + 1e-6)
    assert tau.min() >= 1e-9 and tau.max() <= 1.5e-6


def test_random_scattering_recipe():
    s = scenegen.random_scattering(21, 8)
    assert s.shape == (8, 8) and s.dtype == np.float32
    assert np.all((s[:, 0] >= 0.2) & (s[:, 0] <= 0.7))     # S
    assert np.all((s[:, 1] >= 0.05) & (s[:, 1] <= 0.5))    # K_x
    assert np.allclose(s[:, 2:5].sum(axis=1), 1.0, atol=1e-6) and np.all(s[:, 2:5] > 0)   # lobe weights
    assert np.all((s[:, 5:7] >= 2.0) & (s[:, 5:7] <= 15.0))  # concentrations
    assert np.array_equal(s, scenegen.random_scattering(21, 8))
