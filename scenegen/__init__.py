"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *builds inputs*: triangle meshes, material tables, transmitter and
receiver positions, and seeded random tensors.  It contains none of the method's
arithmetic (no ray tracing, no field or CFR computation), so both the GPU library
and the CPU oracle may consume its output without sharing any computation.

Scenes (the five workloads; every coordinate is exactly representable in FP32):

* ``tiny_box``       closed 10x8x3 m concrete room, 12 triangles, 16 Rx, 1e4 rays, depth 2, 3.5 GHz.
* ``street_canyon``  64 seeded boxes on a 500x500 m ground (770 triangles), 4096 Rx,
                     1e6 rays, depth 3, 3.5 GHz.
* ``indoor_diff``    20x15x4 m room with 40 obstacles (about 5.1k triangles), 8 materials
                     with hidden ground truth, 1024 Rx on a random walk, 1024 subcarriers
                     of 48.828125 kHz around 1.272 GHz.
* ``room_corridor``  about 20k triangles, per-triangle ground-truth materials drawn from
                     smooth random fields, 1e5 Rx, 256 subcarriers.
* ``city_batch``     16 procedural cities of 1k-50k triangles, 65,536 Rx split unevenly.

The scene geometry follows the paper's setting of a triangle-mesh scene whose
objects carry materials (Sec. II-D, Sec. IV-A); the concrete sizes are synthetic
stand-ins for the paper's institute model and DICHASUS measurement campaign, which
are not available.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "Scene", "tiny_box", "street_canyon", "indoor_diff", "room_corridor", "city_batch",
    "box_faces", "random_cfr_inputs", "random_fields_inputs", "random_mlp_params", "random_scattering",
    "ground_plane",
    "CONCRETE", "GLASS", "GROUND", "SPEED_OF_LIGHT", "VACUUM_PERMITTIVITY",
]

# CODATA 2018 values (the paper names the constants but does not print them).
SPEED_OF_LIGHT = 299792458.0
VACUUM_PERMITTIVITY = 8.8541878128e-12

# (eps_r, sigma [S/m]) used as frequency-independent constants.
CONCRETE = (5.24, 0.0462)
GLASS = (6.31, 0.0036)
GROUND = (15.0, 0.035)


@dataclasses.dataclass
class Scene:
    name: str
    verts: np.ndarray          # (V, 3) float32
    tris: np.ndarray           # (T, 3) int32, normal = (v1-v0) x (v2-v0)
    tri_material: np.ndarray   # (T,) int32 index into the material table
    eps_r: np.ndarray          # (M,) float32 relative permittivity (ground truth)
    sigma: np.ndarray          # (M,) float32 conductivity [S/m] (ground truth)
    is_pec: np.ndarray         # (M,) uint8, 1 = perfect electric conductor
    tx: np.ndarray             # (3,) float64, FP32-exact
    rx: np.ndarray             # (R, 3) float64, FP32-exact
    n_rays: int
    max_depth: int
    freq_hz: float             # frequency at which path coefficients are evaluated
    f_center_hz: float         # CFR centre frequency
    delta_f_hz: float          # CFR subcarrier spacing
    n_sub: int                 # number of subcarriers
    per_triangle: bool = False  # materials indexed by triangle instead of by material id
    seed: int = 0
    tri_object: Optional[np.ndarray] = None   # (T,) object index of each triangle (when meaningful)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_rx(self) -> int:
        return int(self.rx.shape[0])

    @property
    def n_materials(self) -> int:
        return int(self.eps_r.shape[0])

    def subset_rx(self, idx) -> "Scene":
        return dataclasses.replace(self, rx=np.ascontiguousarray(self.rx[idx]))

    def with_rays(self, n_rays: int, max_depth: Optional[int] = None) -> "Scene":
        return dataclasses.replace(self, n_rays=int(n_rays),
                                   max_depth=self.max_depth if max_depth is None else int(max_depth))


def _f32(x):
    """Round to the nearest FP32 value and return as float64 (exact)."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


class _MeshBuilder:
    def __init__(self):
        self.verts: List[np.ndarray] = []
        self.tris: List[np.ndarray] = []
        self.mats: List[np.ndarray] = []
        self.nv = 0

    def add(self, v: np.ndarray, t: np.ndarray, mat: int):
        self.verts.append(v.astype(np.float32))
        self.tris.append((t + self.nv).astype(np.int32))
        self.mats.append(np.full(t.shape[0], mat, np.int32))
        self.nv += v.shape[0]

    def add_mats(self, v: np.ndarray, t: np.ndarray, mats: np.ndarray):
        self.verts.append(v.astype(np.float32))
        self.tris.append((t + self.nv).astype(np.int32))
        self.mats.append(mats.astype(np.int32))
        self.nv += v.shape[0]

    def build(self):
        return (np.ascontiguousarray(np.concatenate(self.verts)),
                np.ascontiguousarray(np.concatenate(self.tris)),
                np.ascontiguousarray(np.concatenate(self.mats)))


def _axis_coords(lo: float, hi: float, n: int) -> np.ndarray:
    c = np.linspace(lo, hi, n + 1)
    c[0], c[-1] = lo, hi
    return np.asarray(c, np.float32)


def box_faces(lo, hi, subdiv=(1, 1, 1), inward=False, skip_faces=()):
    """Triangles of an axis-aligned box [lo, hi], each face split into a grid of quads.

    ``subdiv[a]`` is the number of cells along axis ``a``.  Every quad is split along
    its diagonal into two triangles with the same winding, so the geometric normal
    (v1-v0)x(v2-v0) points out of the box (into it when ``inward``).  Coordinates of
    shared edges are taken from one per-axis table, so adjacent faces share exact
    vertex positions.  ``skip_faces`` lists faces to omit as (axis, side) pairs,
    side 0 = low, 1 = high.  Returns (verts (V,3) f32, tris (T,3) i32, face_id (T,)).
    """
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    coords = [_axis_coords(lo[a], hi[a], int(subdiv[a])) for a in range(3)]
    verts, tris, fids = [], [], []
    nv = 0
    fid = 0
    for f in range(3):
        for side in (0, 1):
            if (f, side) in skip_faces:
                fid += 1
                continue
            outward_sign = 1 if side == 1 else -1
            sign = -outward_sign if inward else outward_sign
            a, b = (f + 1) % 3, (f + 2) % 3      # e_a x e_b = +e_f
            if sign < 0:
                a, b = b, a
            ca, cb = coords[a], coords[b]
            na, nb = len(ca), len(cb)
            grid = np.zeros((na, nb, 3), np.float32)
            grid[:, :, f] = coords[f][-1] if side == 1 else coords[f][0]
            grid[:, :, a] = ca[:, None]
            grid[:, :, b] = cb[None, :]
            v = grid.reshape(-1, 3)
            idx = np.arange(na * nb).reshape(na, nb)
            p00 = idx[:-1, :-1].ravel()
            p10 = idx[1:, :-1].ravel()
            p11 = idx[1:, 1:].ravel()
            p01 = idx[:-1, 1:].ravel()
            t = np.concatenate([np.stack([p00, p10, p11], 1), np.stack([p00, p11, p01], 1)])
            # interleave the two triangles of each quad
            t = t.reshape(2, -1, 3).transpose(1, 0, 2).reshape(-1, 3)
            verts.append(v)
            tris.append(t + nv)
            fids.append(np.full(t.shape[0], fid, np.int32))
            nv += v.shape[0]
            fid += 1
    return (np.concatenate(verts).astype(np.float32), np.concatenate(tris).astype(np.int32),
            np.concatenate(fids))


# --------------------------------------------------------------------------- C0

def tiny_box() -> Scene:
    """Closed 10x8x3 m room, 2 triangles per face with inward normals, concrete walls."""
    v, t, _ = box_faces((0, 0, 0), (10, 8, 3), (1, 1, 1), inward=True)
    xs = np.array([1.25, 3.75, 6.25, 8.75])
    ys = np.array([1.0, 3.0, 5.0, 7.0])
    gx, gy = np.meshgrid(xs, ys, indexing="ij")
    rx = np.stack([gx.ravel(), gy.ravel(), np.full(16, 1.5)], 1)
    return Scene(
        name="tiny_box", verts=v, tris=t, tri_material=np.zeros(t.shape[0], np.int32),
        eps_r=np.array([CONCRETE[0]], np.float32), sigma=np.array([CONCRETE[1]], np.float32),
        is_pec=np.zeros(1, np.uint8), tx=_f32([2.0, 2.0, 2.0]), rx=_f32(rx),
        n_rays=10_000, max_depth=2, freq_hz=3.5e9, f_center_hz=3.5e9,
        delta_f_hz=50e6 / 1024, n_sub=1024, seed=0)


# --------------------------------------------------------------------------- C1 / C4

def _place_footprints(rng, n_boxes, half_extent, size_lo, size_hi, gap, keep_out_xy, keep_out_r):
    boxes = []
    tries = 0
    while len(boxes) < n_boxes:
        tries += 1
        if tries > 200000:
            raise RuntimeError("box placement did not converge")
        sx, sy = rng.uniform(size_lo, size_hi, 2)
        cx = rng.uniform(-half_extent + sx / 2 + 1, half_extent - sx / 2 - 1)
        cy = rng.uniform(-half_extent + sy / 2 + 1, half_extent - sy / 2 - 1)
        x0, x1, y0, y1 = cx - sx / 2, cx + sx / 2, cy - sy / 2, cy + sy / 2
        kx, ky = keep_out_xy
        if x0 - keep_out_r <= kx <= x1 + keep_out_r and y0 - keep_out_r <= ky <= y1 + keep_out_r:
            continue
        ok = True
        for (a0, a1, b0, b1) in boxes:
            if x0 < a1 + gap and a0 < x1 + gap and y0 < b1 + gap and b0 < y1 + gap:
                ok = False
                break
        if ok:
            boxes.append((x0, x1, y0, y1))
    return boxes


def _city(rng, n_boxes, subdiv, name, n_rays, max_depth, rx, freq, fc, df, nsub, seed):
    half = 250.0
    mb = _MeshBuilder()
    gv, gt, _ = box_faces((-half, -half, -1.0), (half, half, 0.0), (1, 1, 1))
    # keep only the top face (z = 0, normal +z) of the slab as the ground plane
    keep = np.all(gv[gt][:, :, 2] == 0.0, axis=1)
    mb.add(gv, gt[keep], 3)
    boxes = _place_footprints(rng, n_boxes, half, 10.0, 30.0, 5.0, (0.0, 0.0), 5.0)
    heights = rng.uniform(10.0, 40.0, n_boxes)
    mats = rng.integers(0, 3, n_boxes)
    for (x0, x1, y0, y1), h, m in zip(boxes, heights, mats):
        v, t, _ = box_faces((x0, y0, 0.0), (x1, y1, h), (subdiv, subdiv, subdiv))
        mb.add(v, t, int(m))
    v, t, tm = mb.build()
    eps = np.array([CONCRETE[0], GLASS[0], 1.0, GROUND[0]], np.float32)
    sig = np.array([CONCRETE[1], GLASS[1], 0.0, GROUND[1]], np.float32)
    pec = np.array([0, 0, 1, 0], np.uint8)
    return Scene(name=name, verts=v, tris=t, tri_material=tm, eps_r=eps, sigma=sig, is_pec=pec,
                 tx=_f32([0.0, 0.0, 30.0]), rx=_f32(rx), n_rays=n_rays, max_depth=max_depth,
                 freq_hz=freq, f_center_hz=fc, delta_f_hz=df, n_sub=nsub, seed=seed)


def street_canyon(seed: int = 1) -> Scene:
    """64 boxes (footprints U(10,30) m, heights U(10,40) m) on a 500x500 m ground plane.

    Materials: 0 concrete, 1 glass, 2 metal (PEC), 3 ground.  Tx at (0,0,30) m, Rx on the
    centres of a 64x64 grid at 1.5 m height (receivers inside buildings are kept).
    """
    rng = np.random.default_rng(seed)
    c = -250.0 + (np.arange(64) + 0.5) * (500.0 / 64)
    gx, gy = np.meshgrid(c, c, indexing="ij")
    rx = np.stack([gx.ravel(), gy.ravel(), np.full(64 * 64, 1.5)], 1)
    return _city(rng, 64, 1, "street_canyon", 1_000_000, 3, rx, 3.5e9, 3.5e9, 50e6 / 1024, 1024, seed)


def city_batch(seed: int = 4, n_scenes: int = 16, total_rx: int = 65536, min_rx: int = 256,
               n_rays: int = 10_000_000, max_depth: int = 4) -> List[Scene]:
    """16 procedural cities of uneven size; triangle counts log-uniform in [1k, 50k]."""
    rng = np.random.default_rng(seed)
    w = rng.dirichlet(np.ones(n_scenes))
    extra = total_rx - n_scenes * min_rx
    counts = min_rx + np.floor(w * extra).astype(np.int64)
    counts[np.argmax(w)] += total_rx - counts.sum()
    scenes = []
    for s in range(n_scenes):
        t_target = math.exp(rng.uniform(math.log(1e3), math.log(5e4)))
        n_boxes = int(rng.integers(48, 97))
        sub = max(1, int(round(math.sqrt(t_target / (12.0 * n_boxes)))))
        r = int(counts[s])
        rxy = rng.uniform(-245.0, 245.0, (r, 2))
        rx = np.concatenate([rxy, np.full((r, 1), 1.5)], 1)
        scenes.append(_city(rng, n_boxes, sub, f"city_{s:02d}", n_rays, max_depth, rx,
                            1.272e9, 1.272e9, 50e6 / 256, 256, seed * 1000 + s))
    return scenes


# --------------------------------------------------------------------------- C2

def indoor_diff(seed: int = 2, n_rx: int = 1024) -> Scene:
    """20x15x4 m room (faces 8x8 quads) with 40 box obstacles (faces 3x3 quads).

    Materials 0 floor, 1 ceiling, 2 walls, 3..7 obstacles; hidden ground truth
    eps_r ~ U(2, 10), sigma ~ logU(1e-3, 1).  Rx follow a seeded random walk at 1.5 m.
    """
    rng = np.random.default_rng(seed)
    L = (20.0, 15.0, 4.0)
    mb = _MeshBuilder()
    v, t, fid = box_faces((0, 0, 0), L, (8, 8, 8), inward=True)
    # face ids: 0 x-lo, 1 x-hi, 2 y-lo, 3 y-hi, 4 z-lo (floor), 5 z-hi (ceiling)
    mats = np.where(fid == 4, 0, np.where(fid == 5, 1, 2)).astype(np.int32)
    mb.add_mats(v, t, mats)
    tx = np.array([2.0, 2.0, 3.0])
    boxes = []
    tries = 0
    while len(boxes) < 40:
        tries += 1
        if tries > 100000:
            raise RuntimeError("obstacle placement did not converge")
        s = rng.uniform(0.3, 2.0, 3)
        cx = rng.uniform(0.5 + s[0] / 2, L[0] - 0.5 - s[0] / 2)
        cy = rng.uniform(0.5 + s[1] / 2, L[1] - 0.5 - s[1] / 2)
        x0, x1, y0, y1 = cx - s[0] / 2, cx + s[0] / 2, cy - s[1] / 2, cy + s[1] / 2
        if x0 - 0.5 <= tx[0] <= x1 + 0.5 and y0 - 0.5 <= tx[1] <= y1 + 0.5:
            continue
        if any(x0 < b[1] + 0.2 and b[0] < x1 + 0.2 and y0 < b[3] + 0.2 and b[2] < y1 + 0.2 for b in boxes):
            continue
        boxes.append((x0, x1, y0, y1, s[2]))
    box_mats = rng.integers(3, 8, 40)
    for (x0, x1, y0, y1, h), m in zip(boxes, box_mats):
        v, t, _ = box_faces((x0, y0, 0.0), (x1, y1, h), (3, 3, 3))
        mb.add(v, t, int(m))
    v, t, tm = mb.build()
    eps = rng.uniform(2.0, 10.0, 8).astype(np.float32)
    sig = (10.0 ** rng.uniform(-3.0, 0.0, 8)).astype(np.float32)

    def blocked(p):
        return any(b[0] - 0.2 <= p[0] <= b[1] + 0.2 and b[2] - 0.2 <= p[1] <= b[3] + 0.2 for b in boxes)

    while True:
        p = np.array([rng.uniform(1, L[0] - 1), rng.uniform(1, L[1] - 1)])
        if not blocked(p):
            break
    heading = rng.uniform(0, 2 * np.pi)
    pts = []
    for _ in range(n_rx):
        pts.append(p.copy())
        for _attempt in range(200):
            heading += rng.normal(0.0, 0.3)
            q = p + 0.1 * np.array([np.cos(heading), np.sin(heading)])
            if q[0] < 0.5 or q[0] > L[0] - 0.5:
                heading = np.pi - heading
                continue
            if q[1] < 0.5 or q[1] > L[1] - 0.5:
                heading = -heading
                continue
            if blocked(q):
                heading = rng.uniform(0, 2 * np.pi)
                continue
            p = q
            break
    pts = np.array(pts)
    rx = np.concatenate([pts, np.full((n_rx, 1), 1.5)], 1)
    return Scene(name="indoor_diff", verts=v, tris=t, tri_material=tm, eps_r=eps, sigma=sig,
                 is_pec=np.zeros(8, np.uint8), tx=_f32(tx), rx=_f32(rx), n_rays=1_000_000,
                 max_depth=3, freq_hz=1.272e9, f_center_hz=1.272e9, delta_f_hz=50e6 / 1024,
                 n_sub=1024, seed=seed)


# --------------------------------------------------------------------------- C3

def _smooth_field(rng, pts, n_features=16, length=5.0):
    """Sigmoid of a sum of random Fourier features: a smooth seeded field in (0, 1)."""
    w = rng.normal(0.0, 2 * np.pi / length, (n_features, 3))
    w[:, 2] *= 0.3
    b = rng.uniform(0, 2 * np.pi, n_features)
    amp = rng.normal(0.0, 1.0, n_features) * (2.0 / math.sqrt(n_features))
    z = np.cos(pts @ w.T + b) @ amp
    return 1.0 / (1.0 + np.exp(-z))


def room_corridor(seed: int = 3, n_rx: int = 100_000, target_tris: int = 20_000) -> Scene:
    """A 24x12x3.5 m hall split by a partition wall into a room and a corridor.

    Faces are refined so that the mesh has about ``target_tris`` triangles.  Every
    triangle has its own material (per-triangle mode): ground truth
    eps_r = 2 + 8 s(c), sigma = 10^(-3 + 3 s'(c)) at the centroid c, with s, s'
    smooth random fields.
    """
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = 24.0, 12.0, 3.5
    part = (0.0, 6.0, 0.0, 16.0, 6.2, Lz)   # partition wall box
    area = 2 * (Lx * Ly + Lx * Lz + Ly * Lz)
    px, py, pz = part[3] - part[0], part[4] - part[1], part[5] - part[2]
    area += 2 * (px * py + px * pz + py * pz)
    h = math.sqrt(2 * area / target_tris)

    def nsub(a):
        return max(1, int(round(a / h)))

    mb = _MeshBuilder()
    v, t, fid = box_faces((0, 0, 0), (Lx, Ly, Lz), (nsub(Lx), nsub(Ly), nsub(Lz)), inward=True)
    # objects: 0 floor, 1 ceiling, 2 walls, 3 partition
    mb.add_mats(v, t, np.where(fid == 4, 0, np.where(fid == 5, 1, 2)))
    v, t, _ = box_faces(part[:3], part[3:], (nsub(px), nsub(py), nsub(pz)), skip_faces=((0, 0), (2, 0), (2, 1)))
    mb.add(v, t, 3)
    v, t, objects = mb.build()
    T = t.shape[0]
    cen = v[t].astype(np.float64).mean(axis=1)
    s1 = _smooth_field(rng, cen)
    s2 = _smooth_field(rng, cen)
    eps = (2.0 + 8.0 * s1).astype(np.float32)
    sig = (10.0 ** (-3.0 + 3.0 * s2)).astype(np.float32)
    tx = np.array([4.0, 3.0, 2.5])
    rxs = []
    while len(rxs) < n_rx:
        q = rng.uniform((0.3, 0.3), (Lx - 0.3, Ly - 0.3), (n_rx, 2))
        ok = ~((q[:, 0] <= part[3] + 0.3) & (q[:, 1] >= part[1] - 0.3) & (q[:, 1] <= part[4] + 0.3))
        rxs.extend(q[ok].tolist())
    q = np.array(rxs[:n_rx])
    rx = np.concatenate([q, np.full((n_rx, 1), 1.5)], 1)
    return Scene(name="room_corridor", verts=v, tris=t, tri_material=np.arange(T, dtype=np.int32),
                 eps_r=eps, sigma=sig, is_pec=np.zeros(T, np.uint8), tx=_f32(tx), rx=_f32(rx),
                 n_rays=1_000_000, max_depth=3, freq_hz=1.272e9, f_center_hz=1.272e9,
                 delta_f_hz=50e6 / 256, n_sub=256, per_triangle=True, seed=seed, tri_object=objects)


# --------------------------------------------------------------------------- tensors

def random_cfr_inputs(seed: int, n_rx: int, mean_paths: int, max_tau_s: float = 1.5e-6,
                      empty_every: int = 0):
    """Random per-path coefficients and delays grouped by receiver (uneven counts).

    Returns (a complex64 (P,), tau float64 (P,), rx_offsets int64 (R+1,)).  Every
    ``empty_every``-th receiver gets no paths when ``empty_every`` > 0.
    """
    rng = np.random.default_rng(seed)
    counts = rng.integers(max(1, mean_paths // 2), mean_paths * 3 // 2 + 2, n_rx)
    if empty_every:
        counts[::empty_every] = 0
    offs = np.zeros(n_rx + 1, np.int64)
    offs[1:] = np.cumsum(counts)
    P = int(offs[-1])
    mag = 10.0 ** rng.uniform(-5, -2, P)
    ph = rng.uniform(0, 2 * np.pi, P)
    a = (mag * np.exp(1j * ph)).astype(np.complex64)
    tau = rng.uniform(1e-9, max_tau_s, P)
    return a, tau, offs


def random_fields_inputs(seed: int, n_materials: int):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.5, 12.0, n_materials).astype(np.float32)
    sig = (10.0 ** rng.uniform(-3.0, 0.5, n_materials)).astype(np.float32)
    return eps, sig


def random_scattering(seed: int, n_materials: int) -> np.ndarray:
    """Seeded per-material diffuse-reflection parameters (M x 8 float32):
    [S, K_x, w_1, w_2, w_3, lambda_2, lambda_3, 0] with S ~ U(0.2, 0.7),
    K_x ~ U(0.05, 0.5), (w_1, w_2, w_3) ~ Dirichlet(2, 2, 2), lambda ~ U(2, 15)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n_materials, 8), np.float32)
    out[:, 0] = rng.uniform(0.2, 0.7, n_materials)
    out[:, 1] = rng.uniform(0.05, 0.5, n_materials)
    out[:, 2:5] = rng.dirichlet([2.0, 2.0, 2.0], n_materials)
    out[:, 5:7] = rng.uniform(2.0, 15.0, (n_materials, 2))
    return out


def ground_plane(half: float = 200.0, tx=(0.0, 0.0, 10.0), rx=((25.0, 5.0, 2.0),)) -> Scene:
    """One square ground plane (2 triangles, normal +z, material GROUND) of side
    2 * half centred at the origin, a transmitter and receivers above it."""
    v = np.array([[-half, -half, 0.0], [half, -half, 0.0], [half, half, 0.0], [-half, half, 0.0]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return Scene(name="ground_plane", verts=v, tris=t, tri_material=np.zeros(2, np.int32),
                 eps_r=np.array([GROUND[0]], np.float32), sigma=np.array([GROUND[1]], np.float32),
                 is_pec=np.zeros(1, np.uint8), tx=_f32(tx), rx=_f32(np.asarray(rx, np.float64)),
                 n_rays=100_000, max_depth=1, freq_hz=3.5e9, f_center_hz=3.5e9,
                 delta_f_hz=50e6 / 1024, n_sub=1024, seed=0)


def random_mlp_params(seed: int, d_in: int = 39, width: int = 128, depth: int = 3, d_out: int = 2):
    """He-initialised weights (float32) of the d_in -> width^depth -> d_out ReLU MLP."""
    rng = np.random.default_rng(seed)
    dims = [d_in] + [width] * depth + [d_out]
    Ws, bs = [], []
    for i in range(len(dims) - 1):
        Ws.append((rng.normal(0, math.sqrt(2.0 / dims[i]), (dims[i], dims[i + 1]))).astype(np.float32))
        bs.append((rng.normal(0, 0.01, dims[i + 1])).astype(np.float32))
    return Ws, bs
