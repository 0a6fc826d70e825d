"""Plain FP64 CPU oracle of the differentiable radio ray tracer (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product library never calls it; it shares no code
with the CUDA path.  The heavy geometric loops live in ``rt_oracle.cpp`` (FP64,
compiled by :func:`build`); this module wraps them with numpy and adds the parts
that are clearer in numpy: the loss (a plain definition), and the neural-material
MLP with BF16 rounding emulation.

Paper: Hoydis et al., "Learning Radio Environments by Differentiable Ray Tracing",
arXiv 2311.18558.  Each function cites the equation it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

C0 = 299792458.0
EPS0 = 8.8541878128e-12


def build(force: bool = False) -> str:
    """Compile the FP64 oracle (plain g++, OpenMP, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "orc_scene_create": (P, [P, i32, P, i32]),
            "orc_scene_free": (None, [P]),
            "orc_scene_diag": (f64, [P]),
            "orc_bvh_nodes": (i32, [P]),
            "orc_closest_hit": (None, [P, i64, P, P, f64, P, i32, P, P]),
            "orc_fibonacci": (None, [i64, P]),
            "orc_sbr_rays": (None, [P, P, i64, i32, i32, P]),
            "orc_candidates": (P, [P, P, i64, i32]),
            "orc_candidates_count": (i64, [P]),
            "orc_candidates_get": (None, [P, P]),
            "orc_candidates_free": (None, [P]),
            "orc_image_method": (P, [P, P, P, i32, P]),
            "orc_paths_count": (i64, [P]),
            "orc_paths_get": (None, [P, P, P, P, P, P]),
            "orc_paths_free": (None, [P]),
            "orc_diffuse_paths": (P, [P, P, P, i32, i64, i32]),
            "orc_paths_rays": (None, [P, P]),
            "orc_fields": (None, [P, i64, i32, P, P, P, P, P, P, P, i32, f64, f64, f64, i32, P]),
            "orc_fields_grad": (None, [P, i64, i32, P, P, P, P, P, P, P, i32, f64, f64, f64, P, P, P, P]),
            "orc_cfr": (None, [i64, P, P, P, i32, f64, f64, i32, P]),
            "orc_cfr_grad": (None, [i64, P, P, i32, f64, f64, i32, P, P]),
            "orc_fresnel": (None, [f64, f64, f64, f64, P]),
            "orc_permittivity": (None, [f64, f64, f64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------- geometry

class OracleScene:
    """A triangle scene held by the oracle (FP64 copies of the FP32 vertices)."""

    def __init__(self, scene):
        self.scene = scene
        lib = _load()
        self._v = _c(scene.verts, np.float32)
        self._t = _c(scene.tris, np.int32)
        self.h = lib.orc_scene_create(_p(self._v), self._v.shape[0], _p(self._t), self._t.shape[0])
        self.diag = lib.orc_scene_diag(self.h)
        self.tmin = 1e-6 * self.diag

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_scene_free(self.h)
            self.h = None

    def closest_hit(self, o, d, tmin=None, skip=None, use_bvh=True):
        o = _c(o, np.float64).reshape(-1, 3)
        d = _c(d, np.float64).reshape(-1, 3)
        n = o.shape[0]
        tri = np.empty(n, np.int32)
        t = np.empty(n, np.float64)
        sk = None if skip is None else _c(skip, np.int32)
        _load().orc_closest_hit(self.h, n, _p(o), _p(d), self.tmin if tmin is None else tmin,
                                None if sk is None else _p(sk), int(use_bvh), _p(tri), _p(t))
        return tri, t

    def sbr_rays(self, n_rays, depth, use_bvh=True, tx=None):
        tx = _c(self.scene.tx if tx is None else tx, np.float64)
        out = np.empty((n_rays, depth), np.int32)
        _load().orc_sbr_rays(self.h, _p(tx), n_rays, depth, int(use_bvh), _p(out))
        return out

    def candidates(self, n_rays=None, depth=None, tx=None):
        """Unique candidate sequences (K x depth, -1 padded), LoS first, by (length, lexicographic)."""
        lib = _load()
        n_rays = self.scene.n_rays if n_rays is None else n_rays
        depth = self.scene.max_depth if depth is None else depth
        tx = _c(self.scene.tx if tx is None else tx, np.float64)
        ch = lib.orc_candidates(self.h, _p(tx), n_rays, depth)
        K = lib.orc_candidates_count(ch)
        out = np.empty((K, depth), np.int32)
        lib.orc_candidates_get(ch, _p(out))
        lib.orc_candidates_free(ch)
        return out

    def trace(self, n_rays=None, depth=None, rx=None, tx=None, candidates=None):
        """SBR candidates + image method + visibility + duplicate rule (Sec. II-F).

        Returns a dict with per-path arrays grouped by receiver: rx (P,), depth (P,),
        seq (P, D), pts (P, D+2, 3) = Tx, s_1..s_q, Rx (zero padded), tau (P,),
        rx_offsets (R+1,), and the candidate list.
        """
        lib = _load()
        n_rays = self.scene.n_rays if n_rays is None else n_rays
        depth = self.scene.max_depth if depth is None else depth
        tx = _c(self.scene.tx if tx is None else tx, np.float64)
        rx = _c(self.scene.rx if rx is None else rx, np.float64).reshape(-1, 3)
        ch = lib.orc_candidates(self.h, _p(tx), n_rays, depth)
        K = lib.orc_candidates_count(ch)
        cands = np.empty((K, depth), np.int32)
        lib.orc_candidates_get(ch, _p(cands))
        if candidates is not None:
            lib.orc_candidates_free(ch)
            raise NotImplementedError
        ph = lib.orc_image_method(self.h, _p(tx), _p(rx), rx.shape[0], ch)
        lib.orc_candidates_free(ch)
        P = lib.orc_paths_count(ph)
        out = dict(rx=np.empty(P, np.int32), depth=np.empty(P, np.int32),
                   seq=np.empty((P, depth), np.int32), pts=np.empty((P, depth + 2, 3), np.float64),
                   tau=np.empty(P, np.float64))
        lib.orc_paths_get(ph, _p(out["rx"]), _p(out["depth"]), _p(out["seq"]), _p(out["pts"]), _p(out["tau"]))
        lib.orc_paths_free(ph)
        offs = np.zeros(rx.shape[0] + 1, np.int64)
        np.add.at(offs, out["rx"] + 1, 1)
        out["rx_offsets"] = np.cumsum(offs)
        out["candidates"] = cands
        out["max_depth"] = depth
        return out

    def diffuse_paths(self, n_rays, depth, rx=None, tx=None):
        """Diffuse paths by next-event estimation (Sec. II-F): for every hit s_j of every
        launch ray, the path Tx -> s_1..s_{j-1} (specular) -> s_j (diffuse) -> Rx when Rx
        is on the incidence side of t_j and sees s_j.  Same dict layout as :meth:`trace`
        plus ``ray`` (the launch ray of each path); ordered by (receiver, ray, j)."""
        lib = _load()
        tx = _c(self.scene.tx if tx is None else tx, np.float64)
        rx = _c(self.scene.rx if rx is None else rx, np.float64).reshape(-1, 3)
        ph = lib.orc_diffuse_paths(self.h, _p(tx), _p(rx), rx.shape[0], int(n_rays), int(depth))
        P = lib.orc_paths_count(ph)
        out = dict(rx=np.empty(P, np.int32), depth=np.empty(P, np.int32),
                   seq=np.empty((P, depth), np.int32), pts=np.empty((P, depth + 2, 3), np.float64),
                   tau=np.empty(P, np.float64), ray=np.empty(P, np.int32))
        lib.orc_paths_get(ph, _p(out["rx"]), _p(out["depth"]), _p(out["seq"]), _p(out["pts"]), _p(out["tau"]))
        lib.orc_paths_rays(ph, _p(out["ray"]))
        lib.orc_paths_free(ph)
        offs = np.zeros(rx.shape[0] + 1, np.int64)
        np.add.at(offs, out["rx"] + 1, 1)
        out["rx_offsets"] = np.cumsum(offs)
        out["max_depth"] = depth
        out["n_rays"] = int(n_rays)
        return out

    def fields(self, paths, eps_r=None, sigma=None, freq=None, gain_tx=1.0, gain_rx=1.0, ni_mode=0):
        """Path coefficients a_i (complex128) of Eq. cfr_cont for the given paths."""
        sc = self.scene
        eps_r = _c(sc.eps_r if eps_r is None else eps_r, np.float32)
        sigma = _c(sc.sigma if sigma is None else sigma, np.float32)
        freq = sc.freq_hz if freq is None else freq
        P = int(paths["depth"].shape[0])
        D = int(paths["seq"].shape[1])
        a = np.empty(2 * P, np.float64)
        dep, seq, pts = _c(paths["depth"], np.int32), _c(paths["seq"], np.int32), _c(paths["pts"], np.float64)
        tm, pec = _c(sc.tri_material, np.int32), _c(sc.is_pec, np.uint8)
        _load().orc_fields(self.h, P, D, _p(dep), _p(seq), _p(pts), _p(tm), _p(eps_r), _p(sigma), _p(pec),
                           int(sc.per_triangle), float(freq), float(gain_tx), float(gain_rx), int(ni_mode), _p(a))
        return a[0::2] + 1j * a[1::2]

    def fields_grad(self, paths, grad_a, eps_r=None, sigma=None, freq=None, gain_tx=1.0, gain_rx=1.0):
        """dL/d eps_r, dL/d sigma (per material or triangle) and dL/d (g_T, g_R) given dL/da."""
        sc = self.scene
        eps_r = _c(sc.eps_r if eps_r is None else eps_r, np.float32)
        sigma = _c(sc.sigma if sigma is None else sigma, np.float32)
        freq = sc.freq_hz if freq is None else freq
        P = int(paths["depth"].shape[0])
        D = int(paths["seq"].shape[1])
        ga = np.empty(2 * P, np.float64)
        ga[0::2] = np.real(grad_a)
        ga[1::2] = np.imag(grad_a)
        ge = np.zeros(eps_r.shape[0], np.float64)
        gs = np.zeros(eps_r.shape[0], np.float64)
        gg = np.zeros(2, np.float64)
        dep, seq, pts = _c(paths["depth"], np.int32), _c(paths["seq"], np.int32), _c(paths["pts"], np.float64)
        tm, pec = _c(sc.tri_material, np.int32), _c(sc.is_pec, np.uint8)
        _load().orc_fields_grad(self.h, P, D, _p(dep), _p(seq), _p(pts), _p(tm), _p(eps_r), _p(sigma), _p(pec),
                                int(sc.per_triangle), float(freq), float(gain_tx), float(gain_rx), _p(ga),
                                _p(ge), _p(gs), _p(gg))
        return ge, gs, gg


def fibonacci(n: int) -> np.ndarray:
    out = np.empty((n, 3), np.float32)
    _load().orc_fibonacci(n, _p(out))
    return out


def fresnel(eps_r, sigma, freq, cos_i):
    """(r_perp, r_par, d r_perp/d eta, d r_par/d eta) of Eq. fresnel-1/2."""
    out = np.empty(8, np.float64)
    _load().orc_fresnel(float(eps_r), float(sigma), float(freq), float(cos_i), _p(out))
    return complex(out[0], out[1]), complex(out[2], out[3]), complex(out[4], out[5]), complex(out[6], out[7])


def permittivity(eps_r, sigma, freq):
    out = np.empty(2, np.float64)
    _load().orc_permittivity(float(eps_r), float(sigma), float(freq), _p(out))
    return complex(out[0], out[1])


# ----------------------------------------------------------------------------- CFR and loss

def cfr(a, tau, rx_offsets, f_center, delta_f, n_sub):
    """H[r, n] = sum_i a_i exp(-j 2 pi (f_c + n df) tau_i), n = -N/2..N/2-1 (Sec. II-A)."""
    a = np.asarray(a, np.complex128)
    ai = np.empty(2 * a.shape[0], np.float64)
    ai[0::2], ai[1::2] = a.real, a.imag
    tau = _c(tau, np.float64)
    offs = _c(rx_offsets, np.int64)
    R = offs.shape[0] - 1
    H = np.empty(2 * R * n_sub, np.float64)
    _load().orc_cfr(a.shape[0], _p(ai), _p(tau), _p(offs), R, float(f_center), float(delta_f), int(n_sub), _p(H))
    return (H[0::2] + 1j * H[1::2]).reshape(R, n_sub)


def cfr_grad(tau, rx_offsets, f_center, delta_f, n_sub, grad_H):
    """g_a[i] = sum_n g_H[r(i), n] conj(exp(-j 2 pi f_n tau_i)) (adjoint of :func:`cfr`)."""
    tau = _c(tau, np.float64)
    offs = _c(rx_offsets, np.int64)
    R = offs.shape[0] - 1
    gH = np.asarray(grad_H, np.complex128).reshape(R, n_sub)
    gi = np.empty(2 * R * n_sub, np.float64)
    gi[0::2], gi[1::2] = gH.real.ravel(), gH.imag.ravel()
    ga = np.empty(2 * tau.shape[0], np.float64)
    _load().orc_cfr_grad(tau.shape[0], _p(tau), _p(offs), R, float(f_center), float(delta_f), int(n_sub), _p(gi), _p(ga))
    return ga[0::2] + 1j * ga[1::2]


def power_weights(target_power):
    """w_r = 1 / mean_n P*[r, n] (0 for a receiver without power)."""
    m = np.asarray(target_power, np.float64).mean(axis=1)
    return np.where(m > 0, 1.0 / np.where(m > 0, m, 1.0), 0.0)


def power_mse(H, target_power, weights):
    """MSE on CFR power: L = 1/(R N) sum_{r,n} (w_r (|H[r,n]|^2 - P*[r,n]))^2.

    Returns (L, g_H) with g_H = dL/dRe H + j dL/dIm H = 4 w_r^2 (|H|^2 - P*) H / (R N).
    """
    H = np.asarray(H, np.complex128)
    R, N = H.shape
    w = np.asarray(weights, np.float64)[:, None]
    e = np.abs(H) ** 2 - np.asarray(target_power, np.float64)
    L = float(np.sum((w * e) ** 2) / (R * N))
    gH = 4.0 * w ** 2 * e * H / (R * N)
    return L, gH
