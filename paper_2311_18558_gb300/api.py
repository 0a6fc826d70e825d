"""Thin Python binding of librt103: argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch provides device
memory and the current stream.  Names follow include/rt103.h.
"""
from __future__ import annotations

import ctypes
import sys
from typing import Optional

import numpy as np
import torch

from ._lib import RtError, load

_c = ctypes


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else _c.c_void_p(t.data_ptr())


class Context:
    """A library context on one CUDA device (rt_create).  Each call is ordered on
    the torch stream that is current when the call is made."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = int(device)
        h = _c.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.rt_create(self.device, _c.c_void_p(torch.cuda.current_stream().cuda_stream), _c.byref(h))
        if st != 0:
            raise RtError(st, "rt_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.rt_destroy(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the process releases everything; calling into CUDA
        # while Python and the runtime tear down is not safe
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        self.lib.rt_set_stream(self.h, _c.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def check(self, st: int, what: str):
        if st != 0:
            msg = self.lib.rt_last_error(self.h).decode()
            raise RtError(st, f"{what}: {msg}")

    def set_profiling(self, flags: int):
        """Instrumentation: bit 0 trace stage timing, bit 1 traversal counters."""
        self._stream()
        self.check(self.lib.rt_set_profiling(self.h, int(flags)), "rt_set_profiling")

    def profile(self):
        """(kernel launches so far, trace stage ms [8], counters [8])."""
        n = _c.c_int64()
        ms = (_c.c_double * 8)()
        cnt = (_c.c_int64 * 8)()
        self._stream()
        self.check(self.lib.rt_profile_read(self.h, _c.byref(n), ms, cnt), "rt_profile_read")
        return int(n.value), list(ms), list(cnt)

    def status_word(self) -> int:
        """Synchronise and return (and clear) the sticky device status word."""
        v = _c.c_int32(0)
        self._stream()
        self.check(self.lib.rt_status_word(self.h, _c.byref(v)), "rt_status_word")
        return int(v.value)


class Scene:
    """A triangle mesh uploaded to the device with its BVH (rt_scene_upload)."""

    def __init__(self, ctx: Context, verts, tris, tri_material, is_pec):
        self.ctx = ctx
        self._v = np.ascontiguousarray(verts, np.float32)
        self._t = np.ascontiguousarray(tris, np.int32)
        self._m = np.ascontiguousarray(tri_material, np.int32)
        self._p = np.ascontiguousarray(is_pec, np.uint8)
        h = _c.c_void_p()
        ctx._stream()
        ctx.check(ctx.lib.rt_scene_upload(ctx.h, self._v.ctypes.data_as(_c.c_void_p), self._v.shape[0],
                                          self._t.ctypes.data_as(_c.c_void_p), self._t.shape[0],
                                          self._m.ctypes.data_as(_c.c_void_p), self._p.shape[0],
                                          self._p.ctypes.data_as(_c.c_void_p), _c.byref(h)), "rt_scene_upload")
        self.h = h
        nt, nn, dg = _c.c_int32(), _c.c_int32(), _c.c_double()
        ctx.lib.rt_scene_info(h, _c.byref(nt), _c.byref(nn), _c.byref(dg))
        self.n_tris, self.n_nodes, self.diag = nt.value, nn.value, dg.value
        self.n_materials = int(self._p.shape[0])

    @classmethod
    def from_synthetic(cls, ctx: Context, sc) -> "Scene":
        return cls(ctx, sc.verts, sc.tris, sc.tri_material, sc.is_pec)

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.rt_scene_free(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the process releases everything; calling into CUDA
        # while Python and the runtime tear down is not safe
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class _PathsHandle:
    """Owns one library paths object; frees it when the last reference (the Paths
    object or a device view of its arrays) goes, or on close()."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def close(self):
        if self.h:
            self.ctx.lib.rt_paths_free(self.h)
            self.h = None

    def __del__(self):
        # at interpreter exit the process releases everything; calling into CUDA
        # while Python and the runtime tear down is not safe
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class _DeviceView:
    """A library-owned device array exposed through __cuda_array_interface__ (no
    copy); it keeps the owning paths handle alive.  Read it only."""

    def __init__(self, ptr: int, n: int, typestr: str, owner: _PathsHandle):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}
        self._owner = owner


class Paths:
    """Traced (or imported) paths with their frozen geometry records.  ``rx_offsets``
    and ``tau`` are read-only views of the library's arrays (valid while the object
    is open)."""

    def __init__(self, ctx: Context, scene: Scene, h, n_rx: int, max_depth: int):
        self.ctx, self.scene, self.h = ctx, scene, h
        self._handle = _PathsHandle(ctx, h)
        self.n_rx, self.max_depth = int(n_rx), int(max_depth)
        p, k = _c.c_int64(), _c.c_int64()
        ctx.lib.rt_paths_count(h, _c.byref(p), _c.byref(k))
        self.n_paths, self.n_candidates = int(p.value), int(k.value)
        off, tau = _c.c_void_p(), _c.c_void_p()
        ctx.check(ctx.lib.rt_paths_device_views(h, _c.byref(off), _c.byref(tau)), "rt_paths_device_views")
        dev = torch.device("cuda", ctx.device)
        self.rx_offsets = torch.as_tensor(_DeviceView(off.value, self.n_rx + 1, "<i8", self._handle), device=dev)
        self.tau = torch.as_tensor(_DeviceView(tau.value, self.n_paths, "<f8", self._handle), device=dev)

    def resolve(self):
        """Waits for a trace that returned without waiting (rt_set_trace_async) and
        fixes n_paths to the paths it found (rt_paths_resolve); a no-op otherwise."""
        self.ctx._stream()
        self.ctx.check(self.ctx.lib.rt_paths_resolve(self.h), "rt_paths_resolve")
        p, k = _c.c_int64(), _c.c_int64()
        self.ctx.lib.rt_paths_count(self.h, _c.byref(p), _c.byref(k))
        if int(p.value) != self.n_paths:
            self.n_paths, self.n_candidates = int(p.value), int(k.value)
            self.tau = self.tau[: self.n_paths]
        return self

    def export(self):
        """Triangle sequences, depths, receivers, delays and points as device tensors."""
        self.resolve()
        dev = torch.device("cuda", self.ctx.device)
        P, D = self.n_paths, self.max_depth
        out = dict(seq=torch.empty((P, D), dtype=torch.int32, device=dev),
                   depth=torch.empty(P, dtype=torch.int32, device=dev),
                   rx=torch.empty(P, dtype=torch.int32, device=dev),
                   tau=torch.empty(P, dtype=torch.float64, device=dev),
                   pts=torch.empty((P, D + 2, 3), dtype=torch.float64, device=dev))
        self.ctx._stream()
        if P:
            self.ctx.check(self.ctx.lib.rt_paths_export(self.h, _ptr(out["seq"]), _ptr(out["depth"]), _ptr(out["rx"]),
                                                        _ptr(out["tau"]), _ptr(out["pts"])), "rt_paths_export")
        out["rx_offsets"] = self.rx_offsets
        return out

    def candidates(self) -> torch.Tensor:
        dev = torch.device("cuda", self.ctx.device)
        out = torch.empty((max(self.n_candidates, 1), self.max_depth), dtype=torch.int32, device=dev)
        self.ctx._stream()
        self.ctx.check(self.ctx.lib.rt_paths_candidates(self.h, _ptr(out)), "rt_paths_candidates")
        return out[: self.n_candidates]

    def close(self):
        """Frees the library's paths now (the rx_offsets and tau views die with them)."""
        if getattr(self, "_handle", None) is not None:
            self._handle.close()
        self.h = None


def trace_paths(ctx: Context, scene: Scene, tx, rx: torch.Tensor, n_rays: int, max_depth: int) -> Paths:
    """Specular path tracing (rt_trace_paths); rx is a CUDA float64 (R, 3) tensor."""
    rx = rx.to(device=torch.device("cuda", ctx.device), dtype=torch.float64).contiguous()
    txa = (_c.c_double * 3)(*[float(v) for v in tx])
    h = _c.c_void_p()
    ctx._stream()
    ctx.check(ctx.lib.rt_trace_paths(ctx.h, scene.h, txa, _ptr(rx), rx.shape[0], int(n_rays), int(max_depth),
                                     _c.byref(h)), "rt_trace_paths")
    return Paths(ctx, scene, h, rx.shape[0], max_depth)


def import_paths(ctx: Context, scene: Scene, rx_idx, depth, seq, pts, n_rx: int) -> Paths:
    """Paths given by their receivers, depths, triangle sequences and points (rt_paths_import)."""
    dev = torch.device("cuda", ctx.device)
    rx_idx = torch.as_tensor(rx_idx, dtype=torch.int32).to(dev).contiguous()
    depth = torch.as_tensor(depth, dtype=torch.int32).to(dev).contiguous()
    seq = torch.as_tensor(seq, dtype=torch.int32).to(dev).contiguous()
    pts = torch.as_tensor(pts, dtype=torch.float64).to(dev).contiguous()
    D = int(seq.shape[1])
    h = _c.c_void_p()
    ctx._stream()
    ctx.check(ctx.lib.rt_paths_import(ctx.h, scene.h, int(seq.shape[0]), D, int(n_rx), _ptr(rx_idx), _ptr(depth),
                                      _ptr(seq), _ptr(pts), _c.byref(h)), "rt_paths_import")
    return Paths(ctx, scene, h, n_rx, D)


def eval_fields(ctx: Context, paths: Paths, eps_r: torch.Tensor, sigma: torch.Tensor, freq_hz: float,
                gain_tx: float = 1.0, gain_rx: float = 1.0, per_triangle: bool = False,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Path coefficients a_i (complex64) of Eq. cfr_cont (rt_eval_fields)."""
    dev = torch.device("cuda", ctx.device)
    a = out if out is not None else torch.empty(paths.n_paths, dtype=torch.complex64, device=dev)
    ctx._stream()
    ctx.check(ctx.lib.rt_eval_fields(ctx.h, paths.h, _ptr(eps_r), _ptr(sigma), int(per_triangle), float(freq_hz),
                                     float(gain_tx), float(gain_rx), _ptr(a), None), "rt_eval_fields")
    return a


def eval_fields_backward(ctx: Context, paths: Paths, eps_r, sigma, freq_hz, grad_a, grad_eps=None, grad_sigma=None,
                         grad_gain=None, gain_tx=1.0, gain_rx=1.0, per_triangle=False):
    """Accumulates dL/deps_r, dL/dsigma, dL/d(g_T, g_R) given dL/da (rt_eval_fields_backward)."""
    dev = torch.device("cuda", ctx.device)
    if grad_eps is None:
        grad_eps = torch.zeros_like(eps_r, dtype=torch.float32)
    if grad_sigma is None:
        grad_sigma = torch.zeros_like(sigma, dtype=torch.float32)
    if grad_gain is None:
        grad_gain = torch.zeros(2, dtype=torch.float32, device=dev)
    ctx._stream()
    ctx.check(ctx.lib.rt_eval_fields_backward(ctx.h, paths.h, _ptr(eps_r), _ptr(sigma), int(per_triangle),
                                              float(freq_hz), float(gain_tx), float(gain_rx),
                                              _ptr(grad_a.contiguous()), _ptr(grad_eps), _ptr(grad_sigma),
                                              _ptr(grad_gain)), "rt_eval_fields_backward")
    return grad_eps, grad_sigma, grad_gain


def cfr(ctx: Context, rx_offsets: torch.Tensor, a: torch.Tensor, tau: torch.Tensor, f_center_hz: float,
        delta_f_hz: float, n_sub: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """H[r, n] of Sec. II-A (rt_cfr); complex64 (R, N), column n + N/2."""
    R = rx_offsets.shape[0] - 1
    H = out if out is not None else torch.empty((R, n_sub), dtype=torch.complex64, device=a.device)
    ctx._stream()
    ctx.check(ctx.lib.rt_cfr(ctx.h, _ptr(rx_offsets), R, _ptr(a), _ptr(tau), float(f_center_hz), float(delta_f_hz),
                             int(n_sub), _ptr(H)), "rt_cfr")
    return H


def cfr_backward(ctx: Context, rx_offsets, tau, f_center_hz, delta_f_hz, n_sub, grad_H,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    R = rx_offsets.shape[0] - 1
    ga = out if out is not None else torch.empty(tau.shape[0], dtype=torch.complex64, device=tau.device)
    ctx._stream()
    ctx.check(ctx.lib.rt_cfr_backward(ctx.h, _ptr(rx_offsets), R, _ptr(tau), float(f_center_hz), float(delta_f_hz),
                                      int(n_sub), _ptr(grad_H.contiguous()), _ptr(ga)), "rt_cfr_backward")
    return ga


def cfr_power_mse_fused(ctx: Context, rx_offsets, a, tau, f_center_hz, delta_f_hz, n_sub, target_power, rx_weight,
                        loss=None, grad_a=None, H=None):
    """CFR + power MSE + CFR adjoint in one launch (rt_cfr_power_mse_fused)."""
    R = rx_offsets.shape[0] - 1
    loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=a.device)
    grad_a = grad_a if grad_a is not None else torch.empty_like(a)
    ctx._stream()
    ctx.check(ctx.lib.rt_cfr_power_mse_fused(ctx.h, _ptr(rx_offsets), R, _ptr(a), _ptr(tau), float(f_center_hz),
                                             float(delta_f_hz), int(n_sub), _ptr(target_power), _ptr(rx_weight),
                                             _ptr(loss), _ptr(grad_a), _ptr(H)), "rt_cfr_power_mse_fused")
    return loss, grad_a, H


# ----------------------------------------------------------------------------- antenna patterns

def _lobes(pat):
    return 0 if pat is None else (int(pat.shape[0]) - 1) // 5


def antenna_apply(ctx: Context, paths: Paths, a: torch.Tensor, tx_pattern=None, rx_pattern=None, out=None):
    """a sqrt(G_T G_R) with mixture-of-lobes patterns (rt_antenna_apply); returns (a_out, G_T, G_R)."""
    P = paths.n_paths
    dev = a.device
    a_out = out if out is not None else torch.empty_like(a)
    gt = torch.empty(max(P, 1), dtype=torch.float32, device=dev)[:P] if tx_pattern is not None else None
    gr = torch.empty(max(P, 1), dtype=torch.float32, device=dev)[:P] if rx_pattern is not None else None
    ctx._stream()
    ctx.check(ctx.lib.rt_antenna_apply(ctx.h, paths.h, _ptr(tx_pattern), _lobes(tx_pattern), _ptr(rx_pattern),
                                       _lobes(rx_pattern), _ptr(a.contiguous()), _ptr(a_out), _ptr(gt), _ptr(gr)),
              "rt_antenna_apply")
    return a_out, gt, gr


def antenna_apply_backward(ctx: Context, paths: Paths, a_out, gt, gr, grad_out, tx_pattern=None, rx_pattern=None):
    """Adjoint of antenna_apply: (dL/da, dL/d tx pattern, dL/d rx pattern)."""
    grad_a = torch.empty_like(a_out)
    g_tx = torch.zeros_like(tx_pattern) if tx_pattern is not None else None
    g_rx = torch.zeros_like(rx_pattern) if rx_pattern is not None else None
    ctx._stream()
    ctx.check(ctx.lib.rt_antenna_apply_backward(ctx.h, paths.h, _ptr(tx_pattern), _lobes(tx_pattern),
                                                _ptr(rx_pattern), _lobes(rx_pattern), _ptr(a_out), _ptr(gt), _ptr(gr),
                                                _ptr(grad_out.contiguous()), _ptr(grad_a), _ptr(g_tx), _ptr(g_rx)),
              "rt_antenna_apply_backward")
    return grad_a, g_tx, g_rx


# ----------------------------------------------------------------------------- diffuse reflection

def trace_diffuse(ctx: Context, scene: Scene, tx, rx: torch.Tensor, n_rays: int, max_depth: int) -> Paths:
    """Diffuse paths by next-event estimation from every SBR hit (rt_trace_diffuse)."""
    rx = rx.to(device=torch.device("cuda", ctx.device), dtype=torch.float64).contiguous()
    txa = (_c.c_double * 3)(*[float(v) for v in tx])
    h = _c.c_void_p()
    ctx._stream()
    ctx.check(ctx.lib.rt_trace_diffuse(ctx.h, scene.h, txa, _ptr(rx), rx.shape[0], int(n_rays), int(max_depth),
                                       _c.byref(h)), "rt_trace_diffuse")
    return Paths(ctx, scene, h, rx.shape[0], max_depth)


def eval_fields_diffuse(ctx: Context, paths: Paths, eps_r, sigma, scat, freq_hz: float, gain_tx: float = 1.0,
                        gain_rx: float = 1.0, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Coefficients of diffuse paths (rt_eval_fields_diffuse); scat is (M, 8) float32."""
    dev = torch.device("cuda", ctx.device)
    a = out if out is not None else torch.empty(paths.n_paths, dtype=torch.complex64, device=dev)
    ctx._stream()
    ctx.check(ctx.lib.rt_eval_fields_diffuse(ctx.h, paths.h, _ptr(eps_r), _ptr(sigma), _ptr(scat), float(freq_hz),
                                             float(gain_tx), float(gain_rx), _ptr(a), None), "rt_eval_fields_diffuse")
    return a


def eval_fields_diffuse_backward(ctx: Context, paths: Paths, eps_r, sigma, scat, freq_hz, grad_a, grad_eps=None,
                                 grad_sigma=None, grad_scat=None, gain_tx=1.0, gain_rx=1.0):
    """Accumulates dL/deps_r, dL/dsigma and dL/dscat given dL/da (rt_eval_fields_diffuse_backward)."""
    grad_eps = torch.zeros_like(eps_r, dtype=torch.float32) if grad_eps is None else grad_eps
    grad_sigma = torch.zeros_like(sigma, dtype=torch.float32) if grad_sigma is None else grad_sigma
    grad_scat = torch.zeros_like(scat, dtype=torch.float32) if grad_scat is None else grad_scat
    ctx._stream()
    ctx.check(ctx.lib.rt_eval_fields_diffuse_backward(ctx.h, paths.h, _ptr(eps_r), _ptr(sigma), _ptr(scat),
                                                      float(freq_hz), float(gain_tx), float(gain_rx),
                                                      _ptr(grad_a.contiguous()), _ptr(grad_eps), _ptr(grad_sigma),
                                                      _ptr(grad_scat)), "rt_eval_fields_diffuse_backward")
    return grad_eps, grad_sigma, grad_scat


def scene_wedges(ctx: Context, scene: Scene):
    """Wedges of the scene's mesh (rt_scene_wedges): faces (W, 2) int32 and n (W,) float64."""
    n = _c.c_int32()
    ctx._stream()
    ctx.check(ctx.lib.rt_scene_wedges(ctx.h, scene.h, _c.byref(n), None, None), "rt_scene_wedges")
    faces = np.zeros((max(n.value, 1), 2), np.int32)
    nn = np.zeros(max(n.value, 1), np.float64)
    ctx.check(ctx.lib.rt_scene_wedges(ctx.h, scene.h, _c.byref(n), faces.ctypes.data_as(_c.c_void_p),
                                      nn.ctypes.data_as(_c.c_void_p)), "rt_scene_wedges")
    return faces[: n.value], nn[: n.value]


def trace_diffraction(ctx: Context, scene: Scene, specular: Paths, tx, rx: torch.Tensor) -> Paths:
    """First-order diffraction paths Tx -> edge -> Rx (rt_trace_diffraction); the candidate
    wedges come from the first hits of `specular`, a trace of the same scene and Tx."""
    rx = rx.to(device=torch.device("cuda", ctx.device), dtype=torch.float64).contiguous()
    txa = (_c.c_double * 3)(*[float(v) for v in tx])
    h = _c.c_void_p()
    ctx._stream()
    ctx.check(ctx.lib.rt_trace_diffraction(ctx.h, scene.h, specular.h, txa, _ptr(rx), rx.shape[0], _c.byref(h)),
              "rt_trace_diffraction")
    return Paths(ctx, scene, h, rx.shape[0], 2)


def eval_fields_diffraction(ctx: Context, paths: Paths, eps_r, sigma, freq_hz: float, gain_tx: float = 1.0,
                            gain_rx: float = 1.0, per_triangle: bool = False,
                            out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Coefficients of diffraction paths (rt_eval_fields_diffraction)."""
    dev = torch.device("cuda", ctx.device)
    a = out if out is not None else torch.empty(paths.n_paths, dtype=torch.complex64, device=dev)
    ctx._stream()
    ctx.check(ctx.lib.rt_eval_fields_diffraction(ctx.h, paths.h, _ptr(eps_r), _ptr(sigma), int(per_triangle),
                                                 float(freq_hz), float(gain_tx), float(gain_rx), _ptr(a), None),
              "rt_eval_fields_diffraction")
    return a


def eval_fields_diffraction_backward(ctx: Context, paths: Paths, eps_r, sigma, freq_hz, grad_a, grad_eps=None,
                                     grad_sigma=None, grad_gain=None, gain_tx=1.0, gain_rx=1.0,
                                     per_triangle: bool = False):
    """Accumulates dL/deps_r, dL/dsigma and dL/d(g_T, g_R) given dL/da
    (rt_eval_fields_diffraction_backward)."""
    grad_eps = torch.zeros_like(eps_r, dtype=torch.float32) if grad_eps is None else grad_eps
    grad_sigma = torch.zeros_like(sigma, dtype=torch.float32) if grad_sigma is None else grad_sigma
    grad_gain = torch.zeros(2, dtype=torch.float32, device=eps_r.device) if grad_gain is None else grad_gain
    ctx._stream()
    ctx.check(ctx.lib.rt_eval_fields_diffraction_backward(ctx.h, paths.h, _ptr(eps_r), _ptr(sigma), int(per_triangle),
                                                          float(freq_hz), float(gain_tx), float(gain_rx),
                                                          _ptr(grad_a.contiguous()), _ptr(grad_eps),
                                                          _ptr(grad_sigma), _ptr(grad_gain)),
              "rt_eval_fields_diffraction_backward")
    return grad_eps, grad_sigma, grad_gain


def set_diffuse_phases(ctx: Context, paths: Paths, chi=None):
    """Attaches per-path random phases (n_paths x 2 float32, radians) of Eq.
    scattered_field to diffuse paths, or clears them (rt_set_diffuse_phases).  The
    tensor is kept referenced by the paths object."""
    if chi is not None:
        chi = chi.to(device=torch.device("cuda", ctx.device), dtype=torch.float32).contiguous()
        if chi.shape != (paths.n_paths, 2):
            raise ValueError("chi must have shape (n_paths, 2)")
    ctx.check(ctx.lib.rt_set_diffuse_phases(ctx.h, paths.h, _ptr(chi)), "rt_set_diffuse_phases")
    paths.chi = chi


def specular_reduction(ctx: Context, paths: Paths, scat, a, out=None):
    """a prod_b sqrt(1 - S_b^2) over the bounces of each specular path (rt_specular_reduction)."""
    out = out if out is not None else torch.empty_like(a)
    ctx._stream()
    ctx.check(ctx.lib.rt_specular_reduction(ctx.h, paths.h, _ptr(scat), _ptr(a.contiguous()), _ptr(out)),
              "rt_specular_reduction")
    return out


def specular_reduction_backward(ctx: Context, paths: Paths, scat, a_out, grad_out, grad_scat=None):
    """Adjoint of specular_reduction: (dL/da, dL/dscat accumulated into grad_scat)."""
    grad_a = torch.empty_like(grad_out)
    grad_scat = torch.zeros_like(scat, dtype=torch.float32) if grad_scat is None else grad_scat
    ctx._stream()
    ctx.check(ctx.lib.rt_specular_reduction_backward(ctx.h, paths.h, _ptr(scat), _ptr(a_out),
                                                     _ptr(grad_out.contiguous()), _ptr(grad_a), _ptr(grad_scat)),
              "rt_specular_reduction_backward")
    return grad_a, grad_scat


def rx_merge(ctx: Context, off1, off2, x1, x2, off_out=None):
    """Per-receiver concatenation [x1 of r | x2 of r] (rt_rx_merge); 8-byte dtypes.  Returns (x, offsets)."""
    if x1.element_size() != 8 or x2.dtype != x1.dtype:
        raise ValueError("rx_merge takes two tensors of one 8-byte dtype (complex64 or float64)")
    R = off1.shape[0] - 1
    out = torch.empty(x1.shape[0] + x2.shape[0], dtype=x1.dtype, device=x1.device)
    off_out = off_out if off_out is not None else torch.empty(R + 1, dtype=torch.int64, device=x1.device)
    ctx._stream()
    ctx.check(ctx.lib.rt_rx_merge(ctx.h, R, _ptr(off1), _ptr(off2), _ptr(x1.contiguous()), _ptr(x2.contiguous()),
                                  _ptr(out), _ptr(off_out)), "rt_rx_merge")
    return out, off_out


def rx_split(ctx: Context, off1, off2, x, n1=None, n2=None):
    """Adjoint of rx_merge: the two per-receiver parts of x (rt_rx_split); n1, n2 are
    the part sizes (read from the offsets when not given)."""
    if x.element_size() != 8:
        raise ValueError("rx_split takes an 8-byte dtype (complex64 or float64)")
    n1 = int(off1[-1].item()) if n1 is None else int(n1)
    n2 = int(off2[-1].item()) if n2 is None else int(n2)
    d1 = torch.empty(n1, dtype=x.dtype, device=x.device)
    d2 = torch.empty(n2, dtype=x.dtype, device=x.device)
    R = off1.shape[0] - 1
    ctx._stream()
    ctx.check(ctx.lib.rt_rx_split(ctx.h, R, _ptr(off1), _ptr(off2), _ptr(x.contiguous()), _ptr(d1), _ptr(d2)),
              "rt_rx_split")
    return d1, d2


# ----------------------------------------------------------------------------- CIR, loss and metrics

def cir(ctx: Context, H: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """CIR by N-point IDFT of every row of H (rt_cir); columns l + N/2."""
    H = H.contiguous()
    h = out if out is not None else torch.empty_like(H)
    ctx._stream()
    ctx.check(ctx.lib.rt_cir(ctx.h, _ptr(H), int(H.shape[0]), int(H.shape[1]), _ptr(h)), "rt_cir")
    return h


def cir_stats(ctx: Context, H: torch.Tensor, delta_f_hz: float):
    """Channel gain P and RMS delay spread tau_RMS [s] per receiver (rt_cir_stats)."""
    H = H.contiguous()
    R = int(H.shape[0])
    P = torch.empty(R, dtype=torch.float32, device=H.device)
    t = torch.empty(R, dtype=torch.float32, device=H.device)
    ctx._stream()
    ctx.check(ctx.lib.rt_cir_stats(ctx.h, _ptr(H), R, int(H.shape[1]), float(delta_f_hz), _ptr(P), _ptr(t)),
              "rt_cir_stats")
    return P, t


def power_scale_ema(ctx: Context, P_meas: torch.Tensor, P_pred: torch.Tensor, decay: float, state: torch.Tensor):
    """Moving-average power scale of the measurements (rt_power_scale_ema); state = {alpha, initialised}."""
    ctx._stream()
    ctx.check(ctx.lib.rt_power_scale_ema(ctx.h, _ptr(P_meas.contiguous()), _ptr(P_pred.contiguous()),
                                         int(P_meas.shape[0]), float(decay), _ptr(state)), "rt_power_scale_ema")
    return state


def delay_spread_power_loss(ctx: Context, H: torch.Tensor, delta_f_hz: float, P_meas: torch.Tensor,
                            tau_meas: torch.Tensor, alpha_state: Optional[torch.Tensor] = None, loss=None,
                            grad_H=None, P_pred=None, tau_pred=None):
    """Eq. loss averaged over the receivers and dL/dH (rt_delay_spread_power_loss)."""
    H = H.contiguous()
    R = int(H.shape[0])
    loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=H.device)
    grad_H = grad_H if grad_H is not None else torch.empty_like(H)
    ctx._stream()
    ctx.check(ctx.lib.rt_delay_spread_power_loss(ctx.h, _ptr(H), R, int(H.shape[1]), float(delta_f_hz),
                                                 _ptr(P_meas.contiguous()), _ptr(tau_meas.contiguous()),
                                                 _ptr(alpha_state), _ptr(loss), _ptr(grad_H), _ptr(P_pred),
                                                 _ptr(tau_pred)), "rt_delay_spread_power_loss")
    return loss, grad_H


def cir_metrics(ctx: Context, P_meas, tau_meas, P_pred, tau_pred, alpha_state=None):
    """ALE [dB] and RAE per receiver (rt_cir_metrics)."""
    n = int(P_meas.shape[0])
    ale = torch.empty(n, dtype=torch.float32, device=P_meas.device)
    rae = torch.empty(n, dtype=torch.float32, device=P_meas.device)
    ctx._stream()
    ctx.check(ctx.lib.rt_cir_metrics(ctx.h, _ptr(P_meas.contiguous()), _ptr(tau_meas.contiguous()),
                                     _ptr(P_pred.contiguous()), _ptr(tau_pred.contiguous()), n, _ptr(alpha_state),
                                     _ptr(ale), _ptr(rae)), "rt_cir_metrics")
    return ale, rae


# ----------------------------------------------------------------------------- neural materials

MLP_IN, MLP_IN_PAD, MLP_WIDTH, MLP_OUT = 39, 40, 128, 2
MLP_NW = MLP_IN_PAD * MLP_WIDTH + 2 * MLP_WIDTH * MLP_WIDTH + MLP_WIDTH * MLP_OUT   # 38144
MLP_NB = 3 * MLP_WIDTH + MLP_OUT                                                    # 386
MLP_ACT = MLP_IN_PAD + 3 * MLP_WIDTH                                                # 424


def pack_mlp(Ws, bs, device="cuda"):
    """Packs [W1 (39x128), W2, W3 (128x128), W4 (128x2)] and biases into the flat
    FP32 layout of rt_mlp_forward (W1 padded with a zero row to 40 x 128)."""
    W1 = np.zeros((MLP_IN_PAD, MLP_WIDTH), np.float32)
    W1[:MLP_IN] = Ws[0]
    w = np.concatenate([W1.ravel()] + [np.asarray(W, np.float32).ravel() for W in Ws[1:]])
    b = np.concatenate([np.asarray(x, np.float32).ravel() for x in bs])
    assert w.size == MLP_NW and b.size == MLP_NB
    return torch.tensor(w, device=device), torch.tensor(b, device=device)


def mlp_forward(ctx: Context, scene: Scene, w_bf16: torch.Tensor, b: torch.Tensor, save_act: bool = True):
    """(eps_r, sigma, act) per triangle from the neural-material MLP (rt_mlp_forward)."""
    dev = torch.device("cuda", ctx.device)
    assert w_bf16.dtype == torch.bfloat16 and w_bf16.numel() == MLP_NW
    eps = torch.empty(scene.n_tris, dtype=torch.float32, device=dev)
    sig = torch.empty(scene.n_tris, dtype=torch.float32, device=dev)
    act = torch.empty((scene.n_tris, MLP_ACT), dtype=torch.bfloat16, device=dev) if save_act else None
    ctx._stream()
    ctx.check(ctx.lib.rt_mlp_forward(ctx.h, scene.h, _ptr(w_bf16.contiguous()), _ptr(b.contiguous()), _ptr(eps),
                                     _ptr(sig), _ptr(act)), "rt_mlp_forward")
    return eps, sig, act


def mlp_backward(ctx: Context, scene: Scene, w_bf16, act, eps, sig, grad_eps, grad_sigma, grad_w=None, grad_b=None,
                 dz=None):
    """Accumulates dL/dW (FP32, packed) and dL/db (rt_mlp_backward)."""
    dev = torch.device("cuda", ctx.device)
    grad_w = grad_w if grad_w is not None else torch.zeros(MLP_NW, dtype=torch.float32, device=dev)
    grad_b = grad_b if grad_b is not None else torch.zeros(MLP_NB, dtype=torch.float32, device=dev)
    dz = dz if dz is not None else torch.empty((scene.n_tris, 3 * MLP_WIDTH), dtype=torch.float32, device=dev)
    ctx._stream()
    ctx.check(ctx.lib.rt_mlp_backward(ctx.h, scene.h, _ptr(w_bf16.contiguous()), _ptr(act), _ptr(eps), _ptr(sig),
                                      _ptr(grad_eps.contiguous()), _ptr(grad_sigma.contiguous()), _ptr(dz),
                                      _ptr(grad_w), _ptr(grad_b)), "rt_mlp_backward")
    return grad_w, grad_b


# ----------------------------------------------------------------------------- batches and tuning

def trace_batch(ctx: Context, scenes, txs, rxs, n_rays: int, max_depth: int) -> Paths:
    """Traces several scenes in one pipeline (rt_trace_batch).  Returns one Paths
    over all receivers, scene after scene, with attributes scene_rx_offsets and
    scene_tri_offsets (numpy, n_scenes + 1)."""
    dev = torch.device("cuda", ctx.device)
    rx_list = [torch.as_tensor(np.asarray(r) if not isinstance(r, torch.Tensor) else r, dtype=torch.float64)
               for r in rxs]
    counts = np.array([r.shape[0] for r in rx_list], np.int32)
    rx_all = torch.cat([r.to(dev) for r in rx_list]).contiguous()
    tx = np.ascontiguousarray(np.asarray(txs, np.float64).reshape(-1, 3))
    n = len(scenes)
    handles = (_c.c_void_p * n)(*[s.h.value for s in scenes])
    h = _c.c_void_p()
    ctx._stream()
    ctx.check(ctx.lib.rt_trace_batch(ctx.h, handles, n, tx.ctypes.data_as(_c.c_void_p), _ptr(rx_all),
                                     counts.ctypes.data_as(_c.c_void_p), int(n_rays), int(max_depth), _c.byref(h)),
              "rt_trace_batch")
    p = Paths(ctx, list(scenes), h, int(counts.sum()), max_depth)
    ns = _c.c_int32()
    rx_off = np.zeros(n + 1, np.int64)
    tri_off = np.zeros(n + 1, np.int64)
    ctx.lib.rt_paths_batch_info(h, _c.byref(ns), rx_off.ctypes.data_as(_c.c_void_p), tri_off.ctypes.data_as(_c.c_void_p))
    p.scene_rx_offsets, p.scene_tri_offsets = rx_off, tri_off
    p._rx_all = rx_all
    return p


def set_cfr_tensor_cores(ctx: Context, enable: bool):
    """CFR contraction on the tensor cores (default) or on the SIMT units (rt_set_cfr_tensor_cores)."""
    ctx.check(ctx.lib.rt_set_cfr_tensor_cores(ctx.h, int(bool(enable))), "rt_set_cfr_tensor_cores")


def set_trace_async(ctx: Context, enable: bool):
    """trace_paths returns without waiting for the GPU (rt_set_trace_async); its paths then
    hold slots until Paths.resolve()."""
    ctx.check(ctx.lib.rt_set_trace_async(ctx.h, int(bool(enable))), "rt_set_trace_async")


def set_wait_limit(ctx: Context, polls: int):
    """Poll limit of the CFR kernels' waits on other CTAs; 0 restores the default (rt_set_wait_limit)."""
    ctx.check(ctx.lib.rt_set_wait_limit(ctx.h, int(polls)), "rt_set_wait_limit")


def set_tuning(ctx: Context, sbr: int, pairs: int, vis: int):
    ctx.check(ctx.lib.rt_set_tuning(ctx.h, int(sbr), int(pairs), int(vis)), "rt_set_tuning")


def autotune_trace(ctx: Context, scene: Scene, tx, rx: torch.Tensor, n_rays: int, max_depth: int):
    """Runs the tracing autotuner on this workload; returns ([sbr, pairs, vis] blocks per SM, summed stage ms)."""
    rx = rx.to(device=torch.device("cuda", ctx.device), dtype=torch.float64).contiguous()
    txa = (_c.c_double * 3)(*[float(v) for v in tx])
    chosen = (_c.c_int32 * 3)()
    ms = _c.c_double()
    ctx._stream()
    ctx.check(ctx.lib.rt_autotune_trace(ctx.h, scene.h, txa, _ptr(rx), rx.shape[0], int(n_rays), int(max_depth),
                                        chosen, _c.byref(ms)), "rt_autotune_trace")
    return list(chosen), float(ms.value)
