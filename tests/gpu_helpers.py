"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np
import torch

import oracle


def path_key_set(rx, depth, seq):
    return {(int(r), tuple(int(x) for x in s[:q])) for r, q, s in zip(rx, depth, seq)}


def gpu_trace(rt, ctx, sc, n_rays=None, depth=None, rx=None):
    n_rays = sc.n_rays if n_rays is None else n_rays
    depth = sc.max_depth if depth is None else depth
    rx = sc.rx if rx is None else rx
    scene = rt.Scene.from_synthetic(ctx, sc)
    rxt = torch.tensor(np.asarray(rx), dtype=torch.float64, device="cuda")
    p = rt.trace_paths(ctx, scene, sc.tx, rxt, n_rays, depth)
    ex = {k: v.cpu().numpy() for k, v in p.export().items()}
    return scene, p, ex


def oracle_trace(sc, n_rays=None, depth=None, rx=None):
    o = oracle.OracleScene(sc)
    tr = o.trace(n_rays=n_rays, depth=depth, rx=rx)
    return o, tr


def assert_same_paths(ex, tr, diag, tau_rtol=1e-12):
    """Exact path-set parity: same (receiver, triangle sequence) pairs in the same
    order, delays to FP64 rounding, points within 1e-9 of the scene diagonal."""
    ks_gpu = path_key_set(ex["rx"], ex["depth"], ex["seq"])
    ks_orc = path_key_set(tr["rx"], tr["depth"], tr["seq"])
    missing = sorted(ks_orc - ks_gpu)[:10]
    extra = sorted(ks_gpu - ks_orc)[:10]
    assert not missing and not extra, f"paths only in oracle: {missing}; only on GPU: {extra}"
    assert np.array_equal(ex["rx"], tr["rx"])
    assert np.array_equal(ex["depth"], tr["depth"])
    assert np.array_equal(ex["seq"], tr["seq"])
    assert np.array_equal(ex["rx_offsets"], tr["rx_offsets"])
    if len(tr["tau"]):
        np.testing.assert_allclose(ex["tau"], tr["tau"], rtol=tau_rtol, atol=0)
        for i in range(len(tr["tau"])):
            q = tr["depth"][i]
            np.testing.assert_allclose(ex["pts"][i, : q + 2], tr["pts"][i, : q + 2], rtol=0, atol=1e-9 * diag)


def rel_err_per_item(x, ref):
    x = np.asarray(x)
    ref = np.asarray(ref)
    return np.abs(x - ref) / np.maximum(np.abs(ref), 1e-300)


def normwise_rows(x, ref):
    num = np.linalg.norm(np.asarray(x) - np.asarray(ref), axis=-1)
    den = np.linalg.norm(np.asarray(ref), axis=-1)
    return num, den


def assert_grad_close(got, ref, rtol=1e-4, floor=1e-3, what=""):
    """Gradient parity: normwise within rtol, and every entry whose magnitude exceeds
    floor * max|ref| within rtol relative on its own, so that a small entry (a material
    with few paths) cannot be wrong under the cover of a large one."""
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    assert np.linalg.norm(got - ref) <= rtol * np.linalg.norm(ref), (what, got, ref)
    big = np.abs(ref) > floor * np.abs(ref).max()
    rel = np.abs(got[big] - ref[big]) / np.abs(ref[big])
    assert rel.size == 0 or rel.max() <= rtol, (what, np.flatnonzero(big)[np.argmax(rel)], rel.max(), got, ref)
