"""GPU neural-material kernels (BF16 weights and layer inputs, FP32 sums) vs the
FP64 oracle with BF16 emulation (Sec. III-D).

Tolerances are set by BF16 storage: a feature computed in FP32 on the GPU and in
FP64 in the oracle can round to neighbouring BF16 values, which also flips the
occasional ReLU mask.  Forward outputs: 1e-3 normwise.  Weight gradients sum
activation x dZ over all 20k rows, so each product carries up to one BF16 unit
roundoff (2^-8 relative) of disagreement: 2^-8 normwise."""
import numpy as np
import pytest
import torch

import scenegen
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2311_18558_gb300 as rt
    ctx = rt.Context(0)
    sc = scenegen.room_corridor(n_rx=8)
    scene = rt.Scene.from_synthetic(ctx, sc)
    Ws, bs = scenegen.random_mlp_params(7)
    Ws = [w * 0.5 for w in Ws]
    bs[-1] = np.array([np.log(0.05), np.log(3.0)], np.float32)
    V = sc.verts.astype(np.float64)
    cen = V[sc.tris].mean(axis=1)
    lo, hi = V.min(0), V.max(0)
    x = mlp.encode(mlp.normalize(cen, lo, hi))
    return rt, ctx, sc, scene, Ws, bs, x


def test_mlp_forward(setup):
    rt, ctx, sc, scene, Ws, bs, x = setup
    w, b = rt.pack_mlp(Ws, bs)
    eps, sig, act = rt.mlp_forward(ctx, scene, w.to(torch.bfloat16), b)
    out, _, _ = mlp.forward(x, Ws, bs, bf16=True)
    eps_ref, sig_ref = mlp.materials(out)
    e, s = eps.cpu().numpy(), sig.cpu().numpy()
    assert np.linalg.norm(e - eps_ref) <= 1e-3 * np.linalg.norm(eps_ref)
    assert np.linalg.norm(s - sig_ref) <= 1e-3 * np.linalg.norm(sig_ref)
    assert np.isfinite(e).all() and (e >= 1).all() and (s > 0).all()


def test_mlp_backward(setup):
    rt, ctx, sc, scene, Ws, bs, x = setup
    w, b = rt.pack_mlp(Ws, bs)
    w16 = w.to(torch.bfloat16)
    eps, sig, act = rt.mlp_forward(ctx, scene, w16, b)
    rng = np.random.default_rng(5)
    ge = rng.normal(size=sc.n_tris).astype(np.float32)
    gs = rng.normal(size=sc.n_tris).astype(np.float32)
    gw, gb = rt.mlp_backward(ctx, scene, w16, act, eps, sig, torch.tensor(ge, device="cuda"),
                             torch.tensor(gs, device="cuda"))
    gW_ref, gb_ref = mlp.backward(x, Ws, bs, ge, gs, bf16=True)
    gw_ref_packed = np.concatenate([gW_ref[0].ravel(), np.zeros(128), gW_ref[1].ravel(), gW_ref[2].ravel(),
                                    gW_ref[3].ravel()])
    got = gw.cpu().numpy()
    tol = 2.0 ** -8
    assert np.linalg.norm(got - gw_ref_packed) <= tol * np.linalg.norm(gw_ref_packed)
    gbr = np.concatenate(gb_ref)
    assert np.linalg.norm(gb.cpu().numpy() - gbr) <= tol * np.linalg.norm(gbr)
    # per layer as well (the small last layer must not hide behind the large ones)
    o = [0, 40 * 128, 40 * 128 + 128 * 128, 40 * 128 + 2 * 128 * 128, 38144]
    ref_layers = [np.concatenate([gW_ref[0].ravel(), np.zeros(128)]), gW_ref[1].ravel(), gW_ref[2].ravel(),
                  gW_ref[3].ravel()]
    for li in range(4):
        r = ref_layers[li]
        assert np.linalg.norm(got[o[li]:o[li + 1]] - r) <= tol * np.linalg.norm(r), li


def test_mlp_autograd_module(setup):
    rt, ctx, sc, scene, Ws, bs, x = setup
    m = rt.NeuralMaterials(Ws, bs)
    eps, sig = m(ctx, scene)
    (eps.sum() + 2.0 * sig.sum()).backward()
    assert m.w.grad is not None and torch.isfinite(m.w.grad).all() and m.w.grad.abs().sum() > 0
    assert torch.isfinite(m.b.grad).all()
