"""What the trained network gains over the method without it (Sec. III-D).

Scene: the room-and-corridor mesh whose ground-truth eps_r and sigma vary
smoothly from triangle to triangle.  Both calibrations run Algorithm 1 (Adam) on
the CFR power of the same training receivers through the library kernels:
  - plain: one (eps_r, sigma) per object (floor, ceiling, walls, partition), the
    per-material calibration of Sec. III-C in the log domain;
  - neural: the MLP of Sec. III-D at every triangle centroid.
The neural model must reach a clearly lower loss on held-out receivers.
"""
import numpy as np
import pytest
import torch

import scenegen

pytestmark = pytest.mark.gpu


def test_neural_materials_beat_per_object_calibration():
    import paper_2311_18558_gb300 as rt
    sc = scenegen.room_corridor(n_rx=1536)
    ctx = rt.Context(0)
    scene_tri = rt.Scene.from_synthetic(ctx, sc)                       # per-triangle materials
    scene_obj = rt.Scene(ctx, sc.verts, sc.tris, sc.tri_object, np.zeros(4, np.uint8))   # per object
    dev = "cuda"
    rx_tr = torch.tensor(sc.rx[:1280], device=dev)
    rx_te = torch.tensor(sc.rx[1280:], device=dev)
    n_rays = 300_000
    fc, df, N, f = sc.f_center_hz, sc.delta_f_hz, sc.n_sub, sc.freq_hz
    eg = torch.tensor(sc.eps_r, device=dev)
    sg = torch.tensor(sc.sigma, device=dev)

    def target(p):
        a = rt.eval_fields(ctx, p, eg, sg, f, per_triangle=True)
        T = (rt.cfr(ctx, p.rx_offsets, a, p.tau, fc, df, N).abs() ** 2).float().contiguous()
        m = T.mean(1)
        w = torch.where(m > 0, 1 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).float()
        return T, w.contiguous()

    tri_tr = rt.trace_paths(ctx, scene_tri, sc.tx, rx_tr, n_rays, 3)
    tri_te = rt.trace_paths(ctx, scene_tri, sc.tx, rx_te, n_rays, 3)
    obj_tr = rt.trace_paths(ctx, scene_obj, sc.tx, rx_tr, n_rays, 3)
    obj_te = rt.trace_paths(ctx, scene_obj, sc.tx, rx_te, n_rays, 3)
    assert obj_tr.n_paths == tri_tr.n_paths and obj_te.n_paths == tri_te.n_paths
    Ttr, wtr = target(tri_tr)
    Tte, wte = target(tri_te)

    plain = rt.LogMaterials(np.full(4, 4.0), np.full(4, 0.05)).cuda()
    opt_p = torch.optim.Adam(plain.parameters(), lr=0.05)
    Ws, bs = scenegen.random_mlp_params(11)
    Ws = [w * 0.5 for w in Ws]
    bs[-1] = np.array([np.log(0.05), np.log(3.0)], np.float32)
    neural = rt.NeuralMaterials(Ws, bs)
    opt_n = torch.optim.Adam(neural.parameters(), lr=3e-3)

    def plain_loss(p, T, w):
        e, s = plain()
        return rt.calibration_loss(ctx, p, e.contiguous(), s.contiguous(), T, w, f, fc, df, N)

    def neural_loss(p, T, w):
        e, s = neural(ctx, scene_tri)
        return rt.calibration_loss(ctx, p, e, s, T, w, f, fc, df, N, per_triangle=True)

    with torch.no_grad():
        start = (plain_loss(obj_te, Tte, wte).item(), neural_loss(tri_te, Tte, wte).item())
    for _ in range(150):
        L = plain_loss(obj_tr, Ttr, wtr)
        opt_p.zero_grad()
        L.backward()
        opt_p.step()
        L2 = neural_loss(tri_tr, Ttr, wtr)
        opt_n.zero_grad()
        L2.backward()
        opt_n.step()
    with torch.no_grad():
        held_plain = plain_loss(obj_te, Tte, wte).item()
        held_neural = neural_loss(tri_te, Tte, wte).item()
    assert held_plain < start[0] and held_neural < start[1]
    assert held_neural < 0.25 * held_plain, (start, held_plain, held_neural)
    assert ctx.status_word() == 0
