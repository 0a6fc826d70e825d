"""First-order diffraction on the GPU (rt_trace_diffraction, rt_eval_fields_diffraction
and its adjoint) against the FP64 oracle (oracle/diffraction.py; Sec. II-D Eq.
diffraction, Sec. II-F).

* The wedge table equals the oracle's (faces and exterior angles).
* Path sets are identical: the same (receiver, incidence face, other face) in the
  same order; delays within 1e-12 relative, points of diffraction within
  1e-9 of the scene diagonal.  Street canyon (concrete, glass, metal, ground) on a
  receiver subset and at full size in the benchmark's launch configuration
  (10^6 rays, 4096 receivers), indoor obstacles, ragged receiver counts.
* Coefficients within 1e-4 relative per path (FP32 against FP64), antenna gains
  and per-triangle materials included.
* Gradients with respect to eps_r, sigma (both faces) and the gains within 1e-4,
  normwise and per entry, against the oracle's autograd.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from gpu_helpers import assert_grad_close, rel_err_per_item
from oracle import diffraction as od

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def _trace(rt, ctx, sc, n_rays, rx=None, depth=None):
    rx = sc.rx if rx is None else rx
    scene = rt.Scene.from_synthetic(ctx, sc)
    rxt = torch.tensor(np.asarray(rx), dtype=torch.float64, device="cuda")
    spec = rt.trace_paths(ctx, scene, sc.tx, rxt, n_rays, sc.max_depth if depth is None else depth)
    dif = rt.trace_diffraction(ctx, scene, spec, sc.tx, rxt)
    ex = {k: v.cpu().numpy() for k, v in dif.export().items()}
    return scene, spec, dif, ex


def _assert_same(ex, dp, diag):
    assert np.array_equal(ex["rx"], dp["rx"])
    assert np.array_equal(ex["seq"], dp["faces"])
    assert np.array_equal(ex["rx_offsets"], dp["rx_offsets"])
    assert np.all(ex["depth"] == 1)
    if len(dp["tau"]):
        np.testing.assert_allclose(ex["tau"], dp["tau"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(ex["pts"][:, :3], dp["pts"], rtol=0, atol=1e-9 * diag)


def _dev(x, dtype=torch.float32):
    return torch.as_tensor(np.asarray(x), dtype=dtype, device="cuda").contiguous()


@pytest.mark.parametrize("name", ["street_canyon", "indoor_diff"])
def test_wedge_table_matches_oracle(rt, ctx, name):
    sc = getattr(scenegen, name)()
    scene = rt.Scene.from_synthetic(ctx, sc)
    faces, n = rt.scene_wedges(ctx, scene)
    W = od.wedges(oracle.OracleScene(sc))
    assert np.array_equal(faces, W["faces"])
    np.testing.assert_allclose(n, W["n"], rtol=0, atol=1e-12)
    assert len(n) > 100


@pytest.mark.parametrize("name,n_rays,step", [("street_canyon", 200_000, 61), ("indoor_diff", 200_000, 37),
                                              ("street_canyon", 33_333, 1001)])
def test_paths_and_coefficients(rt, ctx, name, n_rays, step):
    sc = getattr(scenegen, name)()
    rx = sc.rx[::step]
    scene, spec, dif, ex = _trace(rt, ctx, sc, n_rays, rx)
    sco = sc.subset_rx(np.arange(0, sc.n_rx, step))
    o = oracle.OracleScene(sco)
    dp = od.paths(o, n_rays=n_rays)
    assert len(dp["tau"]) > 0
    _assert_same(ex, dp, o.diag)
    for gt, gr in ((1.0, 1.0), (2.0, 0.5)):
        a = rt.eval_fields_diffraction(ctx, dif, _dev(sc.eps_r), _dev(sc.sigma), sc.freq_hz, gt, gr).cpu().numpy()
        ref = od.fields(sco, dp, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64), gain_tx=gt,
                        gain_rx=gr).numpy()
        err = rel_err_per_item(a, ref)
        assert err.max() <= 1e-4, (err.max(), np.argmax(err))
    assert ctx.status_word() == 0


def test_full_street_canyon_bench_configuration(rt, ctx):
    # the benchmark's launch configuration: 10^6 launch rays, every receiver
    sc = scenegen.street_canyon()
    scene, spec, dif, ex = _trace(rt, ctx, sc, sc.n_rays)
    o = oracle.OracleScene(sc)
    dp = od.paths(o, n_rays=sc.n_rays)
    assert len(dp["tau"]) > 10_000
    _assert_same(ex, dp, o.diag)
    a = rt.eval_fields_diffraction(ctx, dif, _dev(sc.eps_r), _dev(sc.sigma), sc.freq_hz).cpu().numpy()
    pick = np.arange(0, len(dp["tau"]), 37)
    sub = {k: (v[pick] if isinstance(v, np.ndarray) and v.shape[:1] == dp["tau"].shape else v) for k, v in dp.items()}
    ref = od.fields(sc, sub, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64)).numpy()
    assert rel_err_per_item(a[pick], ref).max() <= 1e-4
    assert ctx.status_word() == 0


@pytest.mark.parametrize("name", ["street_canyon", "indoor_diff"])
def test_backward_matches_oracle(rt, ctx, name):
    sc = getattr(scenegen, name)()
    step = 97 if name == "street_canyon" else 29
    scene, spec, dif, ex = _trace(rt, ctx, sc, 200_000, sc.rx[::step])
    sco = sc.subset_rx(np.arange(0, sc.n_rx, step))
    dp = od.paths(oracle.OracleScene(sco), n_rays=200_000)
    P = len(dp["tau"])
    rng = np.random.default_rng(3)
    g = (rng.normal(size=P) + 1j * rng.normal(size=P)).astype(np.complex64)
    gt, gr = 1.3, 0.7
    ge, gs, gg = rt.eval_fields_diffraction_backward(ctx, dif, _dev(sc.eps_r), _dev(sc.sigma), sc.freq_hz,
                                                     _dev(g, torch.complex64), gain_tx=gt, gain_rx=gr)
    e = torch.tensor(sc.eps_r.astype(np.float64), requires_grad=True)
    s = torch.tensor(sc.sigma.astype(np.float64), requires_grad=True)
    a = od.fields(sco, dp, e, s, gain_tx=gt, gain_rx=gr)
    (torch.as_tensor(g.astype(np.complex128)).conj() * a).real.sum().backward()
    assert_grad_close(ge.cpu().numpy(), e.grad.numpy(), what="eps_r")
    assert_grad_close(gs.cpu().numpy(), s.grad.numpy(), what="sigma")
    ra = float((np.conj(g.astype(np.complex128)) * a.detach().numpy()).real.sum())
    assert_grad_close(gg.cpu().numpy(), [ra / (2 * gt), ra / (2 * gr)], what="gains")
    # the autograd wrapper gives the same gradients
    ep = _dev(sc.eps_r).requires_grad_(True)
    sp = _dev(sc.sigma).requires_grad_(True)
    ad = rt.EvalFieldsDiffraction.apply(ep, sp, ctx, dif, sc.freq_hz, gt, gr)
    (_dev(g, torch.complex64).conj() * ad).real.sum().backward()
    torch.testing.assert_close(ep.grad, ge, rtol=1e-5, atol=1e-12)
    assert ctx.status_word() == 0


def test_per_triangle_materials(rt, ctx):
    sc = scenegen.street_canyon()
    rng = np.random.default_rng(9)
    T = sc.n_tris
    sc.per_triangle = True
    sc.tri_material = np.arange(T, dtype=np.int32)
    sc.eps_r = rng.uniform(2, 10, T).astype(np.float32)
    sc.sigma = (10 ** rng.uniform(-3, 0, T)).astype(np.float32)
    sc.is_pec = np.zeros(T, np.uint8)
    step = 131
    scene, spec, dif, ex = _trace(rt, ctx, sc, 100_000, sc.rx[::step])
    sco = sc.subset_rx(np.arange(0, sc.n_rx, step))
    dp = od.paths(oracle.OracleScene(sco), n_rays=100_000)
    a = rt.eval_fields_diffraction(ctx, dif, _dev(sc.eps_r), _dev(sc.sigma), sc.freq_hz,
                                   per_triangle=True).cpu().numpy()
    ref = od.fields(sco, dp, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64)).numpy()
    assert rel_err_per_item(a, ref).max() <= 1e-4
    g = (rng.normal(size=len(a)) + 1j * rng.normal(size=len(a))).astype(np.complex64)
    ge, gs, _ = rt.eval_fields_diffraction_backward(ctx, dif, _dev(sc.eps_r), _dev(sc.sigma), sc.freq_hz,
                                                    _dev(g, torch.complex64), per_triangle=True)
    e = torch.tensor(sc.eps_r.astype(np.float64), requires_grad=True)
    s = torch.tensor(sc.sigma.astype(np.float64), requires_grad=True)
    (torch.as_tensor(g.astype(np.complex128)).conj() * od.fields(sco, dp, e, s)).real.sum().backward()
    assert_grad_close(ge.cpu().numpy(), e.grad.numpy(), what="eps_r per triangle")
    assert_grad_close(gs.cpu().numpy(), s.grad.numpy(), what="sigma per triangle")


def test_antenna_pattern_on_diffraction_paths(rt, ctx):
    # departure and arrival directions are recorded like those of specular paths
    sc = scenegen.street_canyon()
    scene, spec, dif, ex = _trace(rt, ctx, sc, 100_000, sc.rx[::257])
    a = rt.eval_fields_diffraction(ctx, dif, _dev(sc.eps_r), _dev(sc.sigma), sc.freq_hz)
    pat = torch.tensor([1.0, 1.0, 3.0, 0.0, 0.0, 1.0], device="cuda")   # eta, one lobe up
    a_out, gt, _ = rt.antenna_apply(ctx, dif, a, pat)
    pts = ex["pts"]
    k1 = (pts[:, 1] - pts[:, 0]) / np.linalg.norm(pts[:, 1] - pts[:, 0], axis=1, keepdims=True)
    lam = 3.0
    G = 4 * np.pi * lam * np.exp(lam * (k1[:, 2] - 1)) / (2 * np.pi * (1 - np.exp(-2 * lam)))
    np.testing.assert_allclose(gt.cpu().numpy(), G, rtol=1e-5)
    assert ctx.status_word() == 0


def test_empty_and_rejected(rt, ctx):
    # inside a closed room every edge is concave: no wedges, no paths
    sc = scenegen.tiny_box()
    scene, spec, dif, ex = _trace(rt, ctx, sc, 10_000)
    assert dif.n_paths == 0 and np.all(ex["rx_offsets"] == 0)
    a = rt.eval_fields_diffraction(ctx, dif, _dev(sc.eps_r), _dev(sc.sigma), sc.freq_hz)
    assert a.numel() == 0
    # a specular trace of another scene, and the specular field call on diffraction paths
    other = rt.Scene.from_synthetic(ctx, scenegen.street_canyon())
    with pytest.raises(rt.RtError):
        rt.trace_diffraction(ctx, other, spec, sc.tx, torch.tensor(sc.rx, device="cuda"))
    sc2 = scenegen.street_canyon()
    _, _, dif2, _ = _trace(rt, ctx, sc2, 20_000, sc2.rx[::512])
    with pytest.raises(rt.RtError):
        rt.eval_fields(ctx, dif2, _dev(sc2.eps_r), _dev(sc2.sigma), sc2.freq_hz)
    assert ctx.status_word() == 0


def test_calibration_gradient_with_diffraction(rt, ctx):
    # specular and diffraction paths of each receiver merged into one CFR, power MSE,
    # autograd through the library back to eps_r and sigma, against the oracle's
    # FP64 chain (CFR adjoint, split, specular adjoint + diffraction autograd)
    sc = scenegen.street_canyon()
    step, n_rays = 127, 200_000
    rx = sc.rx[::step]
    scene, spec, dif, ex = _trace(rt, ctx, sc, n_rays, rx)
    sco = sc.subset_rx(np.arange(0, sc.n_rx, step))
    o = oracle.OracleScene(sco)
    tr = o.trace(n_rays=n_rays)
    dp = od.paths(o, n_rays=n_rays)
    fc, df, N, f = sc.f_center_hz, sc.delta_f_hz * 4, 256, sc.freq_hz
    R = len(rx)

    def merge(x1, o1, x2, o2):
        out, off = [], [0]
        for r in range(R):
            out += [x1[o1[r]:o1[r + 1]], x2[o2[r]:o2[r + 1]]]
            off.append(off[-1] + (o1[r + 1] - o1[r]) + (o2[r + 1] - o2[r]))
        return np.concatenate(out), np.array(off, np.int64)

    def oracle_a(eps, sig):
        a_s = o.fields(tr, eps_r=eps, sigma=sig)
        a_d = od.fields(sco, dp, eps, sig).detach().numpy()
        return a_s, a_d

    tau_m, off_m = merge(tr["tau"], tr["rx_offsets"], dp["tau"], dp["rx_offsets"])
    a_s, a_d = oracle_a(sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64))
    T = np.abs(oracle.cfr(merge(a_s, tr["rx_offsets"], a_d, dp["rx_offsets"])[0], tau_m, off_m, fc, df, N)) ** 2
    w = oracle.power_weights(T)
    eps0 = (sc.eps_r * 1.3).astype(np.float32)
    sig0 = (sc.sigma * 0.6).astype(np.float32)
    # oracle chain
    a_s, a_d = oracle_a(eps0.astype(np.float64), sig0.astype(np.float64))
    a_m = merge(a_s, tr["rx_offsets"], a_d, dp["rx_offsets"])[0]
    L_ref, gH = oracle.power_mse(oracle.cfr(a_m, tau_m, off_m, fc, df, N), T, w)
    ga = oracle.cfr_grad(tau_m, off_m, fc, df, N, gH)
    ga_s = np.concatenate([ga[off_m[r]:off_m[r] + tr["rx_offsets"][r + 1] - tr["rx_offsets"][r]] for r in range(R)])
    ga_d = np.concatenate([ga[off_m[r + 1] - (dp["rx_offsets"][r + 1] - dp["rx_offsets"][r]):off_m[r + 1]]
                           for r in range(R)])
    ge_s, gs_s, _ = o.fields_grad(tr, ga_s, eps_r=eps0, sigma=sig0)
    e = torch.tensor(eps0.astype(np.float64), requires_grad=True)
    s = torch.tensor(sig0.astype(np.float64), requires_grad=True)
    (torch.as_tensor(ga_d).conj() * od.fields(sco, dp, e, s)).real.sum().backward()
    ge_ref, gs_ref = ge_s + e.grad.numpy(), gs_s + s.grad.numpy()
    # library
    ep = _dev(eps0).requires_grad_(True)
    sp = _dev(sig0).requires_grad_(True)
    a1 = rt.EvalFields.apply(ep, sp, ctx, spec, f, 1.0, 1.0, False)
    a2 = rt.EvalFieldsDiffraction.apply(ep, sp, ctx, dif, f)
    am = rt.RxMerge.apply(a1, a2, spec.rx_offsets, dif.rx_offsets, ctx)
    taum, offm = rt.rx_merge(ctx, spec.rx_offsets, dif.rx_offsets, spec.tau, dif.tau)
    assert np.array_equal(offm.cpu().numpy(), off_m)
    loss = rt.CfrPowerMSE.apply(am, taum, offm, _dev(T), _dev(w), ctx, fc, df, N)
    loss.backward()
    assert abs(loss.item() - L_ref) <= 1e-4 * L_ref
    assert_grad_close(ep.grad.cpu().numpy(), ge_ref, what="eps_r")
    assert_grad_close(sp.grad.cpu().numpy(), gs_ref, what="sigma")
    assert ctx.status_word() == 0
