"""Diffuse reflection on the GPU (rt_trace_diffuse, rt_eval_fields_diffuse and its
adjoint, rt_specular_reduction and its adjoint, rt_rx_merge / rt_rx_split) vs the
FP64 oracle (oracle/rt_oracle.cpp next-event estimation, oracle/diffuse.py).

Tolerances: path sets identical (receiver, depth, triangles, order), points within
1e-9 of the scene diagonal, delays within 1e-12 relative (FP64 on both sides);
coefficients within 2e-5 relative (FP32 chain of <= 3 Fresnel products, the
pattern's exponentials and a square root); gradients within 1e-4 normwise per
parameter group; merge and split bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import scenegen
from gpu_helpers import assert_grad_close
from oracle import diffuse as od

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import paper_2311_18558_gb300 as rt
    return rt


@pytest.fixture(scope="module")
def ctx(rt):
    return rt.Context(0)


def _trace_both(rt, ctx, sc, n_rays, depth, rx):
    scene = rt.Scene.from_synthetic(ctx, sc)
    p = rt.trace_diffuse(ctx, scene, sc.tx, torch.tensor(np.asarray(rx), dtype=torch.float64, device="cuda"),
                         n_rays, depth)
    ex = {k: v.cpu().numpy() for k, v in p.export().items()}
    o = oracle.OracleScene(sc)
    tr = o.diffuse_paths(n_rays, depth, rx=rx)
    return scene, p, ex, o, tr


def _assert_same(ex, tr, diag):
    assert ex["rx"].shape == tr["rx"].shape, (ex["rx"].shape, tr["rx"].shape)
    assert np.array_equal(ex["rx_offsets"], tr["rx_offsets"])
    assert np.array_equal(ex["rx"], tr["rx"])
    assert np.array_equal(ex["depth"], tr["depth"])
    assert np.array_equal(ex["seq"], tr["seq"])
    if len(tr["tau"]):
        np.testing.assert_allclose(ex["tau"], tr["tau"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(ex["pts"], tr["pts"], rtol=0, atol=1e-9 * diag)


@pytest.mark.parametrize("n_rays", [1, 33, 1000])
def test_closed_room_path_sets(rt, ctx, n_rays):
    sc = scenegen.tiny_box()
    scene, p, ex, o, tr = _trace_both(rt, ctx, sc, n_rays, 2, sc.rx)
    assert p.n_paths == sc.n_rx * n_rays * 2
    _assert_same(ex, tr, o.diag)
    assert ctx.status_word() == 0


@pytest.mark.parametrize("name,n_rays,depth,step", [("indoor", 3000, 3, 64), ("street", 20000, 3, 256)])
def test_path_sets(rt, ctx, name, n_rays, depth, step):
    sc = scenegen.indoor_diff() if name == "indoor" else scenegen.street_canyon()
    rx = sc.rx[::step]
    scene, p, ex, o, tr = _trace_both(rt, ctx, sc, n_rays, depth, rx)
    assert p.n_paths > 1000
    _assert_same(ex, tr, o.diag)
    assert ctx.status_word() == 0


@pytest.fixture(scope="module")
def indoor(rt, ctx):
    sc = scenegen.indoor_diff()
    rx = sc.rx[::64]
    scene, p, ex, o, tr = _trace_both(rt, ctx, sc, 3000, 3, rx)
    _assert_same(ex, tr, o.diag)
    sc2 = sc.subset_rx(np.arange(0, sc.n_rx, 64))
    return sc2, scene, p, tr


def _scat(seed, M):
    return scenegen.random_scattering(seed, M)


def test_fields_match_oracle(rt, ctx, indoor):
    sc, scene, p, tr = indoor
    scat = _scat(7, sc.n_materials)
    a = rt.eval_fields_diffuse(ctx, p, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
                               torch.tensor(scat, device="cuda"), sc.freq_hz).cpu().numpy()
    ref = od.fields(sc, tr, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64), scat.astype(np.float64),
                    sc.freq_hz, 3000).numpy()
    assert np.all(a.imag == 0)
    np.testing.assert_allclose(a.real, ref.real, rtol=2e-5, atol=1e-6 * np.abs(ref).max())
    # antenna patterns apply to diffuse paths through the same records
    a_id, _, _ = rt.antenna_apply(ctx, p, torch.tensor(a, device="cuda"))
    assert np.array_equal(a_id.cpu().numpy(), a)
    assert ctx.status_word() == 0


def test_fields_gain_and_pec(rt, ctx):
    # a PEC material and antenna gains: a scales by sqrt(g_T g_R)
    sc = scenegen.street_canyon()
    rx = sc.rx[::512]
    scene, p, ex, o, tr = _trace_both(rt, ctx, sc, 5000, 2, rx)
    assert sc.is_pec.any()
    scat = _scat(3, sc.n_materials)
    args = (torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
            torch.tensor(scat, device="cuda"), sc.freq_hz)
    a1 = rt.eval_fields_diffuse(ctx, p, *args).cpu().numpy()
    a4 = rt.eval_fields_diffuse(ctx, p, *args, gain_tx=2.0, gain_rx=8.0).cpu().numpy()
    np.testing.assert_allclose(a4, 4.0 * a1, rtol=1e-6)
    ref = od.fields(sc.subset_rx(np.arange(0, sc.n_rx, 512)), tr, sc.eps_r.astype(np.float64),
                    sc.sigma.astype(np.float64), scat.astype(np.float64), sc.freq_hz, 5000).numpy()
    np.testing.assert_allclose(a1.real, ref.real, rtol=2e-5, atol=1e-6 * np.abs(ref).max())


def test_backward_matches_oracle(rt, ctx, indoor):
    sc, scene, p, tr = indoor
    scat = _scat(11, sc.n_materials)
    rng = np.random.default_rng(4)
    P = p.n_paths
    g = (rng.normal(size=P) + 1j * rng.normal(size=P)).astype(np.complex64)
    ge, gs, gc = rt.eval_fields_diffuse_backward(
        ctx, p, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
        torch.tensor(scat, device="cuda"), sc.freq_hz, torch.tensor(g, device="cuda"))
    e = torch.tensor(sc.eps_r.astype(np.float64), requires_grad=True)
    s = torch.tensor(sc.sigma.astype(np.float64), requires_grad=True)
    c = torch.tensor(scat[:, :7].astype(np.float64), requires_grad=True)
    a = od.fields(sc, tr, e, s, c, sc.freq_hz, 3000)
    (torch.as_tensor(g.astype(np.complex128)).conj() * a).real.sum().backward()
    for got, ref in ((ge, e.grad), (gs, s.grad)):
        got, ref = got.cpu().numpy(), ref.numpy()
        assert_grad_close(got, ref)
    gc = gc.cpu().numpy()
    assert np.all(gc[:, 7] == 0)
    for col in range(7):
        ref = c.grad[:, col].numpy()
        assert_grad_close(gc[:, col], ref, what=col)


def test_specular_reduction(rt, ctx):
    sc = scenegen.indoor_diff()
    rx = sc.rx[::64]
    scene = rt.Scene.from_synthetic(ctx, sc)
    p = rt.trace_paths(ctx, scene, sc.tx, torch.tensor(rx, device="cuda"), 200_000, 3)
    tr = {k: v.cpu().numpy() for k, v in p.export().items()}
    a = rt.eval_fields(ctx, p, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
                       sc.freq_hz)
    scat = _scat(5, sc.n_materials)
    sd = torch.tensor(scat, device="cuda")
    out = rt.specular_reduction(ctx, p, sd, a)
    ref = od.specular_reduction(sc, tr, scat[:, :7].astype(np.float64), a.cpu().numpy().astype(np.complex128))
    np.testing.assert_allclose(out.cpu().numpy(), ref.numpy(), rtol=1e-6, atol=0)
    rng = np.random.default_rng(6)
    g = (rng.normal(size=p.n_paths) + 1j * rng.normal(size=p.n_paths)).astype(np.complex64)
    ga, gc = rt.specular_reduction_backward(ctx, p, sd, out, torch.tensor(g, device="cuda"))
    c = torch.tensor(scat[:, :7].astype(np.float64), requires_grad=True)
    a_in = torch.as_tensor(a.cpu().numpy().astype(np.complex128))
    y = od.specular_reduction(sc, tr, c, a_in)
    (torch.as_tensor(g.astype(np.complex128)).conj() * y).real.sum().backward()
    ref_S = c.grad[:, 0].numpy()
    assert np.linalg.norm(gc.cpu().numpy()[:, 0] - ref_S) <= 1e-4 * np.linalg.norm(ref_S)
    fac = (ref.numpy() / np.where(a_in.numpy() == 0, 1, a_in.numpy())).real
    np.testing.assert_allclose(ga.cpu().numpy(), g * fac, rtol=1e-5, atol=1e-30)


def test_rx_merge_split(rt, ctx):
    rng = np.random.default_rng(8)
    R = 37
    c1 = rng.integers(0, 5, R)
    c2 = rng.integers(0, 7, R)
    c1[3] = c2[3] = 0
    o1 = np.concatenate([[0], np.cumsum(c1)])
    o2 = np.concatenate([[0], np.cumsum(c2)])
    x1 = (rng.normal(size=o1[-1]) + 1j * rng.normal(size=o1[-1])).astype(np.complex64)
    x2 = (rng.normal(size=o2[-1]) + 1j * rng.normal(size=o2[-1])).astype(np.complex64)
    ref = np.concatenate([np.concatenate([x1[o1[r]:o1[r + 1]], x2[o2[r]:o2[r + 1]]]) for r in range(R)])
    d = lambda v: torch.tensor(v, device="cuda")  # noqa: E731
    out, off = rt.rx_merge(ctx, d(o1), d(o2), d(x1), d(x2))
    assert np.array_equal(out.cpu().numpy(), ref)
    assert np.array_equal(off.cpu().numpy(), o1 + o2)
    s1, s2 = rt.rx_split(ctx, d(o1), d(o2), out)
    assert np.array_equal(s1.cpu().numpy(), x1) and np.array_equal(s2.cpu().numpy(), x2)
    t1, t2 = rng.uniform(size=o1[-1]), rng.uniform(size=o2[-1])
    tref = np.concatenate([np.concatenate([t1[o1[r]:o1[r + 1]], t2[o2[r]:o2[r + 1]]]) for r in range(R)])
    tout, _ = rt.rx_merge(ctx, d(o1), d(o2), d(t1), d(t2))
    assert np.array_equal(tout.cpu().numpy(), tref)


def test_scattering_calibration(rt, ctx):
    # hidden S, K_x and scattering patterns are recovered from CFR powers of the
    # specular + diffuse paths: eval_fields -> specular share, eval_fields_diffuse ->
    # per-receiver merge -> CFR + power MSE, with L = 30 material embeddings
    sc = scenegen.indoor_diff()
    dev = "cuda"
    rx = torch.tensor(sc.rx[::16], device=dev)
    scene = rt.Scene.from_synthetic(ctx, sc)
    ps = rt.trace_paths(ctx, scene, sc.tx, rx, 200_000, 2)
    pd = rt.trace_diffuse(ctx, scene, sc.tx, rx, 4000, 2)
    tau, off = rt.rx_merge(ctx, ps.rx_offsets, pd.rx_offsets, ps.tau, pd.tau)
    fc, df, N = sc.f_center_hz, sc.delta_f_hz, 256
    eps = torch.tensor(sc.eps_r, device=dev)
    sig = torch.tensor(sc.sigma, device=dev)
    hidden = torch.tensor(_scat(21, sc.n_materials), device=dev)

    def forward(scat):
        a_s = rt.SpecularReduction.apply(rt.EvalFields.apply(eps, sig, ctx, ps, sc.freq_hz, 1.0, 1.0, False),
                                         scat, ctx, ps)
        a_d = rt.EvalFieldsDiffuse.apply(eps, sig, scat, ctx, pd, sc.freq_hz)
        return rt.RxMerge.apply(a_s, a_d, ps.rx_offsets, pd.rx_offsets, ctx)
    with torch.no_grad():
        T = (rt.cfr(ctx, off, forward(hidden), tau, fc, df, N).abs() ** 2).float().contiguous()
    m = T.mean(1)
    w = torch.where(m > 0, 1 / torch.where(m > 0, m, torch.ones_like(m)), torch.zeros_like(m)).contiguous()
    M = sc.n_materials
    emb = rt.MaterialEmbeddings(sc.eps_r, sc.sigma, L=30, S_init=np.full(M, 0.4), K_x_init=np.full(M, 0.25)).to(dev)
    pat = rt.ScatteringPattern(M, lam_init=6.0).to(dev)
    opt = torch.optim.Adam([emb.v, emb.w_S, emb.w_Kx, *pat.parameters()], lr=0.01)
    losses = []
    for _ in range(150):
        S, Kx = emb.scattering()
        wts, lam = pat()
        scat = rt.pack_scattering(S, Kx, wts, lam)
        L = rt.CfrPowerMSE.apply(forward(scat), tau, off, T, w, ctx, fc, df, N)
        opt.zero_grad()
        L.backward()
        opt.step()
        losses.append(L.item())
    assert losses[-1] < 0.1 * losses[0], losses[::15]
    assert ctx.status_word() == 0


def test_diffuse_rejects_bad_arguments(rt, ctx):
    # host-side validation: nothing is launched, the status word stays clear
    sc = scenegen.tiny_box()
    scene = rt.Scene.from_synthetic(ctx, sc)
    rxt = torch.tensor(sc.rx, dtype=torch.float64, device="cuda")
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.trace_diffuse(ctx, scene, sc.tx, rxt, 1000, 5)
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.trace_diffuse(ctx, scene, sc.tx, rxt, 0, 2)
    with pytest.raises(rt.RtError, match="NUMERIC"):
        rt.trace_diffuse(ctx, scene, (float("nan"), 0.0, 0.0), rxt, 10, 2)
    pd = rt.trace_diffuse(ctx, scene, sc.tx, rxt, 100, 2)
    ps = rt.trace_paths(ctx, scene, sc.tx, rxt, 1000, 2)
    eps = torch.tensor(sc.eps_r, device="cuda")
    sig = torch.tensor(sc.sigma, device="cuda")
    scat = torch.tensor(_scat(1, sc.n_materials), device="cuda")
    a = torch.zeros(ps.n_paths, dtype=torch.complex64, device="cuda")
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.eval_fields(ctx, pd, eps, sig, sc.freq_hz)            # diffuse paths in the specular kernel
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.eval_fields_diffuse(ctx, ps, eps, sig, scat, sc.freq_hz)   # and the reverse
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.specular_reduction(ctx, pd, scat, torch.zeros(pd.n_paths, dtype=torch.complex64, device="cuda"))
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.eval_fields_diffuse(ctx, pd, eps, sig, scat, -1.0)
    with pytest.raises(rt.RtError, match="INVALID_ARG"):
        rt.eval_fields_diffuse(ctx, pd, eps, sig, scat, sc.freq_hz, gain_tx=0.0)
    with pytest.raises(ValueError):
        rt.rx_merge(ctx, ps.rx_offsets, pd.rx_offsets, a, torch.zeros(pd.n_paths, device="cuda"))
    assert ctx.status_word() == 0


def test_random_phases(rt, ctx, indoor):
    # per-path random phases of Eq. scattered_field (inputs): coefficients and the
    # adjoint against the oracle with the same phases, then cleared again
    sc, scene, p, tr = indoor
    scat = _scat(13, sc.n_materials)
    rng = np.random.default_rng(17)
    chi = rng.uniform(0, 2 * np.pi, (p.n_paths, 2)).astype(np.float32)
    rt.set_diffuse_phases(ctx, p, torch.tensor(chi, device="cuda"))
    try:
        eps_d, sig_d = torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda")
        scat_d = torch.tensor(scat, device="cuda")
        a = rt.eval_fields_diffuse(ctx, p, eps_d, sig_d, scat_d, sc.freq_hz).cpu().numpy()
        ref = od.fields(sc, tr, sc.eps_r.astype(np.float64), sc.sigma.astype(np.float64), scat.astype(np.float64),
                        sc.freq_hz, 3000, chi=chi.astype(np.float64)).numpy()
        np.testing.assert_allclose(a, ref, rtol=2e-5, atol=1e-6 * np.abs(ref).max())
        g = (rng.normal(size=p.n_paths) + 1j * rng.normal(size=p.n_paths)).astype(np.complex64)
        ge, gs, gcat = rt.eval_fields_diffuse_backward(ctx, p, eps_d, sig_d, scat_d, sc.freq_hz,
                                                        torch.tensor(g, device="cuda"))
        e = torch.tensor(sc.eps_r.astype(np.float64), requires_grad=True)
        s = torch.tensor(sc.sigma.astype(np.float64), requires_grad=True)
        c = torch.tensor(scat[:, :7].astype(np.float64), requires_grad=True)
        af = od.fields(sc, tr, e, s, c, sc.freq_hz, 3000, chi=chi.astype(np.float64))
        (torch.as_tensor(g.astype(np.complex128)).conj() * af).real.sum().backward()
        for got, ref_g in ((ge, e.grad), (gs, s.grad)):
            assert_grad_close(got.cpu().numpy(), ref_g.numpy())
        gcat = gcat.cpu().numpy()
        for col in range(7):
            ref_c = c.grad[:, col].numpy()
            assert_grad_close(gcat[:, col], ref_c, what=col)
    finally:
        rt.set_diffuse_phases(ctx, p, None)
    a0 = rt.eval_fields_diffuse(ctx, p, torch.tensor(sc.eps_r, device="cuda"), torch.tensor(sc.sigma, device="cuda"),
                                torch.tensor(scat, device="cuda"), sc.freq_hz)
    assert torch.all(a0.imag == 0)
    assert ctx.status_word() == 0
