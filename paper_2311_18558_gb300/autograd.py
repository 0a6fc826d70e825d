"""torch.autograd glue over the library's hand-written adjoint kernels.

The calibration of Algorithm 1 (arXiv 2311.18558, Sec. III-G) differentiates the
field computation with the path geometry held fixed (Sec. II-F): gradients flow
from the loss through the CFR (rt_cfr_backward or the fused kernel) into the
path coefficients and from there into eps_r, sigma (rt_eval_fields_backward).
PyTorch only stores the parameters and runs the optimiser.
"""
from __future__ import annotations

import torch

from . import api


class EvalFields(torch.autograd.Function):
    """a = eval_fields(eps_r, sigma) with the hand-written adjoint as backward."""

    @staticmethod
    def forward(fctx, eps_r, sigma, ctx, paths, freq_hz, gain_tx, gain_rx, per_triangle):
        eps_r = eps_r.contiguous()
        sigma = sigma.contiguous()
        a = api.eval_fields(ctx, paths, eps_r, sigma, freq_hz, gain_tx, gain_rx, per_triangle)
        fctx.save_for_backward(eps_r, sigma)
        fctx.args = (ctx, paths, freq_hz, gain_tx, gain_rx, per_triangle)
        return a

    @staticmethod
    def backward(fctx, grad_a):
        eps_r, sigma = fctx.saved_tensors
        ctx, paths, freq_hz, gain_tx, gain_rx, per_triangle = fctx.args
        ge, gs, _ = api.eval_fields_backward(ctx, paths, eps_r, sigma, freq_hz, grad_a.contiguous(),
                                             gain_tx=gain_tx, gain_rx=gain_rx, per_triangle=per_triangle)
        return ge, gs, None, None, None, None, None, None


class Cfr(torch.autograd.Function):
    """H = cfr(a) (Sec. II-A) with rt_cfr_backward as backward."""

    @staticmethod
    def forward(fctx, a, tau, rx_offsets, ctx, f_center_hz, delta_f_hz, n_sub):
        H = api.cfr(ctx, rx_offsets, a.contiguous(), tau, f_center_hz, delta_f_hz, n_sub)
        fctx.args = (ctx, rx_offsets, tau, f_center_hz, delta_f_hz, n_sub)
        return H

    @staticmethod
    def backward(fctx, grad_H):
        ctx, rx_offsets, tau, fc, df, n = fctx.args
        return api.cfr_backward(ctx, rx_offsets, tau, fc, df, n, grad_H.contiguous()), None, None, None, None, None, None


class CfrPowerMSE(torch.autograd.Function):
    """Loss L = 1/(R N) sum (w_r (|H|^2 - P*))^2 of the CFR of a; the forward
    launch also produces dL/da, which backward scales by the incoming gradient."""

    @staticmethod
    def forward(fctx, a, tau, rx_offsets, target_power, rx_weight, ctx, f_center_hz, delta_f_hz, n_sub):
        loss, grad_a, _ = api.cfr_power_mse_fused(ctx, rx_offsets, a.contiguous(), tau, f_center_hz, delta_f_hz,
                                                  n_sub, target_power, rx_weight)
        fctx.save_for_backward(grad_a)
        return loss[0]

    @staticmethod
    def backward(fctx, g):
        (grad_a,) = fctx.saved_tensors
        return grad_a * g, None, None, None, None, None, None, None, None


class DelaySpreadPowerLoss(torch.autograd.Function):
    """The paper's loss (Eq. loss): mean over receivers of SMAPE(tau_RMS, tau^_RMS) +
    SMAPE(alpha P, P^) of the CIRs of H; the forward launch also produces dL/dH."""

    @staticmethod
    def forward(fctx, H, P_meas, tau_meas, alpha_state, ctx, delta_f_hz):
        loss, grad_H = api.delay_spread_power_loss(ctx, H, delta_f_hz, P_meas, tau_meas, alpha_state)
        fctx.save_for_backward(grad_H)
        return loss[0]

    @staticmethod
    def backward(fctx, g):
        (grad_H,) = fctx.saved_tensors
        return grad_H * g, None, None, None, None, None


def paper_calibration_loss(ctx, paths, eps_r, sigma, P_meas, tau_meas, alpha_state, freq_hz, f_center_hz,
                           delta_f_hz, n_sub, decay=0.99, update_scale=True, per_triangle=False):
    """One step of Algorithm 1 with the paper's loss: a = eval_fields(eps_r, sigma),
    H = CFR(a), the power scale alpha updated by its moving average from this
    batch (Eq. scaling_param; no gradient), then Eq. loss.  alpha_state is the
    2-float device state of rt_power_scale_ema."""
    a = EvalFields.apply(eps_r, sigma, ctx, paths, freq_hz, 1.0, 1.0, per_triangle)
    H = Cfr.apply(a, paths.tau, paths.rx_offsets, ctx, f_center_hz, delta_f_hz, n_sub)
    if update_scale:
        with torch.no_grad():
            P_pred, _ = api.cir_stats(ctx, H.detach(), delta_f_hz)
            api.power_scale_ema(ctx, P_meas, P_pred, decay, alpha_state)
    return DelaySpreadPowerLoss.apply(H, P_meas, tau_meas, alpha_state, ctx, delta_f_hz)


class AntennaApply(torch.autograd.Function):
    """a sqrt(G_T(departure) G_R(arrival)) with packed mixture-of-lobes patterns
    (either may be None for a unit gain), rt_antenna_apply_backward as backward."""

    @staticmethod
    def forward(fctx, a, tx_pattern, rx_pattern, ctx, paths):
        tx = tx_pattern.contiguous() if tx_pattern is not None else None
        rx = rx_pattern.contiguous() if rx_pattern is not None else None
        a_out, gt, gr = api.antenna_apply(ctx, paths, a, tx, rx)
        fctx.save_for_backward(a_out, *(t for t in (gt, gr, tx, rx) if t is not None))
        fctx.flags = (gt is not None, gr is not None)
        fctx.args = (ctx, paths)
        return a_out

    @staticmethod
    def backward(fctx, grad_out):
        saved = list(fctx.saved_tensors)
        a_out = saved.pop(0)
        has_t, has_r = fctx.flags
        gt = saved.pop(0) if has_t else None
        gr = saved.pop(0) if has_r else None
        tx = saved.pop(0) if has_t else None
        rx = saved.pop(0) if has_r else None
        ctx, paths = fctx.args
        ga, gtx, grx = api.antenna_apply_backward(ctx, paths, a_out, gt, gr, grad_out, tx, rx)
        return ga, gtx, grx, None, None


class AntennaPattern(torch.nn.Module):
    """Trainable pattern of Sec. III-B: weights by a softmax, concentrations by an
    exponential, mean directions normalised, radiation efficiency by a sigmoid;
    forward() returns the packed physical parameters of rt_antenna_apply."""

    def __init__(self, n_lobes=3, lam_init=2.0, eta_init=0.9, seed=0):
        super().__init__()
        g = torch.Generator().manual_seed(seed)
        self.w_logit = torch.nn.Parameter(torch.zeros(n_lobes))
        self.log_lam = torch.nn.Parameter(torch.full((n_lobes,), float(torch.log(torch.tensor(lam_init)))))
        self.mu_raw = torch.nn.Parameter(torch.randn(n_lobes, 3, generator=g))
        self.eta_logit = torch.nn.Parameter(torch.logit(torch.tensor(float(eta_init))))

    def forward(self):
        w = torch.softmax(self.w_logit, 0)
        lam = torch.exp(self.log_lam)
        mu = torch.nn.functional.normalize(self.mu_raw, dim=1)
        lobes = torch.cat([w[:, None], lam[:, None], mu], 1).reshape(-1)
        return torch.cat([torch.sigmoid(self.eta_logit)[None], lobes])


class LogMaterials(torch.nn.Module):
    """Per-material parameters in the log domain of Eq. trainable_materials_1/2:
    sigma = exp(w_sigma), eps_r = 1 + exp(w_eps) (read-out vector v = 1, L = 1)."""

    def __init__(self, eps_r_init, sigma_init):
        super().__init__()
        eps_r_init = torch.as_tensor(eps_r_init, dtype=torch.float32)
        sigma_init = torch.as_tensor(sigma_init, dtype=torch.float32)
        self.w_eps = torch.nn.Parameter(torch.log(eps_r_init - 1.0))
        self.w_sigma = torch.nn.Parameter(torch.log(sigma_init))

    def forward(self):
        return 1.0 + torch.exp(self.w_eps), torch.exp(self.w_sigma)


class MaterialEmbeddings(torch.nn.Module):
    """The over-parametrised materials of Eq. trainable_materials_1/2: per material
    two embeddings w_1, w_2 in L dimensions and one read-out vector v shared by all
    materials, sigma = exp(v . w_1), eps_r = 1 + exp(v . w_2).  Initialised so that
    v . w reproduces the given starting values (v = 1 / sqrt(L), w = v value * sqrt(L)
    / L plus a small seeded spread that leaves v . w unchanged)."""

    def __init__(self, eps_r_init, sigma_init, L=30, seed=0, spread=0.1, S_init=None, K_x_init=None):
        super().__init__()
        eps_r_init = torch.as_tensor(eps_r_init, dtype=torch.float32)
        sigma_init = torch.as_tensor(sigma_init, dtype=torch.float32)
        M = eps_r_init.shape[0]
        g = torch.Generator().manual_seed(seed)
        v = torch.full((L,), L ** -0.5)

        def embed(value):
            # noise orthogonal to v, so that v . w starts at the requested value
            n = torch.randn(M, L, generator=g) * spread
            n -= (n @ v)[:, None] * v[None, :]
            return torch.nn.Parameter(value[:, None] * v[None, :] + n)
        self.v = torch.nn.Parameter(v)
        self.w_sigma = embed(torch.log(sigma_init))
        self.w_eps = embed(torch.log(eps_r_init - 1.0))
        # S = sigmoid(v . w_3), K_x = sigmoid(v . w_4) (Eq. trainable_materials_4), when asked for
        self.w_S = embed(torch.logit(torch.as_tensor(S_init, dtype=torch.float32))) if S_init is not None else None
        self.w_Kx = (embed(torch.logit(torch.as_tensor(K_x_init, dtype=torch.float32)))
                     if K_x_init is not None else None)

    def forward(self):
        return 1.0 + torch.exp(self.w_eps @ self.v), torch.exp(self.w_sigma @ self.v)

    def scattering(self):
        """(S, K_x) per material, sigmoid(v . w_3) and sigmoid(v . w_4)."""
        return torch.sigmoid(self.w_S @ self.v), torch.sigmoid(self.w_Kx @ self.v)


class EvalFieldsDiffuse(torch.autograd.Function):
    """a = eval_fields_diffuse(eps_r, sigma, scat) for diffuse paths, with
    rt_eval_fields_diffuse_backward as backward (scat is the (M, 8) table)."""

    @staticmethod
    def forward(fctx, eps_r, sigma, scat, ctx, paths, freq_hz, gain_tx=1.0, gain_rx=1.0):
        eps_r, sigma, scat = eps_r.contiguous(), sigma.contiguous(), scat.contiguous()
        a = api.eval_fields_diffuse(ctx, paths, eps_r, sigma, scat, freq_hz, gain_tx, gain_rx)
        fctx.save_for_backward(eps_r, sigma, scat)
        fctx.args = (ctx, paths, freq_hz, gain_tx, gain_rx)
        return a

    @staticmethod
    def backward(fctx, grad_a):
        eps_r, sigma, scat = fctx.saved_tensors
        ctx, paths, freq_hz, gain_tx, gain_rx = fctx.args
        ge, gs, gc = api.eval_fields_diffuse_backward(ctx, paths, eps_r, sigma, scat, freq_hz, grad_a.contiguous(),
                                                      gain_tx=gain_tx, gain_rx=gain_rx)
        return ge, gs, gc, None, None, None, None, None


class EvalFieldsDiffraction(torch.autograd.Function):
    """a = eval_fields_diffraction(eps_r, sigma) for diffraction paths (Sec. II-D Eq.
    diffraction), with rt_eval_fields_diffraction_backward as backward."""

    @staticmethod
    def forward(fctx, eps_r, sigma, ctx, paths, freq_hz, gain_tx=1.0, gain_rx=1.0, per_triangle=False):
        eps_r, sigma = eps_r.contiguous(), sigma.contiguous()
        a = api.eval_fields_diffraction(ctx, paths, eps_r, sigma, freq_hz, gain_tx, gain_rx, per_triangle)
        fctx.save_for_backward(eps_r, sigma)
        fctx.args = (ctx, paths, freq_hz, gain_tx, gain_rx, per_triangle)
        return a

    @staticmethod
    def backward(fctx, grad_a):
        eps_r, sigma = fctx.saved_tensors
        ctx, paths, freq_hz, gain_tx, gain_rx, per_triangle = fctx.args
        ge, gs, _ = api.eval_fields_diffraction_backward(ctx, paths, eps_r, sigma, freq_hz, grad_a.contiguous(),
                                                         gain_tx=gain_tx, gain_rx=gain_rx,
                                                         per_triangle=per_triangle)
        return ge, gs, None, None, None, None, None, None


class SpecularReduction(torch.autograd.Function):
    """a prod_b sqrt(1 - S_b^2) for specular paths (Eq. specular_reflection)."""

    @staticmethod
    def forward(fctx, a, scat, ctx, paths):
        scat = scat.contiguous()
        out = api.specular_reduction(ctx, paths, scat, a.contiguous())
        fctx.save_for_backward(out, scat)
        fctx.args = (ctx, paths)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        out, scat = fctx.saved_tensors
        ctx, paths = fctx.args
        ga, gc = api.specular_reduction_backward(ctx, paths, scat, out, grad_out.contiguous())
        return ga, gc, None, None


class RxMerge(torch.autograd.Function):
    """Per-receiver concatenation of two coefficient lists (rt_rx_merge), with
    rt_rx_split as backward."""

    @staticmethod
    def forward(fctx, x1, x2, off1, off2, ctx):
        out, _ = api.rx_merge(ctx, off1, off2, x1, x2)
        fctx.args = (ctx, off1, off2, x1.shape[0], x2.shape[0])
        return out

    @staticmethod
    def backward(fctx, g):
        ctx, off1, off2, n1, n2 = fctx.args
        g1, g2 = api.rx_split(ctx, off1, off2, g.contiguous(), n1, n2)
        return g1, g2, None, None, None


class ScatteringPattern(torch.nn.Module):
    """Per-material trainable scattering pattern of Sec. III-C: mixture weights
    (w_1, w_2, w_3) by a softmax and concentrations lambda_2, lambda_3 by an
    exponential; forward() returns (w (M, 3), lambda (M, 2))."""

    def __init__(self, n_materials, lam_init=5.0, w_init=(1 / 3, 1 / 3, 1 / 3)):
        super().__init__()
        w0 = torch.log(torch.as_tensor(w_init, dtype=torch.float32))
        self.w_logit = torch.nn.Parameter(w0.repeat(n_materials, 1))
        self.log_lam = torch.nn.Parameter(torch.full((n_materials, 2), float(torch.log(torch.tensor(lam_init)))))

    def forward(self):
        return torch.softmax(self.w_logit, 1), torch.exp(self.log_lam)


def pack_scattering(S, K_x, w, lam):
    """The (M, 8) float32 table of rt_eval_fields_diffuse: S, K_x, w_1..w_3, lambda_2, lambda_3, 0."""
    M = S.shape[0]
    return torch.cat([S[:, None], K_x[:, None], w, lam, torch.zeros(M, 1, dtype=S.dtype, device=S.device)],
                     1).float().contiguous()


def calibration_loss(ctx, paths, eps_r, sigma, target_power, rx_weight, freq_hz, f_center_hz, delta_f_hz, n_sub,
                     gain_tx=1.0, gain_rx=1.0, per_triangle=False):
    """One forward pass of Algorithm 1's inner loop: RT(p; Omega) -> CFR -> loss."""
    a = EvalFields.apply(eps_r, sigma, ctx, paths, freq_hz, gain_tx, gain_rx, per_triangle)
    return CfrPowerMSE.apply(a, paths.tau, paths.rx_offsets, target_power, rx_weight, ctx, f_center_hz, delta_f_hz,
                             n_sub)


class NeuralMaterialsFn(torch.autograd.Function):
    """(eps_r, sigma) per triangle = MLP(positional encoding of the centroid), with
    the BF16 weights rounded from the FP32 master weights; the gradient of the
    BF16 weights is applied to the masters (straight through the rounding)."""

    @staticmethod
    def forward(fctx, w, b, ctx, scene):
        w16 = w.detach().to(torch.bfloat16).contiguous()
        eps, sig, act = api.mlp_forward(ctx, scene, w16, b.detach())
        fctx.save_for_backward(w16, act, eps, sig)
        fctx.args = (ctx, scene)
        return eps, sig

    @staticmethod
    def backward(fctx, g_eps, g_sig):
        w16, act, eps, sig = fctx.saved_tensors
        ctx, scene = fctx.args
        if g_eps is None:
            g_eps = torch.zeros_like(eps)
        if g_sig is None:
            g_sig = torch.zeros_like(sig)
        gw, gb = api.mlp_backward(ctx, scene, w16, act, eps, sig, g_eps, g_sig)
        return gw, gb, None, None


class NeuralMaterials(torch.nn.Module):
    """Neural materials of Sec. III-D evaluated at the triangle centroids."""

    def __init__(self, Ws, bs, device="cuda"):
        super().__init__()
        w, b = api.pack_mlp(Ws, bs, device)
        self.w = torch.nn.Parameter(w)
        self.b = torch.nn.Parameter(b)

    def forward(self, ctx, scene):
        return NeuralMaterialsFn.apply(self.w, self.b, ctx, scene)
