"""CPU checks of the trainable parametrisations (host logic, no kernel call):
the material embeddings of Eq. trainable_materials_1/2 and the packed antenna
pattern of Sec. III-B."""
import numpy as np
import torch

from paper_2311_18558_gb300.autograd import AntennaPattern, LogMaterials, MaterialEmbeddings


def test_embeddings_start_at_given_values():
    eps0 = np.array([2.5, 4.0, 7.0])
    sig0 = np.array([1e-3, 0.05, 0.8])
    for L in (1, 4, 30):
        m = MaterialEmbeddings(eps0, sig0, L=L, seed=L)
        eps, sig = m()
        np.testing.assert_allclose(eps.detach().numpy(), eps0, rtol=1e-5)
        np.testing.assert_allclose(sig.detach().numpy(), sig0, rtol=1e-5)
        assert m.w_eps.shape == (3, L) and m.v.shape == (L,)


def test_embeddings_share_the_readout():
    # the read-out vector v is shared: its gradient collects every material's term,
    # and with L = 1, v = 1 the module is the log parametrisation
    m = MaterialEmbeddings([3.0, 5.0], [0.1, 0.2], L=8, seed=1)
    eps, sig = m()
    (eps.sum() + sig.sum()).backward()
    ge = (eps.detach() - 1.0)[:, None] * m.v.detach()[None, :]
    np.testing.assert_allclose(m.w_eps.grad.numpy(), ge.numpy(), rtol=1e-6)
    gv = ((eps.detach() - 1.0)[:, None] * m.w_eps.detach()).sum(0) + (sig.detach()[:, None] * m.w_sigma.detach()).sum(0)
    np.testing.assert_allclose(m.v.grad.numpy(), gv.numpy(), rtol=1e-5)
    one = MaterialEmbeddings([3.0, 5.0], [0.1, 0.2], L=1)
    log = LogMaterials(np.array([3.0, 5.0]), np.array([0.1, 0.2]))
    for x, y in zip(one(), log()):
        np.testing.assert_allclose(x.detach().numpy(), y.detach().numpy(), rtol=1e-6)


def test_antenna_pattern_packing():
    pat = AntennaPattern(n_lobes=3, lam_init=2.0, eta_init=0.9, seed=0)
    p = pat().detach().numpy()
    assert p.shape == (1 + 5 * 3,)
    lob = p[1:].reshape(3, 5)
    np.testing.assert_allclose(p[0], 0.9, rtol=1e-6)
    np.testing.assert_allclose(lob[:, 0].sum(), 1.0, rtol=1e-6)
    np.testing.assert_allclose(lob[:, 1], 2.0, rtol=1e-6)
    np.testing.assert_allclose(np.linalg.norm(lob[:, 2:5], axis=1), 1.0, rtol=1e-6)
    assert torch.is_tensor(pat()) and pat().requires_grad
