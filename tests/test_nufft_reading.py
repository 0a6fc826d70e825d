"""The non-uniform FFT that evaluates the CFR of receivers with many paths on the
GPU, checked as mathematics in FP64 on the CPU.  The CFR itself is the direct
sum of Sec. II-A, and the oracle computes it that way.  On the GPU, receivers
with more than 4096 paths go through a non-uniform FFT instead, so its parameters
must keep the approximation far inside the parity tolerance:
  an exponential-of-semicircle kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)),
  W = 8 cells wide, beta = 2.3 W, on an oversampled grid of M = 2N cells, with the
  deconvolution M phi_hat(n) = W/2 int_{-1}^{1} phi(z) cos(pi n W z / M) dz
  taken by 256-node Gauss-Legendre quadrature.
For one path the error per entry is about 4e-7 of |c|, the kernel's aliasing.  For
thousands of paths the errors partly cancel, and the error stays below 1e-7 of
sum_i |c_i|, whether the delays spread over the whole grid or cluster on a few
cells.  This is written from the method's definition; it shares nothing with the
CUDA code."""
import numpy as np
import pytest

W = 8
BETA = 2.3 * W


def _phi(z):
    q = 1.0 - z * z
    return np.where(q > 0, np.exp(BETA * (np.sqrt(np.clip(q, 0.0, None)) - 1.0)), 0.0)


def _exact(c, x, N):
    n = np.arange(N) - N // 2
    return (c[None, :] * np.exp(-2j * np.pi * n[:, None] * x[None, :])).sum(1)


def _nufft(c, x, N, nodes=256):
    M = 2 * N
    n = np.arange(N) - N // 2
    b = np.zeros(M, complex)
    xm = M * x
    l0 = np.ceil(xm - W / 2).astype(np.int64)
    for k in range(W):
        l = l0 + k
        np.add.at(b, l % M, c * _phi((l - xm) * 2.0 / W))
    B = np.fft.fft(b)   # sum_l b[l] exp(-j 2 pi k l / M)
    zq, wq = np.polynomial.legendre.leggauss(nodes)
    mphi = 0.5 * W * (wq[None, :] * _phi(zq)[None, :] * np.cos(np.pi * n[:, None] * W * zq[None, :] / M)).sum(1)
    return B[n % M] / mphi


@pytest.mark.parametrize("N", [256, 1024, 4096])
@pytest.mark.parametrize("spread", ["uniform", "clustered"])
def test_many_paths_error_below_1e7_of_total_magnitude(N, spread):
    rng = np.random.default_rng(N + (0 if spread == "uniform" else 1))
    P = 3000
    if spread == "uniform":
        x = rng.uniform(0.0, 1.0, P)
    else:   # indoor-like delays, 10-200 ns at 48.8 kHz spacing: a few cells of the grid
        x = (48828.125 * rng.uniform(10e-9, 200e-9, P)) % 1.0
    c = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    err = np.abs(_nufft(c, x, N) - _exact(c, x, N)).max() / np.abs(c).sum()
    assert err < 1e-7


def test_deconvolution_quadrature_converged():
    # 256 nodes against 512: the deconvolution factors agree to FP64 rounding
    N, M = 1024, 2048
    n = np.arange(N) - N // 2
    vals = []
    for nodes in (256, 512):
        zq, wq = np.polynomial.legendre.leggauss(nodes)
        vals.append((wq[None, :] * _phi(zq)[None, :] * np.cos(np.pi * n[:, None] * W * zq[None, :] / M)).sum(1))
    assert np.max(np.abs(vals[0] - vals[1]) / np.abs(vals[1])) < 1e-12


@pytest.mark.parametrize("x", [37.0 / 2048, 0.0, 0.5, 0.3, 0.999])
def test_lone_path_error_below_5e7(x):
    # on a grid cell (l0 = M x - W/2, offset -W/2) or between cells
    N = 1024
    c = np.array([0.5 - 0.25j])
    err = np.abs(_nufft(c, np.array([x]), N) - _exact(c, np.array([x]), N)).max() / np.abs(c).sum()
    assert err < 5e-7
