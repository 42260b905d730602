"""Pins of the finite-difference gradients and the flat adjoint (CPU)."""
import math

import numpy as np

from oracle import flat, grad
from synth import grf, vector_noise


def test_grad_symbols():
    shape = (16, 12, 8)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = (2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny, 2 * np.pi * 5 / nz)
    th = k[0] * x + k[1] * y + k[2] * z
    u = np.sin(th)
    g4, g2 = grad.grad4(u), grad.grad2(u)
    for a in range(3):
        s4 = (8 * math.sin(k[a]) - math.sin(2 * k[a])) / 6.0
        np.testing.assert_allclose(g4[a], s4 * np.cos(th), atol=1e-13)
        np.testing.assert_allclose(g2[a], math.sin(k[a]) * np.cos(th), atol=1e-13)


def test_grad_transposes():
    rng = np.random.default_rng(4)
    u = rng.standard_normal((8, 12, 16))
    w = rng.standard_normal((3, 8, 12, 16))
    assert abs(float((grad.grad4(u) * w).sum()) - float((u * grad.grad4_T(w)).sum())) < 1e-11
    assert abs(float((grad.grad2(u) * w).sum()) - float((u * grad.grad2_T(w)).sum())) < 1e-11


def test_flat_loss_gradient_against_differences():
    # loss = sum(w * grad4(phi)), phi = zero-mean solve of A phi = F - mean(F);
    # dL/dF = P A^+ P grad4^T w (P the mean projection); L is linear in F
    n = 16
    F = grf(n, 4)
    w = vector_noise(n, 5).astype(np.float64)
    g = flat.fft_solve(grad.grad4_T(w))
    g -= g.mean()
    rng = np.random.default_rng(6)

    def loss(FF):
        return float((w * grad.grad4(flat.fft_solve(FF))).sum())

    for _ in range(4):
        v = rng.standard_normal(F.shape)
        fd = (loss(F + 1e-3 * v) - loss(F - 1e-3 * v)) / 2e-3
        assert abs(fd - float((g * v).sum())) < 1e-9 * max(1.0, abs(fd))
