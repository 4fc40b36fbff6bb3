"""Pins of the oracle's Fourier-layer network (oracle/fno.py) against things other than
itself: numpy's FFT for the truncated spectral transform, central finite differences
for every parameter group of the hand-derived gradient, the closed form of Adam's
first step, translation equivariance and the standard normal distribution function."""
import numpy as np
import pytest
from scipy.stats import norm

import synthetic_media as sm
from oracle import fno as F

TINY = F.FnoDims(n=8, c_in=3, width=3, modes=2, layers=2, hidden=5, c_out=2)


def tiny_params(seed=0, D=TINY):
    th = sm.fno_initial_params(D.c_in, D.width, D.modes, D.layers, D.hidden, D.c_out, seed)
    # larger spectral weights than the initial ones, so the spectral branch matters
    parts = F.unpack(th.copy(), D)
    rng = np.random.default_rng(seed + 1)
    for l in range(D.layers):
        R = parts[f"R{l}"]
        parts[f"R{l}"] = (rng.standard_normal(R.shape) + 1j * rng.standard_normal(R.shape)) * 0.3
    return F.pack(parts, D)


def test_param_count_matches_generator():
    D = F.FnoDims(n=256)
    assert F.param_count(D) == sm.fno_initial_params().size
    assert F.param_count(TINY) == tiny_params().size
    th = tiny_params()
    assert np.array_equal(F.pack(F.unpack(th, TINY), TINY), th)


def test_spectral_conv_is_truncated_rfft2():
    """The explicit truncated DFT pair equals numpy's rfft2 / irfft2 with the modes outside
    kx < M, ky in [0, M) U [n - M, n) set to zero."""
    rng = np.random.default_rng(1)
    n, M, C = 16, 5, 3
    v = rng.standard_normal((2, C, n, n))
    V = F.spectral_forward(v, M)
    full = np.fft.rfft2(v)                    # [.., ky, kx], kx = 0 .. n/2
    ky = F.ky_list(n, M)
    assert np.allclose(V, full[:, :, ky, :M], rtol=0, atol=1e-12)
    R = rng.standard_normal((2 * M, M, C, C)) + 1j * rng.standard_normal((2 * M, M, C, C))
    Y = F.mix(V, R)
    pad = np.zeros((2, C, n, n // 2 + 1), dtype=complex)
    pad[:, :, ky, :M] = Y
    z_np = np.fft.irfft2(pad, s=(n, n))
    z = F.spectral_inverse(Y, n, 1.0 / n**2, 2.0 / n**2)
    assert np.allclose(z, z_np, rtol=0, atol=1e-12 * np.abs(z_np).max())


def test_network_spectral_branch_is_truncated_irfft2():
    """Inside the network: with the lift the identity, W_0 = 0 and b_0 = 0, layer 0's
    pre-activation is the spectral convolution alone, which must equal numpy's irfft2 of
    the truncated rfft2 spectrum mixed by R_0 (pins the weights the forward pass hands
    the inverse transform, including the doubling of the kx >= 1 modes)."""
    D = F.FnoDims(n=16, c_in=3, width=3, modes=5, layers=1, hidden=4, c_out=2)
    parts = F.unpack(tiny_params(8, D), D)
    rng = np.random.default_rng(9)
    parts["P"] = np.eye(3)
    parts["p"] = np.zeros(3)
    parts["W0"] = np.zeros((3, 3))
    parts["b0"] = np.zeros(3)
    R = rng.standard_normal(parts["R0"].shape) + 1j * rng.standard_normal(parts["R0"].shape)
    parts["R0"] = R
    a = rng.standard_normal((2, 3, D.n, D.n))
    _, cache = F.forward(F.pack(parts, D), a, D, keep=True)
    ky = F.ky_list(D.n, D.modes)
    pad = np.zeros((2, 3, D.n, D.n // 2 + 1), dtype=complex)
    pad[:, :, ky, :D.modes] = F.mix(np.fft.rfft2(a)[:, :, ky, :D.modes], R)
    z_np = np.fft.irfft2(pad, s=(D.n, D.n))
    assert np.allclose(cache["h"][0], z_np, rtol=0, atol=1e-12 * np.abs(z_np).max())


def test_gelu_is_x_times_normal_cdf():
    x = np.linspace(-6, 6, 101)
    assert np.allclose(F.gelu(x), x * norm.cdf(x), rtol=0, atol=1e-15)
    h = 1e-6
    assert np.allclose(F.gelu_prime(x), (F.gelu(x + h) - F.gelu(x - h)) / (2 * h), atol=1e-8)


def _loss_of(theta, a, t, D):
    return F.loss(F.forward(theta, a, D), t)[0]


def test_gradient_matches_finite_differences():
    """Central differences on every parameter group (a dropped term, a wrong sign or a
    transposed operand in any group's gradient fails here)."""
    D = TINY
    rng = np.random.default_rng(2)
    th = tiny_params(3)
    a = rng.standard_normal((2, D.c_in, D.n, D.n))
    t = rng.standard_normal((2, D.c_out, D.n, D.n))
    y, cache = F.forward(th, a, D, keep=True)
    L, dy, _ = F.loss(y, t)
    g = F.backward(th, cache, dy, D)
    eps = 1e-6
    off = 0
    for name, shape in F.param_shapes(D):
        sz = int(np.prod(shape))
        for j in rng.choice(sz, size=min(sz, 6), replace=False):
            e = np.zeros_like(th)
            e[off + j] = eps
            fd = (_loss_of(th + e, a, t, D) - _loss_of(th - e, a, t, D)) / (2 * eps)
            assert abs(fd - g[off + j]) <= 1e-7 + 1e-5 * abs(fd), (name, j, fd, g[off + j])
        off += sz
    # and a random direction through all parameters at once
    d = rng.standard_normal(th.size)
    fd = (_loss_of(th + eps * d, a, t, D) - _loss_of(th - eps * d, a, t, D)) / (2 * eps)
    assert abs(fd - g @ d) <= 1e-6 * abs(fd)


def test_translation_equivariance():
    """Every operation commutes with periodic shifts of the grid: shifting the input
    shifts the output (pins the twiddle indices of the transform pair)."""
    D = F.FnoDims(n=16, c_in=3, width=4, modes=3, layers=2, hidden=6, c_out=2)
    th = tiny_params(4, D)
    a = np.random.default_rng(5).standard_normal((1, D.c_in, D.n, D.n))
    y = F.forward(th, a, D)
    ys = F.forward(th, np.roll(a, (3, -5), axis=(2, 3)), D)
    assert np.allclose(ys, np.roll(y, (3, -5), axis=(2, 3)), rtol=0, atol=1e-12)


def test_adam_first_step_is_signed_lr():
    """After one step from zero moments, m_hat = g and v_hat = g^2, so every parameter
    moves by lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    th1, m, v = F.adam_step(th, np.zeros(50), np.zeros(50), g, 1, lr, eps=eps)
    assert np.allclose(th1 - th, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=0)
    # a second step with the same gradient keeps the same direction and size
    th2, _, _ = F.adam_step(th1, m, v, g, 2, lr, eps=eps)
    assert np.allclose(th2 - th1, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=0)


def test_loss_is_relative_error():
    rng = np.random.default_rng(7)
    t = rng.standard_normal((3, 2, 4, 4))
    L, dy, rel = F.loss(1.1 * t, t)
    assert np.allclose(rel, 0.1) and abs(L - 0.01) < 1e-15


def test_bf16_round():
    x = np.array([1.0, 1 + 2.0**-8, 1 + 2.0**-7, 1 + 3 * 2.0**-8, -3.14159, 1e-30])
    r = F.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0            # tie to even (down)
    assert r[2] == 1 + 2.0**-7                    # representable
    assert r[3] == 1 + 2.0**-6                    # tie to even (up)
    assert abs(r[4] + 3.140625) < 1e-12
    assert np.all(np.abs(r - x) <= 2.0**-8 * np.abs(x))   # half a unit in the last place
