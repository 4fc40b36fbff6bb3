"""Pins of the oracle's pseudospectral pieces against the definitions of Section 2.1-2.2.

The FFT-based routines are compared with dense matrices written out from the
unitary DFT's sum (Section 2.1) on tiny grids, and with closed forms.
"""
import numpy as np
import pytest

import oracle as O
import synthetic_media as sm


def _dense_ops(d, n, s):
    F, K = O.dft_matrix(d, n)
    k2 = np.sum(K.astype(float) ** 2, axis=1)
    Fi = F.conj().T
    L = Fi @ np.diag(4 * np.pi ** 2 * k2) @ F
    G = Fi @ np.diag(1.0 / (4 * np.pi ** 2 * k2 - s)) @ F
    return F, L, G


@pytest.mark.parametrize("d,n", [(2, 4), (2, 6), (3, 4)])
def test_dft_matrix_unitary(d, n):
    F, _ = O.dft_matrix(d, n)
    assert np.allclose(F.conj().T @ F, np.eye(n ** d), atol=1e-13)


@pytest.mark.parametrize("d,n", [(2, 4), (2, 6), (3, 4)])
def test_green_apply_matches_dense_definition(d, n):
    s = 4 * np.pi ** 2 * 1.37
    _, L, G = _dense_ops(d, n, s)
    x = sm.random_complex_vector(n ** d, 1)
    ref = G @ x
    got = O.apply_green(d, n, s, x)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # G is the inverse of L - s (Eq. G)
    assert np.linalg.norm(G @ ((L - s * np.eye(n ** d)) @ x) - x) <= 1e-12 * np.linalg.norm(x)


def test_green_kernel_is_the_convolution_kernel():
    d, n, s = 2, 6, 4 * np.pi ** 2 * 0.61
    _, _, G = _dense_ops(d, n, s)
    g = O.green_kernel(d, n, s)
    pts = np.array([(j % n, j // n) for j in range(n * n)])
    Gc = np.empty((n * n, n * n))
    for i in range(n * n):
        for j in range(n * n):
            dd = (pts[i] - pts[j]) % n
            Gc[i, j] = g[dd[1], dd[0]]
    assert np.allclose(Gc, G.real, atol=1e-14, rtol=0)
    assert np.max(np.abs(G.imag)) < 1e-14
    # real and even: g(m) = g(-m)
    assert np.allclose(g, np.roll(np.flip(g), 1, axis=(0, 1)), atol=1e-15)


def test_integral_reformulation_identity():
    """(L - s)(I + G q) u = (L - s + q) u (Section 2.2)."""
    d, n = 2, 6
    s = 4 * np.pi ** 2 * 2.3
    _, L, G = _dense_ops(d, n, s)
    rng = np.random.default_rng(3)
    q = rng.standard_normal(n * n) * 50
    u = sm.random_complex_vector(n * n, 4)
    lhs = (L - s * np.eye(n * n)) @ O.apply_operator(d, n, s, q, u)
    rhs = (L - s * np.eye(n * n) + np.diag(q)) @ u
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


@pytest.mark.parametrize("d,n,k0", [(2, 16, (3, -5)), (2, 16, (-8, 2)), (3, 8, (1, -4, 2))])
def test_plane_wave_closed_form(d, n, k0):
    """G e^{2 pi i k0.x} = e^{2 pi i k0.x} / (4 pi^2 |k0|^2 - s) (Eq. G, diagonal in Fourier)."""
    s = 4 * np.pi ** 2 * 7.31
    x = sm.grid_coords(d, n)
    f = np.exp(2j * np.pi * sum(k0[a] * x[a] for a in range(d))).ravel()
    got = O.apply_green(d, n, s, f)
    ref = f / (4 * np.pi ** 2 * sum(k * k for k in k0) - s)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_helmholtz_shift_split():
    d, n = 2, 32
    c = sm.grf_velocity(d, n, 0.1, 5)
    omega = 2 * np.pi * 3.3
    s, q = O.helmholtz_shift(d, n, omega, c)
    assert abs(np.mean(q)) < 1e-10 * s
    assert np.allclose(-s + q, -(omega ** 2) / c ** 2, rtol=1e-14, atol=1e-9)


def test_helmholtz_shift_perturbs_resonant_s():
    """c = 1, omega = 2 pi 5: s / 4 pi^2 = 25 = |(3,4)|^2 makes L - s singular."""
    d, n = 2, 32
    c = np.ones(n * n)
    omega = 2 * np.pi * 5
    s, q = O.helmholtz_shift(d, n, omega, c)
    assert O.resonance_gap(d, n, s) >= 1e-6
    assert s != omega ** 2
    assert np.allclose(-s + q, -(omega ** 2), rtol=0, atol=1e-9)


def test_schrodinger_shift_split():
    d, n, ell, E = 2, 32, 4.0, 3.0
    V = sm.lattice_wells_potential(d, n, ell, 11)
    s, q = O.schrodinger_shift(d, n, ell, E, V)
    assert abs(np.mean(q)) < 1e-10 * abs(s)
    assert np.allclose(-s + q, ell ** 2 * V - ell ** 2 * E, rtol=1e-14, atol=1e-9)
