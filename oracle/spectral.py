"""Pseudospectral pieces of the method (Section 2.1 and Eq. G of the paper). Test infrastructure.

Conventions (shared with the library only as documented conventions, no code):
  * grid J = {0..n-1}^d, flat index j0 + n*j1 (+ n^2*j2); numpy arrays of shape
    (n,)*d are indexed arr[j_{d-1}, ..., j_0];
  * Fourier grid K = {-n/2..n/2-1}^d stored in FFT order (index i <-> k = i for
    i < n/2, k = i - n otherwise), so the Nyquist row carries k = -n/2.
"""
from __future__ import annotations

import itertools

import numpy as np

FOUR_PI2 = 4.0 * np.pi * np.pi


def wavenumber_grid(d: int, n: int) -> np.ndarray:
    """|k|^2 for every k in K (Section 2.1), array of shape (n,)*d in FFT order."""
    k1 = np.fft.fftfreq(n, d=1.0 / n)  # 0,1,..,n/2-1,-n/2,..,-1
    ks = np.meshgrid(*([k1] * d), indexing="ij")
    return sum(k * k for k in ks)


def laplacian_symbol(d: int, n: int) -> np.ndarray:
    """Diagonal of L in Fourier space: 4 pi^2 |k|^2 (Section 2.1, definition of L)."""
    return FOUR_PI2 * wavenumber_grid(d, n)


def green_symbol(d: int, n: int, s: float) -> np.ndarray:
    """1 / (4 pi^2 |k|^2 - s), the Fourier diagonal of G = (L - s)^{-1} (Eq. G)."""
    den = laplacian_symbol(d, n) - s
    if np.any(den == 0.0):
        raise ValueError("L - s is singular: s equals 4 pi^2 |k|^2 for some k")
    return 1.0 / den


def resonance_gap(d: int, n: int, s: float) -> float:
    """min_k |kappa - |k|^2| / max(1, kappa), kappa = s / (4 pi^2).

    The paper assumes L - s invertible and perturbs s if needed (Section 2.2).
    Reading: s is perturbed when this gap is below 1e-6 (see helmholtz_shift).
    """
    kappa = s / FOUR_PI2
    return float(np.min(np.abs(kappa - wavenumber_grid(d, n))) / max(1.0, abs(kappa)))


def _perturb_if_resonant(d: int, n: int, s: float) -> float:
    # Section 2.2: "L - s ... invertible ... by perturbing s slightly if necessary".
    # Reading: shift s by 1e-3 * 4 pi^2 (i.e. kappa by 1e-3) until the gap exceeds 1e-6.
    while resonance_gap(d, n, s) < 1e-6:
        s += 1e-3 * FOUR_PI2
    return s


def helmholtz_shift(d: int, n: int, omega: float, c: np.ndarray):
    """Section 2.1: s = int omega^2/c^2, q = s - omega^2/c^2 (grid-mean quadrature).

    Returns (s, q) with q flat float64.  The sum (-s + q) = -omega^2/c^2 does not
    depend on s, so the perturbation of s for invertibility keeps the problem.
    """
    w2c2 = omega * omega / (np.asarray(c, dtype=np.float64) ** 2)
    s = _perturb_if_resonant(d, n, float(np.mean(w2c2)))
    return s, (s - w2c2).ravel()


def schrodinger_shift(d: int, n: int, ell: float, E: float, V: np.ndarray):
    """Section 2.1: s = int (l^2 E - l^2 V(l y)), q = l^2 V - l^2 E + s.

    The right-hand side of the rescaled equation is l^2 f (Eq. schr); the caller
    scales f.  Returns (s, q).
    """
    l2 = ell * ell
    pot = l2 * np.asarray(V, dtype=np.float64) - l2 * E
    s = _perturb_if_resonant(d, n, float(np.mean(-pot)))
    return s, (pot + s).ravel()


def apply_green(d: int, n: int, s: float, x: np.ndarray) -> np.ndarray:
    """G x = F^{-1} diag(1/(4 pi^2|k|^2 - s)) F x (Eq. G) via numpy FFTs.

    With the unitary F of Section 2.1 the two n^{-d/2} factors combine into the
    1/N that numpy's ifftn carries, so F^{-1} D F = ifftn(D * fftn(.)).
    """
    shape = (n,) * d
    X = np.asarray(x, dtype=np.complex128).reshape(shape)
    return np.fft.ifftn(green_symbol(d, n, s) * np.fft.fftn(X)).ravel()


def apply_operator(d: int, n: int, s: float, q: np.ndarray, x: np.ndarray) -> np.ndarray:
    """(I + G q) x, the integral operator of Section 2.2."""
    x = np.asarray(x, dtype=np.complex128)
    return x + apply_green(d, n, s, np.asarray(q) * x)


def green_kernel(d: int, n: int, s: float) -> np.ndarray:
    """Convolution kernel g with G(i, j) = g[(i - j) mod n] (Eq. G).

    g = F^{-1} applied to the symbol with the 1/N of the unitary pair; it is real
    because the symbol is real and even in k.  Returned with shape (n,)*d.
    """
    return np.fft.ifftn(green_symbol(d, n, s)).real


def dft_matrix(d: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Dense unitary DFT of Section 2.1 written out from its sum, for tiny n.

    Returns (F, kvec) where F[kk, jj] = n^{-d/2} exp(-2 pi i j.k / n), rows over
    K = {-n/2..n/2-1}^d (in lexicographic order of k, axis 0 fastest) and
    columns over J in flat order.  Used only to pin the FFT-based routines.
    """
    pts = list(itertools.product(range(n), repeat=d))  # (j_{d-1},...,j_0)
    J = np.array([p[::-1] for p in pts])  # axis-0 first
    kr = np.arange(-n // 2, n // 2)
    kpts = list(itertools.product(kr, repeat=d))
    K = np.array([p[::-1] for p in kpts])
    phase = -2j * np.pi * (K @ J.T) / n
    return np.exp(phase) / n ** (d / 2.0), K
