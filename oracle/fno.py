"""Fourier-layer network for the GMRES initial guess: plain FP64 forward pass, backward
pass and Adam step.  TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; this is the Fourier neural operator of Li et al.
(Fourier Neural Operator for Parametric Partial Differential Equations, ICLR 2021,
Section 4, the 2D network), used to supply the starting vector of the solve, with the
optimiser of Kingma and Ba (Adam, ICLR 2015, Algorithm 1).  Everything below is the
plain definition written out with dense numpy arrays: explicit truncated DFT
matrices, a loop over layers, and hand-derived gradients (no autodiff).

Tensors are (B, C, n, n) float64 arrays whose last axis is j0 and second-to-last j1,
i.e. the flat index j0 + n j1 of the solver's grids in C order.

Network (L Fourier layers, width W, M modes per axis, hidden width H):
  v_0     = P a + p                                  (pointwise lift, c_in -> W)
  h_l     = W_l v_l + b_l + K_l v_l                  (l = 0 .. L-1)
  v_{l+1} = gelu(h_l)  for l < L-1,  v_L = h_{L-1}   (no activation on the last layer)
  e       = Q1 v_L + c1,  y = Q2 gelu(e) + c2        (projection W -> H -> c_out)
Spectral convolution K v (modes kx = 0..M-1 along j0, ky in {0..M-1} U {n-M..n-1}
along j1, R_l(ky, kx) a complex W x W matrix per mode):
  V(ky, kx)_i = sum_{j0, j1} v_i(j1, j0) exp(-2 pi i (kx j0 + ky j1) / n)
  Y(ky, kx)_o = sum_i V(ky, kx)_i R(ky, kx)[i, o]
  (K v)_o(j1, j0) = (1/n^2) sum_{ky, kx} c_kx Re(Y(ky, kx)_o exp(+2 pi i (kx j0 + ky j1) / n))
with c_0 = 1 and c_kx = 2 for kx >= 1: the real inverse transform of the truncated,
Hermitian-completed spectrum (numpy's irfft2 of the zero-padded modes).
gelu(x) = x Phi(x), Phi the standard normal distribution function.

Loss: the mean over the batch of the squared relative error ||y_b - t_b||^2 / ||t_b||^2.

Parameter vector (float64, this order; matrices row-major, complex entries as
(re, im) pairs):
  P [W, c_in], p [W];
  per layer: R [2M, M, W, W] complex (ky index: 0..M-1 then n-M..n-1), W_l [W, W], b_l [W];
  Q1 [H, W], c1 [H], Q2 [c_out, H], c2 [c_out].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import erf


@dataclass(frozen=True)
class FnoDims:
    n: int
    c_in: int = 3
    width: int = 32
    modes: int = 16
    layers: int = 4
    hidden: int = 128
    c_out: int = 2


def param_shapes(D: FnoDims) -> list[tuple[str, tuple[int, ...]]]:
    """Names and shapes in the order of the flat parameter vector (complex R counted
    as a trailing axis of 2)."""
    W, M = D.width, D.modes
    out = [("P", (W, D.c_in)), ("p", (W,))]
    for l in range(D.layers):
        out += [(f"R{l}", (2 * M, M, W, W, 2)), (f"W{l}", (W, W)), (f"b{l}", (W,))]
    out += [("Q1", (D.hidden, W)), ("c1", (D.hidden,)), ("Q2", (D.c_out, D.hidden)),
            ("c2", (D.c_out,))]
    return out


def param_count(D: FnoDims) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(D)))


def unpack(theta: np.ndarray, D: FnoDims) -> dict:
    """Views of the flat vector; R_l returned as complex arrays [2M, M, W, W]."""
    out, off = {}, 0
    for name, shape in param_shapes(D):
        sz = int(np.prod(shape))
        a = theta[off:off + sz].reshape(shape)
        out[name] = a[..., 0] + 1j * a[..., 1] if name.startswith("R") else a
        off += sz
    return out


def pack(parts: dict, D: FnoDims) -> np.ndarray:
    chunks = []
    for name, shape in param_shapes(D):
        a = parts[name]
        if name.startswith("R"):
            a = np.stack([a.real, a.imag], axis=-1)
        chunks.append(np.asarray(a, dtype=np.float64).reshape(-1))
    return np.concatenate(chunks)


# ------------------------------------------------------------------ elementwise pieces
def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_prime(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


# ------------------------------------------------------------------ truncated DFT
def ky_list(n: int, M: int) -> np.ndarray:
    return np.concatenate([np.arange(M), np.arange(n - M, n)])


def dft_mats(n: int, M: int):
    """Fx[kx, j0] = exp(-2 pi i kx j0 / n) (M x n), Fy[ky', j1] = exp(-2 pi i ky j1 / n) (2M x n)."""
    j = np.arange(n)
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(M), j) / n)
    Fy = np.exp(-2j * np.pi * np.outer(ky_list(n, M), j) / n)
    return Fx, Fy


def spectral_forward(v: np.ndarray, M: int) -> np.ndarray:
    """V[b, c, ky', kx] = sum_{j1, j0} v[b, c, j1, j0] Fy[ky', j1] Fx[kx, j0]."""
    n = v.shape[-1]
    Fx, Fy = dft_mats(n, M)
    return np.einsum("bcyx,ky,qx->bckq", v, Fy, Fx, optimize=True)


def spectral_inverse(Y: np.ndarray, n: int, w0: float, w1: float) -> np.ndarray:
    """z[b, c, j1, j0] = Re sum_{ky', kx} w_kx Y[b, c, ky', kx] conj(Fy[ky', j1]) conj(Fx[kx, j0])
    with w_0 = w0 and w_kx = w1 for kx >= 1 (the forward pass uses 1/n^2 and 2/n^2)."""
    M = Y.shape[-1]
    Fx, Fy = dft_mats(n, M)
    w = np.full(M, w1)
    w[0] = w0
    return np.einsum("bckq,ky,qx,q->bcyx", Y, Fy.conj(), Fx.conj(), w, optimize=True).real


def mix(V: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Y[b, o, k] = sum_i V[b, i, k] R[k][i, o] for every kept mode k = (ky', kx)."""
    return np.einsum("bikq,kqio->bokq", V, R)


def pointwise(Wm: np.ndarray, x: np.ndarray, bias=None) -> np.ndarray:
    y = np.einsum("oi,biyx->boyx", Wm, x)
    if bias is not None:
        y = y + bias[None, :, None, None]
    return y


# ------------------------------------------------------------------ network
def forward(theta: np.ndarray, a: np.ndarray, D: FnoDims, keep: bool = False):
    """Network output y (B, c_out, n, n) for inputs a (B, c_in, n, n); with keep=True
    also the intermediate values the backward pass needs."""
    P = unpack(theta, D)
    n, M = D.n, D.modes
    cache = {"a": a, "v": [], "V": [], "h": []}
    v = pointwise(P["P"], a, P["p"])
    for l in range(D.layers):
        V = spectral_forward(v, M)
        z = spectral_inverse(mix(V, P[f"R{l}"]), n, 1.0 / n**2, 2.0 / n**2)
        h = pointwise(P[f"W{l}"], v, P[f"b{l}"]) + z
        cache["v"].append(v)
        cache["V"].append(V)
        cache["h"].append(h)
        v = gelu(h) if l < D.layers - 1 else h
    e = pointwise(P["Q1"], v, P["c1"])
    ge = gelu(e)
    y = pointwise(P["Q2"], ge, P["c2"])
    cache.update(vL=v, e=e, ge=ge)
    return (y, cache) if keep else y


def loss(y: np.ndarray, t: np.ndarray):
    """Mean squared relative error and its gradient with respect to y."""
    B = y.shape[0]
    diff = y - t
    num = np.sum(diff.reshape(B, -1) ** 2, axis=1)
    den = np.sum(t.reshape(B, -1) ** 2, axis=1)
    L = float(np.mean(num / den))
    dy = 2.0 * diff / (B * den[:, None, None, None])
    return L, dy, np.sqrt(num / den)


def backward(theta: np.ndarray, cache: dict, dy: np.ndarray, D: FnoDims) -> np.ndarray:
    """Gradient of the loss with respect to theta, given dL/dy (chain rule, layer by layer)."""
    P = unpack(theta, D)
    n = D.n
    G = {}
    # projection
    G["Q2"] = np.einsum("boyx,biyx->oi", dy, cache["ge"])
    G["c2"] = dy.sum(axis=(0, 2, 3))
    dge = np.einsum("oi,boyx->biyx", P["Q2"], dy)
    de = dge * gelu_prime(cache["e"])
    G["Q1"] = np.einsum("boyx,biyx->oi", de, cache["vL"])
    G["c1"] = de.sum(axis=(0, 2, 3))
    dv = np.einsum("oi,boyx->biyx", P["Q1"], de)
    for l in reversed(range(D.layers)):
        h, v, V = cache["h"][l], cache["v"][l], cache["V"][l]
        dh = dv * gelu_prime(h) if l < D.layers - 1 else dv
        G[f"W{l}"] = np.einsum("boyx,biyx->oi", dh, v)
        G[f"b{l}"] = dh.sum(axis=(0, 2, 3))
        # z = Re(sum w Y e^{+i theta}): dL/dRe Y + i dL/dIm Y = w * (forward DFT of dh)
        w = np.full(D.modes, 2.0 / n**2)
        w[0] = 1.0 / n**2
        dY = spectral_forward(dh, D.modes) * w[None, None, None, :]
        # Y = V R: dR[k][i, o] = sum_b dY[b, o, k] conj(V[b, i, k]); dV = sum_o dY conj(R)
        G[f"R{l}"] = np.einsum("bokq,bikq->kqio", dY, V.conj())
        dV = np.einsum("bokq,kqio->bikq", dY, P[f"R{l}"].conj())
        # V = sum v e^{-i theta} (v real): dL/dv = Re sum dV e^{+i theta}
        dv = np.einsum("oi,boyx->biyx", P[f"W{l}"], dh) + spectral_inverse(dV, n, 1.0, 1.0)
    G["P"] = np.einsum("boyx,biyx->oi", dv, cache["a"])
    G["p"] = dv.sum(axis=(0, 2, 3))
    return pack(G, D)


def adam_step(theta, m, v, g, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) with bias-corrected moments; step >= 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1**step)
    vh = v / (1.0 - beta2**step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (8-bit significand), ties to even, as
    float64.  The parity tests give the oracle the weights the kernels actually use."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
