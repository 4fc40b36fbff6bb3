"""Sparsifying stencil Q and the truncated C = Q G (Section 2.3 of the paper). Test infrastructure.

Sets (Section 2.3, the partition of J at the leaf level of nested dissection):
a point p belongs to the set type Z = {a : p_a mod b == 0}.  Z = {} is a cell
(the (b-1)^d interior of a leaf box), |Z| = 1 an edge (2D) or face (3D),
|Z| = 2 in 3D an edge, |Z| = d a vertex.  Types are numbered t = sum_{a in Z} 2^a,
so t = 0 is the cell and t = 2^d - 1 the vertex; the reading that each
orientation of an edge/face gets its own T is taken (the paper writes one T
per kind and remarks that T does not depend on the translate).

Canonical instance of type t: the translate whose leaf box has origin 0,
  S_t     = {p : p_a = 0 for a in Z, 1 <= p_a <= b-1 otherwise},
  gamma_t = {p : -1 <= p_a <= 1 for a in Z, 0 <= p_a <= b otherwise}  (Section 2.3, gamma),
  beta_t  = gamma_t minus S_t.
Every list of points is ordered with axis 0 fastest (lexicographic in
(p_{d-1}, ..., p_0)); T_t has rows in S order and columns in beta order, Q_t
and C_t have rows in S order and columns in gamma order.
"""
from __future__ import annotations

import itertools

import numpy as np

from .spectral import green_kernel


def set_types(d: int) -> list[tuple[int, ...]]:
    """Z for t = 0 .. 2^d-1 (bit a of t set <=> axis a in Z)."""
    return [tuple(a for a in range(d) if (t >> a) & 1) for t in range(1 << d)]


def _box_points(ranges_per_axis) -> np.ndarray:
    """Cartesian product, rows = points (p_0..p_{d-1}), axis 0 fastest."""
    rev = list(reversed(ranges_per_axis))
    pts = [p[::-1] for p in itertools.product(*rev)]
    return np.array(pts, dtype=np.int64).reshape(len(pts), len(ranges_per_axis))


def canonical_set(d: int, b: int, t: int) -> np.ndarray:
    """S_t of Section 2.3 for the leaf box at origin 0 (cell, face, edge or vertex)."""
    return _box_points([[0] if (t >> a) & 1 else list(range(1, b)) for a in range(d)])


def canonical_gamma(d: int, b: int, t: int) -> np.ndarray:
    """gamma(S_t): points within l-infinity distance 1 of S_t (Section 2.3), unwrapped."""
    return _box_points([list(range(-1, 2)) if (t >> a) & 1 else list(range(0, b + 1))
                        for a in range(d)])


def canonical_beta(d: int, b: int, t: int) -> np.ndarray:
    """beta(S_t) = gamma(S_t) minus S_t, in gamma order."""
    S = {tuple(p) for p in canonical_set(d, b, t)}
    return np.array([p for p in canonical_gamma(d, b, t) if tuple(p) not in S], dtype=np.int64)


def flat_index(pts: np.ndarray, n: int) -> np.ndarray:
    """Periodic flat index sum_a (p_a mod n) n^a."""
    pts = np.mod(pts, n)
    return sum(pts[:, a] * n ** a for a in range(pts.shape[1]))


def green_block(g: np.ndarray, n: int, rows: np.ndarray, cols_flat: np.ndarray) -> np.ndarray:
    """Dense G(rows, cols) with G(i, j) = g[(i - j) mod n] (Eq. G as a convolution).

    rows: (r, d) integer points; cols_flat: flat indices of the column points.
    """
    d = rows.shape[1]
    gf = g.ravel()
    col_pts = np.stack([(cols_flat // n ** a) % n for a in range(d)], axis=1)
    out = np.empty((rows.shape[0], cols_flat.size), dtype=np.float64)
    for r in range(rows.shape[0]):
        diff = np.mod(rows[r][None, :] - col_pts, n)
        out[r] = gf[sum(diff[:, a] * n ** a for a in range(d))]
    return out


def matlab_pinv(B: np.ndarray):
    """Pseudoinverse with Matlab's default cutoff (the paper's code is Matlab, Section 3).

    Reading: singular values at or below max(size(B)) * eps(sigma_max) are dropped,
    eps(x) = 2^(floor(log2 x) - 52).  Returns (pinv, rank, singular values).
    """
    U, sig, Vh = np.linalg.svd(B, full_matrices=False)
    if sig.size == 0 or sig[0] == 0.0:
        return np.zeros((B.shape[1], B.shape[0])), 0, sig
    tol = max(B.shape) * 2.0 ** (np.floor(np.log2(sig[0])) - 52)
    r = int(np.sum(sig > tol))
    pinv = (Vh[:r].T / sig[:r]) @ U[:, :r].T
    return pinv, r, sig


def _q_and_c(g: np.ndarray, n: int, S: np.ndarray, gam: np.ndarray, T: np.ndarray):
    """Q(S, gamma) = [I, -T] on the columns (S, beta) in gamma order and
    C(S, gamma) = Q(S, gamma) G(gamma, gamma) (Section 2.3)."""
    S_set = {tuple(p) for p in S}
    in_S = np.array([tuple(p) in S_set for p in gam])
    Qg = np.zeros((S.shape[0], gam.shape[0]))
    Qg[:, np.nonzero(in_S)[0]] = np.eye(S.shape[0])
    Qg[:, np.nonzero(~in_S)[0]] = -T
    Ggg = green_block(g, n, gam, flat_index(gam, n))
    return Qg, Qg @ Ggg


def tables_from_T(d: int, n: int, b: int, s: float, Ts: list) -> list[dict]:
    """The set-type tables of Section 2.3 from given T_S (one |S| x |beta| array per
    type t, rows in S order, columns in beta order): Q(S, gamma) = [I, -T_S] and
    C(S, gamma) = Q(S, gamma) G(gamma, gamma), as stencil_tables forms them."""
    g = green_kernel(d, n, s)
    out = []
    for t, T in enumerate(Ts):
        S = canonical_set(d, b, t)
        gam = canonical_gamma(d, b, t)
        Q, C = _q_and_c(g, n, S, gam, np.asarray(T, dtype=np.float64))
        out.append(dict(t=t, S=S, gamma=gam, beta=canonical_beta(d, b, t), T=T, Q=Q, C=C))
    return out


def stencil_tables(d: int, n: int, b: int, s: float, origin=None, types=None,
                   keep_blocks: bool = False) -> list[dict]:
    """T_t, Q_t(S, gamma) and C_t(S, gamma) for every set type (Section 2.3).

    For each type: A = G(S, gamma^c), B = G(beta, gamma^c),
    T = A pinv(B), Q(S, gamma) = [I, -T] on columns (S, beta) placed in gamma
    order, C(S, gamma) = Q(S, gamma) G(gamma, gamma).  `origin` translates the
    instance (the paper notes T is the same for every translate; a test pins it).
    Each entry also carries the pinv rank, the singular values of B and the
    annihilation ratio ||A - T B||_F / ||A||_F; with keep_blocks the dense A, B
    and A - T B are kept too.
    """
    if n % b or n // b < 2:
        raise ValueError("need n divisible by b with n/b >= 2")
    g = green_kernel(d, n, s)
    N = n ** d
    o = np.zeros(d, dtype=np.int64) if origin is None else np.asarray(origin, dtype=np.int64)
    out = []
    for t in (range(1 << d) if types is None else types):
        S = canonical_set(d, b, t) + o
        gam = canonical_gamma(d, b, t) + o
        beta = canonical_beta(d, b, t) + o
        gam_flat = flat_index(gam, n)
        mask = np.ones(N, dtype=bool)
        mask[gam_flat] = False
        comp = np.nonzero(mask)[0]
        A = green_block(g, n, S, comp)
        B = green_block(g, n, beta, comp)
        Bp, rank, sig = matlab_pinv(B)
        T = A @ Bp
        Qg, C = _q_and_c(g, n, S, gam, T)
        resid = A - T @ B
        tab = dict(t=t, S=S - o, gamma=gam - o, beta=beta - o, T=T, Q=Qg, C=C,
                   rank=rank, sigma=sig,
                   ratio=float(np.linalg.norm(resid) / np.linalg.norm(A)))
        if keep_blocks:
            tab.update(A=A, B=B, resid=resid)
        out.append(tab)
    return out


def pointwise_stencil_tables(d: int, n: int, b: int, s: float) -> list[dict]:
    """The per-point sparsifying stencils mu(j) = gamma({j}) (the construction the
    paper's set stencils generalise, Section 2.3): for every point j of every set
    type, independently, A = G(j, gamma({j})^c), B = G(beta_j, gamma({j})^c) with
    gamma({j}) the 3^d neighbourhood of j and beta_j = gamma({j}) minus j,
    T_j = A pinv(B), Q(j, gamma({j})) = [1, -T_j], C(j, gamma({j})) =
    Q(j, gamma({j})) G(gamma({j}), gamma({j})).  Returned in the set tables' layout
    (rows in S order, columns in gamma(S) order, zero outside gamma({j}))."""
    g = green_kernel(d, n, s)
    N = n ** d
    offs = _box_points([range(-1, 2)] * d)  # gamma({0}), axis 0 fastest
    out = []
    for t in range(1 << d):
        S = canonical_set(d, b, t)
        gam = canonical_gamma(d, b, t)
        col = {tuple(p): i for i, p in enumerate(gam)}
        Q = np.zeros((S.shape[0], gam.shape[0]))
        C = np.zeros_like(Q)
        rank = None
        for a, p in enumerate(S):
            gj = p + offs
            gj_flat = flat_index(gj, n)
            mask = np.ones(N, dtype=bool)
            mask[gj_flat] = False
            comp = np.nonzero(mask)[0]
            centre = np.all(gj == p, axis=1)
            beta = gj[~centre]
            A = green_block(g, n, p[None, :], comp)
            Bm = green_block(g, n, beta, comp)
            Bp, rank, _ = matlab_pinv(Bm)
            Tj = (A @ Bp)[0]
            qrow = np.zeros(gj.shape[0])
            qrow[centre] = 1.0
            qrow[~centre] = -Tj
            crow = qrow @ green_block(g, n, gj, gj_flat)
            cols = [col[tuple(x)] for x in gj]
            Q[a, cols] = qrow
            C[a, cols] = crow
        out.append(dict(t=t, S=S, gamma=gam, Q=Q, C=C, rank=rank))
    return out


def annihilation_ratio(tab: dict) -> float:
    """||Q(S,gamma) G(gamma,gamma^c)||_F / ||G(S,gamma^c)||_F = ||A - T B|| / ||A|| (Eq. Qc)."""
    return tab["ratio"]
