"""Right-preconditioned GMRES (Saad and Schultz 1986), the outer iteration of Section 2. Test infrastructure.

Readings (the paper only states "GMRES with relative tolerance 1e-6", Section 3):
  * system (I + G q) u = g with g = G f, right preconditioner M = P^{-1} Q,
    zero initial guess;
  * Arnoldi with classical Gram-Schmidt applied twice, complex Givens rotations;
  * stop when the Givens residual estimate |gamma_{k+1}| / ||g|| <= tol, form
    u = u0 + M (V_k y), then compute the true residual ||g - A u|| / ||g||; if
    that is above tol, restart from u (the iteration count keeps running).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _givens(a: complex, b: complex):
    """Unitary [[c, s], [-conj(s), c]] (c real) that maps (a, b) to (r, 0)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, 1.0 + 0.0j
    r = np.hypot(abs(a), abs(b))
    c = abs(a) / r
    s = (a / abs(a)) * np.conj(b) / r
    return c, s


def gmres_right(apply_A, apply_M, g: np.ndarray, tol: float = 1e-8, maxit: int = 500):
    """Solve A u = g with right preconditioner M.  Returns a dict with
    u, iters, hist (estimate per iteration, relative to ||g||), true_relres."""
    g = np.asarray(g, dtype=np.complex128)
    N = g.size
    bnorm = np.linalg.norm(g)
    u = np.zeros(N, dtype=np.complex128)
    hist = [1.0]
    total = 0
    if bnorm == 0.0:
        return dict(u=u, iters=0, hist=hist, true_relres=0.0)
    r = g.copy()
    true_rel = 1.0
    while True:
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or total >= maxit:
            true_rel = beta / bnorm
            break
        m = maxit - total
        V = np.zeros((m + 1, N), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        gam = np.zeros(m + 1, dtype=np.complex128)
        gam[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = apply_A(apply_M(V[j]))
            h = np.zeros(j + 1, dtype=np.complex128)
            for _ in range(2):  # classical Gram-Schmidt, twice
                c = V[: j + 1].conj() @ w
                w = w - V[: j + 1].T @ c
                h += c
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):  # earlier rotations on the new column
                t0 = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t0
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            gam[j + 1] = -np.conj(sn[j]) * gam[j]
            gam[j] = cs[j] * gam[j]
            total += 1
            k = j + 1
            hist.append(abs(gam[j + 1]) / bnorm)
            if abs(gam[j + 1]) / bnorm <= tol or hn == 0.0 or total >= maxit:
                break
            V[j + 1] = w / hn
        y = sla.solve_triangular(H[:k, :k], gam[:k])
        u = u + apply_M(V[:k].T @ y)
        r = g - apply_A(u)
        true_rel = np.linalg.norm(r) / bnorm
        if true_rel <= tol or total >= maxit:
            break
    return dict(u=u, iters=total, hist=hist, true_relres=float(true_rel))
