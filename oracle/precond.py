"""Sparse Q, C, P = Q + C q and the preconditioner u <= P^{-1} Q g (Section 2.2). Test infrastructure.

P is assembled entry by entry from the per-type tables of stencil.py: row j of
the set instance S (translate of S_t by the leaf-box origin o) has
  Q(j, i) = Q_t[a, c],  C(j, i) = C_t[a, c],  P(j, i) = Q(j, i) + C(j, i) q_i
for i = o + gamma_t[c] (mod n), a the position of j in S (Section 2.2: P = Q + C q
has the pattern of Q).  P is then factored exactly; P^{-1} does not depend on
the ordering, so SuperLU's own column ordering (or a dense LU for small N) is
used instead of the paper's nested dissection.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .stencil import flat_index, stencil_tables


def _leaf_origins(d: int, n: int, b: int) -> np.ndarray:
    m = n // b
    idx = np.indices((m,) * d).reshape(d, -1).T  # rows (i_0..i_{d-1}) in C order of (i_0,...)
    return idx * b


def assemble_sparse(d: int, n: int, b: int, tables: list[dict], q: np.ndarray | None):
    """Global sparse Q, C and P = Q + C diag(q) (CSR, float64), Section 2.2-2.3."""
    N = n ** d
    origins = _leaf_origins(d, n, b)
    rows_l, cols_l, qv_l, cv_l = [], [], [], []
    for tab in tables:
        S, gam = tab["S"], tab["gamma"]
        for o in origins:
            r = flat_index(S + o, n)
            c = flat_index(gam + o, n)
            rows_l.append(np.repeat(r, c.size))
            cols_l.append(np.tile(c, r.size))
            qv_l.append(tab["Q"].ravel())
            cv_l.append(tab["C"].ravel())
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    Qv = np.concatenate(qv_l)
    Cv = np.concatenate(cv_l)
    Qm = sp.csr_matrix((Qv, (rows, cols)), shape=(N, N))
    Cm = sp.csr_matrix((Cv, (rows, cols)), shape=(N, N))
    if q is None:
        return Qm, Cm, None
    Pv = Qv + Cv * np.asarray(q, dtype=np.float64)[cols]
    Pm = sp.csr_matrix((Pv, (rows, cols)), shape=(N, N))
    return Qm, Cm, Pm


class SparsifyingPreconditioner:
    """M r = P^{-1} (Q r) with P = Q + C q factored exactly (Section 2.2).

    factor: "dense" (scipy LU with partial pivoting), "splu" (SuperLU), "auto"
    (dense for N <= 4096) or None (assemble only, for residual checks at large N).
    """

    def __init__(self, d: int, n: int, b: int, s: float, q: np.ndarray, tables=None,
                 factor: str | None = "auto"):
        self.d, self.n, self.b, self.s = d, n, b, s
        self.N = n ** d
        self.tables = tables if tables is not None else stencil_tables(d, n, b, s)
        self.Q, self.C, self.P = assemble_sparse(d, n, b, self.tables, q)
        if factor == "auto":
            factor = "dense" if self.N <= 4096 else "splu"
        self.kind = factor
        if factor == "dense":
            self._lu = sla.lu_factor(self.P.toarray())
        elif factor == "splu":
            self._lu = spla.splu(self.P.tocsc())
        elif factor is None:
            self._lu = None
        else:
            raise ValueError(factor)

    def solve_P(self, y: np.ndarray) -> np.ndarray:
        """P^{-1} y for complex y (P is real: real and imaginary parts solved apart)."""
        y = np.asarray(y, dtype=np.complex128)
        if self.kind == "dense":
            return sla.lu_solve(self._lu, y.real) + 1j * sla.lu_solve(self._lu, y.imag)
        if self.kind == "splu":
            return self._lu.solve(np.ascontiguousarray(y.real)) + \
                1j * self._lu.solve(np.ascontiguousarray(y.imag))
        raise RuntimeError("preconditioner was assembled without a factorisation")

    def apply_Q(self, r: np.ndarray) -> np.ndarray:
        return self.Q @ np.asarray(r, dtype=np.complex128)

    def apply(self, r: np.ndarray) -> np.ndarray:
        """u <= P^{-1} Q r (Section 2.2)."""
        return self.solve_P(self.apply_Q(r))

    def apply_residual(self, r: np.ndarray, z: np.ndarray) -> float:
        """||P z - Q r|| / ||Q r||: checks any candidate z = P^{-1} Q r without a factor."""
        Qr = self.apply_Q(r)
        return float(np.linalg.norm(self.P @ np.asarray(z) - Qr) / np.linalg.norm(Qr))


def sampled_rows(d: int, n: int, b: int, tables: list[dict], q: np.ndarray, rows: np.ndarray):
    """Rows of Q and P = Q + C q for the listed grid points, one by one (Section 2.2-2.3).

    Returns a list of (cols, Q_row, P_row): row j belongs to the set of type
    t = sum_{a : j_a mod b = 0} 2^a of the leaf box with origin b * floor(j / b);
    its entries sit on gamma(S) of that instance.  Lets a caller check
    (P z - Q r) at sampled rows of a grid too large to assemble.
    """
    out = []
    q = np.asarray(q, dtype=np.float64)
    for j in np.asarray(rows):
        p = np.array([(j // n ** a) % n for a in range(d)], dtype=np.int64)
        t = sum(1 << a for a in range(d) if p[a] % b == 0)
        o = (p // b) * b
        tab = tables[t]
        loc = p - o
        a_idx = int(np.nonzero(np.all(tab["S"] == loc[None, :], axis=1))[0][0])
        cols = flat_index(tab["gamma"] + o, n)
        Qr = tab["Q"][a_idx]
        out.append((cols, Qr, Qr + tab["C"][a_idx] * q[cols]))
    return out


def sampled_apply_residual(d, n, b, tables, q, r, z, rows) -> float:
    """||(P z - Q r)[rows]|| / ||(Q r)[rows]|| from rows computed one by one."""
    num = den = 0.0
    for cols, Qr, Pr in sampled_rows(d, n, b, tables, q, rows):
        qr = Qr @ np.asarray(r)[cols]
        pz = Pr @ np.asarray(z)[cols]
        num += abs(pz - qr) ** 2
        den += abs(qr) ** 2
    return float(np.sqrt(num / den))
