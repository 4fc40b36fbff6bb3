"""Per-point sparsifying stencils (sp_opts.stencil = 1): each point j gets its own
stencil on gamma({j}), its 3^d neighbourhood (the per-point construction that the
paper's set stencils of Section 2.3 generalise).  Host checks of the library's
tables against the oracle, which computes every point's T_j independently, and
pins: the stencil rows live on gamma({j}) only, the centre weight is 1, all
points share one T (translation invariance: the oracle does not assume it), and
T_j is the least-squares fit A ~ T_j B (normal equations (A - T_j B) B^T = 0)."""
import numpy as np
import pytest

import oracle as O

CASES = [(2, 16, 2, 1.37), (2, 32, 4, 3.3), (3, 8, 2, 1.37), (2, 40, 5, 4.1), (3, 12, 3, 2.2)]


def _B():
    import os
    from paper_1409_0297_gb300 import build as bld
    if not os.path.exists(bld.LIB):
        bld.build()
    from paper_1409_0297_gb300 import binding as B
    return B


@pytest.mark.parametrize("d,n,b,kappa", CASES)
def test_pointwise_tables_match_oracle(d, n, b, kappa):
    B = _B()
    s = 4 * np.pi ** 2 * kappa
    orc = O.pointwise_stencil_tables(d, n, b, s)
    for t in range(1 << d):
        Q, C, rank, _ = B.sp_stencil_table(d, n, b, s, t, kind=1)
        assert rank == 3 ** d - 1
        assert np.linalg.norm(Q - orc[t]["Q"]) <= 1e-10 * np.linalg.norm(orc[t]["Q"])
        assert np.linalg.norm(C - orc[t]["C"]) <= 1e-10 * np.linalg.norm(orc[t]["C"])


@pytest.mark.parametrize("d,n,b,kappa", CASES)
def test_pointwise_structure_and_invariance(d, n, b, kappa):
    s = 4 * np.pi ** 2 * kappa
    orc = O.pointwise_stencil_tables(d, n, b, s)
    ref = None
    for tab in orc:
        S, gam, Q = tab["S"], tab["gamma"], tab["Q"]
        for a, p in enumerate(S):
            near = np.all(np.abs(gam - p) <= 1, axis=1)
            assert np.all(Q[a, ~near] == 0.0)
            assert Q[a, np.nonzero(np.all(gam == p, axis=1))[0][0]] == 1.0
            # the weights on gamma({p}) in neighbour order (axis 0 fastest)
            offs = gam[near] - p
            order = np.lexsort(offs.T[::-1])
            row = Q[a, np.nonzero(near)[0][order]]
            if ref is None:
                ref = row
            assert np.allclose(row, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_pointwise_least_squares_pin():
    """T_j minimises ||A - T B||: (A - T B) B^T = 0, with A, B built here directly."""
    d, n, b, kappa = 2, 16, 2, 1.37
    s = 4 * np.pi ** 2 * kappa
    g = O.green_kernel(d, n, s)
    tab = O.pointwise_stencil_tables(d, n, b, s)[0]
    p = tab["S"][0]
    offs = np.array([(i, j) for j in (-1, 0, 1) for i in (-1, 0, 1)])
    gj = p + offs
    from oracle.stencil import flat_index
    flat = flat_index(gj, n)
    comp = np.setdiff1d(np.arange(n ** d), flat)
    A = O.green_block(g, n, p[None, :], comp)
    Bm = O.green_block(g, n, gj[np.any(offs != 0, axis=1)], comp)
    col = {tuple(x): i for i, x in enumerate(tab["gamma"])}
    T = -tab["Q"][0, [col[tuple(x)] for x in gj[np.any(offs != 0, axis=1)]]]
    resid = (A - T[None, :] @ Bm) @ Bm.T
    assert np.linalg.norm(resid) <= 1e-10 * np.linalg.norm(A) * np.linalg.norm(Bm)


@pytest.mark.parametrize("d,n,b", [(2, 16, 2), (3, 8, 2)])
def test_pointwise_C_is_QG_on_each_stencil(d, n, b):
    """Row a of a per-point table holds C(j, gamma({j})) = (Q G)(j, gamma({j})) for the
    point j = S[a], with G the dense Green's matrix of the whole grid (Eq. G), and zero
    on the rest of gamma(S): the truncation keeps exactly the point's own stencil."""
    s = 4 * np.pi ** 2 * 1.37
    g = O.green_kernel(d, n, s)
    N = n ** d
    pts = np.stack([(np.arange(N) // n ** a) % n for a in range(d)], axis=1)
    G = O.green_block(g, n, pts, np.arange(N))
    from oracle.stencil import flat_index
    for tab in O.pointwise_stencil_tables(d, n, b, s):
        gam_flat = flat_index(tab["gamma"], n)
        for a, p in enumerate(tab["S"]):
            qrow = np.zeros(N)
            np.add.at(qrow, gam_flat, tab["Q"][a])
            qg = qrow @ G
            near = np.all(np.abs(tab["gamma"] - p) <= 1, axis=1)
            assert np.allclose(tab["C"][a, near], qg[gam_flat[near]], rtol=0,
                               atol=1e-12 * np.abs(qg).max())
            assert not np.any(tab["C"][a, ~near])

