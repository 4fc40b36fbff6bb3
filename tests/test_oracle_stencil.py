"""Pins of the oracle's stencil Q, C and P (Section 2.2-2.3) against what the paper fixes.

  * the set partition and neighbourhood sizes stated in Section 2.3;
  * T_S = G(S, gamma^c) G(beta, gamma^c)^+ satisfies the least-squares normal
    equations and equals an independent LAPACK least-squares solve;
  * T_S does not depend on the translate of S, and orientations of one kind
    are axis permutations of each other (G is symmetric under axis swaps);
  * Q(S, S) = I, C = (Q G) on the pattern of Q, P = Q + C q with the pattern of Q.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from oracle.stencil import flat_index


@pytest.mark.parametrize("d,n,b", [(2, 8, 2), (2, 12, 3), (2, 16, 4), (3, 8, 2), (3, 8, 4)])
def test_sets_partition_the_grid(d, n, b):
    """Cells (b-1)^d, faces (b-1)^2, edges b-1, vertices 1; translates partition J."""
    N = n ** d
    hits = np.zeros(N, dtype=int)
    m = n // b
    for t, Z in enumerate(O.set_types(d)):
        S = O.canonical_set(d, b, t)
        assert len(S) == (b - 1) ** (d - len(Z))
        gam = O.canonical_gamma(d, b, t)
        assert len(gam) == (b + 1) ** (d - len(Z)) * 3 ** len(Z)
        # every point of gamma is within l-inf distance 1 of S, and S is inside gamma
        for p in gam:
            assert np.min(np.max(np.abs(S - p), axis=1)) <= 1
        beta = O.canonical_beta(d, b, t)
        assert len(beta) == len(gam) - len(S)
        for idx in itertools.product(range(m), repeat=d):
            hits[flat_index(S + b * np.array(idx), n)] += 1
    assert np.all(hits == 1)
    # a point's type is the set of axes where its coordinate is a multiple of b
    cell = O.canonical_set(d, b, 0)
    assert np.all(cell % b != 0)


def test_cell_gamma_is_leaf_box_closure():
    d, b = 2, 5
    gam = O.canonical_gamma(d, b, 0)
    assert len(gam) == (b + 1) ** 2
    assert gam.min() == 0 and gam.max() == b


@pytest.mark.parametrize("d,n,b", [(2, 16, 4), (2, 24, 3), (3, 8, 2), (3, 16, 4)])
def test_T_least_squares(d, n, b):
    s = 4 * np.pi ** 2 * (n / 6) ** 2 * 1.013
    for tab in O.stencil_tables(d, n, b, s, keep_blocks=True):
        A, B, T = tab["A"], tab["B"], tab["T"]
        assert tab["rank"] == B.shape[0]
        # normal equations (A - T B) B^T = 0
        ne = (A - T @ B) @ B.T
        assert np.linalg.norm(ne) <= 1e-10 * np.linalg.norm(A) * np.linalg.norm(B)
        # independent route: LAPACK least squares of B^T X = A^T
        X = sla.lstsq(B.T, A.T, lapack_driver="gelsy")[0]
        assert np.linalg.norm(X.T - T) <= 1e-9 * np.linalg.norm(T)
        # the stencil annihilates most of G(S, gamma^c) (Eq. Qc); T = 0 would give 1
        assert tab["ratio"] < 0.05
        # Q(S, gamma) = [I, -T] on (S, beta)
        Q = tab["Q"]
        gam = [tuple(p) for p in tab["gamma"]]
        pos_S = [gam.index(tuple(p)) for p in tab["S"]]
        pos_b = [gam.index(tuple(p)) for p in tab["beta"]]
        assert np.array_equal(Q[:, pos_S], np.eye(len(pos_S)))
        assert np.array_equal(Q[:, pos_b], -T)


def test_matlab_pinv_truncation():
    rng = np.random.default_rng(0)
    U = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    V = np.linalg.qr(rng.standard_normal((40, 6)))[0]
    sig = np.array([3.0, 1.0, 1e-3, 1e-8, 1e-12, 1e-15])
    B = (U * sig) @ V.T
    P, r, _ = O.matlab_pinv(B)
    # cutoff 40 * eps(3) = 40 * 2^-51 ~ 1.8e-14: the last singular value is dropped
    assert r == 5
    ref = (V[:, :5] / sig[:5]) @ U[:, :5].T
    assert np.linalg.norm(P - ref) <= 1e-2 * np.linalg.norm(ref)
    # the cutoff scales with the larger dimension: 5e-15 lies between 6 eps(3) = 2.7e-15
    # and 40 eps(3) = 1.8e-14, so it is dropped (a cutoff on the smaller dimension keeps it)
    sig2 = np.array([3.0, 1.0, 1e-3, 1e-8, 5e-15, 1e-16])
    _, r2, s2 = O.matlab_pinv((U * sig2) @ V.T)
    assert 6 * 2.0 ** -51 < s2[4] < 40 * 2.0 ** -51
    assert r2 == 4


@pytest.mark.parametrize("d,n,b,origin", [(2, 16, 4, (4, 8)), (2, 24, 3, (21, 6)), (3, 8, 2, (2, 4, 6))])
def test_T_translation_invariance(d, n, b, origin):
    s = 4 * np.pi ** 2 * 3.71
    t0 = O.stencil_tables(d, n, b, s)
    t1 = O.stencil_tables(d, n, b, s, origin=origin)
    for a, c in zip(t0, t1):
        assert np.linalg.norm(a["T"] - c["T"]) <= 1e-10 * np.linalg.norm(a["T"])
        assert np.linalg.norm(a["C"] - c["C"]) <= 1e-10 * np.linalg.norm(a["C"])


@pytest.mark.parametrize("d,n,b", [(2, 16, 4), (3, 12, 3)])
def test_T_axis_permutation_symmetry(d, n, b):
    """G is invariant under a permutation of the axes, so T of an orientation is the
    T of another orientation with rows and columns permuted accordingly."""
    s = 4 * np.pi ** 2 * 2.17
    tabs = O.stencil_tables(d, n, b, s)
    for perm in itertools.permutations(range(d)):
        for t in range(1 << d):
            tp = sum(1 << perm[a] for a in range(d) if (t >> a) & 1)
            A, B = tabs[t], tabs[tp]
            S = [tuple(p) for p in B["S"]]
            be = [tuple(p) for p in B["beta"]]

            def moved(p):
                q = [0] * d
                for a in range(d):
                    q[perm[a]] = p[a]
                return tuple(q)

            rows = [S.index(moved(p)) for p in A["S"]]
            cols = [be.index(moved(p)) for p in A["beta"]]
            assert np.linalg.norm(B["T"][np.ix_(rows, cols)] - A["T"]) <= 1e-9 * np.linalg.norm(A["T"])


def _dense_G(d, n, s):
    g = O.green_kernel(d, n, s)
    N = n ** d
    pts = np.stack([(np.arange(N) // n ** a) % n for a in range(d)], axis=1)
    return O.green_block(g, n, pts, np.arange(N))


@pytest.mark.parametrize("d,n,b", [(2, 16, 4), (2, 16, 2), (3, 8, 2)])
def test_C_is_QG_on_the_pattern_and_P(d, n, b):
    s = 4 * np.pi ** 2 * 4.9
    tabs = O.stencil_tables(d, n, b, s)
    rng = np.random.default_rng(9)
    q = rng.standard_normal(n ** d) * 30
    Qs, Cs, Ps = O.assemble_sparse(d, n, b, tabs, q)
    Q, C, P = Qs.toarray(), Cs.toarray(), Ps.toarray()
    G = _dense_G(d, n, s)
    QG = Q @ G
    # structural pattern: row j of a set S is supported on gamma(S) (Section 2.2, mu(j))
    pattern = np.zeros((n ** d, n ** d), dtype=bool)
    for tab in tabs:
        for o in itertools.product(range(0, n, b), repeat=d):
            rws = flat_index(tab["S"] + np.array(o), n)
            cls = flat_index(tab["gamma"] + np.array(o), n)
            pattern[np.ix_(rws, cls)] = True
    assert np.all(pattern[Q != 0])
    assert np.allclose(C[pattern], QG[pattern], rtol=0, atol=1e-12 * np.abs(QG).max())
    assert not np.any(C[~pattern])
    # every row has the full gamma support of its set, rows of Q are [I, -T]
    assert np.array_equal(np.diag(Q), np.ones(n ** d))
    # P = Q + C diag(q) has the pattern of Q
    assert np.allclose(P, Q + C * q[None, :], rtol=0, atol=1e-12 * np.abs(P).max())
    assert np.all(pattern[P != 0]) and np.count_nonzero(P) == np.count_nonzero(pattern)
    # the truncation only drops the far field: Q(I + G q) - P is small compared with P
    full = Q @ (np.eye(n ** d) + G * q[None, :])
    assert np.linalg.norm(full - P) < 0.2 * np.linalg.norm(P)


@pytest.mark.parametrize("d,n,b", [(2, 16, 4), (3, 8, 2), (2, 24, 3)])
def test_tables_from_T_rebuilds_stencil_tables(d, n, b):
    """tables_from_T (Q = [I, -T], C = Q G(gamma, gamma) from a given T) reproduces
    stencil_tables' Q and C exactly when handed its T, and a perturbed T moves Q by
    exactly that perturbation on the beta columns (the identity block stays)."""
    s = 4 * np.pi ** 2 * 2.37
    tabs = O.stencil_tables(d, n, b, s)
    rebuilt = O.tables_from_T(d, n, b, s, [t["T"] for t in tabs])
    for a, c in zip(tabs, rebuilt):
        assert np.array_equal(a["Q"], c["Q"]) and np.array_equal(a["C"], c["C"])
    T0 = tabs[0]["T"] + 1e-3
    Q1 = O.tables_from_T(d, n, b, s, [T0] + [t["T"] for t in tabs[1:]])[0]["Q"]
    diff = Q1 - tabs[0]["Q"]
    assert np.allclose(np.abs(diff).sum(), 1e-3 * tabs[0]["T"].size)
    S_cols = [i for i, p in enumerate(map(tuple, tabs[0]["gamma"])) if p in set(map(tuple, tabs[0]["S"]))]
    assert np.array_equal(Q1[:, S_cols], np.eye(len(S_cols)))
