"""Pins of the oracle's row-by-row checker (Section 2.2-2.3), used at grid sizes too
large to assemble P.

`sampled_rows` rebuilds rows of Q and P = Q + C q one grid point at a time from the
set-type tables (type bits from j mod b, leaf-box origin b floor(j / b)).  Here it is
compared, at every row of grids small enough to assemble, with the assembled sparse
matrices of `assemble_sparse`: same columns, same values, no entry missing.  The
sampled residual over all rows must then equal the global ||P z - Q r|| / ||Q r||,
vanish for z = P^{-1} Q r, and flag a z that is wrong in a single entry, on a face of
a leaf box as well as inside a cell.
"""
import numpy as np
import pytest

import oracle as O
import synthetic_media as sm

CASES = [(2, 16, 4), (3, 8, 2), (2, 32, 4), (2, 24, 3)]


def _problem(d, n, b):
    c = sm.grf_velocity(d, n, 0.15, 3)
    s, q = O.helmholtz_shift(d, n, 2 * np.pi * n / 7, c)
    M = O.SparsifyingPreconditioner(d, n, b, s, q)
    return s, q, M


@pytest.mark.parametrize("d,n,b", CASES)
def test_rows_equal_assembled_matrices(d, n, b):
    s, q, M = _problem(d, n, b)
    N = n ** d
    rows = np.arange(N)
    Qc, Pc = M.Q.tocsr(), M.P.tocsr()
    for j, (cols, Qr, Pr) in zip(rows, O.sampled_rows(d, n, b, M.tables, q, rows)):
        assert len(set(cols.tolist())) == cols.size  # gamma(S) never wraps onto itself here
        qd = np.zeros(N)
        pd = np.zeros(N)
        qd[cols] = Qr
        pd[cols] = Pr
        assert np.array_equal(qd, Qc[j].toarray().ravel())
        assert np.allclose(pd, Pc[j].toarray().ravel(), rtol=1e-15, atol=1e-15 * np.abs(Pr).max())


@pytest.mark.parametrize("d,n,b", CASES)
def test_sampled_residual_equals_global(d, n, b):
    s, q, M = _problem(d, n, b)
    N = n ** d
    r = sm.random_complex_vector(N, 5)
    z = M.apply(r)
    rows = np.arange(N)
    assert O.sampled_apply_residual(d, n, b, M.tables, q, r, z, rows) <= 1e-13
    # any candidate: the full-row sum is the global residual
    y = sm.random_complex_vector(N, 6)
    a = O.sampled_apply_residual(d, n, b, M.tables, q, r, y, rows)
    assert abs(a - M.apply_residual(r, y)) <= 1e-12 * a


@pytest.mark.parametrize("d,n,b", CASES)
def test_single_wrong_entry_is_flagged(d, n, b):
    s, q, M = _problem(d, n, b)
    N = n ** d
    r = sm.random_complex_vector(N, 7)
    z = M.apply(r)
    rows = np.arange(N)
    # a point inside a cell and a point on a face/edge of a leaf box (coordinate 0 mod b)
    cell = sum(1 * n ** a for a in range(d))
    face = sum((b if a == 0 else 1) * n ** a for a in range(d))
    for j in (cell, face):
        zb = z.copy()
        zb[j] += 1e-6 * np.abs(z).max()
        res = O.sampled_apply_residual(d, n, b, M.tables, q, r, zb, rows)
        assert res >= 1e-9, (j, res)
        assert abs(res - M.apply_residual(r, zb)) <= 1e-9 * res


def test_subsample_tracks_full_residual():
    """A random 25% of the rows estimates the full residual of a uniformly wrong z
    within a factor 2 (the estimate the full-size GPU tests rely on)."""
    d, n, b = 2, 32, 4
    s, q, M = _problem(d, n, b)
    N = n ** d
    r = sm.random_complex_vector(N, 8)
    z = M.apply(r) * (1 + 1e-4 * sm.random_complex_vector(N, 9))
    rows = np.random.default_rng(4).choice(N, N // 4, replace=False)
    est = O.sampled_apply_residual(d, n, b, M.tables, q, r, z, rows)
    full = M.apply_residual(r, z)
    assert 0.5 * full <= est <= 2.0 * full
