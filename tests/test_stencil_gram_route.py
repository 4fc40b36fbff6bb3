"""The Gram route of the stencil set-up (sp_opts.setup_route = 1; the T_S of
Section 2.3 from B B^T = (G^2)(beta, beta) - G(beta, gamma) G(gamma, beta) and
A B^T likewise, instead of a TSQR over all of gamma^c) checked on the host against
the library's TSQR + SVD route and against the oracle's pseudoinverse: the Gram
route solves the normal equations, whose condition number is cond(B)^2, so the
tables agree to a few cond(B)^2 eps (cond(B) from the singular values both routes
report; every case here has |beta| <= 64 so all of them are reported)."""
import numpy as np
import pytest

import oracle as O

EPS = np.finfo(float).eps
CASES = [(2, 16, 2, 1.37), (2, 32, 4, 3.3), (2, 64, 8, 7.7), (3, 8, 2, 1.37), (2, 48, 3, 5.5),
         (2, 40, 5, 4.1), (3, 12, 3, 2.2)]  # |beta| <= 64: every singular value returned


def _B():
    import os
    from paper_1409_0297_gb300 import build as bld
    if not os.path.exists(bld.LIB):
        bld.build()
    from paper_1409_0297_gb300 import binding as B
    return B


@pytest.mark.parametrize("d,n,b,kappa", CASES)
def test_gram_route_matches_svd_route_and_oracle(d, n, b, kappa):
    B = _B()
    s = 4 * np.pi ** 2 * kappa
    orc = O.stencil_tables(d, n, b, s)
    for t in range(1 << d):
        Q0, C0, r0, s0 = B.sp_stencil_table(d, n, b, s, t, route=0)
        Q1, C1, r1, s1 = B.sp_stencil_table(d, n, b, s, t, route=1)
        nb = Q0.shape[1] - Q0.shape[0]
        assert nb <= 64 and r0 == r1 == nb  # full rank at these sizes
        cond = s0[0] / s0[nb - 1]
        bound = 8 * cond ** 2 * EPS
        # singular values: sqrt of the eigenvalues of B B^T, relative to sigma_max
        assert np.max(np.abs(s1[:nb] - s0[:nb])) <= bound * s0[0]
        for Qx, Cx in ((Q1, C1),):
            assert np.linalg.norm(Qx - Q0) <= bound * np.linalg.norm(Q0)
            assert np.linalg.norm(Cx - C0) <= bound * np.linalg.norm(C0)
            assert np.linalg.norm(Qx - orc[t]["Q"]) <= bound * np.linalg.norm(orc[t]["Q"])


def test_gram_route_argument_check():
    B = _B()
    with pytest.raises(B.SpError):
        B.sp_stencil_table(2, 16, 2, 4 * np.pi ** 2 * 1.37, 0, route=2)
