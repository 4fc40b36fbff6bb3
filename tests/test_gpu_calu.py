"""Tournament pivoting of the FP32 grid panel (sp_opts.panel_pivoting = 1, the
communication-avoiding LU of Grigori, Demmel and Xiang): 3D 64^3 in the TF32 form,
whose 23816-wide root is factored by the cooperative grid panel.  The factor differs
from the column-by-column one (other pivots) but is as good a preconditioner: the
solve reaches a true residual of 1e-8 by the oracle's FFT operator within a few
iterations of the default, and two factorisations give bit-identical applications."""
import numpy as np
import pytest

import oracle as O
import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tournament_panel_3d64():
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf_3d(64, 8, 0)
    d, n, b = w["d"], w["n"], w["b"]
    s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
    qd = torch.from_numpy(q).cuda()
    fd = torch.from_numpy(np.ascontiguousarray(w["f"])).cuda()
    g = O.apply_green(d, n, s, w["f"])
    its = {}
    for pp in (0, 1):
        S = B.Solver(d, n, b, s, prec=B.SP_PREC_TF32, setup_route=1, panel_pivoting=pp)
        S.factor(qd)
        u = torch.empty(n ** d, dtype=torch.complex128, device="cuda")
        info = S.solve(fd, u)
        true = float(np.linalg.norm(g - O.apply_operator(d, n, s, q, u.cpu().numpy())) / np.linalg.norm(g))
        assert true <= 1e-8, (pp, true, info)
        its[pp] = info["iters"]
        if pp == 1:
            r = torch.from_numpy(sm.random_complex_vector(n ** d, 37)).cuda()
            z1, z2 = torch.empty_like(u), torch.empty_like(u)
            S.apply(r, z1)
            S.factor(qd)
            S.apply(r, z2)
            torch.cuda.synchronize()
            assert torch.equal(z1, z2)
        S.close()
    assert abs(its[1] - its[0]) <= 3, its
