"""The bounded wait of the cooperative grid panel runs out and is reported.

Fronts too tall for a thread-block cluster (the 3D 64^3 root, m = 23816, in the FP32
forms) are factored by the grid panel: every CTA of a front publishes its best pivot
candidate per column and polls its peers' publications.  Each poll gives up after
sp_opts.wait_limit_ns of the GPU's global timer, sets the timeout bit of the status
word and returns, leaving identity interchanges for its panel so later kernels stay in
range.  Here the limit is 1 ns, far shorter than one publication round trip, so the
waits run out; sp_factor must return SP_ERR_TIMEOUT (no fault, no hang).  The context
is then destroyed, and a fresh context with the default limit factors and solves the
same problem to a true residual of 1e-8 (the oracle's FFT operator): the device stays
usable.  The tensor-core pipeline waits keep their fixed limit and are not involved.
"""
import numpy as np
import pytest

import oracle as O
import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_grid_panel_wait_runs_out():
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf_3d(64, 8, 0)
    d, n, b = w["d"], w["n"], w["b"]
    s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
    qd = torch.from_numpy(q).cuda()
    S = B.Solver(d, n, b, s, prec=B.SP_PREC_TF32, setup_route=1, wait_limit_ns=1)
    with pytest.raises(B.SpError) as e:
        S.factor(qd)
    assert e.value.status == B.SP_ERR_TIMEOUT
    S.close()
    torch.cuda.synchronize()
    S = B.Solver(d, n, b, s, prec=B.SP_PREC_TF32, setup_route=1)
    S.factor(qd)
    u = torch.empty(n ** d, dtype=torch.complex128, device="cuda")
    info = S.solve(torch.from_numpy(np.ascontiguousarray(w["f"])).cuda(), u)
    g = O.apply_green(d, n, s, w["f"])
    uh = u.cpu().numpy()
    true = float(np.linalg.norm(g - O.apply_operator(d, n, s, q, uh)) / np.linalg.norm(g))
    assert true <= 1e-8, (true, info)
    S.close()


def test_wait_limit_out_of_range_rejected():
    from paper_1409_0297_gb300 import binding as B
    with pytest.raises(B.SpError) as e:
        B.Solver(2, 32, 4, 4 * np.pi ** 2 * 10.5, wait_limit_ns=-5)
    assert e.value.status == B.SP_ERR_ARG
