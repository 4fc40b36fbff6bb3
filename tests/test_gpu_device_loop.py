"""The device-resident restart cycle (sp_opts.device_loop = 1): each GMRES cycle of
sp_solve is one CUDA graph whose Arnoldi steps repeat under a conditional while node,
the stopping test on the device.  It launches the host-driven loop's kernels in the
host loop's order with the same operands, so every result must be bit-identical to
device_loop = 0: the solution, the iteration and restart counts, the estimate
history and both residuals.  Cases: FP64 and FP32 forms in 2D and 3D, several
restart cycles, the iteration budget running out, a starting vector, a new medium
between solves, the host-buffer solve and several right-hand sides (sp_solve_many,
batched instances)."""
import numpy as np
import pytest

import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("2d_n128_b8", lambda: sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)),
    ("2d_n96_b6_schr", lambda: sm.schrodinger_wells(2, 96, 6, 6.0, 5.0, 17)),
    ("3d_n16_b4", lambda: sm.helmholtz_grf_3d(16, 4, 0)),
]


def _medium(B, w):
    if w["kind"] == "helmholtz":
        return B.sp_medium_helmholtz(w["d"], w["n"], w["omega"], w["c"])
    return B.sp_medium_schrodinger(w["d"], w["n"], w["ell"], w["E"], w["V"])


def _same(a, b):
    ua, ia = a
    ub, ib = b
    assert torch.equal(ua, ub)
    for key in ("iters", "restarts", "est_relres", "true_relres", "status"):
        assert ia[key] == ib[key], key
    assert np.array_equal(np.asarray(ia["hist"]), np.asarray(ib["hist"]))


def _run(B, w, prec, loop, restart=200, maxit=500, x0=False, allow_noconv=False):
    d, n, b = w["d"], w["n"], w["b"]
    s, q = _medium(B, w)
    N = n ** d
    f = torch.from_numpy(np.ascontiguousarray(w["f"])).cuda()
    S = B.Solver(d, n, b, s, prec=prec, restart=restart, maxit=maxit, device_loop=loop)
    S.factor(torch.from_numpy(q).cuda())
    u = torch.empty(N, dtype=torch.complex128, device="cuda")
    if x0:
        u0 = 0.5 * torch.from_numpy(sm.random_complex_vector(N, 61)).cuda() * 1e-3
        info = S.solve_x0(f, u0, u, allow_noconv=allow_noconv)
    else:
        info = S.solve(f, u, allow_noconv=allow_noconv)
    torch.cuda.synchronize()
    S.close()
    return u, info


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_device_loop_bit_identical(name, make, prec):
    from paper_1409_0297_gb300 import binding as B
    w = make()
    a = _run(B, w, prec, 0)
    b = _run(B, w, prec, 1)
    _same(a, b)
    assert b[1]["true_relres"] <= 1e-8 and b[1]["restarts"] == 0


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_device_loop_restarts(prec):
    """restart = 6: several cycles, each one graph launch; the host's restart
    decision from the true residual the graph leaves behind."""
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)
    a = _run(B, w, prec, 0, restart=6)
    b = _run(B, w, prec, 1, restart=6)
    _same(a, b)
    assert b[1]["restarts"] >= 2 and b[1]["true_relres"] <= 1e-8


def test_device_loop_budget_runs_out():
    """maxit = 5 inside the first cycle: the device test stops at the budget and the
    solve reports SP_ERR_NOCONV exactly as the host loop does."""
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)
    a = _run(B, w, 0, 0, maxit=5, allow_noconv=True)
    b = _run(B, w, 0, 1, maxit=5, allow_noconv=True)
    _same(a, b)
    assert b[1]["iters"] == 5 and b[1]["status"] == B.SP_ERR_NOCONV


def test_device_loop_start_vector():
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)
    _same(_run(B, w, 1, 0, x0=True), _run(B, w, 1, 1, x0=True))


def test_device_loop_new_medium_and_host_buffers():
    """Two media of one shift in two different tensors, factored and solved in turn
    on one context (the graph reads the context's copy of the medium), then the
    host-buffer solve; each against a host-loop context."""
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)
    d, n, b = w["d"], w["n"], w["b"]
    s, q = _medium(B, w)
    N = n ** d
    rng = np.random.default_rng(5)
    q2 = q * (1.0 + 0.05 * rng.standard_normal(N))
    f = torch.from_numpy(np.ascontiguousarray(w["f"])).cuda()
    res = {}
    for loop in (0, 1):
        S = B.Solver(d, n, b, s, prec=1, device_loop=loop)
        out = []
        for qq in (q, q2):
            qd = torch.from_numpy(qq).cuda()
            S.factor(qd)
            u = torch.empty(N, dtype=torch.complex128, device="cuda")
            info = S.solve(f, u)
            torch.cuda.synchronize()
            out.append((u, info))
        fh = np.ascontiguousarray(w["f"]).astype(np.complex128)
        uh = np.empty(N, dtype=np.complex128)
        ih = B.sp_solve_host(S.ctx, fh, uh)
        out.append((torch.from_numpy(uh), ih))
        S.close()
        res[loop] = out
    for x, y in zip(res[0], res[1]):
        _same(x, y)
    assert res[1][0][1]["iters"] != res[1][1][1]["iters"] or not torch.equal(res[1][0][0],
                                                                             res[1][1][0])


@pytest.mark.parametrize("prec,restart", [(0, 200), (1, 7)], ids=["fp64", "fp32_restart7"])
def test_device_loop_many_rhs(prec, restart):
    """sp_solve_many through the batched cycle graph (4 Krylov instances, one a zero
    right-hand side) against the host-driven lockstep iteration."""
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)
    d, n, b = w["d"], w["n"], w["b"]
    s, q = _medium(B, w)
    N = n ** d
    F = np.stack([sm.random_gaussian_source(d, n, 2600 + r, 0.05 + 0.02 * r) for r in range(4)])
    F[2] = 0.0
    Fd = torch.from_numpy(F).cuda().contiguous()
    res = []
    for loop in (0, 1):
        S = B.Solver(d, n, b, s, prec=prec, restart=restart, max_rhs=4, device_loop=loop)
        S.factor(torch.from_numpy(q).cuda())
        U = torch.empty_like(Fd)
        infos = S.solve_many(Fd.view(-1), U.view(-1))
        torch.cuda.synchronize()
        res.append((U, infos))
        S.close()
    assert torch.equal(res[0][0], res[1][0])
    for a, c in zip(res[0][1], res[1][1]):
        for key in ("iters", "restarts", "est_relres", "true_relres"):
            assert a[key] == c[key], key
        assert np.array_equal(a["hist"], c["hist"])
    assert res[1][1][2]["iters"] == 0
