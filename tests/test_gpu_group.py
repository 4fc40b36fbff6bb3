"""Problem groups (sp_setup_group): P problems of one grid and leaf size in one
context, every level launch covering the fronts of all P problems and the P GMRES
iterations advancing together.  Each problem of a group must give what a separate
context gives for it: the operator, the Green's function and the stencil apply
bit-identically (the same kernels per vector with that problem's symbol, medium and
tables), the preconditioner to rounding (launch shapes that depend on the number of
fronts may sum in another order), the solve to the same tolerance with the iteration
counts within one.  Several right-hand sides per problem (sp_solve_many on a group)
must give each (right-hand side, problem) the bits of the group's sp_solve for it."""
import numpy as np
import pytest

import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _members(d, n, b):
    if d == 2:
        return [sm.helmholtz_grf(2, n, b, 2 * np.pi * n / 8, 0.05, 4),
                sm.schrodinger_wells(2, n, b, 8.0, 10.0, 7),
                sm.helmholtz_grf(2, n, b, 2 * np.pi * n / 8, 0.05, 9)]
    return [sm.helmholtz_grf_3d(n, b, 0), sm.schrodinger_wells(3, n, b, 4.0, 10.0, 3)]


def _medium(B, w):
    if w["kind"] == "helmholtz":
        return B.sp_medium_helmholtz(w["d"], w["n"], w["omega"], w["c"])
    return B.sp_medium_schrodinger(w["d"], w["n"], w["ell"], w["E"], w["V"])


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


CASES = [(2, 128, 8, 0), (2, 128, 8, 1), (3, 16, 4, 1), (3, 16, 4, 0)]
IDS = ["2d_n128_fp64", "2d_n128_fp32", "3d_n16_fp32", "3d_n16_fp64"]


@pytest.mark.parametrize("d,n,b,prec", CASES, ids=IDS)
def test_group_matches_separate_contexts(d, n, b, prec):
    from paper_1409_0297_gb300 import binding as B
    ws = _members(d, n, b)
    P, N = len(ws), n ** d
    meds = [_medium(B, w) for w in ws]
    shifts = [m[0] for m in meds]
    qs = [torch.from_numpy(m[1]).cuda() for m in meds]
    fs = [torch.from_numpy(np.ascontiguousarray(w["f"])).cuda() for w in ws]
    r = torch.from_numpy(sm.random_complex_vector(P * N, 71)).cuda()
    G = B.Solver(d, n, b, shifts, prec=prec)
    assert G.P == P and B.sp_problems(G.ctx) == P
    G.factor(torch.cat(qs))
    zg, wg, gg, yg, ug = (torch.empty(P * N, dtype=torch.complex128, device="cuda")
                          for _ in range(5))
    G.apply(r, zg)
    G.matvec(r, wg)
    G.green(r, gg)
    G.qapply(r, yg)
    infos = G.solve(torch.cat(fs), ug)
    torch.cuda.synchronize()
    assert len(infos) == P
    # both are exact applications of the same factor that may sum in another order
    # (the sweep variants' bound: 1e-11 relative in FP64, 2e-3 in FP32 at cond(P) ~
    # 1e4-1e5, where FP32 rounding alone reaches cond(P) eps32 ~ 1e-3)
    tol_apply = 1e-11 if prec == 0 else 2e-3
    for p in range(P):
        S = B.Solver(d, n, b, shifts[p], prec=prec)
        S.factor(qs[p])
        sl = slice(p * N, (p + 1) * N)
        rp = r[sl].contiguous()
        z, w, g, y, u = (torch.empty(N, dtype=torch.complex128, device="cuda") for _ in range(5))
        S.apply(rp, z)
        S.matvec(rp, w)
        S.green(rp, g)
        S.qapply(rp, y)
        info = S.solve(fs[p], u)
        torch.cuda.synchronize()
        assert torch.equal(wg[sl], w), p
        assert torch.equal(gg[sl], g), p
        assert torch.equal(yg[sl], y), p
        assert _rel(zg[sl], z) <= tol_apply, p
        assert infos[p]["true_relres"] <= 1e-8, p
        assert abs(infos[p]["iters"] - info["iters"]) <= 1, p
        assert infos[p]["s_used"] == shifts[p]
        assert _rel(ug[sl], u) <= 1e-6, p
        S.close()
    G.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_group_many_rhs_bit_identical(prec):
    """R = 3 right-hand sides of each of the P problems in one sp_solve_many (3 P
    Krylov instances, one of them a zero right-hand side): each (r, p) is
    bit-identical to the group's sp_solve with that right-hand side."""
    from paper_1409_0297_gb300 import binding as B
    d, n, b = 2, 128, 8
    ws = _members(d, n, b)
    P, N, R = len(ws), n ** d, 3
    meds = [_medium(B, w) for w in ws]
    G = B.Solver(d, n, b, [m[0] for m in meds], prec=prec, max_rhs=R)
    G.factor(torch.cat([torch.from_numpy(m[1]).cuda() for m in meds]))
    F = np.stack([np.concatenate([sm.random_gaussian_source(d, n, 4000 + 10 * r + p)
                                  for p in range(P)]) for r in range(R)])
    F[1, N:2 * N] = 0.0
    Fd = torch.from_numpy(F).cuda().contiguous()
    U = torch.empty_like(Fd)
    infos = G.solve_many(Fd.view(-1), U.view(-1))
    torch.cuda.synchronize()
    assert len(infos) == R * P
    for r in range(R):
        u = torch.empty(P * N, dtype=torch.complex128, device="cuda")
        one = G.solve(Fd[r].contiguous(), u)
        torch.cuda.synchronize()
        assert torch.equal(U[r], u), r
        for p in range(P):
            a, c = infos[r * P + p], one[p]
            assert a["iters"] == c["iters"] and a["restarts"] == c["restarts"], (r, p)
            assert np.array_equal(a["hist"], c["hist"]), (r, p)
            assert a["true_relres"] <= 1e-8
    assert infos[1 * P + 1]["iters"] == 0 and torch.count_nonzero(U[1, N:2 * N]) == 0
    G.close()


def test_group_restarts_and_arguments():
    """restart = 6 (several cycles per problem; the problems need different numbers of
    cycles) against separate contexts, and the arguments a group refuses."""
    from paper_1409_0297_gb300 import binding as B
    d, n, b = 2, 128, 8
    ws = _members(d, n, b)
    P, N = len(ws), n ** d
    meds = [_medium(B, w) for w in ws]
    shifts = [m[0] for m in meds]
    qs = [torch.from_numpy(m[1]).cuda() for m in meds]
    fs = [torch.from_numpy(np.ascontiguousarray(w["f"])).cuda() for w in ws]
    G = B.Solver(d, n, b, shifts, prec=1, restart=6)
    G.factor(torch.cat(qs))
    ug = torch.empty(P * N, dtype=torch.complex128, device="cuda")
    infos = G.solve(torch.cat(fs), ug)
    torch.cuda.synchronize()
    assert max(i["restarts"] for i in infos) >= 2
    for p in range(P):
        S = B.Solver(d, n, b, shifts[p], prec=1, restart=6)
        S.factor(qs[p])
        u = torch.empty(N, dtype=torch.complex128, device="cuda")
        info = S.solve(fs[p], u)
        torch.cuda.synchronize()
        assert infos[p]["true_relres"] <= 1e-8
        assert abs(infos[p]["iters"] - info["iters"]) <= 2, p
        S.close()
    with pytest.raises(B.SpError):  # a start vector needs a single-problem context
        G.solve_x0(torch.cat(fs), ug, torch.empty_like(ug))
    G.close()
    with pytest.raises(B.SpError):  # the mixed-precision form takes one problem
        B.Solver(d, n, b, shifts, prec=B.SP_PREC_MIXED)
    with pytest.raises(B.SpError):  # more than 1024 Krylov instances
        B.Solver(d, n, b, shifts * 100, prec=1, max_rhs=4)
