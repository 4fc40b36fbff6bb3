"""Several right-hand sides in one call (sp_solve_many): the GMRES iterations of the
right-hand sides run in lockstep and share every preconditioner application and
operator product (stacked vectors through the same kernels), and every solution,
iteration count and residual history must be bit-identical to sp_solve's for that
right-hand side alone, in each precision form, including right-hand sides that
converge at different iterations, a zero right-hand side and restarts."""
import numpy as np
import pytest

import oracle as O
import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1409_0297_gb300 import binding
    assert torch.cuda.is_available()
    return binding


def problem(name):
    if name == "2d_n128_b8":
        w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)
    else:
        w = sm.helmholtz_grf_3d(16, 4, 0)
    d, n, b = w["d"], w["n"], w["b"]
    s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
    F = [sm.random_gaussian_source(d, n, 2500 + r, 0.05 + 0.03 * r) for r in range(5)]
    F[3] = np.zeros_like(F[3])  # a zero right-hand side stops at once
    return d, n, b, s, q, np.stack(F)


@pytest.mark.parametrize("name", ["2d_n128_b8", "3d_n16_b4"])
@pytest.mark.parametrize("prec,restart", [(0, 200), (1, 200), (3, 200), (0, 7)],
                         ids=["fp64", "fp32", "tf32", "fp64_restart7"])
def test_solve_many_matches_single(B, name, prec, restart):
    d, n, b, s, q, F = problem(name)
    N = n ** d
    S = B.Solver(d, n, b, s, prec=prec, restart=restart, max_rhs=8)
    S.factor(torch.from_numpy(q).cuda())
    Fd = torch.from_numpy(F).cuda().contiguous()
    U = torch.empty_like(Fd)
    infos = S.solve_many(Fd.view(-1), U.view(-1))
    torch.cuda.synchronize()
    Um = U.cpu().numpy()
    for r in range(F.shape[0]):
        u = torch.empty(N, dtype=torch.complex128, device="cuda")
        info = S.solve(Fd[r].contiguous(), u)
        torch.cuda.synchronize()
        assert infos[r]["iters"] == info["iters"], r
        assert infos[r]["restarts"] == info["restarts"], r
        assert np.array_equal(infos[r]["hist"], info["hist"]), r
        assert np.array_equal(Um[r], u.cpu().numpy()), r
        assert infos[r]["true_relres"] <= 1e-8
    if restart == 7:
        assert max(i["restarts"] for i in infos) > 0
    S.close()


def test_solve_many_arguments(B):
    d, n, b, s, q, F = problem("2d_n128_b8")
    S = B.Solver(d, n, b, s, prec=1, max_rhs=2)
    S.factor(torch.from_numpy(q).cuda())
    Fd = torch.from_numpy(F[:3]).cuda().contiguous()
    U = torch.empty_like(Fd)
    with pytest.raises(B.SpError):  # more right-hand sides than max_rhs
        S.solve_many(Fd.view(-1), U.view(-1))
    S.close()
    with pytest.raises(B.SpError):  # max_rhs beyond the sweeps' vector bound
        B.Solver(d, n, b, s, prec=1, max_rhs=9)
