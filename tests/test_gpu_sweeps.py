"""The fused sweeps (one launch per level and direction, a thread-block cluster of up
to 16 CTAs per front on levels with few fronts; sp_opts.sweeps = 2 everywhere, 0 on
the levels with many fronts) against the per-block launch chains (sweeps = 1).  All
apply the same factor exactly (Section 2.3's forward and backward substitutions with
the block inverses), so in FP64 they agree to rounding:
1e-11 relative on grids where cond(P) ~ 1e4-1e5.  The fused path must launch one
forward and one backward kernel per level, and stacked right-hand sides (groups of
four per CTA) must give each vector the same bits as a single-vector application."""
import numpy as np
import pytest

import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("2d_n64_b4", lambda: sm.helmholtz_centre_gaussian_64()),
    ("2d_n512_b16", lambda: sm.helmholtz_grf_512()),
    ("3d_n16_b4", lambda: sm.helmholtz_grf_3d(16, 4, 0)),
    ("2d_n96_b6_schr", lambda: sm.schrodinger_wells(2, 96, 6, 6.0, 5.0, 17)),
]


def _medium(B, w):
    if w["kind"] == "helmholtz":
        return B.sp_medium_helmholtz(w["d"], w["n"], w["omega"], w["c"])
    return B.sp_medium_schrodinger(w["d"], w["n"], w["ell"], w["E"], w["V"])


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_fused_sweeps_match_chains(name, make, prec):
    from paper_1409_0297_gb300 import binding as B
    w = make()
    d, n, b = w["d"], w["n"], w["b"]
    s, q = _medium(B, w)
    N = n ** d
    r = torch.from_numpy(sm.random_complex_vector(N, 51)).cuda()
    out = []
    for sweeps in (2, 1, 0):
        S = B.Solver(d, n, b, s, prec=prec, sweeps=sweeps)
        S.factor(torch.from_numpy(q).cuda())
        z = torch.empty(N, dtype=torch.complex128, device="cuda")
        B.sp_profile(S.ctx, True)
        S.apply(r, z)
        prof = B.sp_profile_read(S.ctx)
        B.sp_profile(S.ctx, False)
        nlev = len(B.sp_front_sizes(d, n, b))
        if sweeps == 2:
            assert prof["forward"][1] == nlev and prof["backward"][1] == nlev, prof
        torch.cuda.synchronize()
        out.append(z.cpu().numpy())
        S.close()
    for z in (out[0], out[2]):
        rel = np.linalg.norm(z - out[1]) / np.linalg.norm(out[1])
        assert rel <= (1e-11 if prec == 0 else 2e-3), rel


@pytest.mark.parametrize("sweeps", [0, 2])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("nrhs", [3, 6])
def test_fused_sweeps_stacked_vectors_bit_identical(prec, nrhs, sweeps):
    """Groups of four vectors per CTA and a partial group give each vector the bits of
    its single-vector application (2D 512^2: the root is fused in clusters of 16)."""
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf_512()
    d, n, b = w["d"], w["n"], w["b"]
    s, q = _medium(B, w)
    N = n ** d
    S = B.Solver(d, n, b, s, prec=prec, max_rhs=8, sweeps=sweeps)
    S.factor(torch.from_numpy(q).cuda())
    F = torch.from_numpy(np.stack([sm.random_gaussian_source(2, n, 60 + i) for i in range(nrhs)])).cuda()
    U = torch.empty_like(F)
    infos = S.solve_many(F.view(-1), U.view(-1))
    for i in range(nrhs):
        u = torch.empty(N, dtype=torch.complex128, device="cuda")
        inf = S.solve(F[i].contiguous(), u)
        assert inf["iters"] == infos[i]["iters"]
        assert torch.equal(u, U[i])
    S.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_launch_overlap_bit_identical(prec):
    """Programmatic dependent launch of the stencil and sweep kernels
    (sp_opts.launch_overlap = 1) runs the same kernels in the same order: the
    preconditioner application and the solve are bit-identical to ordinary launches."""
    from paper_1409_0297_gb300 import binding as B
    w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)
    d, n, b = w["d"], w["n"], w["b"]
    s, q = _medium(B, w)
    N = n ** d
    r = torch.from_numpy(sm.random_complex_vector(N, 52)).cuda()
    f = torch.from_numpy(np.ascontiguousarray(w["f"])).cuda()
    out = []
    for lo in (0, 1):
        S = B.Solver(d, n, b, s, prec=prec, launch_overlap=lo)
        S.factor(torch.from_numpy(q).cuda())
        z = torch.empty(N, dtype=torch.complex128, device="cuda")
        u = torch.empty_like(z)
        S.apply(r, z)
        info = S.solve(f, u)
        torch.cuda.synchronize()
        out.append((z, u, info["iters"]))
        S.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
