"""Parity at the benchmark's own configuration: 2D 512^2, b = 16, both problems of
the pair, against values the FP64 CPU oracle wrote (tests/golden/make_golden_512.py,
which calls only `oracle/` and the seeded generators).

Per problem (Helmholtz on a random-field velocity, rescaled Schroedinger with a
16 x 16 lattice of wells):
  * the stencil tables Q(S, gamma), C(S, gamma) of every set type (Section 2.3) at
    1e-10 relative and the same pseudoinverse rank;
  * the FP64 preconditioner application z = P^{-1} Q r (Section 2.2) at 1e-10
    relative, element by element over all 262144 entries;
  * GMRES (Section 3; tolerance 1e-8): the FP64 form's iteration count within +-1 of
    the oracle's and its residual estimates at 1e-6 relative; every precision form's
    solution within 1e-6 relative of the oracle's u and a true residual
    ||g - (I + G q) u|| / ||g|| <= 1e-8 by the oracle's FFT operator.
The library's contexts are built with the default (TSQR + SVD) set-up route, the
benchmark's choice in 2D.
"""
import os

import numpy as np
import pytest

import oracle as O
import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(kind):
    path = os.path.join(GOLDEN, f"oracle_2d512_{kind}.npz")
    z = np.load(path)
    return {k: z[k] for k in z.files}


def _problem(kind):
    w = sm.helmholtz_grf_512() if kind == "helmholtz" else sm.schrodinger_wells_512()
    if kind == "helmholtz":
        s, q = O.helmholtz_shift(2, 512, w["omega"], w["c"])
        f = w["f"]
    else:
        s, q = O.schrodinger_shift(2, 512, w["ell"], w["E"], w["V"])
        f = w["f"] * w["ell"] ** 2
    return s, q, np.ascontiguousarray(f)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def B():
    from paper_1409_0297_gb300 import binding
    assert torch.cuda.is_available()
    return binding


@pytest.mark.parametrize("kind", ["helmholtz", "schrodinger"])
def test_tables_and_apply_512(B, kind):
    G = _load(kind)
    s, q, f = _problem(kind)
    assert abs(s - float(G["s"])) <= 1e-13 * abs(s)  # numpy's mean may round differently by host
    S = B.Solver(2, 512, 16, s, prec=B.SP_PREC_FP64)
    for t in range(4):
        Q, C, rank = S.table(t)
        assert rank == int(G[f"rank{t}"])
        assert rel(Q, G[f"Q{t}"]) <= 1e-10, (t, rel(Q, G[f"Q{t}"]))
        assert rel(C, G[f"C{t}"]) <= 1e-10, (t, rel(C, G[f"C{t}"]))
    S.factor(torch.from_numpy(q).cuda())
    r = sm.random_complex_vector(512 * 512, int(G["r_seed"]))
    z = torch.empty(512 * 512, dtype=torch.complex128, device="cuda")
    S.apply(torch.from_numpy(r).cuda(), z)
    zh = z.cpu().numpy()
    assert rel(zh, G["z"]) <= 1e-10, rel(zh, G["z"])
    S.close()


@pytest.mark.parametrize("kind", ["helmholtz", "schrodinger"])
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4], ids=["fp64", "fp32", "mixed", "tf32", "tf32x3"])
def test_solve_512_matches_oracle(B, kind, prec):
    G = _load(kind)
    s, q, f = _problem(kind)
    S = B.Solver(2, 512, 16, s, prec=prec)
    S.factor(torch.from_numpy(q).cuda())
    u = torch.empty(512 * 512, dtype=torch.complex128, device="cuda")
    info = S.solve(torch.from_numpy(f).cuda(), u)
    uh = u.cpu().numpy()
    S.close()
    g = O.apply_green(2, 512, s, f)
    true = float(np.linalg.norm(g - O.apply_operator(2, 512, s, q, uh)) / np.linalg.norm(g))
    assert true <= 1e-8, (true, info)
    assert rel(uh, G["u"].astype(np.complex128)) <= 1e-6, rel(uh, G["u"].astype(np.complex128))
    if prec == 0:
        assert abs(info["iters"] - int(G["iters"])) <= 1, (info["iters"], int(G["iters"]))
        h = G["hist"]
        m = min(len(h), len(info["hist"]))
        assert np.allclose(info["hist"][:m], h[:m], rtol=1e-6, atol=1e-12)
