"""The launch-shape autotuner (sp_opts.autotune): the tuned context picks a
Schur-update / block-inverse GEMM tile per level and must give results that are
bit-identical to the untuned context's (every output entry of those GEMMs is summed
in the same order whatever the tile), in the FP64, FP32 and TF32 forms."""
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


CASES = [
    ("2d_n128_b8", lambda: sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 4)),
    ("3d_n16_b4", lambda: sm.helmholtz_grf_3d(16, 4, 0)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [0, 1, 3], ids=["fp64", "fp32", "tf32"])
def test_autotune_is_bit_identical(B, name, make, prec):
    w = make()
    d, n, b = w["d"], w["n"], w["b"]
    s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
    qd = torch.from_numpy(q).cuda()
    fd = torch.from_numpy(w["f"]).cuda()
    out = []
    for tune in (False, True):
        S = B.Solver(d, n, b, s, prec=prec, autotune=tune)
        L = int(np.log2(n // b))
        shapes = [B.sp_tuning(S.ctx, l) for l in range(L + 1)]
        if tune:
            assert all(v["gemm_tile"] in (32, 64) for v in shapes)
        else:
            assert all(v["gemm_tile"] == 0 and v["gen_tile"] == 0 for v in shapes)
        S.factor(qd)
        u = torch.empty(n ** d, dtype=torch.complex128, device="cuda")
        info = S.solve(fd, u)
        torch.cuda.synchronize()
        out.append((u.cpu().numpy(), info["iters"], info["true_relres"]))
        with pytest.raises(B.SpError):
            B.sp_tuning(S.ctx, L + 1)
        S.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][2] <= 1e-8
