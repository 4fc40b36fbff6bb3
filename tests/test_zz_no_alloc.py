"""GPU test of sp_green_static, the allocation-free form of sp_green.

Some callers cannot allocate device memory when they call into the library (a
stream being captured into a CUDA graph, or a fixed memory budget); for them
sp_green_static computes g = G f with a static work array instead of a context.
The test calls it through the C ABI twice in a row and compares each result with
the context-based sp_green and with the FP64 oracle's G f (numpy FFTs), both at
1e-13 relative (the tolerance of the other FFT tests), up to the largest grid the
array holds (64^3 = 2^18 points, every pass through the whole array), and checks
that a grid beyond the array's size is rejected.  It lives in a file collected
last so that a failure here leaves the other tests' results intact; it also passes
when run alone in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
import synthetic_media as sm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,n,b,s", [(2, 512, 16, 4 * np.pi ** 2 * 4096 * 1.0137),
                                     (2, 64, 4, 4 * np.pi ** 2 * 64 * 1.013),
                                     (3, 16, 4, 4 * np.pi ** 2 * 7.3),
                                     (3, 64, 8, 4 * np.pi ** 2 * 64 * 1.0071)])
def test_green_static_matches_sp_green(d, n, b, s):
    from paper_1409_0297_gb300 import binding as B
    assert torch.cuda.is_available()
    N = n ** d
    S = B.Solver(d, n, b, s, setup_route=1)
    for seed in (71, 72):  # two calls in a row share the static work array
        fh = sm.random_complex_vector(N, seed)
        f = torch.from_numpy(fh).cuda()
        g_ref = torch.empty_like(f)
        g = torch.empty_like(f)
        S.green(f, g_ref)
        B.sp_green_static(d, n, s, f.data_ptr(), g.data_ptr(), 0)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(g - g_ref) / torch.linalg.norm(g_ref)).item()
        assert err <= 1e-13, err
        go = O.apply_green(d, n, s, fh)
        gh = g.cpu().numpy()
        assert np.linalg.norm(gh - go) / np.linalg.norm(go) <= 1e-13
    S.close()


def test_green_static_rejects_oversize():
    from paper_1409_0297_gb300 import binding as B
    f = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.SpError) as e:
        B.sp_green_static(2, 1024, 100.0, f.data_ptr(), f.data_ptr() + 16, 0)
    assert e.value.status == B.SP_ERR_ARG
