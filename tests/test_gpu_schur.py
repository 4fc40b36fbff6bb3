"""The Schur-complement update kernels of the factorisation (Section 2.3,
S = F22 - L21 U12) checked in isolation through sp_schur_update.

C -= A B on batched column-major blocks with leading dimensions larger than the
row counts and ragged sizes (several 128 x 128 tensor-core tiles plus a partial
one, K not a multiple of 32).  The reference is numpy in FP64 on the same
inputs; for the tensor-core form the inputs are first rounded to TF32 (10-bit
mantissa, round to nearest with ties away from zero, the rounding the operand
packing applies), so what remains is the FP32 accumulation error, bounded
elementwise by (K + 2) * 2^-24 * (|A| |B|) + 2^-24 |C| (Higham, Thm 3.5 with FP32
unit roundoff).  The split form (3xTF32) is compared with the unrounded FP32
inputs: its extra error is the dropped lo*lo product and the rounding of the low
parts, 4 * 2^-22 |A||B| at most.  A wrong descriptor, swizzle or tile offset
breaks these bounds by orders of magnitude.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1409_0297_gb300 import binding
    assert torch.cuda.is_available()
    return binding


def tf32_round(x):
    """FP32 -> TF32 by rounding the magnitude to 10 mantissa bits, ties away from zero."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


def make(M, N, K, batch, lda, ldb, ldc, dtype, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, K, lda)).astype(dtype)   # column-major: [col][row]
    Bm = rng.standard_normal((batch, N, ldb)).astype(dtype)
    C = rng.standard_normal((batch, N, ldc)).astype(dtype)
    return A, Bm, C


SHAPES = [
    (300, 277, 256, 2),   # 3 x 3 tiles (ragged), sub-block depth
    (260, 390, 512, 1),   # full outer block depth
    (129, 130, 40, 3),    # K not a multiple of 32
    (1000, 64, 200, 1),   # tall
    (17, 900, 33, 2),     # one partial row tile, wide
]


@pytest.mark.parametrize("M,N,K,batch", SHAPES)
@pytest.mark.parametrize("prec", [0, 1, 3, 4], ids=["fp64", "fp32", "tf32", "tf32x3"])
def test_schur_update(B, M, N, K, batch, prec):
    dtype = np.float64 if prec == 0 else np.float32
    lda, ldb, ldc = M + 3, K + 5, M + 7
    A, Bm, C = make(M, N, K, batch, lda, ldb, ldc, dtype, 100 + M + K)
    tA, tB, tC = (torch.from_numpy(x).cuda() for x in (A, Bm, C))
    B.sp_schur_update(prec, M, N, K, tA.data_ptr(), lda, K * lda, tB.data_ptr(), ldb, N * ldb,
                      tC.data_ptr(), ldc, N * ldc, batch)
    torch.cuda.synchronize()
    out = tC.cpu().numpy()
    for f in range(batch):
        a = A[f, :, :M].T.astype(np.float64)   # M x K
        b = Bm[f, :, :K].T.astype(np.float64)  # K x N
        c = C[f, :, :M].T.astype(np.float64)   # M x N
        if prec == 3:
            a = tf32_round(a.astype(np.float32)).astype(np.float64)
            b = tf32_round(b.astype(np.float32)).astype(np.float64)
        ref = c - a @ b
        got = out[f, :, :M].T.astype(np.float64)
        u = 2.0 ** -53 if prec == 0 else 2.0 ** -24
        bound = (K + 2) * u * (np.abs(a) @ np.abs(b)) + u * np.abs(c) + 1e-300
        if prec == 4:
            # 3xTF32: the dropped lo*lo term and the TF32 rounding of the low parts
            # add at most 2^-22 |a||b| each per product (|a_lo| <= 2^-11 |a|)
            bound = bound + 4 * 2.0 ** -22 * (np.abs(a) @ np.abs(b))
        assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
        # rows beyond M and the padding of C are untouched
        assert np.array_equal(out[f, :, M:], C[f, :, M:])


def test_tf32_rounding_is_applied(B):
    """The tensor-core form must see TF32 operands: with A = 1 + 2^-20 (not a TF32
    value) and B = 1, the update is exactly K (the FP32 product would give
    K (1 + 2^-20))."""
    M, N, K = 128, 128, 64
    A = np.full((1, K, M), 1 + 2.0 ** -20, dtype=np.float32)
    Bm = np.ones((1, N, K), dtype=np.float32)
    C = np.zeros((1, N, M), dtype=np.float32)
    tA, tB, tC = (torch.from_numpy(x).cuda() for x in (A, Bm, C))
    B.sp_schur_update(3, M, N, K, tA.data_ptr(), M, K * M, tB.data_ptr(), K, N * K, tC.data_ptr(),
                      M, N * M, 1)
    torch.cuda.synchronize()
    assert np.all(tC.cpu().numpy() == -float(K))


def test_split_recovers_fp32_accuracy(B):
    """With A = 1 + 2^-20 and B = 1 the split form keeps the low part: the update
    is K (1 + 2^-20) to FP32 rounding, where plain TF32 gives exactly K."""
    M, N, K = 128, 128, 64
    A = np.full((1, K, M), 1 + 2.0 ** -20, dtype=np.float32)
    Bm = np.ones((1, N, K), dtype=np.float32)
    C = np.zeros((1, N, M), dtype=np.float32)
    tA, tB, tC = (torch.from_numpy(x).cuda() for x in (A, Bm, C))
    B.sp_schur_update(4, M, N, K, tA.data_ptr(), M, K * M, tB.data_ptr(), K, N * K, tC.data_ptr(),
                      M, N * M, 1)
    torch.cuda.synchronize()
    # K (1 + 2^-20) = 64 + 2^-14; plain TF32 would give 64 (2^-14 away)
    assert np.all(np.abs(tC.cpu().numpy().astype(np.float64) + K * (1 + 2.0 ** -20)) < 2.0 ** -16)


def test_schur_update_arguments(B):
    t = torch.zeros(64, device="cuda", dtype=torch.float32)
    p = t.data_ptr()
    with pytest.raises(B.SpError):  # K beyond the tensor-core kernel's limit (16384)
        B.sp_schur_update(3, 4, 4, 16416, p, 4, 0, p, 16416, 0, p, 4, 0, 1)
    with pytest.raises(B.SpError):  # leading dimension below the row count
        B.sp_schur_update(1, 8, 4, 4, p, 4, 0, p, 4, 0, p, 8, 0, 1)
    with pytest.raises(B.SpError):  # the mixed form has no update kernel of its own
        B.sp_schur_update(2, 4, 4, 4, p, 4, 0, p, 4, 0, p, 4, 0, 1)
    B.sp_schur_update(3, 0, 4, 4, p, 1, 0, p, 4, 0, p, 1, 0, 1)  # empty: nothing to do
