"""GPU parity of the learned-initial-guess kernels (include/sp_fno.h) against the FP64
oracle network (oracle/fno.py), and of the solve from a starting vector (sp_solve_x0).

Both sides get the same bfloat16-rounded weights (the kernels compute with those), so
with FP32 activations what remains is FP32 accumulation (sums of at most a few
thousand terms: relative error ~1e-6, allowance 2e-5 on outputs and 2e-4 on gradient
groups, whose reductions run over every grid point of the batch).  With bfloat16
activations each stored activation carries a relative rounding of 2^-9; through four
layers and the projection the allowance is 3e-2.  A wrong twiddle sign, a transposed
weight or a dropped mode weight c_kx moves the output by O(1) relative.
"""
import numpy as np
import pytest

import oracle as O
import synthetic_media as sm
from oracle import fno as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1409_0297_gb300 import binding
    assert torch.cuda.is_available()
    return binding


SMALL = F.FnoDims(n=64, c_in=3, width=8, modes=6, layers=3, hidden=16, c_out=2)
FULL = F.FnoDims(n=64)  # width 32, 16 modes, 4 layers, hidden 128
WORKLOAD = F.FnoDims(n=256)  # the learned-guess workload's network at its grid size


def params(D, seed):
    th = sm.fno_initial_params(D.c_in, D.width, D.modes, D.layers, D.hidden, D.c_out, seed)
    parts = F.unpack(th.copy(), D)
    rng = np.random.default_rng(seed + 7)
    for l in range(D.layers):  # spectral weights large enough to matter
        R = parts[f"R{l}"]
        parts[f"R{l}"] = (rng.standard_normal(R.shape) + 1j * rng.standard_normal(R.shape)) * (2.0 / D.width)
    return F.bf16_round(F.pack(parts, D))


def inputs(D, batch, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((batch, D.c_in, D.n, D.n))
    t = rng.standard_normal((batch, D.c_out, D.n, D.n))
    return a, t


def dev32(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def make(B, D, th, batch_max, act_fp32):
    return B.Fno(D.n, th.astype(np.float32), D.c_in, D.width, D.modes, D.layers, D.hidden, D.c_out,
                 batch_max=batch_max, act_fp32=act_fp32)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("D", [SMALL, FULL, WORKLOAD], ids=["small", "full", "n256"])
@pytest.mark.parametrize("act_fp32", [True, False], ids=["fp32act", "bf16act"])
def test_forward_matches_oracle(B, D, act_fp32):
    th = params(D, 11)
    a, _ = inputs(D, 2, 12)
    net = make(B, D, th, 3, act_fp32)
    # inputs rounded to FP32 on both sides
    a32 = a.astype(np.float32).astype(np.float64)
    y = torch.empty((2, D.c_out, D.n * D.n), dtype=torch.float32, device="cuda")
    net.forward(dev32(a32), y, 2)
    torch.cuda.synchronize()
    ref = F.forward(th, a32, D)
    got = y.cpu().numpy().reshape(ref.shape).astype(np.float64)
    tol = 2e-5 if act_fp32 else 3e-2
    for b in range(2):
        assert rel(got[b], ref[b]) <= tol, (b, rel(got[b], ref[b]))
    net.close()


@pytest.mark.parametrize("D", [SMALL, FULL, WORKLOAD], ids=["small", "full", "n256"])
def test_gradient_matches_oracle(B, D):
    th = params(D, 21)
    a, t = inputs(D, 2, 22)
    a32, t32 = (x.astype(np.float32).astype(np.float64) for x in (a, t))
    net = make(B, D, th, 2, True)
    loss, g = net.gradient(dev32(a32), dev32(t32), 2)
    y, cache = F.forward(th, a32, D, keep=True)
    L, dy, _ = F.loss(y, t32)
    gref = F.backward(th, cache, dy, D)
    assert abs(loss - L) <= 1e-5 * L
    off = 0
    for name, shape in F.param_shapes(D):
        sz = int(np.prod(shape))
        gg, gr = g[off:off + sz].astype(np.float64), gref[off:off + sz]
        assert rel(gg, gr) <= 2e-4, (name, rel(gg, gr))
        off += sz
    net.close()


def test_adam_steps_match_oracle(B):
    """Two train steps: the kernels' Adam against the oracle's from the same gradients
    (the gradient itself is compared above)."""
    D = SMALL
    th = params(D, 31)
    a, t = inputs(D, 2, 32)
    xa, xt = dev32(a), dev32(t)
    net = make(B, D, th, 2, True)
    lr = 1e-3
    p = th.astype(np.float32).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in (1, 2):
        _, g = net.gradient(xa, xt, 2)
        L = net.train_step(xa, xt, 2, lr, sync=True)
        p, m, v = F.adam_step(p, m, v, g.astype(np.float64), step, lr)
        got = net.params().astype(np.float64)
        assert np.max(np.abs(got - p)) <= 1e-6 * max(1.0, np.max(np.abs(p))), step
        assert L > 0
    net.close()


def test_training_reduces_loss(B):
    D = SMALL
    th = sm.fno_initial_params(D.c_in, D.width, D.modes, D.layers, D.hidden, D.c_out, 41)
    rng = np.random.default_rng(42)
    a = rng.standard_normal((4, D.c_in, D.n, D.n))
    t = np.stack([np.sin(a[:, 1]) + 0.5 * a[:, 0], np.cos(a[:, 2])], axis=1)  # a pointwise map
    xa, xt = dev32(a), dev32(t)
    net = make(B, D, th, 4, False)
    first = net.train_step(xa, xt, 4, 3e-3, sync=True)
    for _ in range(60):
        net.train_step(xa, xt, 4, 3e-3)
    last, _ = net.gradient(xa, xt, 4, want_grad=False)
    assert last < 0.5 * first, (first, last)
    net.close()


def test_features_guess_target(B):
    """x = (q_scale q, g / c) with c = rms|g| e^{i phi}, phi = arg(sum g^2) / 2; for the
    random-phase Gaussian source (g = e^{i theta} G|f| with G real) g / c is real; the
    guess inverts the target's scaling up to FP32 rounding."""
    w = sm.schrodinger_wells(2, 64, 4, 4.0, 10.0, 3)
    s, q = O.schrodinger_shift(2, 64, w["ell"], w["E"], w["V"])
    S = B.Solver(2, 64, 4, s)
    qd = torch.from_numpy(q).cuda()
    S.factor(qd)
    f = torch.from_numpy(w["f"] * w["ell"] ** 2).cuda()
    g = torch.empty_like(f)
    S.green(f, g)
    D = F.FnoDims(n=64)
    net = make(B, D, sm.fno_initial_params(), 1, False)
    x = torch.empty((1, 3, 64 * 64), dtype=torch.float32, device="cuda")
    sc = torch.zeros(1, dtype=torch.complex128, device="cuda")
    net.features(qd, 1e-3, g, x, sc)
    gh = g.cpu().numpy()
    c = np.sqrt(np.mean(np.abs(gh) ** 2)) * np.exp(0.5j * np.angle(np.sum(gh * gh)))
    torch.cuda.synchronize()
    assert abs(sc.item() - c) <= 1e-12 * abs(c)
    xh = x.cpu().numpy()[0]
    assert np.allclose(xh[0], (1e-3 * q).astype(np.float32), rtol=1e-7, atol=0)
    assert np.allclose(xh[1] + 1j * xh[2], gh / c, rtol=0, atol=1e-6 * np.abs(gh / c).max())
    assert np.abs(xh[2]).max() <= 1e-6 * np.abs(xh[1]).max()
    t = torch.empty((1, 2, 64 * 64), dtype=torch.float32, device="cuda")
    net.target(g, sc, t)
    u0 = torch.empty_like(g)
    net.guess(t, sc, u0)
    torch.cuda.synchronize()
    assert rel(u0.cpu().numpy(), gh) <= 1e-7
    net.close()
    S.close()


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "mixed"])
def test_solve_from_starting_vector(B, prec):
    """sp_solve_x0: the exact solution needs no iteration; a perturbed one fewer than
    zero; a start worse than zero falls back to zero (same iterations as sp_solve);
    every solve ends at a true residual <= 1e-8 (the oracle's FFT residual)."""
    w = sm.helmholtz_centre_gaussian_64()
    d, n, b = w["d"], w["n"], w["b"]
    s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
    f = w["f"]
    S = B.Solver(d, n, b, s, prec=prec)
    S.factor(torch.from_numpy(q).cuda())
    fd = torch.from_numpy(f).cuda()
    u = torch.empty_like(fd)
    base = S.solve(fd, u)
    gref = O.apply_green(d, n, s, f)

    def true_res(x):
        return float(np.linalg.norm(gref - O.apply_operator(d, n, s, q, x)) / np.linalg.norm(gref))

    ustar = u.clone()
    u2 = torch.empty_like(u)
    info = S.solve_x0(fd, ustar, u2)
    assert info["iters"] == 0 and info["guess_used"] and info["guess_relres"] <= 1e-8
    rng = np.random.default_rng(5)
    pert = ustar.cpu().numpy() * (1 + 1e-3 * (rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)))
    info = S.solve_x0(fd, torch.from_numpy(pert).cuda(), u2)
    assert info["guess_used"] and info["guess_relres"] < 0.2
    assert info["iters"] < base["iters"] and true_res(u2.cpu().numpy()) <= 1e-8
    bad = torch.from_numpy(100.0 * (rng.standard_normal(n * n) + 0j)).cuda()
    info = S.solve_x0(fd, bad, u2)
    assert not info["guess_used"] and info["guess_relres"] > 1
    assert info["iters"] == base["iters"] and true_res(u2.cpu().numpy()) <= 1e-8
    info = S.solve_x0(fd, None, u2)
    assert info["iters"] == base["iters"] and torch.equal(u2, u)
    # the start may alias the output
    u3 = torch.from_numpy(pert).cuda()
    info = S.solve_x0(fd, u3, u3)
    assert info["guess_used"] and true_res(u3.cpu().numpy()) <= 1e-8
    S.close()


def test_fno_arguments(B):
    D = SMALL
    th = params(D, 51).astype(np.float32)
    with pytest.raises(B.SpError):
        B.Fno(100, th, D.c_in, D.width, D.modes, D.layers, D.hidden, D.c_out)  # n not a multiple of 64
    with pytest.raises(ValueError):
        B.Fno(D.n, th[:-1], D.c_in, D.width, D.modes, D.layers, D.hidden, D.c_out)
    net = make(B, D, th.astype(np.float64), 2, False)
    x = torch.zeros((3, D.c_in, D.n * D.n), dtype=torch.float32, device="cuda")
    y = torch.zeros((3, D.c_out, D.n * D.n), dtype=torch.float32, device="cuda")
    with pytest.raises(B.SpError):
        net.forward(x, y, 3)  # beyond batch_max
    with pytest.raises(B.SpError):
        net.train_step(x, y, 1, -1.0)  # negative learning rate
    net.close()


def test_features_guess_target_with_prior(B):
    """The prior-aware forms (input channels 3-4 = z / c, guess u0 = z + c y, target
    (u - z) / c) against numpy on random device data, and guess_prior inverting
    target_prior up to FP32 rounding of the correction."""
    n = 64
    N = n * n
    D = F.FnoDims(n=n, c_in=5)
    net = make(B, D, sm.fno_initial_params(c_in=5), 1, False)
    rng = np.random.default_rng(77)
    q = rng.standard_normal(N)
    g = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    z = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    u = z + 0.1 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    qd, gd, zd, ud = (torch.from_numpy(a).cuda() for a in (q, g, z, u))
    x = torch.empty((1, 5, N), dtype=torch.float32, device="cuda")
    sc = torch.zeros(1, dtype=torch.complex128, device="cuda")
    net.features_prior(qd, 0.5, gd, zd, x, sc)
    c = np.sqrt(np.mean(np.abs(g) ** 2)) * np.exp(0.5j * np.angle(np.sum(g * g)))
    xh = x.cpu().numpy()[0].astype(np.float64)
    assert abs(sc.item() - c) <= 1e-12 * abs(c)
    assert np.allclose(xh[0], 0.5 * q, rtol=1e-6, atol=1e-6)
    assert np.allclose(xh[1] + 1j * xh[2], g / c, rtol=1e-6, atol=1e-6)
    assert np.allclose(xh[3] + 1j * xh[4], z / c, rtol=1e-6, atol=1e-6)
    t = torch.empty((1, 2, N), dtype=torch.float32, device="cuda")
    net.target_prior(ud, sc, zd, t)
    th = t.cpu().numpy()[0].astype(np.float64)
    assert np.allclose(th[0] + 1j * th[1], (u - z) / c, rtol=1e-6, atol=1e-7)
    u0 = torch.empty(N, dtype=torch.complex128, device="cuda")
    net.guess_prior(t[0], sc, zd, u0)
    back = u0.cpu().numpy()
    assert np.linalg.norm(back - u) <= 1e-6 * np.linalg.norm(u - z) + 1e-12
    net.close()
