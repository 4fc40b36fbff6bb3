"""CPU tests of the C ABI: the library loads, exports every declared symbol, and its
host-only logic (argument checks, nested-dissection sizes, stencil tables, medium
split) agrees with the paper's formulas and with the oracle.  No GPU compute."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import synthetic_media as sm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _binding():
    from paper_1409_0297_gb300 import build as bld
    if not os.path.exists(bld.LIB):
        bld.build()
    from paper_1409_0297_gb300 import binding as B
    return B


def test_header_symbols_exported():
    B = _binding()
    hdr = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("sp.h", "sp_fno.h"))
    declared = set(re.findall(r"\b(sp_[a-z0-9_]+)\s*\(", hdr))
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(B.LIB, name), name
    assert declared == set(B.EXPORTED)


@pytest.mark.parametrize("d,n,b", [(2, 64, 4), (2, 512, 16), (3, 128, 8), (2, 16, 2), (3, 16, 4)])
def test_front_sizes_match_geometry(d, n, b):
    """Level l < L: k = (B-1)^d - 2^d (B/2-1)^d (B-1)^d at the leaves), m = k + (B+1)^d - (B-1)^d;
    root k = m = n^d - 2^d (n/2-1)^d (Section 2.3, Fig. nd)."""
    B_ = _binding()
    lv = B_.sp_front_sizes(d, n, b)
    L = int(np.log2(n // b))
    assert len(lv) == L + 1
    total = 0
    for l, (nf, k, m) in enumerate(lv[:-1]):
        B = b << l
        kk = (B - 1) ** d - (0 if l == 0 else 2 ** d * (B // 2 - 1) ** d)
        assert (nf, k, m) == ((n // B) ** d, kk, kk + (B + 1) ** d - (B - 1) ** d)
        total += nf * k
    root = lv[-1]
    assert root == (1, n ** d - 2 ** d * (n // 2 - 1) ** d, n ** d - 2 ** d * (n // 2 - 1) ** d)
    assert total + root[1] == n ** d  # every unknown is eliminated exactly once


def test_argument_checks_need_no_gpu():
    B = _binding()
    for args in [(2, 48, 4), (2, 64, 3), (4, 64, 4), (2, 8, 8), (2, 64, 1)]:
        with pytest.raises(B.SpError) as e:
            B.sp_setup(*args, s=100.0)
        assert e.value.status == B.SP_ERR_ARG
    # s = 4 pi^2 * 25 hits |k|^2 = 25: L - s singular
    with pytest.raises(B.SpError) as e:
        B.sp_setup(2, 64, 4, 4 * np.pi ** 2 * 25)
    assert e.value.status == B.SP_ERR_RESONANT


def test_group_argument_checks_need_no_gpu():
    """sp_setup_group refuses, before touching the device: no problems, a resonant shift
    among them, the mixed-precision form with several problems, more than 1024 Krylov
    instances (P max_rhs), a bad grid, more than 2^31 - 1 grid points in all (P n^d: the
    fronts' grid indices are ints); and the FP16 factor copy in the plain FP64 form."""
    B = _binding()
    cases = [
        (dict(shifts=[]), B.SP_ERR_ARG),
        (dict(shifts=[100.0, 4 * np.pi ** 2 * 25]), B.SP_ERR_RESONANT),
        (dict(shifts=[100.0, 101.0], prec=B.SP_PREC_MIXED), B.SP_ERR_ARG),
        (dict(shifts=[100.0] * 129, max_rhs=8), B.SP_ERR_ARG),
        (dict(shifts=[100.0, 101.0], n=48, b=4), B.SP_ERR_ARG),
        (dict(shifts=[100.0 + p for p in range(1024)], d=3, n=128, b=8), B.SP_ERR_ARG),
        (dict(shifts=[100.0], factor_storage=1, prec=B.SP_PREC_FP64), B.SP_ERR_ARG),
    ]
    for kw, status in cases:
        o = B.sp_default_opts()
        o.max_rhs = kw.get("max_rhs", 1)
        o.factor_storage = kw.get("factor_storage", 0)
        with pytest.raises(B.SpError) as e:
            B.sp_setup_group(kw.get("d", 2), kw.get("n", 64), kw.get("b", 4), kw["shifts"],
                             kw.get("prec", B.SP_PREC_FP32), o)
        assert e.value.status == status, kw


BAD_OPTS = [("maxit", 0), ("restart", 0), ("restart", 1001), ("tol", 0.0),
            ("tol", float("nan")), ("max_rhs", 0), ("max_rhs", 9), ("setup_route", 2),
            ("stencil", 2), ("inv_block", 100), ("inv_block", 32), ("inv_block", 4096),
            ("tc_epilogue", -1), ("tc_epilogue", 5), ("wait_limit_ns", -1),
            ("wait_limit_ns", 60000000001), ("sweeps", 3), ("panel_pivoting", 2),
            ("launch_overlap", 2), ("device_loop", -1), ("factor_storage", 2)]


@pytest.mark.parametrize("field,value", BAD_OPTS, ids=[f"{f}={v}" for f, v in BAD_OPTS])
def test_option_ranges_checked_before_the_device(field, value):
    """Every sp_opts field outside the range include/sp.h states is refused with
    SP_ERR_ARG by sp_setup before any device work (so this runs without a GPU)."""
    B = _binding()
    o = B.sp_default_opts()
    setattr(o, field, value)
    with pytest.raises(B.SpError) as e:
        B.sp_setup(2, 64, 4, 4 * np.pi ** 2 * 1.37, B.SP_PREC_FP32, o)
    assert e.value.status == B.SP_ERR_ARG


@pytest.mark.parametrize("d,n,b", [(2, 64, 4), (2, 24, 3), (3, 8, 2), (3, 16, 4),
                                   (2, 40, 5), (2, 56, 7), (3, 10, 5)])
def test_host_tables_match_oracle(d, n, b):
    B = _binding()
    s = 4 * np.pi ** 2 * (n / 6) ** 2 * 1.013
    tabs = O.stencil_tables(d, n, b, s)
    for t in range(1 << d):
        Q, C, rank, sig = B.sp_stencil_table(d, n, b, s, t)
        assert rank == tabs[t]["rank"]
        assert np.linalg.norm(Q - tabs[t]["Q"]) <= 1e-11 * np.linalg.norm(tabs[t]["Q"])
        assert np.linalg.norm(C - tabs[t]["C"]) <= 1e-11 * np.linalg.norm(tabs[t]["C"])
        k = min(64, len(tabs[t]["sigma"]))
        assert np.allclose(sig[:k], tabs[t]["sigma"][:k], rtol=1e-10, atol=0)


def test_medium_split_matches_oracle():
    B = _binding()
    d, n = 2, 64
    c = sm.grf_velocity(d, n, 0.1, 3)
    s1, q1 = B.sp_medium_helmholtz(d, n, 2 * np.pi * 7, c)
    s0, q0 = O.helmholtz_shift(d, n, 2 * np.pi * 7, c)
    assert abs(s1 - s0) <= 1e-12 * abs(s0)
    assert np.allclose(q1, q0, rtol=0, atol=1e-9 * abs(s0))
    V = sm.lattice_wells_potential(d, n, 4.0, 5)
    s1, q1 = B.sp_medium_schrodinger(d, n, 4.0, 3.0, V)
    s0, q0 = O.schrodinger_shift(d, n, 4.0, 3.0, V)
    assert abs(s1 - s0) <= 1e-12 * abs(s0)
    assert np.allclose(q1, q0, rtol=0, atol=1e-9 * abs(s0))
    # resonant: c = 1, omega = 2 pi 5 -> s/4pi^2 = 25 is moved off the lattice
    s1, q1 = B.sp_medium_helmholtz(d, n, 2 * np.pi * 5, np.ones(n * n))
    s0, q0 = O.helmholtz_shift(d, n, 2 * np.pi * 5, np.ones(n * n))
    assert abs(s1 - s0) <= 1e-12 * s0 and s1 != (2 * np.pi * 5) ** 2


def test_default_opts_layout():
    """sp_opts as the binding lays it out: the defaults documented in include/sp.h."""
    B = _binding()
    o = B.sp_default_opts()
    assert (o.maxit, o.restart, o.tol, o.pivot_tol) == (500, 200, 1e-8, 1e-14)
    assert (o.device, o.host_threads, o.inner_tol, o.autotune) == (0, 0, 1e-5, 0)
    assert (o.max_rhs, o.setup_route, o.stencil, o.inv_block, o.tc_epilogue) == (1, 0, 0, 0, 0)
    assert o.wait_limit_ns == 0 and o.sweeps == 0 and o.panel_pivoting == 0
    assert o.launch_overlap == 0 and o.device_loop == 1 and o.factor_storage == 0
    # the binding's layouts of sp_opts and sp_info match the build's
    assert B.LIB.sp_abi_size(0) == ctypes.sizeof(B.sp_opts)
    assert B.LIB.sp_abi_size(1) == ctypes.sizeof(B.sp_info)
    assert B.LIB.sp_abi_size(2) == 0


def test_fno_param_count_matches_oracle_layout():
    """The library's parameter count of the network equals the oracle's layout and the
    seeded initial weights' length; dims outside the documented ranges give 0."""
    from oracle import fno as F
    B = _binding()
    for D in (F.FnoDims(n=256), F.FnoDims(n=64, c_in=3, width=8, modes=6, layers=3, hidden=16),
              F.FnoDims(n=128, c_in=5, width=32, modes=16, layers=8, hidden=128, c_out=8)):
        dims = B.sp_fno_dims(D.n, D.c_in, D.width, D.modes, D.layers, D.hidden, D.c_out, 4, 0)
        assert B.sp_fno_param_count(dims) == F.param_count(D)
    assert B.sp_fno_param_count(B.sp_fno_dims(256, 3, 32, 16, 4, 128, 2, 16, 0)) == \
        sm.fno_initial_params().size
    for bad in ((100, 3, 32, 16, 4, 128, 2, 1, 0),    # n not a multiple of 64
                (64, 3, 33, 16, 4, 128, 2, 1, 0),     # width above 32
                (64, 3, 32, 17, 4, 128, 2, 1, 0),     # more than 16 modes
                (64, 3, 32, 16, 4, 129, 2, 1, 0),     # hidden above 128
                (64, 3, 32, 16, 4, 128, 2, 0, 0),     # batch_max 0
                (64, 3, 32, 16, 4, 128, 2, 1, 2)):    # act_fp32 not 0/1
        assert B.sp_fno_param_count(B.sp_fno_dims(*bad)) == 0


def test_medium_schrodinger_at_fixed_shift():
    """q(s) = l^2 V - l^2 E + s: at the context's own s it reproduces sp_medium_schrodinger,
    and q(s') - q(s) = s' - s everywhere (the operator -Laplace - s + q does not change)."""
    B = _binding()
    V = np.random.default_rng(3).uniform(-15, 0, 32 * 32)
    s, q = B.sp_medium_schrodinger(2, 32, 8.0, 10.0, V)
    assert np.array_equal(B.sp_medium_schrodinger_at(2, 32, 8.0, 10.0, V, s), q)
    q2 = B.sp_medium_schrodinger_at(2, 32, 8.0, 10.0, V, s + 7.5)
    assert np.allclose(q2 - q, 7.5, rtol=0, atol=1e-12)


def test_solver_dispatches_scalars_and_groups(monkeypatch):
    """Solver makes a single-problem context for any real scalar shift (float, numpy
    scalar, int) and a problem group for a sequence (list, array), with the options it
    was given; the set-up and destroy calls are replaced by recorders, so no GPU (and
    no library context) is touched."""
    B = _binding()
    calls = []
    monkeypatch.setattr(B, "sp_setup", lambda d, n, b, s, prec, o, st: calls.append(
        ("one", s, o.restart, o.factor_storage)) or 1)
    monkeypatch.setattr(B, "sp_setup_group", lambda d, n, b, sh, prec, o, st: calls.append(
        ("group", list(sh), o.restart, o.factor_storage)) or 2)
    monkeypatch.setattr(B, "sp_destroy", lambda ctx: calls.append(("destroy", ctx)))
    for s in (101.5, np.float64(101.5), 101, np.int64(101)):
        S = B.Solver(2, 64, 4, s, prec=B.SP_PREC_FP32, restart=7, factor_storage=1)
        assert (S.P, S.NP, S.ctx) == (1, 64 * 64, 1)
        assert calls[-1] == ("one", float(s), 7, 1) and isinstance(calls[-1][1], float)
        S.close()
    for sh in ([100.0, 101.0, 102.0], np.array([100.0, 101.0, 102.0])):
        S = B.Solver(2, 64, 4, sh, prec=B.SP_PREC_FP32, restart=7)
        assert (S.P, S.NP, S.ctx) == (3, 3 * 64 * 64, 2)
        assert calls[-1] == ("group", [100.0, 101.0, 102.0], 7, 0)
        S.close()
        assert calls[-1] == ("destroy", 2) and S.ctx is None


def test_host_allocation_failure_is_a_status():
    """A host allocation that fails inside the set-up comes back as SP_ERR_OOM instead
    of an exception crossing the C ABI (which would end the caller's process).  A child
    process caps its address space a little above what it already uses and asks for the
    3D 128^3 nested-dissection structure, whose assembly lists alone need hundreds of MB."""
    import subprocess
    import sys
    code = (
        "import re, resource, sys\n"
        "import numpy as np\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "from paper_1409_0297_gb300 import binding as B\n"
        "vm = int(re.search(r'VmSize:\\s+(\\d+)', open('/proc/self/status').read()).group(1)) * 1024\n"
        "resource.setrlimit(resource.RLIMIT_AS, (vm + (64 << 20), resource.getrlimit(resource.RLIMIT_AS)[1]))\n"
        "try:\n"
        "    B.sp_level_info(3, 128, 8, 0)\n"
        "    print('no error')\n"
        "except B.SpError as e:\n"
        "    print('status', e.status, e.status == B.SP_ERR_OOM)\n")
    _binding()
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == "status 5 True", p.stdout + p.stderr[-2000:]


def test_status_strings():
    """Every status of the header has its own message; an unknown code is named so."""
    B = _binding()
    codes = [B.SP_OK, B.SP_ERR_ARG, B.SP_ERR_RESONANT, B.SP_ERR_SINGULAR, B.SP_ERR_NOCONV,
             B.SP_ERR_OOM, B.SP_ERR_TIMEOUT, B.SP_ERR_CUDA, B.SP_ERR_STATE]
    assert codes == list(range(9))
    msgs = [B.status_str(c) for c in codes]
    assert len(set(msgs)) == len(msgs) and all(msgs)
    assert B.status_str(99) == "unknown status"
    e = B.SpError(B.SP_ERR_ARG, "sp_setup")
    assert "sp_setup" in str(e) and msgs[1] in str(e) and e.status == B.SP_ERR_ARG


def test_solver_rejects_vectors_it_cannot_pass(monkeypatch):
    """The binding only marshals: a vector of the wrong dtype, size, layout or device is
    refused before any library call (here on host tensors, with the set-up and every
    compute call replaced by recorders that must stay silent)."""
    torch = pytest.importorskip("torch")
    B = _binding()
    calls = []
    monkeypatch.setattr(B, "sp_setup", lambda *a: 1)
    monkeypatch.setattr(B, "sp_destroy", lambda ctx: None)
    for name in ("sp_factor", "sp_apply", "sp_solve", "sp_solve_many", "sp_green"):
        monkeypatch.setattr(B, name, lambda *a, _n=name, **k: calls.append(_n))
    S = B.Solver(2, 16, 4, 101.5)
    N = 16 * 16
    bad_vectors = [torch.zeros(N, dtype=torch.complex128),             # host memory
                   torch.zeros(N, dtype=torch.complex64),              # wrong dtype
                   torch.zeros(N - 1, dtype=torch.complex128),         # wrong size
                   torch.zeros(2 * N, dtype=torch.complex128)[::2]]    # not contiguous
    for x in bad_vectors:
        with pytest.raises(ValueError):
            S.apply(x, x)
        with pytest.raises(ValueError):
            S.solve(x, x)
        with pytest.raises(ValueError):
            S.solve_many(x, x)
    with pytest.raises(ValueError):
        S.factor(torch.zeros(N, dtype=torch.float64))
    assert calls == []
    S.close()


@pytest.mark.parametrize("d,n,b", [(2, 64, 4), (3, 16, 4)])
def test_tables_and_host_thread_count(d, n, b):
    """The Gram route computes each table on one thread, so its tables are the same
    bit for bit whatever sp_opts.host_threads is; the TSQR route combines one R factor
    per thread, so its tables agree across thread counts to rounding only."""
    B = _binding()
    s = 4 * np.pi ** 2 * (n / 8) ** 2 * 1.0137 if d == 2 else 4 * np.pi ** 2 * 7.3
    for t in range(1 << d):
        gram = [B.sp_stencil_table(d, n, b, s, t, host_threads=k, route=1) for k in (1, 3, 0)]
        for g in gram[1:]:
            assert np.array_equal(g[0], gram[0][0]) and np.array_equal(g[1], gram[0][1])
        tsqr = [B.sp_stencil_table(d, n, b, s, t, host_threads=k, route=0) for k in (1, 3, 0)]
        for q in tsqr[1:]:
            assert np.abs(q[0] - tsqr[0][0]).max() <= 1e-11 * max(1.0, np.abs(tsqr[0][0]).max())
            assert q[2] == tsqr[0][2]  # the same numerical rank


def test_grid_size_limit():
    """Grid indices are 32-bit, so every call that takes (d, n, b) refuses n^d >= 2^31
    with SP_ERR_ARG instead of overflowing; just below the limit the level sizes still
    follow the closed forms (Section 2.3, Fig. nd), computed here in exact integers."""
    B = _binding()
    for d, n, b in [(2, 65536, 16), (3, 2048, 16), (3, 1 << 20, 2)]:
        with pytest.raises(B.SpError) as e:
            B.sp_front_sizes(d, n, b)
        assert e.value.status == B.SP_ERR_ARG
        with pytest.raises(B.SpError):
            B.sp_level_info(d, n, b, 0)
    for d, n, b in [(3, 1024, 16), (2, 32768, 16)]:
        lv = B.sp_front_sizes(d, n, b)
        L = len(lv) - 1
        assert 2 ** L * b == n
        for l, (nf, k, m) in enumerate(lv[:-1]):
            Bx = b << l
            kk = (Bx - 1) ** d - (0 if l == 0 else 2 ** d * (Bx // 2 - 1) ** d)
            assert (nf, k, m) == ((n // Bx) ** d, kk, kk + (Bx + 1) ** d - (Bx - 1) ** d)
        kr = n ** d - 2 ** d * (n // 2 - 1) ** d
        assert lv[-1] == (1, kr, kr)


def test_medium_helpers_refuse_non_finite_media():
    """The Section 2.1 splits refuse media that have no meaning (a zero or non-finite
    wave speed, a non-finite potential or parameter) with SP_ERR_ARG and leave q
    untouched, instead of handing NaN or infinity to the factorisation."""
    B = _binding()
    n = 16
    c = np.ones(n * n)
    V = np.zeros(n * n)
    for bad in (0.0, np.nan, np.inf):
        cb = c.copy()
        cb[37] = bad
        with pytest.raises(B.SpError) as e:
            B.sp_medium_helmholtz(2, n, 2 * np.pi * 2, cb)
        assert e.value.status == B.SP_ERR_ARG
    for bad in (np.nan, -np.inf):
        Vb = V.copy()
        Vb[5] = bad
        with pytest.raises(B.SpError):
            B.sp_medium_schrodinger(2, n, 4.0, 10.0, Vb)
        with pytest.raises(B.SpError):
            B.sp_medium_schrodinger_at(2, n, 4.0, 10.0, Vb, 100.0)
    with pytest.raises(B.SpError):
        B.sp_medium_helmholtz(2, n, np.nan, c)
    with pytest.raises(B.SpError):
        B.sp_medium_schrodinger(2, n, 4.0, np.inf, V)
    with pytest.raises(B.SpError):
        B.sp_medium_schrodinger_at(2, n, 4.0, 10.0, V, np.nan)
    for s_bad in (np.nan, np.inf):  # the host tables refuse a non-finite shift too
        with pytest.raises(B.SpError) as e:
            B.sp_stencil_table(2, n, 4, s_bad, 0)
        assert e.value.status == B.SP_ERR_ARG
    s, q = B.sp_medium_helmholtz(2, n, 2 * np.pi * 2, c)  # the finite case still splits
    assert np.all(np.isfinite(q)) and np.isfinite(s)


def test_host_buffer_calls_refuse_foreign_arrays(monkeypatch):
    """sp_factor_host / sp_solve_host hand the library plain host memory, so the binding
    refuses arrays of another dtype, non-contiguous or read-only outputs and unequal
    sizes before the library is called (the library entry points are replaced by
    recorders that must stay silent)."""
    B = _binding()
    calls = []

    class Lib:
        def __getattr__(self, name):
            return lambda *a: calls.append(name) or 0
    monkeypatch.setattr(B, "LIB", Lib())
    N = 64
    with pytest.raises(ValueError):
        B.sp_factor_host(1, np.zeros(N, dtype=np.float32))
    with pytest.raises(ValueError):
        B.sp_factor_host(1, np.zeros(2 * N)[::2])
    with pytest.raises(ValueError):
        B.sp_factor_host(1, list(range(N)))
    f = np.zeros(N, dtype=np.complex128)
    with pytest.raises(ValueError):
        B.sp_solve_host(1, f.real.copy(), np.zeros(N, dtype=np.complex128))
    ro = np.zeros(N, dtype=np.complex128)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        B.sp_solve_host(1, f, ro)
    with pytest.raises(ValueError):
        B.sp_solve_host(1, f, np.zeros(N + 1, dtype=np.complex128))
    assert calls == []
    B.sp_factor_host(1, np.zeros(N))  # a valid array reaches the (recorded) library call
    assert calls == ["sp_factor_host"]
