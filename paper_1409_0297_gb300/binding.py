"""ctypes binding of the C ABI in include/sp.h and include/sp_fno.h (argument marshalling only).

Every function below forwards to the function of the same name in
libsp_gb300.so; all arithmetic happens in the library's CUDA kernels.  Device
buffers are passed as integer addresses (e.g. torch.Tensor.data_ptr()); the
convenience class Solver takes torch CUDA tensors and checks their dtype, size
and contiguity before passing the pointers on.  If the library is missing the
import of this module raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsp_gb300.so")

SP_OK, SP_ERR_ARG, SP_ERR_RESONANT, SP_ERR_SINGULAR, SP_ERR_NOCONV = 0, 1, 2, 3, 4
SP_ERR_OOM, SP_ERR_TIMEOUT, SP_ERR_CUDA, SP_ERR_STATE = 5, 6, 7, 8
SP_PREC_FP64, SP_PREC_FP32, SP_PREC_MIXED, SP_PREC_TF32, SP_PREC_TF32X3 = 0, 1, 2, 3, 4

EXPORTED = [
    "sp_abi_size", "sp_default_opts", "sp_setup", "sp_setup_group", "sp_problems", "sp_factor", "sp_apply", "sp_solve", "sp_factor_host",
    "sp_solve_host", "sp_matvec", "sp_green", "sp_qapply", "sp_get_table", "sp_set_table", "sp_stencil_table",
    "sp_front_sizes", "sp_level_info", "sp_costs", "sp_medium_helmholtz", "sp_medium_schrodinger", "sp_profile",
    "sp_profile_read", "sp_green_static", "sp_schur_update", "sp_tc_probe", "sp_tuning", "sp_solve_many",
    "sp_solve_x0", "sp_medium_schrodinger_at", "sp_destroy", "sp_status_str",
    "sp_fno_param_count", "sp_fno_create", "sp_fno_destroy", "sp_fno_set_params",
    "sp_fno_get_params", "sp_fno_forward", "sp_fno_gradient", "sp_fno_train_step",
    "sp_fno_features", "sp_fno_guess", "sp_fno_target", "sp_fno_features_prior",
    "sp_fno_guess_prior", "sp_fno_target_prior",
]
PROF_CLASSES = ["assemble", "lu_panel", "lu_trsm", "lu_gemm", "qapply", "forward", "backward",
                "fft", "krylov", "lu_trinv", "lu_tc"]


class sp_opts(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int), ("restart", ctypes.c_int), ("tol", ctypes.c_double),
                ("pivot_tol", ctypes.c_double), ("device", ctypes.c_int),
                ("host_threads", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("autotune", ctypes.c_int), ("max_rhs", ctypes.c_int),
                ("setup_route", ctypes.c_int), ("stencil", ctypes.c_int),
                ("inv_block", ctypes.c_int), ("tc_epilogue", ctypes.c_int),
                ("wait_limit_ns", ctypes.c_longlong), ("sweeps", ctypes.c_int),
                ("panel_pivoting", ctypes.c_int), ("launch_overlap", ctypes.c_int),
                ("device_loop", ctypes.c_int), ("factor_storage", ctypes.c_int)]


class sp_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("est_relres", ctypes.c_double), ("true_relres", ctypes.c_double),
                ("s_used", ctypes.c_double), ("hist", ctypes.POINTER(ctypes.c_double)),
                ("hist_cap", ctypes.c_int), ("hist_len", ctypes.c_int),
                ("guess_relres", ctypes.c_double), ("guess_used", ctypes.c_int)]


class sp_fno_dims(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("c_in", ctypes.c_int), ("width", ctypes.c_int),
                ("modes", ctypes.c_int), ("layers", ctypes.c_int), ("hidden", ctypes.c_int),
                ("c_out", ctypes.c_int), ("batch_max", ctypes.c_int), ("act_fp32", ctypes.c_int)]


class sp_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


class SpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} (status {status})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1409_0297_gb300.build.build() "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    pI, pD = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "sp_abi_size": (ctypes.c_size_t, [I]),
        "sp_default_opts": (V, [ctypes.POINTER(sp_opts)]),
        "sp_setup": (I, [I, I, I, D, I, ctypes.POINTER(sp_opts), P, ctypes.POINTER(P)]),
        "sp_setup_group": (I, [I, I, I, I, pD, I, ctypes.POINTER(sp_opts), P, ctypes.POINTER(P)]),
        "sp_problems": (I, [P, pI]),
        "sp_factor": (I, [P, P]),
        "sp_apply": (I, [P, P, P]),
        "sp_solve": (I, [P, P, P, ctypes.POINTER(sp_info)]),
        "sp_factor_host": (I, [P, P]),
        "sp_solve_host": (I, [P, P, P, ctypes.POINTER(sp_info)]),
        "sp_matvec": (I, [P, P, P]),
        "sp_green": (I, [P, P, P]),
        "sp_qapply": (I, [P, P, P]),
        "sp_get_table": (I, [P, I, pD, pD, pI, pI, pI]),
        "sp_set_table": (I, [P, I, pD, pD]),
        "sp_stencil_table": (I, [I, I, I, D, I, I, I, I, pD, pD, pI, pI, pI, pD]),
        "sp_front_sizes": (I, [I, I, I, I, pI, pI, pI, pI]),
        "sp_costs": (I, [P, pD, pD, pD]),
        "sp_level_info": (I, [I, I, I, I, pI, pI, pI, pI, pI, pI, pI, pI, pI, pI]),
        "sp_medium_helmholtz": (I, [I, I, D, P, pD, P]),
        "sp_medium_schrodinger": (I, [I, I, D, D, P, pD, P]),
        "sp_profile": (I, [P, I]),
        "sp_profile_read": (I, [P, I, pD, pI, pD]),
        "sp_green_static": (I, [I, I, D, P, P, P]),
        "sp_schur_update": (I, [I, I, I, I, P, I, ctypes.c_longlong, P, I, ctypes.c_longlong, P, I,
                                ctypes.c_longlong, I, P]),
        "sp_tc_probe": (I, [I, I, I, I, I, P, pD]),
        "sp_tuning": (I, [P, I, pI, pI]),
        "sp_solve_many": (I, [P, I, P, P, ctypes.POINTER(sp_info)]),
        "sp_solve_x0": (I, [P, P, P, P, ctypes.POINTER(sp_info)]),
        "sp_medium_schrodinger_at": (I, [I, I, D, D, P, D, P]),
        "sp_fno_param_count": (ctypes.c_longlong, [ctypes.POINTER(sp_fno_dims)]),
        "sp_fno_create": (I, [ctypes.POINTER(sp_fno_dims), P, P, ctypes.POINTER(P)]),
        "sp_fno_destroy": (V, [P]),
        "sp_fno_set_params": (I, [P, P]),
        "sp_fno_get_params": (I, [P, P]),
        "sp_fno_forward": (I, [P, I, P, P]),
        "sp_fno_gradient": (I, [P, I, P, P, P, pD, P]),
        "sp_fno_train_step": (I, [P, I, P, P, ctypes.POINTER(sp_adam), pD]),
        "sp_fno_features": (I, [P, P, D, P, P, P]),
        "sp_fno_guess": (I, [P, P, P, P]),
        "sp_fno_target": (I, [P, P, P, P]),
        "sp_fno_features_prior": (I, [P, P, D, P, P, P, P]),
        "sp_fno_guess_prior": (I, [P, P, P, P, P]),
        "sp_fno_target_prior": (I, [P, P, P, P, P]),
        "sp_destroy": (V, [P]),
        "sp_status_str": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()


def status_str(st: int) -> str:
    return LIB.sp_status_str(st).decode()


def _check(st: int, where: str, ok=(SP_OK,)):
    if st not in ok:
        raise SpError(st, where)
    return st


def _dptr(a):
    """numpy float64 array -> POINTER(c_double)."""
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------------ same-name wrappers
def sp_default_opts() -> sp_opts:
    o = sp_opts()
    LIB.sp_default_opts(ctypes.byref(o))
    return o


def sp_setup(d: int, n: int, b: int, s: float, prec: int = SP_PREC_FP64, opts: sp_opts | None = None,
             stream: int = 0) -> int:
    ctx = ctypes.c_void_p()
    _check(LIB.sp_setup(d, n, b, float(s), prec, ctypes.byref(opts) if opts else None,
                        ctypes.c_void_p(stream), ctypes.byref(ctx)), "sp_setup")
    return ctx.value


def sp_setup_group(d: int, n: int, b: int, shifts, prec: int = SP_PREC_FP64,
                   opts: sp_opts | None = None, stream: int = 0) -> int:
    """A context of len(shifts) problems of one grid and leaf size (a problem group)."""
    import numpy as np
    sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64).ravel())
    ctx = ctypes.c_void_p()
    _check(LIB.sp_setup_group(d, n, b, int(sh.size), _dptr(sh), prec,
                              ctypes.byref(opts) if opts else None, ctypes.c_void_p(stream),
                              ctypes.byref(ctx)), "sp_setup_group")
    return ctx.value


def sp_problems(ctx: int) -> int:
    P = ctypes.c_int()
    _check(LIB.sp_problems(ctx, ctypes.byref(P)), "sp_problems")
    return P.value


def sp_factor(ctx: int, q_dev: int) -> None:
    _check(LIB.sp_factor(ctx, q_dev), "sp_factor")


def _host_array(a, dtype, name: str, writeable: bool = False) -> int:
    """Address of a C-contiguous numpy array of the given dtype (the library reads or
    writes it as plain memory, so anything else is refused here)."""
    import numpy as np
    if not (isinstance(a, np.ndarray) and a.dtype == np.dtype(dtype) and a.flags["C_CONTIGUOUS"]
            and (a.flags["WRITEABLE"] or not writeable)):
        raise ValueError(f"{name}: expected a C-contiguous{' writeable' if writeable else ''} "
                         f"numpy {np.dtype(dtype)} array")
    return a.ctypes.data


def sp_factor_host(ctx: int, q_host) -> None:
    import numpy as np
    _check(LIB.sp_factor_host(ctx, _host_array(q_host, np.float64, "q_host")), "sp_factor_host")


def sp_apply(ctx: int, r_dev: int, z_dev: int) -> None:
    _check(LIB.sp_apply(ctx, r_dev, z_dev), "sp_apply")


def sp_qapply(ctx: int, r_dev: int, y_dev: int) -> None:
    _check(LIB.sp_qapply(ctx, r_dev, y_dev), "sp_qapply")


def sp_matvec(ctx: int, x_dev: int, w_dev: int) -> None:
    _check(LIB.sp_matvec(ctx, x_dev, w_dev), "sp_matvec")


def sp_green(ctx: int, f_dev: int, g_dev: int) -> None:
    _check(LIB.sp_green(ctx, f_dev, g_dev), "sp_green")


def _info(hist_cap: int):
    import numpy as np
    info = sp_info()
    hist = np.zeros(max(1, hist_cap), dtype=np.float64)
    info.hist = _dptr(hist)
    info.hist_cap = hist_cap
    return info, hist


def _info_dict(info, hist, st):
    return dict(status=st, iters=info.iters, restarts=info.restarts, est_relres=info.est_relres,
                true_relres=info.true_relres, s_used=info.s_used,
                hist=hist[: info.hist_len].copy(), guess_relres=info.guess_relres,
                guess_used=bool(info.guess_used))


def _infos(count: int, hist_cap: int):
    infos = (sp_info * count)()
    hists = []
    for i in range(count):
        info, hist = _info(hist_cap)
        infos[i] = info  # copies the struct, including the pointer to hist
        hists.append(hist)
    return infos, hists


def sp_solve(ctx: int, f_dev: int, u_dev: int, hist_cap: int = 1024, allow_noconv=False,
             nprob: int = 1):
    """One info dict; a list of nprob dicts for a group of nprob problems."""
    infos, hists = _infos(nprob, hist_cap)
    st = LIB.sp_solve(ctx, f_dev, u_dev, infos)
    _check(st, "sp_solve", (SP_OK, SP_ERR_NOCONV) if allow_noconv else (SP_OK,))
    out = [_info_dict(infos[i], hists[i], st) for i in range(nprob)]
    return out[0] if nprob == 1 else out


def sp_solve_x0(ctx: int, f_dev: int, u0_dev: int | None, u_dev: int, hist_cap: int = 1024,
                allow_noconv=False) -> dict:
    info, hist = _info(hist_cap)
    st = LIB.sp_solve_x0(ctx, f_dev, u0_dev, u_dev, ctypes.byref(info))
    _check(st, "sp_solve_x0", (SP_OK, SP_ERR_NOCONV) if allow_noconv else (SP_OK,))
    return _info_dict(info, hist, st)


def sp_solve_many(ctx: int, nrhs: int, F_dev: int, U_dev: int, hist_cap: int = 1024,
                  allow_noconv=False, nprob: int = 1) -> list:
    """nrhs right-hand sides of each of the nprob problems (right-hand side r of
    problem p at offset (r nprob + p) N); one info dict per (r, p), in that order."""
    infos, hists = _infos(nrhs * nprob, hist_cap)
    st = LIB.sp_solve_many(ctx, nrhs, F_dev, U_dev, infos)
    _check(st, "sp_solve_many", (SP_OK, SP_ERR_NOCONV) if allow_noconv else (SP_OK,))
    return [_info_dict(infos[i], hists[i], st) for i in range(nrhs * nprob)]


def sp_solve_host(ctx: int, f_host, u_host, hist_cap: int = 1024, allow_noconv=False,
                  nprob: int = 1):
    import numpy as np
    pf = _host_array(f_host, np.complex128, "f_host")
    pu = _host_array(u_host, np.complex128, "u_host", writeable=True)
    if f_host.size != u_host.size:
        raise ValueError("f_host and u_host must have the same number of entries")
    infos, hists = _infos(nprob, hist_cap)
    st = LIB.sp_solve_host(ctx, pf, pu, infos)
    _check(st, "sp_solve_host", (SP_OK, SP_ERR_NOCONV) if allow_noconv else (SP_OK,))
    out = [_info_dict(infos[i], hists[i], st) for i in range(nprob)]
    return out[0] if nprob == 1 else out


def sp_get_table(ctx: int, t: int):
    import numpy as np
    rows, cols, rank = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(LIB.sp_get_table(ctx, t, None, None, ctypes.byref(rows), ctypes.byref(cols),
                            ctypes.byref(rank)), "sp_get_table")
    Q = np.zeros((rows.value, cols.value))
    C = np.zeros((rows.value, cols.value))
    _check(LIB.sp_get_table(ctx, t, _dptr(Q), _dptr(C), ctypes.byref(rows), ctypes.byref(cols),
                            ctypes.byref(rank)), "sp_get_table")
    return Q, C, rank.value


def sp_stencil_table(d: int, n: int, b: int, s: float, t: int, host_threads: int = 0,
                     route: int = 0, kind: int = 0):
    """Host-only stencil tables (no GPU needed): returns (Q, C, rank, sigma).
    route 0: TSQR + SVD, 1: Gram route; kind 0: set stencils, 1: per-point stencils."""
    import numpy as np
    rows, cols, rank = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(LIB.sp_stencil_table(d, n, b, float(s), t, route, kind, host_threads, None, None,
                                ctypes.byref(rows), ctypes.byref(cols), None, None),
           "sp_stencil_table")
    Q = np.zeros((rows.value, cols.value))
    C = np.zeros((rows.value, cols.value))
    sig = np.zeros(64)
    _check(LIB.sp_stencil_table(d, n, b, float(s), t, route, kind, host_threads, _dptr(Q),
                                _dptr(C),
                                ctypes.byref(rows), ctypes.byref(cols), ctypes.byref(rank),
                                _dptr(sig)), "sp_stencil_table")
    nb = 3 ** d - 1 if kind else Q.shape[1] - Q.shape[0]  # |beta| of the pseudoinverse
    return Q, C, rank.value, sig[: min(64, nb)]


def sp_front_sizes(d: int, n: int, b: int):
    cap = 64
    nl = ctypes.c_int()
    nf, k, m = (ctypes.c_int * cap)(), (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
    _check(LIB.sp_front_sizes(d, n, b, cap, ctypes.byref(nl), nf, k, m), "sp_front_sizes")
    return [(nf[i], k[i], m[i]) for i in range(nl.value)]


def sp_level_info(d: int, n: int, b: int, level: int) -> dict:
    """Host-only symbolic data of one nested-dissection level (see include/sp.h)."""
    import numpy as np
    v = [ctypes.c_int() for _ in range(6)]
    _check(LIB.sp_level_info(d, n, b, level, *[ctypes.byref(x) for x in v], None, None, None, None),
           "sp_level_info")
    nf, k, m, mc, kc, nasm = (x.value for x in v)
    gidx = np.zeros(nf * m, dtype=np.int32)
    ea = np.zeros(max(1, (1 << d) * (mc - kc)), dtype=np.int32)
    row = np.zeros(max(1, nasm), dtype=np.int32)
    cvar = np.zeros(max(1, nasm), dtype=np.int32)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _check(LIB.sp_level_info(d, n, b, level, *[ctypes.byref(x) for x in v], ip(gidx), ip(ea),
                             ip(row), ip(cvar)), "sp_level_info")
    return dict(nf=nf, k=k, m=m, mc=mc, kc=kc, gidx=gidx.reshape(nf, m),
                ea_map=ea[: (1 << d) * (mc - kc)].reshape(1 << d, mc - kc) if mc else None,
                asm_row=row[:nasm], asm_cvar=cvar[:nasm])


def sp_costs(ctx: int):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(LIB.sp_costs(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "sp_costs")
    return dict(factor_entries=a.value, factor_flops=b.value, apply_bytes=c.value)


def sp_medium_helmholtz(d: int, n: int, omega: float, c):
    import numpy as np
    c = np.ascontiguousarray(c, dtype=np.float64)
    q = np.empty_like(c)
    s = ctypes.c_double()
    _check(LIB.sp_medium_helmholtz(d, n, float(omega), c.ctypes.data, ctypes.byref(s),
                                   q.ctypes.data), "sp_medium_helmholtz")
    return s.value, q


def sp_medium_schrodinger(d: int, n: int, ell: float, E: float, V):
    import numpy as np
    V = np.ascontiguousarray(V, dtype=np.float64)
    q = np.empty_like(V)
    s = ctypes.c_double()
    _check(LIB.sp_medium_schrodinger(d, n, float(ell), float(E), V.ctypes.data, ctypes.byref(s),
                                     q.ctypes.data), "sp_medium_schrodinger")
    return s.value, q


def sp_medium_schrodinger_at(d: int, n: int, ell: float, E: float, V, s: float):
    import numpy as np
    V = np.ascontiguousarray(V, dtype=np.float64)
    q = np.empty_like(V)
    _check(LIB.sp_medium_schrodinger_at(d, n, float(ell), float(E), V.ctypes.data, float(s),
                                        q.ctypes.data), "sp_medium_schrodinger_at")
    return q


def sp_profile(ctx: int, enable: bool) -> None:
    _check(LIB.sp_profile(ctx, 1 if enable else 0), "sp_profile")


def sp_profile_read(ctx: int) -> dict:
    """{class: (ms, launches, work)} since the last read (work: flops or bytes)."""
    import numpy as np
    k = len(PROF_CLASSES)
    ms, wk = np.zeros(k), np.zeros(k)
    ln = (ctypes.c_int * k)()
    _check(LIB.sp_profile_read(ctx, k, _dptr(ms), ln, _dptr(wk)), "sp_profile_read")
    return {c: (float(ms[i]), int(ln[i]), float(wk[i])) for i, c in enumerate(PROF_CLASSES)}


def sp_green_static(d: int, n: int, s: float, f_dev: int, g_dev: int, stream: int = 0) -> None:
    """g = G f without a context or any allocation (see include/sp.h)."""
    _check(LIB.sp_green_static(d, n, float(s), f_dev, g_dev, stream), "sp_green_static")


def sp_schur_update(prec: int, M: int, N: int, K: int, A_dev: int, lda: int, sA: int, B_dev: int,
                    ldb: int, sB: int, C_dev: int, ldc: int, sC: int, batch: int,
                    stream: int = 0) -> None:
    """C -= A B (column-major, batched) with the factorisation's update kernel."""
    _check(LIB.sp_schur_update(prec, M, N, K, A_dev, lda, sA, B_dev, ldb, sB, C_dev, ldc, sC, batch,
                               stream), "sp_schur_update")


def sp_tc_probe(split: int, M: int, N: int, K: int, reps: int = 10, stream: int = 0) -> float:
    """Device milliseconds per launch of the tcgen05 update kernel on generated
    operands (C[M x N] -= A[M x K] B[K x N]; split = 1: 3xTF32)."""
    ms = ctypes.c_double()
    _check(LIB.sp_tc_probe(split, M, N, K, reps, stream, ctypes.byref(ms)), "sp_tc_probe")
    return ms.value


def sp_tuning(ctx: int, level: int) -> dict:
    """Launch shapes of one level (0 = built-in heuristic)."""
    v = [ctypes.c_int() for _ in range(2)]
    _check(LIB.sp_tuning(ctx, level, *[ctypes.byref(x) for x in v]), "sp_tuning")
    return dict(gemm_tile=v[0].value, gen_tile=v[1].value)


def sp_destroy(ctx: int) -> None:
    LIB.sp_destroy(ctx)


# ------------------------------------------------------------------ convenience class
class Solver:
    """Owns one context.  Vectors are torch complex128 CUDA tensors of n^d entries,
    q a float64 CUDA tensor (factor copies it into the context).  With a sequence of
    shifts s the context is a problem group (sp_setup_group): vectors and q hold P n^d
    entries, problem p's at p n^d, and solve returns one info dict per problem."""

    def __init__(self, d: int, n: int, b: int, s, prec: int = SP_PREC_FP64,
                 maxit: int = 500, restart: int = 200, tol: float = 1e-8, device: int = 0,
                 stream: int = 0, host_threads: int = 0, autotune: bool = False,
                 max_rhs: int = 1, setup_route: int = 0, stencil: int = 0, inv_block: int = 0,
                 tc_epilogue: int = 0, wait_limit_ns: int = 0, sweeps: int = 0,
                 panel_pivoting: int = 0, launch_overlap: int = 0, device_loop: int = 1,
                 factor_storage: int = 0):
        o = sp_default_opts()
        o.maxit, o.restart, o.tol, o.device = maxit, restart, tol, device
        o.host_threads = host_threads
        o.autotune = 1 if autotune else 0
        o.max_rhs = max_rhs
        o.setup_route = setup_route
        o.stencil = stencil
        o.inv_block = inv_block
        o.tc_epilogue = tc_epilogue
        o.wait_limit_ns = wait_limit_ns
        o.sweeps = sweeps
        o.panel_pivoting = panel_pivoting
        o.launch_overlap = launch_overlap
        o.device_loop = device_loop
        o.factor_storage = factor_storage
        self.d, self.n, self.b, self.s, self.prec = d, n, b, s, prec
        self.device = device
        self.N = n ** d
        import numpy as np
        if np.ndim(s) == 0:  # one shift (any real scalar); a sequence makes a group
            self.P = 1
            self.ctx = sp_setup(d, n, b, float(s), prec, o, stream)
        else:
            self.P = len(s)
            self.ctx = sp_setup_group(d, n, b, s, prec, o, stream)
        self.NP = self.P * self.N
        self._q = None

    def _vec(self, x, dtype):
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == dtype and
                x.is_contiguous() and x.numel() == self.NP and x.get_device() == self.device):
            raise ValueError(f"expected a contiguous {dtype} tensor of {self.NP} entries on "
                             f"cuda:{self.device}")
        return x.data_ptr()

    def solve_many(self, F, U, **kw):
        """F, U: contiguous CUDA complex128 tensors of nrhs x P x N entries."""
        import torch
        nrhs = F.numel() // self.NP
        for x in (F, U):
            if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.complex128 and
                    x.is_contiguous() and x.numel() == nrhs * self.NP and nrhs >= 1 and
                    x.get_device() == self.device):
                raise ValueError("expected contiguous complex128 tensors of nrhs x P x N entries "
                                 f"on cuda:{self.device}")
        return sp_solve_many(self.ctx, nrhs, F.data_ptr(), U.data_ptr(), nprob=self.P, **kw)

    def factor(self, q):
        import torch
        p = self._vec(q, torch.float64)
        self._q = q
        sp_factor(self.ctx, p)

    def apply(self, r, z):
        import torch
        sp_apply(self.ctx, self._vec(r, torch.complex128), self._vec(z, torch.complex128))

    def qapply(self, r, y):
        import torch
        sp_qapply(self.ctx, self._vec(r, torch.complex128), self._vec(y, torch.complex128))

    def matvec(self, x, w):
        import torch
        sp_matvec(self.ctx, self._vec(x, torch.complex128), self._vec(w, torch.complex128))

    def green(self, f, g):
        import torch
        sp_green(self.ctx, self._vec(f, torch.complex128), self._vec(g, torch.complex128))

    def solve(self, f, u, **kw):
        import torch
        return sp_solve(self.ctx, self._vec(f, torch.complex128), self._vec(u, torch.complex128),
                        nprob=self.P, **kw)

    def solve_x0(self, f, u0, u, **kw):
        """sp_solve from the starting vector u0 (None: zero)."""
        import torch
        p0 = None if u0 is None else self._vec(u0, torch.complex128)
        return sp_solve_x0(self.ctx, self._vec(f, torch.complex128), p0,
                           self._vec(u, torch.complex128), **kw)

    def table(self, t: int):
        return sp_get_table(self.ctx, t)

    def set_table(self, t: int, Q, C):
        """Replace type t's Q(S, gamma), C(S, gamma) (row-major |S| x |gamma| float64)."""
        import numpy as np
        Qh = np.ascontiguousarray(Q, dtype=np.float64)
        Ch = np.ascontiguousarray(C, dtype=np.float64)
        rows, cols = sp_get_table(self.ctx, t)[0].shape
        if Qh.shape != (rows, cols) or Ch.shape != (rows, cols):
            raise ValueError(f"type {t} tables are {rows} x {cols}")
        _check(LIB.sp_set_table(self.ctx, t, _dptr(Qh), _dptr(Ch)), "sp_set_table")

    def costs(self):
        return sp_costs(self.ctx)

    def close(self):
        if self.ctx:
            sp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ learned initial guess
def sp_fno_param_count(dims: sp_fno_dims) -> int:
    return int(LIB.sp_fno_param_count(ctypes.byref(dims)))


class Fno:
    """Owns one network context of include/sp_fno.h.  Batches are contiguous torch
    float32 CUDA tensors [batch][channels][n*n]; params a float32 host vector in the
    header's order."""

    def __init__(self, n: int, params, c_in: int = 3, width: int = 32, modes: int = 16,
                 layers: int = 4, hidden: int = 128, c_out: int = 2, batch_max: int = 16,
                 act_fp32: bool = False, stream: int = 0):
        import numpy as np
        self.dims = sp_fno_dims(n, c_in, width, modes, layers, hidden, c_out, batch_max,
                                1 if act_fp32 else 0)
        self.np = sp_fno_param_count(self.dims)
        if self.np == 0:
            raise SpError(SP_ERR_ARG, "sp_fno_param_count")
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.np:
            raise ValueError(f"expected {self.np} parameters, got {p.size}")
        self.N = n * n
        h = ctypes.c_void_p()
        _check(LIB.sp_fno_create(ctypes.byref(self.dims), p.ctypes.data, ctypes.c_void_p(stream),
                                 ctypes.byref(h)), "sp_fno_create")
        self.h = h.value

    def _t(self, x, channels, batch, dtype=None):
        import torch
        dtype = dtype or torch.float32
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == dtype and
                x.is_contiguous() and x.numel() >= batch * channels * self.N):
            raise ValueError(f"expected a contiguous CUDA {dtype} tensor of at least "
                             f"{batch} x {channels} x {self.N} entries")
        return x.data_ptr()

    def forward(self, x, y, batch: int):
        _check(LIB.sp_fno_forward(self.h, batch, self._t(x, self.dims.c_in, batch),
                                  self._t(y, self.dims.c_out, batch)), "sp_fno_forward")

    def gradient(self, x, t, batch: int, y=None, want_grad: bool = True):
        """(loss, gradient as a float32 numpy vector or None)."""
        import numpy as np
        loss = ctypes.c_double()
        g = np.empty(self.np, dtype=np.float32) if want_grad else None
        _check(LIB.sp_fno_gradient(self.h, batch, self._t(x, self.dims.c_in, batch),
                                   self._t(t, self.dims.c_out, batch),
                                   None if y is None else self._t(y, self.dims.c_out, batch),
                                   ctypes.byref(loss), None if g is None else g.ctypes.data),
               "sp_fno_gradient")
        return loss.value, g

    def train_step(self, x, t, batch: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                   eps: float = 1e-8, sync: bool = False):
        """One Adam step; returns the loss before the update when sync, else None."""
        opt = sp_adam(lr, beta1, beta2, eps)
        loss = ctypes.c_double()
        _check(LIB.sp_fno_train_step(self.h, batch, self._t(x, self.dims.c_in, batch),
                                     self._t(t, self.dims.c_out, batch), ctypes.byref(opt),
                                     ctypes.byref(loss) if sync else None), "sp_fno_train_step")
        return loss.value if sync else None

    def params(self):
        import numpy as np
        p = np.empty(self.np, dtype=np.float32)
        _check(LIB.sp_fno_get_params(self.h, p.ctypes.data), "sp_fno_get_params")
        return p

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.np:
            raise ValueError(f"expected {self.np} parameters")
        _check(LIB.sp_fno_set_params(self.h, p.ctypes.data), "sp_fno_set_params")

    def features(self, q, q_scale: float, g, x_slot, scale_slot):
        """One problem's input (3 x N floats at x_slot) and its complex scale c
        (scale_slot: one complex128)."""
        import torch
        _check(LIB.sp_fno_features(self.h, self._t(q, 1, 1, torch.float64), float(q_scale),
                                   self._t(g, 1, 1, torch.complex128), self._t(x_slot, 3, 1),
                                   self._t(scale_slot, 0, 0, torch.complex128)), "sp_fno_features")

    def guess(self, y_slot, scale_slot, u0):
        import torch
        _check(LIB.sp_fno_guess(self.h, self._t(y_slot, 2, 1), self._t(scale_slot, 0, 0, torch.complex128),
                                self._t(u0, 1, 1, torch.complex128)), "sp_fno_guess")

    def target(self, u, scale_slot, t_slot):
        import torch
        _check(LIB.sp_fno_target(self.h, self._t(u, 1, 1, torch.complex128),
                                 self._t(scale_slot, 0, 0, torch.complex128), self._t(t_slot, 2, 1)),
               "sp_fno_target")

    def features_prior(self, q, q_scale: float, g, z, x_slot, scale_slot):
        """One problem's input with the prior z (5 x N floats at x_slot) and its scale."""
        import torch
        _check(LIB.sp_fno_features_prior(self.h, self._t(q, 1, 1, torch.float64), float(q_scale),
                                         self._t(g, 1, 1, torch.complex128),
                                         self._t(z, 1, 1, torch.complex128), self._t(x_slot, 5, 1),
                                         self._t(scale_slot, 0, 0, torch.complex128)),
               "sp_fno_features_prior")

    def guess_prior(self, y_slot, scale_slot, z, u0):
        import torch
        _check(LIB.sp_fno_guess_prior(self.h, self._t(y_slot, 2, 1),
                                      self._t(scale_slot, 0, 0, torch.complex128),
                                      self._t(z, 1, 1, torch.complex128),
                                      self._t(u0, 1, 1, torch.complex128)), "sp_fno_guess_prior")

    def target_prior(self, u, scale_slot, z, t_slot):
        import torch
        _check(LIB.sp_fno_target_prior(self.h, self._t(u, 1, 1, torch.complex128),
                                       self._t(scale_slot, 0, 0, torch.complex128),
                                       self._t(z, 1, 1, torch.complex128), self._t(t_slot, 2, 1)),
               "sp_fno_target_prior")

    def close(self):
        if getattr(self, "h", None):
            LIB.sp_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
