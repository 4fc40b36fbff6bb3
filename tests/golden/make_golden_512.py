"""Write the oracle's expected values for the 2D 512^2 workloads (b = 16).

Calls only the FP64 oracle (`oracle/`) and the seeded input generators
(`synthetic_media.py`); nothing here touches the CUDA library.  For each of
the two problems of the 512^2 pair (Helmholtz on a Gaussian-random-field
velocity, Schroedinger with lattice wells) it stores, in
`tests/golden/oracle_2d512_<kind>.npz`:

  s, rank[t], Q[t], C[t]  the stencil tables of Section 2.3 (T_S by the
                          pseudoinverse, Q(S, gamma) = [I, -T_S],
                          C(S, gamma) = Q(S, gamma) G(gamma, gamma)) per set type t;
  sigma[t], rho[t]        the singular values of B = G(beta, gamma^c) and the relative
                          least-squares residual rho = ||A - T B||_F / (||B||_2 ||T||_2)
                          with A = G(S, gamma^c): together they bound how closely two
                          backward-stable pseudoinverse solutions can agree
                          (kappa eps + kappa^2 eps rho, kappa = sigma_max / sigma_min);
  r_seed, z               z = P^{-1} Q r (Section 2.2) for the seeded complex
                          normal r, P = Q + C q factored exactly (SuperLU);
  u, iters, hist, true_relres
                          right-preconditioned GMRES on (I + G q) u = G f to
                          relative residual 1e-8 (u stored in complex64: its
                          rounding, 6e-8 relative, is far below the 1e-6
                          solution tolerance it is used with);
  u_ref, iters_ref, true_relres_ref
                          the same GMRES to relative residual 1e-12: the discrete
                          solution to ~1e-10 (complex64), against which a solution's
                          forward error is measured;
  phase_seconds           wall time of each oracle phase on the host that ran it.

Run from the repository root:  python tests/golden/make_golden_512.py helmholtz
(one problem per process; the two may run side by side).  Each problem takes
5 to 8 minutes on 8 x86 cores: the SuperLU factorisation of P (about 4 minutes)
and one SuperLU solve pair (3 s) per GMRES iteration.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synthetic_media as sm  # noqa: E402

R_SEED = 41
TOL = 1e-8


def problem(kind: str) -> dict:
    return sm.helmholtz_grf_512() if kind == "helmholtz" else sm.schrodinger_wells_512()


def shift_and_rhs(w: dict):
    if w["kind"] == "helmholtz":
        s, q = O.helmholtz_shift(w["d"], w["n"], w["omega"], w["c"])
        f = w["f"]
    else:
        s, q = O.schrodinger_shift(w["d"], w["n"], w["ell"], w["E"], w["V"])
        f = w["f"] * w["ell"] ** 2
    return s, q, f


def main(kind: str) -> None:
    w = problem(kind)
    d, n, b = w["d"], w["n"], w["b"]
    s, q, f = shift_and_rhs(w)
    ph = {}
    t0 = time.time()
    tabs = O.stencil_tables(d, n, b, s, keep_blocks=True)
    ph["tables"] = time.time() - t0
    for tab in tabs:
        tab["rho"] = float(np.linalg.norm(tab.pop("resid")) /
                           (np.linalg.norm(tab.pop("B"), 2) * np.linalg.norm(tab["T"], 2)))
        tab.pop("A")
    t0 = time.time()
    M = O.SparsifyingPreconditioner(d, n, b, s, q, tables=tabs, factor=None)
    ph["assemble"] = time.time() - t0
    t0 = time.time()
    import scipy.sparse.linalg as spla
    M._lu = spla.splu(M.P.tocsc())
    M.kind = "splu"
    ph["factor"] = time.time() - t0
    ph["factor_entries"] = int(M._lu.L.nnz + M._lu.U.nnz)
    r = sm.random_complex_vector(n ** d, R_SEED)
    t0 = time.time()
    z = M.apply(r)
    ph["apply"] = time.time() - t0
    ph["z_backward_residual"] = M.apply_residual(r, z)
    print(f"[{kind}] tables {ph['tables']:.1f}s assemble {ph['assemble']:.1f}s factor "
          f"{ph['factor']:.1f}s apply {ph['apply']:.1f}s  ||Pz-Qr||/||Qr|| "
          f"{ph['z_backward_residual']:.2e}", flush=True)
    g = O.apply_green(d, n, s, f)
    t0 = time.time()
    ref = O.gmres_right(lambda x: O.apply_operator(d, n, s, q, x), M.apply, g, tol=TOL)
    ph["gmres"] = time.time() - t0
    print(f"[{kind}] GMRES {ref['iters']} iterations, true residual "
          f"{ref['true_relres']:.2e}, {ph['gmres']:.0f}s", flush=True)
    t0 = time.time()
    ref12 = O.gmres_right(lambda x: O.apply_operator(d, n, s, q, x), M.apply, g, tol=1e-12)
    ph["gmres_ref"] = time.time() - t0
    print(f"[{kind}] reference GMRES {ref12['iters']} iterations, true residual "
          f"{ref12['true_relres']:.2e}; ||u - u_ref|| / ||u_ref|| = "
          f"{np.linalg.norm(ref['u'] - ref12['u']) / np.linalg.norm(ref12['u']):.3e}", flush=True)
    out = os.path.join(ROOT, "tests", "golden", f"oracle_2d512_{kind}.npz")
    arrays = dict(s=np.float64(s), r_seed=np.int64(R_SEED), z=z.astype(np.complex128),
                  u=ref["u"].astype(np.complex64), iters=np.int64(ref["iters"]),
                  hist=np.asarray(ref["hist"], dtype=np.float64),
                  true_relres=np.float64(ref["true_relres"]),
                  u_ref=ref12["u"].astype(np.complex64), iters_ref=np.int64(ref12["iters"]),
                  true_relres_ref=np.float64(ref12["true_relres"]),
                  phase_names=np.array(sorted(ph)), phase_seconds=np.array([ph[k] for k in sorted(ph)],
                                                                           dtype=np.float64))
    for t, tab in enumerate(tabs):
        arrays[f"Q{t}"] = tab["Q"]
        arrays[f"C{t}"] = tab["C"]
        arrays[f"rank{t}"] = np.int64(tab["rank"])
        arrays[f"sigma{t}"] = np.asarray(tab["sigma"], dtype=np.float64)
        arrays[f"rho{t}"] = np.float64(tab["rho"])
    np.savez_compressed(out, **arrays)
    print(f"[{kind}] wrote {out}", flush=True)


if __name__ == "__main__":
    kinds = sys.argv[1:] or ["helmholtz", "schrodinger"]
    for k in kinds:
        if k not in ("helmholtz", "schrodinger"):
            raise SystemExit(f"unknown problem {k!r}")
        main(k)
