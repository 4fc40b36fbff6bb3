"""Write the oracle's stencil tables for the 3D 128^3 workloads (b = 8).

Calls only the FP64 oracle (`oracle/`) and the seeded input generators
(`synthetic_media.py`).  For each 3D 128^3 problem (Helmholtz on a random-field
velocity, omega = 2 pi 16; rescaled Schroedinger with an 8 x 8 x 8 lattice of
wells, l = 8, E = 10) it stores, in `tests/golden/oracle_3d128_<kind>.npz`, per
set type t (Section 2.3: cell, three faces, three edges, vertex):

  T[t]        T_S = G(S, gamma^c) G(beta, gamma^c)^+, |S| x |beta| (rows in S
              order, columns in beta order; Q and C follow from it by
              oracle.tables_from_T);
  rank[t], sigma[t], rho[t]
              the pseudoinverse's rank, the singular values of
              B = G(beta, gamma^c) and rho = ||A - T B||_F / (||B||_2 ||T||_2);
  s           the shift.

The 128^3 oracle solve itself does not fit a host (its factor alone is hundreds of
gigabytes); the tables do: the dense blocks of one type take up to 12 GB.  Run
from the repository root:  python tests/golden/make_golden_3d128.py [helmholtz|schrodinger]
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synthetic_media as sm  # noqa: E402


def problem(kind: str) -> dict:
    if kind == "helmholtz":
        return sm.helmholtz_grf_3d(128, 8, 0)
    return sm.schrodinger_wells_3d(128, 8, 8.0, 10.0, 0)


def shift(w: dict):
    if w["kind"] == "helmholtz":
        return O.helmholtz_shift(w["d"], w["n"], w["omega"], w["c"])
    return O.schrodinger_shift(w["d"], w["n"], w["ell"], w["E"], w["V"])


def main(kind: str) -> None:
    w = problem(kind)
    d, n, b = w["d"], w["n"], w["b"]
    s, _ = shift(w)
    arrays = dict(s=np.float64(s))
    for t in range(1 << d):
        tab = O.stencil_tables(d, n, b, s, types=[t], keep_blocks=True)[0]
        rho = float(np.linalg.norm(tab["resid"]) / (tab["sigma"][0] * np.linalg.norm(tab["T"], 2)))
        arrays[f"T{t}"] = tab["T"]
        arrays[f"rank{t}"] = np.int64(tab["rank"])
        arrays[f"sigma{t}"] = np.asarray(tab["sigma"], dtype=np.float64)
        arrays[f"rho{t}"] = np.float64(rho)
        print(f"[{kind}] type {t}: T {tab['T'].shape}, rank {tab['rank']}, "
              f"kappa {tab['sigma'][0] / tab['sigma'][-1]:.3g}, rho {rho:.3g}", flush=True)
        del tab
    out = os.path.join(ROOT, "tests", "golden", f"oracle_3d128_{kind}.npz")
    np.savez_compressed(out, **arrays)
    print(f"[{kind}] wrote {out}", flush=True)


if __name__ == "__main__":
    for k in sys.argv[1:] or ["helmholtz", "schrodinger"]:
        if k not in ("helmholtz", "schrodinger"):
            raise SystemExit(f"unknown problem {k!r}")
        main(k)
