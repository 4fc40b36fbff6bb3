"""CPU tests of the nested-dissection symbolic structure built by the library (host logic).

Checked against the paper's geometry (Section 2.3, Fig. nd) and the oracle's sparse P:
  * every grid point is eliminated exactly once, and a front's boundary unknowns
    are eliminated at a later level;
  * the extend-add maps send each child's boundary unknown to the same grid point
    in the parent front;
  * the assembly lists place every structural entry of P (oracle pattern) exactly
    once, into the front of its earlier-eliminated endpoint.
"""
import itertools

import numpy as np
import pytest

import oracle as O


def _B():
    from paper_1409_0297_gb300 import build as bld
    import os
    if not os.path.exists(bld.LIB):
        bld.build()
    from paper_1409_0297_gb300 import binding as B
    return B


CASES = [(2, 16, 4), (2, 32, 4), (2, 16, 2), (2, 24, 3), (3, 8, 2), (3, 16, 4),
         # odd and even leaf sizes other than powers of two, deeper trees
         (2, 20, 5), (2, 56, 7), (2, 48, 6), (2, 40, 5), (3, 10, 5), (3, 12, 3)]


@pytest.mark.parametrize("d,n,b", CASES)
def test_symbolic_consistency(d, n, b):
    B = _B()
    N = n ** d
    L = int(np.log2(n // b))
    lv = [B.sp_level_info(d, n, b, l) for l in range(L + 1)]
    elim_level = np.full(N, -1)
    for l, V in enumerate(lv):
        el = V["gidx"][:, : V["k"]].ravel()
        assert np.all(elim_level[el] == -1)
        elim_level[el] = l
    assert np.all(elim_level >= 0)
    for l, V in enumerate(lv):
        bd = V["gidx"][:, V["k"]:].ravel()
        assert np.all(elim_level[bd] > l)
        # front unknowns of one front are distinct grid points
        for f in range(V["nf"]):
            assert len(set(V["gidx"][f].tolist())) == V["m"]
    # extend-add maps: child boundary point -> same point in the parent front
    for l in range(1, L + 1):
        P, C = lv[l], lv[l - 1]
        nb1 = round(P["nf"] ** (1.0 / d))
        for f in range(P["nf"]):
            bc = [(f // nb1 ** a) % nb1 for a in range(d)]
            for dl in range(1 << d):
                cid = sum((2 * bc[a] + ((dl >> a) & 1)) * (2 * nb1) ** a for a in range(d))
                mp = P["ea_map"][dl]
                assert len(set(mp.tolist())) == len(mp)
                assert np.array_equal(P["gidx"][f][mp], C["gidx"][cid][C["k"]:])


@pytest.mark.parametrize("d,n,b", CASES)
def test_assembly_covers_pattern_of_P_once(d, n, b):
    B = _B()
    s = 4 * np.pi ** 2 * 1.37
    tabs = O.stencil_tables(d, n, b, s)
    Qs, _, _ = O.assemble_sparse(d, n, b, tabs, None)
    Qs = Qs.tocoo()
    pattern = set(zip(Qs.row.tolist(), Qs.col.tolist()))
    L = int(np.log2(n // b))
    seen = set()
    total = 0
    for l in range(L + 1):
        V = B.sp_level_info(d, n, b, l)
        m = V["m"]
        r, c = V["asm_row"].astype(np.int64), V["asm_cvar"].astype(np.int64)
        slots = r + c * m
        assert len(set(slots.tolist())) == len(slots)
        assert np.all((r >= 0) & (r < m) & (c >= 0) & (c < m))
        # the earlier-eliminated endpoint is eliminated in this front
        assert np.all((r < V["k"]) | (c < V["k"]))
        for f in range(V["nf"]):
            g = V["gidx"][f]
            for rr, cc in zip(g[r].tolist(), g[c].tolist()):
                seen.add((rr, cc))
            total += len(slots)
    assert total == len(pattern)
    assert seen == pattern
