// Host-side set-up of the sparsifying preconditioner: Green's kernel, stencil
// tables (Section 2.3) and the periodic nested-dissection structure (Fig. nd).
// Plain C++; no CUDA types.
#pragma once
#include <cstdint>
#include <vector>

namespace sp {

// One stencil type (Section 2.3): cell, face, edge or vertex of a given orientation.
// Type t = sum over axes a with p_a = 0 (mod b) of 2^a.  Offsets are relative to the
// leaf-box origin, d ints per point, points ordered with axis 0 fastest.
struct StencilTable {
  int t = 0, nS = 0, nG = 0, nB = 0, rank = 0;
  std::vector<int> S, G, Bt;        // set, gamma(set), beta(set) = gamma minus set
  std::vector<double> Q, C;          // nS x nG, row-major
  std::vector<double> sigma;         // singular values of G(beta, gamma^c), descending
};

// One level of the nested-dissection tree.  Level 0 holds the leaf boxes of side b,
// level l boxes of side b*2^l, level L the root (the whole torus).  Every front of a
// level has the same size: k eliminated unknowns first, then m - k boundary unknowns.
struct Level {
  int lev = 0, B = 0, nb1 = 0, nf = 0, k = 0, m = 0;
  std::vector<int> off;       // m x d local offsets of the front unknowns (box 0)
  std::vector<int> gidx;      // nf x m global flat indices
  // assembly of the original entries of P whose earlier-eliminated endpoint is
  // eliminated in this front (same list for every front of the level)
  std::vector<int> asm_row;   // front row r of the entry (its column is asm_cvar)
  std::vector<int> asm_tidx;  // index into the concatenated column-major Q/C tables
  std::vector<int> asm_cvar;  // front position of the column point (for q)
  // extend-add: child position delta (0..2^d-1) -> map of the child's m_c - k_c
  // boundary unknowns to positions of this front
  int mc = 0, kc = 0;
  std::vector<int> ea_map;    // 2^d x (mc - kc)
};

struct Symbolic {
  int d = 0, n = 0, b = 0, L = 0;
  std::vector<Level> lv;
};

// g = inverse DFT of 1/(4 pi^2 |k|^2 - s) with the 1/N of the unitary pair (Eq. G):
// G(i, j) = g[(i - j) mod n].  Flat, axis 0 fastest.  The host FFT runs on up to
// `threads` host threads (0 = all); the result does not depend on the count.
std::vector<double> green_kernel(int d, int n, double s, int threads = 0);
// the same for G^2: inverse DFT of 1/(4 pi^2 |k|^2 - s)^2 with the 1/N
std::vector<double> green_kernel_sq(int d, int n, double s, int threads = 0);

// min_k |kappa - |k|^2| / max(1, kappa), kappa = s / (4 pi^2).
double resonance_gap(int d, int n, double s);

// Tables of one type (Section 2.3).  g: the Green kernel.  g2 (the kernel of G^2)
// selects the Gram route for T_S instead of the TSQR + SVD route.  kind 0: the
// paper's set stencils Q(S, gamma(S)); kind 1: per-point stencils Q(j, gamma({j}))
// (the 3^d neighbourhood of each point j), stored in the same |S| x |gamma(S)|
// layout with each row zero outside gamma({j}).
int stencil_table(int d, int n, int b, int t, const std::vector<double>& g, int threads,
                  StencilTable* out, const std::vector<double>* g2 = nullptr, int kind = 0);

// All 2^d tables of one shift s (types t = 0 .. 2^d - 1 into out[0 .. 2^d - 1]):
// the Green kernel (and, for route 1, the kernel of G^2) and then stencil_table for
// every type, on up to `threads` host threads (0 = all); the same tables, bit for
// bit, as stencil_table called type by type.
int stencil_tables(int d, int n, int b, double s, int route, int kind, int threads,
                   StencilTable* out);

// The host set-up of a context of P problems (shifts[0 .. P-1]): tabs gets the
// 2^d tables of every problem, problem-major (problem p's type t at p 2^d + t), as
// stencil_tables makes them; sym the nested-dissection structure, built from the
// sets' geometry while the tables are computed.  0 on success.
int setup_host(int d, int n, int b, int P, const double* shifts, int route, int kind,
               int threads, std::vector<StencilTable>* tabs, Symbolic* sym);

// Nested-dissection structure.
int build_symbolic(int d, int n, int b, const std::vector<StencilTable>& tabs, Symbolic* out);

// Level sizes only (cheap).
int front_sizes(int d, int n, int b, std::vector<int>* nf, std::vector<int>* k,
                std::vector<int>* m);

// 0 if d is 2 or 3, b >= 2 divides n, n / b = 2^L with L >= 1 (stored in *L) and
// n^d < 2^31 (grid indices are ints); 1 otherwise.
int check_grid(int d, int n, int b, int* L);

}  // namespace sp
