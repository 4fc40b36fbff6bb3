// Numeric multifrontal factorisation of P = Q + C q on the periodic nested-dissection
// tree (Section 2.2-2.3, Fig. nd): per level, leaves to root,
//   1. assemble the original entries P(j, i) = Q(j, i) + C(j, i) q_i whose
//      earlier-eliminated endpoint belongs to the front (Section 2.2: P = Q + C q);
//   2. extend-add the children's Schur complements (one launch per child position,
//      so no two threads of a launch add into the same entry);
//   3. blocked right-looking LU of the front with partial pivoting restricted to
//      the k eliminated rows (the paper does not say how fronts are pivoted; this
//      is the reading used throughout): panel factorisation, row-block triangular
//      solve and a tiled Schur-complement update that also forms
//      S = F22 - L21 U12, the block handed to the parent.
// Every front of a level has the same size, so each step is one batched launch
// over all fronts of the level.  Fronts are column-major m x m.  T = double for
// the FP64 form, float for the FP32 preconditioner form.
#include <cfloat>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kNB = 32;       // panel width
constexpr int kTile = 64;     // Schur update tile (kTile x kTile per CTA)

template <class T>
__global__ void assemble_kernel(T* fronts, int m, int nasm, const int* __restrict__ slot,
                                const int* __restrict__ tidx, const int* __restrict__ cvar,
                                const int* __restrict__ gidx, const double* __restrict__ Qcat,
                                const double* __restrict__ Ccat, const double* __restrict__ q) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nasm) return;
  long f = blockIdx.y;
  int ti = tidx[e];
  double qi = q[gidx[f * m + cvar[e]]];
  fronts[f * (long)m * m + slot[e]] = (T)fma(Ccat[ti], qi, Qcat[ti]);
}

template <class T>
__global__ void extend_add_kernel(T* parent, int m, int nb1, const T* __restrict__ child, int mc,
                                  int kc, const int* __restrict__ map, int delta, int d) {
  const int nbd = mc - kc;
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)nbd * nbd) return;
  int f = blockIdx.y;
  // parent box coordinates -> child box id (child grid has 2*nb1 boxes per axis)
  int ff = f, cid = 0, stride = 1;
  for (int a = 0; a < d; ++a) {
    int bc = ff % nb1;
    ff /= nb1;
    cid += (2 * bc + ((delta >> a) & 1)) * stride;
    stride *= 2 * nb1;
  }
  int i = (int)(e % nbd), j = (int)(e / nbd);
  const T v = child[(long)cid * mc * mc + (long)(kc + i) + (long)(kc + j) * mc];
  parent[(long)f * m * m + map[i] + (long)map[j] * m] += v;
}

template <class T>
__global__ void front_scale_kernel(const T* fronts, long mm, double* scale) {
  const T* A = fronts + blockIdx.x * mm;
  double mx = 0;
  for (long i = threadIdx.x; i < mm; i += blockDim.x) mx = fmax(mx, fabs((double)A[i]));
  __shared__ double red[256];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) scale[blockIdx.x] = red[0];
}

// Unblocked LU of the panel columns [j0, j0+jb) of every front (one CTA per front).
// Pivot rows are searched among the eliminated rows [j, k) only; the swap moves
// whole rows (all m columns), LAPACK style.
template <class T>
__global__ void __launch_bounds__(256) lu_panel_kernel(T* fronts, int m, int k, int j0, int jb,
                                                       int* piv, const double* scale,
                                                       double ptol, int* status) {
  T* A = fronts + (long)blockIdx.x * m * m;
  __shared__ double rv[256];
  __shared__ int ri[256];
  __shared__ T prow[kNB];
  __shared__ int s_p;
  const double thresh = ptol * scale[blockIdx.x];
  for (int j = j0; j < j0 + jb; ++j) {
    // argmax |A[r, j]| over r in [j, k), ties to the smallest row
    double best = -1.0;
    int bi = j;
    for (int r = j + threadIdx.x; r < k; r += blockDim.x) {
      double v = fabs((double)A[r + (long)j * m]);
      if (v > best) {
        best = v;
        bi = r;
      }
    }
    rv[threadIdx.x] = best;
    ri[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double o = rv[threadIdx.x + s];
        int oi = ri[threadIdx.x + s];
        if (o > rv[threadIdx.x] || (o == rv[threadIdx.x] && oi < ri[threadIdx.x])) {
          rv[threadIdx.x] = o;
          ri[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      s_p = ri[0];
      piv[(long)blockIdx.x * k + j] = ri[0];
      if (!(rv[0] > thresh)) atomicOr(status, 1);
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        T t = A[j + (long)c * m];
        A[j + (long)c * m] = A[p + (long)c * m];
        A[p + (long)c * m] = t;
      }
      __syncthreads();
    }
    for (int c = j + 1 + threadIdx.x; c < j0 + jb; c += blockDim.x) prow[c - j0] = A[j + (long)c * m];
    __syncthreads();
    T pv = A[j + (long)j * m];
    if (!(fabs((double)pv) > 0.0)) pv = (T)(thresh > 0 ? thresh : 1e-30);
    const T inv = (T)1 / pv;
    for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) {
      T l = A[r + (long)j * m] * inv;
      A[r + (long)j * m] = l;
      for (int c = j + 1; c < j0 + jb; ++c) A[r + (long)c * m] -= l * prow[c - j0];
    }
    __syncthreads();
  }
}

// U12 row block: A[j0:j0+jb, c] = L_pp^{-1} A[j0:j0+jb, c] for c >= j0 + jb.
template <class T>
__global__ void __launch_bounds__(256) lu_trsm_kernel(T* fronts, int m, int j0, int jb) {
  T* A = fronts + (long)blockIdx.y * m * m;
  __shared__ T Lp[kNB][kNB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e % jb, l = e / jb;
    Lp[i][l] = A[(j0 + i) + (long)(j0 + l) * m];
  }
  __syncthreads();
  int c = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  T x[kNB];
  T* col = A + (long)c * m + j0;
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) x[i] = col[i];
#pragma unroll
  for (int i = 1; i < kNB; ++i) {
    if (i < jb) {
      T acc = x[i];
#pragma unroll
      for (int l = 0; l < kNB; ++l)
        if (l < i) acc -= Lp[i][l] * x[l];
      x[i] = acc;
    }
  }
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) col[i] = x[i];
}

// Schur update of the trailing matrix: A[r, c] -= sum_l A[r, j0+l] A[j0+l, c],
// r, c >= j0 + jb.  kTile x kTile per CTA, 4 x 4 per thread.
template <class T>
__global__ void __launch_bounds__(256) lu_gemm_kernel(T* fronts, int m, int j0, int jb, int tiles) {
  T* A = fronts + (long)blockIdx.y * m * m;
  const int base = j0 + jb;
  const int tr = blockIdx.x % tiles, tc = blockIdx.x / tiles;
  const int r0 = base + tr * kTile, c0 = base + tc * kTile;
  __shared__ T As[kNB][kTile];
  __shared__ T Bs[kNB][kTile + 1];
  for (int e = threadIdx.x; e < jb * kTile; e += blockDim.x) {
    int i = e % kTile, l = e / kTile;
    int r = r0 + i;
    As[l][i] = (r < m) ? A[r + (long)(j0 + l) * m] : (T)0;
  }
  for (int e = threadIdx.x; e < jb * kTile; e += blockDim.x) {
    int l = e % jb, jc = e / jb;
    int c = c0 + jc;
    Bs[l][jc] = (c < m) ? A[(j0 + l) + (long)c * m] : (T)0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int l = 0; l < jb; ++l) {
    T av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[l][tx + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = Bs[l][ty + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    int c = c0 + ty + 16 * b;
    if (c >= m) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int r = r0 + tx + 16 * a;
      if (r < m) A[r + (long)c * m] -= acc[a][b];
    }
  }
}

__global__ void lu_perm_kernel(const int* piv, int* perm, int k, int nf) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  int* p = perm + (long)f * k;
  const int* pv = piv + (long)f * k;
  for (int j = 0; j < k; ++j) p[j] = j;
  for (int j = 0; j < k; ++j) {
    int t = p[j];
    p[j] = p[pv[j]];
    p[pv[j]] = t;
  }
}

template <class T>
cudaError_t factor_level_t(int d, DevLevel& L, const DevLevel* child, const double* Qcat,
                           const double* Ccat, const double* q, double ptol, int* status,
                           cudaStream_t st) {
  const long mm = (long)L.m * L.m;
  T* F = (T*)L.front;
  ProfScope pa(PROF_ASSEMBLE, st);
  cudaError_t e = cudaMemsetAsync(F, 0, sizeof(T) * mm * L.nf, st);
  if (e != cudaSuccess) return e;
  int na = 1;
  if (L.nasm > 0) {
    dim3 g((L.nasm + 255) / 256, L.nf);
    assemble_kernel<T><<<g, 256, 0, st>>>(F, L.m, L.nasm, L.asm_slot, L.asm_tidx, L.asm_cvar,
                                          L.gidx, Qcat, Ccat, q);
    ++na;
  }
  double abytes = (double)sizeof(T) * mm * L.nf;
  if (child) {
    const int nbd = L.mc - L.kc;
    long work = (long)nbd * nbd;
    dim3 g((unsigned)((work + 255) / 256), L.nf);
    for (int dl = 0; dl < (1 << d); ++dl)
      extend_add_kernel<T><<<g, 256, 0, st>>>(F, L.m, L.nb1, (const T*)child->front, L.mc, L.kc,
                                               L.ea_map + (long)dl * nbd, dl, d);
    na += 1 << d;
    abytes += (double)sizeof(T) * work * child->nf;
  }
  front_scale_kernel<T><<<L.nf, 256, 0, st>>>(F, mm, L.scale);
  pa.done(abytes, na + 1, st);
  for (int j0 = 0; j0 < L.k; j0 += kNB) {
    int jb = L.k - j0 < kNB ? L.k - j0 : kNB;
    double pf = 0;
    for (int j = j0; j < j0 + jb; ++j) pf += (double)(L.m - j - 1) * (1.0 + 2.0 * (j0 + jb - j - 1));
    ProfScope pp(PROF_LU_PANEL, st);
    lu_panel_kernel<T><<<L.nf, 256, 0, st>>>(F, L.m, L.k, j0, jb, L.piv, L.scale, ptol, status);
    pp.done(pf * L.nf, 1, st);
    int rem = L.m - j0 - jb;
    if (rem > 0) {
      dim3 gt((rem + 255) / 256, L.nf);
      ProfScope pt(PROF_LU_TRSM, st);
      lu_trsm_kernel<T><<<gt, 256, 0, st>>>(F, L.m, j0, jb);
      pt.done((double)rem * jb * (jb - 1) * L.nf, 1, st);
      int tiles = (rem + kTile - 1) / kTile;
      dim3 gg(tiles * tiles, L.nf);
      ProfScope pg(PROF_LU_GEMM, st);
      lu_gemm_kernel<T><<<gg, 256, 0, st>>>(F, L.m, j0, jb, tiles);
      pg.done(2.0 * rem * rem * jb * L.nf, 1, st);
    }
  }
  lu_perm_kernel<<<(L.nf + 127) / 128, 128, 0, st>>>(L.piv, L.perm, L.k, L.nf);
  return cudaGetLastError();
}

}  // namespace

cudaError_t factor_level(int prec, int d, DevLevel& L, const DevLevel* child, const double* Qcat,
                         const double* Ccat, const double* q, double pivot_tol, int* status,
                         cudaStream_t st) {
  if (prec == SP_PREC_FP32)
    return factor_level_t<float>(d, L, child, Qcat, Ccat, q, pivot_tol, status, st);
  return factor_level_t<double>(d, L, child, Qcat, Ccat, q, pivot_tol, status, st);
}

}  // namespace sp
