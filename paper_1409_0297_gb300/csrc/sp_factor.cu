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

// LU of the panel columns [j0, j0+jb) of every front (one CTA per front).  The
// panel rows [j0, m) are staged in shared memory (column-major, leading
// dimension rows = m - j0); pivot rows are searched among the eliminated rows
// [j, k) only.  Row swaps inside the panel happen in shared memory; the same
// swaps are applied here to the columns left of the panel and by the row-block
// solve to the columns right of it (LAPACK-style full-row interchanges).
template <class T>
__global__ void __launch_bounds__(256) lu_panel_kernel(T* fronts, int m, int k, int j0, int jb,
                                                       int* piv, const double* scale,
                                                       double ptol, int* status) {
  extern __shared__ unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);
  __shared__ double wv[8];
  __shared__ int wi[8];
  __shared__ int spiv[kNB];
  T* A = fronts + (long)blockIdx.x * m * m;
  const int rows = m - j0;
  const int kl = k - j0;  // pivot candidates are local rows < kl
  const double thresh = ptol * scale[blockIdx.x];
  for (long e = threadIdx.x; e < (long)rows * jb; e += blockDim.x) {
    int r = (int)(e % rows), c = (int)(e / rows);
    P[e] = A[(j0 + r) + (long)(j0 + c) * m];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jj = 0; jj < jb; ++jj) {
    T* pc = P + (long)jj * rows;
    double best = -1.0;
    int bi = jj;
    for (int r = jj + threadIdx.x; r < kl; r += blockDim.x) {
      double v = fabs((double)pc[r]);
      if (v > best) {
        best = v;
        bi = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      wv[warp] = best;
      wi[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b0 = wv[0];
      int i0 = wi[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (wv[w] > b0 || (wv[w] == b0 && wi[w] < i0)) {
          b0 = wv[w];
          i0 = wi[w];
        }
      spiv[jj] = i0;
      piv[(long)blockIdx.x * k + j0 + jj] = j0 + i0;
      if (!(b0 > thresh)) atomicOr(status, 1);
    }
    __syncthreads();
    const int p = spiv[jj];
    if (p != jj)
      for (int c = threadIdx.x; c < jb; c += blockDim.x) {
        T t = P[jj + (long)c * rows];
        P[jj + (long)c * rows] = P[p + (long)c * rows];
        P[p + (long)c * rows] = t;
      }
    __syncthreads();
    T pv = pc[jj];
    if (!(fabs((double)pv) > 0.0)) pv = (T)(thresh > 0 ? thresh : 1e-30);
    const T inv = (T)1 / pv;
    for (int r = jj + 1 + threadIdx.x; r < rows; r += blockDim.x) {
      T l = pc[r] * inv;
      pc[r] = l;
      for (int c = jj + 1; c < jb; ++c) P[r + (long)c * rows] -= l * P[jj + (long)c * rows];
    }
    __syncthreads();
  }
  for (long e = threadIdx.x; e < (long)rows * jb; e += blockDim.x) {
    int r = (int)(e % rows), c = (int)(e / rows);
    A[(j0 + r) + (long)(j0 + c) * m] = P[e];
  }
  // interchanges on the columns left of the panel
  for (int c = threadIdx.x; c < j0; c += blockDim.x) {
    T* col = A + (long)c * m;
    for (int jj = 0; jj < jb; ++jj) {
      int p = j0 + spiv[jj];
      if (p != j0 + jj) {
        T t = col[j0 + jj];
        col[j0 + jj] = col[p];
        col[p] = t;
      }
    }
  }
}

// Row-block solve right of the panel: interchanges, then
// A[j0:j0+jb, c] = L_pp^{-1} A[j0:j0+jb, c] for c >= j0 + jb (one thread per column).
template <class T>
__global__ void __launch_bounds__(256) lu_trsm_kernel(T* fronts, int m, int k, int j0, int jb,
                                                      const int* piv) {
  T* A = fronts + (long)blockIdx.y * m * m;
  __shared__ T Lp[kNB][kNB + 1];
  __shared__ int sp_[kNB];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e % jb, l = e / jb;
    Lp[i][l] = A[(j0 + i) + (long)(j0 + l) * m];
  }
  for (int e = threadIdx.x; e < jb; e += blockDim.x) sp_[e] = piv[(long)blockIdx.y * k + j0 + e];
  __syncthreads();
  int c = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  T* colg = A + (long)c * m;
  for (int jj = 0; jj < jb; ++jj) {
    int p = sp_[jj];
    if (p != j0 + jj) {
      T t = colg[j0 + jj];
      colg[j0 + jj] = colg[p];
      colg[p] = t;
    }
  }
  T x[kNB];
  T* col = colg + j0;
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

// Batched C[M x N] -= A[M x K] B[K x N], K <= kNB, column-major with leading
// dimensions lda/ldb/ldc and per-batch strides (blockIdx.y = batch).  kTile x
// kTile per CTA, 4 x 4 per thread.  Used for the Schur update of the LU and for
// the triangular inverses.
template <class T>
__global__ void __launch_bounds__(256) gemm_sub_kernel(int M, int N, int K, const T* A, int lda,
                                                       long sA, const T* B, int ldb, long sB,
                                                       T* C, int ldc, long sC, int tilesM) {
  A += blockIdx.y * sA;
  B += blockIdx.y * sB;
  C += blockIdx.y * sC;
  const int tr = blockIdx.x % tilesM, tc = blockIdx.x / tilesM;
  const int r0 = tr * kTile, c0 = tc * kTile;
  __shared__ T As[kNB][kTile];
  __shared__ T Bs[kNB][kTile + 1];
  for (int e = threadIdx.x; e < K * kTile; e += blockDim.x) {
    int i = e % kTile, l = e / kTile;
    int r = r0 + i;
    As[l][i] = (r < M) ? A[r + (long)l * lda] : (T)0;
  }
  for (int e = threadIdx.x; e < K * kTile; e += blockDim.x) {
    int l = e % K, jc = e / K;
    int c = c0 + jc;
    Bs[l][jc] = (c < N) ? B[l + (long)c * ldb] : (T)0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int l = 0; l < K; ++l) {
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
    if (c >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int r = r0 + tx + 16 * a;
      if (r < M) C[r + (long)c * ldc] -= acc[a][b];
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

// ---- explicit triangular inverses for levels with few fronts -------------------
// X (k x k per front, leading dimension k) is set to the identity.
template <class T>
__global__ void set_identity_kernel(T* X, int k, long total) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  long w = e % ((long)k * k);
  int r = (int)(w % k), c = (int)(w / k);
  X[e] = (r == c) ? (T)1 : (T)0;
}

// Diagonal-block step of X = L11^{-1} (unit lower): rows [j0, j0+jb) of X,
// columns [0, ncol), replaced by L_JJ^{-1} times themselves (one thread per column).
template <class T>
__global__ void trinv_lower_diag_kernel(const T* fronts, int m, T* X, int k, int j0, int jb, int ncol) {
  const T* A = fronts + (long)blockIdx.y * m * m;
  T* Xf = X + (long)blockIdx.y * k * k;
  __shared__ T Lp[kNB][kNB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e % jb, l = e / jb;
    Lp[i][l] = A[(j0 + i) + (long)(j0 + l) * m];
  }
  __syncthreads();
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  T* col = Xf + (long)c * k + j0;
  T x[kNB];
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) x[i] = col[i];
#pragma unroll
  for (int i = 1; i < kNB; ++i)
    if (i < jb) {
      T acc = x[i];
#pragma unroll
      for (int l = 0; l < kNB; ++l)
        if (l < i) acc -= Lp[i][l] * x[l];
      x[i] = acc;
    }
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) col[i] = x[i];
}

// Diagonal-block step of X = U11^{-1} (upper, non-unit): rows [j0, j0+jb) of X,
// columns [c_lo, k), replaced by U_JJ^{-1} times themselves.
template <class T>
__global__ void trinv_upper_diag_kernel(const T* fronts, int m, T* X, int k, int j0, int jb) {
  const T* A = fronts + (long)blockIdx.y * m * m;
  T* Xf = X + (long)blockIdx.y * k * k;
  __shared__ T Up[kNB][kNB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e % jb, l = e / jb;
    Up[i][l] = A[(j0 + i) + (long)(j0 + l) * m];
  }
  __syncthreads();
  int c = j0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  T* col = Xf + (long)c * k + j0;
  T x[kNB];
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) x[i] = col[i];
#pragma unroll
  for (int i = kNB - 1; i >= 0; --i)
    if (i < jb) {
      T acc = x[i];
#pragma unroll
      for (int l = 0; l < kNB; ++l)
        if (l > i && l < jb) acc -= Up[i][l] * x[l];
      x[i] = acc / Up[i][i];
    }
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) col[i] = x[i];
}

// F11 <- strict lower part of Linv, upper part (with the diagonal) of Uinv.
template <class T>
__global__ void trinv_store_kernel(T* fronts, int m, const T* Xl, const T* Xu, int k) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)k * k) return;
  int r = (int)(e % k), c = (int)(e / k);
  long f = blockIdx.y;
  T v = (r > c) ? Xl[f * k * k + e] : Xu[f * k * k + e];
  fronts[f * (long)m * m + r + (long)c * m] = v;
}

template <class T>
void gemm_sub(int M, int N, int K, const T* A, int lda, long sA, const T* B, int ldb, long sB,
              T* C, int ldc, long sC, int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  int tilesM = (M + kTile - 1) / kTile, tilesN = (N + kTile - 1) / kTile;
  dim3 g(tilesM * tilesN, batch);
  gemm_sub_kernel<T><<<g, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, tilesM);
}

// Replace L11, U11 of every front of the level by L11^{-1} (strict lower part;
// the unit diagonal is implied) and U11^{-1} (upper part).  The sweeps of such a
// level are then plain matrix-vector products spread over many CTAs.
template <class T>
void invert_triangles(DevLevel& L, T* scratch, cudaStream_t st) {
  const int k = L.k, m = L.m;
  const long kk = (long)k * k, mm = (long)m * m;
  T* F = (T*)L.front;
  T* Xl = scratch;
  T* Xu = scratch + kk * L.nf;
  long tot = kk * L.nf;
  set_identity_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Xl, k, tot);
  set_identity_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Xu, k, tot);
  // L X = I, block rows top to bottom
  for (int j0 = 0; j0 < k; j0 += kNB) {
    int jb = k - j0 < kNB ? k - j0 : kNB;
    int ncol = j0 + jb;
    dim3 g((ncol + 255) / 256, L.nf);
    trinv_lower_diag_kernel<T><<<g, 256, 0, st>>>(F, m, Xl, k, j0, jb, ncol);
    int rows = k - j0 - jb;
    gemm_sub<T>(rows, ncol, jb, F + (j0 + jb) + (long)j0 * m, m, mm, Xl + j0, k, kk,
                Xl + (j0 + jb), k, kk, L.nf, st);
  }
  // U X = I, block rows bottom to top
  int nblk = (k + kNB - 1) / kNB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    int j0 = bi * kNB;
    int jb = k - j0 < kNB ? k - j0 : kNB;
    dim3 g((k - j0 + 255) / 256, L.nf);
    trinv_upper_diag_kernel<T><<<g, 256, 0, st>>>(F, m, Xu, k, j0, jb);
    gemm_sub<T>(j0, k - j0, jb, F + (long)j0 * m, m, mm, Xu + j0 + (long)j0 * k, k, kk,
                Xu + (long)j0 * k, k, kk, L.nf, st);
  }
  dim3 g((unsigned)((kk + 255) / 256), L.nf);
  trinv_store_kernel<T><<<g, 256, 0, st>>>(F, m, Xl, Xu, k);
}

template <class T>
int panel_width(int m) {
  // widest of 32 / 16 / 8 whose staged panel fits in 160 KB of shared memory
  for (int jb = kNB; jb >= 8; jb >>= 1)
    if ((size_t)m * jb * sizeof(T) <= 160 * 1024) return jb;
  return 0;
}

template <class T>
cudaError_t factor_level_t(int d, DevLevel& L, const DevLevel* child, const double* Qcat,
                           const double* Ccat, const double* q, double ptol, int* status,
                           void* scratch, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
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
  const int NB = panel_width<T>(L.m);
  if (NB == 0) return cudaErrorInvalidValue;
  for (int j0 = 0; j0 < L.k; j0 += NB) {
    int jb = L.k - j0 < NB ? L.k - j0 : NB;
    double pf = 0;
    for (int j = j0; j < j0 + jb; ++j) pf += (double)(L.m - j - 1) * (1.0 + 2.0 * (j0 + jb - j - 1));
    ProfScope pp(PROF_LU_PANEL, st);
    size_t sm = sizeof(T) * (size_t)(L.m - j0) * jb;
    lu_panel_kernel<T><<<L.nf, 256, sm, st>>>(F, L.m, L.k, j0, jb, L.piv, L.scale, ptol, status);
    pp.done(pf * L.nf, 1, st);
    int rem = L.m - j0 - jb;
    if (rem > 0) {
      dim3 gt((rem + 255) / 256, L.nf);
      ProfScope pt(PROF_LU_TRSM, st);
      lu_trsm_kernel<T><<<gt, 256, 0, st>>>(F, L.m, L.k, j0, jb, L.piv);
      pt.done((double)rem * jb * (jb - 1) * L.nf, 1, st);
      ProfScope pg(PROF_LU_GEMM, st);
      const int base = j0 + jb;
      gemm_sub<T>(rem, rem, jb, F + base + (long)j0 * L.m, L.m, mm, F + j0 + (long)base * L.m, L.m,
                  mm, F + base + (long)base * L.m, L.m, mm, L.nf, st);
      pg.done(2.0 * rem * rem * jb * L.nf, 1, st);
    }
  }
  lu_perm_kernel<<<(L.nf + 127) / 128, 128, 0, st>>>(L.piv, L.perm, L.k, L.nf);
  if (L.inv) {
    ProfScope pi(PROF_LU_TRINV, st);
    invert_triangles<T>(L, (T*)scratch, st);
    pi.done((2.0 / 3.0) * (double)L.k * L.k * L.k * L.nf, 1, st);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t factor_level(int prec, int d, DevLevel& L, const DevLevel* child, const double* Qcat,
                         const double* Ccat, const double* q, double pivot_tol, int* status,
                         void* scratch, cudaStream_t st) {
  if (prec == SP_PREC_FP32)
    return factor_level_t<float>(d, L, child, Qcat, Ccat, q, pivot_tol, status, scratch, st);
  return factor_level_t<double>(d, L, child, Qcat, Ccat, q, pivot_tol, status, scratch, st);
}

int factor_panel_width(int prec, int m) {
  return prec == SP_PREC_FP32 ? panel_width<float>(m) : panel_width<double>(m);
}

}  // namespace sp
