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
#include <cooperative_groups.h>

#include <functional>
#include <vector>

#include <algorithm>
#include <cfloat>

#include <cuda_fp16.h>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kNB = 32;       // panel width
constexpr int kTile = 64;     // Schur update tile (kTile x kTile per CTA)
constexpr int kTcMinFront = 1024;         // smallest front blocked for the tensor cores
constexpr int kGridPanelCTAs = 152;       // CTAs of a grid-panel launch (one per SM)
constexpr size_t kGridPanelSmem = 200 * 1024;  // staged rows of one grid-panel CTA

template <class T>
__global__ void assemble_kernel(T* fronts, int m, int nasm, const int* __restrict__ row,
                                const int* __restrict__ tidx, const int* __restrict__ cvar,
                                const int* __restrict__ gidx, const double* __restrict__ Qcat,
                                const double* __restrict__ Ccat, const double* __restrict__ q,
                                int nfp, long tstride) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nasm) return;
  long f = blockIdx.y;
  // fronts of a problem group: problem f / nfp reads its own tables (tstride apart)
  const long ti = tidx[e] + (f / nfp) * tstride;
  const int c = cvar[e];
  double qi = q[gidx[f * m + c]];
  fronts[f * (long)m * m + row[e] + (long)c * m] = (T)fma(Ccat[ti], qi, Qcat[ti]);
}

// One launch per child position: the child's Schur block (rows and columns kc..mc-1 of
// its front) is added into the parent front through the map.  Each thread adds kEaU
// entries a block width apart in column-major order: it reads every child value, map
// entry and parent value first and writes afterwards, so kEaU independent read chains
// are in flight (the map is injective within one child position, so no two entries of a
// launch meet in the parent).
constexpr int kEaU = 4;

template <class T>
__global__ void extend_add_kernel(T* parent, int m, int nb1, const T* __restrict__ child, int mc,
                                  int kc, const int* __restrict__ map, int delta, int d) {
  const int nbd = mc - kc;
  const long nn = (long)nbd * nbd;
  const long e0 = (long)blockIdx.x * (kEaU * blockDim.x) + threadIdx.x;
  if (e0 >= nn) return;
  int f = blockIdx.y;
  // parent box coordinates -> child box id (child grid has 2*nb1 boxes per axis)
  int ff = f, cid = 0, stride = 1;
  for (int a = 0; a < d; ++a) {
    int bc = ff % nb1;
    ff /= nb1;
    cid += (2 * bc + ((delta >> a) & 1)) * stride;
    stride *= 2 * nb1;
  }
  cid += ff * stride;  // problem ff of a group: its children follow the earlier problems'
  const T* cf = child + (long)cid * mc * mc + kc + (long)kc * mc;
  T* pf = parent + (long)f * m * m;
  int i = (int)(e0 % nbd), j = (int)(e0 / nbd);
  T v[kEaU];
  long at[kEaU];
#pragma unroll
  for (int u = 0; u < kEaU; ++u) {
    at[u] = -1;
    if (e0 + (long)u * blockDim.x < nn) {
      v[u] = cf[i + (long)j * mc];
      at[u] = map[i] + (long)map[j] * m;
    }
    i += blockDim.x;  // next entry: blockDim.x further in column-major order
    j += i / nbd;
    i %= nbd;
  }
  T p[kEaU];
#pragma unroll
  for (int u = 0; u < kEaU; ++u)
    if (at[u] >= 0) p[u] = pf[at[u]];
#pragma unroll
  for (int u = 0; u < kEaU; ++u)
    if (at[u] >= 0) pf[at[u]] = p[u] + v[u];
}

// FP16 copy of the factor for the chained sweeps (sp_opts.factor_storage = 1), with a
// power-of-two scale per front column: column c of front f is stored as entry /
// 2^(e - 15), with max |entry| = mant 2^e (mant in [0.5, 1)) over the rows the sweeps
// read (all rows for c < k; rows < k, the U12 block, for c >= k), so every stored
// magnitude is below 2^15 (FP16's largest finite value is 65504), the scaling is
// exact, and a column's entries keep FP16's 11 significant bits down to 2^-29 of its
// largest.  One warp per column; columns ld16 = m rounded up to even apart (the pad
// row zero).
__global__ void f16_copy_kernel(const float* fronts, int m, int k, __half* out, float* fsc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= m) return;
  const long f = blockIdx.y, mm = (long)m * m;
  const int ld16 = (m + 1) & ~1;  // even column stride: row pairs load as half2
  const float* col = fronts + f * mm + (long)c * m;
  __half* hc = out + f * (long)m * ld16 + (long)c * ld16;
  const int rows = c < k ? m : k;
  if (lane == 0 && ld16 > m) hc[m] = __float2half_rn(0.f);
  // both passes over the column keep eight loads per lane in flight
  constexpr int kU = 8;
  float mxu[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) mxu[u] = 0.f;
  int r = lane;
  for (; r + 32 * (kU - 1) < rows; r += 32 * kU) {
    float v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) v[u] = col[r + 32 * u];
#pragma unroll
    for (int u = 0; u < kU; ++u) mxu[u] = fmaxf(mxu[u], fabsf(v[u]));
  }
  for (; r < rows; r += 32) mxu[0] = fmaxf(mxu[0], fabsf(col[r]));
  float mx = mxu[0];
#pragma unroll
  for (int u = 1; u < kU; ++u) mx = fmaxf(mx, mxu[u]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;
  if (mx > 0.f) frexpf(mx, &e);
  const float inv = ldexpf(1.0f, 15 - e);
  if (lane == 0) fsc[f * m + c] = ldexpf(1.0f, e - 15);
  r = lane;
  for (; r + 32 * (kU - 1) < rows; r += 32 * kU) {
    float v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) v[u] = col[r + 32 * u];
#pragma unroll
    for (int u = 0; u < kU; ++u) hc[r + 32 * u] = __float2half_rn(v[u] * inv);
  }
  for (; r < rows; r += 32) hc[r] = __float2half_rn(col[r] * inv);
}

// max |entry| of every front: CTAs over (chunk, front), atomicMax on the bit
// pattern (non-negative doubles order like their unsigned integer bits); scale
// must be zeroed first.
template <class T>
__global__ void front_scale_kernel(const T* fronts, long mm, double* scale) {
  const T* A = fronts + blockIdx.y * mm;
  // eight independent loads in flight per thread (a loop-carried max with one load per
  // trip is bound by memory latency, not bandwidth)
  constexpr int kU = 8;
  const long stride = (long)gridDim.x * blockDim.x;
  double mxu[kU];
#pragma unroll
  for (int u = 0; u < kU; ++u) mxu[u] = 0;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (kU - 1) * stride < mm; i += kU * stride) {
    T v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) v[u] = A[i + u * stride];
#pragma unroll
    for (int u = 0; u < kU; ++u) mxu[u] = fmax(mxu[u], fabs((double)v[u]));
  }
  for (; i < mm; i += stride) mxu[0] = fmax(mxu[0], fabs((double)A[i]));
  double mx = mxu[0];
#pragma unroll
  for (int u = 1; u < kU; ++u) mx = fmax(mx, mxu[u]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0)
    atomicMax(reinterpret_cast<unsigned long long*>(scale + blockIdx.y),
              (unsigned long long)__double_as_longlong(mx));
}

// LU of the panel columns [j0, j0+jb) of every front (one CTA per front).  The
// panel rows [j0, m) are staged in shared memory (column-major, leading
// dimension rows = m - j0); pivot rows are searched among the eliminated rows
// [j, k) only.  Row swaps inside the panel happen in shared memory; the same
// swaps are applied to the columns left and right of the panel by the row-block
// solve kernel (LAPACK-style full-row interchanges).
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
}

// Panel LU of a large front by a cluster of kCL CTAs (thread-block cluster, one
// front per cluster).  The panel rows [j0, m) are split in kCL contiguous chunks
// of physical rows ("slots"), each staged in its CTA's shared memory.  Rows are
// never moved during the panel: every CTA keeps the same position <-> slot maps
// and applies the pivot interchanges to the maps only.  Per pivot column each
// CTA folds its best candidate into a 64-bit key (magnitude rounded to FP32 in
// the high word, position in the low word; double-buffered), one cluster
// barrier, then warp 0 of every CTA reads the kCL keys and the pivot row through
// distributed shared memory (the pivot row is final from then on) and updates
// the maps; after one block barrier each thread updates its own slots.  The
// panel is written back in position order.  The pivot is a largest-magnitude
// entry of the column up to FP32 rounding of the magnitudes (ties and
// near-ties go to the smallest position).
constexpr int kCL = 8;
template <class T>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(256)
    lu_panel_cluster_kernel(T* fronts, int m, int k, int j0, int jb, int* piv,
                            const double* scale, double ptol, int* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int f = blockIdx.x / kCL;
  T* A = fronts + (long)f * m * m;
  const int rows = m - j0, kl = k - j0;
  const int chunk = (rows + kCL - 1) / kCL;
  const int rbeg = rank * chunk, rend = min(rows, rbeg + chunk);
  const int nmy = max(0, rend - rbeg);
  extern __shared__ unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);                        // chunk x jb, column-major
  int* pos2slot = reinterpret_cast<int*>(P + (long)chunk * jb);  // rows
  int* slot2pos = pos2slot + rows;                            // rows
  // candidate key: (float bits of |value|) << 32 | (0xffffffff - position), so the
  // largest key is the largest magnitude, ties to the smallest position
  __shared__ unsigned long long ckey[2];
  __shared__ T prow[kNB];
  __shared__ int s_slot;
  const double thresh = ptol * scale[f];
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    pos2slot[i] = i;
    slot2pos[i] = i;
  }
  if (threadIdx.x < 2) ckey[threadIdx.x] = 0ull;
  for (long e = threadIdx.x; e < (long)nmy * jb; e += blockDim.x) {
    int r = (int)(e % nmy), c = (int)(e / nmy);
    P[r + (long)c * chunk] = A[(j0 + rbeg + r) + (long)(j0 + c) * m];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jj = 0; jj < jb; ++jj) {
    // best candidate among my slots whose position is in [jj, kl)
    unsigned long long key = 0ull;
    for (int sl = rbeg + threadIdx.x; sl < rend; sl += blockDim.x) {
      const int ps = slot2pos[sl];
      if (ps < jj || ps >= kl) continue;
      float v = (float)fabs((double)P[(sl - rbeg) + (long)jj * chunk]);
      unsigned long long kk = ((unsigned long long)__float_as_uint(v) << 32) |
                              (unsigned long long)(0xffffffffu - (unsigned)ps);
      key = kk > key ? kk : key;
    }
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ok = __shfl_down_sync(0xffffffffu, key, o);
      key = ok > key ? ok : key;
    }
    if (lane == 0 && key) atomicMax(&ckey[jj & 1], key);
    cl.sync();  // candidates of column jj published
    if (warp == 0) {
      unsigned long long kb = 0ull;
      if (lane < kCL) kb = *cl.map_shared_rank(&ckey[jj & 1], lane);
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ok = __shfl_down_sync(0xffffffffu, kb, o);
        kb = ok > kb ? ok : kb;
      }
      kb = __shfl_sync(0xffffffffu, kb, 0);
      const int p = kb ? (int)(0xffffffffu - (unsigned)(kb & 0xffffffffull)) : jj;
      const double b0 = kb ? (double)__uint_as_float((unsigned)(kb >> 32)) : -1.0;
      const int sb = pos2slot[p];
      // the pivot row (final from now on) from its owner's shared memory
      const int owner = sb / chunk;
      if (lane < jb) prow[lane] = cl.map_shared_rank(P, owner)[(sb - owner * chunk) + (long)lane * chunk];
      __syncwarp();
      if (lane == 0) {
        const int sa = pos2slot[jj];
        pos2slot[jj] = sb;
        pos2slot[p] = sa;
        slot2pos[sb] = jj;
        slot2pos[sa] = p;
        s_slot = sb;
        ckey[(jj + 1) & 1] = 0ull;  // last read before this iteration's barrier
        if (rank == 0) {
          piv[(long)f * k + j0 + jj] = j0 + p;
          if (!(b0 > thresh)) atomicOr(status, 1);
        }
      }
    }
    __syncthreads();
    T pv = prow[jj];
    if (!(fabs((double)pv) > 0.0)) pv = (T)(thresh > 0 ? thresh : 1e-30);
    const T inv = (T)1 / pv;
    for (int sl = rbeg + threadIdx.x; sl < rend; sl += blockDim.x) {
      if (slot2pos[sl] <= jj) continue;
      T* pr = P + (sl - rbeg);
      T l = pr[(long)jj * chunk] * inv;
      pr[(long)jj * chunk] = l;
      for (int c = jj + 1; c < jb; ++c) pr[(long)c * chunk] -= l * prow[c];
    }
  }
  // the pivot rows read by other CTAs are final, but keep this CTA's shared
  // memory alive until every CTA has read its last pivot row
  cl.sync();
  for (long e = threadIdx.x; e < (long)nmy * jb; e += blockDim.x) {
    int r = (int)(e % nmy), c = (int)(e / nmy);
    A[(j0 + slot2pos[rbeg + r]) + (long)(j0 + c) * m] = P[r + (long)c * chunk];
  }
}

// Panel LU of a front too tall for the cluster panel: G CTAs per front in one
// cooperative launch (every CTA resident), the fronts of a level in groups of
// nfl per launch.  CTA g stages the panel rows ("slots") [g c, (g+1) c) of rows
// [j0, m) in shared memory; rows never move during the panel.  A slot is a pivot
// candidate while its starting position is below k (interchanges only exchange
// positions below k) and it has not been a pivot yet.  Per pivot column every
// CTA publishes the row of its best candidate, then (release) one 64-bit word:
// FP32 magnitude in bits 32-63, 2^20 - 1 - slot in bits 8-27, the column tag in
// bits 0-7 (words of one column compare like their keys); each CTA polls the
// words of its front's G CTAs (acquire, all in flight at once), takes the
// largest and copies the winner's row: no other barrier.  The publication slots alternate between two
// buffers by column parity (a CTA cannot publish column j+2 before every CTA has
// published j+1, i.e. finished reading column j).  The pivot positions are
// reconstructed after the panel from the sequence of pivot slots; each CTA then
// writes its rows back in position order.  A poll that does not complete within
// wait_ns (2 s by default) sets bit 2 of *status and the CTA returns without
// writing back (CTA 0 of the front leaves identity interchanges for the panel).
constexpr int kPubWords = 1 + kNB;  // word, row (in units of 8 bytes; T <= 8 bytes)
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <class T>
__global__ void __launch_bounds__(256) lu_panel_grid_kernel(T* fronts, int m, int k, int j0, int jb,
                                                            int f0, int G, int* piv,
                                                            const double* scale, double ptol,
                                                            int* status,
                                                            unsigned long long* pub,
                                                            unsigned long long wait_ns) {
  const int f = f0 + blockIdx.x / G, g = blockIdx.x % G;
  T* A = fronts + (long)f * m * m;
  const int rows = m - j0, kl = k - j0;
  const int chunk = (rows + G - 1) / G;
  const int s0 = min(rows, g * chunk), s1 = min(rows, s0 + chunk), nmy = s1 - s0;
  // publication slots of this front: [parity][g][kPubWords]
  unsigned long long* pf = pub + (long)f * 2 * kGridPanelMaxG * kPubWords;
  extern __shared__ unsigned long long smraw_u64[];
  T* P = reinterpret_cast<T*>(smraw_u64);                      // chunk x jb, column-major
  unsigned char* elim = reinterpret_cast<unsigned char*>(P + (long)chunk * jb);
  __shared__ T prow[kNB];
  __shared__ unsigned long long wkey[8];
  __shared__ int pslot[kNB];
  __shared__ int ds[2 * kNB], dp[2 * kNB];
  __shared__ int s_nd, s_abort;
  const double thresh = ptol * scale[f];
  for (long e = threadIdx.x; e < (long)nmy * jb; e += blockDim.x) {
    const int r = (int)(e % nmy), c = (int)(e / nmy);
    P[r + (long)c * chunk] = A[(j0 + s0 + r) + (long)(j0 + c) * m];
  }
  for (int r = threadIdx.x; r < nmy; r += blockDim.x) elim[r] = 0;
  if (threadIdx.x == 0) s_abort = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  for (int jj = 0; jj < jb; ++jj) {
    const unsigned long long tag = (unsigned long long)(jj + 1);
    unsigned long long key = 0ull;
    for (int r = threadIdx.x; r < nmy; r += blockDim.x) {
      const int sl = s0 + r;
      if (sl >= kl || elim[r]) continue;
      const float v = (float)fabs((double)P[r + (long)jj * chunk]);
      const unsigned long long kk = ((unsigned long long)__float_as_uint(v) << 32) |
                                    ((unsigned long long)(0xFFFFFu - (unsigned)sl) << 8);
      key = kk > key ? kk : key;
    }
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ok = __shfl_down_sync(0xffffffffu, key, o);
      key = ok > key ? ok : key;
    }
    if (lane == 0) wkey[warp] = key;
    __syncthreads();
    unsigned long long* base = pf + (long)(jj & 1) * kGridPanelMaxG * kPubWords;
    if (warp == 0) {
      unsigned long long kb = wkey[lane & 7];
      for (int o = 4; o > 0; o >>= 1) {
        unsigned long long ok = __shfl_down_sync(0xffffffffu, kb, o);
        kb = ok > kb ? ok : kb;
      }
      if (lane == 0) {
        unsigned long long* mine = base + (long)g * kPubWords;
        if (kb) {
          const int r = (int)(0xFFFFFu - (unsigned)((kb >> 8) & 0xFFFFFu)) - s0;
          T* row = reinterpret_cast<T*>(mine + 1);
          for (int c = 0; c < jb; ++c) row[c] = P[r + (long)c * chunk];
        }
        st_release64(mine, kb | tag);  // orders the row stores before the word
      }
      // the G words of this column, all loads in flight at once
      constexpr int kPer = (kGridPanelMaxG + 31) / 32;
      unsigned long long w[kPer];
      bool rdy[kPer];
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        w[i] = 0ull;
        rdy[i] = lane + 32 * i >= G;
      }
      const unsigned long long t0 = gtimer_ns();
      bool ok = true;
      while (true) {
#pragma unroll
        for (int i = 0; i < kPer; ++i)
          if (!rdy[i]) w[i] = ld_acquire64(base + (long)(lane + 32 * i) * kPubWords);
        bool mine_ok = true;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          if (!rdy[i]) rdy[i] = (w[i] & 0xFFull) == tag;
          mine_ok = mine_ok && rdy[i];
        }
        if (__all_sync(0xffffffffu, mine_ok)) break;
        if (gtimer_ns() - t0 > wait_ns) {
          ok = false;
          break;
        }
      }
      __syncwarp();  // the lanes' acquires order the row reads of every lane below
      unsigned long long best = 0ull;
#pragma unroll
      for (int i = 0; i < kPer; ++i)
        if (lane + 32 * i < G) best = w[i] > best ? w[i] : best;
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
        best = ob > best ? ob : best;
      }
      best = __shfl_sync(0xffffffffu, best, 0);
      int sb = (int)(0xFFFFFu - (unsigned)((best >> 8) & 0xFFFFFu));
      const bool valid = ok && (best >> 8) != 0ull && sb >= 0 && sb < rows;
      if (!valid) {
        if (lane == 0) {
          s_abort = 1;
          atomicOr(status, ok ? 1 : 2);
        }
        sb = 0;
      } else {
        const T* orow = reinterpret_cast<const T*>(base + (long)(sb / chunk) * kPubWords + 1);
        if (lane < jb) prow[lane] = __ldcg(orow + lane);
      }
      if (lane == 0) {
        pslot[jj] = sb;
        if (sb >= s0 && sb < s1) elim[sb - s0] = 1;
      }
    }
    __syncthreads();
    if (s_abort) {
      // the panel stops here; later kernels of the factorisation still read this
      // panel's interchanges, so leave in-range (identity) ones
      if (g == 0)
        for (int c = threadIdx.x; c < jb; c += blockDim.x) piv[(long)f * k + j0 + c] = j0 + c;
      return;
    }
    T pv = prow[jj];
    if (g == 0 && threadIdx.x == 0 && !(fabs((double)pv) > thresh)) atomicOr(status, 1);
    if (!(fabs((double)pv) > 0.0)) pv = (T)(thresh > 0 ? thresh : 1e-30);
    const T inv = (T)1 / pv;
    for (int r = threadIdx.x; r < nmy; r += blockDim.x) {
      if (elim[r]) continue;
      T* pr = P + r;
      const T l = pr[(long)jj * chunk] * inv;
      pr[(long)jj * chunk] = l;
      for (int c = jj + 1; c < jb; ++c) pr[(long)c * chunk] -= l * prow[c];
    }
  }
  // positions: replay the interchanges (pivot slot pslot[jj] moves to position jj,
  // the slot at jj moves to the pivot's position); displaced slots in ds/dp
  if (threadIdx.x == 0) {
    int nd = 0;
    for (int jj = 0; jj < jb; ++jj) {
      const int sb = pslot[jj];
      int p = sb, ib = -1, sa = jj, ia = -1;
      for (int i = 0; i < nd; ++i) {
        if (ds[i] == sb) {
          p = dp[i];
          ib = i;
        }
      }
      for (int i = 0; i < nd; ++i)
        if (dp[i] == jj) {
          sa = ds[i];
          ia = i;
        }
      if (ia < 0)
        for (int i = 0; i < nd; ++i)
          if (ds[i] == sa) ia = i;
      if (ib < 0) {
        ib = nd++;
        ds[ib] = sb;
      }
      dp[ib] = jj;
      if (sa != sb) {
        if (ia < 0) {
          ia = nd++;
          ds[ia] = sa;
        }
        dp[ia] = p;
      }
      if (g == 0) piv[(long)f * k + j0 + jj] = j0 + p;
    }
    s_nd = nd;
  }
  __syncthreads();
  const int nd = s_nd;
  for (long e = threadIdx.x; e < (long)nmy * jb; e += blockDim.x) {
    const int r = (int)(e % nmy), c = (int)(e / nmy);
    const int sl = s0 + r;
    int pos = sl;
    for (int i = 0; i < nd; ++i)
      if (ds[i] == sl) pos = dp[i];
    A[(j0 + pos) + (long)(j0 + c) * m] = P[r + (long)c * chunk];
  }
}

// ---- tournament pivoting of the grid panel (FP32 forms) -------------------------
// Communication-avoiding LU of the panel (Grigori, Demmel and Xiang, "CALU", 2011):
// instead of one publication round per pivot column, the jb pivot rows are chosen
// by a tournament, then every row is eliminated against them at once.
//   1. each CTA runs partial-pivoting elimination on its candidate rows (slot below
//      k - j0) and publishes the ORIGINAL values of its jb winners (read again
//      from the front, which the panel does not change until its write-back);
//   2. the first CTA of every group of kCaluGroup CTAs gathers the group's winners,
//      runs the same elimination on them and publishes its jb winners' originals;
//   3. every CTA gathers the groups' winners and runs the same elimination, which
//      fixes the panel's pivot rows in order and their factored values [L11 | U11]
//      (every CTA computes identical values from identical inputs);
//   4. every other row gets its multipliers l = a U11^{-1} from its original values;
//   5. the interchanges and the write-back are those of lu_panel_grid_kernel.
// Pivots are chosen by FP32 magnitude with ties to the smaller slot.  Each wait on a
// publication gives up after wait_ns (status bit 2, identity interchanges, return).
constexpr int kCaluGroup = 16;
constexpr int kCaluMaxGroups = (kGridPanelMaxG + kCaluGroup - 1) / kCaluGroup;
constexpr int kCaluRow = kNB + 1;  // words of a published row: jb values, then the slot
constexpr long kCaluTagWords = 256;  // u64 words: tags of level 1 (G) and level 2 (groups)
constexpr long kCaluFrontWords =
    kCaluTagWords + ((long)(kGridPanelMaxG + kCaluMaxGroups) * kNB * kCaluRow + 1) / 2;
constexpr size_t kCaluBuf = sizeof(float) * (size_t)kCaluGroup * kNB * kCaluRow;  // gather buffer

// Partial-pivoting elimination of the rows [0, R) of the shared-memory matrix
// M(r, c) = M[r rs + c cs] (jb columns), candidates cand(r); up to jb pivots in order
// into sel[] (row indices), *nsel their count.  Rows are owned round-robin by the
// threads; two barriers per pivot.  used: R bytes of shared memory.
template <class Cand, class Slot>
__device__ void calu_gepp(float* M, int rs, int cs, int R, int jb, Cand cand, Slot slot,
                          unsigned char* used, int* sel, int* nsel, unsigned long long* wkey) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto keyof = [&](int r, int c) -> unsigned long long {
    const float v = fabsf(M[r * rs + c * cs]);
    return ((unsigned long long)__float_as_uint(v) << 32) |
           ((unsigned long long)(0xFFFFFu - (unsigned)slot(r)) << 12) | (unsigned long long)r;
  };
  for (int r = threadIdx.x; r < R; r += blockDim.x) used[r] = cand(r) ? 0 : 1;
  __syncthreads();
  unsigned long long key = 0ull;
  for (int r = threadIdx.x; r < R; r += blockDim.x)
    if (!used[r]) {
      const unsigned long long kk = keyof(r, 0);  // nonzero even for a zero entry (slot field)
      key = (kk > key) ? kk : key;
    }
  int n = 0;
  for (int jj = 0; jj < jb; ++jj) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_down_sync(0xffffffffu, key, o);
      key = ok > key ? ok : key;
    }
    if (lane == 0) wkey[warp] = key;
    __syncthreads();
    unsigned long long kb = 0ull;
    for (int w = 0; w < nw; ++w) kb = wkey[w] > kb ? wkey[w] : kb;
    // a candidate row always carries a key > 0 (its slot field is nonzero)
    if (kb == 0ull) break;
    const int p = (int)(kb & 0xFFFull);
    if (threadIdx.x == 0) sel[jj] = p;
    n = jj + 1;
    float pv = M[p * rs + jj * cs];
    if (!(fabsf(pv) > 0.f)) pv = 1e-30f;
    const float inv = 1.f / pv;
    key = 0ull;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      if (used[r]) continue;
      if (r == p) {
        used[r] = 1;
        continue;
      }
      const float l = M[r * rs + jj * cs] * inv;
      M[r * rs + jj * cs] = l;
      for (int c = jj + 1; c < jb; ++c) M[r * rs + c * cs] -= l * M[p * rs + c * cs];
      if (jj + 1 < jb) {
        const unsigned long long kk = keyof(r, jj + 1);
        key = kk > key ? kk : key;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *nsel = n;
  __syncthreads();
}

__global__ void __launch_bounds__(256) lu_panel_calu_kernel(float* fronts, int m, int k, int j0,
                                                             int jb, int f0, int G, int* piv,
                                                             const double* scale, double ptol,
                                                             int* status, unsigned long long* pub,
                                                             unsigned long long wait_ns) {
  const int fl = blockIdx.x / G, g = blockIdx.x % G;
  const int f = f0 + fl;
  float* A = fronts + (long)f * m * m;
  const int rows = m - j0, kl = k - j0;
  const int chunk = (rows + G - 1) / G;
  const int s0 = min(rows, g * chunk), s1 = min(rows, s0 + chunk), nmy = s1 - s0;
  const int ngroups = (G + kCaluGroup - 1) / kCaluGroup;
  unsigned long long* tags = pub + (long)f * kCaluFrontWords;  // [G] then [ngroups]
  float* cand1 = reinterpret_cast<float*>(tags + kCaluTagWords);  // [G][jb][kCaluRow]
  float* cand2 = cand1 + (long)kGridPanelMaxG * kNB * kCaluRow;   // [groups][jb][kCaluRow]
  extern __shared__ unsigned long long smraw_u64[];
  float* P = reinterpret_cast<float*>(smraw_u64);              // chunk x jb, column-major
  float* Bf = P + (long)chunk * jb;                              // gather buffer, row-major
  unsigned char* used = reinterpret_cast<unsigned char*>(Bf + (long)kCaluGroup * kNB * kCaluRow);
  // used: max(chunk, kCaluGroup jb) bytes; pivj: chunk ints after it
  int* pivj = reinterpret_cast<int*>(used + ((max(chunk, kCaluGroup * kNB) + 15) & ~15));
  __shared__ float UF[kNB][kNB + 1];
  __shared__ int sel[kNB], pslot[kNB], bslot[kCaluGroup * kNB];
  __shared__ unsigned long long wkey[8];
  __shared__ int s_n, s_abort;
  __shared__ int ds[2 * kNB], dp[2 * kNB];
  __shared__ int s_nd, s_ok;
  __shared__ int cnt[kGridPanelMaxG], offs[kGridPanelMaxG + 1];
  const double thresh = ptol * scale[f];
  if (threadIdx.x == 0) s_abort = 0;
  // ---- 1. local tournament on the chunk
  for (long e = threadIdx.x; e < (long)nmy * jb; e += blockDim.x) {
    const int r = (int)(e % nmy), c = (int)(e / nmy);
    P[r + (long)c * chunk] = A[(j0 + s0 + r) + (long)(j0 + c) * m];
  }
  __syncthreads();
  calu_gepp(P, 1, chunk, nmy, jb, [&](int r) { return s0 + r < kl; }, [&](int r) { return s0 + r; },
            used, sel, &s_n, wkey);
  const int n1 = s_n;
  {
    float* out = cand1 + (long)g * kNB * kCaluRow;  // this CTA's level-1 block of its front
    for (int e = threadIdx.x; e < n1 * jb; e += blockDim.x) {
      const int i = e / jb, c = e % jb;
      const int r = sel[i];
      out[(long)i * kCaluRow + c] = A[(j0 + s0 + r) + (long)(j0 + c) * m];
      if (c == 0) out[(long)i * kCaluRow + jb] = __int_as_float(s0 + r);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release64(tags + g, ((unsigned long long)n1 << 8) | 1ull);
  }
  // bounded wait for the tags [t0, t1) of `tags`; returns the candidate counts in cnt
  auto wait_tags = [&](const unsigned long long* tg, int t0, int t1) -> bool {
    if (threadIdx.x < 32) {
      const unsigned long long tstart = gtimer_ns();
      bool ok = true;
      for (int i = t0 + (int)threadIdx.x; i < t1; i += 32) {
        unsigned long long v = ld_acquire64(tg + i);
        while ((v & 0xFFull) != 1ull) {
          if (gtimer_ns() - tstart > wait_ns) {
            ok = false;
            break;
          }
          v = ld_acquire64(tg + i);
        }
        if (!ok) break;
        cnt[i - t0] = (int)(v >> 8);
      }
      ok = __all_sync(0xffffffffu, ok);
      if (threadIdx.x == 0) s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
  };
  // gathers the candidate blocks [b0, b1) of `src` (counts in cnt) into Bf (row-major,
  // kCaluRow words per row; block b's rows start at offs[b - b0])
  auto gather = [&](const float* src, int b0, int b1) -> int {
    if (threadIdx.x == 0) {
      offs[0] = 0;
      for (int b = b0; b < b1; ++b) offs[b - b0 + 1] = offs[b - b0] + cnt[b - b0];
    }
    __syncthreads();
    const int tot = offs[b1 - b0];
    for (int b = b0; b < b1; ++b) {
      const float* blk = src + (long)b * kNB * kCaluRow;
      const int nb = cnt[b - b0], o = offs[b - b0];
      for (int e = threadIdx.x; e < nb * kCaluRow; e += blockDim.x)
        Bf[(long)o * kCaluRow + e] = __ldcg(blk + e);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tot; i += blockDim.x) bslot[i] = __float_as_int(Bf[(long)i * kCaluRow + jb]);
    __syncthreads();
    return tot;
  };
  // ---- 2. group tournament (first CTA of each group)
  const int grp = g / kCaluGroup;
  if (g % kCaluGroup == 0) {
    const int b0 = grp * kCaluGroup, b1 = min(G, b0 + kCaluGroup);
    if (!wait_tags(tags, b0, b1)) {
      if (threadIdx.x == 0) {
        s_abort = 1;
        atomicOr(status, 2);
      }
    } else {
      const int tot = gather(cand1, b0, b1);
      calu_gepp(Bf, kCaluRow, 1, tot, jb, [&](int) { return true; }, [&](int r) { return bslot[r]; },
                used, sel, &s_n, wkey);
      const int n2 = s_n;
      float* out = cand2 + (long)grp * kNB * kCaluRow;
      // the winners' original rows: re-read from the level-1 area (Bf was eliminated)
      for (int e = threadIdx.x; e < n2 * kCaluRow; e += blockDim.x) {
        const int i = e / kCaluRow, c = e % kCaluRow;
        const int r = sel[i];
        // row r of Bf came from level-1 block b at row r - offs[b - b0]
        int b = b0;
        while (b + 1 < b1 && r >= offs[b + 1 - b0]) ++b;
        out[(long)i * kCaluRow + c] =
            __ldcg(cand1 + (long)b * kNB * kCaluRow + (long)(r - offs[b - b0]) * kCaluRow + c);
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) st_release64(tags + G + grp, ((unsigned long long)n2 << 8) | 1ull);
    }
  }
  __syncthreads();
  // ---- 3. final tournament (every CTA)
  if (!s_abort) {
    if (!wait_tags(tags + G, 0, ngroups)) {
      if (threadIdx.x == 0) {
        s_abort = 1;
        atomicOr(status, 2);
      }
    }
  }
  __syncthreads();
  if (s_abort) {
    if (g == 0)
      for (int c = threadIdx.x; c < jb; c += blockDim.x) piv[(long)f * k + j0 + c] = j0 + c;
    return;
  }
  {
    const int tot = gather(cand2, 0, ngroups);
    calu_gepp(Bf, kCaluRow, 1, tot, jb, [&](int) { return true; }, [&](int r) { return bslot[r]; },
              used, sel, &s_n, wkey);
    if (s_n < jb) {  // fewer candidates than columns: cannot happen inside k
      if (threadIdx.x == 0) atomicOr(status, 1);
    }
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
      const int j = e / jb, c = e % jb;
      UF[j][c] = j < s_n ? Bf[(long)sel[j] * kCaluRow + c] : (c == j ? 1.f : 0.f);
    }
    for (int j = threadIdx.x; j < jb; j += blockDim.x) pslot[j] = j < s_n ? bslot[sel[j]] : -1;
    __syncthreads();
    for (int j = threadIdx.x; j < jb; j += blockDim.x) {
      float d = UF[j][j];
      if (g == 0 && !(fabs((double)d) > thresh)) atomicOr(status, 1);
      if (!(fabsf(d) > 0.f)) UF[j][j] = (float)(thresh > 0 ? thresh : 1e-30);
    }
  }
  // ---- 4. rows of the chunk: pivot rows take their factored values, the others
  // their multipliers from the original values
  for (int r = threadIdx.x; r < nmy; r += blockDim.x) pivj[r] = -1;
  __syncthreads();
  for (int j = threadIdx.x; j < jb; j += blockDim.x)
    if (pslot[j] >= s0 && pslot[j] < s1) pivj[pslot[j] - s0] = j;
  for (long e = threadIdx.x; e < (long)nmy * jb; e += blockDim.x) {
    const int r = (int)(e % nmy), c = (int)(e / nmy);
    P[r + (long)c * chunk] = A[(j0 + s0 + r) + (long)(j0 + c) * m];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nmy; r += blockDim.x) {
    float* pr = P + r;
    const int j = pivj[r];
    if (j >= 0) {
      for (int c = 0; c < jb; ++c) pr[(long)c * chunk] = UF[j][c];
      continue;
    }
    for (int c = 0; c < jb; ++c) {
      float a = pr[(long)c * chunk];
      for (int i = 0; i < c; ++i) a -= pr[(long)i * chunk] * UF[i][c];
      pr[(long)c * chunk] = a / UF[c][c];
    }
  }
  // ---- 5. positions of the interchanges (pivot slot pslot[jj] to position jj) and
  // the write-back, as in lu_panel_grid_kernel
  if (threadIdx.x == 0) {
    int nd = 0;
    for (int jj = 0; jj < jb; ++jj) {
      const int sb = pslot[jj];
      int p = sb, ib = -1, sa = jj, ia = -1;
      for (int i = 0; i < nd; ++i) {
        if (ds[i] == sb) {
          p = dp[i];
          ib = i;
        }
      }
      for (int i = 0; i < nd; ++i)
        if (dp[i] == jj) {
          sa = ds[i];
          ia = i;
        }
      if (ia < 0)
        for (int i = 0; i < nd; ++i)
          if (ds[i] == sa) ia = i;
      if (ib < 0) {
        ib = nd++;
        ds[ib] = sb;
      }
      dp[ib] = jj;
      if (sa != sb) {
        if (ia < 0) {
          ia = nd++;
          ds[ia] = sa;
        }
        dp[ia] = p;
      }
      if (g == 0) piv[(long)f * k + j0 + jj] = j0 + p;
    }
    s_nd = nd;
  }
  __syncthreads();
  const int nd = s_nd;
  for (long e = threadIdx.x; e < (long)nmy * jb; e += blockDim.x) {
    const int r = (int)(e % nmy), c = (int)(e / nmy);
    const int sl = s0 + r;
    int pos = sl;
    for (int i = 0; i < nd; ++i)
      if (ds[i] == sl) pos = dp[i];
    A[(j0 + pos) + (long)(j0 + c) * m] = P[r + (long)c * chunk];
  }
}

// Interchanges of the panel's pivots and the row-block solve
// A[j0:j0+jb, c] = L_pp^{-1} A[j0:j0+jb, c] on the columns c in [c_lo, c_hi)
// outside the panel [j0, j0+jb): columns left of the panel get the interchanges
// only, columns right of it the interchanges (when do_swap) and the solve.  One
// thread per column.  The full-front form is c_lo = 0, c_hi = m, do_swap = 1.
template <class T>
__global__ void __launch_bounds__(256) lu_trsm_kernel(T* fronts, int m, int k, int j0, int jb,
                                                      const int* piv, int c_lo, int c_hi,
                                                      int do_swap) {
  T* A = fronts + (long)blockIdx.y * m * m;
  __shared__ T Lp[kNB][kNB + 1];
  __shared__ int sp_[kNB];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e % jb, l = e / jb;
    Lp[i][l] = A[(j0 + i) + (long)(j0 + l) * m];
  }
  for (int e = threadIdx.x; e < jb; e += blockDim.x) sp_[e] = piv[(long)blockIdx.y * k + j0 + e];
  __syncthreads();
  const int nleft = max(0, min(j0, c_hi) - c_lo);
  const int rbeg = max(j0 + jb, c_lo);
  const int cc = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = cc < nleft ? c_lo + cc : rbeg + (cc - nleft);
  if (c >= c_hi) return;
  T* colg = A + (long)c * m;
  if (do_swap)
    for (int jj = 0; jj < jb; ++jj) {
      int p = sp_[jj];
      if (p != j0 + jj) {
        T t = colg[j0 + jj];
        colg[j0 + jj] = colg[p];
        colg[p] = t;
      }
    }
  if (cc < nleft) return;
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

// Row interchanges piv[p0 .. p0+cnt) (in order) on the columns [a0, a1) and
// [b0, b1) of every front; one thread per column.
template <class T>
__global__ void lu_laswp_kernel(T* fronts, int m, int k, int p0, int cnt, const int* piv, int a0,
                                int a1, int b0, int b1) {
  T* A = fronts + (long)blockIdx.y * m * m;
  const int cc = blockIdx.x * blockDim.x + threadIdx.x;
  const int na = a1 - a0;
  const int c = cc < na ? a0 + cc : b0 + (cc - na);
  if (c >= (cc < na ? a1 : b1)) return;
  const int* pv = piv + (long)blockIdx.y * k;
  T* col = A + (long)c * m;
  for (int j = p0; j < p0 + cnt; ++j) {
    const int p = pv[j];
    if (p != j) {
      T t = col[j];
      col[j] = col[p];
      col[p] = t;
    }
  }
}

// Batched C[M x N] -= A[M x K] B[K x N], K <= kNB, column-major with leading
// dimensions lda/ldb/ldc and per-batch strides (blockIdx.y = batch).  TILE x TILE
// per CTA (TILE = 64: 4 x 4 per thread, TILE = 32: 2 x 2 per thread; the launcher
// picks the one that wastes less work on the padding of the last tile row and
// column).  Used for the Schur update of the LU.
template <class T, int TILE>
__global__ void __launch_bounds__(256) gemm_sub_kernel(int M, int N, int K, const T* A, int lda,
                                                       long sA, const T* B, int ldb, long sB,
                                                       T* C, int ldc, long sC, int tilesM) {
  constexpr int R = TILE / 16;
  A += blockIdx.y * sA;
  B += blockIdx.y * sB;
  C += blockIdx.y * sC;
  const int tr = blockIdx.x % tilesM, tc = blockIdx.x / tilesM;
  const int r0 = tr * TILE, c0 = tc * TILE;
  __shared__ T As[kNB][TILE];
  __shared__ T Bs[kNB][TILE + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  // FP32: this thread's C entries are loaded first, so their latency overlaps the
  // staging of A and B and the products (the update is bound by C traffic); FP64
  // is bound by the FP64 pipe and keeps its registers for occupancy
  constexpr bool kPre = sizeof(T) == sizeof(float);
  T cpre[R][R];
  if constexpr (kPre) {
#pragma unroll
    for (int b = 0; b < R; ++b) {
      const int c = c0 + ty + 16 * b;
#pragma unroll
      for (int a = 0; a < R; ++a) {
        const int r = r0 + tx + 16 * a;
        cpre[a][b] = (r < M && c < N) ? C[r + (long)c * ldc] : (T)0;
      }
    }
  }
  for (int e = threadIdx.x; e < K * TILE; e += blockDim.x) {
    int i = e % TILE, l = e / TILE;
    int r = r0 + i;
    As[l][i] = (r < M) ? A[r + (long)l * lda] : (T)0;
  }
  for (int e = threadIdx.x; e < K * TILE; e += blockDim.x) {
    int l = e % K, jc = e / K;
    int c = c0 + jc;
    Bs[l][jc] = (c < N) ? B[l + (long)c * ldb] : (T)0;
  }
  __syncthreads();
  T acc[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) acc[a][b] = 0;
  for (int l = 0; l < K; ++l) {
    T av[R], bv[R];
#pragma unroll
    for (int a = 0; a < R; ++a) av[a] = As[l][tx + 16 * a];
#pragma unroll
    for (int b = 0; b < R; ++b) bv[b] = Bs[l][ty + 16 * b];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int b = 0; b < R; ++b) {
    int c = c0 + ty + 16 * b;
    if (c >= N) continue;
#pragma unroll
    for (int a = 0; a < R; ++a) {
      int r = r0 + tx + 16 * a;
      if (r < M) {
        if constexpr (kPre) C[r + (long)c * ldc] = cpre[a][b] - acc[a][b];
        else C[r + (long)c * ldc] -= acc[a][b];
      }
    }
  }
}

// Batched C = beta C + alpha A B (column-major, any K) with triangle-aware K
// ranges: tri_a = 1 when A is lower triangular (A[r, l] = 0 for l > r), 2 when
// upper (A[r, l] = 0 for l < r); tri_b = 1 when B is lower (B[l, c] = 0 for
// l < c), 2 when upper (B[l, c] = 0 for l > c).  Zero tiles are skipped, entries
// inside a computed tile must hold their zeros.  beta is 0 or 1.
template <class T, int TILE>
__global__ void __launch_bounds__(256) gemm_gen_kernel(int M, int N, int K, T alpha, int beta_one,
                                                       const T* A, int lda, long sA, const T* B,
                                                       int ldb, long sB, T* C, int ldc, long sC,
                                                       int tilesM, int tri_a, int tri_b, int nb2,
                                                       long sA2, long sB2, long sC2) {
  constexpr int R = TILE / 16;  // outputs per thread along each dimension
  // batch index = outer * nb2 + inner with strides (sA, sB, sC) and (sA2, sB2, sC2)
  const long bo = blockIdx.y / nb2, bi = blockIdx.y % nb2;
  A += bo * sA + bi * sA2;
  B += bo * sB + bi * sB2;
  C += bo * sC + bi * sC2;
  const int tr = blockIdx.x % tilesM, tc = blockIdx.x / tilesM;
  const int r0 = tr * TILE, c0 = tc * TILE;
  int klo = 0, khi = K;
  if (tri_a == 1) khi = min(khi, r0 + TILE);
  if (tri_a == 2) klo = max(klo, r0);
  if (tri_b == 1) klo = max(klo, c0);
  if (tri_b == 2) khi = min(khi, c0 + TILE);
  __shared__ T As[kNB][TILE];
  __shared__ T Bs[kNB][TILE + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) acc[a][b] = 0;
  for (int k0 = klo; k0 < khi; k0 += kNB) {
    const int kc = min(kNB, khi - k0);
    for (int e = threadIdx.x; e < kNB * TILE; e += blockDim.x) {
      int i = e % TILE, l = e / TILE;
      int r = r0 + i;
      As[l][i] = (r < M && l < kc) ? A[r + (long)(k0 + l) * lda] : (T)0;
    }
    for (int e = threadIdx.x; e < kNB * TILE; e += blockDim.x) {
      int l = e % kNB, jc = e / kNB;
      int c = c0 + jc;
      Bs[l][jc] = (c < N && l < kc) ? B[(k0 + l) + (long)c * ldb] : (T)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < kNB; ++l) {
      T av[R], bv[R];
#pragma unroll
      for (int a = 0; a < R; ++a) av[a] = As[l][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < R; ++b) bv[b] = Bs[l][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < R; ++b) {
    int c = c0 + ty + 16 * b;
    if (c >= N) continue;
#pragma unroll
    for (int a = 0; a < R; ++a) {
      int r = r0 + tx + 16 * a;
      if (r < M) {
        T v = alpha * acc[a][b];
        if (beta_one) v += C[r + (long)c * ldc];
        C[r + (long)c * ldc] = v;
      }
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
// Inverse of every 32 x 32 diagonal block of L11 (unit lower; upper == 0) or U11
// (upper == 1) of every front, written to the matching diagonal block of X
// (entry (i, j) at i + j ldx, front stride sX).  One CTA per (block, front);
// thread c solves column c by substitution.
template <class T>
__global__ void trinv_diag32_kernel(const T* fronts, int m, T* X, int ldx, long sX, int k,
                                    int upper) {
  const int j0 = blockIdx.x * kNB;
  const int jb = min(kNB, k - j0);
  const T* A = fronts + (long)blockIdx.y * m * m;
  T* Xf = X + (long)blockIdx.y * sX;
  __shared__ T Bk[kNB][kNB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e % jb, l = e / jb;
    Bk[i][l] = A[(j0 + i) + (long)(j0 + l) * m];
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c >= jb) return;
  T x[kNB];
#pragma unroll
  for (int i = 0; i < kNB; ++i) x[i] = (i == c) ? (T)1 : (T)0;
  if (!upper) {
#pragma unroll
    for (int i = 0; i < kNB; ++i)
      if (i < jb) {
        T acc = x[i];
#pragma unroll
        for (int l = 0; l < kNB; ++l)
          if (l < i) acc -= Bk[i][l] * x[l];
        x[i] = acc;
      }
  } else {
#pragma unroll
    for (int i = kNB - 1; i >= 0; --i)
      if (i < jb) {
        T acc = x[i];
#pragma unroll
        for (int l = 0; l < kNB; ++l)
          if (l > i && l < jb) acc -= Bk[i][l] * x[l];
        x[i] = acc / Bk[i][i];
      }
  }
  T* col = Xf + j0 + (long)(j0 + c) * ldx;
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) col[i] = x[i];
}

// In-place inversion of the 32 x 32 diagonal blocks of L11 (unit lower) and U11
// (upper) of every front: afterwards the block's strict lower part holds the
// block of L11^{-1} and its upper part (with the diagonal) the block of U11^{-1}.
// The sweeps then resolve a diagonal block with a 32 x 32 matrix-vector product
// instead of 32 dependent steps and 32 divisions.  One CTA (32 threads) per
// (block, front); thread c computes column c of both inverses.
template <class T>
__global__ void diag32_inplace_kernel(T* fronts, int m, int k) {
  const int j0 = blockIdx.x * kNB;
  const int jb = min(kNB, k - j0);
  T* A = fronts + (long)blockIdx.y * m * m;
  __shared__ T Bk[kNB][kNB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e % jb, l = e / jb;
    Bk[i][l] = A[(j0 + i) + (long)(j0 + l) * m];
  }
  __syncthreads();
  const int c = threadIdx.x;
  T xl[kNB], xu[kNB];
#pragma unroll
  for (int i = 0; i < kNB; ++i) xl[i] = xu[i] = (i == c) ? (T)1 : (T)0;
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) {
      T acc = xl[i];
#pragma unroll
      for (int l = 0; l < kNB; ++l)
        if (l < i) acc -= Bk[i][l] * xl[l];
      xl[i] = acc;
    }
#pragma unroll
  for (int i = kNB - 1; i >= 0; --i)
    if (i < jb) {
      T acc = xu[i];
#pragma unroll
      for (int l = 0; l < kNB; ++l)
        if (l > i && l < jb) acc -= Bk[i][l] * xu[l];
      xu[i] = acc / Bk[i][i];
    }
  if (c >= jb) return;
  T* col = A + j0 + (long)(j0 + c) * m;
#pragma unroll
  for (int i = 0; i < kNB; ++i)
    if (i < jb) col[i] = (i > c) ? xl[i] : xu[i];
}

// F11 <- strict lower part of Linv, upper part (with the diagonal) of Uinv, on
// the diagonal blocks of size Bsz only (the off-diagonal blocks keep L11, U11).
// X entry (r, c) at r + c Bsz (front stride sX); one thread per block entry.
template <class T>
__global__ void trinv_store_kernel(T* fronts, int m, const T* Xl, const T* Xu, long sX, int k,
                                   int Bsz) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long bb = (long)Bsz * Bsz;
  const long blk = e / bb, rem = e % bb;
  const long r = blk * Bsz + rem % Bsz, c = blk * Bsz + rem / Bsz;
  if (r >= k || c >= k) return;
  const long f = blockIdx.y;
  const long x = f * sX + r + c * Bsz;
  fronts[f * (long)m * m + r + c * m] = (r > c) ? Xl[x] : Xu[x];
}

template <class T>
void gemm_sub(int M, int N, int K, const T* A, int lda, long sA, const T* B, int ldb, long sB,
              T* C, int ldc, long sC, int batch, cudaStream_t st, int tile = 0) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  // padded work of 64- and 32-wide tiles relative to M N
  const double w64 = (double)((M + 63) / 64 * 64) * ((N + 63) / 64 * 64);
  const double w32 = (double)((M + 31) / 32 * 32) * ((N + 31) / 32 * 32);
  if (tile == 32 || (tile == 0 && w64 > 1.1 * w32)) {
    int tilesM = (M + 31) / 32, tilesN = (N + 31) / 32;
    dim3 g(tilesM * tilesN, batch);
    gemm_sub_kernel<T, 32><<<g, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, tilesM);
  } else {
    int tilesM = (M + 63) / 64, tilesN = (N + 63) / 64;
    dim3 g(tilesM * tilesN, batch);
    gemm_sub_kernel<T, 64><<<g, 256, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, tilesM);
  }
}

template <class T>
void gemm_gen(int M, int N, int K, T alpha, bool beta_one, const T* A, int lda, long sA,
              const T* B, int ldb, long sB, T* C, int ldc, long sC, int batch, int tri_a,
              int tri_b, cudaStream_t st, int nb2 = 1, long sA2 = 0, long sB2 = 0, long sC2 = 0,
              int tile = 0) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0 || nb2 <= 0) return;
  int tilesM = (M + kTile - 1) / kTile, tilesN = (N + kTile - 1) / kTile;
  if (tile == 32 || (tile == 0 && (long)tilesM * tilesN * batch * nb2 < 304)) {
    // small problem: 32 x 32 tiles give four times the CTAs
    tilesM = (M + 31) / 32;
    tilesN = (N + 31) / 32;
    dim3 g(tilesM * tilesN, batch * nb2);
    gemm_gen_kernel<T, 32><<<g, 256, 0, st>>>(M, N, K, alpha, beta_one ? 1 : 0, A, lda, sA, B, ldb,
                                              sB, C, ldc, sC, tilesM, tri_a, tri_b, nb2, sA2, sB2,
                                              sC2);
    return;
  }
  dim3 g(tilesM * tilesN, batch * nb2);
  gemm_gen_kernel<T, kTile><<<g, 256, 0, st>>>(M, N, K, alpha, beta_one ? 1 : 0, A, lda, sA, B, ldb,
                                               sB, C, ldc, sC, tilesM, tri_a, tri_b, nb2, sA2, sB2,
                                               sC2);
}

// Replace the diagonal blocks (size Bsz, a power of two >= 32) of L11 and U11 of
// every front of the level by the blocks of L11^{-1} (strict lower part; the unit
// diagonal is implied) and U11^{-1} (upper part).  The sweeps of such a level are
// then short chains of matrix-vector products spread over many CTAs.
// Recursive doubling on the diagonal blocks (32, 64, 128, ... up to Bsz):
//   [A 0; B C]^{-1} = [A^{-1} 0; -C^{-1} (B A^{-1}), C^{-1}]
//   [A B; 0 C]^{-1} = [A^{-1}, -(A^{-1} B) C^{-1}; 0 C^{-1}]
// with the two products of each merge as batched GEMMs over fronts and pairs.
// Storage: the inverses Xl, Xu keep entry (i, j) of a diagonal block at
// i + j Bsz (a column-major array with leading dimension Bsz whose columns
// overlap: the diagonal blocks never collide, and a pair's diagonal step is
// 2 s (1 + Bsz) everywhere), k (Bsz + 1) entries per front; the work array W
// holds pair p's product at rows [2ps, 2ps+s) of a k x Bsz/2 block per front.
template <class T>
void invert_triangles(DevLevel& L, T* scratch, int Bsz, cudaStream_t st) {
  const int k = L.k, m = L.m, nf = L.nf;
  const long mm = (long)m * m;
  const int ldx = Bsz;
  const long sX = (long)k * (Bsz + 1), sW = (long)k * (Bsz / 2);
  T* F = (T*)L.front;
  T* Xl = scratch;
  T* Xu = scratch + sX * nf;
  T* W = scratch + 2 * sX * nf;
  cudaMemsetAsync(Xl, 0, sizeof(T) * sX * nf, st);
  cudaMemsetAsync(Xu, 0, sizeof(T) * sX * nf, st);
  const int nb = (k + kNB - 1) / kNB;
  dim3 gd(nb, nf);
  trinv_diag32_kernel<T><<<gd, kNB, 0, st>>>(F, m, Xl, ldx, sX, k, 0);
  trinv_diag32_kernel<T><<<gd, kNB, 0, st>>>(F, m, Xu, ldx, sX, k, 1);
  for (int s = kNB; s < k && s < Bsz; s *= 2) {
    // pairs p: A at [2ps, 2ps+s), C at [2ps+s, min(2ps+2s, k)); the pairs with a
    // full-size C go in one batched launch (fronts x pairs), a ragged last pair in
    // a second one.
    const int npairs = (k + 2 * s - 1) / (2 * s);
    const int last_c = k - ((npairs - 1) * 2 * s + s);
    const int nfull = (last_c >= s) ? npairs : npairs - 1;
    const long ps_x = 2L * s * (1 + ldx), ps_m = 2L * s * (1 + m), ps_w = 2L * s;
    for (int pass = 0; pass < 2; ++pass) {
      int cnt, p0, sc;
      if (pass == 0) {
        cnt = nfull;
        p0 = 0;
        sc = s;
      } else {
        if (nfull == npairs || last_c <= 0) continue;
        cnt = 1;
        p0 = npairs - 1;
        sc = last_c;
      }
      if (cnt <= 0) continue;
      const int a0 = p0 * 2 * s, c0 = a0 + s;
      // lower: W = B Ainv (B = L[c0.., a0..], Ainv lower), Xl[c0.., a0..] = -Cinv W
      gemm_gen<T>(sc, s, s, (T)1, false, F + c0 + (long)a0 * m, m, mm, Xl + a0 + (long)a0 * ldx,
                  ldx, sX, W + a0, k, sW, nf, 0, 1, st, cnt, ps_m, ps_x, ps_w, L.gen_tile);
      gemm_gen<T>(sc, s, sc, (T)-1, false, Xl + c0 + (long)c0 * ldx, ldx, sX, W + a0, k, sW,
                  Xl + c0 + (long)a0 * ldx, ldx, sX, nf, 1, 0, st, cnt, ps_x, ps_w, ps_x,
                  L.gen_tile);
      // upper: W = Ainv B (B = U[a0.., c0..], Ainv upper), Xu[a0.., c0..] = -W Cinv
      gemm_gen<T>(s, sc, s, (T)1, false, Xu + a0 + (long)a0 * ldx, ldx, sX, F + a0 + (long)c0 * m,
                  m, mm, W + a0, k, sW, nf, 2, 0, st, cnt, ps_x, ps_m, ps_w, L.gen_tile);
      gemm_gen<T>(s, sc, sc, (T)-1, false, W + a0, k, sW, Xu + c0 + (long)c0 * ldx, ldx, sX,
                  Xu + a0 + (long)c0 * ldx, ldx, sX, nf, 0, 2, st, cnt, ps_w, ps_x, ps_x,
                  L.gen_tile);
    }
  }
  const long nbk = (k + Bsz - 1) / Bsz;
  dim3 g((unsigned)((nbk * Bsz * Bsz + 255) / 256), nf);
  trinv_store_kernel<T><<<g, 256, 0, st>>>(F, m, Xl, Xu, sX, k, Bsz);
}

// Panel staging: one CTA when the 32-column panel fits in 160 KB of shared
// memory, else a cluster of kCL CTAs (each holding m / kCL rows) when that fits,
// else the cooperative grid panel working in global memory.
template <class T>
int panel_width(int m) {
  return m > 0 ? kNB : 0;
}
// Fronts per launch (nfl) and CTAs per front (G) of the grid panel for `rows`
// panel rows: every CTA's rows fit in kGridPanelSmem, nfl G <= kGridPanelCTAs.
template <class T>
void grid_panel_shape(int nf, int rows, int* nfl, int* G) {
  const long cmax = (long)(kGridPanelSmem / (sizeof(T) * kNB + 1));
  const int gmin = (int)std::max<long>(1, (rows + cmax - 1) / cmax);
  *nfl = std::max(1, std::min(nf, kGridPanelCTAs / gmin));
  *G = std::max(1, std::min(kGridPanelMaxG, std::min(kGridPanelCTAs / *nfl, (rows + 31) / 32)));
}

// the tournament panel's shared memory: the chunk (jb floats per row), the gather
// buffer, the row flags and the pivot map
size_t calu_smem(int chunk) {
  return sizeof(float) * (size_t)chunk * kNB + kCaluBuf +
         (size_t)((std::max(chunk, kCaluGroup * kNB) + 15) & ~15) + sizeof(int) * (size_t)chunk;
}
void calu_shape(int nf, int rows, int* nfl, int* G) {
  const long per_row = sizeof(float) * kNB + 1 + sizeof(int);
  const long cmax = (long)(kGridPanelSmem - kCaluBuf - kCaluGroup * kNB - 16) / per_row;
  const int gmin = (int)std::max<long>(1, (rows + cmax - 1) / cmax);
  *nfl = std::max(1, std::min(nf, kGridPanelCTAs / gmin));
  *G = std::max(1, std::min(kGridPanelMaxG, std::min(kGridPanelCTAs / *nfl, (rows + 31) / 32)));
}

template <class T>
int panel_kind(int m) {  // 0 one CTA, 1 cluster, 2 grid
  if ((size_t)m * kNB * sizeof(T) <= 160 * 1024) return 0;
  if ((size_t)((m + kCL - 1) / kCL) * kNB * sizeof(T) + 2 * sizeof(int) * (size_t)m <= 160 * 1024)
    return 1;
  return 2;
}

// Panel LU of columns [j0, j0+jb) followed by the interchanges and the row-block
// solve on the columns [c_lo, c_hi) outside the panel.
template <class T>
void panel_step(DevLevel& L, T* F, int j0, int jb, int c_lo, int c_hi, double ptol, int* status,
                const FactorWork& W, cudaStream_t st) {
  double pf = 0;
  for (int j = j0; j < j0 + jb; ++j) pf += (double)(L.m - j - 1) * (1.0 + 2.0 * (j0 + jb - j - 1));
  ProfScope pp(PROF_LU_PANEL, st);
  const int kind = panel_kind<T>(L.m);
  if (kind == 2 && sizeof(T) == sizeof(float) && W.calu) {
    const int rows = L.m - j0;
    if (rows >= (1 << 20)) return;  // slot field of the pivot key; factor_level_t rejects it
    int nfl, G;
    calu_shape(L.nf, rows, &nfl, &G);
    const int chunk = (rows + G - 1) / G;
    for (int f0 = 0; f0 < L.nf; f0 += nfl) {
      const int nfg = std::min(nfl, L.nf - f0);
      // fresh publication tags for every launch (graph replays reuse the buffer)
      for (int fi = 0; fi < nfg; ++fi)
        cudaMemsetAsync(W.gpub + (size_t)(f0 + fi) * kCaluFrontWords, 0,
                        sizeof(unsigned long long) * kCaluTagWords, st);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(nfg * G));
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = calu_smem(chunk);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, lu_panel_calu_kernel, (float*)F, L.m, L.k, j0, jb, f0, G, L.piv,
                         (const double*)L.scale, ptol, status, W.gpub, W.wait_ns);
    }
  } else if (kind == 2) {
    const int rows = L.m - j0;
    if (rows >= (1 << 20)) return;  // slot field of the pivot word; factor_level_t rejects it
    int nfl, G;
    grid_panel_shape<T>(L.nf, rows, &nfl, &G);
    const int chunk = (rows + G - 1) / G;
    const size_t sm = sizeof(T) * (size_t)chunk * jb + (size_t)chunk;
    for (int f0 = 0; f0 < L.nf; f0 += nfl) {
      const int nfg = std::min(nfl, L.nf - f0);
      // fresh publication tags for every launch (graph replays reuse the buffer)
      cudaMemsetAsync(W.gpub + (size_t)f0 * 2 * kGridPanelMaxG * kPubWords, 0,
                      sizeof(unsigned long long) * (size_t)nfg * 2 * kGridPanelMaxG * kPubWords,
                      st);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(nfg * G));
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = sm;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, lu_panel_grid_kernel<T>, F, L.m, L.k, j0, jb, f0, G, L.piv,
                         (const double*)L.scale, ptol, status, W.gpub, W.wait_ns);
    }
  } else if (kind == 1) {
    size_t sm = sizeof(T) * (size_t)((L.m - j0 + kCL - 1) / kCL) * jb +
                2 * sizeof(int) * (size_t)(L.m - j0);
    lu_panel_cluster_kernel<T><<<L.nf * kCL, 256, sm, st>>>(F, L.m, L.k, j0, jb, L.piv, L.scale,
                                                            ptol, status);
  } else {
    size_t sm = sizeof(T) * (size_t)(L.m - j0) * jb;
    lu_panel_kernel<T><<<L.nf, 256, sm, st>>>(F, L.m, L.k, j0, jb, L.piv, L.scale, ptol, status);
  }
  pp.done(pf * L.nf, 1, st);
  const int nleft = std::max(0, std::min(j0, c_hi) - c_lo);
  const int nright = std::max(0, c_hi - std::max(j0 + jb, c_lo));
  const int ncols = nleft + nright;
  if (ncols > 0) {
    // one thread per column; narrow CTAs when few fronts would leave SMs idle
    const int tb = ((long)((ncols + 255) / 256) * L.nf >= 152) ? 256 : 64;
    dim3 gt((ncols + tb - 1) / tb, L.nf);
    ProfScope pt(PROF_LU_TRSM, st);
    lu_trsm_kernel<T><<<gt, tb, 0, st>>>(F, L.m, L.k, j0, jb, L.piv, c_lo, c_hi, 1);
    pt.done((double)nright * jb * (jb - 1) * L.nf, 1, st);
  }
}

// C -= A B on the fronts (M x N x K sub-blocks at the given offsets, leading
// dimension m, front stride m^2): SIMT tiles for K <= 32, else the general GEMM
// or, for the tensor-core form, TF32 tensor cores.
template <class T>
void schur_update(DevLevel& L, T* F, int M, int N, int K, long offA, long offB, long offC,
                  const FactorWork& W, int* status, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  const long mm = (long)L.m * L.m;
  const double fl = 2.0 * M * N * K * L.nf;
  if (K <= kNB) {
    ProfScope pg(PROF_LU_GEMM, st);
    gemm_sub<T>(M, N, K, F + offA, L.m, mm, F + offB, L.m, mm, F + offC, L.m, mm, L.nf, st,
                L.gemm_tile);
    pg.done(fl, 1, st);
    return;
  }
  if constexpr (sizeof(T) == sizeof(float)) {
    if (W.tc) {
      ProfScope pc(PROF_LU_TC, st);
      tc_schur_update(M, N, K, (const float*)(F + offA), L.m, mm, (const float*)(F + offB), L.m, mm,
                      (float*)(F + offC), L.m, mm, L.nf, W.packA, W.packB, W.tc_split, status, st,
                      W.tc_epi);
      pc.done(fl, 3, st);
      return;
    }
  }
  ProfScope pg(PROF_LU_GEMM, st);
  gemm_gen<T>(M, N, K, (T)-1, true, F + offA, L.m, mm, F + offB, L.m, mm, F + offC, L.m, mm, L.nf,
              0, 0, st);
  pg.done(fl, 1, st);
}

template <class T>
cudaError_t factor_level_t(int d, DevLevel& L, const DevLevel* child, const double* Qcat,
                           const double* Ccat, const double* q, double ptol, int* status,
                           const FactorWork& W, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(lu_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(lu_panel_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(lu_panel_grid_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGridPanelSmem + 1024);
    cudaFuncSetAttribute(lu_panel_calu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGridPanelSmem + 1024);
    attr = true;
  }
  const long mm = (long)L.m * L.m;
  const int m = L.m, k = L.k;
  T* F = (T*)L.front;
  ProfScope pa(PROF_ASSEMBLE, st);
  cudaError_t e = cudaMemsetAsync(F, 0, sizeof(T) * mm * L.nf, st);
  if (e != cudaSuccess) return e;
  int na = 1;
  if (L.nasm > 0) {
    dim3 g((L.nasm + 255) / 256, L.nf);
    assemble_kernel<T><<<g, 256, 0, st>>>(F, L.m, L.nasm, L.asm_row, L.asm_tidx, L.asm_cvar,
                                          L.gidx, Qcat, Ccat, q, L.nfp > 0 ? L.nfp : L.nf,
                                          W.tab_stride);
    ++na;
  }
  double abytes = (double)sizeof(T) * mm * L.nf;
  if (child) {
    const int nbd = L.mc - L.kc;
    long work = (long)nbd * nbd;
    dim3 g((unsigned)((work + 256 * kEaU - 1) / (256 * kEaU)), L.nf);
    for (int dl = 0; dl < (1 << d); ++dl)
      extend_add_kernel<T><<<g, 256, 0, st>>>(F, L.m, L.nb1, (const T*)child->front, L.mc, L.kc,
                                               L.ea_map + (long)dl * nbd, dl, d);
    na += 1 << d;
    abytes += (double)sizeof(T) * work * child->nf;
  }
  cudaMemsetAsync(L.scale, 0, sizeof(double) * L.nf, st);
  {
    long chunks = std::min<long>(std::max<long>(1, mm / (256 * 16)), std::max<long>(1, 1216 / L.nf));
    dim3 gs((unsigned)chunks, L.nf);
    front_scale_kernel<T><<<gs, 256, 0, st>>>(F, mm, L.scale);
  }
  pa.done(abytes, na + 1, st);
  const int NB = panel_width<T>(m);
  if (NB == 0 || m >= (1 << 20)) return cudaErrorInvalidValue;
  const int OB = factor_outer_block(sizeof(T) == sizeof(float) ? SP_PREC_FP32 : SP_PREC_FP64, W.tc,
                                    m, k);
  if (OB == 0) {
    // right-looking LU with a Schur update after every 32-column panel
    for (int j0 = 0; j0 < k; j0 += NB) {
      const int jb = std::min(NB, k - j0);
      panel_step<T>(L, F, j0, jb, 0, m, ptol, status, W, st);
      const int base = j0 + jb, rem = m - base;
      schur_update<T>(L, F, rem, rem, jb, base + (long)j0 * m, j0 + (long)base * m,
                      base + (long)base * m, W, status, st);
    }
  } else {
    // Two-level blocked LU.  An outer block [J0, e1) of OB columns is factored in
    // sub-blocks [J1, e2) of IB columns; a sub-block is factored by 32-column
    // panel steps whose interchanges, row-block solves and updates stay inside it,
    // then its interchanges go to the rest of the outer block, its row band
    // [J1, e2) x [e2, e1) is solved and the outer block's remaining columns get
    // one update of depth IB.  After the outer block its interchanges go to the
    // other columns, the row band U12 = L11^{-1} A12 is solved in the same
    // sub-block pattern, and the trailing matrix gets one update of depth OB.
    // The updates of depth > 32 run on the tensor cores in the tensor-core forms.
    // block sizes from the outer block down to the panels: OB, 256, 32.  (A third
    // level of 128 columns, whose depth-128 updates would run on the tensor cores
    // too, leaves too much TF32 rounding in the columns next to the panels: at 3D
    // 128^3 one Helmholtz medium's preconditioner stalled GMRES at 0.42 with it.)
    const int IB = std::min(OB, kTcSubBlock);
    std::vector<int> bsz = {OB};
    if (IB < OB) bsz.push_back(IB);
    bsz.push_back(NB);
    auto laswp = [&](int p0, int cnt, int a0, int a1, int b0, int b1) {
      const int ncols = std::max(0, a1 - a0) + std::max(0, b1 - b0);
      if (ncols <= 0 || cnt <= 0) return;
      ProfScope pt(PROF_LU_TRSM, st);
      dim3 g((ncols + 255) / 256, L.nf);
      lu_laswp_kernel<T><<<g, 256, 0, st>>>(F, m, k, p0, cnt, L.piv, a0, std::max(a0, a1), b0,
                                            std::max(b0, b1));
      pt.done(0, 1, st);
    };
    // row band [r0, r1) x [c0, c1) solved with the unit lower block at [r0, r1): the
    // rows split in blocks of bsz[lev] (recursively down to 32-row solve steps), each
    // block's update of the rows below it of depth bsz[lev]
    std::function<void(int, int, int, int, int)> band = [&](int r0, int r1, int c0, int c1,
                                                            int lev) {
      if (c1 <= c0 || r1 <= r0) return;
      const int bs = bsz[lev];
      if (bs == NB) {
        for (int j0 = r0; j0 < r1; j0 += NB) {
          const int jb = std::min(NB, r1 - j0);
          {
            const int ncol = c1 - c0;
            const int tb = ((long)((ncol + 255) / 256) * L.nf >= 152) ? 256 : 64;
            dim3 gt((ncol + tb - 1) / tb, L.nf);
            ProfScope pt(PROF_LU_TRSM, st);
            lu_trsm_kernel<T><<<gt, tb, 0, st>>>(F, m, k, j0, jb, L.piv, c0, c1, 0);
            pt.done((double)ncol * jb * (jb - 1) * L.nf, 1, st);
          }
          const int base = j0 + jb;
          schur_update<T>(L, F, r1 - base, c1 - c0, jb, base + (long)j0 * m, j0 + (long)c0 * m,
                          base + (long)c0 * m, W, status, st);
        }
        return;
      }
      for (int B0 = r0; B0 < r1; B0 += bs) {
        const int B1 = std::min(r1, B0 + bs);
        band(B0, B1, c0, c1, lev + 1);
        schur_update<T>(L, F, r1 - B1, c1 - c0, B1 - B0, B1 + (long)B0 * m, B0 + (long)c0 * m,
                        B1 + (long)c0 * m, W, status, st);
      }
    };
    // LU of the columns [J, e) (rows J .. m) whose width is at most bsz[lev]: sub-blocks
    // of bsz[lev + 1] columns factored in turn (32-column panel steps at the bottom),
    // each followed by its interchanges on the block's other columns, the row band of
    // the block's columns to its right and their update of depth bsz[lev + 1]
    std::function<void(int, int, int)> block = [&](int J, int e, int lev) {
      const int bs = bsz[lev + 1];
      if (bs == NB) {
        for (int j0 = J; j0 < e; j0 += NB) {
          const int jb = std::min(NB, e - j0);
          panel_step<T>(L, F, j0, jb, J, e, ptol, status, W, st);
          const int base = j0 + jb;
          schur_update<T>(L, F, m - base, e - base, jb, base + (long)j0 * m, j0 + (long)base * m,
                          base + (long)base * m, W, status, st);
        }
        return;
      }
      for (int J1 = J; J1 < e; J1 += bs) {
        const int e2 = std::min(e, J1 + bs);
        block(J1, e2, lev + 1);
        laswp(J1, e2 - J1, J, J1, e2, e);
        if (e2 < e) {
          band(J1, e2, e2, e, lev + 2);
          schur_update<T>(L, F, m - e2, e - e2, e2 - J1, e2 + (long)J1 * m, J1 + (long)e2 * m,
                          e2 + (long)e2 * m, W, status, st);
        }
      }
    };
    for (int J0 = 0; J0 < k; J0 += OB) {
      const int e1 = std::min(k, J0 + OB);
      block(J0, e1, 0);
      laswp(J0, e1 - J0, 0, J0, e1, m);
      if (e1 < m) {
        band(J0, e1, e1, m, 1);
        schur_update<T>(L, F, m - e1, m - e1, e1 - J0, e1 + (long)J0 * m, J0 + (long)e1 * m,
                        e1 + (long)e1 * m, W, status, st);
      }
    }
  }
  lu_perm_kernel<<<(L.nf + 127) / 128, 128, 0, st>>>(L.piv, L.perm, L.k, L.nf);
  ProfScope pi(PROF_LU_TRINV, st);
  double bw = 0;
  if (L.inv) {
    invert_triangles<T>(L, (T*)W.inv, L.ib, st);
    const int Bz = L.ib < L.k ? L.ib : L.k;
    bw = (2.0 / 3.0) * (double)Bz * Bz * L.k * L.nf;
  } else {
    dim3 gd((L.k + kNB - 1) / kNB, L.nf);
    diag32_inplace_kernel<T><<<gd, kNB, 0, st>>>(F, L.m, L.k);
    bw = (2.0 / 3.0) * (double)kNB * kNB * L.k * L.nf;
  }
  pi.done(bw, 1, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t factor_level(int prec, int d, DevLevel& L, const DevLevel* child, const double* Qcat,
                         const double* Ccat, const double* q, double pivot_tol, int* status,
                         const FactorWork& W, cudaStream_t st) {
  if (prec == SP_PREC_FP32)
    return factor_level_t<float>(d, L, child, Qcat, Ccat, q, pivot_tol, status, W, st);
  return factor_level_t<double>(d, L, child, Qcat, Ccat, q, pivot_tol, status, W, st);
}

cudaError_t schur_update_raw(int prec, bool tc, bool split, int M, int N, int K, const void* A,
                             int lda, long sA, const void* B, int ldb, long sB, void* C, int ldc,
                             long sC, int batch, float* packA, float* packB, int* status,
                             cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (prec == SP_PREC_FP32 && tc)
    return tc_schur_update(M, N, K, (const float*)A, lda, sA, (const float*)B, ldb, sB, (float*)C,
                           ldc, sC, batch, packA, packB, split, status, st);
  if (prec == SP_PREC_FP32) {
    if (K <= kNB)
      gemm_sub<float>(M, N, K, (const float*)A, lda, sA, (const float*)B, ldb, sB, (float*)C, ldc,
                      sC, batch, st);
    else
      gemm_gen<float>(M, N, K, -1.f, true, (const float*)A, lda, sA, (const float*)B, ldb, sB,
                      (float*)C, ldc, sC, batch, 0, 0, st);
  } else {
    if (K <= kNB)
      gemm_sub<double>(M, N, K, (const double*)A, lda, sA, (const double*)B, ldb, sB, (double*)C,
                       ldc, sC, batch, st);
    else
      gemm_gen<double>(M, N, K, -1.0, true, (const double*)A, lda, sA, (const double*)B, ldb, sB,
                       (double*)C, ldc, sC, batch, 0, 0, st);
  }
  return cudaGetLastError();
}

int factor_outer_block(int prec, bool tc, int m, int k) {
  // the tensor-core form blocks the fronts whose trailing updates are large
  // enough to fill the GPU with 128 x 128 tiles
  if (prec == SP_PREC_FP32 && tc && m >= kTcMinFront && k > kNB) return kTcMaxK;
  return 0;
}

size_t invert_scratch_elems(int nf, int k, int ib) {
  return (size_t)nf * ((size_t)2 * k * (ib + 1) + (size_t)k * (ib / 2));
}

cudaError_t factor_copy16(DevLevel& L, cudaStream_t st) {
  if (!L.front16) return cudaSuccess;
  dim3 g((unsigned)((L.m + 7) / 8), L.nf);
  f16_copy_kernel<<<g, 256, 0, st>>>((const float*)L.front, L.m, L.k, (__half*)L.front16,
                                     L.fscale16);
  return cudaGetLastError();
}

size_t grid_panel_pub_words(int nf) {
  return (size_t)nf * std::max<size_t>((size_t)2 * kGridPanelMaxG * kPubWords, kCaluFrontWords);
}

bool factor_grid_panel(int prec, int m) {
  return prec == SP_PREC_FP32 ? panel_kind<float>(m) == 2 : panel_kind<double>(m) == 2;
}

int factor_panel_width(int prec, int m) {
  return prec == SP_PREC_FP32 ? panel_width<float>(m) : panel_width<double>(m);
}

}  // namespace sp
