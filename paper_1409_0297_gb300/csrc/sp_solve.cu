// Preconditioner application z = P^{-1} Q r (Section 2.2, "u <= P^{-1} Q g"):
//   1. the sparsifying stencil y_S = r_S - T_S r_beta(S) for every set instance
//      (Section 2.3, Q(S, gamma) = [I, -T_S]);
//   2. the forward sweep of the multifrontal factor, leaves to root: per front
//      y1 = L11^{-1} Pi b1 and the update b2 - L21 y1 handed to the parent;
//   3. the backward sweep, root to leaves: x1 = U11^{-1} (y1 - U12 x2).
// Levels with many fronts: one CTA per front, right-hand side in shared memory,
// triangular solves blocked by 32 (the inverse of each 32 x 32 diagonal block is
// formed at factor time; the block step is a 32 x 32 matrix-vector product, then
// all warps apply the block's columns with coalesced column reads of the
// column-major front).
// Levels with few fronts (the 512 x 512 diagonal blocks of L11, U11 replaced by
// their inverses at factor time): the sweep is a short chain of matrix-vector
// products (the diagonal blocks 16 rows per CTA; after each diagonal block the
// rows below (forward) or above (backward) take that column block's contribution,
// one row per thread), so the large upper fronts spread over the whole GPU.
// VT = double2 (FP64 form) or float2 (FP32 form).
#include <cooperative_groups.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kBS = 32;
constexpr size_t kVecSmem = 192 * 1024;  // largest vector staged in shared memory

template <class VT> struct Scalar;
template <> struct Scalar<double2> { using T = double; };
template <> struct Scalar<float2> { using T = float; };

// Factor entries as the sweeps compute with them: FP64 and FP32 fronts as stored, the
// FP16 copy (sp_opts.factor_storage = 1) widened to FP32; its power-of-two column
// scales multiply the vector entries as they are staged (exact), so
// sum_c A[r, c] v[c] = sum_c A16[r, c] (scale[c] v[c])
__device__ __forceinline__ double fac(double a) { return a; }
__device__ __forceinline__ float fac(float a) { return a; }
__device__ __forceinline__ float fac(__half a) { return __half2float(a); }
template <class VT> __device__ __forceinline__ VT vscale(VT v, const float* sc, long c) {
  if (sc) {
    const float s = sc[c];
    v.x *= s;
    v.y *= s;
  }
  return v;
}

template <class VT> __device__ __forceinline__ VT vzero();
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0, 0); }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0, 0); }

template <class VT> __device__ __forceinline__ VT from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }

template <class VT, class T>
__device__ __forceinline__ void axpy_neg(VT& acc, T a, VT x) {  // acc -= a * x
  acc.x = fma(-a, x.x, acc.x);
  acc.y = fma(-a, x.y, acc.y);
}
template <class VT, class T>
__device__ __forceinline__ void axpy(VT& acc, T a, VT x) {  // acc += a * x
  using C = decltype(acc.x);
  acc.x = fma((C)a, x.x, acc.x);
  acc.y = fma((C)a, x.y, acc.y);
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel's last CTAs drain; it waits
// here, before touching anything that kernel wrote (a no-op for ordinary launches).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// kernel<<<g, b, smem, st>>>(args) with programmatic stream serialisation when pdl
template <class... KArgs, class... Args>
void launch_k(bool pdl, void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t st,
              Args... args) {
  if (!pdl) {
    kern<<<g, b, smem, st>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// y[S instance] = self * r[S instance] - T_t r[B instance], B = beta (self = 1, set
// stencils) or gamma (self = 0, per-point stencils); one CTA per instance of type t
// (and per stacked vector, blockIdx.y, vectors N apart).  In a problem group of P
// problems vector v belongs to problem v % P, whose tables are t_stride apart.
template <class VT, class T>
__global__ void qapply_kernel(int d, int n, int nl, int nS, int nB, int self,
                              const int* __restrict__ Soff, const int* __restrict__ Boff,
                              const T* __restrict__ Tt, const double2* __restrict__ r, VT* y,
                              long N, int P, long t_stride) {
  pdl_wait();
  extern __shared__ unsigned char smraw[];
  VT* rb = reinterpret_cast<VT*>(smraw);
  r += blockIdx.y * N;
  y += blockIdx.y * N;
  Tt += (blockIdx.y % P) * t_stride;
  int box = blockIdx.x, o[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    o[a] = (box % nl) * (n / nl);
    box /= nl;
  }
  for (int c = threadIdx.x; c < nB; c += blockDim.x) {
    long g = 0, s = 1;
    for (int a = 0; a < d; ++a) {
      g += (long)wrapi(o[a] + Boff[c * d + a], n) * s;
      s *= n;
    }
    rb[c] = from_d2<VT>(r[g]);
  }
  __syncthreads();
  for (int a0 = threadIdx.x; a0 < nS; a0 += blockDim.x) {
    long g = 0, s = 1;
    for (int a = 0; a < d; ++a) {
      g += (long)wrapi(o[a] + Soff[a0 * d + a], n) * s;
      s *= n;
    }
    VT acc = self ? from_d2<VT>(r[g]) : VT{0, 0};
    for (int c = 0; c < nB; ++c) axpy_neg(acc, Tt[a0 + (long)c * nS], rb[c]);
    y[g] = acc;
  }
}

// The same product tiled over instances, so a chunk of T_t staged in shared memory
// serves kQIt instances at once (the kernel above re-reads the whole T_t from L2
// for every instance).  CTA (instance block, stacked vector, row tile): rows
// [z kQRt, z kQRt + kQRt) of S for kQIt consecutive instances; per 32-column chunk
// of B the CTA stages T_t(rows, chunk) and the gathered r(B chunk, instances) in
// shared memory (the next chunk's loads in flight meanwhile); each thread keeps 4 rows x
// 2 instances.  Every output is summed in
// the order of the kernel above (self term first, then the columns of B in order),
// so both give the same bits.
constexpr int kQRt = 64, kQIt = 32, kQK = 32;
// grid index of the point at offset off from an instance's origin o
__device__ __forceinline__ long q_addr(int d, int n, const int* o, const int* off) {
  long g = wrapi(o[0] + off[0], n);
  if (d > 1) g += (long)wrapi(o[1] + off[1], n) * n;
  if (d > 2) g += (long)wrapi(o[2] + off[2], n) * n * n;
  return g;
}
template <class VT, class T>
__global__ void __launch_bounds__(256) qgemm_kernel(int d, int n, int nl, int nS, int nB, int self,
                                                    const int* __restrict__ Soff,
                                                    const int* __restrict__ Boff,
                                                    const T* __restrict__ Tt,
                                                    const double2* __restrict__ r, VT* y, long N,
                                                    int P, long t_stride, long ninst) {
  pdl_wait();
  __shared__ T Ts[kQK][kQRt];
  __shared__ VT Rs[kQK][kQIt];
  __shared__ int org[kQIt][3];
  r += blockIdx.y * N;
  y += blockIdx.y * N;
  Tt += (blockIdx.y % P) * t_stride;
  const long i0 = (long)blockIdx.x * kQIt;
  const int row0 = blockIdx.z * kQRt;
  const int tid = threadIdx.x, ig = tid & 15, rg = tid >> 4;
  const int side = n / nl;
  if (tid < kQIt) {
    long box = i0 + tid;
    for (int a = 0; a < 3; ++a) {
      org[tid][a] = (a < d) ? (int)(box % nl) * side : 0;
      if (a < d) box /= nl;
    }
  }
  __syncthreads();
  VT acc[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int row = row0 + rg * 4 + q, ii = ig * 2 + j;
      acc[q][j] = VT{0, 0};
      if (self && row < nS && i0 + ii < ninst)
        acc[q][j] = from_d2<VT>(r[q_addr(d, n, org[ii], Soff + row * d)]);
    }
  // the next chunk's T entries and gathered r values are loaded into registers while
  // the current chunk is multiplied (each thread 8 of T, 4 of r)
  constexpr int kTe = kQK * kQRt / 256, kRe = kQK * kQIt / 256;
  T tpre[kTe];
  VT rpre[kRe];
  auto fetch = [&](int k0) {
    const int kc = min(kQK, nB - k0);
#pragma unroll
    for (int u = 0; u < kTe; ++u) {
      const int e = tid + 256 * u, rr = e % kQRt, kk = e / kQRt;
      tpre[u] = (row0 + rr < nS && kk < kc) ? Tt[(row0 + rr) + (long)(k0 + kk) * nS] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kRe; ++u) {
      const int e = tid + 256 * u, ii = e % kQIt, kk = e / kQIt;
      rpre[u] = (kk < kc && i0 + ii < ninst)
                    ? from_d2<VT>(r[q_addr(d, n, org[ii], Boff + (k0 + kk) * d)])
                    : VT{0, 0};
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < nB; k0 += kQK) {
    const int kc = min(kQK, nB - k0);
#pragma unroll
    for (int u = 0; u < kTe; ++u) {
      const int e = tid + 256 * u;
      Ts[e / kQRt][e % kQRt] = tpre[u];
    }
#pragma unroll
    for (int u = 0; u < kRe; ++u) {
      const int e = tid + 256 * u;
      Rs[e / kQIt][e % kQIt] = rpre[u];
    }
    __syncthreads();
    if (k0 + kQK < nB) fetch(k0 + kQK);
    for (int kk = 0; kk < kc; ++kk) {
      const VT r0 = Rs[kk][ig * 2], r1 = Rs[kk][ig * 2 + 1];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T t = Ts[kk][rg * 4 + q];
        axpy_neg(acc[q][0], t, r0);
        axpy_neg(acc[q][1], t, r1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int row = row0 + rg * 4 + q, ii = ig * 2 + j;
      if (row < nS && i0 + ii < ninst) y[q_addr(d, n, org[ii], Soff + row * d)] = acc[q][j];
    }
}

// Gathers the front's right-hand side: the stencil output at the eliminated
// unknowns plus the children's update vectors (one child position at a time, so
// no two threads add into one entry).  b: m entries of shared memory.
template <class VT>
__device__ void gather_rhs(int d, int f, int m, int k, int nb1, const int* __restrict__ gidx,
                           const VT* __restrict__ rhsQ, const VT* __restrict__ cupd, int mc,
                           int kc, const int* __restrict__ ea_map, VT* b) {
  for (int v = threadIdx.x; v < m; v += blockDim.x)
    b[v] = (v < k) ? rhsQ[gidx[(long)f * m + v]] : vzero<VT>();
  __syncthreads();
  if (cupd) {
    const int nbd = mc - kc;
    for (int dl = 0; dl < (1 << d); ++dl) {
      int ff = f, cid = 0, stride = 1;
      for (int a = 0; a < d; ++a) {
        int bc = ff % nb1;
        ff /= nb1;
        cid += (2 * bc + ((dl >> a) & 1)) * stride;
        stride *= 2 * nb1;
      }
      cid += ff * stride;  // problem ff of a group
      const VT* cu = cupd + (long)cid * nbd;
      const int* mp = ea_map + (long)dl * nbd;
      for (int i = threadIdx.x; i < nbd; i += blockDim.x) {
        VT v = cu[i];
        VT& t = b[mp[i]];
        t.x += v.x;
        t.y += v.y;
      }
      __syncthreads();
    }
  }
}

// Forward sweep of one level, one CTA per front.
template <class VT, class T>
__global__ void __launch_bounds__(256) forward_kernel(
    int d, const T* __restrict__ fronts, int m, int k, int nb1, const int* __restrict__ gidx,
    const int* __restrict__ perm, const VT* __restrict__ rhsQ, const VT* __restrict__ cupd, int mc,
    int kc, const int* __restrict__ ea_map, VT* upd, VT* yout, long N, long custr) {
  pdl_wait();
  extern __shared__ unsigned char smraw[];
  VT* b = reinterpret_cast<VT*>(smraw);  // m
  VT* b1 = b + m;                         // k (permuted eliminated part)
  __shared__ T Ld[kBS][kBS + 1];
  __shared__ VT yd[kBS];
  const int f = blockIdx.x;
  {  // stacked vector blockIdx.y
    const long v = blockIdx.y, nf = gridDim.x;
    rhsQ += v * N;
    if (cupd) cupd += v * custr;
    upd += v * nf * (m - k);
    yout += v * nf * k;
  }
  const T* A = fronts + (long)f * m * m;
  gather_rhs(d, f, m, k, nb1, gidx, rhsQ, cupd, mc, kc, ea_map, b);
  const int* pr = perm + (long)f * k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) b1[j] = b[pr[j]];
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) b[j] = b1[j];
  for (int jb = 0; jb < k; jb += kBS) {
    const int bs = min(kBS, k - jb);
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
      int i = e % bs, j = e / bs;
      Ld[i][j] = A[(jb + i) + (long)(jb + j) * m];
    }
    __syncthreads();
    // y_J = Linv_JJ b_J (the diagonal block holds the inverse, unit diagonal
    // implied): 8 threads per row, partial sums reduced with shuffles
    {
      const int i = threadIdx.x >> 3, cl = threadIdx.x & 7;
      VT acc = vzero<VT>();
      if (i < bs)
        for (int l = cl; l < i; l += 8) axpy(acc, Ld[i][l], b[jb + l]);
      for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, 8);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, 8);
      }
      if (cl == 0 && i < bs) {
        VT bi = b[jb + i];
        yd[i] = VT{bi.x + acc.x, bi.y + acc.y};
      }
      __syncthreads();
      if (threadIdx.x < bs) b[jb + threadIdx.x] = yd[threadIdx.x];
    }
    __syncthreads();
    for (int r = jb + bs + threadIdx.x; r < m; r += blockDim.x) {
      VT acc = b[r];
      const T* Ar = A + r + (long)jb * m;
      for (int j = 0; j < bs; ++j) axpy_neg(acc, __ldcs(Ar + (long)j * m), b[jb + j]);
      b[r] = acc;
    }
    __syncthreads();
  }
  for (int v = threadIdx.x; v < k; v += blockDim.x) yout[(long)f * k + v] = b[v];
  for (int v = threadIdx.x; v < m - k; v += blockDim.x) upd[(long)f * (m - k) + v] = b[k + v];
}

// Backward sweep of one level, one CTA per front.  x: the global solution.
template <class VT, class T>
__global__ void __launch_bounds__(256) backward_kernel(const T* __restrict__ fronts, int m, int k,
                                                        const int* __restrict__ gidx,
                                                        const VT* __restrict__ yin, double2* x,
                                                        long N) {
  pdl_wait();
  extern __shared__ unsigned char smraw[];
  VT* xb = reinterpret_cast<VT*>(smraw);  // m: x1 then x2
  yin += (long)blockIdx.y * gridDim.x * k;
  x += blockIdx.y * N;
  __shared__ T Ud[kBS][kBS + 1];
  __shared__ VT xd[kBS];
  const int f = blockIdx.x;
  const T* A = fronts + (long)f * m * m;
  const int* gi = gidx + (long)f * m;
  for (int v = k + threadIdx.x; v < m; v += blockDim.x) xb[v] = from_d2<VT>(x[gi[v]]);
  __syncthreads();
  // rhs = y1 - U12 x2
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    VT acc = yin[(long)f * k + i];
    for (int c = k; c < m; ++c) axpy_neg(acc, __ldcs(A + i + (long)c * m), xb[c]);
    xb[i] = acc;
  }
  __syncthreads();
  const int nblk = (k + kBS - 1) / kBS;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int jb = bi * kBS;
    const int bs = min(kBS, k - jb);
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
      int i = e % bs, j = e / bs;
      Ud[i][j] = A[(jb + i) + (long)(jb + j) * m];
    }
    __syncthreads();
    // x_J = Uinv_JJ t_J (the diagonal block holds the inverse, upper part with
    // the diagonal)
    {
      const int i = threadIdx.x >> 3, cl = threadIdx.x & 7;
      VT acc = vzero<VT>();
      if (i < bs)
        for (int l = i + cl; l < bs; l += 8) axpy(acc, Ud[i][l], xb[jb + l]);
      for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o, 8);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o, 8);
      }
      if (cl == 0 && i < bs) xd[i] = acc;
      __syncthreads();
      if (threadIdx.x < bs) xb[jb + threadIdx.x] = xd[threadIdx.x];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < jb; r += blockDim.x) {
      VT acc = xb[r];
      const T* Ar = A + r + (long)jb * m;
      for (int j = 0; j < bs; ++j) axpy_neg(acc, __ldcs(Ar + (long)j * m), xb[jb + j]);
      xb[r] = acc;
    }
    __syncthreads();
  }
  for (int v = threadIdx.x; v < k; v += blockDim.x) x[gi[v]] = to_d2(xb[v]);
}

// ---- sweeps of levels whose L11, U11 hold their inverses -------------------------
// tmp (m per front): Pi b1 (k entries) then b2 (m - k entries).
template <class VT>
__global__ void __launch_bounds__(256) inv_gather_kernel(
    int d, int m, int k, int nb1, const int* __restrict__ gidx, const int* __restrict__ perm,
    const VT* __restrict__ rhsQ, const VT* __restrict__ cupd, int mc, int kc,
    const int* __restrict__ ea_map, VT* tmp, long N, long custr) {
  pdl_wait();
  extern __shared__ unsigned char smraw[];
  VT* b = reinterpret_cast<VT*>(smraw);
  const int f = blockIdx.x;
  rhsQ += blockIdx.y * N;
  if (cupd) cupd += blockIdx.y * custr;
  tmp += (long)blockIdx.y * gridDim.x * m;
  gather_rhs(d, f, m, k, nb1, gidx, rhsQ, cupd, mc, kc, ea_map, b);
  const int* pr = perm + (long)f * k;
  VT* t = tmp + (long)f * m;
  for (int j = threadIdx.x; j < k; j += blockDim.x) t[j] = b[pr[j]];
  for (int j = k + threadIdx.x; j < m; j += blockDim.x) t[j] = b[j];
}

// The same for fronts whose right-hand side does not fit in shared memory: the
// front's work vector tmp is assembled in place in global memory, the eliminated
// part permuted through the forward-result buffer y (free at this point).
template <class VT>
__global__ void __launch_bounds__(1024) inv_gather_global_kernel(
    int d, int m, int k, int nb1, const int* __restrict__ gidx, const int* __restrict__ perm,
    const VT* __restrict__ rhsQ, const VT* __restrict__ cupd, int mc, int kc,
    const int* __restrict__ ea_map, VT* tmp, VT* ybuf, long N, long custr) {
  pdl_wait();
  const int f = blockIdx.x;
  rhsQ += blockIdx.y * N;
  if (cupd) cupd += blockIdx.y * custr;
  tmp += (long)blockIdx.y * gridDim.x * m;
  ybuf += (long)blockIdx.y * gridDim.x * k;
  VT* t = tmp + (long)f * m;
  for (int v = threadIdx.x; v < m; v += blockDim.x)
    t[v] = (v < k) ? rhsQ[gidx[(long)f * m + v]] : vzero<VT>();
  __syncthreads();
  if (cupd) {
    const int nbd = mc - kc;
    for (int dl = 0; dl < (1 << d); ++dl) {
      int ff = f, cid = 0, stride = 1;
      for (int a = 0; a < d; ++a) {
        int bc = ff % nb1;
        ff /= nb1;
        cid += (2 * bc + ((dl >> a) & 1)) * stride;
        stride *= 2 * nb1;
      }
      cid += ff * stride;  // problem ff of a group
      const VT* cu = cupd + (long)cid * nbd;
      const int* mp = ea_map + (long)dl * nbd;
      for (int i = threadIdx.x; i < nbd; i += blockDim.x) {
        VT v = cu[i];
        VT& tt = t[mp[i]];
        tt.x += v.x;
        tt.y += v.y;
      }
      __syncthreads();
    }
  }
  const int* pr = perm + (long)f * k;
  VT* y = ybuf + (long)f * k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) y[j] = t[pr[j]];
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) t[j] = y[j];
}

// Diagonal-block products of the levels whose diagonal blocks (size L.ib) hold
// the inverses of those of L11 / U11; [j0, j1) is the block.
//   mode 0 (forward):  y[r] = tmp[r] + sum_{j0<=c<r} Linv[r,c] tmp[c]
//   mode 3 (backward): y[r] = x[r] = sum_{r<=c<j1} Uinv[r,c] tmp[c]
// (in the backward sweep y holds x1).  RB rows per CTA, 256 / RB column lanes per
// row, partial sums reduced in shared memory in a fixed order; the off-diagonal
// products go through gemv_kernel below.
template <class VT, class T, int RB>
__global__ void __launch_bounds__(256) inv_gemv_kernel(int mode, const T* __restrict__ fronts,
                                                        int m, int k, int j0, int j1,
                                                        const int* __restrict__ gidx, VT* tmp,
                                                        VT* y, double2* x, long N,
                                                        const float* __restrict__ fsc, int lda) {
  pdl_wait();
  extern __shared__ unsigned char smraw[];
  VT* v = reinterpret_cast<VT*>(smraw);  // tmp[j0 .. j1)
  {  // stacked vector blockIdx.z
    const long vz = blockIdx.z, nf = gridDim.y;
    tmp += vz * nf * m;
    y += vz * nf * k;
    if (x) x += vz * N;
  }
  constexpr int CL = 256 / RB;  // column lanes per row
  __shared__ VT red[CL][RB + 1];
  const int f = blockIdx.y;
  const T* A = fronts + (long)f * m * lda;  // columns lda apart (m, or the FP16 copy's even m)
  VT* tf = tmp + (long)f * m;
  VT* yf = y + (long)f * k;
  const float* sc = fsc ? fsc + (long)f * m : nullptr;  // column scales of the FP16 copy
  for (int c = j0 + threadIdx.x; c < j1; c += blockDim.x) v[c - j0] = vscale(tf[c], sc, c);
  __syncthreads();
  const int tx = threadIdx.x % RB, ty = threadIdx.x / RB;
  const int r0 = j0 + blockIdx.x * RB;
  const int r = r0 + tx;
  // column range of the row block: the lower triangle up to the block's last row
  // (mode 0) or the upper triangle from its first row (mode 3)
  const int cb = (mode == 0) ? j0 : max(r0, j0);
  const int ce = (mode == 0) ? min(r0 + RB, j1) : j1;
  VT acc = vzero<VT>();
  if (r < j1) {
#pragma unroll 4
    for (int c = cb + ty; c < ce; c += CL) {
      const bool use = (mode == 0) ? (c < r) : (c >= r);
      if (use) axpy(acc, fac(A[r + (long)c * lda]), v[c - j0]);
    }
  }
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && r < j1) {
    VT s = red[0][tx];
    for (int l = 1; l < CL; ++l) {
      s.x += red[l][tx].x;
      s.y += red[l][tx].y;
    }
    if (mode == 0) {
      const VT o = tf[r];
      yf[r] = VT{o.x + s.x, o.y + s.y};
    } else {
      yf[r] = s;
      x[gidx[(long)f * m + r]] = to_d2(s);
    }
  }
}

// Off-diagonal products of the sweeps for fronts of any size,
//   out[r] op= sum_{c in [vlo, vhi)} A[r, c] v[c],   r in [rlo, rhi),
// with v = y (vsrc 0) or x at the front's grid points (vsrc 1), and
//   op 0: tmp[r] -= s   op 1: upd[r - k] = tmp[r] - s   op 2: tmp[r] = y[r] - s.
// One thread per row, 256 rows per CTA (a warp reads 128 contiguous bytes of a
// column of the column-major front), v staged in shared memory in chunks of
// 1024, the column range split over gridDim.y when the rows alone would leave
// the GPU idle.  With one split the kernel applies op itself; with several it
// writes partial sums part[(split nf + f) rows + (r - rlo)], which
// gemv_finish_kernel adds in split order (the result does not depend on timing).
struct GemvArgs {
  int rlo, rhi, vlo, vhi, vsrc, op;
};
template <class VT>
__device__ __forceinline__ void gemv_out(int op, int m, int k, int r, VT s, VT* tf, const VT* yf,
                                         VT* upd, int f) {
  if (op == 1) {
    VT o = tf[r];
    upd[(long)f * (m - k) + (r - k)] = VT{o.x - s.x, o.y - s.y};
  } else if (op == 2) {
    VT o = yf[r];
    tf[r] = VT{o.x - s.x, o.y - s.y};
  } else {
    VT o = tf[r];
    tf[r] = VT{o.x - s.x, o.y - s.y};
  }
}
// NV: vectors per thread (compile-time bound; nv <= NV run), stacked vector-major
// (level work vectors nf m / nf k / nf (m - k) apart, global ones N apart).  Each
// vector is summed in the same order for every NV, so stacking vectors never
// changes a result.
template <class VT, class T, int NV>
__global__ void __launch_bounds__(256) gemv_kernel(GemvArgs ga, const T* __restrict__ fronts,
                                                    int m, int k, const int* __restrict__ gidx,
                                                    VT* tmp, VT* y, VT* upd, const double2* x,
                                                    int nsplit, VT* part, int nv, long N,
                                                    const float* __restrict__ fsc) {
  pdl_wait();
  constexpr int CH = 1024 / NV;  // columns of one staged chunk
  __shared__ VT vs[CH * NV];     // vs[j NV + v]
  const int f = blockIdx.z, sp = blockIdx.y, nf = gridDim.z;
  const T* A = fronts + (long)f * m * m;
  const float* sc = fsc ? fsc + (long)f * m : nullptr;  // column scales of the FP16 copy
  const long tstr = (long)nf * m, ystr = (long)nf * k, ustr = (long)nf * (m - k);
  const int r = ga.rlo + blockIdx.x * 256 + threadIdx.x;
  const int per = (ga.vhi - ga.vlo + nsplit - 1) / nsplit;
  const int cb = ga.vlo + sp * per, ce = min(ga.vhi, cb + per);
  VT acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = vzero<VT>();
  for (int c0 = cb; c0 < ce; c0 += CH) {
    const int cn = min(CH, ce - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn * nv; i += 256) {
      const int j = i / nv, v = i - j * nv;
      vs[j * NV + v] = vscale(ga.vsrc ? from_d2<VT>(x[v * N + gidx[(long)f * m + c0 + j]])
                                      : y[v * ystr + (long)f * k + c0 + j],
                              sc, c0 + j);
    }
    __syncthreads();
    if (r < ga.rhi) {
      const T* Ar = A + r + (long)c0 * m;
      int j = 0;
      // 8 column loads in flight per thread: a launch costs (columns of a split) / 8
      // memory latencies at least (16 was measured slower on the large 3D launches)
      for (; j + 8 <= cn; j += 8) {
        decltype(fac(T())) a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fac(Ar[(long)(j + u) * m]);
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < NV; ++v)
            if (v < nv) axpy(acc[v], a[u], vs[(j + u) * NV + v]);
      }
      for (; j < cn; ++j) {
        const auto a = fac(Ar[(long)j * m]);
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v < nv) axpy(acc[v], a, vs[j * NV + v]);
      }
    }
  }
  if (r >= ga.rhi) return;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v >= nv) break;
    if (nsplit == 1)
      gemv_out(ga.op, m, k, r, acc[v], tmp + v * tstr + (long)f * m, y + v * ystr + (long)f * k,
               upd + v * ustr, f);
    else
      part[(((long)sp * nv + v) * nf + f) * (ga.rhi - ga.rlo) + (r - ga.rlo)] = acc[v];
  }
}
// gemv_kernel on the FP16 copy of the factor (columns ld16 = m rounded up to even
// apart): each thread owns a pair of rows (r0, r0 + 1), r0 even, and reads both with
// one half2 load, so a warp still moves 128 contiguous bytes of a column per load;
// the column scales multiply the staged vector entries.
template <class VT, int NV>
__global__ void __launch_bounds__(256) gemv16_kernel(GemvArgs ga, const __half* __restrict__ fronts,
                                                     int m, int ld16, int k,
                                                     const int* __restrict__ gidx, VT* tmp, VT* y,
                                                     VT* upd, const double2* x, int nsplit, VT* part,
                                                     int nv, long N, const float* __restrict__ fsc) {
  pdl_wait();
  constexpr int CH = 1024 / NV;
  __shared__ VT vs[CH * NV];
  const int f = blockIdx.z, sp = blockIdx.y, nf = gridDim.z;
  const __half* A = fronts + (long)f * m * ld16;
  const float* sc = fsc + (long)f * m;
  const long tstr = (long)nf * m, ystr = (long)nf * k, ustr = (long)nf * (m - k);
  const int r0 = (ga.rlo & ~1) + 2 * (blockIdx.x * 256 + threadIdx.x);
  const int per = (ga.vhi - ga.vlo + nsplit - 1) / nsplit;
  const int cb = ga.vlo + sp * per, ce = min(ga.vhi, cb + per);
  VT acc0[NV], acc1[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc0[v] = acc1[v] = vzero<VT>();
  const bool live = r0 < ga.rhi;
  for (int c0 = cb; c0 < ce; c0 += CH) {
    const int cn = min(CH, ce - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cn * nv; i += 256) {
      const int j = i / nv, v = i - j * nv;
      vs[j * NV + v] = vscale(ga.vsrc ? from_d2<VT>(x[v * N + gidx[(long)f * m + c0 + j]])
                                      : y[v * ystr + (long)f * k + c0 + j],
                              sc, c0 + j);
    }
    __syncthreads();
    if (live) {
      const __half2* Ar = reinterpret_cast<const __half2*>(A + r0 + (long)c0 * ld16);
      const long cs = ld16 / 2;  // column stride in half2
      int j = 0;
      for (; j + 8 <= cn; j += 8) {
        __half2 h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) h[u] = Ar[(long)(j + u) * cs];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float2 a = __half22float2(h[u]);
#pragma unroll
          for (int v = 0; v < NV; ++v)
            if (v < nv) {
              axpy(acc0[v], a.x, vs[(j + u) * NV + v]);
              axpy(acc1[v], a.y, vs[(j + u) * NV + v]);
            }
        }
      }
      for (; j < cn; ++j) {
        const float2 a = __half22float2(Ar[(long)j * cs]);
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v < nv) {
            axpy(acc0[v], a.x, vs[j * NV + v]);
            axpy(acc1[v], a.y, vs[j * NV + v]);
          }
      }
    }
  }
  if (!live) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = r0 + h;
    if (r < ga.rlo || r >= ga.rhi) continue;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (v >= nv) break;
      const VT a = h ? acc1[v] : acc0[v];
      if (nsplit == 1)
        gemv_out(ga.op, m, k, r, a, tmp + v * tstr + (long)f * m, y + v * ystr + (long)f * k,
                 upd + v * ustr, f);
      else
        part[(((long)sp * nv + v) * nf + f) * (ga.rhi - ga.rlo) + (r - ga.rlo)] = a;
    }
  }
}

template <class VT>
__global__ void gemv_finish_kernel(GemvArgs ga, int m, int k, VT* tmp, VT* y, VT* upd, int nsplit,
                                   const VT* __restrict__ part) {
  pdl_wait();
  const int f = blockIdx.y, nf = gridDim.y, v = blockIdx.z, nv = gridDim.z;
  const int r = ga.rlo + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ga.rhi) return;
  VT s = vzero<VT>();
  for (int sp = 0; sp < nsplit; ++sp) {
    const VT p = part[(((long)sp * nv + v) * nf + f) * (ga.rhi - ga.rlo) + (r - ga.rlo)];
    s.x += p.x;
    s.y += p.y;
  }
  gemv_out(ga.op, m, k, r, s, tmp + (long)v * nf * m + (long)f * m,
           y + (long)v * nf * k + (long)f * k, upd + (long)v * nf * (m - k), f);
}

template <class VT>
cudaError_t q_apply_t(int d, int n, int nl, const std::vector<QTypeDev>& types, const void* Tt,
                      const double2* r, VT* y, int nv, long N, cudaStream_t st, bool pdl, int P,
                      long t_stride) {
  using T = typename Scalar<VT>::T;
  long ninst = 1;
  for (int a = 0; a < d; ++a) ninst *= nl;
  ProfScope ps(PROF_QAPPLY, st);
  double bytes = 0;
  for (const auto& ty : types) {
    size_t smem = sizeof(VT) * (ty.na > 0 ? ty.na : 1);
    // the tiled product for the large FP32 tables (cells; faces in 3D), where the
    // per-instance kernel's re-reads of T_t from L2 dominate; FP64 products are bound
    // by the FP64 pipe either way and small tables stay in L1 (both kernels give the
    // same bits)
    if (sizeof(T) == sizeof(float) && ninst >= kQIt && ty.nS >= kQRt / 2) {
      dim3 g((unsigned)((ninst + kQIt - 1) / kQIt), nv * P, (unsigned)((ty.nS + kQRt - 1) / kQRt));
      launch_k(pdl, qgemm_kernel<VT, T>, dim3(g), dim3(256), 0, st, d, n, nl, ty.nS, ty.na,
               ty.self, ty.S, ty.A, (const T*)Tt + ty.t_off, r, y, N, P, t_stride, ninst);
    } else {
      dim3 g((unsigned)ninst, nv * P);
      launch_k(pdl, qapply_kernel<VT, T>, dim3(g), dim3(128), smem, st, d, n, nl, ty.nS, ty.na,
               ty.self, ty.S, ty.A, (const T*)Tt + ty.t_off, r, y, N, P, t_stride);
    }
    bytes += (double)ninst * nv * P * ty.nS * (sizeof(double2) + sizeof(VT)) +
             sizeof(T) * ty.nS * ty.na;
  }
  ps.done(bytes, (int)types.size(), st);
  return cudaGetLastError();
}

size_t sweep_smem(int m, int k, size_t vt) { return vt * (size_t)(m + k); }

template <class VT, class T>
void set_attrs() {
  cudaFuncSetAttribute(forward_kernel<VT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(backward_kernel<VT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(inv_gather_kernel<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(inv_gemv_kernel<VT, T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(inv_gemv_kernel<VT, T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(inv_gemv_kernel<VT, __half, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(inv_gemv_kernel<VT, __half, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

constexpr int kGemvTarget = 1216;  // CTAs a row-parallel product aims for (8 per SM)
constexpr int kMaxVec = 8;         // stacked vectors of one sweep launch

// Column splits of one row-parallel product: enough CTAs that the active rows fill
// kGemvTarget CTAs of 256 (a CTA of a 64-row front holds 64 active threads, so such
// fronts split 4 times as far), at least 32 columns per split.  Whenever it splits,
// splits x fronts x rows stays below 2 kGemvTarget 256 (sweep_partial_bytes).
int gemv_splits(int rows, int cols, int nf) {
  const long rpt = std::min(256, rows);
  const long tiles = (long)((rows + 255) / 256) * nf;
  if (cols < 64) return 1;
  const long want = ((long)kGemvTarget * 256 + rpt * tiles - 1) / (rpt * tiles);
  return (int)std::max<long>(1, std::min<long>(want, cols / 32));
}

// One off-diagonal product (gemv_kernel, + gemv_finish_kernel when split) for nv
// stacked vectors.
// The factor comes from the level's FP16 copy when it has one (T = __half, scaled
// per front), else from the fronts.
template <class VT, class T>
int gemv(const GemvArgs& ga, DevLevel& L, const double2* x, void* part, int nv, long N,
         cudaStream_t st) {
  const T* fr = (const T*)L.front;
  const int rows = ga.rhi - ga.rlo, cols = ga.vhi - ga.vlo;
  if (rows <= 0) return 0;
  int ns = cols > 0 ? gemv_splits(rows, cols, L.nf) : 1;
  if (!part) ns = 1;
  dim3 g((rows + 255) / 256, ns, L.nf);
  if (L.front16) {  // row pairs from the FP16 copy
    const int ld16 = (L.m + 1) & ~1;
    const int pairs = ((ga.rhi + 1) >> 1) - (ga.rlo >> 1);
    // a thread's column walk is a chain of memory latencies: as many CTAs as the FP32
    // form launches, so twice the column splits, within the partial-sum buffer's
    // bound (splits x fronts x rows <= 2 kGemvTarget 256)
    if (part && cols > 0) {
      const long cap = std::max<long>(1, (2L * kGemvTarget * 256) / ((long)L.nf * rows));
      ns = (int)std::min<long>(gemv_splits(pairs, cols, L.nf), cap);
    }
    dim3 g16((pairs + 255) / 256, ns, L.nf);
    if (nv == 1)
      launch_k(L.pdl != 0, gemv16_kernel<VT, 1>, dim3(g16), dim3(256), 0, st, ga,
               (const __half*)L.front16, L.m, ld16, L.k, L.gidx, (VT*)L.tmp, (VT*)L.y, (VT*)L.upd,
               x, ns, (VT*)part, 1, N, (const float*)L.fscale16);
    else
      launch_k(L.pdl != 0, gemv16_kernel<VT, kMaxVec>, dim3(g16), dim3(256), 0, st, ga,
               (const __half*)L.front16, L.m, ld16, L.k, L.gidx, (VT*)L.tmp, (VT*)L.y, (VT*)L.upd,
               x, ns, (VT*)part, nv, N, (const float*)L.fscale16);
  } else if (nv == 1)
    launch_k(L.pdl != 0, gemv_kernel<VT, T, 1>, dim3(g), dim3(256), 0, st, ga, fr, L.m, L.k,
             L.gidx, (VT*)L.tmp, (VT*)L.y, (VT*)L.upd, x, ns, (VT*)part, 1, N,
             (const float*)nullptr);
  else
    launch_k(L.pdl != 0, gemv_kernel<VT, T, kMaxVec>, dim3(g), dim3(256), 0, st, ga, fr, L.m, L.k,
             L.gidx, (VT*)L.tmp, (VT*)L.y, (VT*)L.upd, x, ns, (VT*)part, nv, N,
             (const float*)nullptr);
  if (ns == 1) return 1;
  dim3 gf((rows + 255) / 256, L.nf, nv);
  launch_k(L.pdl != 0, gemv_finish_kernel<VT>, dim3(gf), dim3(256), 0, st, ga, L.m, L.k, (VT*)L.tmp, (VT*)L.y, (VT*)L.upd, ns,
                                             (const VT*)part);
  return 2;
}

// One inv_gemv launch over rows [rlo, rhi) of every front and stacked vector: 16
// rows per CTA, or 4 rows per CTA (64 column lanes) when that leaves fewer CTAs
// than SMs.
template <class VT, class T>
void inv_gemv(int mode, DevLevel& L, int j0, int j1, int rlo, int rhi, size_t smem, double2* x,
              int nv, long N, cudaStream_t st) {
  const T* fr = (const T*)(L.front16 ? L.front16 : L.front);
  const float* fsc = L.front16 ? L.fscale16 : nullptr;
  const int lda = L.front16 ? ((L.m + 1) & ~1) : L.m;
  const int rows = rhi - rlo;
  if ((long)((rows + 15) / 16) * L.nf >= 152) {
    dim3 g((rows + 15) / 16, L.nf, nv);
    launch_k(L.pdl != 0, inv_gemv_kernel<VT, T, 16>, dim3(g), dim3(256), smem, st, mode, fr, L.m,
             L.k, j0, j1, L.gidx, (VT*)L.tmp, (VT*)L.y, x, N, fsc, lda);
  } else {
    dim3 g((rows + 3) / 4, L.nf, nv);
    launch_k(L.pdl != 0, inv_gemv_kernel<VT, T, 4>, dim3(g), dim3(256), smem, st, mode, fr, L.m,
             L.k, j0, j1, L.gidx, (VT*)L.tmp, (VT*)L.y, x, N, fsc, lda);
  }
}

template <class VT>
cudaError_t fused_level(bool fwd, int d, DevLevel& L, const DevLevel* child, const void* rhsQ,
                        double2* x, int nv, long N, cudaStream_t st);

template <class VT>
cudaError_t forward_t(int d, DevLevel& L, const DevLevel* child, const void* rhsQ, void* part,
                      int nv, long N, cudaStream_t st) {
  using T = typename Scalar<VT>::T;
  static bool attr = false;
  if (!attr) {
    set_attrs<VT, T>();
    attr = true;
  }
  if (nv < 1 || nv > kMaxVec) return cudaErrorInvalidValue;
  const double kk = L.k, mk = L.m - L.k;
  ProfScope ps(PROF_FORWARD, st);
  const VT* cup = child ? (const VT*)child->upd : nullptr;
  const long custr = child ? (long)child->nf * (child->m - child->k) : 0;
  int launches = 1;
  if (L.fused_c > 0) {
    cudaError_t e = fused_level<VT>(true, d, L, child, rhsQ, nullptr, nv, N, st);
    if (e != cudaSuccess) return e;
  } else if (!L.inv) {
    dim3 g(L.nf, nv);
    launch_k(L.pdl != 0, forward_kernel<VT, T>, dim3(g), dim3(256), sweep_smem(L.m, L.k, sizeof(VT)), st,
        d, (const T*)L.front, L.m, L.k, L.nb1, L.gidx, L.perm, (const VT*)rhsQ, cup, L.mc, L.kc,
        L.ea_map, (VT*)L.upd, (VT*)L.y, N, custr);
  } else {
    dim3 g(L.nf, nv);
    if (sizeof(VT) * (size_t)L.m <= kVecSmem)
      launch_k(L.pdl != 0, inv_gather_kernel<VT>, dim3(g), dim3(256), sizeof(VT) * L.m, st, 
          d, L.m, L.k, L.nb1, L.gidx, L.perm, (const VT*)rhsQ, cup, L.mc, L.kc, L.ea_map,
          (VT*)L.tmp, N, custr);
    else
      launch_k(L.pdl != 0, inv_gather_global_kernel<VT>, dim3(g), dim3(1024), 0, st, d, L.m, L.k, L.nb1, L.gidx, L.perm,
                                                        (const VT*)rhsQ, cup, L.mc, L.kc,
                                                        L.ea_map, (VT*)L.tmp, (VT*)L.y, N,
                                                        custr);
    launches = 1;
    // right-looking: after the diagonal block [j0, j1) of y, the rows below take
    // that column block's contribution; the last block's rows are those of L21,
    // which hand their result to the parent as the update vector
    for (int j0 = 0; j0 < L.k; j0 += L.ib) {
      const int j1 = min(L.k, j0 + L.ib);
      if (L.front16)
        inv_gemv<VT, __half>(0, L, j0, j1, j0, j1, sizeof(VT) * (j1 - j0), nullptr, nv, N, st);
      else
        inv_gemv<VT, T>(0, L, j0, j1, j0, j1, sizeof(VT) * (j1 - j0), nullptr, nv, N, st);
      ++launches;
      if (j1 < L.m) {
        const GemvArgs ga{j1, L.m, j0, j1, 0, j1 == L.k ? 1 : 0};
        launches += gemv<VT, T>(ga, L, nullptr, part, nv, N, st);
      }
    }
  }
  ps.done(L.nf * (L.front16 ? 2.0 : (double)sizeof(T)) * (kk * (kk - 1) / 2 + mk * kk), launches,
          st);
  return cudaGetLastError();
}

template <class VT>
cudaError_t backward_t(DevLevel& L, double2* x, void* part, int nv, long N, cudaStream_t st) {
  using T = typename Scalar<VT>::T;
  if (nv < 1 || nv > kMaxVec) return cudaErrorInvalidValue;
  const double kk = L.k, mk = L.m - L.k;
  ProfScope ps(PROF_BACKWARD, st);
  int launches = 1;
  if (L.fused_c > 0) {
    cudaError_t e = fused_level<VT>(false, 0, L, nullptr, nullptr, x, nv, N, st);
    if (e != cudaSuccess) return e;
  } else if (!L.inv) {
    dim3 g(L.nf, nv);
    launch_k(L.pdl != 0, backward_kernel<VT, T>, dim3(g), dim3(256), sizeof(VT) * (size_t)L.m, st, 
        (const T*)L.front, L.m, L.k, L.gidx, (const VT*)L.y, x, N);
  } else {
    launches = 0;
    if (L.m > L.k) {
      const GemvArgs ga{0, L.k, L.k, L.m, 1, 2};  // t = y1 - U12 x2
      launches += gemv<VT, T>(ga, L, x, part, nv, N, st);
    } else {
      // root: t = y1 (the stacked vectors' fronts are consecutive rows of both)
      cudaMemcpy2DAsync(L.tmp, sizeof(VT) * L.m, L.y, sizeof(VT) * L.k, sizeof(VT) * L.k,
                        (size_t)L.nf * nv, cudaMemcpyDeviceToDevice, st);
    }
    // right-looking: after the diagonal block [j0, j1) of x1, the rows above take
    // that column block's contribution
    const int nbk = (L.k + L.ib - 1) / L.ib;
    for (int bi = nbk - 1; bi >= 0; --bi) {
      const int j0 = bi * L.ib, j1 = min(L.k, j0 + L.ib);
      if (L.front16)
        inv_gemv<VT, __half>(3, L, j0, j1, j0, j1, sizeof(VT) * (j1 - j0), x, nv, N, st);
      else
        inv_gemv<VT, T>(3, L, j0, j1, j0, j1, sizeof(VT) * (j1 - j0), x, nv, N, st);
      ++launches;
      if (j0 > 0) {
        const GemvArgs ga{0, j0, j0, j1, 0, 0};
        launches += gemv<VT, T>(ga, L, x, part, nv, N, st);
      }
    }
  }
  ps.done(L.nf * (L.front16 ? 2.0 : (double)sizeof(T)) * (kk * (kk + 1) / 2 + mk * kk), launches,
          st);
  return cudaGetLastError();
}


// ---- fused sweeps of the inverse-form levels -------------------------------------
// One launch per level and direction instead of a chain of gather / diagonal-block /
// row-product launches: a thread-block cluster of C CTAs per front (C = 1 on levels
// with many fronts) holds the front's work vectors in shared memory and walks the
// diagonal blocks itself.  Rows are owned in slabs of 32 (slab s by cluster rank
// s mod C); a warp reads 32 consecutive rows of a column of the column-major front
// (one 128-byte line in FP32).  A result that other CTAs of the cluster need (the
// forward y of a diagonal block, the next block's right-hand side, the backward x)
// is written into every CTA's copy through distributed shared memory before a
// cluster barrier.  Every CTA runs the same sequence of barriers (the loop bounds
// depend only on k, m and the block size), and each vector is summed in an order
// that does not depend on how many vectors share the launch.
namespace cg = cooperative_groups;

struct FusedArgs {
  int d, m, k, ib, nb1, mc, kc, nv;
  int stream;  // factor loads with the evict-first hint (a level larger than a quarter of L2)
  const void* front;
  const int* gidx;
  const int* perm;
  const int* ea_map;
  const void* rhsQ;   // forward: stencil output (N per vector)
  const void* cupd;   // forward: child update vectors (custr per vector)
  void* upd;          // forward: nf (m - k) per vector
  void* y;            // forward output / backward input: nf k per vector
  double2* x;         // backward: global solution (N per vector)
  long N, custr;
};

template <int NT>
struct FusedShape {
  static constexpr int W = NT / 32;
};

// dst[v ld + i] = val on this CTA and, with C > 1, on every other CTA of the cluster
template <class VT>
__device__ __forceinline__ void bcast(VT* dst, VT val, int C, cg::cluster_group& cl) {
  if (C == 1) {
    *dst = val;
    return;
  }
  for (int q = 0; q < C; ++q) *cl.map_shared_rank(dst, q) = val;
}

__device__ __forceinline__ void csync(int C, cg::cluster_group& cl) {
  if (C == 1)
    __syncthreads();
  else
    cl.sync();
}

// Row products of the rows [r0, r1) owned by this CTA against columns [c0, c1):
//   s_v(r) = sum_c A[r + c m] src[v ls + c]      (mask 0: every column,
//   mask 1: c < r only, mask 2: c >= r only), then epi(r, v, s_v(r)).
// Owned slabs are spread over the warps; when they are fewer than the warps, the
// columns of each slab are split over several warps and the partial sums added in
// split order through shared memory (red: W x 32 x NV).  Every thread of the CTA
// must call this (it contains __syncthreads).
template <class T>
__device__ __forceinline__ T ld_front(const T* p, bool stream) {
  return stream ? __ldcs(p) : *p;  // streaming (evict-first) for the large leaf level
}

template <class VT, class T, int NT, int NV, class Epi>
__device__ void rows_times(const T* __restrict__ A, int m, int r0, int r1, int c0, int c1, int mask,
                           const VT* src, int ls, int nv, int C, int q, VT* red, bool stream,
                           Epi epi) {
  constexpr int W = NT / 32;
  constexpr int U = sizeof(T) == 4 ? 16 : 8;  // column loads in flight per thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (r1 <= r0 || c1 <= c0) return;  // uniform: every thread sees the same bounds
  const int s_lo = r0 >> 5, s_hi = (r1 - 1) >> 5;
  const int first = s_lo + ((q - s_lo % C) % C + C) % C;  // first owned slab >= s_lo
  const int nown = first > s_hi ? 0 : (s_hi - first) / C + 1;
  if (nown == 0) return;  // uniform within the CTA
  const int P = nown >= W ? 1 : W / nown;  // column splits per slab
  auto slab_sum = [&](int i, int p, int np, VT* acc) {
    const int s = first + i * C;
    const int r = s * 32 + lane;
    int cb = c0, ce = c1;
    if (mask == 1) ce = min(ce, s * 32 + 32);
    if (mask == 2) cb = max(cb, s * 32);
    const int per = (ce - cb + np - 1) / np;
    const int pb = cb + p * per, pe = min(ce, pb + per);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = VT{0, 0};
    if (r < r0 || r >= r1) return;
    const T* Ar = A + r;
    int c = pb;
    for (; c + U <= pe; c += U) {
      T a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int cc = c + u;
        const bool use = mask == 0 || (mask == 1 ? cc < r : cc >= r);
        a[u] = use ? ld_front(Ar + (long)cc * m, stream) : (T)0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v < nv) axpy(acc[v], a[u], src[v * ls + c + u]);
    }
    for (; c < pe; ++c) {
      const bool use = mask == 0 || (mask == 1 ? c < r : c >= r);
      const T a = use ? ld_front(Ar + (long)c * m, stream) : (T)0;
#pragma unroll
      for (int v = 0; v < NV; ++v)
        if (v < nv) axpy(acc[v], a, src[v * ls + c]);
    }
  };
  VT acc[NV];
  if (P == 1) {
    for (int i = warp; i < nown; i += W) {
      slab_sum(i, 0, 1, acc);
      const int r = (first + i * C) * 32 + lane;
      if (r >= r0 && r < r1)
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (v < nv) epi(r, v, acc[v]);
    }
    return;
  }
  const int i = warp % nown, p = warp / nown;
  if (p < P) {
    slab_sum(i, p, P, acc);
#pragma unroll
    for (int v = 0; v < NV; ++v) red[(warp * 32 + lane) * NV + v] = acc[v];
  }
  __syncthreads();
  if (p == 0) {
    const int r = (first + i * C) * 32 + lane;
    if (r >= r0 && r < r1) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (v >= nv) break;
        VT sum = red[(warp * 32 + lane) * NV + v];
        for (int pp = 1; pp < P; ++pp) {
          const VT t = red[((warp + pp * nown) * 32 + lane) * NV + v];
          sum.x += t.x;
          sum.y += t.y;
        }
        epi(r, v, sum);
      }
    }
  }
  __syncthreads();
}

// shared memory of the fused kernels: tv (NV x m), yv (NV x k), red (W x 32 x NV)
template <class VT, int NT, int NV>
size_t fused_smem(int m, int k) {
  return sizeof(VT) * ((size_t)NV * m + (size_t)NV * k + (size_t)NT * NV);
}

// Forward sweep of an inverse-form level: per front, t = [Pi b1; b2] gathered, then
// for each diagonal block J: y_J = t_J + Linv_JJ t_J (strict lower part; unit
// diagonal), t_r -= L[r, J] y_J for the rows below; out: y (k), upd = t[k, m).
template <class VT, class T, int NT, int NV>
__global__ void __launch_bounds__(NT) fused_forward_kernel(FusedArgs a) {
  pdl_wait();
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const int f = blockIdx.x / C, nf = gridDim.x / C;
  const int m = a.m, k = a.k, nv = a.nv;
  extern __shared__ __align__(16) unsigned char smraw[];
  VT* tv = reinterpret_cast<VT*>(smraw);  // NV x m
  VT* yv = tv + (size_t)NV * m;            // NV x k
  VT* red = yv + (size_t)NV * k;           // W x 32 x NV
  const T* A = static_cast<const T*>(a.front) + (long)f * m * m;
  const long v0 = (long)blockIdx.y * NV;  // first vector of this CTA's group
  const VT* rhsQ = static_cast<const VT*>(a.rhsQ);
  const VT* cupd = static_cast<const VT*>(a.cupd);
  for (int v = 0; v < nv; ++v) {
    gather_rhs(a.d, f, m, k, a.nb1, a.gidx, rhsQ + (v0 + v) * a.N,
               cupd ? cupd + (v0 + v) * a.custr : nullptr, a.mc, a.kc, a.ea_map, tv + v * m);
    const int* pr = a.perm + (long)f * k;
    for (int j = threadIdx.x; j < k; j += NT) yv[v * k + j] = tv[v * m + pr[j]];
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += NT) tv[v * m + j] = yv[v * k + j];
    __syncthreads();
  }
  // every CTA of the cluster has finished using yv as the permutation buffer (and has
  // started) before any y value is written into it
  csync(C, cl);
  for (int j0 = 0; j0 < k; j0 += a.ib) {
    const int j1 = min(k, j0 + a.ib);
    rows_times<VT, T, NT, NV>(A, m, j0, j1, j0, j1, 1, tv, m, nv, C, q, red, a.stream,
                              [&](int r, int v, VT s) {
                                const VT o = tv[v * m + r];
                                bcast(&yv[v * k + r], VT{o.x + s.x, o.y + s.y}, C, cl);
                              });
    csync(C, cl);
    const int nxt = min(k, j1 + a.ib);
    rows_times<VT, T, NT, NV>(A, m, j1, m, j0, j1, 0, yv, k, nv, C, q, red, a.stream,
                              [&](int r, int v, VT s) {
                                VT& o = tv[v * m + r];
                                const VT val = VT{o.x - s.x, o.y - s.y};
                                if (r < nxt)
                                  bcast(&o, val, C, cl);
                                else
                                  o = val;
                              });
    csync(C, cl);
  }
  // outputs of the rows this CTA owns
  VT* yout = static_cast<VT*>(a.y);
  VT* upd = static_cast<VT*>(a.upd);
  for (int v = 0; v < nv; ++v) {
    for (int r = threadIdx.x; r < m; r += NT) {
      if (((r >> 5) % C) != q) continue;
      if (r < k)
        yout[(v0 + v) * nf * (long)k + (long)f * k + r] = yv[v * k + r];
      else
        upd[(v0 + v) * nf * (long)(m - k) + (long)f * (m - k) + (r - k)] = tv[v * m + r];
    }
  }
}

// Backward sweep of an inverse-form level: x2 gathered from the global solution,
// t = y1 - U12 x2, then for each diagonal block J from the last: x_J = Uinv_JJ t_J
// (upper part with the diagonal), t_r -= U[r, J] x_J for the rows above; x_J goes
// to the global solution.  tv holds x (NV x m), yv the right-hand sides t (NV x k).
template <class VT, class T, int NT, int NV>
__global__ void __launch_bounds__(NT) fused_backward_kernel(FusedArgs a) {
  pdl_wait();
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int q = (int)cl.block_rank();
  const int f = blockIdx.x / C, nf = gridDim.x / C;
  const int m = a.m, k = a.k, nv = a.nv;
  extern __shared__ __align__(16) unsigned char smraw[];
  VT* xv = reinterpret_cast<VT*>(smraw);  // NV x m
  VT* tv = xv + (size_t)NV * m;            // NV x k
  VT* red = tv + (size_t)NV * k;
  const T* A = static_cast<const T*>(a.front) + (long)f * m * m;
  const long v0 = (long)blockIdx.y * NV;
  const int* gi = a.gidx + (long)f * m;
  const VT* yin = static_cast<const VT*>(a.y);
  for (int v = 0; v < nv; ++v)
    for (int c = k + threadIdx.x; c < m; c += NT) xv[v * m + c] = from_d2<VT>(a.x[(v0 + v) * a.N + gi[c]]);
  csync(C, cl);  // every CTA of the cluster has started before the first remote write
  const int nblk = (k + a.ib - 1) / a.ib;
  const int last0 = (nblk - 1) * a.ib;
  // t = y1 - U12 x2 on the owned rows (the rows of the last block to every CTA)
  if (m > k) {
    rows_times<VT, T, NT, NV>(A, m, 0, k, k, m, 0, xv, m, nv, C, q, red, a.stream, [&](int r, int v, VT s) {
      const VT o = yin[(v0 + v) * nf * (long)k + (long)f * k + r];
      const VT val = VT{o.x - s.x, o.y - s.y};
      if (r >= last0)
        bcast(&tv[v * k + r], val, C, cl);
      else
        tv[v * k + r] = val;
    });
  } else {
    for (int v = 0; v < nv; ++v)
      for (int r = threadIdx.x; r < k; r += NT)
        tv[v * k + r] = yin[(v0 + v) * nf * (long)k + (long)f * k + r];
  }
  csync(C, cl);
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int j0 = bi * a.ib, j1 = min(k, j0 + a.ib);
    rows_times<VT, T, NT, NV>(A, m, j0, j1, j0, j1, 2, tv, k, nv, C, q, red, a.stream,
                              [&](int r, int v, VT s) {
                                bcast(&xv[v * m + r], s, C, cl);
                                a.x[(v0 + v) * a.N + gi[r]] = to_d2(s);
                              });
    csync(C, cl);
    const int prv = max(0, j0 - a.ib);
    rows_times<VT, T, NT, NV>(A, m, 0, j0, j0, j1, 0, xv, m, nv, C, q, red, a.stream,
                              [&](int r, int v, VT s) {
                                VT& o = tv[v * k + r];
                                const VT val = VT{o.x - s.x, o.y - s.y};
                                if (r >= prv)
                                  bcast(&o, val, C, cl);
                                else
                                  o = val;
                              });
    csync(C, cl);
  }
}

constexpr size_t kFusedSmemMax = 200 * 1024;

// cluster size and block size of a level's fused sweep: enough CTAs to cover the
// GPU (C = 1 when the fronts alone give 2 per SM), at most 16 per front
struct FusedCfg {
  int C = 0, NT = 0;
};
FusedCfg fused_config(int nf, int num_sms, int max_cluster) {
  FusedCfg c;
  int C = 1;
  while (C < max_cluster && (long)nf * C < 2L * num_sms) C *= 2;
  c.C = C;
  c.NT = C == 1 ? 256 : ((long)nf * C < num_sms ? 1024 : 512);
  return c;
}

template <class VT, class T, int NT, int NV>
cudaError_t fused_launch_t(bool fwd, const FusedArgs& a, int nf, int C, int groups,
                           cudaStream_t st) {
  const size_t smem = fused_smem<VT, NT, NV>(a.m, a.k);
  if (smem > kFusedSmemMax) return cudaErrorInvalidValue;
  auto kern = fwd ? fused_forward_kernel<VT, T, NT, NV> : fused_backward_kernel<VT, T, NT, NV>;
  // the attributes are set once per kernel, to the largest size any level may ask
  // for: a launch captured into a graph keeps its own request, and lowering the
  // attribute later would make that graph's launch fail
  static bool attr_fwd = false, attr_bwd = false;
  bool& attr = fwd ? attr_fwd : attr_bwd;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFusedSmemMax);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nf * C), (unsigned)groups);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class VT, class T, int NV>
cudaError_t fused_launch_nt(bool fwd, const FusedArgs& a, int nf, const FusedCfg& fc, int groups,
                            cudaStream_t st) {
  if (fc.NT == 256) return fused_launch_t<VT, T, 256, NV>(fwd, a, nf, fc.C, groups, st);
  if (fc.NT == 512) return fused_launch_t<VT, T, 512, NV>(fwd, a, nf, fc.C, groups, st);
  return fused_launch_t<VT, T, 1024, NV>(fwd, a, nf, fc.C, groups, st);
}

// vectors per launch of a fused sweep (1 when only one vector's work vectors fit;
// 0 when not even that fits)
template <class VT>
int fused_group(int m, int k, int NT, int nv) {
  if (nv > 1 && fused_smem<VT, 1024, 4>(m, k) <= kFusedSmemMax) return 4;  // any NT <= 1024
  (void)NT;
  return fused_smem<VT, 1024, 1>(m, k) <= kFusedSmemMax ? 1 : 0;
}

template <class VT>
cudaError_t fused_level(bool fwd, int d, DevLevel& L, const DevLevel* child, const void* rhsQ,
                        double2* x, int nv, long N, cudaStream_t st) {
  using T = typename Scalar<VT>::T;
  const FusedCfg fc{L.fused_c, L.fused_nt};
  FusedArgs a{};
  a.d = d;
  a.m = L.m;
  a.k = L.k;
  a.ib = L.ib;
  a.nb1 = L.nb1;
  a.mc = L.mc;
  a.kc = L.kc;
  a.front = L.front;
  a.gidx = L.gidx;
  a.perm = L.perm;
  a.ea_map = L.ea_map;
  a.rhsQ = rhsQ;
  a.cupd = child ? child->upd : nullptr;
  a.upd = L.upd;
  a.y = L.y;
  a.x = x;
  a.N = N;
  a.custr = child ? (long)child->nf * (child->m - child->k) : 0;
  {
    // the factor entries one sweep reads: k(k-1)/2 + k(m-k) per front
    const double bytes = (double)L.nf * sizeof(T) *
                         ((double)L.k * (L.k - 1) / 2 + (double)L.k * (L.m - L.k));
    a.stream = bytes > 32.0 * 1024 * 1024 ? 1 : 0;
  }
  const int g = fused_group<VT>(L.m, L.k, fc.NT, nv);
  if (g == 0) return cudaErrorInvalidValue;
  // g = 1: one vector per CTA (NV = 1), every vector in its own blockIdx.y;
  // g = 4: groups of four vectors per CTA sharing the factor reads, a last partial
  // group (fewer than four) in a launch of its own
  int done = 0;
  while (done < nv) {
    const int left = nv - done;
    const int groups = g == 1 ? left : (left >= g ? left / g : 1);
    const int per = g == 1 ? 1 : std::min(g, left);
    FusedArgs b = a;
    b.nv = per;
    const long vt = (long)done;  // every vector-indexed pointer advances by `done` vectors
    b.rhsQ = rhsQ ? static_cast<const VT*>(rhsQ) + vt * N : nullptr;
    b.cupd = a.cupd ? static_cast<const VT*>(a.cupd) + vt * a.custr : nullptr;
    b.upd = static_cast<VT*>(L.upd) + vt * (long)L.nf * (L.m - L.k);
    b.y = static_cast<VT*>(L.y) + vt * (long)L.nf * L.k;
    b.x = x ? x + vt * N : nullptr;
    cudaError_t e = g == 1 ? fused_launch_nt<VT, T, 1>(fwd, b, L.nf, fc, groups, st)
                           : fused_launch_nt<VT, T, 4>(fwd, b, L.nf, fc, groups, st);
    if (e != cudaSuccess) return e;
    done += groups * per;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t q_apply(int prec, int d, int n, int nl, const std::vector<QTypeDev>& types,
                    const double* Tcat, const float* Tcat32, const double2* r, void* y,
                    cudaStream_t st, int nv, bool pdl, int P, long t_stride) {
  long N = 1;
  for (int a = 0; a < d; ++a) N *= n;
  if (prec == SP_PREC_FP32)
    return q_apply_t<float2>(d, n, nl, types, Tcat32, r, (float2*)y, nv, N, st, pdl, P, t_stride);
  return q_apply_t<double2>(d, n, nl, types, Tcat, r, (double2*)y, nv, N, st, pdl, P, t_stride);
}

cudaError_t forward_level(int prec, int d, DevLevel& L, const DevLevel* child, const void* rhsQ,
                          void* part, cudaStream_t st, int nv, long N) {
  if (prec == SP_PREC_FP32) return forward_t<float2>(d, L, child, rhsQ, part, nv, N, st);
  return forward_t<double2>(d, L, child, rhsQ, part, nv, N, st);
}

cudaError_t backward_level(int prec, int d, DevLevel& L, double2* x, void* part, cudaStream_t st,
                           int nv, long N) {
  (void)d;
  if (prec == SP_PREC_FP32) return backward_t<float2>(L, x, part, nv, N, st);
  return backward_t<double2>(L, x, part, nv, N, st);
}

int sweep_max_vectors() { return kMaxVec; }

int sweep_max_cluster() {
  // 16 CTAs per cluster (non-portable) when a cluster of 16 of the largest fused
  // kernels (1024 threads, the FP64 shared memory of a 2044-wide root) can be resident
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 8;
  static int cache[64] = {0};
  if (cache[dev]) return cache[dev];
  int best = 8;
  auto kern = fused_forward_kernel<double2, double, 1024, 1>;
  const size_t smem = fused_smem<double2, 1024, 1>(2048, 2048);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax) ==
          cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) best = 16;
  }
  cudaGetLastError();  // a refused query leaves no error behind
  cache[dev] = best;
  return best;
}

bool sweep_fused_config(int prec, int nf, int m, int k, int num_sms, int max_cluster,
                        bool clusters, int* C, int* NT) {
  const int g = prec == SP_PREC_FP32 ? fused_group<float2>(m, k, 1024, 1)
                                     : fused_group<double2>(m, k, 1024, 1);
  if (g == 0) return false;
  const FusedCfg fc = fused_config(nf, num_sms, max_cluster);
  if (fc.C > 1 && !clusters) return false;
  *C = fc.C;
  *NT = fc.NT;
  return true;
}

size_t sweep_partial_bytes(int nv) {
  return (size_t)2 * kGemvTarget * 256 * sizeof(double2) * (size_t)nv;
}

}  // namespace sp
