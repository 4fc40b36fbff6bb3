// Preconditioner application z = P^{-1} Q r (Section 2.2, "u <= P^{-1} Q g"):
//   1. the sparsifying stencil y_S = Q(S, gamma(S)) r_gamma(S) for every set
//      instance (Section 2.3, Q(S, gamma) = [I, -T_S]);
//   2. the forward sweep of the multifrontal factor, leaves to root: per front
//      y1 = L11^{-1} Pi b1 and the update b2 - L21 y1 handed to the parent;
//   3. the backward sweep, root to leaves: x1 = U11^{-1} (y1 - U12 x2).
// One CTA per front; the front's right-hand side lives in shared memory.  The
// triangular solves are blocked by 32: one warp resolves the 32 x 32 diagonal
// block with shuffles, then all warps apply the block's columns to the rows
// below (forward) or above (backward) with coalesced column reads of the
// column-major front.  VT = double2 (FP64 form) or float2 (FP32 form).
#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kBS = 32;

template <class VT> struct Scalar;
template <> struct Scalar<double2> { using T = double; };
template <> struct Scalar<float2> { using T = float; };

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

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// y[S instance] = Q_t r[gamma instance]; one CTA per instance of type t.
template <class VT, class T>
__global__ void qapply_kernel(int d, int n, int nl, int nS, int nG, const int* __restrict__ Soff,
                              const int* __restrict__ Goff, const T* __restrict__ Qt,
                              const double2* __restrict__ r, VT* y) {
  extern __shared__ unsigned char smraw[];
  VT* rg = reinterpret_cast<VT*>(smraw);
  int box = blockIdx.x, o[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    o[a] = (box % nl) * (n / nl);
    box /= nl;
  }
  for (int c = threadIdx.x; c < nG; c += blockDim.x) {
    long g = 0, s = 1;
    for (int a = 0; a < d; ++a) {
      g += (long)wrapi(o[a] + Goff[c * d + a], n) * s;
      s *= n;
    }
    rg[c] = from_d2<VT>(r[g]);
  }
  __syncthreads();
  for (int a0 = threadIdx.x; a0 < nS; a0 += blockDim.x) {
    VT acc = vzero<VT>();
    for (int c = 0; c < nG; ++c) axpy_neg(acc, -Qt[a0 + (long)c * nS], rg[c]);
    long g = 0, s = 1;
    for (int a = 0; a < d; ++a) {
      g += (long)wrapi(o[a] + Soff[a0 * d + a], n) * s;
      s *= n;
    }
    y[g] = acc;
  }
}

// Forward sweep of one level, one CTA per front.
template <class VT, class T>
__global__ void __launch_bounds__(256) forward_kernel(
    int d, const T* __restrict__ fronts, int m, int k, int nb1, const int* __restrict__ gidx,
    const int* __restrict__ perm, const VT* __restrict__ rhsQ, const VT* __restrict__ cupd, int mc,
    int kc, const int* __restrict__ ea_map, VT* upd, VT* yout) {
  extern __shared__ unsigned char smraw[];
  VT* b = reinterpret_cast<VT*>(smraw);  // m
  VT* b1 = b + m;                         // k (permuted eliminated part)
  const int f = blockIdx.x;
  const T* A = fronts + (long)f * m * m;
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
  const int* pr = perm + (long)f * k;
  for (int j = threadIdx.x; j < k; j += blockDim.x) b1[j] = b[pr[j]];
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) b[j] = b1[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jb = 0; jb < k; jb += kBS) {
    const int bs = min(kBS, k - jb);
    if (warp == 0) {
      VT val = (lane < bs) ? b[jb + lane] : vzero<VT>();
      for (int j = 0; j < bs; ++j) {
        VT yj;
        yj.x = __shfl_sync(0xffffffffu, val.x, j);
        yj.y = __shfl_sync(0xffffffffu, val.y, j);
        if (lane > j && lane < bs) axpy_neg(val, A[(jb + lane) + (long)(jb + j) * m], yj);
      }
      if (lane < bs) b[jb + lane] = val;
    }
    __syncthreads();
    for (int r = jb + bs + threadIdx.x; r < m; r += blockDim.x) {
      VT acc = b[r];
      for (int j = 0; j < bs; ++j) axpy_neg(acc, A[r + (long)(jb + j) * m], b[jb + j]);
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
                                                        const VT* __restrict__ yin, double2* x) {
  extern __shared__ unsigned char smraw[];
  VT* xb = reinterpret_cast<VT*>(smraw);  // m: x1 then x2
  const int f = blockIdx.x;
  const T* A = fronts + (long)f * m * m;
  const int* gi = gidx + (long)f * m;
  for (int v = k + threadIdx.x; v < m; v += blockDim.x) xb[v] = from_d2<VT>(x[gi[v]]);
  __syncthreads();
  // rhs = y1 - U12 x2
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    VT acc = yin[(long)f * k + i];
    for (int c = k; c < m; ++c) axpy_neg(acc, A[i + (long)c * m], xb[c]);
    xb[i] = acc;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nblk = (k + kBS - 1) / kBS;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int jb = bi * kBS;
    const int bs = min(kBS, k - jb);
    if (warp == 0) {
      VT val = (lane < bs) ? xb[jb + lane] : vzero<VT>();
      for (int j = bs - 1; j >= 0; --j) {
        if (lane == j) {
          const T dgi = A[(jb + j) + (long)(jb + j) * m];
          val.x /= dgi;
          val.y /= dgi;
        }
        VT xj;
        xj.x = __shfl_sync(0xffffffffu, val.x, j);
        xj.y = __shfl_sync(0xffffffffu, val.y, j);
        if (lane < j) axpy_neg(val, A[(jb + lane) + (long)(jb + j) * m], xj);
      }
      if (lane < bs) xb[jb + lane] = val;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < jb; r += blockDim.x) {
      VT acc = xb[r];
      for (int j = 0; j < bs; ++j) axpy_neg(acc, A[r + (long)(jb + j) * m], xb[jb + j]);
      xb[r] = acc;
    }
    __syncthreads();
  }
  for (int v = threadIdx.x; v < k; v += blockDim.x) x[gi[v]] = to_d2(xb[v]);
}

template <class VT>
cudaError_t q_apply_t(int d, int n, int nl, const std::vector<QTypeDev>& types, const void* Qt,
                      const double2* r, VT* y, cudaStream_t st) {
  using T = typename Scalar<VT>::T;
  long ninst = 1;
  for (int a = 0; a < d; ++a) ninst *= nl;
  ProfScope ps(PROF_QAPPLY, st);
  double bytes = 0;
  for (const auto& ty : types) {
    size_t smem = sizeof(VT) * ty.nG;
    qapply_kernel<VT, T><<<(unsigned)ninst, 128, smem, st>>>(
        d, n, nl, ty.nS, ty.nG, ty.S, ty.G, (const T*)Qt + ty.tab_off, r, y);
    bytes += (double)ninst * ty.nS * (sizeof(double2) + sizeof(VT)) + sizeof(T) * ty.nS * ty.nG;
  }
  ps.done(bytes, (int)types.size(), st);
  return cudaGetLastError();
}

size_t sweep_smem(int m, int k, size_t vt) { return vt * (size_t)(m + k); }

}  // namespace

cudaError_t q_apply(int prec, int d, int n, int nl, const std::vector<QTypeDev>& types,
                    const double* Qcat, const float* Qcat32, const double2* r, void* y,
                    cudaStream_t st) {
  if (prec == SP_PREC_FP32) return q_apply_t<float2>(d, n, nl, types, Qcat32, r, (float2*)y, st);
  return q_apply_t<double2>(d, n, nl, types, Qcat, r, (double2*)y, st);
}

cudaError_t forward_level(int prec, int d, DevLevel& L, const DevLevel* child, const void* rhsQ,
                          cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(forward_kernel<double2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(forward_kernel<float2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(backward_kernel<double2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(backward_kernel<float2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const double fs = prec == SP_PREC_FP32 ? 4.0 : 8.0;
  const double kk = L.k, mk = L.m - L.k;
  ProfScope ps(PROF_FORWARD, st);
  if (prec == SP_PREC_FP32) {
    size_t sm = sweep_smem(L.m, L.k, sizeof(float2));
    forward_kernel<float2, float><<<L.nf, 256, sm, st>>>(
        d, (const float*)L.front, L.m, L.k, L.nb1, L.gidx, L.perm, (const float2*)rhsQ,
        child ? (const float2*)child->upd : nullptr, L.mc, L.kc, L.ea_map, (float2*)L.upd,
        (float2*)L.y);
  } else {
    size_t sm = sweep_smem(L.m, L.k, sizeof(double2));
    forward_kernel<double2, double><<<L.nf, 256, sm, st>>>(
        d, (const double*)L.front, L.m, L.k, L.nb1, L.gidx, L.perm, (const double2*)rhsQ,
        child ? (const double2*)child->upd : nullptr, L.mc, L.kc, L.ea_map, (double2*)L.upd,
        (double2*)L.y);
  }
  ps.done(L.nf * fs * (kk * (kk - 1) / 2 + mk * kk), 1, st);
  return cudaGetLastError();
}

cudaError_t backward_level(int prec, int d, DevLevel& L, double2* x, cudaStream_t st) {
  (void)d;
  const double fs = prec == SP_PREC_FP32 ? 4.0 : 8.0;
  const double kk = L.k, mk = L.m - L.k;
  ProfScope ps(PROF_BACKWARD, st);
  if (prec == SP_PREC_FP32) {
    size_t sm = sizeof(float2) * (size_t)L.m;
    backward_kernel<float2, float><<<L.nf, 256, sm, st>>>((const float*)L.front, L.m, L.k, L.gidx,
                                                         (const float2*)L.y, x);
  } else {
    size_t sm = sizeof(double2) * (size_t)L.m;
    backward_kernel<double2, double><<<L.nf, 256, sm, st>>>((const double*)L.front, L.m, L.k,
                                                           L.gidx, (const double2*)L.y, x);
  }
  ps.done(L.nf * fs * (kk * (kk + 1) / 2 + mk * kk), 1, st);
  return cudaGetLastError();
}

}  // namespace sp
