// FP64 complex FFT passes for the pseudospectral operator (Section 2.1, Eq. G).
//
//   G x = F^{-1} diag(1/(4 pi^2 |k|^2 - s)) F x       (Eq. G)
//   A x = x + G (q x)                                   (Section 2.2)
//
// The n^d transform is done axis by axis.  Each CTA owns W complete 1D lines of
// length n of one axis, stages them in shared memory (coalesced: along axis 0 the
// lines are contiguous, along the other axes W neighbouring lines give W
// consecutive elements per row), runs radix-2 butterflies in shared memory and
// writes the lines back.  Fused pointwise work:
//   first pass   x -> q x              (PRE_Q)
//   last axis    forward, * D/N, inverse in one pass (MID), so the spectrum never
//                leaves shared memory between the forward and inverse transform
//   final pass   out = x + result      (POST_ADD)
// Forward transforms are decimation-in-time (bit-reversed load), inverse ones
// decimation-in-frequency (bit-reversed store), so no extra permutation pass is
// needed.  n must be a power of two (<= 4096).
#include <cstdio>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

struct PassArgs {
  const double2* in;
  double2* out;
  const double* q;      // PRE_Q
  const double* Dn;     // MID
  const double2* addx;  // POST_ADD
  const double2* tw;
  long S;               // stride between consecutive elements of a line
  long nlines;          // number of lines of this axis
  int n, logn, W, pad;
  int mode;             // 0 forward, 1 inverse, 2 middle (forward, scale, inverse)
};

// global address of element i of line t
__device__ __forceinline__ long line_addr(const PassArgs& a, long t, int i) {
  long lo = t % a.S, hi = t / a.S;
  return lo + hi * a.S * a.n + (long)i * a.S;
}

__device__ __forceinline__ void dit_stages(double2* sm, const PassArgs& a, bool conj_tw) {
  const int n = a.n, half_n = n >> 1, ld = n + a.pad;
  const int work = a.W * half_n;
  for (int s = 1; s <= a.logn; ++s) {
    const int half = 1 << (s - 1);
    for (int it = threadIdx.x; it < work; it += blockDim.x) {
      int w = it / half_n, p = it - w * half_n;
      int jj = p & (half - 1);
      int i0 = ((p >> (s - 1)) << s) + jj;
      int i1 = i0 + half;
      double2 t = __ldg(&a.tw[jj << (a.logn - s)]);
      if (conj_tw) t.y = -t.y;
      double2* row = sm + w * ld;
      double2 u = row[i0], v = cmul(row[i1], t);
      row[i0] = cadd(u, v);
      row[i1] = csub(u, v);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void dif_stages(double2* sm, const PassArgs& a, bool conj_tw) {
  const int n = a.n, half_n = n >> 1, ld = n + a.pad;
  const int work = a.W * half_n;
  for (int s = a.logn; s >= 1; --s) {
    const int half = 1 << (s - 1);
    for (int it = threadIdx.x; it < work; it += blockDim.x) {
      int w = it / half_n, p = it - w * half_n;
      int jj = p & (half - 1);
      int i0 = ((p >> (s - 1)) << s) + jj;
      int i1 = i0 + half;
      double2 t = __ldg(&a.tw[jj << (a.logn - s)]);
      if (conj_tw) t.y = -t.y;
      double2* row = sm + w * ld;
      double2 u = row[i0], v = row[i1];
      row[i0] = cadd(u, v);
      row[i1] = cmul(csub(u, v), t);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) fft_pass_kernel(PassArgs a) {
  extern __shared__ double2 sm[];
  const int n = a.n, ld = n + a.pad, W = a.W;
  const long t0 = (long)blockIdx.x * W;
  const int total = W * n;
  const bool axis0 = (a.S == 1);
  const bool bitrev_load = (a.mode != 1);  // forward transforms are DIT
  // ---- load (coalesced), optional q multiply, bit-reversed placement for DIT
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int w, i;
    if (axis0) {
      w = e / n;
      i = e - w * n;
    } else {
      i = e / W;
      w = e - i * W;
    }
    long t = t0 + w;
    if (t >= a.nlines) continue;
    long g = line_addr(a, t, i);
    double2 v = a.in[g];
    if (a.q) {
      double qq = a.q[g];
      v.x *= qq;
      v.y *= qq;
    }
    int pos = bitrev_load ? (int)(__brev((unsigned)i) >> (32 - a.logn)) : i;
    sm[w * ld + pos] = v;
  }
  __syncthreads();
  if (a.mode == 0) {
    dit_stages(sm, a, false);
  } else if (a.mode == 1) {
    dif_stages(sm, a, true);
  } else {
    dit_stages(sm, a, false);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      int w, i;
      if (axis0) {
        w = e / n;
        i = e - w * n;
      } else {
        i = e / W;
        w = e - i * W;
      }
      long t = t0 + w;
      if (t >= a.nlines) continue;
      double dn = a.Dn[line_addr(a, t, i)];
      double2* p = &sm[w * ld + i];
      p->x *= dn;
      p->y *= dn;
    }
    __syncthreads();
    dif_stages(sm, a, true);
  }
  const bool bitrev_store = (a.mode != 0);  // inverse transforms are DIF
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int w, i;
    if (axis0) {
      w = e / n;
      i = e - w * n;
    } else {
      i = e / W;
      w = e - i * W;
    }
    long t = t0 + w;
    if (t >= a.nlines) continue;
    long g = line_addr(a, t, i);
    int pos = bitrev_store ? (int)(__brev((unsigned)i) >> (32 - a.logn)) : i;
    double2 v = sm[w * ld + pos];
    if (a.addx) v = cadd(v, a.addx[g]);
    a.out[g] = v;
  }
}

int lines_per_cta(int n, long nlines) {
  // enough lines for >= 256 butterflies per stage, at most 64 KB of lines, and
  // at least ~2 CTAs per SM on 152 SMs when the grid allows it
  int W = 1;
  while (W * n < 2 * kThreads && W < 64) W <<= 1;
  while (W > 1 && (long)W * n * 16 > 64 * 1024) W >>= 1;
  while (W > 1 && nlines / W < 304) W >>= 1;
  return W;
}

cudaError_t run_pass(const FftPlan& P, int axis, int mode, const double2* in, double2* out,
                     const double* q, const double2* addx, cudaStream_t st) {
  PassArgs a{};
  a.mode = mode;
  a.in = in;
  a.out = out;
  a.q = q;
  a.Dn = (mode == 2) ? P.Dn : nullptr;
  a.addx = addx;
  a.tw = P.tw;
  a.n = P.n;
  a.logn = P.logn;
  long S = 1;
  for (int i = 0; i < axis; ++i) S *= P.n;
  a.S = S;
  long N = 1;
  for (int i = 0; i < P.d; ++i) N *= P.n;
  a.nlines = N / P.n;
  a.W = lines_per_cta(P.n, a.nlines);
  // axis > 0 lines are grouped W at a time inside one S-block: W must divide S
  if (axis > 0)
    while (a.W > 1 && (S % a.W)) a.W >>= 1;
  a.pad = 1;
  size_t smem = (size_t)a.W * (P.n + a.pad) * sizeof(double2);
  long grid = (a.nlines + a.W - 1) / a.W;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  ProfScope ps(PROF_FFT, st);
  fft_pass_kernel<<<(unsigned)grid, kThreads, smem, st>>>(a);
  ps.done((double)N * (32.0 + (q ? 8.0 : 0.0) + (mode == 2 ? 8.0 : 0.0) + (addx ? 16.0 : 0.0)), 1, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t fft_green_apply(const FftPlan& P, const double2* x, const double* q, bool add_x,
                            double2* out, cudaStream_t st) {
  cudaError_t e;
  const int d = P.d;
  // forward along axes 0..d-2, middle pass on axis d-1, inverse along d-2..0
  const double2* src = x;
  for (int ax = 0; ax < d - 1; ++ax) {
    e = run_pass(P, ax, 0, src, P.tmp, ax == 0 ? q : nullptr, nullptr, st);
    if (e != cudaSuccess) return e;
    src = P.tmp;
  }
  e = run_pass(P, d - 1, 2, src, P.tmp, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  for (int ax = d - 2; ax >= 0; --ax) {
    bool last = (ax == 0);
    e = run_pass(P, ax, 1, P.tmp, last ? out : P.tmp, nullptr, (last && add_x) ? x : nullptr, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sp
