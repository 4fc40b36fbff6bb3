// Complex FFT passes for the pseudospectral operator (Section 2.1, Eq. G), in
// FP64 (double2) and, for the inner solve of the mixed-precision form, FP32 (float2).
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
// needed.  n = R M with M a power of two and R = 1 or 3: for R = 3 the line is
// split by j mod 3 into three M-point lines (element j = 3 j' + r goes to
// sub-line r at the bit-reversed position of j'), the three M-point transforms
// run side by side, and one radix-3 step combines them in place,
//   X[k1 + M k2] = sum_r w_n^(r k1) w_3^(r k2) Y_r[k1],
// which leaves the spectrum in natural order (sub-line k2 holds X[k1 + M k2]);
// the inverse runs the conjugate steps in the opposite order.
#include <cstdio>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kThreads = 256;

template <class VT> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <class VT>
struct PassArgs {
  using T = typename Real<VT>::T;
  const VT* in;
  VT* out;
  const T* q;      // PRE_Q
  const T* Dn;     // MID
  const VT* addx;  // POST_ADD
  const VT* tw;         // w_n^t = exp(-2 pi i t / n), t < n / 2
  long S;               // stride between consecutive elements of a line
  long nlines;          // number of lines of this axis, all vectors
  long vlines, vstride; // lines per vector, entries per vector (vectors stacked)
  int n, W, pad;
  int R, M, logM;       // n = R M, R in {1, 3}, M = 2^logM
  int mode;             // 0 forward, 1 inverse, 2 middle (forward, scale, inverse)
  int qper;             // q and Dn per vector: vector v reads those of v % qper (vstride apart)
};

// position in the staged row of element i of a line in permuted (DIT input /
// DIF output) order
template <int R, class VT>
__device__ __forceinline__ int perm_pos(const PassArgs<VT>& a, int i) {
  const int r = i % R, j = i / R;
  return r * a.M + (a.logM ? (int)(__brev((unsigned)j) >> (32 - a.logM)) : 0);
}
// w_n^t for 0 <= t < n (w_n^(t + n/2) = -w_n^t)
template <class VT>
__device__ __forceinline__ VT tw_at(const PassArgs<VT>& a, int t) {
  const int h = a.n >> 1;
  if (t < h) return a.tw[t];
  VT v = a.tw[t - h];
  v.x = -v.x;
  v.y = -v.y;
  return v;
}

// address of element i of line t within its vector (q and the symbol are shared
// by every vector), and the offset of that vector
template <class VT>
__device__ __forceinline__ long line_addr(const PassArgs<VT>& a, long t, int i) {
  const long tl = t % a.vlines;
  long lo = tl % a.S, hi = tl / a.S;
  return lo + hi * a.S * a.n + (long)i * a.S;
}
template <class VT>
__device__ __forceinline__ long vec_off(const PassArgs<VT>& a, long t) {
  return (t / a.vlines) * a.vstride;
}

// radix-2 stages of the W R sub-lines of length M (sub-line r of row w at
// offset r M); the M-point twiddle w_M^t is w_n^(R t)
template <int R, class VT>
__device__ __forceinline__ void dit_stages(VT* sm, const PassArgs<VT>& a, bool conj_tw) {
  const int M = a.M, half_m = M >> 1, ld = a.n + a.pad;
  const int work = a.W * R * half_m;
  for (int s = 1; s <= a.logM; ++s) {
    const int half = 1 << (s - 1);
    for (int it = threadIdx.x; it < work; it += blockDim.x) {
      int u = it / half_m, p = it - u * half_m;
      int w = u / R, r = u - w * R;
      int jj = p & (half - 1);
      int i0 = ((p >> (s - 1)) << s) + jj;
      int i1 = i0 + half;
      VT t = a.tw[(jj << (a.logM - s)) * R];
      if (conj_tw) t.y = -t.y;
      VT* row = sm + w * ld + r * M;
      VT x0 = row[i0], v = cmul(row[i1], t);
      row[i0] = cadd(x0, v);
      row[i1] = csub(x0, v);
    }
    __syncthreads();
  }
}

template <int R, class VT>
__device__ __forceinline__ void dif_stages(VT* sm, const PassArgs<VT>& a, bool conj_tw) {
  const int M = a.M, half_m = M >> 1, ld = a.n + a.pad;
  const int work = a.W * R * half_m;
  for (int s = a.logM; s >= 1; --s) {
    const int half = 1 << (s - 1);
    for (int it = threadIdx.x; it < work; it += blockDim.x) {
      int u = it / half_m, p = it - u * half_m;
      int w = u / R, r = u - w * R;
      int jj = p & (half - 1);
      int i0 = ((p >> (s - 1)) << s) + jj;
      int i1 = i0 + half;
      VT t = a.tw[(jj << (a.logM - s)) * R];
      if (conj_tw) t.y = -t.y;
      VT* row = sm + w * ld + r * M;
      VT x0 = row[i0], v = row[i1];
      row[i0] = cadd(x0, v);
      row[i1] = cmul(csub(x0, v), t);
    }
    __syncthreads();
  }
}

// The same transforms with the radix-2 stages taken two at a time (radix 4): three
// twiddle products and one barrier per pair of stages instead of four and two.
//   DIT stages s, s+1 (h = 2^(s-1)): with t1 = w_{2h}^j, t2 = w_{4h}^j,
//     u0 = x0, u1 = t1 x1, u2 = t2 x2, u3 = t1 t2 x3 (x_q at base + j + q h),
//     y0 = (u0 + u1) + (u2 + u3), y2 = (u0 + u1) - (u2 + u3),
//     y1 = (u0 - u1) - i (u2 - u3), y3 = (u0 - u1) + i (u2 - u3);
//   DIF stages s, s-1 (q = 2^(s-2)) of the conjugate (inverse) transform: with
//     t1 = conj w_{4q}^j, t2 = conj w_{2q}^j, s0 = x0 + x2, s1 = x0 - x2, s2 = x1 + x3,
//     s3 = x1 - x3 (x_r at base + j + r q): y0 = s0 + s2, y1 = (s0 - s2) t2,
//     y2 = (s1 + i s3) t1, y3 = (s1 - i s3) t1 t2.
// An odd stage count leaves one radix-2 stage (first for DIT, last for DIF).
template <class VT>
__device__ __forceinline__ VT mul_i(VT v) {  // i v
  VT r;
  r.x = -v.y;
  r.y = v.x;
  return r;
}
template <int R, class VT>
__device__ __forceinline__ void dit_stages4(VT* sm, const PassArgs<VT>& a) {
  const int M = a.M, ld = a.n + a.pad;
  int s = 1;
  if (a.logM & 1) {  // one radix-2 stage first (twiddle 1)
    const int work = a.W * R * (M >> 1);
    for (int it = threadIdx.x; it < work; it += blockDim.x) {
      const int u = it / (M >> 1), p = it - u * (M >> 1);
      const int w = u / R, r = u - w * R;
      VT* row = sm + w * ld + r * M;
      const int i0 = 2 * p;
      const VT x0 = row[i0], x1 = row[i0 + 1];
      row[i0] = cadd(x0, x1);
      row[i0 + 1] = csub(x0, x1);
    }
    __syncthreads();
    s = 2;
  }
  const int quarter = M >> 2;
  const int work = a.W * R * quarter;
  for (; s + 1 <= a.logM; s += 2) {
    const int h = 1 << (s - 1);
    for (int it = threadIdx.x; it < work; it += blockDim.x) {
      const int u = it / quarter, p = it - u * quarter;
      const int w = u / R, r = u - w * R;
      const int j = p & (h - 1);
      const int base = ((p >> (s - 1)) << (s + 1)) + j;
      VT* row = sm + w * ld + r * M;
      const VT t1 = a.tw[(j << (a.logM - s)) * R];
      const VT t2 = a.tw[(j << (a.logM - s - 1)) * R];
      const VT t3 = tw_at(a, (3 * j << (a.logM - s - 1)) * R);
      const VT u0 = row[base], u1 = cmul(row[base + h], t1);
      const VT u2 = cmul(row[base + 2 * h], t2), u3 = cmul(row[base + 3 * h], t3);
      const VT s0 = cadd(u0, u1), s1 = csub(u0, u1), s2 = cadd(u2, u3), s3 = mul_i(csub(u2, u3));
      row[base] = cadd(s0, s2);
      row[base + 2 * h] = csub(s0, s2);
      row[base + h] = csub(s1, s3);
      row[base + 3 * h] = cadd(s1, s3);
    }
    __syncthreads();
  }
}
template <int R, class VT>
__device__ __forceinline__ void dif_stages4_conj(VT* sm, const PassArgs<VT>& a) {
  const int M = a.M, ld = a.n + a.pad;
  const int quarter = M >> 2;
  const int work4 = a.W * R * quarter;
  int s = a.logM;
  for (; s >= 2; s -= 2) {
    const int q = 1 << (s - 2);
    for (int it = threadIdx.x; it < work4; it += blockDim.x) {
      const int u = it / quarter, p = it - u * quarter;
      const int w = u / R, r = u - w * R;
      const int j = p & (q - 1);
      const int base = ((p >> (s - 2)) << s) + j;
      VT* row = sm + w * ld + r * M;
      VT t1 = a.tw[(j << (a.logM - s)) * R];
      VT t2 = a.tw[(j << (a.logM - s + 1)) * R];
      VT t3 = tw_at(a, (3 * j << (a.logM - s)) * R);
      t1.y = -t1.y;
      t2.y = -t2.y;
      t3.y = -t3.y;
      const VT x0 = row[base], x1 = row[base + q], x2 = row[base + 2 * q], x3 = row[base + 3 * q];
      const VT s0 = cadd(x0, x2), s1 = csub(x0, x2), s2 = cadd(x1, x3), s3 = mul_i(csub(x1, x3));
      row[base] = cadd(s0, s2);
      row[base + q] = cmul(csub(s0, s2), t2);
      row[base + 2 * q] = cmul(cadd(s1, s3), t1);
      row[base + 3 * q] = cmul(csub(s1, s3), t3);
    }
    __syncthreads();
  }
  if (s == 1) {  // one radix-2 stage last (twiddle 1)
    const int work = a.W * R * (M >> 1);
    for (int it = threadIdx.x; it < work; it += blockDim.x) {
      const int u = it / (M >> 1), p = it - u * (M >> 1);
      const int w = u / R, r = u - w * R;
      VT* row = sm + w * ld + r * M;
      const int i0 = 2 * p;
      const VT x0 = row[i0], x1 = row[i0 + 1];
      row[i0] = cadd(x0, x1);
      row[i0 + 1] = csub(x0, x1);
    }
    __syncthreads();
  }
}

// radix-3 step over the three sub-lines of every row (R = 3 only).  Forward:
// X[k1 + M k2] = sum_r w_3^(r k2) (w_n^(r k1) Y_r[k1]); inverse (conjugate):
// Z_r[k1] = w_n^(-r k1) sum_k2 w_3^(-r k2) X[k1 + M k2].
template <class VT>
__device__ __forceinline__ void radix3_step(VT* sm, const PassArgs<VT>& a, bool inverse) {
  using T = typename Real<VT>::T;
  const int M = a.M, ld = a.n + a.pad;
  const T h3 = (T)0.86602540378443864676372317075294;  // sin(2 pi / 3)
  for (int it = threadIdx.x; it < a.W * M; it += blockDim.x) {
    const int w = it / M, k1 = it - w * M;
    VT* row = sm + w * ld;
    VT w1 = tw_at(a, k1), w2 = tw_at(a, 2 * k1);
    if (!inverse) {
      const VT a0 = row[k1], b1 = cmul(row[M + k1], w1), b2 = cmul(row[2 * M + k1], w2);
      const VT t1 = cadd(b1, b2), t2 = csub(b1, b2);
      VT mm = a0;
      mm.x -= (T)0.5 * t1.x;
      mm.y -= (T)0.5 * t1.y;
      VT rot;  // -i sin(2 pi / 3) t2
      rot.x = h3 * t2.y;
      rot.y = -h3 * t2.x;
      row[k1] = cadd(a0, t1);
      row[M + k1] = cadd(mm, rot);
      row[2 * M + k1] = csub(mm, rot);
    } else {
      const VT x0 = row[k1], x1 = row[M + k1], x2 = row[2 * M + k1];
      const VT u1 = cadd(x1, x2), u2 = csub(x1, x2);
      VT mm = x0;
      mm.x -= (T)0.5 * u1.x;
      mm.y -= (T)0.5 * u1.y;
      VT rot;  // +i sin(2 pi / 3) u2
      rot.x = -h3 * u2.y;
      rot.y = h3 * u2.x;
      w1.y = -w1.y;
      w2.y = -w2.y;
      row[k1] = cadd(x0, u1);
      row[M + k1] = cmul(cadd(mm, rot), w1);
      row[2 * M + k1] = cmul(csub(mm, rot), w2);
    }
  }
  __syncthreads();
}

template <class VT, int R>
__global__ void __launch_bounds__(kThreads) fft_pass_kernel(PassArgs<VT> a) {
  using T = typename Real<VT>::T;
  extern __shared__ unsigned char smraw[];
  VT* sm = reinterpret_cast<VT*>(smraw);
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
    VT v = a.in[vec_off(a, t) + g];
    if (a.q) {
      T qq = a.q[(a.qper > 1 ? (t / a.vlines) % a.qper * a.vstride : 0) + g];
      v.x *= qq;
      v.y *= qq;
    }
    int pos = bitrev_load ? perm_pos<R>(a, i) : i;
    sm[w * ld + pos] = v;
  }
  __syncthreads();
  if (a.mode == 0) {
    dit_stages4<R>(sm, a);
    if (R == 3) radix3_step(sm, a, false);
  } else if (a.mode == 1) {
    if (R == 3) radix3_step(sm, a, true);
    dif_stages4_conj<R>(sm, a);
  } else {
    dit_stages4<R>(sm, a);
    if (R == 3) radix3_step(sm, a, false);
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
      T dn = a.Dn[(a.qper > 1 ? (t / a.vlines) % a.qper * a.vstride : 0) + line_addr(a, t, i)];
      VT* p = &sm[w * ld + i];
      p->x *= dn;
      p->y *= dn;
    }
    __syncthreads();
    if (R == 3) radix3_step(sm, a, true);
    dif_stages4_conj<R>(sm, a);
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
    long g = vec_off(a, t) + line_addr(a, t, i);
    int pos = bitrev_store ? perm_pos<R>(a, i) : i;
    VT v = sm[w * ld + pos];
    if (a.addx) v = cadd(v, a.addx[g]);
    a.out[g] = v;
  }
}

int lines_per_cta(int n, long nlines, int esize) {
  // enough lines for >= 256 butterflies per stage, at most 64 KB of lines, and
  // at least ~2 CTAs per SM on 152 SMs when the grid allows it
  int W = 1;
  while (W * n < 2 * kThreads && W < 64) W <<= 1;
  while (W > 1 && (long)W * n * esize > 64 * 1024) W >>= 1;
  while (W > 1 && nlines / W < 304) W >>= 1;
  return W;
}

template <class VT>
cudaError_t run_pass(int d, int n, const VT* tw, const typename Real<VT>::T* Dn, int axis,
                     int mode, const VT* in, VT* out, const typename Real<VT>::T* q,
                     const VT* addx, int nvec, int qper, cudaStream_t st) {
  PassArgs<VT> a{};
  a.mode = mode;
  a.qper = qper;
  a.in = in;
  a.out = out;
  a.q = q;
  a.Dn = (mode == 2) ? Dn : nullptr;
  a.addx = addx;
  a.tw = tw;
  a.n = n;
  a.R = (n % 3 == 0) ? 3 : 1;
  a.M = n / a.R;
  a.logM = 0;
  while ((1 << a.logM) < a.M) ++a.logM;
  long S = 1;
  for (int i = 0; i < axis; ++i) S *= n;
  a.S = S;
  long N = 1;
  for (int i = 0; i < d; ++i) N *= n;
  a.vlines = N / n;
  a.vstride = N;
  a.nlines = a.vlines * nvec;
  a.W = lines_per_cta(n, a.nlines, (int)sizeof(VT));
  // axis > 0 lines are grouped W at a time inside one S-block: W must divide S
  if (axis > 0)
    while (a.W > 1 && (S % a.W)) a.W >>= 1;
  a.pad = 1;
  size_t smem = (size_t)a.W * (n + a.pad) * sizeof(VT);
  long grid = (a.nlines + a.W - 1) / a.W;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(fft_pass_kernel<VT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(fft_pass_kernel<VT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const double es = sizeof(VT);
  ProfScope ps(PROF_FFT, st);
  if (a.R == 3)
    fft_pass_kernel<VT, 3><<<(unsigned)grid, kThreads, smem, st>>>(a);
  else
    fft_pass_kernel<VT, 1><<<(unsigned)grid, kThreads, smem, st>>>(a);
  ps.done((double)N * nvec * (2 * es + (q ? es / 2 : 0.0) + (mode == 2 ? es / 2 : 0.0) +
                             (addx ? es : 0.0)),
          1, st);
  return cudaGetLastError();
}

template <class VT>
cudaError_t green_apply_t(int d, int n, const VT* tw, const typename Real<VT>::T* Dn,
                          VT* tmp, const VT* x, const typename Real<VT>::T* q, bool add_x, VT* out,
                          int nvec, int qper, cudaStream_t st) {
  cudaError_t e;
  // forward along axes 0..d-2, middle pass on axis d-1, inverse along d-2..0
  const VT* src = x;
  for (int ax = 0; ax < d - 1; ++ax) {
    e = run_pass<VT>(d, n, tw, Dn, ax, 0, src, tmp, ax == 0 ? q : nullptr, nullptr, nvec, qper, st);
    if (e != cudaSuccess) return e;
    src = tmp;
  }
  e = run_pass<VT>(d, n, tw, Dn, d - 1, 2, src, tmp, nullptr, nullptr, nvec, qper, st);
  if (e != cudaSuccess) return e;
  for (int ax = d - 2; ax >= 0; --ax) {
    bool last = (ax == 0);
    e = run_pass<VT>(d, n, tw, Dn, ax, 1, tmp, last ? out : tmp, nullptr,
                     (last && add_x) ? x : nullptr, nvec, qper, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

__global__ void to_float_kernel(const double* a, float* b, long N) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) b[i] = (float)a[i];
}

}  // namespace

cudaError_t fft_green_apply(const FftPlan& P, const double2* x, const double* q, bool add_x,
                            double2* out, cudaStream_t st, int nvec, int qper) {
  if (qper < 1 || nvec % qper) return cudaErrorInvalidValue;
  return green_apply_t<double2>(P.d, P.n, P.tw, P.Dn, P.tmp, x, q, add_x, out, nvec, qper, st);
}

cudaError_t fft_green_apply32(const FftPlan& P, const float2* x, const float* q, bool add_x,
                              float2* out, cudaStream_t st) {
  return green_apply_t<float2>(P.d, P.n, P.tw32, P.Dn32, P.tmp32, x, q, add_x, out, 1, 1, st);
}

cudaError_t to_float(const double* a, float* b, long N, cudaStream_t st) {
  to_float_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(a, b, N);
  return cudaGetLastError();
}

}  // namespace sp
