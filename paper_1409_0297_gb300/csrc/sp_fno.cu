// Fourier-layer network for the learned initial guess of the solve: forward pass,
// backward pass, Adam, and the packing of features, guesses and targets.
//
// The network is the Fourier neural operator of Li et al. (ICLR 2021, Section 4):
// a pointwise lift, L Fourier layers v <- gelu(W v + b + K v) with K a truncated
// spectral convolution, and a two-layer pointwise projection; Adam follows Kingma and
// Ba (ICLR 2015, Algorithm 1).  Weights are used as bfloat16 (an FP32 master copy is
// updated by Adam), activations are stored as bfloat16 (or FP32 for checks) and every
// product accumulates in FP32.
//
// Layout: tensors [b][c][j0 + n j1].  The truncated transform keeps kx = 0..M-1 along
// axis 0 and ky in {0..M-1} U {n-M..n-1} along axis 1; it runs as two dense stages
// (rows: a real-to-complex DFT of each grid row onto M modes; columns: a complex DFT
// of each mode column onto 2M modes), each a small contraction against a twiddle
// table held in shared memory.  The inverse stage along rows is fused into the
// kernel that adds the pointwise branch, the bias and the activation, so the spatial
// output of the spectral branch never goes to memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <vector>

#include "sp_fno.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTP = 128;          // points per CTA of the pointwise kernels
constexpr int kRowsCta = 64;      // grid rows per CTA of the row transform
constexpr int kRowPitch = kRowsCta + 4;
constexpr int kWgChunk = 2048;    // points per CTA of the weight-gradient reduction
constexpr int kWgSub = 64;
constexpr int kLossChunks = 64;   // CTAs per sample of the loss reduction
constexpr int kNormBlocks = 256;

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

// gelu(x) = x Phi(x) and its derivative Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// ------------------------------------------------------------------ pointwise linear
// Y[b][o][p] = act(sum_i Wt(o, i) X[b][i][p] + bias[o]), optionally times
// gelu'(aux[b][o][p]).  Wt(o, i) = W[o ldw + i] (trans = 0) or W[i ldw + o] (trans = 1).
// gelu: pre (if not null) receives the value before the activation.
template <class TX, class TY, class TA>
__global__ void __launch_bounds__(kTP)
    chan_linear_kernel(const TX* __restrict__ X, int ci, const bf16* __restrict__ W, int ldw,
                       int trans, const bf16* __restrict__ bias, int co, long P, int gelu,
                       TY* __restrict__ pre, TY* __restrict__ Y, const TA* __restrict__ aux) {
  extern __shared__ float4 smf4[];
  float* sm = reinterpret_cast<float*>(smf4);
  const int co8 = (co + 7) & ~7;
  float* Ws = sm;             // [ci][co8]
  float* bs = Ws + ci * co8;  // [co8]
  float* Xs = bs + co8;       // [ci][kTP]
  for (int idx = threadIdx.x; idx < ci * co8; idx += kTP) {
    const int i = idx / co8, o = idx % co8;
    float w = 0.f;
    if (o < co) w = __bfloat162float(trans ? W[(long)i * ldw + o] : W[(long)o * ldw + i]);
    Ws[idx] = w;
  }
  for (int o = threadIdx.x; o < co8; o += kTP)
    bs[o] = (bias != nullptr && o < co) ? __bfloat162float(bias[o]) : 0.f;
  const int b = blockIdx.y;
  const long p = (long)blockIdx.x * kTP + threadIdx.x;
  const bool live = p < P;
  const TX* Xb = X + (long)b * ci * P;
  for (int i = 0; i < ci; ++i) Xs[i * kTP + threadIdx.x] = live ? ldf(Xb + (long)i * P + p) : 0.f;
  __syncthreads();
  if (!live) return;
  for (int o0 = 0; o0 < co; o0 += 8) {
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = bs[o0 + j];
    for (int i = 0; i < ci; ++i) {
      const float x = Xs[i * kTP + threadIdx.x];
      const float4 w0 = *reinterpret_cast<const float4*>(Ws + i * co8 + o0);
      const float4 w1 = *reinterpret_cast<const float4*>(Ws + i * co8 + o0 + 4);
      acc[0] = fmaf(w0.x, x, acc[0]);
      acc[1] = fmaf(w0.y, x, acc[1]);
      acc[2] = fmaf(w0.z, x, acc[2]);
      acc[3] = fmaf(w0.w, x, acc[3]);
      acc[4] = fmaf(w1.x, x, acc[4]);
      acc[5] = fmaf(w1.y, x, acc[5]);
      acc[6] = fmaf(w1.z, x, acc[6]);
      acc[7] = fmaf(w1.w, x, acc[7]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (o0 + j < co) {
        const long idx = ((long)b * co + o0 + j) * P + p;
        float v = acc[j];
        if (gelu) {
          if (pre != nullptr) stf(pre + idx, v);
          v = gelu_f(v);
        }
        if (aux != nullptr) v *= gelu_d(ldf(aux + idx));
        stf(Y + idx, v);
      }
    }
  }
}

// ------------------------------------------------------------------ weight gradients
// part[(b nchunk + chunk)][o ci + i] = sum over the chunk's points of dY[b][o][p] X[b][i][p],
// part[..][co ci + o] = sum dY[b][o][p].  Each thread owns a 4 x 4 block of (o, i).
// With Q2 != nullptr the rows are not read from dY but formed on the fly as the
// projection's hidden-layer gradient de[h][p] = (sum_o Q2[o][h] dY[o][p]) gelu'(E[h][p])
// (dY then has c2 channels, co = H), so de never goes to memory.
template <class TX, class TE>
__global__ void __launch_bounds__(256)
    chan_wgrad_kernel(const float* __restrict__ dY, int co, const TX* __restrict__ X, int ci,
                      long P, float* __restrict__ part, const TE* __restrict__ E,
                      const bf16* __restrict__ Q2, int c2) {
  extern __shared__ float4 smf4[];
  float* sm = reinterpret_cast<float*>(smf4);
  const int co4 = (co + 3) & ~3, ci4 = (ci + 3) & ~3;
  const int pco = co4 + 4, pci = ci4 + 4;
  float* sY = sm;                  // [kWgSub][pco]
  float* sX = sY + kWgSub * pco;   // [kWgSub][pci]
  float* sQ = sX + kWgSub * pci;   // [c2][co] (de mode)
  if (Q2 != nullptr)
    for (int idx = threadIdx.x; idx < c2 * co; idx += 256) sQ[idx] = __bfloat162float(Q2[idx]);
  const int nib = ci4 / 4, nblk = (co4 / 4) * nib;
  const int t = threadIdx.x;
  const int ob = t / nib, ib = t % nib;
  const bool owner = t < nblk;
  float acc[16];
  float accb[4];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) accb[j] = 0.f;
  const int b = blockIdx.y;
  const long c0 = (long)blockIdx.x * kWgChunk;
  const long c1 = c0 + kWgChunk < P ? c0 + kWgChunk : P;
  const float* Yb = dY + (long)b * co * P;
  const TX* Xb = X + (long)b * ci * P;
  __syncthreads();
  for (long s0 = c0; s0 < c1; s0 += kWgSub) {
    __syncthreads();
    if (Q2 == nullptr) {
      for (int idx = t; idx < co4 * kWgSub; idx += 256) {
        const int o = idx / kWgSub, q = idx % kWgSub;
        const long p = s0 + q;
        sY[q * pco + o] = (o < co && p < c1) ? Yb[(long)o * P + p] : 0.f;
      }
    } else {
      const float* Db = dY + (long)b * c2 * P;
      const TE* Eb = E + (long)b * co * P;
      for (int idx = t; idx < co4 * kWgSub; idx += 256) {
        const int h = idx / kWgSub, q = idx % kWgSub;
        const long p = s0 + q;
        float v = 0.f;
        if (h < co && p < c1) {
          for (int o = 0; o < c2; ++o) v = fmaf(sQ[o * co + h], Db[(long)o * P + p], v);
          v *= gelu_d(ldf(Eb + (long)h * P + p));
        }
        sY[q * pco + h] = v;
      }
    }
    for (int idx = t; idx < ci4 * kWgSub; idx += 256) {
      const int i = idx / kWgSub, q = idx % kWgSub;
      const long p = s0 + q;
      sX[q * pci + i] = (i < ci && p < c1) ? ldf(Xb + (long)i * P + p) : 0.f;
    }
    __syncthreads();
    if (owner) {
      for (int q = 0; q < kWgSub; ++q) {
        const float4 y = *reinterpret_cast<const float4*>(sY + q * pco + 4 * ob);
        const float4 x = *reinterpret_cast<const float4*>(sX + q * pci + 4 * ib);
        const float yv[4] = {y.x, y.y, y.z, y.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r * 4 + c] = fmaf(yv[r], xv[c], acc[r * 4 + c]);
          accb[r] += yv[r];
        }
      }
    }
  }
  if (owner) {
    float* out = part + ((long)b * gridDim.x + blockIdx.x) * (long)(co * ci + co);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int o = 4 * ob + r;
      if (o >= co) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = 4 * ib + c;
        if (i < ci) out[o * ci + i] = acc[r * 4 + c];
      }
      if (ib == 0) out[co * ci + o] = accb[r];
    }
  }
}

// Projection backward to the last layer's output: for every point,
// de_h = (sum_o Q2[o][h] dy_o) gelu'(e_h) and dv_i = sum_h Q1[h][i] de_h (H <= 128,
// W <= 32, c2 <= 8); de stays in registers.
template <class TA>
__global__ void __launch_bounds__(kTP)
    proj_bwd_kernel(const float* __restrict__ dy, int c2, const TA* __restrict__ e, int H,
                    const bf16* __restrict__ Q2, const bf16* __restrict__ Q1, int W, long P,
                    float* __restrict__ dv) {
  __shared__ __align__(16) float Q1s[128 * 32];  // [h][i], row pitch 32
  __shared__ float Q2s[8 * 128];                 // [o][h], row pitch 128
  for (int idx = threadIdx.x; idx < 128 * 32; idx += kTP) {
    const int h = idx >> 5, i = idx & 31;
    Q1s[idx] = (h < H && i < W) ? __bfloat162float(Q1[h * W + i]) : 0.f;
  }
  for (int idx = threadIdx.x; idx < 8 * 128; idx += kTP) {
    const int o = idx >> 7, h = idx & 127;
    Q2s[idx] = (o < c2 && h < H) ? __bfloat162float(Q2[o * H + h]) : 0.f;
  }
  __syncthreads();
  const int b = blockIdx.y;
  const long p = (long)blockIdx.x * kTP + threadIdx.x;
  if (p >= P) return;
  float d[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) d[o] = o < c2 ? dy[((long)b * c2 + o) * P + p] : 0.f;
  float acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0.f;
  const int W4 = (W + 3) >> 2;
  const TA* eb = e + (long)b * H * P + p;
  for (int h = 0; h < H; ++h) {
    float a = 0.f;
#pragma unroll
    for (int o = 0; o < 8; ++o) a = fmaf(Q2s[o * 128 + h], d[o], a);
    const float de = a * gelu_d(ldf(eb + (long)h * P));
    const float4* q = reinterpret_cast<const float4*>(Q1s + h * 32);
#pragma unroll
    for (int i4 = 0; i4 < 8; ++i4)
      if (i4 < W4) {
        const float4 w = q[i4];
        acc[4 * i4] = fmaf(w.x, de, acc[4 * i4]);
        acc[4 * i4 + 1] = fmaf(w.y, de, acc[4 * i4 + 1]);
        acc[4 * i4 + 2] = fmaf(w.z, de, acc[4 * i4 + 2]);
        acc[4 * i4 + 3] = fmaf(w.w, de, acc[4 * i4 + 3]);
      }
  }
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (i < W) dv[((long)b * W + i) * P + p] = acc[i];
}

// grad[j] = sum over the nparts partials (fixed order) of part[k][j], j < len
__global__ void sum_parts_kernel(const float* __restrict__ part, int nparts, int len,
                                 float* __restrict__ grad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  float s = 0.f;
  for (int k = 0; k < nparts; ++k) s += part[(long)k * len + j];
  grad[j] = s;
}

// ------------------------------------------------------------------ truncated DFT
// Rows: A[row][kx] = sum_j0 X[row][j0] e^{-2 pi i kx j0 / n}, row = (b C + c) n + j1.
// Thread (kx, row group of 4) with the rows staged transposed, x[j0][row].
template <class TX>
__global__ void __launch_bounds__(256)
    dft_rows_fwd_kernel(const TX* __restrict__ X, long rows, int n, int M,
                        const float2* __restrict__ twr, float2* __restrict__ A) {
  extern __shared__ float4 smf4[];
  float* xs = reinterpret_cast<float*>(smf4);                 // [n][kRowPitch]
  float2* tw = reinterpret_cast<float2*>(xs + n * kRowPitch);  // [n][16]
  const long r0 = (long)blockIdx.x * kRowsCta;
  const int t = threadIdx.x;
  for (int idx = t; idx < n * 16; idx += 256) tw[idx] = twr[idx];
  for (int idx = t; idx < n * (kRowsCta / 4); idx += 256) {
    const int j0 = idx % n, g = idx / n;
    const long r = r0 + 4 * g;
    float4 v;
    v.x = r + 0 < rows ? ldf(X + (r + 0) * n + j0) : 0.f;
    v.y = r + 1 < rows ? ldf(X + (r + 1) * n + j0) : 0.f;
    v.z = r + 2 < rows ? ldf(X + (r + 2) * n + j0) : 0.f;
    v.w = r + 3 < rows ? ldf(X + (r + 3) * n + j0) : 0.f;
    *reinterpret_cast<float4*>(xs + j0 * kRowPitch + 4 * g) = v;
  }
  __syncthreads();
  const int kx = t & 15, rg = t >> 4;
  if (kx >= M) return;
  float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < n; ++j0) {
    const float4 x = *reinterpret_cast<const float4*>(xs + j0 * kRowPitch + 4 * rg);
    const float2 w = tw[j0 * 16 + kx];
    ar[0] = fmaf(x.x, w.x, ar[0]);
    ai[0] = fmaf(x.x, w.y, ai[0]);
    ar[1] = fmaf(x.y, w.x, ar[1]);
    ai[1] = fmaf(x.y, w.y, ai[1]);
    ar[2] = fmaf(x.z, w.x, ar[2]);
    ai[2] = fmaf(x.z, w.y, ai[2]);
    ar[3] = fmaf(x.w, w.x, ar[3]);
    ai[3] = fmaf(x.w, w.y, ai[3]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long r = r0 + 4 * rg + q;
    if (r < rows) A[r * M + kx] = make_float2(ar[q], ai[q]);
  }
}

__device__ __forceinline__ int ky_of(int kq, int n, int M) { return kq < M ? kq : n - 2 * M + kq; }

// Columns: V[bc][ky'][kx] = s_kx sum_j1 A[bc][j1][kx] e^{-2 pi i ky j1 / n}
// (s_0 = s0, s_kx = s1 for kx >= 1); one CTA per (b, c).
__global__ void __launch_bounds__(256)
    dft_cols_fwd_kernel(const float2* __restrict__ A, int n, int M, const float2* __restrict__ twb,
                        float s0, float s1, float2* __restrict__ V) {
  extern __shared__ float4 smf4[];
  float2* As = reinterpret_cast<float2*>(smf4);  // [n][M]
  float2* tb = As + n * M;                        // [n]
  const long bc = blockIdx.x;
  const int t = threadIdx.x;
  for (int idx = t; idx < n * M; idx += 256) As[idx] = A[bc * n * M + idx];
  for (int idx = t; idx < n; idx += 256) tb[idx] = twb[idx];
  __syncthreads();
  const int kx = t & 15, g = t >> 4;
  if (kx >= M) return;
  const int K2 = 2 * M;
  const float s = kx == 0 ? s0 : s1;
  for (int kq = g; kq < K2; kq += 16) {
    const int ky = ky_of(kq, n, M);
    float re = 0.f, im = 0.f;
    int e = 0;
    for (int j1 = 0; j1 < n; ++j1) {
      const float2 a = As[j1 * M + kx], w = tb[e];
      re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
      im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
      e += ky;
      if (e >= n) e -= n;
    }
    V[(bc * K2 + kq) * M + kx] = make_float2(s * re, s * im);
  }
}

// Columns, inverse: Bc[bc][j1][kx] = sum_ky' Y[bc][ky'][kx] e^{+2 pi i ky j1 / n}.
// Thread (kx, g) owns the n / 16 rows j1 = g, g + 16, ...; the twiddle index of a mode
// advances by 16 ky (mod n) from one of its rows to the next.  n % 16 == 0.
__global__ void __launch_bounds__(256)
    dft_cols_inv_kernel(const float2* __restrict__ Y, int n, int M, const float2* __restrict__ twb,
                        float2* __restrict__ Bc) {
  extern __shared__ float4 smf4[];
  const int K2 = 2 * M;
  float2* Ys = reinterpret_cast<float2*>(smf4);  // [2M][M]
  float2* tb = Ys + K2 * M;                       // [n]
  const long bc = blockIdx.x;
  const int t = threadIdx.x;
  for (int idx = t; idx < K2 * M; idx += 256) Ys[idx] = Y[bc * K2 * M + idx];
  for (int idx = t; idx < n; idx += 256) tb[idx] = twb[idx];
  __syncthreads();
  const int kx = t & 15, g = t >> 4;
  if (kx >= M) return;
  const int R = n >> 4;  // rows per thread, <= 32
  float re[32], im[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) re[r] = im[r] = 0.f;
  for (int kq = 0; kq < K2; ++kq) {
    const int ky = ky_of(kq, n, M);
    const float2 y = Ys[kq * M + kx];
    int e = (int)(((long)ky * g) % n);
    const int step = (int)(((long)ky * 16) % n);
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (r < R) {
        const float2 w = tb[e];  // e^{+i theta} = conj(w)
        re[r] = fmaf(y.x, w.x, fmaf(y.y, w.y, re[r]));
        im[r] = fmaf(y.y, w.x, fmaf(-y.x, w.y, im[r]));
        e += step;
        if (e >= n) e -= n;
      }
  }
#pragma unroll
  for (int r = 0; r < 32; ++r)
    if (r < R) Bc[(bc * n + g + 16 * r) * M + kx] = make_float2(re[r], im[r]);
}

// Mode mixing: Y[b][o][k] = sum_i V[b][i][k] R[k][i][o]; one CTA per mode k.
__global__ void __launch_bounds__(256)
    spec_mix_kernel(const float2* __restrict__ V, const bf16* __restrict__ R, int B, int W, int K,
                    float2* __restrict__ Y) {
  extern __shared__ float4 smf4[];
  float2* Rs = reinterpret_cast<float2*>(smf4);  // [W][W]
  float2* Vs = Rs + W * W;                        // [B][W]
  const int k = blockIdx.x, t = threadIdx.x;
  const bf16* Rk = R + (long)k * W * W * 2;
  for (int idx = t; idx < W * W; idx += 256)
    Rs[idx] = make_float2(__bfloat162float(Rk[2 * idx]), __bfloat162float(Rk[2 * idx + 1]));
  for (int idx = t; idx < B * W; idx += 256) Vs[idx] = V[(long)idx * K + k];
  __syncthreads();
  for (int idx = t; idx < B * W; idx += 256) {
    const int b = idx / W, o = idx % W;
    float re = 0.f, im = 0.f;
    for (int i = 0; i < W; ++i) {
      const float2 v = Vs[b * W + i], r = Rs[i * W + o];
      re = fmaf(v.x, r.x, fmaf(-v.y, r.y, re));
      im = fmaf(v.x, r.y, fmaf(v.y, r.x, im));
    }
    Y[(long)idx * K + k] = make_float2(re, im);
  }
}

// Mode mixing, backward: dV[b][i][k] = sum_o dY[b][o][k] conj(R[k][i][o]) and
// dR[k][i][o] = sum_b dY[b][o][k] conj(V[b][i][k]) (written as (re, im) floats).
__global__ void __launch_bounds__(256)
    spec_mix_bwd_kernel(const float2* __restrict__ dY, const float2* __restrict__ V,
                        const bf16* __restrict__ R, int B, int W, int K, float2* __restrict__ dV,
                        float* __restrict__ dR) {
  extern __shared__ float4 smf4[];
  float2* Rs = reinterpret_cast<float2*>(smf4);  // [W][W]
  float2* Ds = Rs + W * W;                        // [B][W]
  float2* Vs = Ds + B * W;                        // [B][W]
  const int k = blockIdx.x, t = threadIdx.x;
  const bf16* Rk = R + (long)k * W * W * 2;
  for (int idx = t; idx < W * W; idx += 256)
    Rs[idx] = make_float2(__bfloat162float(Rk[2 * idx]), __bfloat162float(Rk[2 * idx + 1]));
  for (int idx = t; idx < B * W; idx += 256) {
    Ds[idx] = dY[(long)idx * K + k];
    Vs[idx] = V[(long)idx * K + k];
  }
  __syncthreads();
  for (int idx = t; idx < B * W; idx += 256) {
    const int b = idx / W, i = idx % W;
    float re = 0.f, im = 0.f;
    for (int o = 0; o < W; ++o) {
      const float2 d = Ds[b * W + o], r = Rs[i * W + o];
      re = fmaf(d.x, r.x, fmaf(d.y, r.y, re));
      im = fmaf(d.y, r.x, fmaf(-d.x, r.y, im));
    }
    dV[(long)idx * K + k] = make_float2(re, im);
  }
  float* dRk = dR + (long)k * W * W * 2;
  for (int idx = t; idx < W * W; idx += 256) {
    const int i = idx / W, o = idx % W;
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
      const float2 d = Ds[b * W + o], v = Vs[b * W + i];
      re = fmaf(d.x, v.x, fmaf(d.y, v.y, re));
      im = fmaf(d.y, v.x, fmaf(-d.x, v.y, im));
    }
    dRk[2 * idx] = re;
    dRk[2 * idx + 1] = im;
  }
}

// Layer output: out[b][o][j1][j0] = sum_i Wt(o, i) X[b][i][j1][j0] + bias[o]
//   + sum_kx w_kx Re(Bc[b][o][j1][kx] e^{+2 pi i kx j0 / n}),  w_0 = w0, w_kx = w1;
// with gelu, pre <- the value and out <- gelu(value).  One CTA per grid row (b, j1);
// a thread keeps its point's C inputs and M twiddles in registers and reads the
// weight row and the row's spectral coefficients as float4 broadcasts.  C <= 32, M <= 16.
template <class TX, class TY>
__global__ void __launch_bounds__(256)
    combine_kernel(const TX* __restrict__ X, int C, const bf16* __restrict__ W, int trans,
                   const bf16* __restrict__ bias, const float2* __restrict__ Bc, int n, int M,
                   const float2* __restrict__ twr, float w0, float w1, int gelu,
                   TY* __restrict__ pre, TY* __restrict__ out) {
  __shared__ __align__(16) float Ws[32 * 32];   // [o][i], row pitch 32
  __shared__ float bs[32];
  __shared__ __align__(16) float2 Bs[32 * 16];  // [o][kx], row pitch 16
  const int j1 = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
  for (int idx = t; idx < 32 * 32; idx += blockDim.x) {
    const int o = idx >> 5, i = idx & 31;
    float w = 0.f;
    if (o < C && i < C) w = __bfloat162float(trans ? W[i * C + o] : W[o * C + i]);
    Ws[idx] = w;
  }
  for (int o = t; o < 32; o += blockDim.x)
    bs[o] = (bias != nullptr && o < C) ? __bfloat162float(bias[o]) : 0.f;
  for (int idx = t; idx < 32 * 16; idx += blockDim.x) {
    const int o = idx >> 4, kx = idx & 15;
    Bs[idx] = (o < C && kx < M) ? Bc[(((long)b * C + o) * n + j1) * M + kx] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const long P = (long)n * n;
  const int C4 = (C + 3) >> 2, M2 = (M + 1) >> 1;
  for (int j0 = t; j0 < n; j0 += blockDim.x) {
    const long p = (long)j1 * n + j0;
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = i < C ? ldf(X + ((long)b * C + i) * P + p) : 0.f;
    float2 tw[16];
#pragma unroll
    for (int kx = 0; kx < 16; ++kx) {
      float2 w = kx < M ? twr[j0 * 16 + kx] : make_float2(0.f, 0.f);
      const float s = kx == 0 ? w0 : w1;
      tw[kx] = make_float2(s * w.x, s * w.y);
    }
    for (int o = 0; o < C; ++o) {
      float acc = bs[o];
      const float4* wr = reinterpret_cast<const float4*>(Ws + o * 32);
#pragma unroll
      for (int i4 = 0; i4 < 8; ++i4)
        if (i4 < C4) {
          const float4 w = wr[i4];
          acc = fmaf(w.x, x[4 * i4], acc);
          acc = fmaf(w.y, x[4 * i4 + 1], acc);
          acc = fmaf(w.z, x[4 * i4 + 2], acc);
          acc = fmaf(w.w, x[4 * i4 + 3], acc);
        }
      // Re(B e^{+i theta}) with tw = s e^{-i theta}
      const float4* br = reinterpret_cast<const float4*>(Bs + o * 16);
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2)
        if (k2 < M2) {
          const float4 bb = br[k2];
          acc = fmaf(bb.x, tw[2 * k2].x, fmaf(bb.y, tw[2 * k2].y, acc));
          acc = fmaf(bb.z, tw[2 * k2 + 1].x, fmaf(bb.w, tw[2 * k2 + 1].y, acc));
        }
      const long idx = ((long)b * C + o) * P + p;
      if (gelu) {
        if (pre != nullptr) stf(pre + idx, acc);
        acc = gelu_f(acc);
      }
      stf(out + idx, acc);
    }
  }
}

// dh = dv gelu'(h)
template <class TA>
__global__ void gelu_bwd_kernel(const float* __restrict__ dv, const TA* __restrict__ h, long len,
                                float* __restrict__ dh) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x)
    dh[i] = dv[i] * gelu_d(ldf(h + i));
}

// ------------------------------------------------------------------ loss
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// part[b][chunk] = (sum (y - t)^2, sum t^2) over one chunk of sample b's len values
__global__ void __launch_bounds__(256)
    loss_partial_kernel(const float* __restrict__ y, const float* __restrict__ t, long len,
                        double2* __restrict__ part) {
  __shared__ double red[8];
  const int b = blockIdx.y;
  const long per = (len + gridDim.x - 1) / gridDim.x;
  const long i0 = (long)blockIdx.x * per, i1 = i0 + per < len ? i0 + per : len;
  double s1 = 0.0, s2 = 0.0;
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double tv = t[(long)b * len + i], d = (double)y[(long)b * len + i] - tv;
    s1 += d * d;
    s2 += tv * tv;
  }
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) part[(long)b * gridDim.x + blockIdx.x] = make_double2(s1, s2);
}

// loss = mean_b S1_b / S2_b; scale[b] = 2 / (B S2_b) (the gradient factor); rel[b] = sqrt(S1/S2)
__global__ void loss_finish_kernel(const double2* __restrict__ part, int B, int nchunk,
                                   double* __restrict__ loss, float* __restrict__ scale) {
  if (threadIdx.x != 0) return;
  double L = 0.0;
  for (int b = 0; b < B; ++b) {
    double s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      s1 += part[(long)b * nchunk + c].x;
      s2 += part[(long)b * nchunk + c].y;
    }
    const double r = s2 > 0.0 ? s1 / s2 : 0.0;
    L += r;
    scale[b] = s2 > 0.0 ? (float)(2.0 / (B * s2)) : 0.f;
  }
  *loss = L / B;
}

__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ t, long len,
                                 int B, const float* __restrict__ scale, float* __restrict__ dy) {
  const long total = len * B;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    dy[i] = (y[i] - t[i]) * scale[i / len];
}

// ------------------------------------------------------------------ Adam
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, bf16* __restrict__ wb, long np, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * bc1) / (sqrtf(vi * bc2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, long np, bf16* __restrict__ wb) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

// ------------------------------------------------------------------ features / guess / target
// Per problem the complex scale c = sigma e^{i phi}, sigma = rms |g| and
// phi = arg(sum g^2) / 2: the solution is complex-linear in g, so dividing by c turns a
// source e^{i theta} r (r real, as every real-shaped source) into the real field +-r
// and the network meets the same problem whatever the source's phase.
__global__ void __launch_bounds__(256)
    norm_partial_kernel(const double2* __restrict__ g, long N, double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0, sr = 0.0, si = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double2 v = g[i];
    s += v.x * v.x + v.y * v.y;
    sr += v.x * v.x - v.y * v.y;
    si += 2.0 * v.x * v.y;
  }
  s = block_sum(s, red);
  sr = block_sum(sr, red);
  si = block_sum(si, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = s;
    part[3 * blockIdx.x + 1] = sr;
    part[3 * blockIdx.x + 2] = si;
  }
}

__global__ void scale_kernel(const double* __restrict__ part, int nb, long N, double2* __restrict__ c) {
  if (threadIdx.x != 0) return;
  double s = 0.0, sr = 0.0, si = 0.0;
  for (int i = 0; i < nb; ++i) {
    s += part[3 * i];
    sr += part[3 * i + 1];
    si += part[3 * i + 2];
  }
  const double sigma = sqrt(s / (double)N);
  const double phi = (sr == 0.0 && si == 0.0) ? 0.0 : 0.5 * atan2(si, sr);
  *c = make_double2(sigma * cos(phi), sigma * sin(phi));
}

// 1 / c (0 for c = 0)
__device__ __forceinline__ double2 inv_scale(double2 c) {
  const double m = c.x * c.x + c.y * c.y;
  return m > 0.0 ? make_double2(c.x / m, -c.y / m) : make_double2(0.0, 0.0);
}

__global__ void features_kernel(const double* __restrict__ q, double qs, const double2* __restrict__ g,
                                const double2* __restrict__ c, long N, float* __restrict__ x) {
  const double2 ic = inv_scale(*c);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double2 v = g[i];
    x[i] = (float)(qs * q[i]);
    x[N + i] = (float)(v.x * ic.x - v.y * ic.y);
    x[2 * N + i] = (float)(v.x * ic.y + v.y * ic.x);
  }
}

__global__ void guess_kernel(const float* __restrict__ y, const double2* __restrict__ c, long N,
                             double2* __restrict__ u0) {
  const double2 cc = *c;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double yr = y[i], yi = y[N + i];
    u0[i] = make_double2(cc.x * yr - cc.y * yi, cc.x * yi + cc.y * yr);
  }
}

__global__ void target_kernel(const double2* __restrict__ u, const double2* __restrict__ c, long N,
                              float* __restrict__ t) {
  const double2 ic = inv_scale(*c);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double2 v = u[i];
    t[i] = (float)(v.x * ic.x - v.y * ic.y);
    t[N + i] = (float)(v.x * ic.y + v.y * ic.x);
  }
}

// the same with a prior estimate z of the solution (the preconditioner applied to g):
// x[3] + i x[4] = z / c; the guess adds the network's correction to z, the target is
// the correction (u - z) / c
__global__ void features_prior_kernel(const double2* __restrict__ z, const double2* __restrict__ c,
                                      long N, float* __restrict__ x) {
  const double2 ic = inv_scale(*c);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double2 v = z[i];
    x[3 * N + i] = (float)(v.x * ic.x - v.y * ic.y);
    x[4 * N + i] = (float)(v.x * ic.y + v.y * ic.x);
  }
}

__global__ void guess_prior_kernel(const float* __restrict__ y, const double2* __restrict__ c,
                                   const double2* __restrict__ z, long N, double2* __restrict__ u0) {
  const double2 cc = *c;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double yr = y[i], yi = y[N + i];
    const double2 zi = z[i];
    u0[i] = make_double2(zi.x + (cc.x * yr - cc.y * yi), zi.y + (cc.x * yi + cc.y * yr));
  }
}

__global__ void target_prior_kernel(const double2* __restrict__ u, const double2* __restrict__ c,
                                    const double2* __restrict__ z, long N, float* __restrict__ t) {
  const double2 ic = inv_scale(*c);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double2 v = make_double2(u[i].x - z[i].x, u[i].y - z[i].y);
    t[i] = (float)(v.x * ic.x - v.y * ic.y);
    t[N + i] = (float)(v.x * ic.y + v.y * ic.x);
  }
}

unsigned grid_for(long len, int threads) {
  long g = (len + threads - 1) / threads;
  if (g > 152L * 16) g = 152L * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

bool dims_ok(const sp_fno_dims* D) {
  return D && D->n >= 64 && D->n <= 512 && D->n % 64 == 0 && D->c_in >= 1 && D->c_in <= 32 &&
         D->width >= 1 && D->width <= 32 && D->modes >= 1 && D->modes <= 16 &&
         2 * D->modes <= D->n && D->layers >= 1 && D->layers <= 8 && D->hidden >= 1 &&
         D->hidden <= 128 && D->c_out >= 1 && D->c_out <= 8 && D->batch_max >= 1 &&
         D->batch_max <= 256 && (D->act_fp32 == 0 || D->act_fp32 == 1);
}

long long count_params(const sp_fno_dims* D) {
  const long long W = D->width, M = D->modes;
  long long n = W * D->c_in + W;
  n += D->layers * (2 * M * M * W * W * 2 + W * W + W);
  n += (long long)D->hidden * W + D->hidden + (long long)D->c_out * D->hidden + D->c_out;
  return n;
}

}  // namespace

struct sp_fno {
  sp_fno_dims D{};
  cudaStream_t st = nullptr;
  long long np = 0;
  long P = 0;
  int K = 0;
  long long offP = 0, offQ1 = 0, offQ2 = 0;
  std::vector<long long> offR, offW;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  bf16* wb = nullptr;
  long long step = 0;
  float2 *twr = nullptr, *twb = nullptr;
  std::vector<void*> vv, hh;
  void *e = nullptr, *ge = nullptr;
  std::vector<float2*> Vh;
  float2 *A = nullptr, *Yh = nullptr, *dVh = nullptr, *Bc = nullptr;
  float *y = nullptr, *dy = nullptr, *dv[2] = {nullptr, nullptr}, *dh = nullptr;
  float *part = nullptr, *lscale = nullptr;
  double2* lpart = nullptr;
  double *dloss = nullptr, *npart = nullptr, *hloss = nullptr;
  std::vector<void*> allocs;
  ~sp_fno() {
    for (void* p : allocs) cudaFree(p);
    if (hloss) cudaFreeHost(hloss);
  }
};

namespace {

template <class T>
cudaError_t dalloc(sp_fno* f, T** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return e;
  f->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return cudaSuccess;
}

sp_status cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return SP_OK;
  if (e == cudaErrorMemoryAllocation) return SP_ERR_OOM;
  return SP_ERR_CUDA;
}

#define FNO_CK(x)                        \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return cuda_st(e_); \
  } while (0)

constexpr size_t kLinSmemMax = (128 * kTP + 128 * 128 + 128) * sizeof(float);
constexpr size_t kWgSmemMax = ((size_t)kWgSub * (132 + 132) + 8 * 128) * sizeof(float);
constexpr size_t kRowsSmemMax = 512 * kRowPitch * sizeof(float) + 512 * 16 * sizeof(float2);
constexpr size_t kColsSmemMax = (512 * 16 + 512) * sizeof(float2);

template <class TA>
cudaError_t set_attrs(int mixB, int W) {
  cudaError_t e;
  const size_t mix = (size_t)(W * W + 2 * mixB * W) * sizeof(float2);
  if ((e = cudaFuncSetAttribute(chan_linear_kernel<float, TA, TA>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(chan_linear_kernel<TA, TA, TA>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(chan_linear_kernel<TA, float, TA>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(chan_wgrad_kernel<TA, float>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(chan_wgrad_kernel<TA, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kWgSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(chan_wgrad_kernel<float, float>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(dft_rows_fwd_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kRowsSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(dft_rows_fwd_kernel<float>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowsSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(dft_cols_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kColsSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(dft_cols_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kColsSmemMax))) return e;
  if ((e = cudaFuncSetAttribute(spec_mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mix))) return e;
  return cudaFuncSetAttribute(spec_mix_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mix);
}

template <class TX, class TY, class TA>
void linear(sp_fno* f, int B, const TX* X, int ci, const bf16* W, int ldw, int trans,
            const bf16* bias, int co, int gelu, TY* pre, TY* Y, const TA* aux) {
  const int co8 = (co + 7) & ~7;
  const size_t smem = (size_t)(ci * co8 + co8 + ci * kTP) * sizeof(float);
  dim3 grid((unsigned)((f->P + kTP - 1) / kTP), (unsigned)B);
  chan_linear_kernel<TX, TY, TA><<<grid, kTP, smem, f->st>>>(X, ci, W, ldw, trans, bias, co, f->P,
                                                             gelu, pre, Y, aux);
}

// gradient of a pointwise layer's weight [co][ci] and bias [co] (adjacent in the
// parameter vector at off)
template <class TX, class TE = float>
void wgrad(sp_fno* f, int B, const float* dY, int co, const TX* X, int ci, long long off,
           const TE* E = nullptr, const bf16* Q2 = nullptr, int c2 = 0) {
  const int nchunk = (int)((f->P + kWgChunk - 1) / kWgChunk);
  const int co4 = (co + 3) & ~3, ci4 = (ci + 3) & ~3;
  const size_t smem = ((size_t)kWgSub * (co4 + 4 + ci4 + 4) + (size_t)c2 * co) * sizeof(float);
  chan_wgrad_kernel<TX, TE><<<dim3((unsigned)nchunk, (unsigned)B), 256, smem, f->st>>>(
      dY, co, X, ci, f->P, f->part, E, Q2, c2);
  const int len = co * ci + co;
  sum_parts_kernel<<<(len + 255) / 256, 256, 0, f->st>>>(f->part, B * nchunk, len, f->g + off);
}

template <class TX>
void dft_forward(sp_fno* f, int B, const TX* X, float s0, float s1, float2* V) {
  const int n = f->D.n, M = f->D.modes, C = f->D.width;
  const long rows = (long)B * C * n;
  const size_t rs = (size_t)n * kRowPitch * sizeof(float) + (size_t)n * 16 * sizeof(float2);
  dft_rows_fwd_kernel<TX><<<(unsigned)((rows + kRowsCta - 1) / kRowsCta), 256, rs, f->st>>>(
      X, rows, n, M, f->twr, f->A);
  const size_t cs = (size_t)(n * M + n) * sizeof(float2);
  dft_cols_fwd_kernel<<<(unsigned)(B * C), 256, cs, f->st>>>(f->A, n, M, f->twb, s0, s1, V);
}

void dft_cols_inverse(sp_fno* f, int B, const float2* Y) {
  const int n = f->D.n, M = f->D.modes, C = f->D.width;
  const size_t cs = (size_t)(2 * M * M + n) * sizeof(float2);
  dft_cols_inv_kernel<<<(unsigned)(B * C), 256, cs, f->st>>>(Y, n, M, f->twb, f->Bc);
}

template <class TA>
cudaError_t forward_t(sp_fno* f, int B, const float* x) {
  const sp_fno_dims& D = f->D;
  const int W = D.width, L = D.layers, n = D.n;
  const bf16* wb = f->wb;
  linear<float, TA, TA>(f, B, x, D.c_in, wb + f->offP, D.c_in, 0, wb + f->offP + (long long)W * D.c_in,
                        W, 0, nullptr, (TA*)f->vv[0], (const TA*)nullptr);
  const float inv2 = 1.f / ((float)n * (float)n);
  for (int l = 0; l < L; ++l) {
    dft_forward<TA>(f, B, (const TA*)f->vv[l], 1.f, 1.f, f->Vh[l]);
    const size_t ms = (size_t)(W * W + B * W) * sizeof(float2);
    spec_mix_kernel<<<f->K, 256, ms, f->st>>>(f->Vh[l], wb + f->offR[l], B, W, f->K, f->Yh);
    dft_cols_inverse(f, B, f->Yh);
    const bool act = l < L - 1;
    const bf16* Wl = wb + f->offW[l];
    combine_kernel<TA, TA><<<dim3((unsigned)n, (unsigned)B), 256, 0, f->st>>>(
        (const TA*)f->vv[l], W, Wl, 0, Wl + W * W, f->Bc, n, D.modes, f->twr, inv2, 2.f * inv2,
        act ? 1 : 0, act ? (TA*)f->hh[l] : (TA*)nullptr, (TA*)f->vv[l + 1]);
  }
  const int H = D.hidden;
  linear<TA, TA, TA>(f, B, (const TA*)f->vv[L], W, wb + f->offQ1, W, 0, wb + f->offQ1 + (long long)H * W,
                     H, 1, (TA*)f->e, (TA*)f->ge, (const TA*)nullptr);
  linear<TA, float, TA>(f, B, (const TA*)f->ge, H, wb + f->offQ2, H, 0,
                        wb + f->offQ2 + (long long)D.c_out * H, D.c_out, 0, (float*)nullptr, f->y,
                        (const TA*)nullptr);
  return cudaGetLastError();
}

template <class TA>
cudaError_t backward_t(sp_fno* f, int B, const float* x, const float* t) {
  const sp_fno_dims& D = f->D;
  const int W = D.width, L = D.layers, n = D.n, H = D.hidden, co = D.c_out;
  const bf16* wb = f->wb;
  const long len = (long)co * f->P;
  loss_partial_kernel<<<dim3(kLossChunks, (unsigned)B), 256, 0, f->st>>>(f->y, t, len, f->lpart);
  loss_finish_kernel<<<1, 32, 0, f->st>>>(f->lpart, B, kLossChunks, f->dloss, f->lscale);
  loss_grad_kernel<<<grid_for(len * B, 256), 256, 0, f->st>>>(f->y, t, len, B, f->lscale, f->dy);
  // projection: dQ2 from (dy, gelu(e)); dQ1 and dv from de = (Q2^T dy) gelu'(e), formed
  // on the fly in both kernels
  wgrad<TA>(f, B, f->dy, co, (const TA*)f->ge, H, f->offQ2);
  wgrad<TA, TA>(f, B, f->dy, H, (const TA*)f->vv[L], W, f->offQ1, (const TA*)f->e, wb + f->offQ2, co);
  int cur = 0;
  proj_bwd_kernel<TA><<<dim3((unsigned)((f->P + kTP - 1) / kTP), (unsigned)B), kTP, 0, f->st>>>(
      f->dy, co, (const TA*)f->e, H, wb + f->offQ2, wb + f->offQ1, W, f->P, f->dv[cur]);
  const float inv2 = 1.f / ((float)n * (float)n);
  const long act_len = (long)B * W * f->P;
  for (int l = L - 1; l >= 0; --l) {
    const float* dhp = f->dv[cur];
    if (l < L - 1) {
      gelu_bwd_kernel<TA><<<grid_for(act_len, 256), 256, 0, f->st>>>(f->dv[cur], (const TA*)f->hh[l],
                                                                      act_len, f->dh);
      dhp = f->dh;
    }
    wgrad<TA>(f, B, dhp, W, (const TA*)f->vv[l], W, f->offW[l]);
    // spectral branch: dY = w_kx DFT(dh), dV = dY conj(R), dR = dY conj(V), dv += Re IDFT(dV)
    dft_forward<float>(f, B, dhp, inv2, 2.f * inv2, f->Yh);
    const size_t ms = (size_t)(W * W + 2 * B * W) * sizeof(float2);
    spec_mix_bwd_kernel<<<f->K, 256, ms, f->st>>>(f->Yh, f->Vh[l], wb + f->offR[l], B, W, f->K, f->dVh,
                                                  f->g + f->offR[l]);
    dft_cols_inverse(f, B, f->dVh);
    const int nxt = cur ^ 1;
    combine_kernel<float, float><<<dim3((unsigned)n, (unsigned)B), 256, 0, f->st>>>(
        dhp, W, wb + f->offW[l], 1, nullptr, f->Bc, n, D.modes, f->twr, 1.f, 1.f, 0, (float*)nullptr,
        f->dv[nxt]);
    cur = nxt;
  }
  wgrad<float>(f, B, f->dv[cur], W, x, D.c_in, f->offP);  // lift
  return cudaGetLastError();
}

sp_status run_forward(sp_fno* f, int B, const float* x) {
  return cuda_st(f->D.act_fp32 ? forward_t<float>(f, B, x) : forward_t<bf16>(f, B, x));
}

sp_status run_backward(sp_fno* f, int B, const float* x, const float* t) {
  return cuda_st(f->D.act_fp32 ? backward_t<float>(f, B, x, t) : backward_t<bf16>(f, B, x, t));
}

}  // namespace

extern "C" {

long long sp_fno_param_count(const sp_fno_dims* dims) {
  return dims_ok(dims) ? count_params(dims) : 0;
}

}  // extern "C"

namespace {

// Everything sp_fno_create does after allocating the handle: sizes, device buffers,
// twiddles and the parameters.  On failure the caller deletes f, which frees every
// device buffer recorded so far.
sp_status fno_init(sp_fno* f, const sp_fno_dims* dims, const float* params_host, void* stream) {
  f->D = *dims;
  f->st = (cudaStream_t)stream;
  const sp_fno_dims& D = f->D;
  const int W = D.width, M = D.modes, L = D.layers, n = D.n, H = D.hidden, B = D.batch_max;
  f->np = count_params(&D);
  f->P = (long)n * n;
  f->K = 2 * M * M;
  long long off = 0;
  f->offP = off;
  off += (long long)W * D.c_in + W;
  for (int l = 0; l < L; ++l) {
    f->offR.push_back(off);
    off += 2LL * f->K * W * W;
    f->offW.push_back(off);
    off += (long long)W * W + W;
  }
  f->offQ1 = off;
  off += (long long)H * W + H;
  f->offQ2 = off;
  const size_t es = D.act_fp32 ? sizeof(float) : sizeof(bf16);
  const size_t act = (size_t)B * W * f->P * es;
  cudaError_t e = cudaSuccess;
  f->allocs.reserve((size_t)3 * L + 32);  // every dalloc below records without reallocating
  auto fail = [](cudaError_t err) { return cuda_st(err); };
  if ((e = dalloc(f, &f->w, f->np * sizeof(float))) || (e = dalloc(f, &f->m, f->np * sizeof(float))) ||
      (e = dalloc(f, &f->v, f->np * sizeof(float))) || (e = dalloc(f, &f->g, f->np * sizeof(float))) ||
      (e = dalloc(f, &f->wb, f->np * sizeof(bf16))) ||
      (e = dalloc(f, &f->twr, (size_t)n * 16 * sizeof(float2))) ||
      (e = dalloc(f, &f->twb, (size_t)n * sizeof(float2))))
    return fail(e);
  f->vv.assign(L + 1, nullptr);
  f->hh.assign(L, nullptr);
  f->Vh.assign(L, nullptr);
  for (int l = 0; l <= L; ++l)
    if ((e = dalloc(f, &f->vv[l], act))) return fail(e);
  for (int l = 0; l < L; ++l)
    if ((e = dalloc(f, &f->hh[l], act)) || (e = dalloc(f, &f->Vh[l], (size_t)B * W * f->K * sizeof(float2))))
      return fail(e);
  const int nchunk = (int)((f->P + kWgChunk - 1) / kWgChunk);
  long long plen = (long long)W * D.c_in + W;
  plen = std::max(plen, (long long)W * W + W);
  plen = std::max(plen, (long long)H * W + H);
  plen = std::max(plen, (long long)D.c_out * H + D.c_out);
  if ((e = dalloc(f, &f->e, (size_t)B * H * f->P * es)) || (e = dalloc(f, &f->ge, (size_t)B * H * f->P * es)) ||
      (e = dalloc(f, &f->A, (size_t)B * W * n * M * sizeof(float2))) ||
      (e = dalloc(f, &f->Bc, (size_t)B * W * n * M * sizeof(float2))) ||
      (e = dalloc(f, &f->Yh, (size_t)B * W * f->K * sizeof(float2))) ||
      (e = dalloc(f, &f->dVh, (size_t)B * W * f->K * sizeof(float2))) ||
      (e = dalloc(f, &f->y, (size_t)B * D.c_out * f->P * sizeof(float))) ||
      (e = dalloc(f, &f->dy, (size_t)B * D.c_out * f->P * sizeof(float))) ||
      (e = dalloc(f, &f->dv[0], (size_t)B * W * f->P * sizeof(float))) ||
      (e = dalloc(f, &f->dv[1], (size_t)B * W * f->P * sizeof(float))) ||
      (e = dalloc(f, &f->dh, (size_t)B * W * f->P * sizeof(float))) ||
      (e = dalloc(f, &f->part, (size_t)B * nchunk * plen * sizeof(float))) ||
      (e = dalloc(f, &f->lpart, (size_t)B * kLossChunks * sizeof(double2))) ||
      (e = dalloc(f, &f->lscale, (size_t)B * sizeof(float))) || (e = dalloc(f, &f->dloss, sizeof(double))) ||
      (e = dalloc(f, &f->npart, (size_t)3 * kNormBlocks * sizeof(double))))
    return fail(e);
  if ((e = cudaMallocHost(&f->hloss, sizeof(double)))) return fail(e);
  if ((e = D.act_fp32 ? set_attrs<float>(B, W) : set_attrs<bf16>(B, W))) return fail(e);
  // twiddles e^{-2 pi i m / n}, with the product kx j0 reduced mod n before the angle
  std::vector<float2> twr((size_t)n * 16), twb(n);
  const double tau = 6.283185307179586476925286766559;
  for (int j0 = 0; j0 < n; ++j0)
    for (int kx = 0; kx < 16; ++kx) {
      const double a = tau * (double)((long)kx * j0 % n) / n;
      twr[(size_t)j0 * 16 + kx] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
  for (int mm = 0; mm < n; ++mm) {
    const double a = tau * mm / n;
    twb[mm] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  if ((e = cudaMemcpyAsync(f->twr, twr.data(), twr.size() * sizeof(float2), cudaMemcpyHostToDevice, f->st)) ||
      (e = cudaMemcpyAsync(f->twb, twb.data(), twb.size() * sizeof(float2), cudaMemcpyHostToDevice, f->st)) ||
      (e = cudaStreamSynchronize(f->st)))
    return fail(e);
  return sp_fno_set_params(f, params_host);
}

}  // namespace

extern "C" {

sp_status sp_fno_create(const sp_fno_dims* dims, const float* params_host, void* stream,
                        sp_fno** out) {
  if (!out || !params_host || !dims_ok(dims)) return SP_ERR_ARG;
  *out = nullptr;
  sp_fno* f = new (std::nothrow) sp_fno;
  if (!f) return SP_ERR_OOM;
  sp_status s;
  try {
    s = fno_init(f, dims, params_host, stream);
  } catch (const std::exception&) {  // host memory: no exception crosses the ABI
    s = SP_ERR_OOM;
  }
  if (s != SP_OK) {
    delete f;
    return s;
  }
  *out = f;
  return SP_OK;
}

void sp_fno_destroy(sp_fno* f) {
  if (!f) return;
  cudaStreamSynchronize(f->st);
  delete f;
}

sp_status sp_fno_set_params(sp_fno* f, const float* params_host) {
  if (!f || !params_host) return SP_ERR_ARG;
  FNO_CK(cudaMemcpyAsync(f->w, params_host, f->np * sizeof(float), cudaMemcpyHostToDevice, f->st));
  FNO_CK(cudaMemsetAsync(f->m, 0, f->np * sizeof(float), f->st));
  FNO_CK(cudaMemsetAsync(f->v, 0, f->np * sizeof(float), f->st));
  to_bf16_kernel<<<grid_for(f->np, 256), 256, 0, f->st>>>(f->w, f->np, f->wb);
  FNO_CK(cudaGetLastError());
  f->step = 0;
  return cuda_st(cudaStreamSynchronize(f->st));
}

sp_status sp_fno_get_params(sp_fno* f, float* params_host) {
  if (!f || !params_host) return SP_ERR_ARG;
  FNO_CK(cudaMemcpyAsync(params_host, f->w, f->np * sizeof(float), cudaMemcpyDeviceToHost, f->st));
  return cuda_st(cudaStreamSynchronize(f->st));
}

sp_status sp_fno_forward(sp_fno* f, int batch, const float* x_dev, float* y_dev) {
  if (!f || !x_dev || !y_dev || batch < 1 || batch > f->D.batch_max) return SP_ERR_ARG;
  sp_status s = run_forward(f, batch, x_dev);
  if (s != SP_OK) return s;
  return cuda_st(cudaMemcpyAsync(y_dev, f->y, (size_t)batch * f->D.c_out * f->P * sizeof(float),
                                 cudaMemcpyDeviceToDevice, f->st));
}

sp_status sp_fno_gradient(sp_fno* f, int batch, const float* x_dev, const float* t_dev, float* y_dev,
                          double* loss_host, float* grad_host) {
  if (!f || !x_dev || !t_dev || batch < 1 || batch > f->D.batch_max) return SP_ERR_ARG;
  sp_status s = run_forward(f, batch, x_dev);
  if (s == SP_OK) s = run_backward(f, batch, x_dev, t_dev);
  if (s != SP_OK) return s;
  if (y_dev)
    FNO_CK(cudaMemcpyAsync(y_dev, f->y, (size_t)batch * f->D.c_out * f->P * sizeof(float),
                           cudaMemcpyDeviceToDevice, f->st));
  if (grad_host)
    FNO_CK(cudaMemcpyAsync(grad_host, f->g, f->np * sizeof(float), cudaMemcpyDeviceToHost, f->st));
  FNO_CK(cudaMemcpyAsync(f->hloss, f->dloss, sizeof(double), cudaMemcpyDeviceToHost, f->st));
  FNO_CK(cudaStreamSynchronize(f->st));
  if (loss_host) *loss_host = *f->hloss;
  return SP_OK;
}

sp_status sp_fno_train_step(sp_fno* f, int batch, const float* x_dev, const float* t_dev,
                            const sp_adam* opt, double* loss_host) {
  if (!f || !x_dev || !t_dev || !opt || batch < 1 || batch > f->D.batch_max || !(opt->lr > 0.0) ||
      !(opt->beta1 >= 0.0 && opt->beta1 < 1.0) || !(opt->beta2 >= 0.0 && opt->beta2 < 1.0) ||
      !(opt->eps > 0.0))
    return SP_ERR_ARG;
  sp_status s = run_forward(f, batch, x_dev);
  if (s == SP_OK) s = run_backward(f, batch, x_dev, t_dev);
  if (s != SP_OK) return s;
  f->step += 1;
  const double bc1 = 1.0 / (1.0 - std::pow(opt->beta1, (double)f->step));
  const double bc2 = 1.0 / (1.0 - std::pow(opt->beta2, (double)f->step));
  adam_kernel<<<grid_for(f->np, 256), 256, 0, f->st>>>(f->w, f->m, f->v, f->g, f->wb, f->np,
                                                       (float)opt->lr, (float)opt->beta1,
                                                       (float)opt->beta2, (float)opt->eps, (float)bc1,
                                                       (float)bc2);
  FNO_CK(cudaGetLastError());
  if (loss_host) {
    FNO_CK(cudaMemcpyAsync(f->hloss, f->dloss, sizeof(double), cudaMemcpyDeviceToHost, f->st));
    FNO_CK(cudaStreamSynchronize(f->st));
    *loss_host = *f->hloss;
  }
  return SP_OK;
}

sp_status sp_fno_features(sp_fno* f, const double* q_dev, double q_scale, const void* g_dev,
                          float* x_dev, void* scale_dev) {
  if (!f || !q_dev || !g_dev || !x_dev || !scale_dev || f->D.c_in != 3) return SP_ERR_ARG;
  const long N = f->P;
  norm_partial_kernel<<<kNormBlocks, 256, 0, f->st>>>((const double2*)g_dev, N, f->npart);
  scale_kernel<<<1, 32, 0, f->st>>>(f->npart, kNormBlocks, N, (double2*)scale_dev);
  features_kernel<<<grid_for(N, 256), 256, 0, f->st>>>(q_dev, q_scale, (const double2*)g_dev,
                                                       (const double2*)scale_dev, N, x_dev);
  return cuda_st(cudaGetLastError());
}

sp_status sp_fno_features_prior(sp_fno* f, const double* q_dev, double q_scale, const void* g_dev,
                                const void* z_dev, float* x_dev, void* scale_dev) {
  if (!f || !q_dev || !g_dev || !z_dev || !x_dev || !scale_dev || f->D.c_in != 5) return SP_ERR_ARG;
  const long N = f->P;
  norm_partial_kernel<<<kNormBlocks, 256, 0, f->st>>>((const double2*)g_dev, N, f->npart);
  scale_kernel<<<1, 32, 0, f->st>>>(f->npart, kNormBlocks, N, (double2*)scale_dev);
  features_kernel<<<grid_for(N, 256), 256, 0, f->st>>>(q_dev, q_scale, (const double2*)g_dev,
                                                       (const double2*)scale_dev, N, x_dev);
  features_prior_kernel<<<grid_for(N, 256), 256, 0, f->st>>>((const double2*)z_dev,
                                                             (const double2*)scale_dev, N, x_dev);
  return cuda_st(cudaGetLastError());
}

sp_status sp_fno_guess_prior(sp_fno* f, const float* y_dev, const void* scale_dev, const void* z_dev,
                             void* u0_dev) {
  if (!f || !y_dev || !scale_dev || !z_dev || !u0_dev || f->D.c_out != 2) return SP_ERR_ARG;
  guess_prior_kernel<<<grid_for(f->P, 256), 256, 0, f->st>>>(
      y_dev, (const double2*)scale_dev, (const double2*)z_dev, f->P, (double2*)u0_dev);
  return cuda_st(cudaGetLastError());
}

sp_status sp_fno_target_prior(sp_fno* f, const void* u_dev, const void* scale_dev, const void* z_dev,
                              float* t_dev) {
  if (!f || !u_dev || !scale_dev || !z_dev || !t_dev || f->D.c_out != 2) return SP_ERR_ARG;
  target_prior_kernel<<<grid_for(f->P, 256), 256, 0, f->st>>>(
      (const double2*)u_dev, (const double2*)scale_dev, (const double2*)z_dev, f->P, t_dev);
  return cuda_st(cudaGetLastError());
}

sp_status sp_fno_guess(sp_fno* f, const float* y_dev, const void* scale_dev, void* u0_dev) {
  if (!f || !y_dev || !scale_dev || !u0_dev || f->D.c_out != 2) return SP_ERR_ARG;
  guess_kernel<<<grid_for(f->P, 256), 256, 0, f->st>>>(y_dev, (const double2*)scale_dev, f->P,
                                                       (double2*)u0_dev);
  return cuda_st(cudaGetLastError());
}

sp_status sp_fno_target(sp_fno* f, const void* u_dev, const void* scale_dev, float* t_dev) {
  if (!f || !u_dev || !scale_dev || !t_dev || f->D.c_out != 2) return SP_ERR_ARG;
  target_kernel<<<grid_for(f->P, 256), 256, 0, f->st>>>((const double2*)u_dev, (const double2*)scale_dev,
                                                        f->P, t_dev);
  return cuda_st(cudaGetLastError());
}

}  // extern "C"
