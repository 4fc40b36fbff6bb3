// FP64 Arnoldi / GMRES kernels (Saad and Schultz; the outer iteration of Section 2):
// classical Gram-Schmidt applied twice, norms, Givens rotations and the solution
// update.  Reductions are two-phase (per-CTA partials, then a fixed-order sum) so
// results are deterministic run to run.
#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kThr = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void chunk_of(long N, long* c0, long* c1) {
  long per = (N + gridDim.x - 1) / gridDim.x;
  *c0 = (long)blockIdx.x * per;
  *c1 = min(N, *c0 + per);
}

// The Krylov basis V is read with the evict-first hint (it is larger than L2 at
// 512^2 and streams through it every iteration), so the preconditioner's data stays.
// partial[j * nblk + blk] = sum over the CTA's chunk of conj(V_j) w.  Each thread
// walks its elements of the chunk with w[i] in registers and accumulates eight
// vectors at a time (independent FMA chains; w is re-read once per eight
// vectors, V once); the sums are reduced over the CTA in shared memory in a fixed
// order.
__device__ void chunk_dots(const double2* V, long ldv, int nv, const double2* w, long c0, long c1,
                           double2* partial) {
  constexpr int kJ = 8;
  __shared__ double2 red[kJ][kThr / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j0 = 0; j0 < nv; j0 += kJ) {
    const int nj = min(kJ, nv - j0);
    double sr[kJ], si[kJ];
#pragma unroll
    for (int q = 0; q < kJ; ++q) sr[q] = si[q] = 0.0;
    for (long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
      const double2 wi = w[i];
#pragma unroll
      for (int q = 0; q < kJ; ++q) {
        if (q < nj) {
          const double2 v = __ldcs(V + (long)(j0 + q) * ldv + i);  // conj(v) w; evict-first
          sr[q] = fma(v.x, wi.x, fma(v.y, wi.y, sr[q]));
          si[q] = fma(v.x, wi.y, fma(-v.y, wi.x, si[q]));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kJ; ++q) {
      const double a = warp_sum(sr[q]), b = warp_sum(si[q]);
      if (lane == 0) red[q][warp] = make_double2(a, b);
    }
    __syncthreads();
    if (threadIdx.x < nj) {
      double a = 0, b = 0;
      for (int x = 0; x < nw; ++x) {
        a += red[threadIdx.x][x].x;
        b += red[threadIdx.x][x].y;
      }
      partial[(long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = make_double2(a, b);
    }
    __syncthreads();
  }
}

// jdev != null: the vector count is *jdev + 1, read on the device (the
// device-resident iteration; nv is then only the launch bound).
__global__ void __launch_bounds__(kThr) dots_kernel(const double2* V, long ldv, int nv,
                                                    const double2* w, long N, double2* partial,
                                                    const int* jdev) {
  if (jdev) nv = *jdev + 1;
  long c0, c1;
  chunk_of(N, &c0, &c1);
  chunk_dots(V, ldv, nv, w, c0, c1, partial);
}

__global__ void __launch_bounds__(kThr) update_dots_kernel(const double2* V, long ldv, int nv,
                                                           double2* w, long N, const double2* h,
                                                           double2* partial, const int* jdev) {
  if (jdev) nv = *jdev + 1;
  __shared__ double2 hs[1024];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  long c0, c1;
  chunk_of(N, &c0, &c1);
  for (long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    // w_i - sum_j V_j[i] h_j with four independent partial sums (FP64 FMA latency)
    double ax[4] = {0, 0, 0, 0}, ay[4] = {0, 0, 0, 0};
    int j = 0;
    for (; j + 4 <= nv; j += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 v = __ldcs(V + (long)(j + q) * ldv + i), hj = hs[j + q];
        ax[q] = fma(v.x, hj.x, fma(-v.y, hj.y, ax[q]));
        ay[q] = fma(v.x, hj.y, fma(v.y, hj.x, ay[q]));
      }
    }
    for (; j < nv; ++j) {
      const double2 v = __ldcs(V + (long)j * ldv + i), hj = hs[j];
      ax[0] = fma(v.x, hj.x, fma(-v.y, hj.y, ax[0]));
      ay[0] = fma(v.x, hj.y, fma(v.y, hj.x, ay[0]));
    }
    const double2 wi = w[i];
    w[i] = make_double2(wi.x - ((ax[0] + ax[1]) + (ax[2] + ax[3])),
                        wi.y - ((ay[0] + ay[1]) + (ay[2] + ay[3])));
  }
  if (partial) {
    __syncthreads();
    chunk_dots(V, ldv, nv, w, c0, c1, partial);
  }
}

// out[j] = sum_b partial[j * nblk + b]  (one warp per j, fixed order)
__global__ void reduce_partials_kernel(const double2* partial, int nblk, int nv, double2* out,
                                       const int* jdev) {
  if (jdev) nv = *jdev + 1;
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= nv) return;
  double sr = 0, si = 0;
  for (int b = lane; b < nblk; b += 32) {
    double2 p = partial[(long)j * nblk + b];
    sr += p.x;
    si += p.y;
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  if (lane == 0) out[j] = make_double2(sr, si);
}

__global__ void __launch_bounds__(kThr) norm2_kernel(const double2* w, long N, double2* partial) {
  long c0, c1;
  chunk_of(N, &c0, &c1);
  double s = 0;
  for (long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    double2 v = w[i];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  __shared__ double red[kThr / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partial[blockIdx.x] = make_double2(t, 0);
  }
}

__global__ void sqrt_kernel(const double2* s, double* out) { out[0] = sqrt(s[0].x); }

__global__ void scale_kernel(const double2* x, long N, const double* nrm, double2* y) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double a = nrm[0] > 0 ? 1.0 / nrm[0] : 0.0;
  double2 v = x[i];
  y[i] = make_double2(v.x * a, v.y * a);
}

__global__ void sub_kernel(const double2* a, const double2* b, long N, double2* y) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  y[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void start_kernel(const double2* r, long N, const double* nrm, double2* V0, double2* gam,
                             int len) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double beta = nrm[0];
  if (i < N) {
    double a = beta > 0 ? 1.0 / beta : 0.0;
    V0[i] = make_double2(r[i].x * a, r[i].y * a);
  }
  if (i < len) gam[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
}

__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

// Column j of the Hessenberg matrix, earlier rotations, a new rotation, the
// residual estimate |gamma_{j+1}|.  Single thread.
__global__ void givens_kernel(double2* H, int ldh, int j, const double2* h1, const double2* h2,
                              const double* nrm, double* cs, double2* sn, double2* gam,
                              double* est, const int* jdev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (jdev) j = *jdev;
  double2* col = H + (long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
  col[j + 1] = make_double2(nrm[0], 0.0);
  for (int i = 0; i < j; ++i) {
    double c = cs[i];
    double2 s = sn[i], a = col[i], b = col[i + 1];
    // [c, s; -conj(s), c] (a, b)
    double2 t0 = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
    double2 t1 = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    col[i] = t0;
    col[i + 1] = t1;
  }
  double2 a = col[j], b = col[j + 1];
  double c;
  double2 s;
  double aa = cabs2(a), bb = cabs2(b);
  if (bb == 0.0) {
    c = 1.0;
    s = make_double2(0, 0);
  } else if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1, 0);
  } else {
    double r = hypot(aa, bb);
    c = aa / r;
    // s = (a/|a|) conj(b) / r
    double2 ua = make_double2(a.x / aa, a.y / aa);
    s = make_double2((ua.x * b.x + ua.y * b.y) / r, (ua.y * b.x - ua.x * b.y) / r);
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
  col[j + 1] = make_double2(0, 0);
  double2 g = gam[j];
  gam[j + 1] = make_double2(-(s.x * g.x + s.y * g.y), -(s.x * g.y - s.y * g.x));
  gam[j] = make_double2(c * g.x, c * g.y);
  est[0] = cabs2(gam[j + 1]);
  est[1] = nrm[0];
}

// y = R^{-1} gam (upper triangular, column-major, leading dimension ldh); one CTA
__global__ void trisolve_kernel(const double2* H, int ldh, int k, const double2* gam, double2* y,
                                const int* kdev) {
  if (kdev) k = *kdev;
  __shared__ double2 g[1024];
  for (int i = threadIdx.x; i < k; i += blockDim.x) g[i] = gam[i];
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    __shared__ double2 yj;
    if (threadIdx.x == 0) {
      double2 r = H[j + (long)j * ldh], v = g[j];
      double den = r.x * r.x + r.y * r.y;
      yj = make_double2((v.x * r.x + v.y * r.y) / den, (v.y * r.x - v.x * r.y) / den);
      y[j] = yj;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      double2 r = H[i + (long)j * ldh];
      g[i].x -= r.x * yj.x - r.y * yj.y;
      g[i].y -= r.x * yj.y + r.y * yj.x;
    }
    __syncthreads();
  }
}

__global__ void combine_kernel(const double2* Z, long ldz, int k, const double2* y, long N,
                               double2* u, const int* kdev) {
  if (kdev) k = *kdev;
  __shared__ double2 ys[1024];
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double2 acc = u[i];
  for (int j = 0; j < k; ++j) {
    double2 z = Z[(long)j * ldz + i], c = ys[j];
    acc.x += z.x * c.x - z.y * c.y;
    acc.y += z.x * c.y + z.y * c.x;
  }
  u[i] = acc;
}

}  // namespace

cudaError_t kr_dots(const double2* V, long ldv, int nv, const double2* w, long N, KrylovWork& K,
                    double2* h_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  dots_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv, w, N, K.partial, nullptr);
  reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h_out, nullptr);
  ps.done(16.0 * N * (nv + 1), 2, st);
  return cudaGetLastError();
}

cudaError_t kr_update_dots(const double2* V, long ldv, int nv, double2* w, long N,
                           const double2* h, KrylovWork& K, double2* h2_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  update_dots_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv, w, N, h, h2_out ? K.partial : nullptr,
                                              nullptr);
  if (h2_out)
    reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h2_out, nullptr);
  ps.done(16.0 * N * (nv + 2), h2_out ? 2 : 1, st);
  return cudaGetLastError();
}

cudaError_t kr_norm(const double2* w, long N, KrylovWork& K, double* nrm_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  norm2_kernel<<<K.nblk, kThr, 0, st>>>(w, N, K.partial);
  reduce_partials_kernel<<<1, 32, 0, st>>>(K.partial, K.nblk, 1, K.h + 1023, nullptr);
  sqrt_kernel<<<1, 1, 0, st>>>(K.h + 1023, nrm_out);
  ps.done(16.0 * N, 3, st);
  return cudaGetLastError();
}

cudaError_t kr_scale(const double2* x, long N, const double* nrm, double2* y, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  scale_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(x, N, nrm, y);
  ps.done(32.0 * N, 1, st);
  return cudaGetLastError();
}

cudaError_t kr_sub(const double2* a, const double2* b, long N, double2* y, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  sub_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(a, b, N, y);
  ps.done(48.0 * N, 1, st);
  return cudaGetLastError();
}

cudaError_t kr_givens(double2* H, int ldh, int j, const double2* h1, const double2* h2,
                      const double* nrm, double* cs, double2* sn, double2* gam, double* est,
                      cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  givens_kernel<<<1, 32, 0, st>>>(H, ldh, j, h1, h2, nrm, cs, sn, gam, est, nullptr);
  ps.done(0.0, 1, st);
  return cudaGetLastError();
}

cudaError_t kr_update_solution(const double2* H, int ldh, int k, const double2* gam, double2* y,
                               const double2* Z, long ldz, long N, double2* u, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  trisolve_kernel<<<1, 256, 0, st>>>(H, ldh, k, gam, y, nullptr);
  combine_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(Z, ldz, k, y, N, u, nullptr);
  ps.done(16.0 * N * (k + 2), 2, st);
  return cudaGetLastError();
}

cudaError_t kr_trisolve(const double2* H, int ldh, int k, const double2* gam, double2* y,
                        cudaStream_t st) {
  trisolve_kernel<<<1, 256, 0, st>>>(H, ldh, k, gam, y, nullptr);
  return cudaGetLastError();
}

cudaError_t kr_combine(const double2* Z, long ldz, int k, const double2* y, long N, double2* u,
                       cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  combine_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(Z, ldz, k, y, N, u, nullptr);
  ps.done(16.0 * N * (k + 2), 1, st);
  return cudaGetLastError();
}

cudaError_t kr_start(const double2* r, long N, const double* nrm, double2* V0, double2* gam,
                     int len, cudaStream_t st) {
  long n = N > len ? N : len;
  ProfScope ps(PROF_KRYLOV, st);
  start_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(r, N, nrm, V0, gam, len);
  ps.done(32.0 * N, 1, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Device-resident restart cycle: the Arnoldi step's column index j lives in device
// memory (LoopHead), every kernel of the step reads it there, and the stopping test
// runs on the device and ends the conditional (while) node of the CUDA graph that
// repeats the step, so a whole cycle runs without a host round trip.  The
// arithmetic is that of the host-driven iteration above, kernel for kernel.
namespace {

__global__ void loop_begin_kernel(LoopHead* h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    h->j = 0;
    h->cont = 1;
  }
}

// dst[j * dst_ld + i] = src[j * src_ld + i], j = *jp (an ld of 0: a fixed vector)
__global__ void copy_col_kernel(const double2* src, long src_ld, double2* dst, long dst_ld,
                                const int* jp, long N) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const long j = *jp;
  dst[j * dst_ld + i] = src[j * src_ld + i];
}

// One thread: count the iteration, record the estimate, and either advance j or
// stop the cycle (k columns) and end the while node.  The test is the host loop's:
// estimate <= tol, the iteration budget, a zero new column (breakdown) or a full
// basis.
__global__ void loop_step_kernel(LoopHead* h, double* hist, const double* est,
                                 const double* bnorm, double tol, int maxit, int restart,
                                 cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = h->j + 1, total = h->total + 1;
  const double rel = est[0] / bnorm[0];
  h->total = total;
  h->est_rel = rel;
  if (total <= maxit) hist[total - 1] = rel;
  if (rel <= tol || total >= maxit || est[1] == 0.0 || k == restart) {
    h->k = k;
    h->cont = 0;
    cudaGraphSetConditional(cond, 0);
  } else {
    h->j = k;
    h->cont = 1;
  }
}

// V[j] = w / nrm for the column the step advanced to (nothing when it stopped)
__global__ void loop_scale_kernel(const double2* w, long N, const double* nrm, double2* V,
                                  const LoopHead* h) {
  if (!h->cont) return;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double a = nrm[0] > 0 ? 1.0 / nrm[0] : 0.0;
  const double2 v = w[i];
  V[(long)h->j * N + i] = make_double2(v.x * a, v.y * a);
}

__global__ void loop_finish_kernel(LoopHead* h, const double* nrm) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    h->bnorm = nrm[2];
    h->rnorm = nrm[3];
  }
}

}  // namespace

cudaError_t kr_loop_begin(LoopHead* h, cudaStream_t st) {
  loop_begin_kernel<<<1, 32, 0, st>>>(h);
  return cudaGetLastError();
}

cudaError_t kr_copy_col(const double2* src, long src_ld, double2* dst, long dst_ld, const int* jp,
                        long N, cudaStream_t st) {
  copy_col_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(src, src_ld, dst, dst_ld, jp, N);
  return cudaGetLastError();
}

cudaError_t kr_dots_dev(const double2* V, long ldv, int nv_max, const int* jp, const double2* w,
                        long N, KrylovWork& K, double2* h_out, cudaStream_t st) {
  dots_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv_max, w, N, K.partial, jp);
  reduce_partials_kernel<<<(nv_max + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv_max, h_out, jp);
  return cudaGetLastError();
}

cudaError_t kr_update_dots_dev(const double2* V, long ldv, int nv_max, const int* jp, double2* w,
                               long N, const double2* h, KrylovWork& K, double2* h2_out,
                               cudaStream_t st) {
  update_dots_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv_max, w, N, h,
                                              h2_out ? K.partial : nullptr, jp);
  if (h2_out)
    reduce_partials_kernel<<<(nv_max + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv_max, h2_out,
                                                             jp);
  return cudaGetLastError();
}

cudaError_t kr_givens_dev(double2* H, int ldh, const int* jp, const double2* h1, const double2* h2,
                          const double* nrm, double* cs, double2* sn, double2* gam, double* est,
                          cudaStream_t st) {
  givens_kernel<<<1, 32, 0, st>>>(H, ldh, 0, h1, h2, nrm, cs, sn, gam, est, jp);
  return cudaGetLastError();
}

cudaError_t kr_loop_step(LoopHead* h, double* hist, const double* est, const double* bnorm,
                         double tol, int maxit, int restart, cudaGraphConditionalHandle cond,
                         cudaStream_t st) {
  loop_step_kernel<<<1, 32, 0, st>>>(h, hist, est, bnorm, tol, maxit, restart, cond);
  return cudaGetLastError();
}

cudaError_t kr_loop_scale(const double2* w, long N, const double* nrm, double2* V,
                          const LoopHead* h, cudaStream_t st) {
  loop_scale_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(w, N, nrm, V, h);
  return cudaGetLastError();
}

cudaError_t kr_update_solution_dev(const double2* H, int ldh, const int* kp, const double2* gam,
                                   double2* y, const double2* Z, long ldz, long N, double2* u,
                                   cudaStream_t st) {
  trisolve_kernel<<<1, 256, 0, st>>>(H, ldh, 0, gam, y, kp);
  combine_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(Z, ldz, 0, y, N, u, kp);
  return cudaGetLastError();
}

cudaError_t kr_loop_finish(LoopHead* h, const double* nrm, cudaStream_t st) {
  loop_finish_kernel<<<1, 32, 0, st>>>(h, nrm);
  return cudaGetLastError();
}

}  // namespace sp

// ---------------------------------------------------------------------------------
// FP32 vector kernels of the inner solve of the mixed-precision form (GMRES-IR):
// Krylov vectors in complex64, per-thread sums in FP32, everything from the warp
// reductions on in FP64, Hessenberg matrix and rotations in FP64 (the kernels
// above).
namespace sp {

namespace {

__device__ __forceinline__ void chunk_dots32(const float2* V, long ldv, int nv, const float2* w,
                                             long c0, long c1, double2* partial) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < nv; j += nw) {
    const float2* v = V + (long)j * ldv;
    float sr = 0.f, si = 0.f;
    for (long i = c0 + lane; i < c1; i += 32) {
      float2 a = v[i], b = w[i];
      sr = fmaf(a.x, b.x, fmaf(a.y, b.y, sr));
      si = fmaf(a.x, b.y, fmaf(-a.y, b.x, si));
    }
    double dr = warp_sum((double)sr), di = warp_sum((double)si);
    if (lane == 0) partial[(long)j * gridDim.x + blockIdx.x] = make_double2(dr, di);
  }
}

__global__ void __launch_bounds__(kThr) dots32_kernel(const float2* V, long ldv, int nv,
                                                      const float2* w, long N, double2* partial) {
  long c0, c1;
  chunk_of(N, &c0, &c1);
  chunk_dots32(V, ldv, nv, w, c0, c1, partial);
}

__global__ void __launch_bounds__(kThr) update_dots32_kernel(const float2* V, long ldv, int nv,
                                                             float2* w, long N, const double2* h,
                                                             double2* partial) {
  __shared__ float2 hs[1024];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) hs[j] = make_float2((float)h[j].x, (float)h[j].y);
  __syncthreads();
  long c0, c1;
  chunk_of(N, &c0, &c1);
  for (long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    float2 acc = w[i];
    for (int j = 0; j < nv; ++j) {
      float2 v = V[(long)j * ldv + i], hj = hs[j];
      acc.x -= fmaf(v.x, hj.x, -v.y * hj.y);
      acc.y -= fmaf(v.x, hj.y, v.y * hj.x);
    }
    w[i] = acc;
  }
  if (partial) {
    __syncthreads();
    chunk_dots32(V, ldv, nv, w, c0, c1, partial);
  }
}

__global__ void __launch_bounds__(kThr) norm32_kernel(const float2* w, long N, double2* partial) {
  long c0, c1;
  chunk_of(N, &c0, &c1);
  float s = 0.f;
  for (long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    float2 v = w[i];
    s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
  }
  __shared__ double red[kThr / 32];
  double ds = warp_sum((double)s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ds;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partial[blockIdx.x] = make_double2(t, 0);
  }
}

__global__ void scale32_kernel(float2* x, long N, const double* nrm) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float a = nrm[0] > 0 ? (float)(1.0 / nrm[0]) : 0.f;
  float2 v = x[i];
  x[i] = make_float2(v.x * a, v.y * a);
}

// y = x / nrm[0] rounded to complex64; gam = [1, 0, ...]
__global__ void start32_kernel(const double2* x, long N, const double* nrm, float2* y,
                               double2* gam, int len) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double a = nrm[0] > 0 ? 1.0 / nrm[0] : 0.0;
    y[i] = make_float2((float)(x[i].x * a), (float)(x[i].y * a));
  }
  if (i < len) gam[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
}

__global__ void widen_kernel(const float2* x, long N, double2* y) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) y[i] = make_double2(x[i].x, x[i].y);
}

__global__ void narrow_kernel(const double2* x, long N, float2* y) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

// y[0..k) *= s[0]
__global__ void scale_y_kernel(double2* y, int k, const double* s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) y[i] = make_double2(y[i].x * s[0], y[i].y * s[0]);
}

}  // namespace

cudaError_t kr32_dots(const float2* V, long ldv, int nv, const float2* w, long N, KrylovWork& K,
                      double2* h_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  dots32_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv, w, N, K.partial);
  reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h_out, nullptr);
  ps.done(8.0 * N * (nv + 1), 2, st);
  return cudaGetLastError();
}

cudaError_t kr32_update_dots(const float2* V, long ldv, int nv, float2* w, long N, const double2* h,
                             KrylovWork& K, double2* h2_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  update_dots32_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv, w, N, h, h2_out ? K.partial : nullptr);
  if (h2_out)
    reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h2_out, nullptr);
  ps.done(8.0 * N * (nv + 2), h2_out ? 2 : 1, st);
  return cudaGetLastError();
}

cudaError_t kr32_norm(const float2* w, long N, KrylovWork& K, double* nrm_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  norm32_kernel<<<K.nblk, kThr, 0, st>>>(w, N, K.partial);
  reduce_partials_kernel<<<1, 32, 0, st>>>(K.partial, K.nblk, 1, K.h + 1023, nullptr);
  sqrt_kernel<<<1, 1, 0, st>>>(K.h + 1023, nrm_out);
  ps.done(8.0 * N, 3, st);
  return cudaGetLastError();
}

cudaError_t kr32_scale(float2* x, long N, const double* nrm, cudaStream_t st) {
  scale32_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(x, N, nrm);
  return cudaGetLastError();
}

cudaError_t kr32_start(const double2* x, long N, const double* nrm, float2* y, double2* gam,
                       int len, cudaStream_t st) {
  long n = N > len ? N : len;
  start32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, N, nrm, y, gam, len);
  return cudaGetLastError();
}

cudaError_t kr_widen(const float2* x, long N, double2* y, cudaStream_t st) {
  widen_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(x, N, y);
  return cudaGetLastError();
}

cudaError_t kr_narrow(const double2* x, long N, float2* y, cudaStream_t st) {
  narrow_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(x, N, y);
  return cudaGetLastError();
}

cudaError_t kr_scale_y(double2* y, int k, const double* s, cudaStream_t st) {
  scale_y_kernel<<<(k + 255) / 256, 256, 0, st>>>(y, k, s);
  return cudaGetLastError();
}

}  // namespace sp
