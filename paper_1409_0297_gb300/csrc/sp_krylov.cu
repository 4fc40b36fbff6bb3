// FP64 Arnoldi / GMRES kernels (Saad and Schultz; the outer iteration of Section 2):
// classical Gram-Schmidt applied twice, norms, Givens rotations and the solution
// update.  Reductions are two-phase (per-CTA partials, then a fixed-order sum) so
// results are deterministic run to run.  Each step exists twice: for one Krylov
// process with its column index passed by the host, and batched over the instances
// of a KBatch (blockIdx.y = instance) with each instance's column index and state in
// device memory; both call the same device functions, so an instance of the
// batched form computes the bits the single form computes.
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

// w_i -= sum_j V_j[i] hs_j over the chunk, four independent partial sums (FP64 FMA
// latency); hs in shared memory
__device__ void chunk_update(const double2* V, long ldv, int nv, double2* w, long c0, long c1,
                             const double2* hs) {
  for (long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
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
}

// partial[blockIdx.x] = (sum over the chunk of |w_i|^2, 0)
__device__ void chunk_norm2(const double2* w, long c0, long c1, double2* partial) {
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

// sum_b partial[j * nblk + b] in a fixed order; called by one whole warp
__device__ double2 warp_reduce_partial(const double2* partial, int nblk, int j) {
  const int lane = threadIdx.x & 31;
  double sr = 0, si = 0;
  for (int b = lane; b < nblk; b += 32) {
    double2 p = partial[(long)j * nblk + b];
    sr += p.x;
    si += p.y;
  }
  return make_double2(warp_sum(sr), warp_sum(si));
}

__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }

// Column j of the Hessenberg matrix, earlier rotations, a new rotation, the
// residual estimate |gamma_{j+1}|.  Single thread.
__device__ void givens_col(double2* H, int ldh, int j, const double2* h1, const double2* h2,
                           double nrm, double* cs, double2* sn, double2* gam, double* est) {
  double2* col = H + (long)j * ldh;
  for (int i = 0; i <= j; ++i) col[i] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
  col[j + 1] = make_double2(nrm, 0.0);
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
  est[1] = nrm;
}

// y = R^{-1} gam (upper triangular, column-major, leading dimension ldh); one CTA
__device__ void trisolve_cta(const double2* H, int ldh, int k, const double2* gam, double2* y) {
  __shared__ double2 g[1024];
  __shared__ double2 yj;
  for (int i = threadIdx.x; i < k; i += blockDim.x) g[i] = gam[i];
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
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

// u[i] += sum_j Z_j[i] ys_j
__device__ __forceinline__ void combine_at(const double2* Z, long ldz, int k, const double2* ys,
                                           long i, double2* u) {
  double2 acc = u[i];
  for (int j = 0; j < k; ++j) {
    double2 z = Z[(long)j * ldz + i], c = ys[j];
    acc.x += z.x * c.x - z.y * c.y;
    acc.y += z.x * c.y + z.y * c.x;
  }
  u[i] = acc;
}

// ---- one Krylov process

__global__ void __launch_bounds__(kThr) dots_kernel(const double2* V, long ldv, int nv,
                                                    const double2* w, long N, double2* partial) {
  long c0, c1;
  chunk_of(N, &c0, &c1);
  chunk_dots(V, ldv, nv, w, c0, c1, partial);
}

__global__ void __launch_bounds__(kThr) update_dots_kernel(const double2* V, long ldv, int nv,
                                                           double2* w, long N, const double2* h,
                                                           double2* partial) {
  __shared__ double2 hs[1024];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  long c0, c1;
  chunk_of(N, &c0, &c1);
  chunk_update(V, ldv, nv, w, c0, c1, hs);
  if (partial) {
    __syncthreads();
    chunk_dots(V, ldv, nv, w, c0, c1, partial);
  }
}

// out[j] = sum_b partial[j * nblk + b]  (one warp per j, fixed order)
__global__ void reduce_partials_kernel(const double2* partial, int nblk, int nv, double2* out) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= nv) return;
  const double2 s = warp_reduce_partial(partial, nblk, j);
  if ((threadIdx.x & 31) == 0) out[j] = s;
}

__global__ void __launch_bounds__(kThr) norm2_kernel(const double2* w, long N, double2* partial) {
  long c0, c1;
  chunk_of(N, &c0, &c1);
  chunk_norm2(w, c0, c1, partial);
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

__device__ __forceinline__ void start_at(const double2* r, long N, double beta, double2* V0,
                                         double2* gam, int len, long i) {
  if (i < N) {
    double a = beta > 0 ? 1.0 / beta : 0.0;
    V0[i] = make_double2(r[i].x * a, r[i].y * a);
  }
  if (i < len) gam[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
}

__global__ void start_kernel(const double2* r, long N, const double* nrm, double2* V0, double2* gam,
                             int len) {
  start_at(r, N, nrm[0], V0, gam, len, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void givens_kernel(double2* H, int ldh, int j, const double2* h1, const double2* h2,
                              const double* nrm, double* cs, double2* sn, double2* gam,
                              double* est) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  givens_col(H, ldh, j, h1, h2, nrm[0], cs, sn, gam, est);
}

__global__ void trisolve_kernel(const double2* H, int ldh, int k, const double2* gam, double2* y) {
  trisolve_cta(H, ldh, k, gam, y);
}

__global__ void combine_kernel(const double2* Z, long ldz, int k, const double2* y, long N,
                               double2* u) {
  __shared__ double2 ys[1024];
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  combine_at(Z, ldz, k, ys, i, u);
}

// ---- batched over the instances of a KBatch (blockIdx.y or the thread = instance).
// An instance takes part in the Arnoldi steps while head.cont is set and in the
// cycle's start and solution update when run is set.

__device__ __forceinline__ bool inst_cont(const KBatch& b, int i) { return b.head[i].cont != 0; }

__global__ void kb_begin_kernel(KBatch b, int I) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  b.head[i].j = 0;
  b.head[i].cont = b.run[i];
}

__global__ void kb_start_kernel(KBatch b, const double2* r, int len) {
  const int i = blockIdx.y;
  if (!b.run[i]) return;
  start_at(r + i * b.N, b.N, b.nrm[i * 4 + 3], b.V + i * b.sV, b.gam + i * b.sG, len,
           (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// dst_i = V_i[j_i] (to_z = 0) or Z_i[j_i] = src_i (to_z = 1)
__global__ void kb_copy_kernel(KBatch b, double2* vec, int to_z) {
  const int i = blockIdx.y;
  if (!inst_cont(b, i)) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b.N) return;
  const long j = b.head[i].j;
  if (to_z)
    b.Z[i * b.sZ + j * b.N + e] = vec[i * b.N + e];
  else
    vec[i * b.N + e] = b.V[i * b.sV + j * b.N + e];
}

__global__ void __launch_bounds__(kThr) kb_dots_kernel(KBatch b) {
  const int i = blockIdx.y;
  if (!inst_cont(b, i)) return;
  long c0, c1;
  chunk_of(b.N, &c0, &c1);
  chunk_dots(b.V + i * b.sV, b.N, b.head[i].j + 1, b.w + i * b.N, c0, c1, b.partial + i * b.sP);
}

// w_i -= V_i h_i (h = h1 if second = 0, else h2); then, if second = 0, h2 = V_i^H w_i
// partials
__global__ void __launch_bounds__(kThr) kb_update_dots_kernel(KBatch b, int second) {
  const int i = blockIdx.y;
  if (!inst_cont(b, i)) return;
  const int nv = b.head[i].j + 1;
  const double2* h = (second ? b.h2 : b.h1) + i * b.sh;
  __shared__ double2 hs[1024];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  long c0, c1;
  chunk_of(b.N, &c0, &c1);
  const double2* V = b.V + i * b.sV;
  double2* w = b.w + i * b.N;
  chunk_update(V, b.N, nv, w, c0, c1, hs);
  if (!second) {
    __syncthreads();
    chunk_dots(V, b.N, nv, w, c0, c1, b.partial + i * b.sP);
  }
}

// out_i[j] = sum_b partial_i[j * nblk + b] for j <= j_i (out = h1 if which = 0, else h2)
__global__ void kb_reduce_kernel(KBatch b, int which) {
  const int i = blockIdx.y;
  if (!inst_cont(b, i)) return;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j > b.head[i].j) return;
  const double2 s = warp_reduce_partial(b.partial + i * b.sP, b.nblk, j);
  if ((threadIdx.x & 31) == 0) (which ? b.h2 : b.h1)[i * b.sh + j] = s;
}

// partials of |x_i|^2 (x with instance stride N); active = 1: only instances in a step
__global__ void __launch_bounds__(kThr) kb_norm2_kernel(KBatch b, const double2* x, int active) {
  const int i = blockIdx.y;
  if (active && !inst_cont(b, i)) return;
  long c0, c1;
  chunk_of(b.N, &c0, &c1);
  chunk_norm2(x + i * b.N, c0, c1, b.partial + i * b.sP);
}

// nrm_i[slot] = sqrt(sum of the partials); one warp per instance
__global__ void kb_norm_finish_kernel(KBatch b, int slot, int active) {
  const int i = blockIdx.x;
  if (active && !inst_cont(b, i)) return;
  const double2 s = warp_reduce_partial(b.partial + i * b.sP, b.nblk, 0);
  if (threadIdx.x == 0) b.nrm[i * 4 + slot] = sqrt(s.x);
}

__global__ void kb_givens_kernel(KBatch b) {
  const int i = blockIdx.x;
  if (threadIdx.x != 0 || !inst_cont(b, i)) return;
  givens_col(b.H + i * b.sH, b.ldh, b.head[i].j, b.h1 + i * b.sh, b.h2 + i * b.sh, b.nrm[i * 4],
             b.cs + i * b.sG, b.sn + i * b.sG, b.gam + i * b.sG, b.est + i * 4);
}

// One thread per instance: count the iteration, record the estimate, and either
// advance j or stop the instance's cycle (k columns).  The test is the host loop's:
// estimate <= tol, the iteration budget, a zero new column (breakdown) or a full
// basis.  When no instance goes on, the while node ends.
__global__ void kb_step_kernel(KBatch b, int I, double* hist, int hstride, double tol, int maxit,
                               int restart, cudaGraphConditionalHandle cond) {
  const int i = threadIdx.x;
  int goes_on = 0;
  if (i < I && b.head[i].cont) {
    LoopHead* h = b.head + i;
    const double* est = b.est + i * 4;
    const int k = h->j + 1, total = h->total + 1;
    const double rel = est[0] / b.nrm[i * 4 + 2];
    h->total = total;
    h->est_rel = rel;
    if (total <= maxit) hist[(long)i * hstride + total - 1] = rel;
    if (rel <= tol || total >= maxit || est[1] == 0.0 || k == restart) {
      h->k = k;
      h->cont = 0;
    } else {
      h->j = k;
      goes_on = 1;
    }
  }
  if (!__syncthreads_or(goes_on) && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
}

// V_i[j_i] = w_i / nrm_i for the instances that advanced
__global__ void kb_scale_kernel(KBatch b) {
  const int i = blockIdx.y;
  if (!inst_cont(b, i)) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b.N) return;
  const double nrm = b.nrm[i * 4];
  const double a = nrm > 0 ? 1.0 / nrm : 0.0;
  const double2 v = b.w[i * b.N + e];
  b.V[i * b.sV + (long)b.head[i].j * b.N + e] = make_double2(v.x * a, v.y * a);
}

__global__ void kb_trisolve_kernel(KBatch b) {
  const int i = blockIdx.x;
  if (!b.run[i]) return;
  trisolve_cta(b.H + i * b.sH, b.ldh, b.head[i].k, b.gam + i * b.sG, b.y + i * b.sh);
}

__global__ void kb_combine_kernel(KBatch b, double2* U) {
  const int i = blockIdx.y;
  if (!b.run[i]) return;
  const int k = b.head[i].k;
  __shared__ double2 ys[1024];
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = b.y[i * b.sh + j];
  __syncthreads();
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b.N) return;
  combine_at(b.Z + i * b.sZ, b.N, k, ys, e, U + i * b.N);
}

__global__ void kb_finish_kernel(KBatch b, int I) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  b.head[i].bnorm = b.nrm[i * 4 + 2];
  b.head[i].rnorm = b.nrm[i * 4 + 3];
}

// nrm_i[to] = nrm_i[from]
__global__ void kb_copy_nrm_kernel(KBatch b, int I, int from, int to) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < I) b.nrm[i * 4 + to] = b.nrm[i * 4 + from];
}

inline unsigned blocks_of(long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t kr_dots(const double2* V, long ldv, int nv, const double2* w, long N, KrylovWork& K,
                    double2* h_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  dots_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv, w, N, K.partial);
  reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h_out);
  ps.done(16.0 * N * (nv + 1), 2, st);
  return cudaGetLastError();
}

cudaError_t kr_update_dots(const double2* V, long ldv, int nv, double2* w, long N,
                           const double2* h, KrylovWork& K, double2* h2_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  update_dots_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv, w, N, h, h2_out ? K.partial : nullptr);
  if (h2_out) reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h2_out);
  ps.done(16.0 * N * (nv + 2), h2_out ? 2 : 1, st);
  return cudaGetLastError();
}

cudaError_t kr_norm(const double2* w, long N, KrylovWork& K, double* nrm_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  norm2_kernel<<<K.nblk, kThr, 0, st>>>(w, N, K.partial);
  reduce_partials_kernel<<<1, 32, 0, st>>>(K.partial, K.nblk, 1, K.h + 1023);
  sqrt_kernel<<<1, 1, 0, st>>>(K.h + 1023, nrm_out);
  ps.done(16.0 * N, 3, st);
  return cudaGetLastError();
}

cudaError_t kr_scale(const double2* x, long N, const double* nrm, double2* y, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  scale_kernel<<<blocks_of(N), 256, 0, st>>>(x, N, nrm, y);
  ps.done(32.0 * N, 1, st);
  return cudaGetLastError();
}

cudaError_t kr_sub(const double2* a, const double2* b, long N, double2* y, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  sub_kernel<<<blocks_of(N), 256, 0, st>>>(a, b, N, y);
  ps.done(48.0 * N, 1, st);
  return cudaGetLastError();
}

cudaError_t kr_givens(double2* H, int ldh, int j, const double2* h1, const double2* h2,
                      const double* nrm, double* cs, double2* sn, double2* gam, double* est,
                      cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  givens_kernel<<<1, 32, 0, st>>>(H, ldh, j, h1, h2, nrm, cs, sn, gam, est);
  ps.done(0.0, 1, st);
  return cudaGetLastError();
}

cudaError_t kr_update_solution(const double2* H, int ldh, int k, const double2* gam, double2* y,
                               const double2* Z, long ldz, long N, double2* u, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  trisolve_kernel<<<1, 256, 0, st>>>(H, ldh, k, gam, y);
  combine_kernel<<<blocks_of(N), 256, 0, st>>>(Z, ldz, k, y, N, u);
  ps.done(16.0 * N * (k + 2), 2, st);
  return cudaGetLastError();
}

cudaError_t kr_trisolve(const double2* H, int ldh, int k, const double2* gam, double2* y,
                        cudaStream_t st) {
  trisolve_kernel<<<1, 256, 0, st>>>(H, ldh, k, gam, y);
  return cudaGetLastError();
}

cudaError_t kr_combine(const double2* Z, long ldz, int k, const double2* y, long N, double2* u,
                       cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  combine_kernel<<<blocks_of(N), 256, 0, st>>>(Z, ldz, k, y, N, u);
  ps.done(16.0 * N * (k + 2), 1, st);
  return cudaGetLastError();
}

cudaError_t kr_start(const double2* r, long N, const double* nrm, double2* V0, double2* gam,
                     int len, cudaStream_t st) {
  long n = N > len ? N : len;
  ProfScope ps(PROF_KRYLOV, st);
  start_kernel<<<blocks_of(n), 256, 0, st>>>(r, N, nrm, V0, gam, len);
  ps.done(32.0 * N, 1, st);
  return cudaGetLastError();
}

// ---- batched

cudaError_t kb_begin(const KBatch& b, int I, cudaStream_t st) {
  kb_begin_kernel<<<blocks_of(I), 256, 0, st>>>(b, I);
  return cudaGetLastError();
}

cudaError_t kb_start(const KBatch& b, int I, const double2* r, int len, cudaStream_t st) {
  const long n = b.N > len ? b.N : len;
  kb_start_kernel<<<dim3(blocks_of(n), I), 256, 0, st>>>(b, r, len);
  return cudaGetLastError();
}

cudaError_t kb_copy_in(const KBatch& b, int I, double2* dst, cudaStream_t st) {
  kb_copy_kernel<<<dim3(blocks_of(b.N), I), 256, 0, st>>>(b, dst, 0);
  return cudaGetLastError();
}

cudaError_t kb_copy_out(const KBatch& b, int I, const double2* src, cudaStream_t st) {
  kb_copy_kernel<<<dim3(blocks_of(b.N), I), 256, 0, st>>>(b, const_cast<double2*>(src), 1);
  return cudaGetLastError();
}

cudaError_t kb_arnoldi(const KBatch& b, int I, int nv_max, cudaStream_t st) {
  const dim3 gd(b.nblk, I), gr((nv_max + 7) / 8, I);
  // classical Gram-Schmidt, twice
  kb_dots_kernel<<<gd, kThr, 0, st>>>(b);
  kb_reduce_kernel<<<gr, 256, 0, st>>>(b, 0);
  kb_update_dots_kernel<<<gd, kThr, 0, st>>>(b, 0);
  kb_reduce_kernel<<<gr, 256, 0, st>>>(b, 1);
  kb_update_dots_kernel<<<gd, kThr, 0, st>>>(b, 1);
  kb_norm2_kernel<<<gd, kThr, 0, st>>>(b, b.w, 1);
  kb_norm_finish_kernel<<<I, 32, 0, st>>>(b, 0, 1);
  kb_givens_kernel<<<I, 32, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t kb_norm(const KBatch& b, int I, const double2* x, int slot, cudaStream_t st) {
  kb_norm2_kernel<<<dim3(b.nblk, I), kThr, 0, st>>>(b, x, 0);
  kb_norm_finish_kernel<<<I, 32, 0, st>>>(b, slot, 0);
  return cudaGetLastError();
}

cudaError_t kb_step(const KBatch& b, int I, double* hist, int hstride, double tol, int maxit,
                    int restart, cudaGraphConditionalHandle cond, cudaStream_t st) {
  if (I > 1024) return cudaErrorInvalidValue;
  kb_step_kernel<<<1, (I + 31) / 32 * 32, 0, st>>>(b, I, hist, hstride, tol, maxit, restart, cond);
  kb_scale_kernel<<<dim3(blocks_of(b.N), I), 256, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t kb_update_solution(const KBatch& b, int I, double2* U, cudaStream_t st) {
  kb_trisolve_kernel<<<I, 256, 0, st>>>(b);
  kb_combine_kernel<<<dim3(blocks_of(b.N), I), 256, 0, st>>>(b, U);
  return cudaGetLastError();
}

cudaError_t kb_finish(const KBatch& b, int I, cudaStream_t st) {
  kb_finish_kernel<<<blocks_of(I), 256, 0, st>>>(b, I);
  return cudaGetLastError();
}

cudaError_t kb_copy_nrm(const KBatch& b, int I, int from, int to, cudaStream_t st) {
  kb_copy_nrm_kernel<<<blocks_of(I), 256, 0, st>>>(b, I, from, to);
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
  reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h_out);
  ps.done(8.0 * N * (nv + 1), 2, st);
  return cudaGetLastError();
}

cudaError_t kr32_update_dots(const float2* V, long ldv, int nv, float2* w, long N, const double2* h,
                             KrylovWork& K, double2* h2_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  update_dots32_kernel<<<K.nblk, kThr, 0, st>>>(V, ldv, nv, w, N, h, h2_out ? K.partial : nullptr);
  if (h2_out) reduce_partials_kernel<<<(nv + 7) / 8, 256, 0, st>>>(K.partial, K.nblk, nv, h2_out);
  ps.done(8.0 * N * (nv + 2), h2_out ? 2 : 1, st);
  return cudaGetLastError();
}

cudaError_t kr32_norm(const float2* w, long N, KrylovWork& K, double* nrm_out, cudaStream_t st) {
  ProfScope ps(PROF_KRYLOV, st);
  norm32_kernel<<<K.nblk, kThr, 0, st>>>(w, N, K.partial);
  reduce_partials_kernel<<<1, 32, 0, st>>>(K.partial, K.nblk, 1, K.h + 1023);
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
