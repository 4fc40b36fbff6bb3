// C ABI of the library (include/sp.h): context set-up (single problems and problem
// groups), factorisation, preconditioner application and the GMRES driver.  Every
// vector operation is a device kernel.  By default a GMRES restart cycle is one CUDA
// graph whose Arnoldi step repeats under a conditional while node, the stopping test
// on the device, and the host reads the cycle's outcome once (the true residual
// decides a restart); with device_loop = 0 the host reads two scalars per iteration
// (the Givens estimate and the new Arnoldi norm) to decide whether to stop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <memory>
#include <new>
#include <vector>

#include "sp_internal.h"

using namespace sp;

namespace sp {
thread_local Profiler* g_prof = nullptr;

cudaEvent_t Profiler::get() {
  if (used < pool.size()) return pool[used++];
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  pool.push_back(e);
  ++used;
  return e;
}
int Profiler::begin(int cls, cudaStream_t st) {
  Rec r{cls, get(), get(), 0.0, 0};
  cudaEventRecord(r.a, st);
  recs.push_back(r);
  return (int)recs.size() - 1;
}
void Profiler::end(int tok, double work, int launches, cudaStream_t st) {
  Rec& r = recs[tok];
  r.work = work;
  r.launches = launches;
  cudaEventRecord(r.b, st);
}
cudaError_t Profiler::read(double* ms, int* launches, double* work, int cap) {
  for (int c = 0; c < cap; ++c) {
    if (ms) ms[c] = 0;
    if (launches) launches[c] = 0;
    if (work) work[c] = 0;
  }
  cudaError_t err = cudaSuccess;
  for (auto& r : recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) err = e;
    float t = 0;
    cudaEventElapsedTime(&t, r.a, r.b);
    if (r.cls < cap) {
      if (ms) ms[r.cls] += t;
      if (launches) launches[r.cls] += r.launches;
      if (work) work[r.cls] += r.work;
    }
  }
  recs.clear();
  used = 0;
  return err;
}
void Profiler::destroy() {
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
  recs.clear();
  used = 0;
}
}  // namespace sp

struct sp_ctx {
  int d = 0, n = 0, b = 0, L = 0, nl = 0;
  long N = 0;
  double s = 0;
  sp_precision prec = SP_PREC_FP64;
  sp_opts opts{};
  cudaStream_t stream = nullptr;
  std::vector<StencilTable> tabs;
  Symbolic sym;
  std::vector<DevLevel> lv;
  std::vector<QTypeDev> qtypes;
  std::vector<void*> allocs;
  double* Qcat = nullptr;
  double* Ccat = nullptr;
  double* Tcat = nullptr;
  float* Tcat32 = nullptr;
  FactorWork work;          // triangular-inverse scratch, tensor-core operand buffers
  FftPlan fft;
  const double* q = nullptr;  // current medium (caller's or qbuf)
  double* qbuf = nullptr;     // used by sp_factor_host
  int* status = nullptr;
  void* rhsQ = nullptr;       // N vector (VT) of Q r
  void* gemv_part = nullptr;  // partial sums of the split row products of the sweeps
  // Krylov workspace
  int maxv = 0;
  double2 *V = nullptr, *Z = nullptr, *H = nullptr, *gam = nullptr, *sn = nullptr;
  double2 *h1 = nullptr, *h2 = nullptr, *y = nullptr;
  double *cs = nullptr, *nrm = nullptr, *est = nullptr;
  double2 *g = nullptr, *r = nullptr, *t = nullptr, *fbuf = nullptr, *ubuf = nullptr;
  double* host_sc = nullptr;  // pinned scalars
  KrylovWork K;
  Profiler prof;
  bool profiling = false;
  bool factored = false;
  bool mixed = false;          // SP_PREC_MIXED: prec is FP32 for the factor and sweeps
  float* q32 = nullptr;        // complex64 operator of the inner solve
  float2* z32 = nullptr;
  // CUDA graphs of the preconditioner application and of the factorisation,
  // captured once at set-up on an internal stream and replayed on `stream`
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_apply = nullptr, g_factor = nullptr;
  double2* app_in = nullptr;   // fixed input / output of the apply graph (max_rhs N: the
  double2* app_out = nullptr;  // block input and output of sp_solve_many)
  double2* blk_w = nullptr;    // max_rhs N: operator outputs of sp_solve_many
  cudaGraphExec_t g_block[9] = {};  // block applications of nv = 2 ... max_rhs stacked
  bool g_block_tried[9] = {};       // vectors, captured on first use
  // problem group: P problems of one grid and leaf size (shifts[p]); vectors of the
  // context hold P N entries, problem p's at p N
  int P = 1;
  long NP = 0;
  std::vector<double> shifts;
  long t_stride = 0;  // entries between two problems' T tables (Tcat, Tcat32)
  int IM = 1;         // Krylov instances the workspace holds: P max_rhs
  // batched Krylov processes (sp_solve and sp_solve_many through the cycle graphs):
  // per-instance state on the device and pinned copies, one cycle graph per
  // right-hand-side count R (R P instances) and the medium pointer it was captured with
  LoopHead* heads = nullptr;
  LoopHead* host_heads = nullptr;
  double* hist = nullptr;  // IM x maxit estimates
  double* host_hist = nullptr;
  int* run = nullptr;
  int* host_run = nullptr;
  cudaGraphExec_t g_cycle[9] = {};
  const double* g_cycle_q[9] = {};
  double factor_entries = 0, factor_flops = 0, apply_bytes = 0;
};

namespace {

// Makes the context's profiler current for the duration of one API call.
struct ProfGuard {
  Profiler* saved;
  explicit ProfGuard(sp_ctx* c) : saved(g_prof) { g_prof = (c && c->profiling) ? &c->prof : nullptr; }
  ~ProfGuard() { g_prof = saved; }
};

const double kPi = 3.141592653589793238462643383279502884;

template <class P>
cudaError_t dalloc(sp_ctx* c, P** p, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  c->allocs.push_back(v);
  *p = (P*)v;
  return cudaSuccess;
}

template <class P>
cudaError_t upload(sp_ctx* c, P** p, const std::vector<P>& h) {
  cudaError_t e = dalloc(c, p, h.size() * sizeof(P));
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*p, h.data(), h.size() * sizeof(P), cudaMemcpyHostToDevice);
  return e;
}

sp_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SP_OK;
  if (e == cudaErrorMemoryAllocation) return SP_ERR_OOM;
  return SP_ERR_CUDA;
}

#define SP_CK(x)                              \
  do {                                        \
    cudaError_t e_ = (x);                     \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

double shift_gap(int d, int n, double s) { return resonance_gap(d, n, s); }

double perturb_shift(int d, int n, double s) {
  int guard = 0;
  while (shift_gap(d, n, s) < 1e-6 && guard++ < 1000000) s += 1e-3 * 4.0 * kPi * kPi;
  return s;
}

sp_status apply_block(sp_ctx* c, int nv, const double2* r, double2* z, cudaStream_t st);

sp_status apply_direct(sp_ctx* c, const double2* r, double2* z, cudaStream_t st) {
  return apply_block(c, 1, r, z, st);
}

// z = P^{-1} Q r: the captured graph when there is one and no kernel timing is
// requested (the graph reads app_in and writes app_out), else direct launches.
sp_status apply_impl(sp_ctx* c, const double2* r, double2* z) {
  cudaStream_t st = c->stream;
  if (c->g_apply && !c->profiling) {
    const size_t bytes = sizeof(double2) * (size_t)c->NP;
    SP_CK(cudaMemcpyAsync(c->app_in, r, bytes, cudaMemcpyDeviceToDevice, st));
    SP_CK(cudaGraphLaunch(c->g_apply, st));
    SP_CK(cudaMemcpyAsync(z, c->app_out, bytes, cudaMemcpyDeviceToDevice, st));
    return SP_OK;
  }
  return apply_direct(c, r, z, st);
}

sp_status factor_direct(sp_ctx* c, const double* q, cudaStream_t st) {
  SP_CK(cudaMemsetAsync(c->status, 0, sizeof(int), st));
  for (int l = 0; l <= c->L; ++l)
    SP_CK(factor_level(c->prec, c->d, c->lv[l], l ? &c->lv[l - 1] : nullptr, c->Qcat, c->Ccat, q,
                       c->opts.pivot_tol, c->status, c->work, st));
  for (int l = 0; l <= c->L; ++l) SP_CK(factor_copy16(c->lv[l], st));
  return SP_OK;
}

// Smallest of reps timings of fn() on stream st with CUDA events (ms).
template <class Fn>
float time_ms(cudaStream_t st, int reps, Fn fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  float best = 1e30f;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return best;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, st);
    fn();
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float t = 0;
    cudaEventElapsedTime(&t, a, b);
    best = std::min(best, t);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

// Greedy per-level autotuning of the factorisation's GEMM tiles (shapes that
// leave every result bit-identical: each output entry is summed in the same
// order): each candidate of a level is timed on that level alone (a level's
// factorisation re-assembles its fronts from its children), bottom-up, with the
// medium in qbuf (zero at set-up: P = Q).
sp_status autotune(sp_ctx* c) {
  cudaStream_t st = c->stream;
  SP_CK(cudaMemsetAsync(c->status, 0, sizeof(int), st));
  sp_status fs = factor_direct(c, c->qbuf, st);  // warm-up; leaves a valid factor
  if (fs != SP_OK) return fs;
  for (int l = 0; l <= c->L; ++l) {
    DevLevel& D = c->lv[l];
    const DevLevel* ch = l ? &c->lv[l - 1] : nullptr;
    auto run = [&]() {
      factor_level(c->prec, c->d, D, ch, c->Qcat, c->Ccat, c->qbuf, c->opts.pivot_tol, c->status,
                   c->work, st);
    };
    int* knobs[2] = {&D.gemm_tile, &D.gen_tile};
    for (int kn = 0; kn < (D.inv ? 2 : 1); ++kn) {
      int best = 0;
      float tbest = 1e30f;
      for (int cand : {32, 64}) {
        *knobs[kn] = cand;
        run();  // first launch of a shape outside the timing
        const float t = time_ms(st, 2, run);
        if (t < tbest) {
          tbest = t;
          best = cand;
        }
      }
      *knobs[kn] = best;
    }
    run();
  }
  SP_CK(cudaGetLastError());
  SP_CK(cudaMemsetAsync(c->status, 0, sizeof(int), st));
  SP_CK(cudaStreamSynchronize(st));
  return cuda_status(cudaGetLastError());
}

// Captures fn(cap stream) into an executable graph; leaves *out null on failure
// (the callers then launch directly).
template <class Fn>
void capture_graph(sp_ctx* c, cudaGraphExec_t* out, Fn fn) {
  *out = nullptr;
  if (!c->cap) return;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  sp_status st = fn(c->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (st == SP_OK && e == cudaSuccess && g) {
    if (cudaGraphInstantiate(out, g, 0) != cudaSuccess) *out = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
}

// Application of the preconditioner to nv stacked vectors of the context (each P N
// entries, nv P problem vectors N apart): stencil, forward sweep, backward sweep.
sp_status apply_block(sp_ctx* c, int nv, const double2* r, double2* z, cudaStream_t st) {
  SP_CK(q_apply(c->prec, c->d, c->n, c->nl, c->qtypes, c->Tcat, c->Tcat32, r, c->rhsQ, st, nv,
                c->opts.launch_overlap != 0, c->P, c->t_stride));
  for (int l = 0; l <= c->L; ++l)
    SP_CK(forward_level(c->prec, c->d, c->lv[l], l ? &c->lv[l - 1] : nullptr, c->rhsQ,
                        c->gemv_part, st, nv, c->NP));
  for (int l = c->L; l >= 0; --l)
    SP_CK(backward_level(c->prec, c->d, c->lv[l], z, c->gemv_part, st, nv, c->NP));
  return SP_OK;
}

// The instances' Krylov workspace slices (instance i = r P + p: right-hand side r of
// problem p; every vector N entries, instance i's at i N).
KBatch make_batch(sp_ctx* c) {
  KBatch b;
  const long N = c->N;
  const int mv = c->maxv, restart = c->opts.restart;
  b.V = c->V;
  b.Z = c->Z;
  b.H = c->H;
  b.gam = c->gam;
  b.sn = c->sn;
  b.cs = c->cs;
  b.h1 = c->h1;
  b.h2 = c->h2;
  b.y = c->y;
  b.nrm = c->nrm;
  b.est = c->est;
  b.partial = c->K.partial;
  b.w = c->t;
  b.head = c->heads;
  b.run = c->run;
  b.N = N;
  b.sV = (long)mv * N;
  b.sZ = (long)restart * N;
  b.sH = (long)mv * restart;
  b.sG = mv + 1;
  b.sh = 1024;
  b.sP = (long)c->K.nblk * 1024;
  b.ldh = mv;
  b.nblk = c->K.nblk;
  return b;
}

// One GMRES restart cycle of R P instances as one CUDA graph: V_0 = r / |r| for the
// running instances, then a conditional while node whose body is one Arnoldi step of
// every instance still in its cycle (the apply of the R stacked vectors, the operator,
// Gram-Schmidt twice, the Givens rotation, the stopping test; the test ends the node
// when no instance goes on), then u += Z y, the true residual r = g - A u and a copy
// of the heads and estimates to the host.  The graph works on the context's own
// vectors (u in ubuf) and its copy of the medium (c->q = qbuf, which sp_factor
// refills), so one capture serves every later factorisation; it is captured again
// only if that pointer ever changes.
sp_status build_cycle_graph(sp_ctx* c, int R) {
  if (c->g_cycle[R]) {
    cudaGraphExecDestroy(c->g_cycle[R]);
    c->g_cycle[R] = nullptr;
  }
  if (!c->cap) return SP_ERR_CUDA;
  cudaStream_t s = c->cap;
  const long N = c->N;
  const int I = R * c->P, mv = c->maxv, maxit = c->opts.maxit;
  const KBatch b = make_batch(c);
  cudaGraph_t g = nullptr;
  SP_CK(cudaGraphCreate(&g, 0));
  struct Owner {
    cudaGraph_t g;
    ~Owner() { cudaGraphDestroy(g); }
  } owner{g};
  cudaGraphConditionalHandle cond = 0;
  SP_CK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  cudaGraph_t body = nullptr;
  auto outer = [&]() -> sp_status {
    SP_CK(kb_start(b, I, c->r, mv + 1, s));
    SP_CK(kb_begin(b, I, s));
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    SP_CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd));
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t wn = nullptr;
    SP_CK(cudaGraphAddNode(&wn, g, deps, nullptr, nd, &p));
    body = p.conditional.phGraph_out[0];
    SP_CK(cudaStreamUpdateCaptureDependencies(s, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
    SP_CK(kb_update_solution(b, I, c->ubuf, s));
    SP_CK(fft_green_apply(c->fft, c->ubuf, c->q, true, c->t, s, I, c->P));
    SP_CK(kr_sub(c->g, c->t, (long)I * N, c->r, s));
    SP_CK(kb_norm(b, I, c->r, 3, s));
    SP_CK(kb_finish(b, I, s));
    SP_CK(cudaMemcpyAsync(c->host_heads, c->heads, sizeof(LoopHead) * I, cudaMemcpyDeviceToHost, s));
    SP_CK(cudaMemcpyAsync(c->host_hist, c->hist, sizeof(double) * maxit * I,
                          cudaMemcpyDeviceToHost, s));
    return SP_OK;
  };
  SP_CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  sp_status so = outer();
  cudaGraph_t got = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &got);
  if (so != SP_OK) return so;
  SP_CK(e);
  if (!body) return SP_ERR_CUDA;
  auto step = [&]() -> sp_status {
    SP_CK(kb_copy_in(b, I, c->app_in, s));
    sp_status a = apply_block(c, R, c->app_in, c->app_out, s);
    if (a != SP_OK) return a;
    SP_CK(kb_copy_out(b, I, c->app_out, s));
    SP_CK(fft_green_apply(c->fft, c->app_out, c->q, true, b.w, s, I, c->P));
    SP_CK(kb_arnoldi(b, I, mv, s));
    SP_CK(kb_step(b, I, c->hist, maxit, c->opts.tol, maxit, c->opts.restart, cond, s));
    return SP_OK;
  };
  SP_CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  sp_status sb = step();
  got = nullptr;
  e = cudaStreamEndCapture(s, &got);
  if (sb != SP_OK) return sb;
  SP_CK(e);
  SP_CK(cudaGraphInstantiate(&c->g_cycle[R], g, 0));
  c->g_cycle_q[R] = c->q;
  return SP_OK;
}

}  // namespace

extern "C" {

size_t sp_abi_size(int which) {
  switch (which) {
    case 0: return sizeof(sp_opts);
    case 1: return sizeof(sp_info);
    default: return 0;
  }
}

void sp_default_opts(sp_opts* o) {
  if (!o) return;
  o->maxit = 500;
  o->restart = 200;
  o->tol = 1e-8;
  o->pivot_tol = 1e-14;
  o->device = 0;
  o->host_threads = 0;
  o->inner_tol = 1e-5;
  o->autotune = 0;
  o->max_rhs = 1;
  o->setup_route = 0;
  o->stencil = 0;
  o->inv_block = 0;
  o->tc_epilogue = 0;
  o->wait_limit_ns = 0;
  o->sweeps = 0;
  o->panel_pivoting = 0;
  o->launch_overlap = 0;
  o->device_loop = 1;
  o->factor_storage = 0;
}

const char* sp_status_str(sp_status st) {
  switch (st) {
    case SP_OK: return "ok";
    case SP_ERR_ARG: return "invalid argument";
    case SP_ERR_RESONANT: return "L - s is numerically singular (resonant shift)";
    case SP_ERR_SINGULAR: return "singular front pivot";
    case SP_ERR_NOCONV: return "GMRES did not reach the tolerance";
    case SP_ERR_OOM: return "out of memory (device or host) or no host thread for the set-up";
    case SP_ERR_TIMEOUT: return "device wait timed out";
    case SP_ERR_CUDA: return "CUDA runtime error";
    case SP_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

sp_status sp_front_sizes(int d, int n, int b, int cap, int* nlevels, int* nfronts, int* k, int* m) {
  std::vector<int> nf, kk, mm;
  if (!nlevels || front_sizes(d, n, b, &nf, &kk, &mm)) return SP_ERR_ARG;
  *nlevels = (int)nf.size();
  for (int i = 0; i < (int)nf.size() && i < cap; ++i) {
    if (nfronts) nfronts[i] = nf[i];
    if (k) k[i] = kk[i];
    if (m) m[i] = mm[i];
  }
  return SP_OK;
}

sp_status sp_stencil_table(int d, int n, int b, double s, int t, int route, int kind,
                           int host_threads, double* Q_out, double* C_out, int* rows, int* cols,
                           int* rank, double* sigma_out) {
  if ((route != 0 && route != 1) || (kind != 0 && kind != 1) || !std::isfinite(s))
    return SP_ERR_ARG;
  int L;
  if (check_grid(d, n, b, &L) || t < 0 || t >= (1 << d)) return SP_ERR_ARG;
  if (!rows || !cols) return SP_ERR_ARG;
  long nS = 1, nG = 1;
  for (int a = 0; a < d; ++a) {
    bool z = (t >> a) & 1;
    nS *= z ? 1 : (b - 1);
    nG *= z ? 3 : (b + 1);
  }
  *rows = (int)nS;
  *cols = (int)nG;
  if (!Q_out && !C_out && !sigma_out && !rank) return SP_OK;
  if (shift_gap(d, n, s) < 1e-6) return SP_ERR_RESONANT;
  try {
    std::vector<double> g = green_kernel(d, n, s, host_threads), g2;
    if (route == 1) g2 = green_kernel_sq(d, n, s, host_threads);
    StencilTable tb;
    if (stencil_table(d, n, b, t, g, host_threads, &tb, route == 1 ? &g2 : nullptr, kind))
      return SP_ERR_ARG;
    if (Q_out) std::memcpy(Q_out, tb.Q.data(), tb.Q.size() * sizeof(double));
    if (C_out) std::memcpy(C_out, tb.C.data(), tb.C.size() * sizeof(double));
    if (rank) *rank = tb.rank;
    if (sigma_out)
      for (int i = 0; i < std::min<int>(64, (int)tb.sigma.size()); ++i) sigma_out[i] = tb.sigma[i];
  } catch (const std::exception&) {  // host memory, or the set-up's host threads
    return SP_ERR_OOM;
  }
  return SP_OK;
}

sp_status sp_level_info(int d, int n, int b, int level, int* nf, int* k, int* m, int* mc, int* kc,
                        int* nasm, int* gidx, int* ea_map, int* asm_row, int* asm_cvar) {
  int L;
  if (check_grid(d, n, b, &L) || level < 0 || level > L) return SP_ERR_ARG;
  try {
    // the assembly lists need the table geometry only, not the values
    std::vector<StencilTable> tabs(1 << d);
    for (int t = 0; t < (1 << d); ++t) {
      StencilTable& tb = tabs[t];
      tb.t = t;
      tb.nS = 1;
      tb.nG = 1;
      int lo[3], hi[3], glo[3], ghi[3];
      for (int a = 0; a < d; ++a) {
        bool z = (t >> a) & 1;
        lo[a] = z ? 0 : 1;
        hi[a] = z ? 0 : b - 1;
        glo[a] = z ? -1 : 0;
        ghi[a] = z ? 1 : b;
        tb.nS *= hi[a] - lo[a] + 1;
        tb.nG *= ghi[a] - glo[a] + 1;
      }
      for (int c = 0; c < tb.nS; ++c) {
        int cc = c;
        for (int a = 0; a < d; ++a) {
          int span = hi[a] - lo[a] + 1;
          tb.S.push_back(lo[a] + cc % span);
          cc /= span;
        }
      }
      for (int c = 0; c < tb.nG; ++c) {
        int cc = c;
        for (int a = 0; a < d; ++a) {
          int span = ghi[a] - glo[a] + 1;
          tb.G.push_back(glo[a] + cc % span);
          cc /= span;
        }
      }
    }
    Symbolic sym;
    if (build_symbolic(d, n, b, tabs, &sym)) return SP_ERR_ARG;
    const Level& V = sym.lv[level];
    if (nf) *nf = V.nf;
    if (k) *k = V.k;
    if (m) *m = V.m;
    if (mc) *mc = V.mc;
    if (kc) *kc = V.kc;
    if (nasm) *nasm = (int)V.asm_row.size();
    if (gidx) std::memcpy(gidx, V.gidx.data(), V.gidx.size() * sizeof(int));
    if (ea_map && !V.ea_map.empty()) std::memcpy(ea_map, V.ea_map.data(), V.ea_map.size() * sizeof(int));
    if (asm_row) std::memcpy(asm_row, V.asm_row.data(), V.asm_row.size() * sizeof(int));
    if (asm_cvar) std::memcpy(asm_cvar, V.asm_cvar.data(), V.asm_cvar.size() * sizeof(int));
  } catch (const std::exception&) {  // host memory, or the set-up's host threads
    return SP_ERR_OOM;
  }
  return SP_OK;
}

sp_status sp_medium_helmholtz(int d, int n, double omega, const double* c_host, double* s_out,
                              double* q_host) {
  if ((d != 2 && d != 3) || n < 2 || !c_host || !s_out || !q_host || !std::isfinite(omega))
    return SP_ERR_ARG;
  long N = 1;
  for (int a = 0; a < d; ++a) N *= n;
  double sum = 0;
  for (long j = 0; j < N; ++j) {
    if (!(std::isfinite(c_host[j]) && c_host[j] != 0.0)) return SP_ERR_ARG;
    sum += omega * omega / (c_host[j] * c_host[j]);
  }
  double s = perturb_shift(d, n, sum / (double)N);
  for (long j = 0; j < N; ++j) q_host[j] = s - omega * omega / (c_host[j] * c_host[j]);
  *s_out = s;
  return SP_OK;
}

sp_status sp_medium_schrodinger(int d, int n, double ell, double E, const double* V_host,
                                double* s_out, double* q_host) {
  if ((d != 2 && d != 3) || n < 2 || !V_host || !s_out || !q_host || !std::isfinite(ell) ||
      !std::isfinite(E))
    return SP_ERR_ARG;
  long N = 1;
  for (int a = 0; a < d; ++a) N *= n;
  const double l2 = ell * ell;
  double sum = 0;
  for (long j = 0; j < N; ++j) {
    if (!std::isfinite(V_host[j])) return SP_ERR_ARG;
    sum += -(l2 * V_host[j] - l2 * E);
  }
  double s = perturb_shift(d, n, sum / (double)N);
  for (long j = 0; j < N; ++j) q_host[j] = (l2 * V_host[j] - l2 * E) + s;
  *s_out = s;
  return SP_OK;
}

sp_status sp_medium_schrodinger_at(int d, int n, double ell, double E, const double* V_host,
                                   double s, double* q_host) {
  if ((d != 2 && d != 3) || n < 2 || !V_host || !q_host || !std::isfinite(ell) ||
      !std::isfinite(E) || !std::isfinite(s))
    return SP_ERR_ARG;
  long N = 1;
  for (int a = 0; a < d; ++a) N *= n;
  const double l2 = ell * ell;
  for (long j = 0; j < N; ++j)
    if (!std::isfinite(V_host[j])) return SP_ERR_ARG;
  for (long j = 0; j < N; ++j) q_host[j] = (l2 * V_host[j] - l2 * E) + s;
  return SP_OK;
}

void sp_destroy(sp_ctx* c) {
  if (!c) return;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(c->opts.device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  if (c->host_sc) cudaFreeHost(c->host_sc);
  c->prof.destroy();
  if (c->g_apply) cudaGraphExecDestroy(c->g_apply);
  for (auto& g : c->g_block)
    if (g) cudaGraphExecDestroy(g);
  if (c->g_factor) cudaGraphExecDestroy(c->g_factor);
  for (auto& g : c->g_cycle)
    if (g) cudaGraphExecDestroy(g);
  if (c->host_heads) cudaFreeHost(c->host_heads);
  if (c->host_hist) cudaFreeHost(c->host_hist);
  if (c->host_run) cudaFreeHost(c->host_run);
  if (c->cap) cudaStreamDestroy(c->cap);
  cudaSetDevice(dev);
  delete c;
}

static sp_status setup_impl(int d, int n, int b, int P, const double* shifts, sp_precision prec,
                            const sp_opts* opts, void* stream, sp_ctx** out) {
  if (!out || !shifts || P < 1) return SP_ERR_ARG;
  *out = nullptr;
  int L;
  if (check_grid(d, n, b, &L)) return SP_ERR_ARG;
  {  // the device FFT handles n = 2^p and n = 3 2^p
    const int m2 = (n % 3 == 0) ? n / 3 : n;
    if (m2 < 2 || (m2 & (m2 - 1))) return SP_ERR_ARG;
  }
  {  // grid indices of a group's fronts are ints offset by p N: P n^d must fit
    long long NP = P;
    for (int a = 0; a < d; ++a) NP *= n;
    if (NP > 2147483647LL) return SP_ERR_ARG;
  }
  if (prec != SP_PREC_FP64 && prec != SP_PREC_FP32 && prec != SP_PREC_MIXED &&
      prec != SP_PREC_TF32 && prec != SP_PREC_TF32X3)
    return SP_ERR_ARG;
  const bool mixed = (prec == SP_PREC_MIXED);
  const bool tc = (prec == SP_PREC_TF32 || prec == SP_PREC_TF32X3);
  const bool split = (prec == SP_PREC_TF32X3);
  if (mixed || tc) prec = SP_PREC_FP32;
  if (mixed && P > 1) return SP_ERR_ARG;
  for (int p = 0; p < P; ++p) {
    if (!(std::isfinite(shifts[p]))) return SP_ERR_ARG;
    if (shift_gap(d, n, shifts[p]) < 1e-6) return SP_ERR_RESONANT;
  }
  const double s = shifts[0];
  std::unique_ptr<sp_ctx> c(new (std::nothrow) sp_ctx());
  if (!c) return SP_ERR_OOM;
  sp_default_opts(&c->opts);
  if (opts) c->opts = *opts;
  if (c->opts.maxit < 1 || c->opts.restart < 1 || c->opts.restart > 1000 || !(c->opts.tol > 0))
    return SP_ERR_ARG;
  if (c->opts.max_rhs < 1 || c->opts.max_rhs > sweep_max_vectors()) return SP_ERR_ARG;
  if (c->opts.setup_route != 0 && c->opts.setup_route != 1) return SP_ERR_ARG;
  if (c->opts.stencil != 0 && c->opts.stencil != 1) return SP_ERR_ARG;
  {
    const int ib = c->opts.inv_block;
    if (ib != 0 && (ib < 64 || ib > 2048 || (ib & (ib - 1)) != 0)) return SP_ERR_ARG;
  }
  if (c->opts.tc_epilogue < 0 || c->opts.tc_epilogue > 4) return SP_ERR_ARG;
  if (c->opts.wait_limit_ns < 0 || c->opts.wait_limit_ns > 60000000000LL) return SP_ERR_ARG;
  if (c->opts.sweeps < 0 || c->opts.sweeps > 2) return SP_ERR_ARG;
  if (c->opts.panel_pivoting != 0 && c->opts.panel_pivoting != 1) return SP_ERR_ARG;
  if (c->opts.launch_overlap != 0 && c->opts.launch_overlap != 1) return SP_ERR_ARG;
  if (c->opts.device_loop != 0 && c->opts.device_loop != 1) return SP_ERR_ARG;
  if (c->opts.factor_storage != 0 && c->opts.factor_storage != 1) return SP_ERR_ARG;
  if (c->opts.factor_storage == 1 && prec == SP_PREC_FP64) return SP_ERR_ARG;
  const size_t RH = (size_t)c->opts.max_rhs;
  // every Krylov instance (right-hand side of a problem) is one thread of the batched
  // stopping test
  if ((size_t)P * RH > 1024) return SP_ERR_ARG;
  c->P = P;
  c->shifts.assign(shifts, shifts + P);
  c->IM = (int)(P * RH);
  const size_t IM = (size_t)c->IM;
  c->d = d;
  c->n = n;
  c->b = b;
  c->L = L;
  c->nl = n / b;
  c->s = s;
  c->prec = prec;
  c->mixed = mixed;
  c->work.tc = tc;
  c->work.tc_split = split;
  c->work.tc_epi = c->opts.tc_epilogue;
  c->work.wait_ns = c->opts.wait_limit_ns > 0 ? (unsigned long long)c->opts.wait_limit_ns
                                              : 2000000000ull;
  c->work.calu = c->opts.panel_pivoting == 1 ? 1 : 0;
  if (mixed && !(c->opts.inner_tol > 0 && c->opts.inner_tol < 1)) return SP_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  c->N = 1;
  for (int a = 0; a < d; ++a) c->N *= n;
  const long N = c->N;
  c->NP = (long)P * N;
  const long NP = c->NP;
  SP_CK(cudaSetDevice(c->opts.device));
  // ---- host set-up: Green's kernel, stencil tables, symbolic structure
  try {
    // tables of every problem, problem-major (problem p's type t at p 2^d + t), and
    // the symbolic structure, which depends on the sets only (the same for every problem)
    if (setup_host(d, n, b, P, shifts, c->opts.setup_route, c->opts.stencil,
                   c->opts.host_threads, &c->tabs, &c->sym))
      return SP_ERR_ARG;
  } catch (const std::exception&) {  // host memory, or the set-up's host threads
    return SP_ERR_OOM;
  }
  // ---- tables on the device (column-major per type, concatenated): Q and C on
  // gamma for the assembly, T on beta for the stencil apply
  {
    std::vector<double> Qc, Cc, Tc;
    std::vector<float> T32;
    // problem after problem (all have the same table shapes): the offsets of the
    // first problem address every problem's tables, tab_stride / t_stride apart
    long off = 0, toff = 0;
    for (int pt = 0; pt < (P << d); ++pt) {
      const int t = pt & ((1 << d) - 1);
      const StencilTable& tb = c->tabs[pt];
      QTypeDev qt;
      qt.nS = tb.nS;
      qt.nG = tb.nG;
      qt.nB = tb.nB;
      qt.tab_off = off;
      qt.t_off = toff;
      for (int col = 0; col < tb.nG; ++col)
        for (int a = 0; a < tb.nS; ++a) {
          Qc.push_back(tb.Q[(size_t)a * tb.nG + col]);
          Cc.push_back(tb.C[(size_t)a * tb.nG + col]);
        }
      // T = -Q restricted to the beta columns (gamma order lists beta in beta order)
      std::vector<int> bcols;
      {
        int sidx = 0;
        for (int gi = 0; gi < tb.nG; ++gi) {
          bool inS = sidx < tb.nS;
          for (int a = 0; a < d && inS; ++a)
            if (tb.G[(size_t)gi * d + a] != tb.S[(size_t)sidx * d + a]) inS = false;
          if (inS) ++sidx;
          else bcols.push_back(gi);
        }
      }
      if ((int)bcols.size() != tb.nB) return SP_ERR_ARG;
      // per-point stencils: Q(S, S) is not the identity, so the apply runs over
      // every column of gamma
      if (c->opts.stencil == 1) {
        bcols.resize(tb.nG);
        for (int gi = 0; gi < tb.nG; ++gi) bcols[gi] = gi;
      }
      qt.na = (int)bcols.size();
      qt.self = c->opts.stencil == 1 ? 0 : 1;
      for (int cb = 0; cb < qt.na; ++cb)
        for (int a = 0; a < tb.nS; ++a) {
          double v = -tb.Q[(size_t)a * tb.nG + bcols[cb]];
          Tc.push_back(v);
          T32.push_back((float)v);
        }
      off += (long)tb.nS * tb.nG;
      toff += (long)tb.nS * qt.na;
      if (pt == (1 << d) - 1) {
        c->work.tab_stride = off;
        c->t_stride = toff;
      }
      if (pt != t) continue;
      SP_CK(upload(c.get(), &qt.S, tb.S));
      SP_CK(upload(c.get(), &qt.G, tb.G));
      SP_CK(upload(c.get(), &qt.Bt, tb.Bt));
      qt.A = qt.self ? qt.Bt : qt.G;
      c->qtypes.push_back(qt);
    }
    SP_CK(upload(c.get(), &c->Qcat, Qc));
    SP_CK(upload(c.get(), &c->Ccat, Cc));
    SP_CK(upload(c.get(), &c->Tcat, Tc));
    SP_CK(upload(c.get(), &c->Tcat32, T32));
  }
  // ---- levels
  const size_t fsz = (prec == SP_PREC_FP32) ? sizeof(float) : sizeof(double);
  const size_t vsz = (prec == SP_PREC_FP32) ? sizeof(float2) : sizeof(double2);
  c->lv.resize(L + 1);
  size_t scratch_bytes = 0, pack_floats = 0, gp_words = 0;
  int num_sms = 152;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, c->opts.device);
  const int max_cluster = c->opts.sweeps == 2 ? sweep_max_cluster() : 8;
  for (int l = 0; l <= L; ++l) {
    const Level& S = c->sym.lv[l];
    DevLevel& D = c->lv[l];
    D.nfp = S.nf;
    D.nf = P * S.nf;
    D.k = S.k;
    D.m = S.m;
    D.nb1 = S.nb1;
    D.mc = S.mc;
    D.kc = S.kc;
    D.nasm = (int)S.asm_row.size();
    if (P == 1) {
      SP_CK(upload(c.get(), &D.gidx, S.gidx));
    } else {  // problem p's fronts index its vector segment [p N, (p + 1) N)
      std::vector<int> gg;
      gg.reserve(S.gidx.size() * P);
      for (int p = 0; p < P; ++p)
        for (int v : S.gidx) gg.push_back(v + (int)((long)p * N));
      SP_CK(upload(c.get(), &D.gidx, gg));
    }
    SP_CK(upload(c.get(), &D.asm_row, S.asm_row));
    SP_CK(upload(c.get(), &D.asm_tidx, S.asm_tidx));
    SP_CK(upload(c.get(), &D.asm_cvar, S.asm_cvar));
    SP_CK(upload(c.get(), &D.ea_map, S.ea_map));
    SP_CK(dalloc(c.get(), &D.front, fsz * (size_t)D.nf * S.m * S.m));
    SP_CK(dalloc(c.get(), &D.perm, sizeof(int) * (size_t)D.nf * std::max(1, S.k)));
    SP_CK(dalloc(c.get(), &D.piv, sizeof(int) * (size_t)D.nf * std::max(1, S.k)));
    SP_CK(dalloc(c.get(), &D.scale, sizeof(double) * D.nf));
    SP_CK(dalloc(c.get(), &D.upd, vsz * RH * (size_t)D.nf * std::max(1, S.m - S.k)));
    SP_CK(dalloc(c.get(), &D.y, vsz * RH * (size_t)D.nf * std::max(1, S.k)));
    if (factor_panel_width(prec, S.m) == 0) return SP_ERR_ARG;  // front too large to stage
    // few fronts: keep the inverses of the diagonal blocks of L11 and U11 so the
    // sweeps spread over the GPU; in the FP32 form every level does (the block
    // inverses cost little in FP32 and the sweeps become matrix-vector products)
    D.inv = D.nf < 152 || prec == SP_PREC_FP32 || vsz * (size_t)(S.m + S.k) > 192 * 1024;
    // block inverses: 2048-wide blocks where the fronts are huge (the sweeps of the 3D
    // root become 48 instead of 189 launch pairs; measured 3D 128^3 TF32: sweeps
    // 1.95 -> 1.51 s per solve for +0.1 s of inversion), 512 elsewhere (in 2D the
    // larger inverses cost more than the launches they save)
    D.ib = c->opts.inv_block > 0 ? c->opts.inv_block : (S.k >= 32768 ? 2048 : kInvBlockSize);
    D.pdl = c->opts.launch_overlap;
    if (D.inv && c->opts.sweeps != 1) {
      int C = 0, NT = 0;
      if (sweep_fused_config(prec, D.nf, S.m, S.k, num_sms, max_cluster, c->opts.sweeps == 2, &C,
                             &NT)) {
        D.fused_c = C;
        D.fused_nt = NT;
      }
    }
    if (D.inv && D.fused_c == 0 && c->opts.factor_storage == 1) {
      SP_CK(dalloc(c.get(), &D.front16, (size_t)2 * D.nf * S.m * ((S.m + 1) & ~1)));
      SP_CK(dalloc(c.get(), &D.fscale16, sizeof(float) * D.nf * S.m));
    }
    if (D.inv) {
      SP_CK(dalloc(c.get(), &D.tmp, vsz * RH * (size_t)D.nf * S.m));
      scratch_bytes = std::max(scratch_bytes, fsz * invert_scratch_elems(D.nf, S.k, D.ib));
    }
    if (factor_grid_panel(prec, S.m)) gp_words = std::max(gp_words, grid_panel_pub_words(D.nf));
    if (factor_outer_block(prec, tc, S.m, S.k) > 0)
      pack_floats = std::max(pack_floats, tc_pack_floats(S.m, kTcMaxK, D.nf, split));
    double k = S.k, mk = S.m - S.k;
    c->factor_entries += D.nf * (k * k + 2 * k * mk);
    c->factor_flops += D.nf * ((2.0 / 3.0) * k * k * k + 2 * k * k * mk + 2 * k * mk * mk);
  }
  c->apply_bytes = c->factor_entries * fsz;
  if (c->opts.factor_storage == 1) {  // the chained levels' sweeps read half as many bytes
    double e16 = 0;
    for (const DevLevel& D : c->lv)
      if (D.front16) e16 += D.nf * ((double)D.k * D.k + 2.0 * D.k * (D.m - D.k));
    c->apply_bytes -= e16 * (fsz - 2);
  }
  if (scratch_bytes) SP_CK(dalloc(c.get(), &c->work.inv, scratch_bytes));
  SP_CK(dalloc(c.get(), &c->gemv_part, sweep_partial_bytes((int)RH)));
  if (gp_words) SP_CK(dalloc(c.get(), &c->work.gpub, sizeof(unsigned long long) * gp_words));
  if (pack_floats) {
    SP_CK(dalloc(c.get(), &c->work.packA, sizeof(float) * pack_floats));
    SP_CK(dalloc(c.get(), &c->work.packB, sizeof(float) * pack_floats));
  }
  // ---- FFT plan
  {
    FftPlan& P = c->fft;
    P.d = d;
    P.n = n;
    P.logn = 0;
    while ((1 << P.logn) < n) ++P.logn;
    std::vector<double2> tw(n / 2);
    for (int t = 0; t < n / 2; ++t) {
      double a = 2.0 * kPi * (double)t / (double)n;
      tw[t] = make_double2(std::cos(a), -std::sin(a));
    }
    SP_CK(upload(c.get(), &P.tw, tw));
    std::vector<double> Dn(NP);
    for (int p = 0; p < c->P; ++p)
      for (long j = 0; j < N; ++j) {
        long r = j;
        double k2 = 0;
        for (int a = 0; a < d; ++a) {
          int i = (int)(r % n);
          r /= n;
          int k = i < n / 2 ? i : i - n;
          k2 += (double)k * k;
        }
        Dn[p * N + j] = 1.0 / (4.0 * kPi * kPi * k2 - shifts[p]) / (double)N;
      }
    SP_CK(upload(c.get(), &P.Dn, Dn));
    SP_CK(dalloc(c.get(), &P.tmp, sizeof(double2) * N * IM));
    if (mixed) {
      std::vector<float2> tw32(tw.size());
      for (size_t i = 0; i < tw.size(); ++i) tw32[i] = make_float2((float)tw[i].x, (float)tw[i].y);
      std::vector<float> Dn32(Dn.begin(), Dn.end());
      SP_CK(upload(c.get(), &P.tw32, tw32));
      SP_CK(upload(c.get(), &P.Dn32, Dn32));
      SP_CK(dalloc(c.get(), &P.tmp32, sizeof(float2) * N));
      SP_CK(dalloc(c.get(), &c->q32, sizeof(float) * N));
      SP_CK(dalloc(c.get(), &c->z32, sizeof(float2) * N));
    }
  }
  // ---- solve workspace
  c->maxv = c->opts.restart + 1;
  SP_CK(dalloc(c.get(), &c->rhsQ, vsz * NP * RH));
  SP_CK(dalloc(c.get(), &c->status, sizeof(int)));
  SP_CK(dalloc(c.get(), &c->qbuf, sizeof(double) * NP));
  // Krylov workspace, one slice per instance (right-hand side r of problem p: slice
  // r P + p; slice 0 is sp_solve's on a single-problem context)
  SP_CK(dalloc(c.get(), &c->V, sizeof(double2) * N * c->maxv * IM));
  SP_CK(dalloc(c.get(), &c->Z, sizeof(double2) * N * c->opts.restart * IM));
  SP_CK(dalloc(c.get(), &c->H, sizeof(double2) * c->maxv * c->opts.restart * IM));
  SP_CK(dalloc(c.get(), &c->gam, sizeof(double2) * (c->maxv + 1) * IM));
  SP_CK(dalloc(c.get(), &c->sn, sizeof(double2) * (c->maxv + 1) * IM));
  SP_CK(dalloc(c.get(), &c->cs, sizeof(double) * (c->maxv + 1) * IM));
  SP_CK(dalloc(c.get(), &c->h1, sizeof(double2) * 1024 * IM));
  SP_CK(dalloc(c.get(), &c->h2, sizeof(double2) * 1024 * IM));
  SP_CK(dalloc(c.get(), &c->y, sizeof(double2) * 1024 * IM));
  SP_CK(dalloc(c.get(), &c->nrm, sizeof(double) * 4 * IM));
  SP_CK(dalloc(c.get(), &c->est, sizeof(double) * 4 * IM));
  SP_CK(dalloc(c.get(), &c->g, sizeof(double2) * N * IM));
  SP_CK(dalloc(c.get(), &c->r, sizeof(double2) * N * IM));
  SP_CK(dalloc(c.get(), &c->t, sizeof(double2) * N * IM));
  SP_CK(dalloc(c.get(), &c->fbuf, sizeof(double2) * NP));
  SP_CK(dalloc(c.get(), &c->ubuf, sizeof(double2) * N * IM));
  c->K.nblk = (int)std::min<long>(304, std::max<long>(1, (N + 1023) / 1024));
  SP_CK(dalloc(c.get(), &c->K.partial, sizeof(double2) * (size_t)c->K.nblk * 1024 * IM));
  SP_CK(dalloc(c.get(), &c->K.h, sizeof(double2) * 1024));
  SP_CK(cudaMallocHost(&c->host_sc, 8 * sizeof(double) * IM));
  SP_CK(dalloc(c.get(), &c->heads, sizeof(LoopHead) * IM));
  SP_CK(dalloc(c.get(), &c->hist, sizeof(double) * c->opts.maxit * IM));
  SP_CK(dalloc(c.get(), &c->run, sizeof(int) * IM));
  SP_CK(cudaMallocHost(&c->host_heads, sizeof(LoopHead) * IM));
  SP_CK(cudaMallocHost(&c->host_hist, sizeof(double) * c->opts.maxit * IM));
  SP_CK(cudaMallocHost(&c->host_run, sizeof(int) * IM));
  SP_CK(dalloc(c.get(), &c->app_in, sizeof(double2) * N * IM));
  SP_CK(dalloc(c.get(), &c->app_out, sizeof(double2) * N * IM));
  if (IM > 1) SP_CK(dalloc(c.get(), &c->blk_w, sizeof(double2) * N * IM));
  SP_CK(cudaMemsetAsync(c->qbuf, 0, sizeof(double) * NP, c->stream));
  // only this context's streams are synchronised: a device-wide synchronisation
  // would break a graph capture that another thread's context has in progress
  SP_CK(cudaStreamSynchronize(c->stream));
  if (c->opts.autotune) {
    sp_status ts = autotune(c.get());
    if (ts != SP_OK) return ts;
  }
  // graphs (a failed capture only means direct launches later)
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap = nullptr;
  }
  {
    sp_ctx* cc = c.get();
    capture_graph(cc, &cc->g_apply, [cc](cudaStream_t s) {
      return apply_direct(cc, cc->app_in, cc->app_out, s);
    });
    capture_graph(cc, &cc->g_factor, [cc](cudaStream_t s) { return factor_direct(cc, cc->qbuf, s); });
  }
  if (c->cap) SP_CK(cudaStreamSynchronize(c->cap));
  SP_CK(cudaStreamSynchronize(c->stream));
  *out = c.release();
  return SP_OK;
}

sp_status sp_setup(int d, int n, int b, double s, sp_precision prec, const sp_opts* opts,
                   void* stream, sp_ctx** out) try {
  return setup_impl(d, n, b, 1, &s, prec, opts, stream, out);
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_setup_group(int d, int n, int b, int P, const double* shifts, sp_precision prec,
                         const sp_opts* opts, void* stream, sp_ctx** out) try {
  return setup_impl(d, n, b, P, shifts, prec, opts, stream, out);
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_problems(const sp_ctx* c, int* P) {
  if (!c || !P) return SP_ERR_ARG;
  *P = c->P;
  return SP_OK;
}

sp_status sp_factor(sp_ctx* c, const double* q_dev) try {
  if (!c || !q_dev) return SP_ERR_ARG;
  ProfGuard pg_(c);
  SP_CK(cudaSetDevice(c->opts.device));
  cudaStream_t st = c->stream;
  c->factored = false;
  // the context keeps its own copy of q: the factor graph and the operator read it
  if (q_dev != c->qbuf)
    SP_CK(cudaMemcpyAsync(c->qbuf, q_dev, sizeof(double) * c->NP, cudaMemcpyDeviceToDevice, st));
  c->q = c->qbuf;
  if (c->g_factor && !c->profiling) {
    SP_CK(cudaGraphLaunch(c->g_factor, st));
  } else {
    sp_status fs = factor_direct(c, c->qbuf, st);
    if (fs != SP_OK) return fs;
  }
  if (c->mixed) SP_CK(to_float(c->qbuf, c->q32, c->N, st));
  int hs = 0;
  SP_CK(cudaMemcpyAsync(&hs, c->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SP_CK(cudaStreamSynchronize(st));
  if (hs & 2) return SP_ERR_TIMEOUT;
  if (hs) return SP_ERR_SINGULAR;
  c->factored = true;
  return SP_OK;
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_factor_host(sp_ctx* c, const double* q_host) try {
  if (!c || !q_host) return SP_ERR_ARG;
  SP_CK(cudaSetDevice(c->opts.device));
  SP_CK(cudaMemcpyAsync(c->qbuf, q_host, sizeof(double) * c->NP, cudaMemcpyHostToDevice, c->stream));
  return sp_factor(c, c->qbuf);
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_apply(sp_ctx* c, const void* r_dev, void* z_dev) {
  if (!c || !r_dev || !z_dev || r_dev == z_dev) return SP_ERR_ARG;
  ProfGuard pg_(c);
  if (!c->factored) return SP_ERR_STATE;
  SP_CK(cudaSetDevice(c->opts.device));
  return apply_impl(c, (const double2*)r_dev, (double2*)z_dev);
}

sp_status sp_qapply(sp_ctx* c, const void* r_dev, void* y_dev) {
  if (!c || !r_dev || !y_dev) return SP_ERR_ARG;
  ProfGuard pg_(c);
  SP_CK(cudaSetDevice(c->opts.device));
  // always the FP64 tables: the output is complex128 in both forms
  return cuda_status(q_apply(SP_PREC_FP64, c->d, c->n, c->nl, c->qtypes, c->Tcat, c->Tcat32,
                             (const double2*)r_dev, y_dev, c->stream, 1, false, c->P,
                             c->t_stride));
}

sp_status sp_matvec(sp_ctx* c, const void* x_dev, void* w_dev) {
  if (!c || !x_dev || !w_dev) return SP_ERR_ARG;
  ProfGuard pg_(c);
  if (!c->q) return SP_ERR_STATE;
  SP_CK(cudaSetDevice(c->opts.device));
  return cuda_status(fft_green_apply(c->fft, (const double2*)x_dev, c->q, true, (double2*)w_dev,
                                     c->stream, c->P, c->P));
}

sp_status sp_green(sp_ctx* c, const void* f_dev, void* g_dev) {
  if (!c || !f_dev || !g_dev) return SP_ERR_ARG;
  ProfGuard pg_(c);
  SP_CK(cudaSetDevice(c->opts.device));
  return cuda_status(fft_green_apply(c->fft, (const double2*)f_dev, nullptr, false,
                                     (double2*)g_dev, c->stream, c->P, c->P));
}

static sp_status solve_mixed(sp_ctx* c, const double2* f, const double2* u0, double2* u,
                             sp_info* info);

// Start of a solve: g = G f and ||g|| (c->nrm + 2); with a starting vector u0 the
// residual r = g - (I + G q) u0 and its norm (c->nrm + 3), kept only when it is below
// ||g|| (otherwise the zero vector, r = g, is the better start).  *bnorm = ||g||,
// *rel0 = the relative residual of the start.
static sp_status solve_start(sp_ctx* c, const double2* f, const double2* u0, double2* u,
                             double* bnorm, double* rel0, sp_info* info) {
  cudaStream_t st = c->stream;
  const long N = c->N;
  double* hsc = c->host_sc;
  if (info) {
    info->iters = 0;
    info->restarts = 0;
    info->hist_len = 0;
    info->s_used = c->s;
    info->guess_relres = 1.0;
    info->guess_used = 0;
  }
  SP_CK(fft_green_apply(c->fft, f, nullptr, false, c->g, st));
  SP_CK(kr_norm(c->g, N, c->K, c->nrm + 2, st));
  if (u0) {
    if (u0 != u) SP_CK(cudaMemcpyAsync(u, u0, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    SP_CK(fft_green_apply(c->fft, u, c->q, true, c->t, st));
    SP_CK(kr_sub(c->g, c->t, N, c->r, st));
    SP_CK(kr_norm(c->r, N, c->K, c->nrm + 3, st));
    SP_CK(cudaMemcpyAsync(hsc + 1, c->nrm + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  SP_CK(cudaMemcpyAsync(hsc, c->nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
  SP_CK(cudaStreamSynchronize(st));
  *bnorm = hsc[0];
  *rel0 = 1.0;
  if (u0 && hsc[0] > 0.0) {
    const double g0 = hsc[1] / hsc[0];
    if (info) info->guess_relres = g0;
    if (g0 < 1.0) {  // the guess beats the zero vector
      if (info) info->guess_used = 1;
      *rel0 = g0;
      return SP_OK;
    }
  }
  SP_CK(cudaMemsetAsync(u, 0, sizeof(double2) * N, st));
  SP_CK(cudaMemcpyAsync(c->r, c->g, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
  SP_CK(cudaMemcpyAsync(c->nrm + 3, c->nrm + 2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return SP_OK;
}

// R right-hand sides of every problem of the context (R P instances; instance
// i = r P + p, right-hand side r of problem p, at offset i N of F and U) through the
// cycle graph of build_cycle_graph: the host waits once per restart cycle, where the
// true residuals decide which instances restart.  u0 (one instance only): the start
// of sp_solve_x0.  Every instance runs the kernels of the host-driven iteration with
// the same operands, so its result is bit-identical to that iteration's for its
// right-hand side and problem.
static sp_status solve_batch(sp_ctx* c, int R, const double2* F, const double2* u0, double2* U,
                             sp_info* infos) {
  cudaStream_t st = c->stream;
  const long N = c->N;
  const int I = R * c->P;
  const double tol = c->opts.tol;
  const int maxit = c->opts.maxit;
  if (R < 1 || R > c->opts.max_rhs || (u0 && I != 1)) return SP_ERR_ARG;
  if (!c->g_cycle[R] || c->g_cycle_q[R] != c->q) {
    SP_CK(cudaStreamSynchronize(st));
    sp_status bs = build_cycle_graph(c, R);
    if (bs != SP_OK) return bs;
  }
  const KBatch b = make_batch(c);
  double2* uw = c->ubuf;
  std::vector<double> bnorm(I, 0.0), rel0(I, 1.0);
  if (u0) {
    sp_status s0 = solve_start(c, F, u0, uw, &bnorm[0], &rel0[0], infos);
    if (s0 != SP_OK) return s0;
  } else {
    if (infos)
      for (int i = 0; i < I; ++i) {
        infos[i].iters = 0;
        infos[i].restarts = 0;
        infos[i].hist_len = 0;
        infos[i].s_used = c->shifts[i % c->P];
        infos[i].guess_relres = 1.0;
        infos[i].guess_used = 0;
      }
    // g_i = G_p f_i, ||g_i||; u = 0, r = g
    SP_CK(fft_green_apply(c->fft, F, nullptr, false, c->g, st, I, c->P));
    SP_CK(kb_norm(b, I, c->g, 2, st));
    SP_CK(cudaMemsetAsync(uw, 0, sizeof(double2) * N * I, st));
    SP_CK(cudaMemcpyAsync(c->r, c->g, sizeof(double2) * N * I, cudaMemcpyDeviceToDevice, st));
    SP_CK(kb_copy_nrm(b, I, 2, 3, st));
    SP_CK(cudaMemcpy2DAsync(c->host_sc, sizeof(double), c->nrm + 2, 4 * sizeof(double),
                            sizeof(double), I, cudaMemcpyDeviceToHost, st));
    SP_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < I; ++i) bnorm[i] = c->host_sc[i];
  }
  auto push = [&](int i, double v) {
    sp_info* in = infos ? infos + i : nullptr;
    if (in && in->hist && in->hist_len < in->hist_cap) in->hist[in->hist_len++] = v;
  };
  std::vector<int> total(I, 0), restarts(I, 0);
  std::vector<double> est(I), tr(I);
  int nrun = 0;
  for (int i = 0; i < I; ++i) {
    push(i, rel0[i]);
    est[i] = tr[i] = rel0[i];
    int run = 0;
    if (bnorm[i] == 0.0) {
      est[i] = tr[i] = 0.0;
      SP_CK(cudaMemsetAsync(uw + i * N, 0, sizeof(double2) * N, st));
    } else if (rel0[i] > tol) {
      run = 1;
      ++nrun;
    }
    c->host_run[i] = run;
  }
  if (nrun) SP_CK(cudaMemsetAsync(c->heads, 0, sizeof(LoopHead) * I, st));
  while (nrun) {
    SP_CK(cudaMemcpyAsync(c->run, c->host_run, sizeof(int) * I, cudaMemcpyHostToDevice, st));
    SP_CK(cudaGraphLaunch(c->g_cycle[R], st));
    SP_CK(cudaStreamSynchronize(st));
    nrun = 0;
    for (int i = 0; i < I; ++i) {
      if (!c->host_run[i]) continue;
      const LoopHead& h = c->host_heads[i];
      for (int t = total[i]; t < h.total && t < maxit; ++t)
        push(i, c->host_hist[(long)i * maxit + t]);
      total[i] = h.total;
      est[i] = h.est_rel;
      tr[i] = h.rnorm / bnorm[i];
      if (tr[i] <= tol || total[i] >= maxit) {
        c->host_run[i] = 0;
      } else {
        ++restarts[i];
        ++nrun;
      }
    }
  }
  if (U != uw) SP_CK(cudaMemcpyAsync(U, uw, sizeof(double2) * N * I, cudaMemcpyDeviceToDevice, st));
  SP_CK(cudaStreamSynchronize(st));
  bool all = true;
  for (int i = 0; i < I; ++i) {
    if (infos) {
      infos[i].iters = total[i];
      infos[i].restarts = restarts[i];
      infos[i].est_relres = est[i];
      infos[i].true_relres = tr[i];
    }
    if (!(tr[i] <= tol)) all = false;
  }
  return all ? SP_OK : SP_ERR_NOCONV;
}

static sp_status solve_impl(sp_ctx* c, const double2* f, const double2* u0, double2* u,
                            sp_info* info) {
  if (c->mixed) return solve_mixed(c, f, u0, u, info);
  if (c->P > 1 || (c->opts.device_loop && !c->profiling))
    return solve_batch(c, 1, f, u0, u, info);
  cudaStream_t st = c->stream;
  const long N = c->N;
  double* hsc = c->host_sc;
  const int restart = c->opts.restart;
  const double tol = c->opts.tol;
  auto push_hist = [&](double v) {
    if (info && info->hist && info->hist_len < info->hist_cap) info->hist[info->hist_len++] = v;
  };
  double bnorm = 0.0, rel0 = 1.0;
  sp_status s0 = solve_start(c, f, u0, u, &bnorm, &rel0, info);
  if (s0 != SP_OK) return s0;
  push_hist(rel0);
  if (bnorm == 0.0) {
    SP_CK(cudaMemsetAsync(u, 0, sizeof(double2) * N, st));
    SP_CK(cudaStreamSynchronize(st));
    if (info) info->true_relres = info->est_relres = 0.0;
    return SP_OK;
  }
  if (rel0 <= tol) {
    if (info) info->true_relres = info->est_relres = rel0;
    return SP_OK;
  }
  int total = 0, restarts = 0;
  double est_rel = rel0, true_rel = rel0;
  const int maxit = c->opts.maxit;
  for (;;) {
    SP_CK(kr_start(c->r, N, c->nrm + 3, c->V, c->gam, c->maxv + 1, st));
    int k = 0;
    for (int j = 0; j < restart; ++j) {
      double2* vj = c->V + (long)j * N;
      double2* zj = c->Z + (long)j * N;
      double2* w = c->V + (long)(j + 1) * N;
      sp_status ss = apply_impl(c, vj, zj);
      if (ss != SP_OK) return ss;
      SP_CK(fft_green_apply(c->fft, zj, c->q, true, w, st));
      // classical Gram-Schmidt, twice
      SP_CK(kr_dots(c->V, N, j + 1, w, N, c->K, c->h1, st));
      SP_CK(kr_update_dots(c->V, N, j + 1, w, N, c->h1, c->K, c->h2, st));
      SP_CK(kr_update_dots(c->V, N, j + 1, w, N, c->h2, c->K, nullptr, st));
      SP_CK(kr_norm(w, N, c->K, c->nrm, st));
      SP_CK(kr_givens(c->H, c->maxv, j, c->h1, c->h2, c->nrm, c->cs, c->sn, c->gam, c->est, st));
      SP_CK(cudaMemcpyAsync(hsc, c->est, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      SP_CK(cudaStreamSynchronize(st));
      ++total;
      k = j + 1;
      est_rel = hsc[0] / bnorm;
      push_hist(est_rel);
      if (est_rel <= tol || total >= maxit || hsc[1] == 0.0) break;
      SP_CK(kr_scale(w, N, c->nrm, w, st));
    }
    SP_CK(kr_update_solution(c->H, c->maxv, k, c->gam, c->y, c->Z, N, N, u, st));
    // true residual r = g - A u
    SP_CK(fft_green_apply(c->fft, u, c->q, true, c->t, st));
    SP_CK(kr_sub(c->g, c->t, N, c->r, st));
    SP_CK(kr_norm(c->r, N, c->K, c->nrm + 3, st));
    SP_CK(cudaMemcpyAsync(hsc + 2, c->nrm + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    SP_CK(cudaStreamSynchronize(st));
    true_rel = hsc[2] / bnorm;
    if (true_rel <= tol || total >= maxit) break;
    ++restarts;
  }
  if (info) {
    info->iters = total;
    info->restarts = restarts;
    info->est_relres = est_rel;
    info->true_relres = true_rel;
  }
  return true_rel <= tol ? SP_OK : SP_ERR_NOCONV;
}

sp_status sp_solve(sp_ctx* c, const void* f_dev, void* u_dev, sp_info* info) try {
  if (!c || !f_dev || !u_dev) return SP_ERR_ARG;
  ProfGuard pg_(c);
  if (!c->factored) return SP_ERR_STATE;
  SP_CK(cudaSetDevice(c->opts.device));
  return solve_impl(c, (const double2*)f_dev, nullptr, (double2*)u_dev, info);
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_solve_x0(sp_ctx* c, const void* f_dev, const void* u0_dev, void* u_dev, sp_info* info) try {
  if (!c || !f_dev || !u_dev || (u0_dev && c->P > 1)) return SP_ERR_ARG;
  ProfGuard pg_(c);
  if (!c->factored) return SP_ERR_STATE;
  SP_CK(cudaSetDevice(c->opts.device));
  return solve_impl(c, (const double2*)f_dev, (const double2*)u0_dev, (double2*)u_dev, info);
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

// GMRES-IR: outer refinement in FP64, inner flexible GMRES in complex64.
static sp_status solve_mixed(sp_ctx* c, const double2* f, const double2* u0, double2* u,
                             sp_info* info) {
  cudaStream_t st = c->stream;
  const long N = c->N;
  double* hsc = c->host_sc;
  const int restart = c->opts.restart;
  const double tol = c->opts.tol, tin = c->opts.inner_tol;
  auto push_hist = [&](double v) {
    if (info && info->hist && info->hist_len < info->hist_cap) info->hist[info->hist_len++] = v;
  };
  float2* V32 = reinterpret_cast<float2*>(c->V);  // (restart + 1) complex64 vectors
  double bnorm = 0.0, rel0 = 1.0;
  sp_status s0 = solve_start(c, f, u0, u, &bnorm, &rel0, info);
  if (s0 != SP_OK) return s0;
  push_hist(rel0);
  if (bnorm == 0.0) {
    SP_CK(cudaMemsetAsync(u, 0, sizeof(double2) * N, st));
    SP_CK(cudaStreamSynchronize(st));
    if (info) info->true_relres = info->est_relres = 0.0;
    return SP_OK;
  }
  if (rel0 <= tol) {
    if (info) info->true_relres = info->est_relres = rel0;
    return SP_OK;
  }
  double rel = rel0, est_rel = rel0;
  int total = 0, outer = 0;
  const int maxit = c->opts.maxit;
  for (;;) {
    // inner: A d = r / ||r|| in complex64, flexible GMRES, Z_j kept in FP64
    SP_CK(kr32_start(c->r, N, c->nrm + 3, V32, c->gam, c->maxv + 1, st));
    int k = 0;
    for (int j = 0; j < restart; ++j) {
      const float2* vj = V32 + (long)j * N;
      double2* zj = c->Z + (long)j * N;
      float2* w = V32 + (long)(j + 1) * N;
      SP_CK(kr_widen(vj, N, c->t, st));
      sp_status ss = apply_impl(c, c->t, zj);
      if (ss != SP_OK) return ss;
      SP_CK(kr_narrow(zj, N, c->z32, st));
      SP_CK(fft_green_apply32(c->fft, c->z32, c->q32, true, w, st));
      SP_CK(kr32_dots(V32, N, j + 1, w, N, c->K, c->h1, st));
      SP_CK(kr32_update_dots(V32, N, j + 1, w, N, c->h1, c->K, c->h2, st));
      SP_CK(kr32_update_dots(V32, N, j + 1, w, N, c->h2, c->K, nullptr, st));
      SP_CK(kr32_norm(w, N, c->K, c->nrm, st));
      SP_CK(kr_givens(c->H, c->maxv, j, c->h1, c->h2, c->nrm, c->cs, c->sn, c->gam, c->est, st));
      SP_CK(cudaMemcpyAsync(hsc, c->est, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      SP_CK(cudaStreamSynchronize(st));
      ++total;
      k = j + 1;
      est_rel = hsc[0] * rel;  // inner estimate scaled to ||g||
      push_hist(est_rel);
      if (hsc[0] <= tin || est_rel <= tol || total >= maxit || hsc[1] == 0.0) break;
      SP_CK(kr32_scale(w, N, c->nrm, st));
    }
    // u += ||r|| Z y
    SP_CK(kr_trisolve(c->H, c->maxv, k, c->gam, c->y, st));
    SP_CK(kr_scale_y(c->y, k, c->nrm + 3, st));
    SP_CK(kr_combine(c->Z, N, k, c->y, N, u, st));
    // FP64 residual
    SP_CK(fft_green_apply(c->fft, u, c->q, true, c->t, st));
    SP_CK(kr_sub(c->g, c->t, N, c->r, st));
    SP_CK(kr_norm(c->r, N, c->K, c->nrm + 3, st));
    SP_CK(cudaMemcpyAsync(hsc + 2, c->nrm + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    SP_CK(cudaStreamSynchronize(st));
    rel = hsc[2] / bnorm;
    ++outer;
    if (rel <= tol || total >= maxit) break;
  }
  if (info) {
    info->iters = total;
    info->restarts = outer - 1;
    info->est_relres = est_rel;
    info->true_relres = rel;
  }
  return rel <= tol ? SP_OK : SP_ERR_NOCONV;
}

// z = P^{-1} Q r for nv stacked vectors (direct launches; each vector's result
// equals apply_direct's for it)
sp_status sp_solve_many(sp_ctx* c, int nrhs, const void* F_dev, void* U_dev, sp_info* infos) try {
  if (!c || !F_dev || !U_dev || nrhs < 1 || nrhs > c->opts.max_rhs) return SP_ERR_ARG;
  if (!c->factored) return SP_ERR_STATE;
  SP_CK(cudaSetDevice(c->opts.device));
  const long N = c->N;
  const double2* F = (const double2*)F_dev;
  double2* U = (double2*)U_dev;
  if (!c->mixed && (c->P > 1 || (c->opts.device_loop && !c->profiling))) {
    ProfGuard pg_(c);
    return solve_batch(c, nrhs, F, nullptr, U, infos);
  }
  if (c->mixed || nrhs == 1) {
    sp_status worst = SP_OK;
    for (int r = 0; r < nrhs; ++r) {
      sp_status s1 = sp_solve(c, F + r * N, U + r * N, infos ? infos + r : nullptr);
      if (s1 != SP_OK && s1 != SP_ERR_NOCONV) return s1;
      if (s1 != SP_OK) worst = s1;
    }
    return worst;
  }
  ProfGuard pg_(c);
  cudaStream_t st = c->stream;
  const int restart = c->opts.restart, maxit = c->opts.maxit, mv = c->maxv;
  const double tol = c->opts.tol;
  double* hsc = c->host_sc;
  // per right-hand side r: slices of the Krylov workspace
  auto V = [&](int r) { return c->V + (long)r * mv * N; };
  auto Z = [&](int r) { return c->Z + (long)r * restart * N; };
  auto H = [&](int r) { return c->H + (long)r * mv * restart; };
  auto GAM = [&](int r) { return c->gam + (long)r * (mv + 1); };
  auto SN = [&](int r) { return c->sn + (long)r * (mv + 1); };
  auto CS = [&](int r) { return c->cs + (long)r * (mv + 1); };
  auto H1 = [&](int r) { return c->h1 + (long)r * 1024; };
  auto H2 = [&](int r) { return c->h2 + (long)r * 1024; };
  auto Y = [&](int r) { return c->y + (long)r * 1024; };
  auto NRM = [&](int r) { return c->nrm + (long)r * 4; };
  auto EST = [&](int r) { return c->est + (long)r * 4; };
  auto Gv = [&](int r) { return c->g + (long)r * N; };
  auto Rv = [&](int r) { return c->r + (long)r * N; };
  auto Tv = [&](int r) { return c->t + (long)r * N; };
  struct Rhs {
    double bnorm = 0, est_rel = 1, true_rel = 1;
    int j = 0, total = 0, restarts = 0;
    bool done = false;
  };
  std::vector<Rhs> R(nrhs);
  auto push_hist = [&](int r, double v) {
    sp_info* in = infos ? infos + r : nullptr;
    if (in && in->hist && in->hist_len < in->hist_cap) in->hist[in->hist_len++] = v;
  };
  if (infos)
    for (int r = 0; r < nrhs; ++r) {
      infos[r].iters = 0;
      infos[r].restarts = 0;
      infos[r].hist_len = 0;
      infos[r].s_used = c->s;
      infos[r].guess_relres = 1.0;
      infos[r].guess_used = 0;
    }
  // g_r = G f_r, ||g_r||
  SP_CK(fft_green_apply(c->fft, F, nullptr, false, c->g, st, nrhs));
  for (int r = 0; r < nrhs; ++r) SP_CK(kr_norm(Gv(r), N, c->K, NRM(r) + 2, st));
  SP_CK(cudaMemcpy2DAsync(hsc, sizeof(double), c->nrm + 2, 4 * sizeof(double), sizeof(double),
                          nrhs, cudaMemcpyDeviceToHost, st));
  SP_CK(cudaMemsetAsync(U, 0, sizeof(double2) * N * nrhs, st));
  SP_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < nrhs; ++r) {
    R[r].bnorm = hsc[r];
    push_hist(r, 1.0);
    if (R[r].bnorm == 0.0) {
      R[r].done = true;
      R[r].est_rel = R[r].true_rel = 0.0;
      continue;
    }
    SP_CK(cudaMemcpyAsync(Rv(r), Gv(r), sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    SP_CK(cudaMemcpyAsync(NRM(r) + 3, NRM(r) + 2, sizeof(double), cudaMemcpyDeviceToDevice, st));
    SP_CK(kr_start(Rv(r), N, NRM(r) + 3, V(r), GAM(r), mv + 1, st));
  }
  // u_r += Z_r y, true residual, then either stop or restart
  auto finish_cycle = [&](int r, int k) -> sp_status {
    Rhs& h = R[r];
    double2* u = U + (long)r * N;
    SP_CK(kr_update_solution(H(r), mv, k, GAM(r), Y(r), Z(r), N, N, u, st));
    SP_CK(fft_green_apply(c->fft, u, c->q, true, Tv(r), st));
    SP_CK(kr_sub(Gv(r), Tv(r), N, Rv(r), st));
    SP_CK(kr_norm(Rv(r), N, c->K, NRM(r) + 3, st));
    SP_CK(cudaMemcpyAsync(hsc, NRM(r) + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    SP_CK(cudaStreamSynchronize(st));
    h.true_rel = hsc[0] / h.bnorm;
    if (h.true_rel <= tol || h.total >= maxit) {
      h.done = true;
    } else {
      ++h.restarts;
      h.j = 0;
      SP_CK(kr_start(Rv(r), N, NRM(r) + 3, V(r), GAM(r), mv + 1, st));
    }
    return SP_OK;
  };
  std::vector<int> act;
  for (;;) {
    act.clear();
    for (int r = 0; r < nrhs; ++r)
      if (!R[r].done) act.push_back(r);
    if (act.empty()) break;
    const int na = (int)act.size();
    const size_t vb = sizeof(double2) * N;
    for (int s = 0; s < na; ++s)
      SP_CK(cudaMemcpyAsync(c->app_in + s * N, V(act[s]) + (long)R[act[s]].j * N, vb,
                            cudaMemcpyDeviceToDevice, st));
    if (!c->g_block_tried[na] && !c->profiling && c->cap) {
      // capture the block application of na vectors once (app_in -> app_out); the
      // capture stream waits for the copies just issued
      c->g_block_tried[na] = true;
      SP_CK(cudaStreamSynchronize(st));
      capture_graph(c, &c->g_block[na], [c, na](cudaStream_t s2) {
        return apply_block(c, na, c->app_in, c->app_out, s2);
      });
    }
    if (c->g_block[na] && !c->profiling) {
      SP_CK(cudaGraphLaunch(c->g_block[na], st));
    } else {
      sp_status ss = apply_block(c, na, c->app_in, c->app_out, st);
      if (ss != SP_OK) return ss;
    }
    SP_CK(fft_green_apply(c->fft, c->app_out, c->q, true, c->blk_w, st, na));
    for (int s = 0; s < na; ++s) {
      const int r = act[s], j = R[r].j;
      double2* w = V(r) + (long)(j + 1) * N;
      SP_CK(cudaMemcpyAsync(Z(r) + (long)j * N, c->app_out + s * N, vb, cudaMemcpyDeviceToDevice,
                            st));
      SP_CK(cudaMemcpyAsync(w, c->blk_w + s * N, vb, cudaMemcpyDeviceToDevice, st));
      // classical Gram-Schmidt, twice
      SP_CK(kr_dots(V(r), N, j + 1, w, N, c->K, H1(r), st));
      SP_CK(kr_update_dots(V(r), N, j + 1, w, N, H1(r), c->K, H2(r), st));
      SP_CK(kr_update_dots(V(r), N, j + 1, w, N, H2(r), c->K, nullptr, st));
      SP_CK(kr_norm(w, N, c->K, NRM(r), st));
      SP_CK(kr_givens(H(r), mv, j, H1(r), H2(r), NRM(r), CS(r), SN(r), GAM(r), EST(r), st));
    }
    SP_CK(cudaMemcpyAsync(hsc, c->est, 4 * sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    SP_CK(cudaStreamSynchronize(st));
    std::vector<double> est(hsc, hsc + 4 * nrhs);
    for (int s = 0; s < na; ++s) {
      const int r = act[s];
      Rhs& h = R[r];
      ++h.total;
      const int k = h.j + 1;
      h.est_rel = est[4 * r] / h.bnorm;
      push_hist(r, h.est_rel);
      if (h.est_rel <= tol || h.total >= maxit || est[4 * r + 1] == 0.0 || k == restart) {
        sp_status fs = finish_cycle(r, k);
        if (fs != SP_OK) return fs;
      } else {
        double2* w = V(r) + (long)k * N;
        SP_CK(kr_scale(w, N, NRM(r), w, st));
        h.j = k;
      }
    }
  }
  bool all = true;
  for (int r = 0; r < nrhs; ++r) {
    if (infos) {
      infos[r].iters = R[r].total;
      infos[r].restarts = R[r].restarts;
      infos[r].est_relres = R[r].est_rel;
      infos[r].true_relres = R[r].true_rel;
    }
    if (!(R[r].true_rel <= tol)) all = false;
  }
  return all ? SP_OK : SP_ERR_NOCONV;
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_solve_host(sp_ctx* c, const void* f_host, void* u_host, sp_info* info) try {
  if (!c || !f_host || !u_host) return SP_ERR_ARG;
  SP_CK(cudaSetDevice(c->opts.device));
  SP_CK(cudaMemcpyAsync(c->fbuf, f_host, sizeof(double2) * c->NP, cudaMemcpyHostToDevice, c->stream));
  sp_status st = sp_solve(c, c->fbuf, c->ubuf, info);
  if (st != SP_OK && st != SP_ERR_NOCONV) return st;
  SP_CK(cudaMemcpyAsync(u_host, c->ubuf, sizeof(double2) * c->NP, cudaMemcpyDeviceToHost, c->stream));
  SP_CK(cudaStreamSynchronize(c->stream));
  return st;
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_schur_update(sp_precision prec, int M, int N, int K, const void* A, int lda,
                          long long sA, const void* B, int ldb, long long sB, void* C, int ldc,
                          long long sC, int batch, void* stream) try {
  if (prec != SP_PREC_FP64 && prec != SP_PREC_FP32 && prec != SP_PREC_TF32 &&
      prec != SP_PREC_TF32X3)
    return SP_ERR_ARG;
  if (M < 0 || N < 0 || K < 0 || batch < 0 || !A || !B || !C) return SP_ERR_ARG;
  if (lda < std::max(1, M) || ldb < std::max(1, K) || ldc < std::max(1, M)) return SP_ERR_ARG;
  if (sA < 0 || sB < 0 || sC < 0 || batch > 65535) return SP_ERR_ARG;
  const bool tc = prec == SP_PREC_TF32 || prec == SP_PREC_TF32X3;
  const bool split = prec == SP_PREC_TF32X3;
  if (tc && K > kTcMaxKProbe) return SP_ERR_ARG;
  if ((long long)M * N * K * batch == 0) return SP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  float *pa = nullptr, *pb = nullptr;
  int* status = nullptr;
  sp_status rs = SP_OK;
  cudaError_t e = cudaSuccess;
  if (tc) {
    e = cudaMalloc(&pa, sizeof(float) * tc_pack_floats(M, K, batch, split));
    if (e == cudaSuccess) e = cudaMalloc(&pb, sizeof(float) * tc_pack_floats(N, K, batch, split));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  }
  if (e == cudaSuccess)
    e = schur_update_raw(tc ? SP_PREC_FP32 : prec, tc, split, M, N, K, A, lda, sA, B, ldb, sB, C,
                         ldc, sC, batch, pa, pb, status, st);
  int hs = 0;
  if (e == cudaSuccess && tc) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  rs = cuda_status(e);
  if (rs == SP_OK && (hs & 2)) rs = SP_ERR_TIMEOUT;
  if (pa) cudaFree(pa);
  if (pb) cudaFree(pb);
  if (status) cudaFree(status);
  return rs;
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_tc_probe(int split, int M, int N, int K, int reps, void* stream, double* ms_per_launch) try {
  if ((split != 0 && split != 1) || !ms_per_launch || reps < 1 || reps > 1000) return SP_ERR_ARG;
  if (M < 128 || N < 256 || K < 32 || M % 128 || N % 256 || K % 32 || M > 16384 || N > 16384 ||
      K > kTcMaxKProbe)
    return SP_ERR_ARG;
  float ms = 0.f;
  int hs = 0;
  cudaError_t e = tc_probe(split != 0, M, N, K, reps, (cudaStream_t)stream, &ms, &hs);
  sp_status rs = cuda_status(e);
  if (rs == SP_OK && (hs & 2)) rs = SP_ERR_TIMEOUT;
  *ms_per_launch = ms;
  return rs;
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_tuning(const sp_ctx* c, int level, int* gemm_tile, int* gen_tile) {
  if (!c || level < 0 || level > c->L) return SP_ERR_ARG;
  const DevLevel& D = c->lv[level];
  if (gemm_tile) *gemm_tile = D.gemm_tile;
  if (gen_tile) *gen_tile = D.gen_tile;
  return SP_OK;
}

sp_status sp_get_table(const sp_ctx* c, int t, double* Q_out, double* C_out, int* rows, int* cols,
                       int* rank) {
  if (!c || t < 0 || t >= (int)c->tabs.size()) return SP_ERR_ARG;
  const StencilTable& tb = c->tabs[t];
  if (rows) *rows = tb.nS;
  if (cols) *cols = tb.nG;
  if (rank) *rank = tb.rank;
  if (Q_out) std::memcpy(Q_out, tb.Q.data(), tb.Q.size() * sizeof(double));
  if (C_out) std::memcpy(C_out, tb.C.data(), tb.C.size() * sizeof(double));
  return SP_OK;
}

sp_status sp_set_table(sp_ctx* c, int t, const double* Q_in, const double* C_in) try {
  if (!c || t < 0 || t >= (int)c->tabs.size() || !Q_in || !C_in) return SP_ERR_ARG;
  StencilTable& tb = c->tabs[t];
  // table t of a group: problem t / 2^d, type t mod 2^d
  const long pg = t >> c->d;
  const QTypeDev& qt = c->qtypes[t & ((1 << c->d) - 1)];
  const long toff = qt.tab_off + pg * c->work.tab_stride, tt_off = qt.t_off + pg * c->t_stride;
  const size_t ne = (size_t)tb.nS * tb.nG;
  for (size_t e = 0; e < ne; ++e)
    if (!std::isfinite(Q_in[e]) || !std::isfinite(C_in[e])) return SP_ERR_ARG;
  // columns of gamma that are not in S (gamma order lists S and beta interleaved)
  std::vector<int> scol, bcols;
  {
    int sidx = 0;
    for (int gi = 0; gi < tb.nG; ++gi) {
      bool inS = sidx < tb.nS;
      for (int a = 0; a < c->d && inS; ++a)
        if (tb.G[(size_t)gi * c->d + a] != tb.S[(size_t)sidx * c->d + a]) inS = false;
      if (inS) {
        scol.push_back(gi);
        ++sidx;
      } else {
        bcols.push_back(gi);
      }
    }
  }
  if (qt.self) {
    if ((int)scol.size() != tb.nS) return SP_ERR_ARG;
    for (int a = 0; a < tb.nS; ++a)
      for (int j = 0; j < tb.nS; ++j)
        if (Q_in[(size_t)a * tb.nG + scol[j]] != (a == j ? 1.0 : 0.0)) return SP_ERR_ARG;
  } else {
    bcols.resize(tb.nG);
    for (int gi = 0; gi < tb.nG; ++gi) bcols[gi] = gi;
  }
  if ((int)bcols.size() != qt.na) return SP_ERR_ARG;
  std::vector<double> Qc(ne), Cc(ne), Tc((size_t)tb.nS * qt.na);
  std::vector<float> T32(Tc.size());
  for (int col = 0; col < tb.nG; ++col)
    for (int a = 0; a < tb.nS; ++a) {
      Qc[(size_t)col * tb.nS + a] = Q_in[(size_t)a * tb.nG + col];
      Cc[(size_t)col * tb.nS + a] = C_in[(size_t)a * tb.nG + col];
    }
  for (int cb = 0; cb < qt.na; ++cb)
    for (int a = 0; a < tb.nS; ++a) {
      const double v = -Q_in[(size_t)a * tb.nG + bcols[cb]];
      Tc[(size_t)cb * tb.nS + a] = v;
      T32[(size_t)cb * tb.nS + a] = (float)v;
    }
  SP_CK(cudaSetDevice(c->opts.device));
  cudaStream_t st = c->stream;
  SP_CK(cudaMemcpyAsync(c->Qcat + toff, Qc.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, st));
  SP_CK(cudaMemcpyAsync(c->Ccat + toff, Cc.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, st));
  SP_CK(cudaMemcpyAsync(c->Tcat + tt_off, Tc.data(), sizeof(double) * Tc.size(),
                        cudaMemcpyHostToDevice, st));
  SP_CK(cudaMemcpyAsync(c->Tcat32 + tt_off, T32.data(), sizeof(float) * T32.size(),
                        cudaMemcpyHostToDevice, st));
  SP_CK(cudaStreamSynchronize(st));
  tb.Q.assign(Q_in, Q_in + ne);
  tb.C.assign(C_in, C_in + ne);
  c->factored = false;
  return SP_OK;
} catch (const std::exception&) {  // host memory or threads: no exception crosses the ABI
  return SP_ERR_OOM;
}

sp_status sp_profile(sp_ctx* c, int enable) {
  if (!c) return SP_ERR_ARG;
  c->profiling = enable != 0;
  return SP_OK;
}

sp_status sp_profile_read(sp_ctx* c, int cap, double* ms, int* launches, double* work) {
  if (!c || cap < PROF_NCLASS) return SP_ERR_ARG;
  SP_CK(cudaSetDevice(c->opts.device));
  return cuda_status(c->prof.read(ms, launches, work, cap));
}

sp_status sp_costs(const sp_ctx* c, double* factor_entries, double* factor_flops,
                   double* apply_bytes) {
  if (!c) return SP_ERR_ARG;
  if (factor_entries) *factor_entries = c->factor_entries;
  if (factor_flops) *factor_flops = c->factor_flops;
  if (apply_bytes) *apply_bytes = c->apply_bytes;
  return SP_OK;
}

}  // extern "C"
