// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/sp.h"
#include "sp_host.h"

namespace sp {

// Levels with few fronts keep the inverses of the diagonal blocks of this size of
// L11 and U11 (the sweep is a chain of k / kInvBlockSize matrix-vector steps).
constexpr int kInvBlockSize = 512;

// Optional per-kernel-class timing with CUDA events on the launching stream.
enum ProfClass {
  PROF_ASSEMBLE = 0,  // zeroing, assembly of P, extend-add, front scale
  PROF_LU_PANEL = 1,
  PROF_LU_TRSM = 2,
  PROF_LU_GEMM = 3,
  PROF_QAPPLY = 4,
  PROF_FORWARD = 5,
  PROF_BACKWARD = 6,
  PROF_FFT = 7,
  PROF_KRYLOV = 8,
  PROF_LU_TRINV = 9,  // explicit triangular inverses of few-front levels
  PROF_LU_TC = 10,    // tensor-core Schur updates of the blocked fronts (with operand packing)
  PROF_NCLASS = 11
};
struct Profiler {
  struct Rec {
    int cls;
    cudaEvent_t a, b;
    double work;
    int launches;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t get();
  int begin(int cls, cudaStream_t st);
  void end(int tok, double work, int launches, cudaStream_t st);
  // sums per class (ms, launches, work) and resets
  cudaError_t read(double* ms, int* launches, double* work, int cap);
  void destroy();
};
extern thread_local Profiler* g_prof;
struct ProfScope {
  int tok = -1;
  ProfScope(int cls, cudaStream_t st) {
    if (g_prof) tok = g_prof->begin(cls, st);
  }
  void done(double work, int launches, cudaStream_t st) {
    if (g_prof && tok >= 0) g_prof->end(tok, work, launches, st);
    tok = -1;
  }
};

// Per-level device data of the multifrontal factor (fronts column-major, m x m).
struct DevLevel {
  int nf = 0, k = 0, m = 0, nb1 = 0, mc = 0, kc = 0, nasm = 0;
  int* gidx = nullptr;      // nf x m
  int* asm_row = nullptr;   // nasm front rows (columns: asm_cvar)
  int* asm_tidx = nullptr;
  int* asm_cvar = nullptr;
  int* ea_map = nullptr;    // 2^d x (mc - kc)
  void* front = nullptr;    // nf x m x m of double (FP64) or float (FP32)
  int* perm = nullptr;      // nf x k row permutation of the eliminated block
  int* piv = nullptr;       // nf x k pivot rows (LAPACK style, 0-based within the front)
  double* scale = nullptr;  // nf: max |entry| of the assembled front
  void* upd = nullptr;      // nf x (m - k) complex update vectors of the forward sweep
  void* y = nullptr;        // nf x k complex forward-sweep results
  bool inv = false;         // L11, U11 replaced by their inverses; sweeps are GEMVs
  void* tmp = nullptr;      // nf x m complex work vector of the GEMV sweeps (inv levels)
  // launch shapes (0 = built-in heuristic; set by the autotuner): Schur-update tile
  // (32 or 64) and general GEMM tile of the block inverses (32 or 64); every output
  // entry keeps its summation order, so the choice never changes a result
  int gemm_tile = 0, gen_tile = 0;
  int ib = kInvBlockSize;   // diagonal-block size of the block inverses (inv levels)
  // fused sweeps (inv levels whose work vectors fit in shared memory): CTAs per
  // front (a thread-block cluster; 0 = the per-block launch chain) and threads per CTA
  int fused_c = 0, fused_nt = 0;
  int pdl = 0;  // launch the level's sweep kernels with programmatic dependent launch
  // fronts per problem: a context of P problems (a problem group) holds P nfp fronts
  // per level, problem p's at [p nfp, (p + 1) nfp) with grid indices offset by p N
  int nfp = 0;
  // FP16 copy of the fronts for the chained sweeps (sp_opts.factor_storage = 1):
  // entry (r, c) of front f stored as entry / fscale16[f m + c] rounded to half, a
  // power-of-two scale per column (the Schur block, rows and columns >= k, not copied)
  void* front16 = nullptr;       // nf m ld16 halves, ld16 = m rounded up to even
  float* fscale16 = nullptr;     // nf m
};

// ---------------------------------------------------------------- FFT (sp_fft.cu)
struct FftPlan {
  int d = 0, n = 0, logn = 0;  // n = 2^p or 3 2^p
  double2* tw = nullptr;   // exp(-2 pi i t / n), t < n/2
  double* Dn = nullptr;    // 1 / (4 pi^2 |k|^2 - s) / N, flat (one per problem of a group)
  double2* tmp = nullptr;  // N work (times the context's max_rhs)
  float2* tw32 = nullptr;  // FP32 copies for the mixed-precision inner solve
  float* Dn32 = nullptr;
  float2* tmp32 = nullptr;
};
// w = x + G (q x) when q != null and add_x; g = G f when q == null and !add_x.
// nvec vectors stacked N apart (the plan's tmp holds nvec N entries).  qper > 1 (a
// problem group): the plan holds qper symbols Dn N apart and q holds qper media N
// apart; vector v uses those of problem v % qper (nvec a multiple of qper).
cudaError_t fft_green_apply(const FftPlan& P, const double2* x, const double* q, bool add_x,
                            double2* out, cudaStream_t st, int nvec = 1, int qper = 1);
cudaError_t fft_green_apply32(const FftPlan& P, const float2* x, const float* q, bool add_x,
                              float2* out, cudaStream_t st);
cudaError_t to_float(const double* a, float* b, long N, cudaStream_t st);

// ---------------------------------------------------------------- factor (sp_factor.cu)
// Work buffers of the factorisation, shared by all levels.
struct FactorWork {
  void* inv = nullptr;        // invert_scratch_elems entries of the factor type (L.inv levels)
  float* packA = nullptr;     // tensor-core operand buffers (tc_pack_floats each)
  float* packB = nullptr;
  bool tc = false;            // Schur updates of the blocked fronts on the tensor cores
  bool tc_split = false;      // ... as 3xTF32 (hi/lo split, FP32 accuracy)
  int tc_epi = 0;             // epilogue of the tensor-core update (tc_schur_update's epi)
  unsigned long long wait_ns = 2000000000ull;  // limit of each grid-panel poll (global timer ns)
  int calu = 0;               // FP32 grid panels by tournament pivoting (0: column by column)
  long tab_stride = 0;        // problem group: entries between two problems' Q / C tables
  // grid panel (fronts too tall for a cluster): per front 2 x kGridPanelMaxG
  // publication slots of grid_panel_pub_words() 8-byte words
  unsigned long long* gpub = nullptr;
};
constexpr int kGridPanelMaxG = 152;
// status bits: 1 = pivot below the threshold, 2 = a bounded device wait ran out
cudaError_t factor_level(int prec, int d, DevLevel& L, const DevLevel* child, const double* Qcat,
                         const double* Ccat, const double* q, double pivot_tol, int* status,
                         const FactorWork& W, cudaStream_t st);
// panel width used for fronts of size m (0 if the staged panel cannot fit)
int factor_panel_width(int prec, int m);
// entries of the triangular-inverse scratch of a level with nf fronts of k eliminated
size_t invert_scratch_elems(int nf, int k, int ib);
// whether fronts of size m use the cooperative grid panel; 8-byte words of its
// publication buffer for nf fronts
bool factor_grid_panel(int prec, int m);
// the level's FP16 copy of its fronts (when it has one; after the factorisation)
cudaError_t factor_copy16(DevLevel& L, cudaStream_t st);
size_t grid_panel_pub_words(int nf);
// outer block width of the blocked LU of a front (0: the 32-column right-looking
// LU with a Schur update after every panel)
int factor_outer_block(int prec, bool tc, int m, int k);

// C[M x N] -= A[M x K] B[K x N] with the kernel the factorisation uses for the
// form (FP64 or FP32 SIMT; FP32 with tc: tensor cores, K <= kTcMaxK)
cudaError_t schur_update_raw(int prec, bool tc, bool split, int M, int N, int K, const void* A,
                             int lda, long sA, const void* B, int ldb, long sB, void* C, int ldc,
                             long sC, int batch, float* packA, float* packB, int* status,
                             cudaStream_t st);

// ---------------------------------------------------------------- tensor cores (sp_tc.cu)
constexpr int kTcMaxK = 1024;      // depth of the factorisation's updates (its operand buffers)
constexpr int kTcSubBlock = 256;   // sub-blocks of an outer block (depth of the updates inside it)
constexpr int kTcMaxKProbe = 16384;  // depth accepted by the stand-alone update and the rate probe
// floats of one packed operand buffer for `rows` rows, K columns, batch fronts
size_t tc_pack_floats(int rows, int K, int batch, bool split);
// C[M x N] -= A[M x K] B[K x N] (column-major, batch strides sA, sB, sC) with
// TF32 tensor-core products and FP32 accumulation (split: 3xTF32); K <= kTcMaxK.
// epi: 0 or 2 = C read a tile ahead through a shared-memory ring (three operand
// stages), 1 = C in registers (four operand stages); both give the same bits.
cudaError_t tc_schur_update(int M, int N, int K, const float* A, int lda, long sA, const float* B,
                            int ldb, long sB, float* C, int ldc, long sC, int batch, float* packA,
                            float* packB, bool split, int* status, cudaStream_t st, int epi = 0);
// rate probe of the same update kernel: C[M x N] -= A[M x K] B[K x N] on
// generated operands packed once, `reps` launches of the product kernel alone
// timed with CUDA events on st; *ms = device milliseconds per launch, *hstatus =
// the status word (bit 2: a pipeline wait ran out).  Allocates and frees its buffers.
cudaError_t tc_probe(bool split, int M, int N, int K, int reps, cudaStream_t st, float* ms,
                     int* hstatus);

// ---------------------------------------------------------------- solve (sp_solve.cu)
struct QTypeDev {
  int nS = 0, nG = 0, nB = 0;
  int* S = nullptr;  // nS x d offsets
  int* G = nullptr;  // nG x d offsets
  int* Bt = nullptr; // nB x d offsets of beta = gamma minus S
  long tab_off = 0;  // offset of the type in the concatenated column-major Q/C tables
  long t_off = 0;    // offset of the type in the concatenated column-major T tables
  // columns of the stencil apply: beta with Q(S, S) = I (set stencils), or all of
  // gamma with no identity term (per-point stencils, where Q(S, S) is not I)
  int na = 0, self = 1;
  int* A = nullptr;  // na x d offsets (Bt or G)
};
// y = Q r per set instance: r_S - T r_beta(S) for set stencils, -T r_gamma(S)
// with T = -Q(S, gamma(S)) for per-point stencils (VT = double2 (FP64) or float2
// (FP32) for y; r is complex128).
// nv stacked vectors (1 <= nv <= sweep_max_vectors()): global vectors (r, y, x,
// the stencil output) N apart, a level's work vectors (tmp nf m, y nf k, upd
// nf (m - k)) vector-major; each vector's result equals its single-vector result.
cudaError_t q_apply(int prec, int d, int n, int nl, const std::vector<QTypeDev>& types,
                    const double* Tcat, const float* Tcat32, const double2* r, void* y,
                    cudaStream_t st, int nv = 1, bool pdl = false, int P = 1,
                    long t_stride = 0);
// part: sweep_partial_bytes(nv) of work for the split row products (shared by levels)
cudaError_t forward_level(int prec, int d, DevLevel& L, const DevLevel* child, const void* rhsQ,
                          void* part, cudaStream_t st, int nv = 1, long N = 0);
cudaError_t backward_level(int prec, int d, DevLevel& L, double2* x, void* part, cudaStream_t st,
                           int nv = 1, long N = 0);
size_t sweep_partial_bytes(int nv = 1);
int sweep_max_vectors();
// launch shape of the fused one-launch-per-level sweep of an inverse-form level
// (false: its work vectors do not fit in shared memory)
bool sweep_fused_config(int prec, int nf, int m, int k, int num_sms, int max_cluster,
                        bool clusters, int* C, int* NT);
// CTAs per cluster the fused sweeps may use on the current device (16 or 8)
int sweep_max_cluster();

// ---------------------------------------------------------------- Krylov (sp_krylov.cu)
struct KrylovWork {
  int nblk = 0;            // CTAs of the reduction kernels
  double2* partial = nullptr;  // nblk x (maxv + 1)
  double2* h = nullptr;        // maxv + 1 (current Hessenberg column, device)
  double* nrm = nullptr;       // scalars
};
// h[0..nv) = V[0..nv)^H w  (V rows of length N, stride ldv)
cudaError_t kr_dots(const double2* V, long ldv, int nv, const double2* w, long N,
                    KrylovWork& K, double2* h_out, cudaStream_t st);
// w -= V h; if h2_out != null also h2 = V^H w (after the update)
cudaError_t kr_update_dots(const double2* V, long ldv, int nv, double2* w, long N,
                           const double2* h, KrylovWork& K, double2* h2_out, cudaStream_t st);
// nrm_out[0] = ||w||_2
cudaError_t kr_norm(const double2* w, long N, KrylovWork& K, double* nrm_out, cudaStream_t st);
// y = x * (1 / nrm[0])
cudaError_t kr_scale(const double2* x, long N, const double* nrm, double2* y, cudaStream_t st);
// y = a - b
cudaError_t kr_sub(const double2* a, const double2* b, long N, double2* y, cudaStream_t st);
// Hessenberg column j: H[0..j] = h1 + h2, H[j+1] = nrm; apply Givens; write estimate.
cudaError_t kr_givens(double2* H, int ldh, int j, const double2* h1, const double2* h2,
                      const double* nrm, double* cs, double2* sn, double2* gam, double* est,
                      cudaStream_t st);
// y = R^{-1} gam (upper triangular k x k in H), then u += Z y
cudaError_t kr_update_solution(const double2* H, int ldh, int k, const double2* gam,
                               double2* y, const double2* Z, long ldz, long N, double2* u,
                               cudaStream_t st);
// y = R^{-1} gam; u += Z y
cudaError_t kr_trisolve(const double2* H, int ldh, int k, const double2* gam, double2* y,
                        cudaStream_t st);
cudaError_t kr_combine(const double2* Z, long ldz, int k, const double2* y, long N, double2* u,
                       cudaStream_t st);
// gam = [beta, 0, ...]; V0 = r / beta
cudaError_t kr_start(const double2* r, long N, const double* nrm, double2* V0, double2* gam,
                     int len, cudaStream_t st);
// Batched Krylov processes ("instances": right-hand sides, problems of a group),
// advanced together with each instance's Arnoldi state in device memory, so that a
// restart cycle of all of them is one CUDA graph: the Arnoldi step repeats under a
// conditional while node until no instance goes on.
struct LoopHead {
  int j;           // column of the instance's current Arnoldi step
  int k;           // columns of the cycle once it stopped
  int total;       // iterations so far, all cycles
  int cont;        // 1 while the instance's cycle goes on
  double est_rel;  // last estimate |gamma_{j+1}| / ||g||
  double bnorm;    // ||g||           (written at the end of the cycle)
  double rnorm;    // ||g - A u||     (written at the end of the cycle)
  double pad;
};
// Instance i's slices: V + i sV (maxv vectors of N), Z + i sZ, H + i sH (leading
// dimension ldh), gam / sn / cs + i sG, h1 / h2 / y + i sh, nrm / est + 4 i,
// partial + i sP (nblk partial sums per column), w + i N (the new vector of a step).
struct KBatch {
  double2 *V = nullptr, *Z = nullptr, *H = nullptr, *gam = nullptr, *sn = nullptr;
  double2 *h1 = nullptr, *h2 = nullptr, *y = nullptr, *partial = nullptr, *w = nullptr;
  double *cs = nullptr, *nrm = nullptr, *est = nullptr;
  LoopHead* head = nullptr;  // I heads
  const int* run = nullptr;  // I flags: the instance runs in this cycle
  long N = 0, sV = 0, sZ = 0, sH = 0, sG = 0, sh = 0, sP = 0;
  int ldh = 0, nblk = 0;
};
// head.j = 0, head.cont = run
cudaError_t kb_begin(const KBatch& b, int I, cudaStream_t st);
// running instances: V_i[0] = r_i / nrm_i[3], gam_i = [nrm_i[3], 0, ...] (len entries)
cudaError_t kb_start(const KBatch& b, int I, const double2* r, int len, cudaStream_t st);
// instances in a step: dst_i = V_i[j_i] / Z_i[j_i] = src_i (vectors N apart)
cudaError_t kb_copy_in(const KBatch& b, int I, double2* dst, cudaStream_t st);
cudaError_t kb_copy_out(const KBatch& b, int I, const double2* src, cudaStream_t st);
// instances in a step: classical Gram-Schmidt twice of w_i against V_i[0..j_i],
// nrm_i[0] = ||w_i||, Hessenberg column j_i and its Givens rotation (est_i)
cudaError_t kb_arnoldi(const KBatch& b, int I, int nv_max, cudaStream_t st);
// nrm_i[slot] = ||x_i|| for every instance (x_i = x + i N)
cudaError_t kb_norm(const KBatch& b, int I, const double2* x, int slot, cudaStream_t st);
// the stopping test of every instance in a step (estimate, budget, breakdown, full
// basis), hist_i[total - 1] = estimate; V_i[j_i + 1] = w_i / nrm_i[0] for those that
// go on; cond = 0 when none does.  I <= 1024.
cudaError_t kb_step(const KBatch& b, int I, double* hist, int hstride, double tol, int maxit,
                    int restart, cudaGraphConditionalHandle cond, cudaStream_t st);
// running instances: y_i = R_i^{-1} gam_i (k_i columns), U_i += Z_i y_i
cudaError_t kb_update_solution(const KBatch& b, int I, double2* U, cudaStream_t st);
// head.bnorm = nrm[2], head.rnorm = nrm[3]
cudaError_t kb_finish(const KBatch& b, int I, cudaStream_t st);
// nrm_i[to] = nrm_i[from]
cudaError_t kb_copy_nrm(const KBatch& b, int I, int from, int to, cudaStream_t st);
// complex64 counterparts for the inner solve of the mixed-precision form
cudaError_t kr32_dots(const float2* V, long ldv, int nv, const float2* w, long N, KrylovWork& K,
                      double2* h_out, cudaStream_t st);
cudaError_t kr32_update_dots(const float2* V, long ldv, int nv, float2* w, long N, const double2* h,
                             KrylovWork& K, double2* h2_out, cudaStream_t st);
cudaError_t kr32_norm(const float2* w, long N, KrylovWork& K, double* nrm_out, cudaStream_t st);
cudaError_t kr32_scale(float2* x, long N, const double* nrm, cudaStream_t st);
// y = x / nrm[0] in complex64, gam = [1, 0, ...]
cudaError_t kr32_start(const double2* x, long N, const double* nrm, float2* y, double2* gam,
                       int len, cudaStream_t st);
cudaError_t kr_widen(const float2* x, long N, double2* y, cudaStream_t st);
cudaError_t kr_narrow(const double2* x, long N, float2* y, cudaStream_t st);
cudaError_t kr_scale_y(double2* y, int k, const double* s, cudaStream_t st);

}  // namespace sp
