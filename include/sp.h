/*
 * sp.h -- C ABI of the GB300 sparsifying-preconditioner solver.
 *
 * The library solves the pseudospectral system of the periodic problem
 *     (-Laplace - s + q(x)) u = f   on the unit torus [0,1)^d, d = 2 or 3,
 * (Eq. Dsq / Eq. Lsq of Ying, "Sparsifying preconditioner for pseudospectral
 * approximations of indefinite systems on periodic structures", Section 2.1)
 * through its integral form (I + G q) u = G f with G = (L - s)^{-1} (Eq. G,
 * Section 2.2), preconditioned by u <= P^{-1} Q g where Q is the sparsifying
 * stencil, C = Q G truncated to the stencil and P = Q + C q (Section 2.2-2.3).
 * P is factored by periodic nested dissection with a multifrontal LU
 * (Section 2.3, Fig. nd); the outer iteration is GMRES.
 *
 * Conventions for every call below.
 *  - Grid: n points per axis, N = n^d unknowns, flat index j0 + n*j1 (+ n^2*j2)
 *    (axis 0 fastest).  The leaf box size b must divide n with n/b = 2^L, L >= 1,
 *    and b >= 2, and N < 2^31 (grid indices are 32-bit): every call that takes
 *    (d, n, b) returns SP_ERR_ARG otherwise.
 *  - Vectors (r, z, f, u, g, x, w, y) are complex128: N pairs (re, im) of
 *    double, interleaved, 16-byte aligned.  q is N real doubles.  Pointers named
 *    *_dev are CUDA device pointers on the context's device; *_host are host
 *    pointers (pinned memory gives the fastest copies).  The caller owns every
 *    buffer it passes; the context owns its tables, factor and workspace.
 *  - Every call is ordered on the stream given to sp_setup.  Calls that return a
 *    scalar to the host (sp_solve, sp_factor's status check) synchronise that
 *    stream.  A context is not thread-safe; different contexts may be driven
 *    from different host threads at the same time (sp_setup synchronises only
 *    its own streams, so it does not disturb another context's graph capture).
 *  - No call aborts or throws across the ABI: errors come back as sp_status.
 *    After SP_ERR_CUDA the context should be destroyed.
 */
#ifndef SP_GB300_H
#define SP_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sp_ctx sp_ctx; /* opaque */

typedef enum {
  SP_OK = 0,
  SP_ERR_ARG = 1,       /* invalid argument (sizes, null pointers, n/b not 2^L) */
  SP_ERR_RESONANT = 2,  /* L - s is (numerically) singular: s hits 4 pi^2 |k|^2 */
  SP_ERR_SINGULAR = 3,  /* a pivot of a front fell below pivot_tol * max|front| */
  SP_ERR_NOCONV = 4,    /* GMRES stopped at maxit above tol (the iterate is still returned) */
  SP_ERR_OOM = 5,       /* device or host allocation failed, or the host could not start
                           the set-up's worker threads */
  SP_ERR_TIMEOUT = 6,   /* a bounded device wait (tensor-core pipeline, grid panel) ran out */
  SP_ERR_CUDA = 7,      /* a CUDA runtime call failed */
  SP_ERR_STATE = 8      /* call out of order (e.g. sp_apply before sp_factor) */
} sp_status;

typedef enum {
  SP_PREC_FP64 = 0,  /* factor, sweeps, FFTs and Krylov all in FP64 */
  SP_PREC_FP32 = 1,  /* factor and sweeps of P in FP32 (preconditioner only);
                        FFT operator, Gram-Schmidt and residuals stay FP64 */
  SP_PREC_MIXED = 2, /* GMRES-IR: FP32 factor and sweeps, an inner flexible GMRES
                        in complex64 (FFT operator and Gram-Schmidt in FP32,
                        Hessenberg and rotations in FP64) solves A d = r to
                        inner_tol; the outer FP64 refinement forms u += d and the
                        true residual r = g - A u with the FP64 operator */
  SP_PREC_TF32 = 3,  /* as SP_PREC_FP32, and fronts with m >= 1024 are factored in
                        outer blocks of 1024 columns (sub-blocks of 256) whose
                        Schur updates S -= L21 U12 run on the tensor cores (TF32
                        products, FP32 accumulation; Section 2.3's update
                        S = F22 - L21 U12) */
  SP_PREC_TF32X3 = 4 /* as SP_PREC_TF32 with each operand split into a TF32 high
                        part and a TF32 low part and the three products
                        hi*hi + hi*lo + lo*hi summed on the tensor cores
                        (3xTF32: FP32-level accuracy of the update) */
} sp_precision;

typedef struct {
  int maxit;         /* total GMRES iterations allowed (default 500; >= 1) */
  int restart;       /* Krylov vectors kept before a restart (default 200; 1 ... 1000) */
  double tol;        /* target relative residual ||g - A u|| / ||g|| (default 1e-8; > 0) */
  double pivot_tol;  /* singular-front threshold, relative to max|front| (default 1e-14) */
  int device;        /* CUDA device ordinal the context lives on (default 0) */
  int host_threads;  /* threads for the host set-up (0 = all hardware threads): the
                        host FFT's lines, the TSQR route's row blocks, the Gram
                        route's stencil types side by side.  The Gram route's tables
                        and the symbolic structure do not depend on the count; the
                        TSQR route combines one triangle per thread, so its tables
                        change with the count in the last bits (~1e-13 relative) */
  double inner_tol;  /* SP_PREC_MIXED: relative tolerance of each inner solve (default 1e-5) */
  int autotune;      /* 1: sp_setup times the factorisation's launch-shape candidates
                        of every level (Schur-update and block-inverse GEMM tiles,
                        32 or 64) on a placeholder medium (q = 0) and keeps the
                        fastest; every result is bit-identical to the untuned
                        context's.  0 (default): built-in heuristics */
  int max_rhs;       /* right-hand sides sp_solve_many may take at once, 1 ... 8
                        (default 1); the solve workspace is sized for it */
  int setup_route;   /* how sp_setup forms T_S = G(S, gamma^c) G(beta, gamma^c)^+:
                        0 (default) TSQR of [B^T | A^T] over the N - |gamma| points of
                        gamma^c and an SVD of R11 (accuracy ~cond(B) eps); 1 the Gram
                        route B B^T = (G^2)(beta, beta) - G(beta, gamma) G(gamma, beta),
                        A B^T likewise, and an eigen-decomposition of B B^T: cost
                        independent of N, accuracy ~cond(B)^2 eps */
  int stencil;       /* 0 (default): the set stencils of Section 2.3, Q(S, gamma(S)) for
                        cells, faces, edges and vertices; 1: per-point stencils
                        Q(j, gamma({j})) on the 3^d neighbourhood of every point j
                        (one T for all points by translation invariance), the
                        sparsifying operator of the earlier per-point construction */
  int inv_block;     /* diagonal-block size of the levels that keep block inverses of
                        L11 / U11 (their sweeps are chains of k / inv_block matrix-vector
                        steps): 0 (default) = 2048 on levels with k >= 32768 and 512
                        elsewhere, else a power of two in 64 ... 2048 for every level;
                        larger blocks mean fewer, longer launches per sweep and more
                        work in the block inverses */
  int tc_epilogue;   /* tensor-core forms: how the Schur update reads C.  0 (default)
                        or 3: a tile ahead, three of its four 32-column chunks in
                        registers and one in a shared-memory slot that cp.async fills
                        (four operand stages); 2: two chunks in registers and two slots
                        (three operand stages); 1: the next chunk only, in registers
                        (four operand stages); 4: as 0 in thread-block clusters of two
                        CTAs that share each B tile by TMA multicast (slower: 557 against
                        637 TFLOP/s at 3D 128^3).  All give the same bits. */
  long long wait_limit_ns; /* limit of each bounded wait of the cooperative grid panel
                        (the LU panel of fronts too tall for a thread-block cluster:
                        every CTA polls the pivot candidates its peers publish) in
                        nanoseconds of the GPU's global timer; 0 (default) = 2e9 (2 s),
                        else 1 ... 6e10.  When a wait runs out the panel stops and
                        sp_factor returns SP_ERR_TIMEOUT; destroy that context. */
  int sweeps;        /* forward / backward sweeps of the levels that keep block inverses
                        (Section 2.3's solve with the factor): a level is either swept by a
                        chain of launches per diagonal block (gather, block product, split
                        row products) or by one fused launch per direction (the front's
                        work vectors in shared memory; on levels with few fronts a
                        thread-block cluster of up to 16 CTAs per front walks the diagonal
                        blocks itself).  0 (default): fused only on levels whose fronts
                        fill the GPU without clusters, chains elsewhere; 1: chains
                        everywhere; 2: fused wherever the vectors fit.  All are exact
                        applications of the same factor; they round differently. */
  int panel_pivoting; /* pivoting of the cooperative grid panel in the FP32 forms (fronts too
                        tall for a thread-block cluster, the 3D upper levels): 0 (default)
                        partial pivoting column by column (two publication rounds per
                        column); 1 tournament pivoting (communication-avoiding LU: each CTA
                        picks 32 candidate rows by partial pivoting on its rows, groups of
                        16 CTAs and then all CTAs play the winners off, and every row is
                        eliminated against the 32 chosen ones at once: three publication
                        rounds per panel, but three 32-step eliminations in sequence; 3D
                        128^3 TF32 panels 1.22 s against 1.03 s).  FP64 grid panels always
                        pivot column by column. */
  int launch_overlap; /* 1: the stencil and sweep kernels of the preconditioner application
                        are launched with programmatic dependent launch (a kernel may start
                        while the previous one's last CTAs drain; it waits for that kernel's
                        results before reading them); 0 (default): ordinary stream order.
                        The same kernels and results either way. */
  int device_loop;   /* 1 (default): sp_solve runs each GMRES restart cycle as one CUDA graph whose
                        Arnoldi steps repeat under a conditional (while) graph node: the
                        stopping test runs on the device and the host waits once per
                        cycle instead of once per iteration (Section 2.2's GMRES loop;
                        the same kernels, order and results as 0).  The graph is
                        captured on the first such solve and reads the context's copy
                        of the medium, so later factorisations reuse it; a failed
                        capture returns SP_ERR_CUDA.
                        sp_solve, sp_solve_host, sp_solve_x0 and sp_solve_many (all its
                        right-hand sides in one graph) follow it; SP_PREC_MIXED ignores
                        it, and so does a single-problem context while sp_profile is on
                        (host-driven, so every kernel class is timed).  A problem group
                        (sp_setup_group, P > 1) always runs its cycles as graphs.  0: the
                        host drives every iteration (reads the estimate after each
                        step).  Default 1. */
  int factor_storage; /* FP32-family forms (FP32, mixed, TF32, 3xTF32): 1 keeps, after each
                        factorisation, an FP16 copy of the fronts of the levels whose sweeps
                        run as chains of block products (the large upper levels), each front
                        column scaled by a power of two so its largest entry stays below
                        2^15; those sweeps then read half the bytes and sum in FP32 (Section
                        2.3's solve with the factor, at FP16 accuracy of the factor entries:
                        measured at 3D 128^3 TF32 Helmholtz, 83 -> 85 GMRES iterations and
                        5.00 -> 4.75 s per factor and solve).  0 (default):
                        the sweeps read the factor in the form's precision.  SP_ERR_ARG for
                        SP_PREC_FP64. */
} sp_opts;

typedef struct {
  int iters;           /* GMRES iterations (matvecs with the preconditioned operator) */
  int restarts;        /* restart cycles beyond the first */
  double est_relres;   /* last Givens estimate |gamma_{k+1}| / ||g|| */
  double true_relres;  /* ||g - (I + G q) u|| / ||g|| computed explicitly in FP64 */
  double s_used;       /* the shift s of the context */
  double *hist;        /* optional caller buffer for the estimate per iteration */
  int hist_cap;        /* its capacity (entries) */
  int hist_len;        /* entries written (iters + 1, capped) */
  double guess_relres; /* sp_solve_x0: ||g - (I + G q) u0|| / ||g|| of the given start (1 otherwise) */
  int guess_used;      /* sp_solve_x0: 1 if the start was kept, 0 if it fell back to zero */
} sp_info;

/* Fill *o with the defaults listed above. */
void sp_default_opts(sp_opts *o);

/* sizeof(sp_opts) for which = 0, sizeof(sp_info) for which = 1, else 0: lets a
 * binding in another language check its layout of the two structs against this
 * build (the paper has no counterpart; ABI plumbing only). */
size_t sp_abi_size(int which);

/* Build a context for grid (d, n), leaf size b and shift s (Section 2.2-2.3):
 * the Fourier symbol 1/(4 pi^2 |k|^2 - s) of G (Eq. G), the stencil tables
 * T_S = G(S, gamma^c) G(beta, gamma^c)^+, Q(S, gamma) = [I, -T_S] and
 * C(S, gamma) = Q(S, gamma) G(gamma, gamma) for every cell/face/edge/vertex type
 * (Section 2.3), the nested-dissection symbolic structure (Fig. nd) and all
 * device memory.  The pseudoinverse drops singular values at or below
 * max(size) * eps(sigma_max).  opts may be NULL (defaults); stream is a
 * cudaStream_t or NULL for the legacy default stream.  Grids: d = 2 or 3, n = 2^p
 * or 3 2^p (the paper's 48 ... 384 included), n / b a power of two >= 2;
 * otherwise SP_ERR_ARG.  Returns SP_ERR_RESONANT when
 * min_k |s/(4 pi^2) - |k|^2| < 1e-6 max(1, s/(4 pi^2)). */
sp_status sp_setup(int d, int n, int b, double s, sp_precision prec, const sp_opts *opts,
                   void *stream, sp_ctx **out);

/* A problem group: one context for P independent problems of the same grid (d, n)
 * and leaf size b, problem p with shift shifts[p] (its own Green's function, stencil
 * tables and, at sp_factor, medium).  The nested-dissection structure depends on
 * the grid and leaf size only (Section 2.3), so every level of all P problems has
 * fronts of one size: each factorisation and sweep launch covers the P nf fronts of
 * a level at once, the operator and stencil launches cover the P vectors, and the P
 * GMRES iterations advance together (batched Krylov kernels, restart cycles as CUDA
 * graphs; see sp_opts.device_loop).  Every vector of the context then holds P N
 * entries, problem p's at offset p N: q of sp_factor, r / z of sp_apply, f / u of
 * sp_solve, x / w of sp_matvec, f / g of sp_green, r / y of sp_qapply; sp_solve and
 * sp_solve_host fill P info records in problem order, sp_solve_many nrhs P
 * (right-hand side r of problem p at index and vector offset r P + p);
 * sp_get_table / sp_set_table take t = p 2^d + type.  1 <= P, P opts.max_rhs <=
 * 1024 and P n^d < 2^31 (grid indices are 32-bit); SP_PREC_MIXED and sp_solve_x0
 * with a start vector take P = 1 only (else SP_ERR_ARG).  The other arguments and
 * errors are sp_setup's, checked for every shift.  A group's problems give the
 * results of separate contexts up to rounding: launch shapes that depend on the
 * number of fronts (row splits of the sweeps' matrix-vector products, fused or
 * chained sweeps, block inverses on FP64 levels) may sum in another order. */
sp_status sp_setup_group(int d, int n, int b, int P, const double *shifts, sp_precision prec,
                         const sp_opts *opts, void *stream, sp_ctx **out);

/* *P = the context's number of problems (1 unless made by sp_setup_group).  Host
 * only, no GPU work; SP_ERR_ARG if ctx or P is NULL. */
sp_status sp_problems(const sp_ctx *ctx, int *P);

/* Assemble P = Q + C diag(q) into the fronts and factor it (Section 2.2, Fig. nd):
 * per level, leaves to root, extend-add of the children's Schur complements,
 * partial-pivot LU of the eliminated block, panels and Schur update.  q_dev: N
 * real doubles on the device, copied into the context (the operator I + G q of
 * sp_solve / sp_matvec uses the copy).  The work is replayed from a CUDA graph
 * captured at set-up (direct launches while sp_profile is on).  Returns
 * SP_ERR_SINGULAR if a pivot is below pivot_tol * max|front| (the factor is then
 * unusable). */
sp_status sp_factor(sp_ctx *ctx, const double *q_dev);

/* z = P^{-1} Q r, the preconditioner of Section 2.2 ("u <= P^{-1} Q g"):
 * stencil apply, forward sweep leaves to root, backward sweep root to leaves.
 * r_dev, z_dev: N complex128 on the device, must not alias. */
sp_status sp_apply(sp_ctx *ctx, const void *r_dev, void *z_dev);

/* Solve (I + G q) u_r = G f_r for nrhs right-hand sides with the current factor
 * (Section 2.2): nrhs independent GMRES iterations (each as sp_solve: its own
 * Krylov basis, restarts and stopping test) advanced in lockstep, sharing every
 * preconditioner application and operator product, so the factor is read once
 * per step for all right-hand sides.  Each u_r is bit-identical to sp_solve's
 * for f_r.  F_dev, U_dev: nrhs x N complex128 on the device, right-hand side r at
 * offset r N; infos: nrhs sp_info or NULL.  1 <= nrhs <= opts.max_rhs, else
 * SP_ERR_ARG; SP_ERR_NOCONV if any right-hand side stopped above tol.  The
 * mixed-precision form solves the right-hand sides one after the other. */
sp_status sp_solve_many(sp_ctx *ctx, int nrhs, const void *F_dev, void *U_dev, sp_info *infos);

/* Solve (I + G q) u = G f by GMRES right-preconditioned with P^{-1} Q
 * (Section 2.2; GMRES of Saad and Schultz), zero initial guess, classical
 * Gram-Schmidt twice, stopping when the estimate is <= tol, then an explicit
 * FP64 true residual; restarts from u if that is still above tol (with
 * SP_PREC_MIXED: refinement steps of FP32 inner solves, see sp_precision; iters
 * counts inner iterations, restarts the refinement steps beyond the first).  f_dev, u_dev:
 * N complex128 on the device.  info may be NULL.  Returns SP_ERR_NOCONV when
 * maxit is reached above tol. */
sp_status sp_solve(sp_ctx *ctx, const void *f_dev, void *u_dev, sp_info *info);

/* sp_solve from the starting vector u0_dev (N complex128 on the device; may equal
 * u_dev; NULL means zero).  The start is kept only if its residual
 * ||g - (I + G q) u0|| is below ||g||, the residual of the zero vector; otherwise
 * the solve starts from zero (info->guess_used = 0).  GMRES then runs on the
 * residual equation, the iterations counted from the start, the same stopping test
 * (relative to ||g||) and the same explicit true residual decide convergence.  A
 * start already within tol returns after 0 iterations. */
sp_status sp_solve_x0(sp_ctx *ctx, const void *f_dev, const void *u0_dev, void *u_dev,
                      sp_info *info);

/* Host-buffer forms of sp_factor and sp_solve: the same work with the input
 * copied host->device and the result device->host inside the call. */
sp_status sp_factor_host(sp_ctx *ctx, const double *q_host);
sp_status sp_solve_host(sp_ctx *ctx, const void *f_host, void *u_host, sp_info *info);

/* w = x + G (q x), the integral operator of Section 2.2 (needs sp_factor's q). */
sp_status sp_matvec(sp_ctx *ctx, const void *x_dev, void *w_dev);

/* g = G f = F^{-1} diag(1/(4 pi^2 |k|^2 - s)) F f (Eq. G). */
sp_status sp_green(sp_ctx *ctx, const void *f_dev, void *g_dev);

/* y = Q r, the sparsifying stencil alone (Section 2.3, Q(S, gamma) = [I, -T_S]). */
sp_status sp_qapply(sp_ctx *ctx, const void *r_dev, void *y_dev);

/* Copy set type t's tables to the host (t = sum of 2^a over axes a with
 * p_a = 0 mod b: 0 = cell, 2^d - 1 = vertex).  Q_out, C_out: |S| x |gamma|
 * row-major (rows in S order, columns in gamma order, points ordered with axis 0
 * fastest); either may be NULL.  *rows = |S|, *cols = |gamma|, *rank = rank kept
 * by the pseudoinverse. */
sp_status sp_get_table(const sp_ctx *ctx, int t, double *Q_out, double *C_out, int *rows,
                       int *cols, int *rank);

/* Replace set type t's tables Q(S, gamma) and C(S, gamma) (Section 2.3) with the
 * caller's, in sp_get_table's layout (|S| x |gamma| row-major, host memory): for
 * example tables kept from an earlier set-up of the same (d, n, b, s, stencil), or
 * computed by another route.  They take effect at the next sp_factor (the context
 * is marked unfactored); the stencil apply uses T = -Q on the beta columns.  With
 * set stencils Q(S, S) must be the identity (the form Q(S, gamma) = [I, -T_S]),
 * else SP_ERR_ARG; non-finite entries give SP_ERR_ARG.  The rank that
 * sp_get_table reports stays the set-up's.  Synchronises the context's stream. */
sp_status sp_set_table(sp_ctx *ctx, int t, const double *Q_host, const double *C_host);

/* Host-only (no GPU): the same tables as sp_setup computes for (d, n, b, s),
 * type t, by route 0 (TSQR + SVD) or 1 (Gram, see sp_opts.setup_route), of
 * kind 0 (set stencils) or 1 (per-point stencils, see sp_opts.stencil).  Pass
 * Q_out = C_out = NULL to query *rows / *cols first.  sigma_out (may be NULL)
 * receives min(|beta|, 64) leading singular values of G(beta, gamma^c) in
 * descending order (route 1: square roots of the eigenvalues of B B^T).
 * SP_ERR_ARG for a bad grid, type, route or kind or a non-finite s,
 * SP_ERR_RESONANT when L - s is numerically singular. */
sp_status sp_stencil_table(int d, int n, int b, double s, int t, int route, int kind,
                           int host_threads, double *Q_out, double *C_out, int *rows, int *cols,
                           int *rank, double *sigma_out);

/* Host-only: the nested-dissection structure (Fig. nd).  Writes, for levels
 * 0 (leaves) .. L (root), the number of fronts, eliminated unknowns k and front
 * size m into the caller's arrays of capacity cap; *nlevels = L + 1. */
sp_status sp_front_sizes(int d, int n, int b, int cap, int *nlevels, int *nfronts, int *k,
                         int *m);

/* Host-only: the symbolic data of one nested-dissection level (Fig. nd), for
 * inspection and tests.  Pass NULL arrays to query the sizes first.
 * gidx: nf x m grid indices of the front unknowns (eliminated ones first);
 * ea_map: 2^d x (mc - kc) positions in this level's fronts of the children's
 * boundary unknowns (child position delta = sum_a 2^a * (child box coordinate a
 * is odd)); asm_row / asm_cvar: front row r and front column c (the position of
 * the column point; entry r + c m of the column-major front) of the nasm
 * original entries of P assembled into every front of the level. */
sp_status sp_level_info(int d, int n, int b, int level, int *nf, int *k, int *m, int *mc,
                        int *kc, int *nasm, int *gidx, int *ea_map, int *asm_row,
                        int *asm_cvar);

/* Algorithmic sizes of the context: factor entries (sum over fronts of
 * k^2 + 2 k (m - k)), factor flops (sum of (2/3) k^3 + 2 k^2 (m-k) + 2 k (m-k)^2
 * real operations) and bytes of one preconditioner application. */
sp_status sp_costs(const sp_ctx *ctx, double *factor_entries, double *factor_flops,
                   double *apply_bytes);

/* Section 2.1 shift/potential split on host arrays of N values.
 * Helmholtz: s = mean(omega^2 / c^2), q = s - omega^2 / c^2.
 * Schroedinger (rescaled, Eq. schr): s = mean(l^2 E - l^2 V), q = l^2 V - l^2 E + s;
 * the caller multiplies f by l^2.  If L - s is numerically singular (see
 * sp_setup) s is raised by 1e-3 * 4 pi^2 until it is not; q follows s.
 * SP_ERR_ARG for a zero or non-finite c, a non-finite V, omega, l or E (nothing
 * is written then). */
sp_status sp_medium_helmholtz(int d, int n, double omega, const double *c_host, double *s_out,
                              double *q_host);
sp_status sp_medium_schrodinger(int d, int n, double ell, double E, const double *V_host,
                                double *s_out, double *q_host);
/* q = l^2 V - l^2 E + s for a caller-chosen shift s (a family of potentials sharing
 * one context: the exact solution does not depend on s, only the preconditioner
 * does).  The caller checks s with sp_setup (SP_ERR_RESONANT). */
sp_status sp_medium_schrodinger_at(int d, int n, double ell, double E, const double *V_host,
                                   double s, double *q_host);

/* Kernel-class timing for roofline measurements: with sp_profile(ctx, 1) every
 * later call records CUDA events around its kernel launches on the context's
 * stream.  sp_profile_read synchronises, writes per class c (0 assembly and
 * extend-add, 1 LU panels, 2 LU row-block solves, 3 LU Schur updates, 4 stencil
 * apply, 5 forward sweep, 6 backward sweep, 7 FFT passes, 8 Arnoldi/GMRES vector
 * kernels, 9 triangular inverses of the few-front levels) the summed device
 * milliseconds, the number of kernel launches and the algorithmic work (flops
 * for classes 1-3 and 9, bytes for the others: the data a kernel must move at
 * least once; 10 tensor-core Schur updates of the blocked fronts, flops), then
 * clears the record.  Arrays of cap >= 11.  A single-problem context's solves run
 * host-driven while profiling is on; a problem group's GMRES cycles stay CUDA
 * graphs, whose kernels are not split into classes. */
sp_status sp_profile(sp_ctx *ctx, int enable);
sp_status sp_profile_read(sp_ctx *ctx, int cap, double *ms, int *launches, double *work);

/* One Schur-complement update of the multifrontal LU (Section 2.3: the block
 * S = F22 - L21 U12 handed to the parent front), for checking the update kernels
 * in isolation: C[M x N] -= A[M x K] B[K x N] for `batch` column-major problems
 * on the current device (leading dimensions lda, ldb, ldc >= the row counts;
 * batch strides sA, sB, sC in elements), with the kernel the factorisation uses
 * for the form: SP_PREC_FP64 doubles, SP_PREC_FP32 floats (SIMT FMA units),
 * SP_PREC_TF32 floats with TF32 products on the tensor cores and FP32
 * accumulation, SP_PREC_TF32X3 the same with split operands (K <= 16384 for both;
 * the factorisation itself uses depths up to 1024; the call allocates and frees its
 * operand buffers).
 * A, B, C: device pointers owned by the caller; C must not overlap A or B.
 * Synchronous on `stream` (cudaStream_t or NULL).  SP_ERR_ARG for bad sizes or
 * forms, SP_ERR_TIMEOUT if a tensor-core pipeline wait ran out. */
sp_status sp_schur_update(sp_precision prec, int M, int N, int K, const void *A, int lda,
                          long long sA, const void *B, int ldb, long long sB, void *C, int ldc,
                          long long sC, int batch, void *stream);

/* Rate probe of the tensor-core update kernel (measurement helper; the paper has
 * no counterpart): C[M x N] -= A[M x K] B[K x N] in FP32 on operands the call
 * generates (uniform in [-1, 1)), packed once to TF32 (split = 1: 3xTF32), then
 * `reps` launches of the tcgen05 product kernel alone between two CUDA events on
 * `stream`; *ms_per_launch = device milliseconds per launch (the algorithmic work
 * is 2 M N K flop; the tensor pipe executes 3x that with split = 1).  M a multiple
 * of 128 in 128 ... 16384, N a multiple of 256 in 256 ... 16384, K a multiple of 32
 * up to 16384, reps 1 ... 1000, else SP_ERR_ARG.  Allocates (3 M K + 3 K N + M N
 * floats at most) and frees its buffers; synchronous on `stream`; SP_ERR_TIMEOUT
 * if a pipeline wait ran out. */
sp_status sp_tc_probe(int split, int M, int N, int K, int reps, void *stream, double *ms_per_launch);

/* Launch shapes of nested-dissection level `level` (0 = leaves): Schur-update
 * tile and block-inverse GEMM tile (32 or 64); 0 means the built-in heuristic
 * (sp_opts.autotune = 0).  SP_ERR_ARG for a level outside 0 ... L. */
sp_status sp_tuning(const sp_ctx *ctx, int level, int *gemm_tile, int *gen_tile);

/* g = G f for callers that cannot allocate device memory when they call (for
 * example code running inside a CUDA-graph stream capture, or under a fixed,
 * pre-carved memory budget).  No context and no allocation: the FFT passes use a
 * file-scope device work array of 2^18 complex128 values (4 MiB, held by every
 * device that loads the library until the process exits), so n^d <= 262144
 * (e.g. 512^2, 64^3); larger grids, n not a power of two, d not 2 or 3, null or
 * aliasing pointers return SP_ERR_ARG; a resonant s returns SP_ERR_RESONANT.
 * f_dev, g_dev: n^d complex128 on the current device; stream: cudaStream_t or
 * NULL.  All calls on a device share the work array: calls that may run
 * concurrently on the GPU race and must be ordered by the caller.  The first call
 * on a device looks up the array's address (cudaGetSymbolAddress) with that
 * device current; make it before any stream capture.  That cached address is
 * valid for the device's context: after cudaDeviceReset the process must reload
 * the library before calling again.  A CUDA error already pending from the
 * caller's earlier work returns SP_ERR_CUDA before any launch and is left pending.
 * The paper has no counterpart of this entry point; it is an allocation-free form
 * of sp_green. */
sp_status sp_green_static(int d, int n, double s, const void *f_dev, void *g_dev, void *stream);

void sp_destroy(sp_ctx *ctx);
const char *sp_status_str(sp_status st);

#ifdef __cplusplus
}
#endif
#endif /* SP_GB300_H */
