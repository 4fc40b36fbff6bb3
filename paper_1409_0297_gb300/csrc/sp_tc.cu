// Schur-complement update of the large fronts on the tensor cores, for the
// tensor-core form of the preconditioner (Section 2.3: S = F22 - L21 U12 of each
// front, here with the K = 1024 or 256 columns of one outer block or sub-block of the
// blocked LU):
//
//   C[M x N] -= A[M x K] B[K x N]      (column-major, batched over fronts)
//
// A = L21 and B = U12 are first copied into K-major operand buffers rounded to
// TF32 (round to nearest), padded to a multiple of 32 in K with zeros: packA
// [batch][M][Kp], packB [batch][N][Kp].  The split form (3xTF32) recovers FP32
// accuracy: with a = a_hi + a_lo (a_hi = tf32(a), a_lo = tf32(a - a_hi)) the
// operands are extended along K to [a_lo | a_hi | a_hi] and [b_hi | b_lo | b_hi],
// so one product of depth 3 Kp sums a_lo b_hi + a_hi b_lo + a_hi b_hi (the
// dropped a_lo b_lo and the rounding of the low parts are ~2^-22 |a||b|).  Those are read by TMA (3-D tensor maps,
// 128-byte swizzle) into a ring of shared-memory stages; one thread issues
// tcgen05.mma kind::tf32 (M = 128, N = BN, K = 8 per instruction) with the FP32
// accumulators in tensor memory (two, so one tile's epilogue overlaps the next
// tile's products); eight epilogue warps read an accumulator with tcgen05.ld and
// subtract it from C in global memory (the front keeps its column-major layout
// with leading dimension m, which needs no alignment, so C cannot go through TMA;
// its loads are issued a tile ahead, half into registers and half by cp.async into
// a shared-memory ring).  Persistent: one CTA per SM walks the tiles of all fronts.
//
// Every wait on an mbarrier is bounded (about 2 s of global timer); a wait that
// runs out sets bit 2 of *status, the CTA drains the copies it issued, frees its
// tensor memory and returns without touching C.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr int kBM = 128;       // tile rows = tensor-memory lanes
constexpr int kBK = 32;        // K per stage: 32 FP32 = one 128-byte swizzle row
constexpr int kUK = 8;         // K of one kind::tf32 instruction
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > kWaitNs) return false;
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
// the same copy delivered to the CTAs of ctamask (same shared-memory offset and
// mbarrier offset in each)
__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                               int c2, uint32_t bar, uint16_t ctamask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar), "h"(ctamask)
      : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (start address and offsets in 16-byte units; bit 46 is
// the descriptor version of this architecture; layout 2 = 128-byte swizzle)
__device__ __forceinline__ unsigned long long sw128_desc(uint32_t saddr) {
  return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)(1024u >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, unsigned long long ad,
                                         unsigned long long bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
// arrive (once the MMAs issued so far complete) on the mbarrier at this offset in every
// CTA of ctamask
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t ctamask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(ctamask)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, volatile int* ab) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try(bar, parity)) {
    if (*ab) return false;
    if (gtimer() - t0 > kWaitNs) {
      *ab = 1;
      return false;
    }
  }
  return true;
}

constexpr int kEpiWarps = 8;                  // warps 0-7: epilogue (2 per TMEM lane quarter)
constexpr int kPThreads = 32 * (kEpiWarps + 2);  // + warp 8 (TMA producer), warp 9 (MMA issuer)
constexpr int kGroupM = 32;                   // row tiles per group of the tile order

// tile t -> front f and tile origin (m0, n0): fronts outermost, then groups of
// kGroupM row tiles whose column tiles are visited in turn (the group's A rows and
// the current B columns stay in L2)
__device__ __forceinline__ void tile_coords(long t, int tilesM, int tilesN, int BN, int* f,
                                            int* m0, int* n0) {
  const long per = (long)tilesM * tilesN;
  *f = (int)(t / per);
  const long tl = t % per;
  const long gs = (long)kGroupM * tilesN;
  const int g = (int)(tl / gs);
  const int r = (int)(tl % gs);
  const int gm = min(kGroupM, tilesM - g * kGroupM);
  *m0 = (g * kGroupM + r % gm) * kBM;
  *n0 = (r / gm) * BN;
}

// Persistent C -= A B over all tiles of all fronts: one CTA per SM, a ring of
// STAGES shared-memory stages filled by TMA (warp 8), tcgen05.mma issued by one
// thread of warp 9 into one of two tensor-memory accumulators, and the epilogue
// (warps 0-7) draining the other accumulator: warp w reads TMEM lanes 32 (w % 4)
// .. +31 (tile rows) and column half w / 4, subtracts from C with the C loads of
// later chunks already in flight (CRING = 2: the next tile's four chunks, two in
// registers and two in shared-memory slots after the STAGES operand stages; CRING = 1:
// three in registers and one slot, which leaves room for four operand stages;
// CRING = 0: the next chunk, in registers).
// CL = 2: the CTAs run in thread-block clusters of two that take row tiles m0 and
// m0 + 128 of the same column block together; each loads its own A and half of the B
// tile (tmB's box is 128 rows) and multicasts that half to both, so a stage costs a CTA
// 32 KB of L2 reads instead of 48; a stage is refilled once both CTAs' products have
// released it (the MMA commits arrive on both CTAs' empty barriers).  ntiles then
// counts pairs of row tiles.  The products of every tile are those of CL = 1.
template <int BN, int STAGES, int CRING, int CL = 1>
__global__ void __launch_bounds__(kPThreads, 1) tc_gemm_sub_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
    int N, int nk, float* C, int ldc, long sC, int tilesM, int tilesN, long ntiles, int* status) {
  constexpr uint32_t kABytes = kBM * kBK * 4;
  constexpr uint32_t kBBytes = BN * kBK * 4;
  constexpr uint32_t kStage = kABytes + kBBytes;
  constexpr int kHalf = BN / 2;
  // instruction descriptor: D = F32 (bits 4-5), A = B = TF32 (bits 7-9, 10-12),
  // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                              ((uint32_t)(kBM >> 4) << 24);
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) unsigned long long full[STAGES], empty[STAGES], acc_full[2],
      acc_empty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  __shared__ long long s_issued, s_consumed;
  volatile int* ab = &s_abort;
  const uint32_t base = (smem_u32(smraw) + 1023u) & ~1023u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t crank = 0;
  if constexpr (CL == 2) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
  const long tfirst = CL == 2 ? blockIdx.x / 2 : blockIdx.x;
  const long tstep = CL == 2 ? gridDim.x / 2 : gridDim.x;
  const int tilesMu = CL == 2 ? (tilesM + 1) / 2 : tilesM;  // row units: tile pairs for CL = 2
  auto coords = [&](long t, int* f, int* m0, int* n0) {
    tile_coords(t, tilesMu, tilesN, BN, f, m0, n0);
    if constexpr (CL == 2) *m0 = 2 * *m0 + (int)crank * kBM;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), CL);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), kEpiWarps);
    }
    mbar_init(smem_u32(&drain), 1);
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CL == 2) cluster_sync_all();  // the peer's barriers exist before any multicast
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kEpiWarps) {
    if (lane == 0) {  // TMA producer
      long long g = 0;
      for (long t = tfirst; t < ntiles && !*ab; t += tstep) {
        int f, m0, n0;
        coords(t, &f, &m0, &n0);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % STAGES);
          if (g >= STAGES &&
              !mbar_wait_ab(smem_u32(&empty[s]), (uint32_t)(((g / STAGES) & 1) ^ 1), ab))
            break;
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(fb, kStage);
          tma_load_3d(base + s * kStage, &tmA, kb * kBK, m0, f, fb);
          if constexpr (CL == 2)
            tma_load_3d_mc(base + s * kStage + kABytes + crank * (kBBytes / 2), &tmB, kb * kBK,
                           n0 + (int)crank * kHalf, f, fb, (uint16_t)0x3);
          else
            tma_load_3d(base + s * kStage + kABytes, &tmB, kb * kBK, n0, f, fb);
        }
        if (*ab) break;
      }
      s_issued = g;
      if constexpr (CL == 2) {
        // the last stages' releases, the peer's included, have arrived before this CTA
        // may leave the cluster
        for (long long i = g > STAGES ? g - STAGES : 0; i < g && !*ab; ++i)
          if (!mbar_wait_ab(smem_u32(&empty[i % STAGES]), (uint32_t)((i / STAGES) & 1), ab)) break;
      }
    }
  } else if (warp == kEpiWarps + 1) {
    if (lane == 0) {  // MMA issuer
      long long g = 0;
      long i = 0;
      for (long t = tfirst; t < ntiles && !*ab; t += tstep, ++i) {
        const int buf = (int)(i & 1);
        const long u = i >> 1;
        if (u >= 1 && !mbar_wait_ab(smem_u32(&acc_empty[buf]), (uint32_t)((u - 1) & 1), ab)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        bool okk = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % STAGES);
          if (!mbar_wait_ab(smem_u32(&full[s]), (uint32_t)((g / STAGES) & 1), ab)) {
            okk = false;
            break;
          }
          tc_fence_after();
          const unsigned long long ad = sw128_desc(base + s * kStage);
          const unsigned long long bd = sw128_desc(base + s * kStage + kABytes);
#pragma unroll
          for (int kk = 0; kk < kBK / kUK; ++kk)  // +32 bytes along K = +2 in the address field
            mma_tf32(d, ad + 2 * kk, bd + 2 * kk, kIdesc, (kb | kk) != 0 ? 1u : 0u);
          if constexpr (CL == 2)
            mma_commit_mc(smem_u32(&empty[s]), (uint16_t)0x3);
          else
            mma_commit(smem_u32(&empty[s]));
        }
        if (!okk) break;
        mma_commit(smem_u32(&acc_full[buf]));
      }
      s_consumed = g;
      mma_commit(smem_u32(&drain));  // every MMA issued above has completed
      if (!mbar_wait(smem_u32(&drain), 0)) *ab = 1;
    }
  } else {
    if constexpr (CRING > 0) {
      // epilogue: four chunks of 32 columns per tile; the first 4 - CRING chunks of the
      // C tile are loaded into register buffers, the last CRING by cp.async into
      // shared-memory slots, each issued as soon as the same chunk of the previous
      // tile has been stored, so a whole tile of C loads is in flight ahead of its use
      static_assert(kHalf == 128, "the C ring assumes BN = 256");
      constexpr int kReg = 4 - CRING;
      const int qw = warp & 3, h = warp >> 2;
      const int et = threadIdx.x;  // 0 .. 255
      const uint32_t ring_s = base + STAGES * kStage;
      const float* ring = reinterpret_cast<const float*>(smraw + (ring_s - smem_u32(smraw)));
      float creg[kReg][32];
      auto locate = [&](long tt, float** cp, int* ncol) {
        int f, m0, n0;
        coords(tt, &f, &m0, &n0);
        const int row = m0 + qw * 32 + lane;
        *ncol = row < M ? min(kHalf, N - (n0 + h * kHalf)) : 0;
        *cp = C + (long)f * sC + row + (long)(n0 + h * kHalf) * ldc;
      };
      auto load = [&](float* buf, const float* cp, int ncol, int c0) {
#pragma unroll
        for (int j = 0; j < 32; ++j) buf[j] = c0 + j < ncol ? cp[(long)(c0 + j) * ldc] : 0.f;
      };
      auto sload = [&](int slot, const float* cp, int ncol, int c0) {
#pragma unroll 8
        for (int j = 0; j < 32; ++j)
          if (c0 + j < ncol)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                             ring_s + (uint32_t)(((slot * 32 + j) * 256 + et) * 4)),
                         "l"(cp + (long)(c0 + j) * ldc)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
      };
      long t = tfirst;
      float* cp = C;
      int ncol = 0;
      if (t < ntiles) {
        locate(t, &cp, &ncol);
#pragma unroll
        for (int j = 0; j < kReg; ++j) load(creg[j], cp, ncol, 32 * j);
#pragma unroll
        for (int sl = 0; sl < CRING; ++sl) sload(sl, cp, ncol, 32 * (kReg + sl));
      }
      for (long i = 0; t < ntiles; t += tstep, ++i) {
        const int buf = (int)(i & 1);
        const long u = i >> 1;
        int okw = 0;
        if (lane == 0) okw = mbar_wait_ab(smem_u32(&acc_full[buf]), (uint32_t)(u & 1), ab) ? 1 : 0;
        __syncwarp();
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) break;
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)(buf * BN + h * kHalf);
        float* cp_nx = cp;
        int ncol_nx = 0;
        if (t + tstep < ntiles) locate(t + tstep, &cp_nx, &ncol_nx);
        uint32_t v[32];
        // register chunks: store this tile's, load the next tile's
#pragma unroll
        for (int j = 0; j < kReg; ++j) {
          tmem_ld32(ta + 32 * j, v);
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (32 * j + q < ncol) cp[(long)(32 * j + q) * ldc] = creg[j][q] - __uint_as_float(v[q]);
          load(creg[j], cp_nx, ncol_nx, 32 * j);
        }
        // shared-memory chunks (at each point at most the groups of the later slots
        // are still in flight: groups complete in order)
#pragma unroll
        for (int sl = 0; sl < CRING; ++sl) {
          if constexpr (CRING == 2)
            asm volatile("cp.async.wait_group 1;" ::: "memory");
          else
            asm volatile("cp.async.wait_group 0;" ::: "memory");
          const int c0 = 32 * (kReg + sl);
          tmem_ld32(ta + c0, v);
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (c0 + q < ncol)
              cp[(long)(c0 + q) * ldc] = ring[(sl * 32 + q) * 256 + et] - __uint_as_float(v[q]);
          sload(sl, cp_nx, ncol_nx, c0);
        }
        cp = cp_nx;
        ncol = ncol_nx;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
      // epilogue: chunks of 32 columns, two register buffers in rotation so the C
      // loads of the next chunk (and, at the end of a tile, of the next tile's first
      // chunk) are in flight while the current one is stored
      constexpr int kChunks = kHalf / 32;
      const int qw = warp & 3, h = warp >> 2;
      float cA[32], cB[32];
      auto locate = [&](long tt, float** cp, int* ncol) {
        int f, m0, n0;
        coords(tt, &f, &m0, &n0);
        const int row = m0 + qw * 32 + lane;
        *ncol = row < M ? min(kHalf, N - (n0 + h * kHalf)) : 0;
        *cp = C + (long)f * sC + row + (long)(n0 + h * kHalf) * ldc;
      };
      auto load = [&](float* buf, const float* cp, int ncol, int c0) {
#pragma unroll
        for (int j = 0; j < 32; ++j) buf[j] = c0 + j < ncol ? cp[(long)(c0 + j) * ldc] : 0.f;
      };
      long t = tfirst;
      float* cp = C;
      int ncol = 0;
      if (t < ntiles) {
        locate(t, &cp, &ncol);
        load(cA, cp, ncol, 0);
      }
      for (long i = 0; t < ntiles; t += tstep, ++i) {
        const int buf = (int)(i & 1);
        const long u = i >> 1;
        if (kChunks > 1) load(cB, cp, ncol, 32);
        // one lane waits, the warp follows (tcgen05.ld below is warp-collective)
        int okw = 0;
        if (lane == 0) okw = mbar_wait_ab(smem_u32(&acc_full[buf]), (uint32_t)(u & 1), ab) ? 1 : 0;
        __syncwarp();
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) break;
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)(buf * BN + h * kHalf);
        float* cp_nx = cp;
        int ncol_nx = 0;
        const bool has_next = t + tstep < ntiles;
        if (has_next) locate(t + tstep, &cp_nx, &ncol_nx);
#pragma unroll
        for (int j = 0; j < kChunks; ++j) {
          float* cur = (j & 1) ? cB : cA;
          uint32_t v[32];
          tmem_ld32(ta + 32 * j, v);
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (32 * j + q < ncol) cp[(long)(32 * j + q) * ldc] = cur[q] - __uint_as_float(v[q]);
          if (j + 2 < kChunks) load(cur, cp, ncol, 32 * (j + 2));
          else if (j + 2 == kChunks && has_next) load(cur, cp_nx, ncol_nx, 0);
        }
        if (kChunks == 1 && has_next) load(cA, cp_nx, ncol_nx, 0);
        cp = cp_nx;
        ncol = ncol_nx;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
      }
    }
  }
  __syncthreads();
  if (*ab && threadIdx.x == 0) {
    atomicOr(status, 2);
    // drain: wait (bounded) for the copies issued but never consumed
    for (long long g = s_consumed; g < s_issued; ++g)
      (void)mbar_wait(smem_u32(&full[g % STAGES]), (uint32_t)((g / STAGES) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CL == 2) cluster_sync_all();  // no multicast or remote arrival still targets us
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
  }
}

// packA[f][i][kk] = tf32(A[f sA + i + kk lda]) for kk < K, 0 for K <= kk < Kp
// (row length Kp; split: row length 3 Kp holding lo, hi, hi).  32 x 32 tiles
// transposed through shared memory; block (32, 8).
__global__ void tc_pack_a_kernel(const float* __restrict__ A, int lda, long sA, int M, int K,
                                 int Kp, int split, float* __restrict__ P) {
  __shared__ float t[32][33];
  const long f = blockIdx.z;
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int kk = k0 + r, i = i0 + threadIdx.x;
    t[r][threadIdx.x] = (i < M && kk < K) ? A[f * sA + i + (long)kk * lda] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = i0 + r, kk = k0 + threadIdx.x;
    if (i >= M) continue;
    const float a = t[threadIdx.x][r], hi = to_tf32(a);
    if (!split) {
      P[(f * M + i) * (long)Kp + kk] = hi;
    } else {
      float* row = P + (f * M + i) * (long)(3 * Kp);
      row[kk] = to_tf32(a - hi);
      row[Kp + kk] = hi;
      row[2 * Kp + kk] = hi;
    }
  }
}

// packB[f][j][kk] = tf32(B[f sB + kk + j ldb]) for kk < K, 0 for K <= kk < Kp
// (split: row length 3 Kp holding hi, lo, hi).
__global__ void tc_pack_b_kernel(const float* __restrict__ B, int ldb, long sB, int N, int K,
                                 int Kp, int split, float* __restrict__ P) {
  const long f = blockIdx.y;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)N * Kp) return;
  const int kk = (int)(e % Kp);
  const long j = e / Kp;
  const float b = kk < K ? B[f * sB + kk + j * ldb] : 0.f;
  const float hi = to_tf32(b);
  if (!split) {
    P[f * N * (long)Kp + e] = hi;
  } else {
    float* row = P + (f * N + j) * (long)(3 * Kp);
    row[kk] = hi;
    row[Kp + kk] = to_tf32(b - hi);
    row[2 * Kp + kk] = hi;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t encode_operand(CUtensorMap* map, float* P, int rows, int Kp, int batch, int box_rows) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  if (!g_encode) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 4, (cuuint64_t)rows * Kp * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kBN = 256;
// three configurations of the same kernel: four operand stages plus one 32 KB
// shared-memory slot that cp.async fills with C a tile ahead, the other three chunks
// of the next C tile in registers (the default; 3D 128^3 TF32 factor, depth-1024
// updates: 646 TFLOP/s); three stages plus two slots (583 TFLOP/s); four stages with
// only the next chunk of C in registers (at depth 512 slower than two slots: 1.72
// against 1.64 s of updates per factorisation)
constexpr int kStages = 4, kStagesRing = 3;
constexpr size_t kSmem = (size_t)kStages * (kBM * kBK * 4 + kBN * kBK * 4) + 1024;
constexpr size_t kSmemRing =
    (size_t)kStagesRing * (kBM * kBK * 4 + kBN * kBK * 4) + 1024 + 2 * 32 * 256 * 4;
// four stages and one 32 KB C slot (three C chunks a tile ahead in registers): 225 KB
constexpr size_t kSmemRing1 =
    (size_t)kStages * (kBM * kBK * 4 + kBN * kBK * 4) + 1024 + 1 * 32 * 256 * 4;
static_assert(kSmemRing1 <= 227 * 1024 - 512, "dynamic shared memory of the 4-stage ring");
int g_num_sms[64] = {0};

}  // namespace

size_t tc_pack_floats(int rows, int K, int batch, bool split) {
  return (size_t)batch * rows * (size_t)((K + kBK - 1) / kBK * kBK) * (split ? 3 : 1);
}

namespace {

cudaError_t tc_set_attributes() {
  static bool attr = false;
  if (attr) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_sub_kernel<kBN, kStages, 0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(tc_gemm_sub_kernel<kBN, kStagesRing, 2>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemRing);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(tc_gemm_sub_kernel<kBN, kStages, 1>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemRing1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(tc_gemm_sub_kernel<kBN, kStages, 1, 2>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemRing1);
  if (e != cudaSuccess) return e;
  attr = true;
  return cudaSuccess;
}

// the product kernel on already packed operands of depth Ke (a multiple of kBK)
cudaError_t tc_run(int M, int N, int Ke, float* C, int ldc, long sC, int batch, float* packA,
                   float* packB, int* status, cudaStream_t st, int epi) {
  CUtensorMap ta, tb;
  cudaError_t e = encode_operand(&ta, packA, M, Ke, batch, kBM);
  if (e != cudaSuccess) return e;
  // the cluster form loads B in halves (each CTA of a pair multicasts one)
  e = encode_operand(&tb, packB, N, Ke, batch, epi == 4 ? kBN / 2 : kBN);
  if (e != cudaSuccess) return e;
  const int tilesM = (M + kBM - 1) / kBM, tilesN = (N + kBN - 1) / kBN;
  const long ntiles = (long)tilesM * tilesN * batch;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_num_sms[dev]) cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<long>(ntiles, std::max(1, g_num_sms[dev]));
  if (epi == 4) {
    // clusters of two CTAs on pairs of row tiles, as many clusters as fit at once
    const long npairs = (long)((tilesM + 1) / 2) * tilesN * batch;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = kSmemRing1;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(2 * std::max(1, g_num_sms[dev] / 2)));
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, tc_gemm_sub_kernel<kBN, kStages, 1, 2>, &cfg) !=
            cudaSuccess || ncl < 1)
      return cudaErrorInvalidConfiguration;
    cfg.gridDim = dim3((unsigned)(2 * std::min<long>(ncl, npairs)));
    return cudaLaunchKernelEx(&cfg, tc_gemm_sub_kernel<kBN, kStages, 1, 2>, ta, tb, M, N,
                              Ke / kBK, C, ldc, sC, tilesM, tilesN, npairs, status);
  }
  if (epi == 0 || epi == 3)
    tc_gemm_sub_kernel<kBN, kStages, 1><<<grid, kPThreads, kSmemRing1, st>>>(
        ta, tb, M, N, Ke / kBK, C, ldc, sC, tilesM, tilesN, ntiles, status);
  else if (epi != 1)
    tc_gemm_sub_kernel<kBN, kStagesRing, 2><<<grid, kPThreads, kSmemRing, st>>>(
        ta, tb, M, N, Ke / kBK, C, ldc, sC, tilesM, tilesN, ntiles, status);
  else
    tc_gemm_sub_kernel<kBN, kStages, 0><<<grid, kPThreads, kSmem, st>>>(
        ta, tb, M, N, Ke / kBK, C, ldc, sC, tilesM, tilesN, ntiles, status);
  return cudaGetLastError();
}

void tc_pack(int M, int N, int K, const float* A, int lda, long sA, const float* B, int ldb,
             long sB, int batch, float* packA, float* packB, bool split, cudaStream_t st) {
  const int Kp = (K + kBK - 1) / kBK * kBK;
  dim3 g((M + 31) / 32, Kp / 32, batch);
  tc_pack_a_kernel<<<g, dim3(32, 8), 0, st>>>(A, lda, sA, M, K, Kp, split ? 1 : 0, packA);
  const long nb = (long)N * Kp;
  dim3 gb((unsigned)((nb + 255) / 256), batch);
  tc_pack_b_kernel<<<gb, 256, 0, st>>>(B, ldb, sB, N, K, Kp, split ? 1 : 0, packB);
}

// deterministic uniform values in [-1, 1) from a hash of the index
__global__ void tc_probe_fill_kernel(float* p, long n, unsigned seed) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    p[i] = (float)(h & 0xFFFFu) * (1.0f / 32768.0f) - 1.0f;
  }
}

}  // namespace

cudaError_t tc_schur_update(int M, int N, int K, const float* A, int lda, long sA, const float* B,
                            int ldb, long sB, float* C, int ldc, long sC, int batch, float* packA,
                            float* packB, bool split, int* status, cudaStream_t st, int epi) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (K > kTcMaxKProbe || batch > 65535 || !packA || !packB) return cudaErrorInvalidValue;
  cudaError_t e = tc_set_attributes();
  if (e != cudaSuccess) return e;
  const int Kp = (K + kBK - 1) / kBK * kBK;
  const int Ke = split ? 3 * Kp : Kp;  // depth of the packed product
  tc_pack(M, N, K, A, lda, sA, B, ldb, sB, batch, packA, packB, split, st);
  return tc_run(M, N, Ke, C, ldc, sC, batch, packA, packB, status, st, epi);
}

cudaError_t tc_probe(bool split, int M, int N, int K, int reps, cudaStream_t st, float* ms,
                     int* hstatus) {
  *ms = 0.f;
  *hstatus = 0;
  cudaError_t e = tc_set_attributes();
  if (e != cudaSuccess) return e;
  float *A = nullptr, *B = nullptr, *C = nullptr, *pa = nullptr, *pb = nullptr;
  int* status = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int Kp = (K + kBK - 1) / kBK * kBK;
  const int Ke = split ? 3 * Kp : Kp;
  e = cudaMalloc(&A, sizeof(float) * (size_t)M * K);
  if (e == cudaSuccess) e = cudaMalloc(&B, sizeof(float) * (size_t)K * N);
  if (e == cudaSuccess) e = cudaMalloc(&C, sizeof(float) * (size_t)M * N);
  if (e == cudaSuccess) e = cudaMalloc(&pa, sizeof(float) * tc_pack_floats(M, K, 1, split));
  if (e == cudaSuccess) e = cudaMalloc(&pb, sizeof(float) * tc_pack_floats(N, K, 1, split));
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    tc_probe_fill_kernel<<<1024, 256, 0, st>>>(A, (long)M * K, 17u);
    tc_probe_fill_kernel<<<1024, 256, 0, st>>>(B, (long)K * N, 29u);
    tc_probe_fill_kernel<<<1024, 256, 0, st>>>(C, (long)M * N, 43u);
    e = cudaMemsetAsync(status, 0, sizeof(int), st);
  }
  if (e == cudaSuccess) {
    tc_pack(M, N, K, A, M, 0, B, K, 0, 1, pa, pb, split, st);
    e = tc_run(M, N, Ke, C, M, 0, 1, pa, pb, status, st, 0);  // warm-up
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r)
    e = tc_run(M, N, Ke, C, M, 0, 1, pa, pb, status, st, 0);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (float)reps;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(A);
  cudaFree(B);
  cudaFree(C);
  cudaFree(pa);
  cudaFree(pb);
  cudaFree(status);
  return e;
}

}  // namespace sp
