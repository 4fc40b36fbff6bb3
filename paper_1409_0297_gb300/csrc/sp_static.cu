// g = G f without a context and without any allocation: the work buffer of the
// FFT passes is a fixed-size array in device global memory, declared at file
// scope in this translation unit.
//
// Who needs this: callers that cannot allocate device memory at the point of
// the call -- code that runs while a stream is being captured into a CUDA graph
// (allocation calls are not allowed there), callers whose memory is carved out
// up front under a hard budget, or a caller that must not hit allocator latency
// inside a timed loop.  They pass their own input and output buffers and the
// library's static work array does the rest.
//
// Limits and sharing: the array holds kStaticMaxN complex128 values (4 MiB), so
// grids with n^d <= 262144 are accepted (e.g. 512^2 or 64^3).  It exists once per
// device that loads the library and is kept until the process exits.  Every call
// on a device uses the same array, so calls whose kernels may run at the same
// time (different streams without ordering between them, or several host
// threads) overwrite each other's intermediate data: order them.  Each call
// writes every entry it later reads, so nothing needs clearing between calls.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress and caches it; make that first
// call before any stream capture starts.  The cached address belongs to the
// device's current CUDA context: after cudaDeviceReset on that device the
// library must be reloaded (the process restarted) before this entry point is
// called again.
//
// Errors: a CUDA error left pending by earlier work of the caller is reported as
// SP_ERR_CUDA before anything is launched, and is not cleared, so it is not
// mistaken for a failure of this call nor hidden from the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "sp_internal.h"

namespace sp {

namespace {

constexpr long kStaticMaxN = 1L << 18;  // complex128 entries of the work array
constexpr int kMaxDevices = 64;
constexpr int kThreadsS = 256;

__device__ __align__(256) double2 g_static_work[kStaticMaxN];

std::mutex g_static_mu;
double2* g_static_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double2 smul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// One pass of 1D transforms along an axis (stride S), lines staged in shared
// memory, twiddles computed in the prologue.  mode 0: forward (decimation in
// time), 1: inverse (decimation in frequency), 2: forward, multiply by the Green
// symbol 1/(4 pi^2 |k|^2 - s) / N computed from the flat index, inverse.
__global__ void __launch_bounds__(kThreadsS) green_static_pass(const double2* in, double2* out,
                                                               int d, int n, int logn, long S,
                                                               long nlines, int mode, double s) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* tw = reinterpret_cast<double2*>(smraw);  // n/2 twiddles
  double2* a = tw + n / 2;                          // one line of n values
  const long t = blockIdx.x;                        // one line per CTA
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)j / (double)n, &sn, &cs);
    tw[j] = make_double2(cs, -sn);  // exp(-2 pi i j / n)
  }
  const long base = (t % S) + (t / S) * S * n;
  const bool bitrev_load = (mode != 1);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int pos = bitrev_load ? (int)(__brev((unsigned)i) >> (32 - logn)) : i;
    a[pos] = in[base + (long)i * S];
  }
  __syncthreads();
  auto dit = [&](bool cj) {
    for (int st = 1; st <= logn; ++st) {
      const int half = 1 << (st - 1);
      for (int p = threadIdx.x; p < n / 2; p += blockDim.x) {
        int jj = p & (half - 1);
        int i0 = ((p >> (st - 1)) << st) + jj, i1 = i0 + half;
        double2 w = tw[jj << (logn - st)];
        if (cj) w.y = -w.y;
        double2 u = a[i0], v = smul(a[i1], w);
        a[i0] = make_double2(u.x + v.x, u.y + v.y);
        a[i1] = make_double2(u.x - v.x, u.y - v.y);
      }
      __syncthreads();
    }
  };
  auto dif = [&](bool cj) {
    for (int st = logn; st >= 1; --st) {
      const int half = 1 << (st - 1);
      for (int p = threadIdx.x; p < n / 2; p += blockDim.x) {
        int jj = p & (half - 1);
        int i0 = ((p >> (st - 1)) << st) + jj, i1 = i0 + half;
        double2 w = tw[jj << (logn - st)];
        if (cj) w.y = -w.y;
        double2 u = a[i0], v = a[i1];
        a[i0] = make_double2(u.x + v.x, u.y + v.y);
        a[i1] = smul(make_double2(u.x - v.x, u.y - v.y), w);
      }
      __syncthreads();
    }
  };
  if (mode == 0) {
    dit(false);
  } else if (mode == 1) {
    dif(true);
  } else {
    dit(false);
    long N = 1;
    for (int q = 0; q < d; ++q) N *= n;
    const double four_pi2 = 39.47841760435743447533796399635;  // 4 pi^2
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      long g = base + (long)i * S, r = g;
      double k2 = 0;
      for (int q = 0; q < d; ++q) {
        int c = (int)(r % n);
        r /= n;
        int kq = c < n / 2 ? c : c - n;
        k2 += (double)kq * kq;
      }
      double dn = 1.0 / ((four_pi2 * k2 - s) * (double)N);
      a[i].x *= dn;
      a[i].y *= dn;
    }
    __syncthreads();
    dif(true);
  }
  const bool bitrev_store = (mode != 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int pos = bitrev_store ? (int)(__brev((unsigned)i) >> (32 - logn)) : i;
    out[base + (long)i * S] = a[pos];
  }
}

}  // namespace

}  // namespace sp

using namespace sp;

extern "C" sp_status sp_green_static(int d, int n, double s, const void* f_dev, void* g_dev,
                                     void* stream) {
  if ((d != 2 && d != 3) || n < 4 || (n & (n - 1)) || !f_dev || !g_dev || f_dev == g_dev)
    return SP_ERR_ARG;
  long N = 1;
  for (int a = 0; a < d; ++a) N *= n;
  if (N > kStaticMaxN) return SP_ERR_ARG;  // beyond the static work array
  if (!(s == s) || resonance_gap(d, n, s) < 1e-6) return SP_ERR_RESONANT;
  if (cudaPeekAtLastError() != cudaSuccess) return SP_ERR_CUDA;  // the caller's, left in place
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SP_ERR_CUDA;
  double2* work = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_work) != cudaSuccess || !p) return SP_ERR_CUDA;
      g_static_ptr[dev] = static_cast<double2*>(p);
    }
    work = g_static_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  const size_t smem = sizeof(double2) * (size_t)(n / 2 + n);
  const long nlines = N / n;
  const double2* x = static_cast<const double2*>(f_dev);
  double2* out = static_cast<double2*>(g_dev);
  // forward along axes 0..d-2 into the work array, middle pass on axis d-1,
  // inverse along d-2..0, the last one into the output
  const double2* src = x;
  long S = 1;
  for (int ax = 0; ax < d - 1; ++ax) {
    green_static_pass<<<(unsigned)nlines, kThreadsS, smem, st>>>(src, work, d, n, logn, S, nlines, 0, s);
    src = work;
    S *= n;
  }
  green_static_pass<<<(unsigned)nlines, kThreadsS, smem, st>>>(src, work, d, n, logn, S, nlines, 2, s);
  for (int ax = d - 2; ax >= 0; --ax) {
    S /= n;
    green_static_pass<<<(unsigned)nlines, kThreadsS, smem, st>>>(work, ax == 0 ? out : work, d, n,
                                                                 logn, S, nlines, 1, s);
  }
  return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ERR_CUDA;
}
