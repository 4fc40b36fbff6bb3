// Host-side set-up: Green's kernel, stencil tables and nested-dissection symbolic
// structure.  See sp_host.h.
#include "sp_host.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <exception>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace sp {

using cd = std::complex<double>;
static const double kPi = 3.141592653589793238462643383279502884;

int check_grid(int d, int n, int b, int* L) {
  if (d != 2 && d != 3) return 1;
  if (b < 2 || n < 2 * b || n % b) return 1;
  {  // grid indices are ints: n^d must stay below 2^31
    long long N = 1;
    for (int a = 0; a < d; ++a) {
      if (N > 2147483647LL / n) return 1;
      N *= n;
    }
  }
  int r = n / b, l = 0;
  while (r > 1) {
    if (r & 1) return 1;
    r >>= 1;
    ++l;
  }
  if (l < 1) return 1;
  if (L) *L = l;
  return 0;
}

// ---------------------------------------------------------------- host threads
// Runs f(i) for i = 0 .. count - 1 on up to nth host threads, the calling thread
// included.  Items come from a shared counter, so when a thread cannot be started the
// running ones take its share; the first exception an item throws is rethrown here
// once every thread has joined.
template <class F>
static void parallel_items(int count, int nth, F f) {
  std::atomic<int> next{0};
  std::mutex mu;
  std::exception_ptr err;
  auto run = [&]() {
    for (int i; (i = next.fetch_add(1)) < count;) {
      try {
        f(i);
      } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        if (!err) err = std::current_exception();
      }
    }
  };
  std::vector<std::thread> th;
  th.reserve((size_t)std::max(0, std::min(nth, count) - 1));  // no reallocation below
  for (int k = 1; k < std::min(nth, count); ++k) {
    try {
      th.emplace_back(run);
    } catch (const std::exception&) {
      break;
    }
  }
  run();
  for (auto& t : th) t.join();
  if (err) std::rethrow_exception(err);
}

// ---------------------------------------------------------------- host FFT
// exp(sign * 2 pi i t / n) with t reduced mod n first.
static cd twiddle(long t, long n, int sign) {
  t %= n;
  if (t < 0) t += n;
  double a = 2.0 * kPi * (double)t / (double)n;
  return cd(std::cos(a), sign * std::sin(a));
}

// The sub-lengths, radices and twiddle factors of the mixed-radix recursion below for
// lines of length n: depth q has length len[q] (n, n / p_0, n / (p_0 p_1), ... > 1),
// smallest prime factor radix[q] and tw[q][t] = twiddle(t, len[q], sign) for
// t = 0 .. len[q] - 1, so the recursion looks its twiddles up instead of evaluating
// cos and sin per term.
struct FftPlan {
  std::vector<int> len, radix;
  std::vector<std::vector<cd>> tw;
};

static FftPlan fft_plan(int n, int sign) {
  FftPlan P;
  for (int m = n; m > 1;) {
    int p = 2;
    while (m % p) ++p;
    P.len.push_back(m);
    P.radix.push_back(p);
    std::vector<cd> w(m);
    for (int t = 0; t < m; ++t) w[t] = twiddle(t, m, sign);
    P.tw.push_back(std::move(w));
    m /= p;
  }
  return P;
}

// Mixed-radix decimation-in-time DFT of the contiguous line x[0..n), n = P.len[q]
// (nothing to do at length 1): the p decimated sub-lines are transformed
// recursively, then X_k = sum_r Sub_r[k mod m] exp(sign 2 pi i r k / n).  scratch
// holds at least 2n values (this depth's sub-lines, then the deeper ones').
static void fft_line(cd* x, const FftPlan& P, int q, cd* scratch) {
  if (q == (int)P.len.size()) return;
  const int n = P.len[q], p = P.radix[q], m = n / p;
  cd* sub = scratch;
  for (int r = 0; r < p; ++r)
    for (int j = 0; j < m; ++j) sub[(size_t)r * m + j] = x[(size_t)j * p + r];
  for (int r = 0; r < p; ++r) fft_line(sub + (size_t)r * m, P, q + 1, scratch + n);
  const cd* w = P.tw[q].data();
  for (int k = 0; k < n; ++k) {
    cd acc = 0.0;
    const int kk = k % m;
    for (int r = 0; r < p; ++r) acc += sub[(size_t)r * m + kk] * w[((long)r * k) % n];
    x[k] = acc;
  }
}

// Transform of the n^d array a along every axis; the lines of an axis are
// independent and split over up to `threads` host threads (0 = all).
static void fft_nd(std::vector<cd>& a, int d, int n, int sign, int threads) {
  size_t N = 1;
  for (int i = 0; i < d; ++i) N *= n;
  const FftPlan P = fft_plan(n, sign);
  const size_t lines = N / n;
  int nth = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
  nth = (int)std::min<size_t>({(size_t)nth, (size_t)64, lines});
  size_t S = 1;
  for (int ax = 0; ax < d; ++ax) {
    // line q of axis ax: element i at base + i S, base = (q mod S) + (q / S) S n
    auto worker = [&](int id) {
      std::vector<cd> line(n), scratch(2 * (size_t)n);
      for (size_t q = id; q < lines; q += nth) {
        const size_t base = (q % S) + (q / S) * S * n;
        for (int i = 0; i < n; ++i) line[i] = a[base + (size_t)i * S];
        fft_line(line.data(), P, 0, scratch.data());
        for (int i = 0; i < n; ++i) a[base + (size_t)i * S] = line[i];
      }
    };
    parallel_items(nth, nth, worker);
    S *= n;
  }
}

static inline int kfreq(int i, int n) { return i < n / 2 ? i : i - n; }

std::vector<double> green_kernel(int d, int n, double s, int threads) {
  size_t N = 1;
  for (int i = 0; i < d; ++i) N *= n;
  std::vector<cd> a(N);
  for (size_t j = 0; j < N; ++j) {
    size_t r = j;
    double k2 = 0;
    for (int ax = 0; ax < d; ++ax) {
      int k = kfreq((int)(r % n), n);
      r /= n;
      k2 += (double)k * k;
    }
    a[j] = 1.0 / (4.0 * kPi * kPi * k2 - s);
  }
  fft_nd(a, d, n, +1, threads);
  std::vector<double> g(N);
  for (size_t j = 0; j < N; ++j) g[j] = a[j].real() / (double)N;
  return g;
}

std::vector<double> green_kernel_sq(int d, int n, double s, int threads) {
  size_t N = 1;
  for (int i = 0; i < d; ++i) N *= n;
  std::vector<cd> a(N);
  for (size_t j = 0; j < N; ++j) {
    size_t r = j;
    double k2 = 0;
    for (int ax = 0; ax < d; ++ax) {
      int k = kfreq((int)(r % n), n);
      r /= n;
      k2 += (double)k * k;
    }
    const double dk = 1.0 / (4.0 * kPi * kPi * k2 - s);
    a[j] = dk * dk;
  }
  fft_nd(a, d, n, +1, threads);
  std::vector<double> g(N);
  for (size_t j = 0; j < N; ++j) g[j] = a[j].real() / (double)N;
  return g;
}

double resonance_gap(int d, int n, double s) {
  double kappa = s / (4.0 * kPi * kPi);
  double best = 1e300;
  // |k|^2 takes integer values; scan all of K in one dimension combinations
  if (d == 2) {
    for (int i = -n / 2; i < n / 2; ++i)
      for (int j = -n / 2; j < n / 2; ++j) best = std::min(best, std::fabs(kappa - (double)(i * i + j * j)));
  } else {
    for (int i = -n / 2; i < n / 2; ++i)
      for (int j = -n / 2; j < n / 2; ++j)
        for (int l = -n / 2; l < n / 2; ++l)
          best = std::min(best, std::fabs(kappa - (double)(i * i + j * j + l * l)));
  }
  return best / std::max(1.0, std::fabs(kappa));
}

// ---------------------------------------------------------------- set geometry
// Cartesian product of per-axis ranges [lo_a, hi_a], axis 0 fastest.
static std::vector<int> box_points(int d, const int* lo, const int* hi) {
  std::vector<int> pts;
  int cnt = 1;
  for (int a = 0; a < d; ++a) cnt *= (hi[a] - lo[a] + 1);
  pts.reserve((size_t)cnt * d);
  int p[3];
  for (int a = 0; a < d; ++a) p[a] = lo[a];
  for (int c = 0; c < cnt; ++c) {
    for (int a = 0; a < d; ++a) pts.push_back(p[a]);
    for (int a = 0; a < d; ++a) {
      if (++p[a] <= hi[a]) break;
      p[a] = lo[a];
    }
  }
  return pts;
}

static void set_geometry(int d, int b, int t, std::vector<int>* S, std::vector<int>* G,
                         std::vector<int>* Bt) {
  int lo[3], hi[3], glo[3], ghi[3];
  for (int a = 0; a < d; ++a) {
    bool z = (t >> a) & 1;
    lo[a] = z ? 0 : 1;
    hi[a] = z ? 0 : b - 1;
    glo[a] = z ? -1 : 0;
    ghi[a] = z ? 1 : b;
  }
  *S = box_points(d, lo, hi);
  *G = box_points(d, glo, ghi);
  Bt->clear();
  int nG = (int)G->size() / d;
  for (int i = 0; i < nG; ++i) {
    bool in = true;
    for (int a = 0; a < d; ++a) {
      int v = (*G)[(size_t)i * d + a];
      if (v < lo[a] || v > hi[a]) in = false;
    }
    if (!in)
      for (int a = 0; a < d; ++a) Bt->push_back((*G)[(size_t)i * d + a]);
  }
}

static inline long flat_of(const int* p, int d, int n) {
  long f = 0, s = 1;
  for (int a = 0; a < d; ++a) {
    int v = p[a] % n;
    if (v < 0) v += n;
    f += (long)v * s;
    s *= n;
  }
  return f;
}

// ---------------------------------------------------------------- dense kernels
// Householder QR of the column-major h x c matrix X (leading dimension h);
// on return its upper c x c triangle is R (rows below are zeroed).
static void house_qr(double* X, int h, int c) {
  for (int j = 0; j < c && j < h; ++j) {
    double* xj = X + (size_t)j * h;
    double nrm2 = 0;
    for (int i = j; i < h; ++i) nrm2 += xj[i] * xj[i];
    if (nrm2 == 0.0) continue;
    double nrm = std::sqrt(nrm2);
    double alpha = xj[j] > 0 ? -nrm : nrm;
    xj[j] -= alpha;
    double vv = 0;
    for (int i = j; i < h; ++i) vv += xj[i] * xj[i];
    if (vv > 0) {
      for (int k = j + 1; k < c; ++k) {
        double* xk = X + (size_t)k * h;
        double d0 = 0, d1 = 0, d2 = 0, d3 = 0;
        int i = j;
        for (; i + 3 < h; i += 4) {
          d0 += xj[i] * xk[i];
          d1 += xj[i + 1] * xk[i + 1];
          d2 += xj[i + 2] * xk[i + 2];
          d3 += xj[i + 3] * xk[i + 3];
        }
        for (; i < h; ++i) d0 += xj[i] * xk[i];
        double f = 2.0 * ((d0 + d1) + (d2 + d3)) / vv;
        for (int ii = j; ii < h; ++ii) xk[ii] -= f * xj[ii];
      }
    }
    xj[j] = alpha;
    for (int i = j + 1; i < h; ++i) xj[i] = 0.0;
  }
}

// One-sided Jacobi SVD of the square column-major r x r matrix A: A V = U_s with
// orthogonal columns; sigma_i = |U_s(:,i)|.  Returns U (normalised), sigma, V.
static void jacobi_svd(int r, std::vector<double> A, std::vector<double>* U,
                       std::vector<double>* sig, std::vector<double>* V) {
  std::vector<double> W(A);
  std::vector<double> Vm((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i) Vm[(size_t)i * r + i] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0;
    for (int i = 0; i < r - 1; ++i)
      for (int j = i + 1; j < r; ++j) {
        double* wi = &W[(size_t)i * r];
        double* wj = &W[(size_t)j * r];
        double al = 0, be = 0, ga = 0;
        for (int k = 0; k < r; ++k) {
          al += wi[k] * wi[k];
          be += wj[k] * wj[k];
          ga += wi[k] * wj[k];
        }
        if (al == 0.0 || be == 0.0) continue;
        double rel = std::fabs(ga) / std::sqrt(al * be);
        if (rel <= 1e-16) continue;
        off = std::max(off, rel);
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int k = 0; k < r; ++k) {
          double a = wi[k], bb = wj[k];
          wi[k] = c * a - s * bb;
          wj[k] = s * a + c * bb;
        }
        double* vi = &Vm[(size_t)i * r];
        double* vj = &Vm[(size_t)j * r];
        for (int k = 0; k < r; ++k) {
          double a = vi[k], bb = vj[k];
          vi[k] = c * a - s * bb;
          vj[k] = s * a + c * bb;
        }
      }
    if (off <= 1e-15) break;
  }
  // sort by descending singular value
  std::vector<double> sv(r);
  for (int i = 0; i < r; ++i) {
    double s2 = 0;
    for (int k = 0; k < r; ++k) s2 += W[(size_t)i * r + k] * W[(size_t)i * r + k];
    sv[i] = std::sqrt(s2);
  }
  std::vector<int> ord(r);
  for (int i = 0; i < r; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b2) { return sv[a] > sv[b2]; });
  U->assign((size_t)r * r, 0.0);
  V->assign((size_t)r * r, 0.0);
  sig->assign(r, 0.0);
  for (int ii = 0; ii < r; ++ii) {
    int i = ord[ii];
    (*sig)[ii] = sv[i];
    for (int k = 0; k < r; ++k) {
      (*U)[(size_t)ii * r + k] = sv[i] > 0 ? W[(size_t)i * r + k] / sv[i] : 0.0;
      (*V)[(size_t)ii * r + k] = Vm[(size_t)i * r + k];
    }
  }
}

// ---------------------------------------------------------------- stencil tables
static int finish_table(int d, int n, StencilTable& T, const std::vector<double>& g,
                        const std::vector<double>& Tm);

// Gram route (g2 given): with B = G(beta, gamma^c), A = G(S, gamma^c) and G
// symmetric, B B^T = (G^2)(beta, beta) - G(beta, gamma) G(gamma, beta) and
// A B^T = (G^2)(S, beta) - G(S, gamma) G(gamma, beta), both |gamma|-sized; then
// T = A B^T pinv(B B^T), the pseudoinverse from the eigen-decomposition of the
// symmetric B B^T (one-sided Jacobi), eigenvalues lambda = sigma(B)^2 cut at the
// same tolerance on sigma as the SVD route.  Cost O(|beta|^2 |gamma|) instead of
// O(|gamma|^2 N); accuracy ~cond(B)^2 eps instead of ~cond(B) eps.
static void gram_route(int d, int n, const StencilTable& T, const std::vector<double>& g,
                       const std::vector<double>& g2, long Np, std::vector<double>* Tm,
                       std::vector<double>* sigma, int* rank_out) {
  const int r = T.nB, p = T.nS, nG = T.nG;
  auto gk = [&](const std::vector<double>& k, const int* x, const int* y) {
    int dp[3];
    for (int a = 0; a < d; ++a) dp[a] = x[a] - y[a];
    return k[flat_of(dp, d, n)];
  };
  // G(beta, gamma) (r x nG) and G(S, gamma) (p x nG), row-major
  std::vector<double> Gbg((size_t)r * nG), Gsg((size_t)p * nG);
  for (int a = 0; a < r; ++a)
    for (int c = 0; c < nG; ++c) Gbg[(size_t)a * nG + c] = gk(g, &T.Bt[(size_t)a * d], &T.G[(size_t)c * d]);
  for (int a = 0; a < p; ++a)
    for (int c = 0; c < nG; ++c) Gsg[(size_t)a * nG + c] = gk(g, &T.S[(size_t)a * d], &T.G[(size_t)c * d]);
  std::vector<double> M((size_t)r * r), AB((size_t)p * r);  // M column-major, AB row-major
  for (int bq = 0; bq < r; ++bq) {
    for (int a = 0; a < r; ++a) {
      double acc = 0;
      for (int c = 0; c < nG; ++c) acc += Gbg[(size_t)a * nG + c] * Gbg[(size_t)bq * nG + c];
      M[(size_t)bq * r + a] = gk(g2, &T.Bt[(size_t)a * d], &T.Bt[(size_t)bq * d]) - acc;
    }
    for (int a = 0; a < p; ++a) {
      double acc = 0;
      for (int c = 0; c < nG; ++c) acc += Gsg[(size_t)a * nG + c] * Gbg[(size_t)bq * nG + c];
      AB[(size_t)a * r + bq] = gk(g2, &T.S[(size_t)a * d], &T.Bt[(size_t)bq * d]) - acc;
    }
  }
  std::vector<double> U, lam, V;
  jacobi_svd(r, M, &U, &lam, &V);
  sigma->assign(r, 0.0);
  for (int i = 0; i < r; ++i) (*sigma)[i] = std::sqrt(std::max(0.0, lam[i]));
  const double smax = r ? (*sigma)[0] : 0.0;
  int rank = 0;
  if (smax > 0) {
    const double tol = (double)std::max<long>(r, Np) * std::ldexp(1.0, std::ilogb(smax) - 52);
    for (int i = 0; i < r; ++i)
      if ((*sigma)[i] > tol) ++rank;
  }
  *rank_out = rank;
  // T[a][q] = sum_i (AB[a] . u_i) v_i[q] / lambda_i
  Tm->assign((size_t)p * r, 0.0);
  for (int a = 0; a < p; ++a)
    for (int i = 0; i < rank; ++i) {
      double w = 0;
      for (int k = 0; k < r; ++k) w += AB[(size_t)a * r + k] * U[(size_t)i * r + k];
      w /= lam[i];
      for (int q = 0; q < r; ++q) (*Tm)[(size_t)a * r + q] += w * V[(size_t)i * r + q];
    }
}

// T, Q and C of a table whose geometry (S, gamma, beta) is already set.
static int set_table(int d, int n, StencilTable& T, const std::vector<double>& g, int threads,
                     const std::vector<double>* g2) {
  T.nS = (int)T.S.size() / d;
  T.nG = (int)T.G.size() / d;
  T.nB = (int)T.Bt.size() / d;
  long N = 1;
  for (int a = 0; a < d; ++a) N *= n;
  std::vector<double> Tm;
  if (g2) {
    int rank = 0;
    gram_route(d, n, T, g, *g2, N - T.nG, &Tm, &T.sigma, &rank);
    T.rank = rank;
    return finish_table(d, n, T, g, Tm);
  }
  // complement of gamma (flat indices)
  std::vector<char> ing(N, 0);
  for (int i = 0; i < T.nG; ++i) ing[flat_of(&T.G[(size_t)i * d], d, n)] = 1;
  std::vector<long> comp;
  comp.reserve(N - T.nG);
  for (long j = 0; j < N; ++j)
    if (!ing[j]) comp.push_back(j);
  const long Np = (long)comp.size();
  const int r = T.nB, p = T.nS, c = r + p;
  // rows of [B^T | A^T]: for column point j, G(beta_q, j) then G(S_a, j)
  std::vector<int> pts;  // r + p points: beta then S
  pts.insert(pts.end(), T.Bt.begin(), T.Bt.end());
  pts.insert(pts.end(), T.S.begin(), T.S.end());
  auto fill_rows = [&](double* X, int h, int row0, long j0, int cnt) {
    for (int rr = 0; rr < cnt; ++rr) {
      long j = comp[j0 + rr];
      int jc[3];
      long jj = j;
      for (int a = 0; a < d; ++a) {
        jc[a] = (int)(jj % n);
        jj /= n;
      }
      for (int col = 0; col < c; ++col) {
        long f = 0, sc = 1;
        for (int a = 0; a < d; ++a) {
          int v = pts[(size_t)col * d + a] - jc[a];
          v %= n;
          if (v < 0) v += n;
          f += v * sc;
          sc *= n;
        }
        X[(size_t)col * h + row0 + rr] = g[f];
      }
    }
  };
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  threads = std::min(threads, 64);
  const int R = 1024;
  long nchunks = (Np + R - 1) / R;
  int nth = (int)std::min<long>(threads, std::max<long>(1, nchunks));
  std::vector<std::vector<double>> Rs(nth);
  auto worker = [&](int id) {
    const int h = c + R;
    std::vector<double> X((size_t)h * c, 0.0);
    bool any = false;
    for (long ch = id; ch < nchunks; ch += nth) {
      long j0 = ch * R;
      int cnt = (int)std::min<long>(R, Np - j0);
      // zero the rows below the current R and the strict lower triangle of R
      for (int col = 0; col < c; ++col) {
        double* xc = &X[(size_t)col * h];
        for (int i = col + 1; i < h; ++i) xc[i] = 0.0;
      }
      fill_rows(X.data(), h, c, j0, cnt);
      house_qr(X.data(), h, c);
      any = true;
    }
    Rs[id].assign((size_t)c * c, 0.0);
    if (any)
      for (int col = 0; col < c; ++col)
        for (int i = 0; i <= col; ++i) Rs[id][(size_t)col * c + i] = X[(size_t)col * h + i];
  };
  parallel_items(nth, nth, worker);
  // combine the per-thread triangles
  std::vector<double> Rf((size_t)c * c, 0.0);
  {
    const int h = nth * c;
    std::vector<double> X((size_t)h * c, 0.0);
    for (int id = 0; id < nth; ++id)
      for (int col = 0; col < c; ++col)
        for (int i = 0; i < c; ++i) X[(size_t)col * h + (size_t)id * c + i] = Rs[id][(size_t)col * c + i];
    house_qr(X.data(), h, c);
    for (int col = 0; col < c; ++col)
      for (int i = 0; i <= col && i < c; ++i) Rf[(size_t)col * c + i] = X[(size_t)col * h + i];
  }
  // R11 (r x r), R12 (r x p); B^T = Q1 R11, A^T = Q1 R12 + Q2 R22, so
  // T^T = pinv(B^T) A^T = pinv(R11) R12 and sigma(R11) = sigma(B).
  std::vector<double> R11((size_t)r * r), R12((size_t)r * p);
  for (int col = 0; col < r; ++col)
    for (int i = 0; i < r; ++i) R11[(size_t)col * r + i] = Rf[(size_t)col * c + i];
  for (int col = 0; col < p; ++col)
    for (int i = 0; i < r; ++i) R12[(size_t)col * r + i] = Rf[(size_t)(r + col) * c + i];
  std::vector<double> U, sg, V;
  jacobi_svd(r, R11, &U, &sg, &V);
  T.sigma = sg;
  double smax = sg.empty() ? 0.0 : sg[0];
  int rank = 0;
  if (smax > 0) {
    double tol = (double)std::max<long>(r, Np) * std::ldexp(1.0, std::ilogb(smax) - 52);
    for (int i = 0; i < r; ++i)
      if (sg[i] > tol) ++rank;
  }
  T.rank = rank;
  // Tt = V diag(1/sigma) U^T R12 (r x p), T = Tt^T (p x r)
  std::vector<double> W((size_t)rank * p, 0.0);  // W = diag(1/s) U^T R12 (rank x p)
  for (int col = 0; col < p; ++col)
    for (int i = 0; i < rank; ++i) {
      double acc = 0;
      for (int k = 0; k < r; ++k) acc += U[(size_t)i * r + k] * R12[(size_t)col * r + k];
      W[(size_t)col * rank + i] = acc / sg[i];
    }
  Tm.assign((size_t)p * r, 0.0);  // row-major p x r
  for (int a = 0; a < p; ++a)
    for (int q = 0; q < r; ++q) {
      double acc = 0;
      for (int i = 0; i < rank; ++i) acc += V[(size_t)i * r + q] * W[(size_t)a * rank + i];
      Tm[(size_t)a * r + q] = acc;
    }
  return finish_table(d, n, T, g, Tm);
}

// Q(S, gamma) = [I, -T] and C(S, gamma) = Q(S, gamma) G(gamma, gamma) from T (row-major
// p x r over (S, beta)).
static int finish_table(int d, int n, StencilTable& T, const std::vector<double>& g,
                        const std::vector<double>& Tm) {
  const int p = T.nS, r = T.nB;
  // Q(S, gamma) = [I, -T] on (S, beta), placed in gamma order
  T.Q.assign((size_t)p * T.nG, 0.0);
  {
    int sidx = 0, bidx = 0;
    for (int gi = 0; gi < T.nG; ++gi) {
      bool inS = false;
      // gamma order lists S and beta points in the same relative order
      if (sidx < p) {
        bool eq = true;
        for (int a = 0; a < d; ++a)
          if (T.G[(size_t)gi * d + a] != T.S[(size_t)sidx * d + a]) eq = false;
        inS = eq;
      }
      if (inS) {
        T.Q[(size_t)sidx * T.nG + gi] = 1.0;
        ++sidx;
      } else {
        for (int a = 0; a < p; ++a) T.Q[(size_t)a * T.nG + gi] = -Tm[(size_t)a * r + bidx];
        ++bidx;
      }
    }
    if (sidx != p || bidx != r) return 2;
  }
  // C(S, gamma) = Q(S, gamma) G(gamma, gamma)
  std::vector<double> Ggg((size_t)T.nG * T.nG);
  for (int i = 0; i < T.nG; ++i)
    for (int j = 0; j < T.nG; ++j) {
      int dp[3];
      for (int a = 0; a < d; ++a) dp[a] = T.G[(size_t)i * d + a] - T.G[(size_t)j * d + a];
      Ggg[(size_t)i * T.nG + j] = g[flat_of(dp, d, n)];
    }
  T.C.assign((size_t)p * T.nG, 0.0);
  for (int a = 0; a < p; ++a)
    for (int i = 0; i < T.nG; ++i) {
      double qa = T.Q[(size_t)a * T.nG + i];
      if (qa == 0.0) continue;
      const double* gr = &Ggg[(size_t)i * T.nG];
      double* cr = &T.C[(size_t)a * T.nG];
      for (int j = 0; j < T.nG; ++j) cr[j] += qa * gr[j];
    }
  return 0;
}

int stencil_table(int d, int n, int b, int t, const std::vector<double>& g, int threads,
                  StencilTable* out, const std::vector<double>* g2, int kind) {
  StencilTable& T = *out;
  T.t = t;
  set_geometry(d, b, t, &T.S, &T.G, &T.Bt);
  if (kind == 0) return set_table(d, n, T, g, threads, g2);
  // per-point stencils: the table of the single point 0 (S = {0}, gamma its 3^d
  // neighbours, axis 0 fastest), the same for every point by translation
  // invariance; row a of the type's table carries it on the columns
  // gamma({S_a}) of gamma(S) and is zero elsewhere
  StencilTable P;
  P.t = -1;
  {
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, glo[3] = {-1, -1, -1}, ghi[3] = {1, 1, 1};
    P.S = box_points(d, lo, hi);
    P.G = box_points(d, glo, ghi);
    const int nG = (int)P.G.size() / d;
    for (int i = 0; i < nG; ++i) {
      bool zero = true;
      for (int a = 0; a < d; ++a)
        if (P.G[(size_t)i * d + a] != 0) zero = false;
      if (!zero)
        for (int a = 0; a < d; ++a) P.Bt.push_back(P.G[(size_t)i * d + a]);
    }
  }
  int e = set_table(d, n, P, g, threads, g2);
  if (e) return e;
  T.nS = (int)T.S.size() / d;
  T.nG = (int)T.G.size() / d;
  T.nB = (int)T.Bt.size() / d;
  T.rank = P.rank;
  T.sigma = P.sigma;
  T.Q.assign((size_t)T.nS * T.nG, 0.0);
  T.C.assign((size_t)T.nS * T.nG, 0.0);
  for (int a = 0; a < T.nS; ++a)
    for (int ie = 0; ie < P.nG; ++ie) {
      int c = -1;
      for (int cc = 0; cc < T.nG && c < 0; ++cc) {
        bool eq = true;
        for (int ax = 0; ax < d; ++ax)
          if (T.G[(size_t)cc * d + ax] != T.S[(size_t)a * d + ax] + P.G[(size_t)ie * d + ax])
            eq = false;
        if (eq) c = cc;
      }
      if (c < 0) return 5;  // gamma({S_a}) lies inside gamma(S) by construction
      T.Q[(size_t)a * T.nG + c] = P.Q[ie];
      T.C[(size_t)a * T.nG + c] = P.C[ie];
    }
  return 0;
}

int stencil_tables(int d, int n, int b, double s, int route, int kind, int threads,
                   StencilTable* out) {
  const int hw = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<double> g, g2;
  parallel_items(route == 1 ? 2 : 1, std::min(2, hw), [&](int i) {
    if (i == 0)
      g = green_kernel(d, n, s, threads);
    else
      g2 = green_kernel_sq(d, n, s, threads);
  });
  const int nt = 1 << d;
  // the Gram route computes a table on one thread, so the types run side by side; the
  // TSQR route spreads each table's row blocks over the threads, one type at a time
  std::vector<int> rc(nt, 0);
  parallel_items(nt, route == 1 ? hw : 1, [&](int t) {
    rc[t] = stencil_table(d, n, b, t, g, threads, &out[t], route == 1 ? &g2 : nullptr, kind);
  });
  for (int t = 0; t < nt; ++t)
    if (rc[t]) return rc[t];
  return 0;
}

// ---------------------------------------------------------------- symbolic ND
int front_sizes(int d, int n, int b, std::vector<int>* nf, std::vector<int>* k,
                std::vector<int>* m) {
  int L;
  if (check_grid(d, n, b, &L)) return 1;
  nf->clear();
  k->clear();
  m->clear();
  auto pw = [&](long x) {
    long r = 1;
    for (int a = 0; a < d; ++a) r *= x;
    return r;
  };
  for (int l = 0; l < L; ++l) {
    long B = (long)b << l;
    long kk = pw(B - 1) - (l == 0 ? 0 : (1L << d) * pw(B / 2 - 1));
    long mm = kk + pw(B + 1) - pw(B - 1);
    nf->push_back((int)pw(n / B));
    k->push_back((int)kk);
    m->push_back((int)mm);
  }
  long kr = pw(n) - (1L << d) * pw(n / 2 - 1);
  nf->push_back(1);
  k->push_back((int)kr);
  m->push_back((int)kr);
  return 0;
}

int build_symbolic(int d, int n, int b, const std::vector<StencilTable>& tabs, Symbolic* out) {
  int L;
  if (check_grid(d, n, b, &L)) return 1;
  Symbolic& S = *out;
  S.d = d;
  S.n = n;
  S.b = b;
  S.L = L;
  S.lv.assign(L + 1, Level());
  long N = 1;
  for (int a = 0; a < d; ++a) N *= n;
  // elimination level of every point
  std::vector<signed char> lev(N);
  for (long j = 0; j < N; ++j) {
    int pc[3];
    long jj = j;
    for (int a = 0; a < d; ++a) {
      pc[a] = (int)(jj % n);
      jj /= n;
    }
    int l = 0;
    for (; l < L; ++l) {
      int B = b << l;
      bool interior = true;
      for (int a = 0; a < d; ++a)
        if (pc[a] % B == 0) interior = false;
      if (interior) break;
    }
    lev[j] = (signed char)l;
  }
  // table offsets in the concatenated column-major tables
  std::vector<long> toff(tabs.size() + 1, 0);
  for (size_t t = 0; t < tabs.size(); ++t) toff[t + 1] = toff[t] + (long)tabs[t].nS * tabs[t].nG;

  std::vector<int> pos(N, -1);
  for (int l = 0; l <= L; ++l) {
    Level& V = S.lv[l];
    V.lev = l;
    V.B = (l < L) ? (b << l) : n;
    V.nb1 = n / V.B;
    V.nf = 1;
    for (int a = 0; a < d; ++a) V.nf *= V.nb1;
    // front unknowns of box 0: eliminated ones, then the boundary
    std::vector<int> el, bd;
    if (l < L) {
      int lo[3], hi[3];
      for (int a = 0; a < d; ++a) {
        lo[a] = 0;
        hi[a] = V.B;
      }
      std::vector<int> cl = box_points(d, lo, hi);
      int ncl = (int)cl.size() / d;
      for (int i = 0; i < ncl; ++i) {
        const int* p = &cl[(size_t)i * d];
        bool onb = false;
        for (int a = 0; a < d; ++a)
          if (p[a] == 0 || p[a] == V.B) onb = true;
        if (onb) {
          bd.insert(bd.end(), p, p + d);
        } else if (lev[flat_of(p, d, n)] == l) {
          el.insert(el.end(), p, p + d);
        }
      }
    } else {
      for (long j = 0; j < N; ++j)
        if (lev[j] == L) {
          long jj = j;
          for (int a = 0; a < d; ++a) {
            el.push_back((int)(jj % n));
            jj /= n;
          }
        }
    }
    V.k = (int)el.size() / d;
    V.m = V.k + (int)bd.size() / d;
    V.off = el;
    V.off.insert(V.off.end(), bd.begin(), bd.end());
    // global indices of every front
    V.gidx.resize((size_t)V.nf * V.m);
    for (int f = 0; f < V.nf; ++f) {
      int bc[3];
      int ff = f;
      for (int a = 0; a < d; ++a) {
        bc[a] = ff % V.nb1;
        ff /= V.nb1;
      }
      for (int v = 0; v < V.m; ++v) {
        int p[3];
        for (int a = 0; a < d; ++a) p[a] = bc[a] * V.B + V.off[(size_t)v * d + a];
        V.gidx[(size_t)f * V.m + v] = (int)flat_of(p, d, n);
      }
    }
    // position map of box 0
    for (int v = 0; v < V.m; ++v) pos[V.gidx[v]] = v;
    // assembly list: P entries (row j of set S, column i in gamma(S)) whose
    // earlier-eliminated endpoint is eliminated in box 0 of this level
    std::vector<std::array<int, 3>> origins;
    {
      int nl = n / b;  // leaf boxes per axis
      int lo = (l < L) ? -1 : 0, hi = (l < L) ? V.B / b : nl - 1;
      std::unordered_map<long, int> uniq;
      int cnt = 1;
      for (int a = 0; a < d; ++a) cnt *= (hi - lo + 1);
      for (int c = 0; c < cnt; ++c) {
        int cc = c;
        std::array<int, 3> o{0, 0, 0};
        long key = 0, sc = 1;
        bool keep = true;
        for (int a = 0; a < d; ++a) {
          int ia = lo + cc % (hi - lo + 1);
          cc /= (hi - lo + 1);
          ia = ((ia % nl) + nl) % nl;
          o[a] = ia * b;
          key += (long)ia * sc;
          sc *= nl;
        }
        if (l == L) {
          // only leaf boxes whose closure (+1 layer) touches a root plane
          keep = false;
          int h2 = n / 2;
          for (int a = 0; a < d && !keep; ++a)
            for (int v = o[a] - 1; v <= o[a] + b + 1; ++v)
              if ((((v % n) + n) % n) % h2 == 0) {
                keep = true;
                break;
              }
        }
        if (!keep) continue;
        if (uniq.count(key)) continue;
        uniq[key] = 1;
        origins.push_back(o);
      }
    }
    // a point is eliminated in box 0 of a level below the root iff all its
    // coordinates lie in [1, B-1] (at the root every point is in the one front)
    auto in_box0 = [&](long e) {
      if (l == L) return true;
      for (int ax = 0; ax < d; ++ax) {
        const int v = (int)(e % n);
        e /= n;
        if (v < 1 || v > V.B - 1) return false;
      }
      return true;
    };
    // per (type, leaf box): flat index, level and box-0 test of every set point and
    // every gamma point, once; the (row, column) scan then compares levels only.  A
    // row eliminated below this level gives no entry here (the earlier endpoint of
    // each of its entries is eliminated earlier).
    std::vector<long> jf, cf;
    std::vector<signed char> jl, cl;
    std::vector<char> cin;
    for (size_t t = 0; t < tabs.size(); ++t) {
      const StencilTable& tb = tabs[t];
      jf.resize(tb.nS);
      jl.resize(tb.nS);
      cf.resize(tb.nG);
      cl.resize(tb.nG);
      cin.resize(tb.nG);
      for (const auto& o : origins) {
        bool any = false;
        for (int a = 0; a < tb.nS; ++a) {
          int pj[3];
          for (int ax = 0; ax < d; ++ax) pj[ax] = o[ax] + tb.S[(size_t)a * d + ax];
          jf[a] = flat_of(pj, d, n);
          jl[a] = lev[jf[a]];
          any |= jl[a] >= l;
        }
        if (!any) continue;
        for (int c = 0; c < tb.nG; ++c) {
          int pi[3];
          for (int ax = 0; ax < d; ++ax) pi[ax] = o[ax] + tb.G[(size_t)c * d + ax];
          cf[c] = flat_of(pi, d, n);
          cl[c] = lev[cf[c]];
          cin[c] = in_box0(cf[c]);
        }
        for (int a = 0; a < tb.nS; ++a) {
          const int lj = jl[a];
          if (lj < l) continue;
          const bool jin = in_box0(jf[a]);
          for (int c = 0; c < tb.nG; ++c) {
            const int li = cl[c];
            if (std::min(lj, li) != l) continue;
            // the earlier-eliminated endpoint (the row on ties) must be in box 0
            if (!(lj <= li ? jin : cin[c])) continue;
            const int rp = pos[jf[a]], cp = pos[cf[c]];
            if (rp < 0 || cp < 0) return 3;  // structural error
            V.asm_row.push_back(rp);
            V.asm_tidx.push_back((int)(toff[t] + a + (long)c * tb.nS));
            V.asm_cvar.push_back(cp);
          }
        }
      }
    }
    // extend-add maps from the children (level l-1)
    if (l >= 1) {
      const Level& C = S.lv[l - 1];
      V.mc = C.m;
      V.kc = C.k;
      int nbd = C.m - C.k;
      V.ea_map.assign((size_t)(1 << d) * nbd, -1);
      int half = C.B;
      for (int dl = 0; dl < (1 << d); ++dl)
        for (int v = 0; v < nbd; ++v) {
          int p[3];
          for (int a = 0; a < d; ++a) p[a] = ((dl >> a) & 1) * half + C.off[(size_t)(C.k + v) * d + a];
          int pp = pos[flat_of(p, d, n)];
          if (pp < 0) return 4;
          V.ea_map[(size_t)dl * nbd + v] = pp;
        }
    }
    // clear the position map
    for (int v = 0; v < V.m; ++v) pos[V.gidx[v]] = -1;
  }
  return 0;
}

int setup_host(int d, int n, int b, int P, const double* shifts, int route, int kind,
               int threads, std::vector<StencilTable>* tabs, Symbolic* sym) {
  // the symbolic structure reads the sets' geometry only, so it is built from
  // geometry-only tables while the tables themselves are computed
  std::vector<StencilTable> geo((size_t)1 << d);
  for (int t = 0; t < (1 << d); ++t) {
    StencilTable& T = geo[t];
    T.t = t;
    set_geometry(d, b, t, &T.S, &T.G, &T.Bt);
    T.nS = (int)T.S.size() / d;
    T.nG = (int)T.G.size() / d;
    T.nB = (int)T.Bt.size() / d;
  }
  tabs->assign((size_t)P << d, StencilTable());
  const int hw = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
  int rs = 0, rt = 0;
  parallel_items(2, std::min(2, hw), [&](int i) {
    if (i == 0) {
      rs = build_symbolic(d, n, b, geo, sym);
      return;
    }
    for (int p = 0; p < P && !rt; ++p)
      rt = stencil_tables(d, n, b, shifts[p], route, kind, threads, tabs->data() + ((size_t)p << d));
  });
  return rt ? rt : rs;
}

}  // namespace sp
