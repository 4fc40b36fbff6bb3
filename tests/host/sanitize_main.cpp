// Host-only driver for the sanitizer test: runs the set-up code of the library
// (Green's kernels, stencil tables by both routes and both stencil kinds, the
// nested-dissection structure, front sizes) on small grids of one and several
// problems, so that AddressSanitizer and UndefinedBehaviorSanitizer see every
// host code path of the set-up, its worker threads included.  No CUDA.
#include <cmath>
#include <cstdio>
#include <vector>

#include "sp_host.h"

int main() {
  using namespace sp;
  const double pi = 3.141592653589793;
  const int cfg[][3] = {{2, 16, 2}, {2, 24, 3}, {2, 32, 4}, {3, 8, 2}, {3, 12, 3}};
  int bad = 0;
  for (const auto& c : cfg) {
    const int d = c[0], n = c[1], b = c[2];
    const double s = d == 2 ? 4 * pi * pi * (n / 8.0) * (n / 8.0) * 1.0137 : 4 * pi * pi * 1.37;
    for (int route = 0; route < 2; ++route)
      for (int kind = 0; kind < 2; ++kind)
        for (int P = 1; P <= 2; ++P) {
          const double shifts[2] = {s, s * 1.01};
          std::vector<StencilTable> tabs;
          Symbolic sym;
          const int rc = setup_host(d, n, b, P, shifts, route, kind, route ? 0 : 3, &tabs, &sym);
          std::vector<int> nf, k, m;
          const int rf = front_sizes(d, n, b, &nf, &k, &m);
          const bool ok = rc == 0 && rf == 0 && tabs.size() == ((size_t)P << d) &&
                          sym.lv.size() == nf.size();
          if (!ok) ++bad;
          std::printf("d %d n %d b %d route %d kind %d P %d: %s\n", d, n, b, route, kind, P,
                      ok ? "ok" : "FAILED");
        }
  }
  return bad ? 1 : 0;
}
