// Host check of the factorisation's lower-triangle index arithmetic
// (csrc/tri_index.cuh, compiled for the host): for 1..8 quadrotors, the
// row-major triangle decoding visits every entry (i, j <= i) once, in order,
// and the two row kinds of the Q^ passes (rows 12 q + 6 .. 12 q + 11 and rows
// 12 q .. 12 q + 5 of every block) together cover the lower triangle of the
// nx x nx block exactly once, each entry in the pass of its row's kind.
// Prints "ok" or the first failure and exits non-zero.
#include <cstdio>
#include <vector>

#include "tri_index.cuh"

namespace {
struct D {
  int nq;
};
}  // namespace

int main() {
  for (int n = 1; n <= 400; ++n) {
    int e = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= i; ++j, ++e) {
        int a, b;
        bipm::tri_index(e, a, b);
        if (a != i || b != j) {
          std::printf("tri_index(%d) = (%d, %d), expected (%d, %d)\n", e, a, b, i, j);
          return 1;
        }
      }
  }
  for (int nq = 1; nq <= 8; ++nq) {
    const D d{nq};
    const int nx = 12 * nq;
    std::vector<int> seen(nx * nx, 0);
    for (int r0 : {6, 0}) {
      const int cnt = bipm::tri_rows_count(d, r0);
      int prev = -1;
      for (int f = 0; f < cnt; ++f) {
        int i, j;
        bipm::tri_rows_entry(d, f, r0, i, j);
        const int ci = i % 12;
        const bool kind = r0 == 6 ? ci >= 6 : ci < 6;
        const int lin = i * (i + 1) / 2 + j;
        if (i < 0 || i >= nx || j < 0 || j > i || !kind || lin <= prev) {
          std::printf("nq %d r0 %d entry %d -> (%d, %d)\n", nq, r0, f, i, j);
          return 1;
        }
        prev = lin;
        ++seen[i * nx + j];
      }
    }
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < nx; ++j)
        if (seen[i * nx + j] != (j <= i ? 1 : 0)) {
          std::printf("nq %d entry (%d, %d) visited %d times\n", nq, i, j, seen[i * nx + j]);
          return 1;
        }
  }
  std::printf("ok\n");
  return 0;
}
