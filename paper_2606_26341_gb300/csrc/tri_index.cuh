// Index arithmetic of the lower-triangle passes of the Riccati recursion
// (row-major lower triangles, and the rows of one kind of every quadrotor
// block); host and device.
#pragma once

#include <math.h>

#include "scalar.cuh"

namespace bipm {

// (i, j), j <= i, of entry e of a row-major lower triangle (e = i (i + 1) / 2 + j)
__host__ __device__ __forceinline__ void tri_index(int e, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > e) --r;
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  i = r;
  j = e - r * (r + 1) / 2;
}

// Lower-triangle entries (i, j), j <= i, of the rows 12 q + r0 .. 12 q + r0 + 5
// of every quadrotor block q of an nx x nx matrix: their count, and entry f in
// row-major order
template <class D>
__host__ __device__ __forceinline__ int tri_rows_count(const D& d, int r0) {
  int n = 0;
  for (int q = 0; q < d.nq; ++q) {
    const int a = 12 * q + r0;
    n += (a + 6) * (a + 7) / 2 - a * (a + 1) / 2;
  }
  return n;
}
template <class D>
__host__ __device__ __forceinline__ void tri_rows_entry(const D& d, int f, int r0, int& i, int& j) {
  int q = 0;
  for (; q + 1 < d.nq; ++q) {
    const int a = 12 * q + r0, cnt = (a + 6) * (a + 7) / 2 - a * (a + 1) / 2;
    if (f < cnt) break;
    f -= cnt;
  }
  const int a = 12 * q + r0;
  tri_index(a * (a + 1) / 2 + f, i, j);
}

}  // namespace bipm
