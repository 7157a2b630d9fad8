// Issue cost of FP64 instructions by active-lane count and kind, against FP32
// FMA: 16 warps per SM run independent register-only loops in which only the
// first `active` lanes of each warp take part; each line reports the SM cycles
// one warp instruction occupies.  The only memory write is one double per
// thread into an array of grid * block elements.
#include <cstdio>
#include <cuda_runtime.h>

template <int KIND>
__global__ void probe(double* out, int iters, int active) {
  const int lane = threadIdx.x & 31;
  double a = 1.0 + threadIdx.x * 1e-7, b = 0.999999, c = 1e-9, d = 0.5;
  float f = 0.0f;
  if (lane < active) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (KIND == 0) {        // independent DFMA chains
          a = fma(a, b, c);
          d = fma(d, b, c);
        } else if (KIND == 1) { // compare + min (DSETP / DMNMX)
          a = fmin(a, d + 0.0);
          d = fmax(d, a * 1.0);
        } else if (KIND == 2) { // FP64 -> FP32 -> FP64 conversions
          f += (float)a;
          a = (double)f * b;
        } else if (KIND == 3) { // division
          a = c / a + 1.0;
        } else if (KIND == 4) { // square root
          a = sqrt(a) + 1.0;
        } else {                // FP32 FMA for comparison
          f = fmaf(f, 0.999f, 1e-3f);
        }
      }
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a + d + f;
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int block = 128, grid = sms * 4;  // 16 warps per SM
  double* out = nullptr;
  cudaMalloc(&out, sizeof(double) * grid * block);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const char* names[] = {"dfma x2", "dmin/dmax", "f64<->f32 cvt", "ddiv", "dsqrt", "ffma"};
  const int iters_for[] = {200, 200, 200, 20, 20, 2000};
  for (int kind = 0; kind < 6; ++kind) {
    for (int active : {32, 12, 4, 1}) {
      void (*k)(double*, int, int) = kind == 0 ? probe<0> : kind == 1 ? probe<1> : kind == 2 ? probe<2>
                                     : kind == 3 ? probe<3> : kind == 4 ? probe<4> : probe<5>;
      int iters = iters_for[kind];
      k<<<grid, block>>>(out, iters, active);  // warm-up
      cudaEventRecord(e0);
      k<<<grid, block>>>(out, iters, active);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      double warp_insts = (double)grid * (block / 32) * iters * 8 * (kind == 0 ? 2 : 1);
      double cycles = ms * 1e-3 * 2.07e9;
      printf("%-14s active %2d: %8.3f ms, %.2f SM-cycles per warp-op (per SM), %.3f lane-ops/clk/SM\n",
             names[kind], active, ms, cycles * sms / warp_insts,
             warp_insts * active / (cycles * sms));
    }
  }
  cudaError_t err = cudaGetLastError();
  printf("status: %s\n", cudaGetErrorString(err));
  cudaFree(out);
  return err == cudaSuccess ? 0 : 1;
}
