// Warm-start encodings on the GPU: network input features from a problem's
// parameters, training targets from a solved trajectory, and the primal
// starting point decoded from a network output.
//
// Defined for the cluttered-environment family (one quadrotor, vertical
// cylinders, a fixed goal):
//   features  (p0 - goal)/10, v0/2, eta0, omega0/2, then for the k_near
//             cylinders nearest to p0 (horizontal centre distance, ties by
//             index) (cx - p0x)/10, (cy - p0y)/10, r; zeros past 30 m or past
//             the cylinder count
//   targets   (x_k - xbar)/S, S = (2,2,2, 2,2,2, .5,.5,.5, 2,2,2), k = 0..N,
//             then (u_k - u_hover)/u_hover, k = 0..N-1
//   decoding  inverse map for k >= 1, x_0 = xbar, slacks = g(x_k)
// Distances and inequality values are formed without fused multiply-adds so
// that rankings and values are reproducible bit for bit.
#include <cuda_runtime.h>

#include <string>

#include "../../include/bipm.h"
#include "common.cuh"

namespace bipm {
void set_last_error(const std::string& msg);
}

using namespace bipm;

namespace {

constexpr double kPosScale = 10.0, kVelScale = 2.0, kRateScale = 2.0, kCutoff = 30.0;

__device__ __forceinline__ double state_scale(int i) { return (i >= 6 && i < 9) ? 0.5 : 2.0; }

int fail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

int warm_dims(const bipm_problem_desc* desc, Dims* d) {
  if (!desc) return fail(BIPM_EINVAL, "null problem description");
  if (desc->n_quads != 1 || desc->n_spheres != 0 || desc->pair_dist > 0.0 || desc->n_moving != 0)
    return fail(BIPM_EINVAL, "the warm start is defined for one quadrotor among cylinders "
                             "(n_quads = 1, n_spheres = 0, n_moving = 0, pair_dist = 0)");
  if (desc->horizon < 1 || desc->horizon > 1000 || desc->n_cylinders < 0 || desc->n_cylinders > 256)
    return fail(BIPM_EINVAL, "horizon must be 1..1000 and n_cylinders 0..256");
  Dims& r = *d;
  r.nq = 1;
  r.N = desc->horizon;
  r.nx = 12;
  r.nu = 4;
  r.n_sph = 0;
  r.n_cyl = desc->n_cylinders;
  r.n_pairs = 0;
  r.n_mov = 0;
  r.ni = r.n_cyl;
  r.n = r.nx * (r.N + 1) + (r.nu + r.ni) * r.N;
  r.m = r.nx * (r.N + 1) + r.ni * r.N;
  r.dt = desc->dt;
  r.pair_d = 0.0;
  r.th_x = 0;
  r.th_ref = 12;
  r.th_sph = 18;
  r.th_cyl = 18;
  r.th_mov = 18 + 3 * r.n_cyl;
  r.n_theta = 18 + 3 * r.n_cyl;
  return 0;
}

__device__ __forceinline__ double sq_dist2(double dx, double dy) {
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// one warp per problem
__global__ void features_kernel(Dims d, const double* __restrict__ theta, int count, int k_near,
                                float* __restrict__ feat) {
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= count) return;
  const double* th = theta + (long long)p * d.n_theta;
  const int F = 12 + 3 * k_near;
  float* out = feat + (long long)p * F;
  const double px = th[0], py = th[1];
  if (lane < 12) {
    double v = th[lane];
    if (lane < 3) v = (v - th[d.th_ref + lane]) / kPosScale;
    else if (lane < 6) v = v / kVelScale;
    else if (lane >= 9) v = v / kRateScale;
    out[lane] = (float)v;
  }
  for (int i = lane; i < 3 * k_near; i += 32) out[12 + i] = 0.0f;
  __syncwarp();
  const double* cyl = th + d.th_cyl;
  for (int j = lane; j < d.n_cyl; j += 32) {
    const double dj = sq_dist2(cyl[3 * j] - px, cyl[3 * j + 1] - py);
    int rank = 0;
    for (int i = 0; i < d.n_cyl; ++i) {
      const double di = sq_dist2(cyl[3 * i] - px, cyl[3 * i + 1] - py);
      rank += (di < dj) || (di == dj && i < j);
    }
    if (rank < k_near && sqrt(dj) <= kCutoff) {
      out[12 + 3 * rank] = (float)((cyl[3 * j] - px) / kPosScale);
      out[13 + 3 * rank] = (float)((cyl[3 * j + 1] - py) / kPosScale);
      out[14 + 3 * rank] = (float)cyl[3 * j + 2];
    }
  }
}

// one thread per target entry
__global__ void encode_kernel(Dims d, const double* __restrict__ theta, const double* __restrict__ x, int count,
                              float* __restrict__ target) {
  const int P = 12 * (d.N + 1) + 4 * d.N;
  const long long total = (long long)count * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / P), o = (int)(e - (long long)p * P);
    const double* th = theta + (long long)p * d.n_theta;
    const double* xp = x + (long long)p * d.n;
    double v;
    if (o < 12 * (d.N + 1)) {
      const int k = o / 12, i = o - 12 * k;
      v = (xp[off_x(d, k) + i] - th[i]) / state_scale(i);
    } else {
      const int q = o - 12 * (d.N + 1), k = q / 4, a = q - 4 * k;
      v = (xp[off_u(d, k) + a] - kHover) / kHover;
    }
    target[e] = (float)v;
  }
}

// one thread per primal entry
__global__ void decode_kernel(Dims d, const double* __restrict__ theta, const float* __restrict__ net,
                              int count, double* __restrict__ xg) {
  const int P = 12 * (d.N + 1) + 4 * d.N;
  const long long total = (long long)count * d.n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / d.n), i = (int)(e - (long long)p * d.n);
    const double* th = theta + (long long)p * d.n_theta;
    const float* o = net + (long long)p * P;
    // locate entry i: stage k, offset inside the stage block
    int k, loc;
    if (i < d.nx + d.nu) {
      k = 0;
      loc = i;
    } else {
      const int blk = d.nx + d.nu + d.ni;
      k = 1 + (i - (d.nx + d.nu)) / blk;
      loc = (i - (d.nx + d.nu)) - (k - 1) * blk;
    }
    double v;
    if (loc < 12) {
      v = k == 0 ? th[loc] : th[loc] + state_scale(loc) * (double)o[12 * k + loc];
    } else if (k < d.N && loc < 16) {
      v = kHover * (1.0 + (double)o[12 * (d.N + 1) + 4 * k + (loc - 12)]);
    } else {
      // slack of cylinder j at the decoded position of stage k (k >= 1)
      const int j = loc - (k < d.N ? 16 : 12);
      const double pxk = th[0] + 2.0 * (double)o[12 * k];
      const double pyk = th[1] + 2.0 * (double)o[12 * k + 1];
      const double* c = th + d.th_cyl + 3 * j;
      v = __dsub_rn(sq_dist2(pxk - c[0], pyk - c[1]), __dmul_rn(c[2], c[2]));
    }
    xg[e] = v;
  }
}

int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152LL * 32 ? 152LL * 32 : b));
}

int launched(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(BIPM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return 0;
}

}  // namespace

extern "C" {

int bipm_warm_features(const bipm_problem_desc* desc, const double* theta, int count, int k_near,
                       float* features, void* cuda_stream) {
  Dims d;
  int rc = warm_dims(desc, &d);
  if (rc) return rc;
  if (count < 0 || k_near < 0 || k_near > 256) return fail(BIPM_EINVAL, "count >= 0 and k_near in 0..256");
  if (count == 0) return 0;
  if (!theta || !features) return fail(BIPM_EINVAL, "null theta or features");
  const int threads = 128;
  const int blocks = (int)(((long long)count * 32 + threads - 1) / threads);
  features_kernel<<<blocks, threads, 0, (cudaStream_t)cuda_stream>>>(d, theta, count, k_near, features);
  return launched("features kernel");
}

int bipm_warm_encode(const bipm_problem_desc* desc, const double* theta, const double* x, int count,
                     float* targets, void* cuda_stream) {
  Dims d;
  int rc = warm_dims(desc, &d);
  if (rc) return rc;
  if (count < 0) return fail(BIPM_EINVAL, "count must be >= 0");
  if (count == 0) return 0;
  if (!theta || !x || !targets) return fail(BIPM_EINVAL, "null theta, x or targets");
  long long total = (long long)count * (12 * (d.N + 1) + 4 * d.N);
  encode_kernel<<<blocks_for(total, 256), 256, 0, (cudaStream_t)cuda_stream>>>(d, theta, x, count, targets);
  return launched("encode kernel");
}

int bipm_warm_decode(const bipm_problem_desc* desc, const double* theta, const float* net_out, int count,
                     double* x_guess, void* cuda_stream) {
  Dims d;
  int rc = warm_dims(desc, &d);
  if (rc) return rc;
  if (count < 0) return fail(BIPM_EINVAL, "count must be >= 0");
  if (count == 0) return 0;
  if (!theta || !net_out || !x_guess) return fail(BIPM_EINVAL, "null theta, net_out or x_guess");
  long long total = (long long)count * d.n;
  decode_kernel<<<blocks_for(total, 256), 256, 0, (cudaStream_t)cuda_stream>>>(d, theta, net_out, count,
                                                                              x_guess);
  return launched("decode kernel");
}

}  // extern "C"
