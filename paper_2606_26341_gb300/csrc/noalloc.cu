// bipm_solve_static: a one-shot batched solve that allocates no memory.
//
// Some callers cannot allocate device memory at the time they need a solve:
// code running inside a CUDA stream capture (where cudaMalloc is not allowed),
// real-time control loops that must not enter the allocator, and hosts whose
// memory budget is fixed up front.  This entry point serves them: its whole
// workspace (slot vectors, derivative blocks, factors, parameters, states and
// the launch record) lives in one file-scope __device__ array of fixed size,
// reserved when the library is loaded and held by every GPU that loads it
// until the process exits.  The caller passes device inputs and outputs only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/bipm.h"
#include "kernels.cuh"

using namespace bipm;

namespace bipm {
void set_last_error(const std::string& msg);  // defined with the other entry points
}

namespace {

// 64 MiB: enough slots for the small NMPC problems this path is meant for
// (a few hundred single-quadrotor problems of horizon 10 at once); larger
// problems get fewer slots, problems needing more than the whole array are
// rejected.
constexpr size_t kStaticBytes = 64u << 20;
static __device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ws_ptr[kMaxDevices] = {nullptr};

int sfail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// device address of the static workspace on the current device (set up once
// per device, with that device current)
int workspace_ptr(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return sfail(BIPM_ECUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return sfail(BIPM_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ws_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess || !p)
      return sfail(BIPM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_ws_ptr[dev] = (unsigned char*)p;
  }
  *out = g_ws_ptr[dev];
  return 0;
}

}  // namespace

extern "C" {

int bipm_solve_static(const bipm_problem_desc* desc, const bipm_options* opt, const double* theta,
                      int count, double* x_out, bipm_result* results, void* cuda_stream) {
  if (!desc || !theta || !results) return sfail(BIPM_EINVAL, "null desc, theta or results");
  if (count < 0) return sfail(BIPM_EINVAL, "count must be >= 0");
  if (desc->n_quads < 1 || desc->n_quads > 8) return sfail(BIPM_EINVAL, "n_quads must be 1..8");
  if (desc->horizon < 1 || desc->horizon > 1000) return sfail(BIPM_EINVAL, "horizon must be 1..1000");
  if (!(desc->dt > 0.0) || !std::isfinite(desc->dt)) return sfail(BIPM_EINVAL, "dt must be > 0");
  if (desc->n_spheres < 0 || desc->n_cylinders < 0 || desc->n_spheres > 256 || desc->n_cylinders > 256)
    return sfail(BIPM_EINVAL, "obstacle counts must be 0..256");
  if (!(desc->pair_dist >= 0.0)) return sfail(BIPM_EINVAL, "pair_dist must be >= 0");
  bipm_options o = opt ? *opt : bipm_options{1e-6, 500, 0.1, 0, 0, 0.0};
  if (!(o.tol > 0.0) || o.max_iter < 0 || !(o.mu_init > 0.0) || o.precision < 0 || o.precision > 2)
    return sfail(BIPM_EINVAL, "bad options");
  if (o.fp32_switch == 0.0) o.fp32_switch = kFp32BarrierMax;
  if (count == 0) return 0;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  Dims d;
  std::memset(&d, 0, sizeof(d));
  d.nq = desc->n_quads;
  d.N = desc->horizon;
  d.nx = 12 * d.nq;
  d.nu = 4 * d.nq;
  d.n_sph = desc->n_spheres;
  d.n_cyl = desc->n_cylinders;
  d.n_pairs = desc->pair_dist > 0.0 ? d.nq * (d.nq - 1) / 2 : 0;
  d.ni = d.nq * d.n_sph + d.nq * d.n_cyl + d.n_pairs;
  d.n = d.nx * (d.N + 1) + (d.nu + d.ni) * d.N;
  d.m = d.nx * (d.N + 1) + d.ni * d.N;
  d.dt = desc->dt;
  d.pair_d = desc->pair_dist;
  d.th_x = 0;
  d.th_ref = 12 * d.nq;
  d.th_sph = d.th_ref + 6 * d.nq;
  d.th_cyl = d.th_sph + 4 * d.n_sph;
  d.n_theta = d.th_cyl + 3 * d.n_cyl;
  const Layout L = make_layout(d, o.precision);
  const size_t tsz = o.precision ? sizeof(float) : sizeof(double);
  const size_t fsz = o.precision == 1 ? sizeof(float) : sizeof(double);

  // carve the static array: launch record and counter, then per-slot regions
  const size_t hdr = align256(sizeof(Params)) + 256;
  const size_t per_slot = align256(L.slot_f64 * sizeof(double)) + align256(L.slot_tb * tsz) +
                          align256(L.fac_size * fsz) + align256(d.n_theta * sizeof(double)) +
                          align256(sizeof(SlotState));
  if (hdr + per_slot > kStaticBytes)
    return sfail(BIPM_EINVAL, "problem too large for the static workspace: one problem needs " +
                                  std::to_string(hdr + per_slot) + " bytes, the workspace holds " +
                                  std::to_string(kStaticBytes));
  int fit = (int)((kStaticBytes - hdr) / per_slot);

  unsigned char* base = nullptr;
  int rc = workspace_ptr(&base);
  if (rc) return rc;

  // one slot per resident warp, at most one per problem and per what fits
  void* kfn = o.precision == 2 ? queue_kernel_df() : o.precision ? queue_kernel_f32() : queue_kernel_f64();
  int smem_per_warp;
  {
    size_t need = scratch_bytes(d.nq, d.nx, d.nu, o.precision == 1 ? 4 : 8);
    size_t need64 = scratch_bytes(d.nq, d.nx, d.nu, 8);
    size_t cap_b = 24 * 1024;
    smem_per_warp = (int)(need64 <= cap_b ? need64 : (need <= cap_b ? need : 128));
  }
  size_t smem = (size_t)smem_per_warp * kWarpsPerBlock;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return sfail(BIPM_ECUDA, "shared memory attribute");
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * kWarpsPerBlock, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return sfail(BIPM_ECUDA, "kernel does not fit on an SM");
  const int slots = std::max(1, std::min({fit, count, sms * per_sm * kWarpsPerBlock}));

  unsigned char* p = base + hdr;
  Params P;
  std::memset(&P, 0, sizeof(P));
  P.d = d;
  P.L = L;
  P.opt.tol = o.tol;
  P.opt.max_iter = o.max_iter;
  P.opt.mu_init = o.mu_init;
  P.opt.precision = o.precision;
  P.opt.fp32_switch = o.fp32_switch;
  P.n_slots = slots;
  P.f64 = (double*)p;
  p += align256(L.slot_f64 * sizeof(double)) * slots;
  P.tb = p;
  p += align256(L.slot_tb * tsz) * slots;
  P.tf = p;
  p += align256(L.fac_size * fsz) * slots;
  P.theta = (double*)p;
  p += align256(d.n_theta * sizeof(double)) * slots;
  P.st = (SlotState*)p;
  P.work_counter = (int*)(base + align256(sizeof(Params)));
  P.smem_per_warp = smem_per_warp;
  // every call shares the array and finds the previous call's contents in it:
  // the queue counter must start at zero; slots are fully reset per problem
  if (cudaMemcpyAsync(base, &P, sizeof(P), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemsetAsync(P.work_counter, 0, sizeof(int), stream) != cudaSuccess)
    return sfail(BIPM_ECUDA, "launch record copy");
  const Params* dP = (const Params*)base;
  int n_queue = count;
  int n_warps = slots;
  int blocks = (slots + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const double* no_guess = nullptr;
  void* args[] = {&dP, &theta, &n_queue, &n_warps, &x_out, &results, &no_guess};
  cudaError_t e = cudaLaunchKernel(kfn, dim3(blocks), dim3(32 * kWarpsPerBlock), args, smem, stream);
  if (e != cudaSuccess) return sfail(BIPM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return sfail(BIPM_ECUDA, std::string("solve: ") + cudaGetErrorString(e));
  return 0;
}

}  // extern "C"
