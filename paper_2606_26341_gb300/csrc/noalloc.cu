// bipm_solve_static: a one-shot batched solve that allocates no memory.
//
// Some callers cannot allocate device memory at the time they need a solve:
// real-time control loops that must stay out of the CUDA allocator (cudaMalloc
// can block, synchronise the device or fail under fragmentation), and
// processes whose device memory is budgeted at start-up and may not grow.
// This entry point serves them: its whole workspace (slot vectors, derivative
// blocks, factors, parameters, states, counters and the launch record) lives
// in one file-scope __device__ array of fixed size, reserved when the library
// is loaded and held by every GPU that loads it until the process exits.  The
// caller passes device inputs and outputs only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/bipm.h"
#include "host_api.h"
#include "kernels.cuh"

using namespace bipm;

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
  Dims d;
  int rc = dims_from_desc(desc, &d);  // the same validation as bipm_create_batch
  if (rc) return rc;
  bipm_options o;
  Options dopt;
  if ((rc = options_from(opt, &o, &dopt))) return rc;
  if (count == 0) return 0;
  cudaStream_t stream = (cudaStream_t)cuda_stream;

  const Layout L = make_layout(d, o.precision);
  const size_t tsz = o.precision ? sizeof(float) : sizeof(double);
  const size_t fsz = o.precision == 1 ? sizeof(float) : sizeof(double);

  // carve the static array: launch record and counters, then per-slot regions
  const size_t hdr = align256(sizeof(Params)) + align256(kCounterInts * sizeof(int));
  const size_t per_slot = align256(L.slot_f64 * sizeof(double)) + align256(L.slot_tb * tsz) +
                          align256(L.fac_size * fsz) + align256(d.n_theta * sizeof(double)) +
                          align256(sizeof(SlotState));
  if (hdr + per_slot > kStaticBytes)
    return sfail(BIPM_EINVAL, "problem too large for the static workspace: one problem needs " +
                                  std::to_string(hdr + per_slot) + " bytes, the workspace holds " +
                                  std::to_string(kStaticBytes));
  int fit = (int)((kStaticBytes - hdr) / per_slot);

  unsigned char* base = nullptr;
  if ((rc = workspace_ptr(&base))) return rc;

  // one slot per resident warp, at most one per problem and per what fits
  void* kfn = queue_kernel_ptr(o.precision, d.nq);
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
  per_sm = std::min(per_sm, o.warps_per_sm / kWarpsPerBlock);
  const int slots = std::max(1, std::min({fit, count, sms * per_sm * kWarpsPerBlock}));

  unsigned char* p = base + hdr;
  Params P;
  std::memset(&P, 0, sizeof(P));
  P.d = d;
  P.L = L;
  P.opt = dopt;
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
  int* counter = (int*)(base + align256(sizeof(Params)));
  P.work_counter = counter;
  P.smem_per_warp = smem_per_warp;
  // one slot per warp and no spare slots: a problem is never parked, so the
  // spare counter is never touched and the visit is unlimited
  P.spare_counter = counter + 1;
  P.n_spare = 0;
  P.visit_cap = 0;
  set_budget(P, counter, o.time_limit_ms);
  // every call shares the array and finds the previous call's contents in it:
  // the counters must start at zero; slots are fully reset per problem
  if (cudaMemcpyAsync(base, &P, sizeof(P), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemsetAsync(counter, 0, kCounterInts * sizeof(int), stream) != cudaSuccess)
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
  if (o.time_limit_ms > 0) {
    int flag = 0;
    e = cudaMemcpy(&flag, counter + 2, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sfail(BIPM_ECUDA, std::string("flag read: ") + cudaGetErrorString(e));
    if (flag)
      return sfail(BIPM_ETIMEOUT, "time limit of " + std::to_string(o.time_limit_ms) +
                                      " ms reached: unfinished problems report RUNNING or EMPTY");
  }
  return 0;
}

}  // extern "C"
