// Warm-start network: a tanh multilayer perceptron trained and evaluated on
// the GPU with bfloat16 tensor-core products and FP32 accumulation.
//
//   a_0 = x;  z_l = a_{l-1} W_l^T + b_l;  a_l = tanh(z_l) (hidden);  out = z_L
//   loss = 1/(2B) sum_b |out_b - t_b|^2
//
// Precision contract: every matrix-product operand (inputs, weights, hidden
// activations, back-propagated errors) is rounded to bfloat16; products
// accumulate in FP32; biases, activations kept for the derivative, the loss
// gradient, the parameter gradient and Adam's master weights and moments are
// FP32.  The products use the warp-level bf16 MMA (m16n8k16) on 64x64 tiles
// staged through shared memory; the network is a small share of a solve, so
// the tiles favour simple, bounds-checked staging over peak throughput.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bipm.h"

namespace bipm {
void set_last_error(const std::string& msg);
}

namespace {

using bf16 = __nv_bfloat16;

constexpr int kMaxLayers = 8;
constexpr int BM = 64, BN = 64, BK = 32, SK = BK + 8;  // shared row: 40 bf16 = 80 bytes
constexpr int kGemmThreads = 128;

int fail(int code, const std::string& msg) {
  bipm::set_last_error(msg);
  return code;
}

#define CUDA_TRY(expr)                                                               \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(BIPM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// ------------------------------------------------------------------ GEMM
// C(i, j) = sum_k A(i, k) B(k, j), i < M, j < N, k < K.
// A is "k-contiguous" (A(i,k) = a[i*lda + k]) or "i-contiguous" (a[k*lda + i]);
// B is "k-contiguous" (B(k,j) = b[j*ldb + k]) or "j-contiguous" (b[k*ldb + j]).
enum Epi : int {
  EPI_BIAS_TANH = 0,  // h = tanh(acc + bias): h32 and bf16(h) into o16
  EPI_BIAS = 1,       // acc + bias into o32
  EPI_TANH_GRAD = 2,  // acc * (1 - h^2), h read from h32: into o32 and bf16 into o16
  EPI_STORE = 3       // acc into o32 (split-K slice blockIdx.z at o32 + z * M * ldo32)
};

struct EpiArgs {
  const float* bias;
  float* h32;
  long long ldh;
  float* o32;
  long long ldo32;
  bf16* o16;
  long long ldo16;
};

template <bool KCONT>
__device__ __forceinline__ void load_tile(bf16 (*S)[SK], const bf16* __restrict__ g, long long ld,
                                          int r0, int rows_total, int k0, int k_end) {
  const int tid = threadIdx.x;
  if (KCONT) {
    // BM rows x BK/8 chunks of 8 consecutive k
    for (int c = tid; c < BM * (BK / 8); c += kGemmThreads) {
      int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
      int gr = r0 + r, gk = k0 + kc;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gr < rows_total) {
        const bf16* src = g + (long long)gr * ld + gk;
        if (gk + 7 < k_end && (((uintptr_t)src) & 15) == 0) {
          v = *reinterpret_cast<const uint4*>(src);
        } else {
          bf16 tmp[8];
          for (int e = 0; e < 8; ++e)
            tmp[e] = (gk + e < k_end) ? src[e] : __float2bfloat16(0.0f);
          memcpy(&v, tmp, 16);
        }
      }
      *reinterpret_cast<uint4*>(&S[r][kc]) = v;
    }
  } else {
    // BK k-rows x BM/8 chunks of 8 consecutive rows of S
    for (int c = tid; c < BK * (BM / 8); c += kGemmThreads) {
      int kk = c / (BM / 8), rc = (c % (BM / 8)) * 8;
      int gk = k0 + kk, gr = r0 + rc;
      bf16 tmp[8];
      if (gk < k_end) {
        const bf16* src = g + (long long)gk * ld + gr;
        if (gr + 7 < rows_total && (((uintptr_t)src) & 15) == 0) {
          uint4 v = *reinterpret_cast<const uint4*>(src);
          memcpy(tmp, &v, 16);
        } else {
          for (int e = 0; e < 8; ++e) tmp[e] = (gr + e < rows_total) ? src[e] : __float2bfloat16(0.0f);
        }
      } else {
        for (int e = 0; e < 8; ++e) tmp[e] = __float2bfloat16(0.0f);
      }
      for (int e = 0; e < 8; ++e) S[rc + e][kk] = tmp[e];
    }
  }
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool AK, bool BKc, int EPI>
__global__ void __launch_bounds__(kGemmThreads)
    gemm_kernel(const bf16* __restrict__ A, long long lda, const bf16* __restrict__ B, long long ldb,
                int M, int N, int K, int k_split, EpiArgs ep) {
  __shared__ __align__(16) bf16 As[BM][SK];
  __shared__ __align__(16) bf16 Bs[BN][SK];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[a][b][r] = 0.0f;

  for (int k0 = kb; k0 < ke; k0 += BK) {
    load_tile<AK>(As, A, lda, m0, M, k0, ke);
    load_tile<BKc>(Bs, B, ldb, n0, N, k0, ke);
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        int r = wm + mi * 16 + g;
        af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * t]);
        af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * t]);
        af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * t + 8]);
        af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        int c = wn + ni * 8 + g;
        bfr[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * t]);
        bfr[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int i = m0 + wm + mi * 16 + g + (r >= 2 ? 8 : 0);
        int j = n0 + wn + ni * 8 + 2 * t + (r & 1);
        if (i >= M || j >= N) continue;
        float v = acc[mi][ni][r];
        if (EPI == EPI_BIAS_TANH) {
          float h = tanhf(v + ep.bias[j]);
          ep.h32[(long long)i * ep.ldh + j] = h;
          ep.o16[(long long)i * ep.ldo16 + j] = __float2bfloat16(h);
        } else if (EPI == EPI_BIAS) {
          ep.o32[(long long)i * ep.ldo32 + j] = v + ep.bias[j];
        } else if (EPI == EPI_TANH_GRAD) {
          float h = ep.h32[(long long)i * ep.ldh + j];
          float dz = v * (1.0f - h * h);
          ep.o32[(long long)i * ep.ldo32 + j] = dz;
          ep.o16[(long long)i * ep.ldo16 + j] = __float2bfloat16(dz);
        } else {
          ep.o32[(long long)blockIdx.z * M * ep.ldo32 + (long long)i * ep.ldo32 + j] = v;
        }
      }
}

// ------------------------------------------------------- elementwise kernels
// row r of a batch: idx[r] (or r without idx) if it lies in [0, n_data); an
// index outside the data is replaced by row 0 and raises *bad
__device__ __forceinline__ long long batch_row(const int* idx, int r, int n_data, int* bad) {
  if (!idx) return r;
  const int i = idx[r];
  if (i < 0 || i >= n_data) {
    *bad = 1;
    return 0;
  }
  return i;
}

// rows of x (optionally gathered through idx) -> bf16 with leading dimension ld
__global__ void to_bf16_rows(const float* __restrict__ x, const int* __restrict__ idx, int rows, int cols,
                             int n_data, bf16* __restrict__ out, int ld, int* __restrict__ bad) {
  long long total = (long long)rows * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / ld), c = (int)(e - (long long)r * ld);
    const long long src = batch_row(idx, r, n_data, bad);
    out[e] = __float2bfloat16(c < cols ? x[src * cols + c] : 0.0f);
  }
}

// output error (out - t) / B in FP32 and bf16; per-block partial sums of the squared error
__global__ void loss_grad_kernel(const float* __restrict__ out, const float* __restrict__ t,
                                 const int* __restrict__ idx, int rows, int cols, int n_data,
                                 float* __restrict__ d32, bf16* __restrict__ d16, int ld,
                                 double* __restrict__ part, int* __restrict__ bad) {
  __shared__ double red[256];
  double acc = 0.0;
  const float inv_b = 1.0f / (float)rows;
  long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
    const long long tr = batch_row(idx, r, n_data, bad);
    float err = out[(long long)r * cols + c] - t[tr * cols + c];
    acc += (double)err * (double)err;
    float g = err * inv_b;
    d32[(long long)r * ld + c] = g;
    d16[(long long)r * ld + c] = __float2bfloat16(g);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void loss_final(const double* __restrict__ part, int n, int rows, double* __restrict__ loss) {
  __shared__ double red[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = 0.5 * red[0] / (double)rows;
}

// column sums of d32 (rows x cols, leading dimension ld) into db
__global__ void colsum_kernel(const float* __restrict__ d32, int rows, int cols, int ld, float* __restrict__ db) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int r = 0;
  for (; r + 3 < rows; r += 4) {
    a0 += d32[(long long)r * ld + c];
    a1 += d32[(long long)(r + 1) * ld + c];
    a2 += d32[(long long)(r + 2) * ld + c];
    a3 += d32[(long long)(r + 3) * ld + c];
  }
  for (; r < rows; ++r) a0 += d32[(long long)r * ld + c];
  db[c] = (a0 + a1) + (a2 + a3);
}

// sum of the split-K slices of a weight gradient (M x N, leading dimension N)
__global__ void splitk_sum(const float* __restrict__ part, int splits, long long mn, float* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn;
       e += (long long)gridDim.x * blockDim.x) {
    float a = 0.0f;
    for (int s = 0; s < splits; ++s) a += part[s * mn + e];
    out[e] = a;
  }
}

// Adam (bias-corrected moments) on the FP32 master parameters
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long long n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    float gi = g[e];
    float mi = b1 * m[e] + (1.0f - b1) * gi;
    float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    float mh = mi / c1, vh = vi / c2;
    p[e] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// master W (rows x cols, FP32) -> bf16 with leading dimension ld (zero padding)
__global__ void pack_weights(const float* __restrict__ w, int rows, int cols, bf16* __restrict__ out, int ld) {
  long long total = (long long)rows * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / ld), c = (int)(e - (long long)r * ld);
    out[e] = __float2bfloat16(c < cols ? w[(long long)r * cols + c] : 0.0f);
  }
}

int grid_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  return (int)std::max(1LL, std::min(b, 152LL * 16));
}

int pad8(int v) { return (v + 7) & ~7; }

}  // namespace

struct bipm_mlp {
  int L = 0;                 // weight layers
  int w[kMaxLayers + 1];     // widths
  int ld[kMaxLayers + 1];    // padded widths (multiples of 8)
  long long offW[kMaxLayers], offb[kMaxLayers];
  long long n_params = 0;
  int max_rows = 0;
  cudaStream_t stream = nullptr;
  float *master = nullptr, *mom1 = nullptr, *mom2 = nullptr, *grad = nullptr;
  bf16* W16[kMaxLayers] = {};
  bf16* act16[kMaxLayers] = {};  // [0] input; [l] output of hidden layer l
  float* h32[kMaxLayers] = {};   // [l] FP32 activations of hidden layer l (l >= 1)
  float* out32 = nullptr;
  float* d32[2] = {};
  bf16* d16[2] = {};
  float* splitk = nullptr;
  long long splitk_elems = 0;
  double* loss_part = nullptr;
  double* loss_dev = nullptr;
  int* bad_index = nullptr;  // set when a batch index lies outside the data
  float* xin = nullptr;      // staging of host inputs / targets
  float* tin = nullptr;
  int adam_t = 0;
  std::vector<void*> allocs;
};

namespace {

constexpr int kLossBlocks = 512;
constexpr int kMaxSplits = 32;
constexpr int kSplitChunk = 512;  // batch rows per split of a weight-gradient product

template <bool AK, bool BKc, int EPI>
cudaError_t gemm(cudaStream_t s, const bf16* A, long long lda, const bf16* B, long long ldb, int M, int N,
                 int K, int splits, const EpiArgs& ep) {
  int k_split = (K + splits - 1) / splits;
  k_split = (k_split + BK - 1) / BK * BK;
  splits = std::max(1, (K + k_split - 1) / k_split);
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
  gemm_kernel<AK, BKc, EPI><<<grid, kGemmThreads, 0, s>>>(A, lda, B, ldb, M, N, K, k_split, ep);
  return cudaGetLastError();
}

// forward pass of `rows` rows already in act16[0]
int forward_rows(bipm_mlp* n, int rows) {
  for (int l = 0; l < n->L; ++l) {
    EpiArgs ep{};
    ep.bias = n->master + n->offb[l];
    if (l < n->L - 1) {
      ep.h32 = n->h32[l + 1];
      ep.ldh = n->ld[l + 1];
      ep.o16 = n->act16[l + 1];
      ep.ldo16 = n->ld[l + 1];
      CUDA_TRY((gemm<true, true, EPI_BIAS_TANH>(n->stream, n->act16[l], n->ld[l], n->W16[l], n->ld[l], rows,
                                                n->w[l + 1], n->w[l], 1, ep)));
    } else {
      ep.o32 = n->out32;
      ep.ldo32 = n->w[l + 1];
      CUDA_TRY((gemm<true, true, EPI_BIAS>(n->stream, n->act16[l], n->ld[l], n->W16[l], n->ld[l], rows,
                                           n->w[l + 1], n->w[l], 1, ep)));
    }
  }
  return 0;
}

// loss, gradient into n->grad (needs act16[0] filled); t rows selected by idx
int backward_rows(bipm_mlp* n, const float* t, const int* idx, int rows, int n_data) {
  const int L = n->L;
  int cur = 0;
  loss_grad_kernel<<<kLossBlocks, 256, 0, n->stream>>>(n->out32, t, idx, rows, n->w[L], n_data, n->d32[cur],
                                                       n->d16[cur], n->ld[L], n->loss_part, n->bad_index);
  CUDA_TRY(cudaGetLastError());
  loss_final<<<1, 256, 0, n->stream>>>(n->loss_part, kLossBlocks, rows, n->loss_dev);
  CUDA_TRY(cudaGetLastError());
  for (int l = L - 1; l >= 0; --l) {
    const int wout = n->w[l + 1], win = n->w[l];
    // dW_l = dZ_l^T a_{l-1}: i over outputs (dZ is i-contiguous), j over inputs, k over rows
    int splits = std::min(kMaxSplits, std::max(1, rows / kSplitChunk));
    EpiArgs ep{};
    ep.o32 = splits > 1 ? n->splitk : n->grad + n->offW[l];
    ep.ldo32 = win;
    CUDA_TRY((gemm<false, false, EPI_STORE>(n->stream, n->d16[cur], n->ld[l + 1], n->act16[l], n->ld[l], wout,
                                            win, rows, splits, ep)));
    if (splits > 1) {
      int k_split = ((rows + splits - 1) / splits + BK - 1) / BK * BK;
      int used = (rows + k_split - 1) / k_split;
      long long mn = (long long)wout * win;
      splitk_sum<<<grid_for(mn), 256, 0, n->stream>>>(n->splitk, used, mn, n->grad + n->offW[l]);
      CUDA_TRY(cudaGetLastError());
    }
    colsum_kernel<<<(wout + 127) / 128, 128, 0, n->stream>>>(n->d32[cur], rows, wout, n->ld[l + 1],
                                                            n->grad + n->offb[l]);
    CUDA_TRY(cudaGetLastError());
    if (l > 0) {
      // dZ_{l-1} = (dZ_l W_l) * (1 - h^2): i over rows, j over inputs, k over outputs
      EpiArgs e2{};
      e2.h32 = n->h32[l];
      e2.ldh = n->ld[l];
      e2.o32 = n->d32[cur ^ 1];
      e2.ldo32 = n->ld[l];
      e2.o16 = n->d16[cur ^ 1];
      e2.ldo16 = n->ld[l];
      CUDA_TRY((gemm<true, false, EPI_TANH_GRAD>(n->stream, n->d16[cur], n->ld[l + 1], n->W16[l], n->ld[l],
                                                 rows, win, wout, 1, e2)));
      cur ^= 1;
    }
  }
  return 0;
}

int pack_all(bipm_mlp* n) {
  for (int l = 0; l < n->L; ++l) {
    long long tot = (long long)n->w[l + 1] * n->ld[l];
    pack_weights<<<grid_for(tot), 256, 0, n->stream>>>(n->master + n->offW[l], n->w[l + 1], n->w[l], n->W16[l],
                                                       n->ld[l]);
    CUDA_TRY(cudaGetLastError());
  }
  return 0;
}

int load_inputs(bipm_mlp* n, const float* x, const int* idx, int rows, int n_data) {
  long long tot = (long long)rows * n->ld[0];
  to_bf16_rows<<<grid_for(tot), 256, 0, n->stream>>>(x, idx, rows, n->w[0], n_data, n->act16[0], n->ld[0],
                                                     n->bad_index);
  CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace

extern "C" {

int bipm_mlp_create(const int* widths, int n_widths, int max_rows, void* stream, bipm_mlp** out) {
  if (!widths || !out) return fail(BIPM_EINVAL, "null widths or out");
  *out = nullptr;
  if (n_widths < 2 || n_widths > kMaxLayers + 1)
    return fail(BIPM_EINVAL, "n_widths must be in [2, " + std::to_string(kMaxLayers + 1) + "]");
  if (max_rows < 1) return fail(BIPM_EINVAL, "max_rows must be >= 1");
  for (int i = 0; i < n_widths; ++i)
    if (widths[i] < 1 || widths[i] > 65536) return fail(BIPM_EINVAL, "widths must be in [1, 65536]");
  bipm_mlp* n = new bipm_mlp();
  n->L = n_widths - 1;
  n->max_rows = max_rows;
  n->stream = (cudaStream_t)stream;
  long long pos = 0;
  int maxw = 0;
  for (int i = 0; i < n_widths; ++i) {
    n->w[i] = widths[i];
    n->ld[i] = pad8(widths[i]);
    maxw = std::max(maxw, n->ld[i]);
  }
  for (int l = 0; l < n->L; ++l) {
    n->offW[l] = pos;
    pos += (long long)n->w[l + 1] * n->w[l];
    n->offb[l] = pos;
    pos += n->w[l + 1];
  }
  n->n_params = pos;
  auto alloc = [&](size_t bytes, void** p) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    n->allocs.push_back(*p);
    return true;
  };
  bool ok = alloc(pos * 4, (void**)&n->master) && alloc(pos * 4, (void**)&n->mom1) &&
            alloc(pos * 4, (void**)&n->mom2) && alloc(pos * 4, (void**)&n->grad);
  for (int l = 0; ok && l < n->L; ++l) ok = alloc((size_t)n->w[l + 1] * n->ld[l] * 2, (void**)&n->W16[l]);
  for (int l = 0; ok && l < n->L; ++l) ok = alloc((size_t)max_rows * n->ld[l] * 2, (void**)&n->act16[l]);
  for (int l = 1; ok && l < n->L; ++l) ok = alloc((size_t)max_rows * n->ld[l] * 4, (void**)&n->h32[l]);
  ok = ok && alloc((size_t)max_rows * n->w[n->L] * 4, (void**)&n->out32);
  for (int i = 0; ok && i < 2; ++i)
    ok = alloc((size_t)max_rows * maxw * 4, (void**)&n->d32[i]) &&
         alloc((size_t)max_rows * maxw * 2, (void**)&n->d16[i]);
  long long wmax = 0;
  for (int l = 0; l < n->L; ++l) wmax = std::max(wmax, (long long)n->w[l + 1] * n->w[l]);
  n->splitk_elems = wmax * kMaxSplits;
  ok = ok && alloc(n->splitk_elems * 4, (void**)&n->splitk) && alloc(kLossBlocks * 8, (void**)&n->loss_part) &&
       alloc(8, (void**)&n->loss_dev) && alloc(sizeof(int), (void**)&n->bad_index) &&
       alloc((size_t)max_rows * n->w[0] * 4, (void**)&n->xin) &&
       alloc((size_t)max_rows * n->w[n->L] * 4, (void**)&n->tin);
  if (!ok) {
    bipm_mlp_destroy(n);
    return fail(BIPM_ENOMEM, "cudaMalloc failed for the network buffers");
  }
  if (cudaMemsetAsync(n->master, 0, pos * 4, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->mom1, 0, pos * 4, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->mom2, 0, pos * 4, n->stream) != cudaSuccess ||
      cudaMemsetAsync(n->bad_index, 0, sizeof(int), n->stream) != cudaSuccess) {
    bipm_mlp_destroy(n);
    return fail(BIPM_ECUDA, "cudaMemsetAsync failed");
  }
  if (pack_all(n)) {
    bipm_mlp_destroy(n);
    return BIPM_ECUDA;
  }
  *out = n;
  return 0;
}

int bipm_mlp_param_count(const bipm_mlp* n, long long* count) {
  if (!n || !count) return fail(BIPM_EINVAL, "null network or count");
  *count = n->n_params;
  return 0;
}

int bipm_mlp_set_params(bipm_mlp* n, const float* params, int on_device) {
  if (!n || !params) return fail(BIPM_EINVAL, "null network or params");
  CUDA_TRY(cudaMemcpyAsync(n->master, params, n->n_params * 4,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->stream));
  CUDA_TRY(cudaMemsetAsync(n->mom1, 0, n->n_params * 4, n->stream));
  CUDA_TRY(cudaMemsetAsync(n->mom2, 0, n->n_params * 4, n->stream));
  n->adam_t = 0;
  int rc = pack_all(n);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(n->stream));
  return 0;
}

int bipm_mlp_get_params(const bipm_mlp* n, float* params, int on_device) {
  if (!n || !params) return fail(BIPM_EINVAL, "null network or params");
  CUDA_TRY(cudaMemcpyAsync(params, n->master, n->n_params * 4,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
  CUDA_TRY(cudaStreamSynchronize(n->stream));
  return 0;
}

int bipm_mlp_forward(bipm_mlp* n, const float* x, int rows, float* out, int on_device) {
  if (!n) return fail(BIPM_EINVAL, "null network");
  if (rows < 0) return fail(BIPM_EINVAL, "rows must be >= 0");
  if (rows == 0) return 0;
  if (!x || !out) return fail(BIPM_EINVAL, "null x or out");
  const int win = n->w[0], wout = n->w[n->L];
  for (int r0 = 0; r0 < rows; r0 += n->max_rows) {
    int rr = std::min(n->max_rows, rows - r0);
    const float* xs = x + (long long)r0 * win;
    if (!on_device) {
      CUDA_TRY(cudaMemcpyAsync(n->xin, xs, (size_t)rr * win * 4, cudaMemcpyHostToDevice, n->stream));
      xs = n->xin;
    }
    int rc = load_inputs(n, xs, nullptr, rr, rr);
    if (!rc) rc = forward_rows(n, rr);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(out + (long long)r0 * wout, n->out32, (size_t)rr * wout * 4,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(n->stream));
  return 0;
}

int bipm_mlp_loss_grad(bipm_mlp* n, const float* x, const float* t, int rows, float* grad, double* loss,
                       int on_device) {
  if (!n) return fail(BIPM_EINVAL, "null network");
  if (rows < 1 || rows > n->max_rows) return fail(BIPM_EINVAL, "rows must be in [1, max_rows]");
  if (!x || !t) return fail(BIPM_EINVAL, "null x or t");
  const float* xs = x;
  const float* ts = t;
  if (!on_device) {
    CUDA_TRY(cudaMemcpyAsync(n->xin, x, (size_t)rows * n->w[0] * 4, cudaMemcpyHostToDevice, n->stream));
    CUDA_TRY(cudaMemcpyAsync(n->tin, t, (size_t)rows * n->w[n->L] * 4, cudaMemcpyHostToDevice, n->stream));
    xs = n->xin;
    ts = n->tin;
  }
  int rc = load_inputs(n, xs, nullptr, rows, rows);
  if (!rc) rc = forward_rows(n, rows);
  if (!rc) rc = backward_rows(n, ts, nullptr, rows, rows);
  if (rc) return rc;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (grad) CUDA_TRY(cudaMemcpyAsync(grad, n->grad, n->n_params * 4, k, n->stream));
  if (loss) CUDA_TRY(cudaMemcpyAsync(loss, n->loss_dev, 8, k, n->stream));
  CUDA_TRY(cudaStreamSynchronize(n->stream));
  return 0;
}

int bipm_mlp_train_step(bipm_mlp* n, const float* x, const float* t, int n_data, const int* idx, int rows,
                        float lr, double* loss) {
  if (!n) return fail(BIPM_EINVAL, "null network");
  if (rows < 1 || rows > n->max_rows) return fail(BIPM_EINVAL, "rows must be in [1, max_rows]");
  if (!x || !t) return fail(BIPM_EINVAL, "null x or t");
  if (n_data < 1 || (!idx && n_data < rows)) return fail(BIPM_EINVAL, "n_data must cover the batch rows");
  int rc = load_inputs(n, x, idx, rows, n_data);
  if (!rc) rc = forward_rows(n, rows);
  if (!rc) rc = backward_rows(n, t, idx, rows, n_data);
  if (rc) return rc;
  n->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = (float)(1.0 - std::pow(0.9, n->adam_t));
  float c2 = (float)(1.0 - std::pow(0.999, n->adam_t));
  adam_kernel<<<grid_for(n->n_params), 256, 0, n->stream>>>(n->master, n->mom1, n->mom2, n->grad, n->n_params,
                                                            lr, b1, b2, c1, c2, 1e-8f);
  CUDA_TRY(cudaGetLastError());
  rc = pack_all(n);
  if (rc) return rc;
  if (loss) {
    int bad = 0;
    CUDA_TRY(cudaMemcpyAsync(loss, n->loss_dev, 8, cudaMemcpyDeviceToHost, n->stream));
    CUDA_TRY(cudaMemcpyAsync(&bad, n->bad_index, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    CUDA_TRY(cudaStreamSynchronize(n->stream));
    if (bad) {
      cudaMemsetAsync(n->bad_index, 0, sizeof(int), n->stream);
      return fail(BIPM_EINVAL, "a batch index lies outside [0, n_data) (row 0 was used in its place)");
    }
  }
  return 0;
}

void bipm_mlp_destroy(bipm_mlp* n) {
  if (!n) return;
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

}  // extern "C"
