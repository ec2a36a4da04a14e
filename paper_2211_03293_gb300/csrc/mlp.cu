// Learned form: a multilayer perceptron (SiLU hidden layers, linear output) with
// bfloat16 weights and activations, FP32 accumulation, trained and evaluated on the
// GPU by the kernels in this file.  It predicts a fast stage's increment from the
// cell state, pressure, stage length and slow forcing; the prediction serves as the
// Newton initial guess of the fast solve, which still decides every result.
//
// Every matrix product goes through one tensor-core GEMM,
//     C[M x N] = A[M x K] * B[N x K]^T        (A, B bfloat16 with K contiguous),
// issued with tcgen05.mma from shared-memory operands into a TMEM accumulator:
//   * one CTA of 4 warps per 128-row tile of C and the whole width N (16..256) of C;
//   * K in chunks of 64: the warps copy the A and B chunks from global memory into
//     the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix,
//     core matrices 128 bytes apart along K and 1024 bytes apart along M/N), one
//     thread issues four K=16 MMAs and commits them to an mbarrier that every
//     thread waits on (bounded) before the chunk's shared memory is reused;
//   * the epilogue reads the accumulator rows with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31) and applies bias and SiLU, or stores plain FP32 partial sums
//     (split K for the weight gradients, whose contraction runs over the batch).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/mri_mlp.h"

namespace mri {
namespace {

constexpr int kTileM = 128;
constexpr int kChunkK = 64;
constexpr int kGemmThreads = 128;
constexpr uint32_t kLBO = 128;     // bytes between core matrices along K
constexpr uint32_t kSBO = 1024;    // bytes between core matrices along M / N
constexpr int kATileBytes = kTileM * kChunkK * 2;   // 16 KB
constexpr int kGemmSmem = 100 * 1024;   // also keeps at most two CTAs (2 x 256 TMEM columns) per SM
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on every mbarrier wait

enum Epi { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_F32 = 2 };

struct GemmArgs {
  const __nv_bfloat16* A;   // [M][lda]
  const __nv_bfloat16* B;   // [N][ldb]
  int M, N, K, lda, ldb;
  int k_per_split;          // multiple of kChunkK
  const float* bias;        // [N] (EPI_HIDDEN / EPI_OUT)
  float* C;                 // [M][ldc] fp32 (z, y, or the split's partial block)
  int ldc;
  long long split_stride;   // elements between the partial blocks of consecutive splits
  __nv_bfloat16* act;       // EPI_HIDDEN: bf16 silu(z) [M][ldact]
  int ldact;
  int* err;                 // set on a bounded wait that ran out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor of tcgen05: start address, leading (K) and stride
// (M/N) byte offsets, all in 16-byte units; descriptor version 1; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, bfloat16 A and
// B, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned long long t0) {
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}

// Copy rows [r0, r0 + rows_tile) x K-chunk [k0, k0 + 64) of a bf16 row-major matrix
// into the core-matrix layout at dst (rows beyond nrows and columns beyond K are zero).
__device__ __forceinline__ void load_tile(unsigned char* dst, const __nv_bfloat16* src, int ld, int r0, int nrows,
                                          int rows_tile, int k0, int K) {
  const int vecs = rows_tile * (kChunkK / 8);
  for (int v = threadIdx.x; v < vecs; v += blockDim.x) {
    const int r = v >> 3, j = v & 7;
    const int gr = r0 + r, gk = k0 + 8 * j;
    int4 val = make_int4(0, 0, 0, 0);
    if (gr < nrows && gk < K) val = *reinterpret_cast<const int4*>(src + (size_t)gr * ld + gk);
    *reinterpret_cast<int4*>(dst + (r >> 3) * kSBO + j * kLBO + (r & 7) * 16) = val;
  }
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

template <int EPI>
__global__ void __launch_bounds__(kGemmThreads) gemm_bf16_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int failed;
  unsigned char* sA = smem;
  unsigned char* sB = smem + kATileBytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTileM;
  const int split = blockIdx.y;
  const int kb = split * g.k_per_split;
  const int ke = min(g.K, kb + g.k_per_split);
  const int Npad = (g.N + 15) & ~15;
  uint32_t ncols = 32;
  while ((int)ncols < Npad) ncols <<= 1;
  const uint32_t mb = smem_u32(&mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = instr_desc(kTileM, Npad);
  const unsigned long long t0 = now_ns();

  uint32_t parity = 0;
  bool any = false;
  for (int k0 = kb; k0 < ke; k0 += kChunkK) {
    load_tile(sA, g.A, g.lda, m0, g.M, kTileM, k0, ke);
    load_tile(sB, g.B, g.ldb, 0, g.N, Npad, k0, ke);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < kChunkK / 16; ++kk) {
        const uint64_t ad = smem_desc(a0 + kk * 2 * kLBO);
        const uint64_t bd = smem_desc(b0 + kk * 2 * kLBO);
        const uint32_t acc = (any || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    any = true;
    if (!mbar_wait(mb, parity, t0)) failed = 1;
    parity ^= 1u;
    __syncthreads();
    if (failed) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: row m of C in TMEM lane 32 warp + lane
  const int m = m0 + 32 * warp + lane;
  if (!failed) {
    for (int c = 0; c < Npad; c += 8) {
      uint32_t r[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int col = c + j;
          if (col >= g.N) break;
          float v = any ? __uint_as_float(r[j]) : 0.0f;
          if (EPI == EPI_F32) {
            g.C[(size_t)split * g.split_stride + (size_t)m * g.ldc + col] = v;
          } else {
            v += g.bias[col];
            g.C[(size_t)m * g.ldc + col] = v;
            if (EPI == EPI_HIDDEN) g.act[(size_t)m * g.ldact + col] = __float2bfloat16_rn(silu_f(v));
          }
        }
      }
    }
  }
  if (failed && threadIdx.x == 0) atomicExch(g.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// ------------------------------------------------------------------ elementwise

// x fp32 [B][n_in] -> bf16 [B][ld] (zero padding columns)
__global__ void to_bf16_kernel(const float* x, int B, int n, int ld, __nv_bfloat16* out) {
  const long long total = (long long)B * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / ld), j = (int)(e % ld);
    out[e] = __float2bfloat16_rn(j < n ? x[(size_t)b * n + j] : 0.0f);
  }
}

// src bf16 [rows][ld_src] -> dst bf16 [cols][ld_dst] (transpose; padding columns zero)
__global__ void transpose_bf16_kernel(const __nv_bfloat16* src, int rows, int cols, int ld_src, __nv_bfloat16* dst,
                                      int ld_dst) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * ld_src + c] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ld_dst) dst[(size_t)c * ld_dst + r] = tile[threadIdx.x][i];
  }
}

// master fp32 W [out][in] -> bf16 W [out][in] and bf16 W^T [in][out]
__global__ void weights_bf16_kernel(const float* W, int nout, int nin, __nv_bfloat16* Wb, __nv_bfloat16* WTb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nout * nin; e += gridDim.x * blockDim.x) {
    const int o = e / nin, i = e % nin;
    const __nv_bfloat16 v = __float2bfloat16_rn(W[e]);
    Wb[e] = v;
    WTb[(size_t)i * nout + o] = v;
  }
}

// loss L = sum_b sum_j m_j (y - t)^2 / (2 B) and dy = m (y - t) / B; y, t [B][n]
__global__ void loss_grad_kernel(const float* y, const float* t, const float* m, int B, int n, float* dy,
                                 float* partial) {
  __shared__ float red[256];
  float acc = 0.0f;
  const float invB = 1.0f / (float)B;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)B * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % n);
    const float r = y[e] - t[e];
    dy[e] = m[j] * r * invB;
    acc += m[j] * r * r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0] * 0.5f * invB;
}

// dz = dA * silu'(z) (hidden layers) or dz = dy (output): bf16 dz [B][ldz] and bf16
// dz^T [N][ldT]; per-block column sums of the FP32 dz for the bias gradient.
__global__ void dz_kernel(const float* dA, int ld_dA, const float* z, int ld_z, int B, int N, int hidden,
                          __nv_bfloat16* dzb, int ldz, __nv_bfloat16* dzT, int ldT, float* colpart, int rows_per_block) {
  const int j = threadIdx.x;   // one thread per column (N <= 256)
  if (j >= N) return;
  const int b0 = blockIdx.x * rows_per_block, b1 = min(B, b0 + rows_per_block);
  float acc = 0.0f;
  for (int b = b0; b < b1; ++b) {
    float v = dA[(size_t)b * ld_dA + j];
    if (hidden) {
      const float zz = z[(size_t)b * ld_z + j];
      const float s = 1.0f / (1.0f + __expf(-zz));
      v *= s * (1.0f + zz * (1.0f - s));
    }
    acc += v;
    const __nv_bfloat16 q = __float2bfloat16_rn(v);
    dzb[(size_t)b * ldz + j] = q;
    dzT[(size_t)j * ldT + b] = q;
  }
  colpart[(size_t)blockIdx.x * N + j] = acc;
}

// out[j] = sum_p part[p][j]  (fixed order: deterministic)
__global__ void colsum_kernel(const float* part, int P, int N, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.0f;
  for (int p = 0; p < P; ++p) s += part[(size_t)p * N + j];
  out[j] = s;
}

// dW[o][i] = sum over splits of the partial blocks [split][o][i]
__global__ void split_sum_kernel(const float* part, int splits, long long stride, int n, float* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int p = 0; p < splits; ++p) s += part[(size_t)p * stride + e];
    out[e] = s;
  }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters
__global__ void adam_kernel(float* w, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float a = b1 * m1[e] + (1.0f - b1) * gg;
    const float v = b2 * m2[e] + (1.0f - b2) * gg * gg;
    m1[e] = a;
    m2[e] = v;
    w[e] -= lr * (a * c1) / (sqrtf(v * c2) + eps);
  }
}

}  // namespace
}  // namespace mri

// ------------------------------------------------------------------ host side

struct mri_mlp {
  int L = 0;
  std::vector<int> dims;      // L + 1 sizes (padded to multiples of 16)
  int batch_max = 0, bpad = 0;
  int device = -1;
  // parameters: FP32 master (W_l then b_l for each l, packed), Adam moments, gradient
  float *params = nullptr, *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
  std::vector<long long> offW, offb;
  long long nparams = 0;
  // bf16 weights and transposes
  std::vector<__nv_bfloat16*> Wb, WTb;
  // activations: bf16 GEMM inputs a_l [B][dims[l]] (l = 0..L-1), fp32 z_l [B][dims[l+1]]
  std::vector<__nv_bfloat16*> act;
  std::vector<float*> z;
  // backward scratch
  float* dA = nullptr;              // [B][256]
  float* dA2 = nullptr;             // [B][256]
  __nv_bfloat16 *dzb = nullptr, *dzT = nullptr, *aT = nullptr;
  float *part = nullptr, *colpart = nullptr, *lossp = nullptr;
  int* err = nullptr;
  int splits = 64;
};

namespace {

using namespace mri;

int gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K, int epi,
         const float* bias, float* C, int ldc, __nv_bfloat16* act, int ldact, int splits, long long split_stride,
         int* err, cudaStream_t st) {
  static bool attr_done[3] = {false, false, false};
  GemmArgs g{};
  g.A = A; g.B = B; g.M = M; g.N = N; g.K = K; g.lda = lda; g.ldb = ldb;
  const int chunks = (K + kChunkK - 1) / kChunkK;
  const int per = (chunks + splits - 1) / splits;
  g.k_per_split = per * kChunkK;
  const int used_splits = (K + g.k_per_split - 1) / g.k_per_split;
  g.bias = bias; g.C = C; g.ldc = ldc; g.split_stride = split_stride; g.act = act; g.ldact = ldact; g.err = err;
  dim3 grid((M + kTileM - 1) / kTileM, used_splits < 1 ? 1 : used_splits);
  cudaError_t e;
  if (epi == EPI_HIDDEN) {
    if (!attr_done[0]) { cudaFuncSetAttribute(gemm_bf16_kernel<EPI_HIDDEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem); attr_done[0] = true; }
    gemm_bf16_kernel<EPI_HIDDEN><<<grid, kGemmThreads, kGemmSmem, st>>>(g);
  } else if (epi == EPI_OUT) {
    if (!attr_done[1]) { cudaFuncSetAttribute(gemm_bf16_kernel<EPI_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem); attr_done[1] = true; }
    gemm_bf16_kernel<EPI_OUT><<<grid, kGemmThreads, kGemmSmem, st>>>(g);
  } else {
    if (!attr_done[2]) { cudaFuncSetAttribute(gemm_bf16_kernel<EPI_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem); attr_done[2] = true; }
    gemm_bf16_kernel<EPI_F32><<<grid, kGemmThreads, kGemmSmem, st>>>(g);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? used_splits : -1;
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

void free_all(mri_mlp* m) {
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(m->params); f(m->m1); f(m->m2); f(m->grad);
  for (auto p : m->Wb) f(p);
  for (auto p : m->WTb) f(p);
  for (auto p : m->act) f(p);
  for (auto p : m->z) f(p);
  f(m->dA); f(m->dA2); f(m->dzb); f(m->dzT); f(m->aT); f(m->part); f(m->colpart); f(m->lossp); f(m->err);
}

int refresh_bf16(mri_mlp* m, cudaStream_t st) {
  for (int l = 0; l < m->L; ++l) {
    const int nin = m->dims[l], nout = m->dims[l + 1];
    weights_bf16_kernel<<<grid_for((long long)nin * nout), 256, 0, st>>>(m->params + m->offW[l], nout, nin, m->Wb[l],
                                                                         m->WTb[l]);
  }
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

}  // namespace

extern "C" int mri_mlp_create(const int* dims, int n_layers, int batch_max, const float* init_params, mri_mlp** out) {
  if (!dims || !out || n_layers < 1 || n_layers > MRI_MLP_MAX_LAYERS || batch_max < 1 || batch_max > (1 << 24))
    return MRI_EINVAL;
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] < 16 || dims[l] > 256 || dims[l] % 16 != 0) return MRI_EINVAL;
  mri_mlp* m = new mri_mlp();
  m->L = n_layers;
  m->dims.assign(dims, dims + n_layers + 1);
  m->batch_max = batch_max;
  m->bpad = (batch_max + 63) / 64 * 64;
  cudaGetDevice(&m->device);
  long long o = 0;
  for (int l = 0; l < n_layers; ++l) {
    m->offW.push_back(o); o += (long long)dims[l] * dims[l + 1];
    m->offb.push_back(o); o += dims[l + 1];
  }
  m->nparams = o;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) { if (cudaMalloc(p, bytes) != cudaSuccess) ok = false; };
  alloc((void**)&m->params, o * 4); alloc((void**)&m->m1, o * 4); alloc((void**)&m->m2, o * 4);
  alloc((void**)&m->grad, o * 4);
  m->Wb.resize(n_layers); m->WTb.resize(n_layers); m->act.resize(n_layers); m->z.resize(n_layers);
  const size_t B = (size_t)m->bpad;
  for (int l = 0; l < n_layers; ++l) {
    alloc((void**)&m->Wb[l], (size_t)dims[l] * dims[l + 1] * 2);
    alloc((void**)&m->WTb[l], (size_t)dims[l] * dims[l + 1] * 2);
    alloc((void**)&m->act[l], B * dims[l] * 2);
    alloc((void**)&m->z[l], B * dims[l + 1] * 4);
  }
  alloc((void**)&m->dA, B * 256 * 4); alloc((void**)&m->dA2, B * 256 * 4);
  alloc((void**)&m->dzb, B * 256 * 2); alloc((void**)&m->dzT, B * 256 * 2); alloc((void**)&m->aT, B * 256 * 2);
  alloc((void**)&m->part, (size_t)m->splits * 256 * 256 * 4);
  alloc((void**)&m->colpart, ((B + 63) / 64) * 256 * 4);   // [row blocks of 64][<= 256 columns]
  alloc((void**)&m->lossp, 4096 * 4);
  alloc((void**)&m->err, 4);
  if (ok && init_params)
    ok = cudaMemcpy(m->params, init_params, o * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) ok = cudaMemset(m->m1, 0, o * 4) == cudaSuccess && cudaMemset(m->m2, 0, o * 4) == cudaSuccess &&
               cudaMemset(m->err, 0, 4) == cudaSuccess && cudaMemset(m->aT, 0, B * 256 * 2) == cudaSuccess &&
               cudaMemset(m->dzT, 0, B * 256 * 2) == cudaSuccess;
  if (ok) ok = refresh_bf16(m, 0) == MRI_OK && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    free_all(m);
    delete m;
    return MRI_ECUDA;
  }
  *out = m;
  return MRI_OK;
}

extern "C" void mri_mlp_free(mri_mlp* m) {
  if (!m) return;
  free_all(m);
  delete m;
}

extern "C" long long mri_mlp_num_params(const mri_mlp* m) { return m ? m->nparams : -1; }

extern "C" int mri_mlp_params(mri_mlp* m, float* host_out, const float* host_in) {
  if (!m) return MRI_EINVAL;
  if (host_out && cudaMemcpy(host_out, m->params, m->nparams * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MRI_ECUDA;
  if (host_in) {
    if (cudaMemcpy(m->params, host_in, m->nparams * 4, cudaMemcpyHostToDevice) != cudaSuccess) return MRI_ECUDA;
    if (refresh_bf16(m, 0) != MRI_OK || cudaDeviceSynchronize() != cudaSuccess) return MRI_ECUDA;
  }
  return MRI_OK;
}

extern "C" int mri_mlp_forward(mri_mlp* m, const float* x, int B, float* y, void* stream) {
  if (!m || !x || !y || B < 1 || B > m->batch_max) return MRI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int L = m->L;
  // the network's raw inputs are the first dims[0] columns of x ([B][dims[0]])
  to_bf16_kernel<<<grid_for((long long)B * m->dims[0]), 256, 0, st>>>(x, B, m->dims[0], m->dims[0], m->act[0]);
  for (int l = 0; l < L; ++l) {
    const int nin = m->dims[l], nout = m->dims[l + 1];
    const bool last = (l == L - 1);
    float* zo = last ? y : m->z[l];
    if (gemm(m->act[l], nin, m->Wb[l], nin, B, nout, nin, last ? EPI_OUT : EPI_HIDDEN, m->params + m->offb[l], zo,
             nout, last ? nullptr : m->act[l + 1], nout, 1, 0, m->err, st) < 0)
      return MRI_ECUDA;
    if (last) continue;
  }
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_mlp_grad(mri_mlp* m, const float* x, const float* t, const float* w_out, int B, float* y,
                            float* loss, void* stream) {
  if (!m || !x || !t || !w_out || !y || B < 1 || B > m->batch_max) return MRI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = mri_mlp_forward(m, x, B, y, stream);
  if (rc != MRI_OK) return rc;
  const int L = m->L, nout = m->dims[L];
  const int lb = grid_for((long long)B * nout) < 1024 ? grid_for((long long)B * nout) : 1024;
  loss_grad_kernel<<<lb, 256, 0, st>>>(y, t, w_out, B, nout, m->dA, m->lossp);
  if (loss) colsum_kernel<<<1, 32, 0, st>>>(m->lossp, lb, 1, loss);
  const int bp = m->bpad;
  const int rows_per_block = 64;
  const int nblk = (B + rows_per_block - 1) / rows_per_block;
  float* dA = m->dA;
  float* dAn = m->dA2;
  for (int l = L - 1; l >= 0; --l) {
    const int nin = m->dims[l], no = m->dims[l + 1];
    // dz_l (bf16, and transposed), bias gradient
    dz_kernel<<<nblk, 256, 0, st>>>(dA, no, m->z[l], no, B, no, l < L - 1 ? 1 : 0, m->dzb, no, m->dzT, bp,
                                    m->colpart, rows_per_block);
    colsum_kernel<<<(no + 127) / 128, 128, 0, st>>>(m->colpart, nblk, no, m->grad + m->offb[l]);
    // dW_l = dz^T a_{l-1}: contraction over the batch, split over it
    dim3 tb(32, 8), tg((nin + 31) / 32, (B + 31) / 32);
    transpose_bf16_kernel<<<tg, tb, 0, st>>>(m->act[l], B, nin, nin, m->aT, bp);
    const long long stride = (long long)no * nin;
    int used = gemm(m->dzT, bp, m->aT, bp, no, nin, B, EPI_F32, nullptr, m->part, nin, nullptr, 0, m->splits,
                    stride, m->err, st);
    if (used < 0) return MRI_ECUDA;
    split_sum_kernel<<<grid_for(stride), 256, 0, st>>>(m->part, used, stride, (int)stride, m->grad + m->offW[l]);
    // dA_{l-1} = dz W_l
    if (l > 0) {
      if (gemm(m->dzb, no, m->WTb[l], no, B, nin, no, EPI_F32, nullptr, dAn, nin, nullptr, 0, 1, 0, m->err, st) < 0)
        return MRI_ECUDA;
      float* tmp = dA; dA = dAn; dAn = tmp;
    }
  }
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_mlp_grad_copy(mri_mlp* m, float* dst, void* stream) {
  if (!m || !dst) return MRI_EINVAL;
  return cudaMemcpyAsync(dst, m->grad, m->nparams * 4, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_mlp_adam(mri_mlp* m, float lr, int step, void* stream) {
  if (!m || step < 1 || !(lr > 0)) return MRI_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f / (1.0f - powf(b1, (float)step)), c2 = 1.0f / (1.0f - powf(b2, (float)step));
  adam_kernel<<<grid_for(m->nparams), 256, 0, st>>>(m->params, m->grad, m->m1, m->m2, (int)m->nparams, lr, b1, b2,
                                                     c1, c2, 1e-8f);
  return refresh_bf16(m, st);
}

extern "C" int mri_mlp_status(mri_mlp* m) {
  if (!m) return MRI_EINVAL;
  int h = 0;
  if (cudaMemcpy(&h, m->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return MRI_ECUDA;
  return h ? MRI_ETIMEOUT : MRI_OK;
}

// ------------------------------------------------------------------ learned-form data

namespace mri {
namespace {

// one thread per (cell, feature): raw feature, then (raw - mean) * inv_std
__global__ void features_kernel(const double* y, const double* p, const double* phi, int K, int ncell, int n,
                                double Hs, const float* mean, const float* inv_std, float* x, int ld) {
  const int nf = 2 * n + 2;
  const long long total = (long long)ncell * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / ld), f = (int)(e % ld);
    float v = 0.0f;
    if (f < nf) {
      double raw;
      const double* yc = y + (size_t)c * n;
      if (f < n - 1) raw = log10(fmax(yc[f], 1e-30));
      else if (f == n - 1) raw = yc[n - 1] * 1e-3;
      else if (f == n) raw = log(p[c] / 101325.0);
      else if (f == n + 1) raw = log10(Hs);
      else {
        const int comp = f - n - 2;
        double acc = 0.0;   // Hs * integral over the stage of the forcing polynomial
        for (int k = 0; k < K; ++k) acc += phi[((size_t)c * K + k) * n + comp] / (k + 1);
        raw = Hs * acc;
      }
      v = ((float)raw - mean[f]) * inv_std[f];
    }
    x[e] = v;
  }
}

// t[c][g n + j] = ((y_seq[c][g][j] - y_in[c][j]) - tmean) * tinv_std, 0 up to ld
__global__ void targets_kernel(const double* y_in, const double* y_seq, int G, int ncell, int n, const float* tmean,
                               const float* tinv_std, float* t, int ld) {
  const long long total = (long long)ncell * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / ld), o = (int)(e % ld);
    float v = 0.0f;
    if (o < G * n) {
      const int j = o % n;
      v = ((float)(y_seq[(size_t)c * G * n + o] - y_in[(size_t)c * n + j]) - tmean[o]) * tinv_std[o];
    }
    t[e] = v;
  }
}

// guess[c][g][j] = y_in[c][j] + tmean[g n + j] + tstd[g n + j] * yhat[c][g n + j]
__global__ void guess_kernel(const double* y_in, const float* yhat, int ld, int G, int ncell, int n,
                             const float* tmean, const float* tstd, double* guess) {
  const long long total = (long long)ncell * G * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / (G * n)), o = (int)(e % (G * n)), j = o % n;
    guess[e] = y_in[(size_t)c * n + j] + (double)(tmean[o] + tstd[o] * yhat[(size_t)c * ld + o]);
  }
}

// step_exp[c] = round(tmean + tstd * yhat[c][col]) clamped to [kmin, kmax]
__global__ void step_exp_kernel(const float* yhat, int ld, int col, int ncell, float tmean, float tstd, int kmin,
                                int kmax, int8_t* step_exp) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const float v = fmaf(tstd, yhat[(size_t)c * ld + col], tmean);
    int k = (int)rintf(v);
    if (!(v == v)) k = 0;
    step_exp[c] = (int8_t)min(kmax, max(kmin, k));
  }
}

// Column moments, pass 1: block (column group of 32, row chunk) sums X and X^2 (FP64)
// over its rows for its 32 columns; 8 row slots per block, combined in a fixed order.
constexpr int kMomChunks = 256;
__global__ void moments_part_kernel(const float* X, long long rows, int cols, int ld, double* part) {
  __shared__ double s1[8][32], s2[8][32];
  const int f = blockIdx.x * 32 + threadIdx.x, slot = threadIdx.y;
  const long long per = (rows + kMomChunks - 1) / kMomChunks;
  const long long r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
  double a = 0.0, b = 0.0;
  if (f < cols)
    for (long long r = r0 + slot; r < r1; r += 8) {
      const double v = X[r * ld + f];
      a += v;
      b = fma(v, v, b);
    }
  s1[slot][threadIdx.x] = a;
  s2[slot][threadIdx.x] = b;
  __syncthreads();
  if (slot == 0 && f < cols) {
    double A = 0.0, B = 0.0;
    for (int k = 0; k < 8; ++k) { A += s1[k][threadIdx.x]; B += s2[k][threadIdx.x]; }
    part[((size_t)blockIdx.y * cols + f) * 2] = A;
    part[((size_t)blockIdx.y * cols + f) * 2 + 1] = B;
  }
}

// pass 2: one thread per column adds the chunks in order: mean, population standard
// deviation (a deviation below floor becomes 1) and its inverse
__global__ void moments_final_kernel(const double* part, long long rows, int cols, float floor_sd, float* mean,
                                     float* inv_std, float* sd_out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= cols) return;
  double A = 0.0, B = 0.0;
  for (int c = 0; c < kMomChunks; ++c) {
    A += part[((size_t)c * cols + f) * 2];
    B += part[((size_t)c * cols + f) * 2 + 1];
  }
  const double m = A / (double)rows;
  const double var = fmax(B / (double)rows - m * m, 0.0);
  double sd = sqrt(var);
  if (!(sd >= (double)floor_sd)) sd = 1.0;
  mean[f] = (float)m;
  inv_std[f] = (float)(1.0 / sd);
  if (sd_out) sd_out[f] = (float)sd;
}

// out[i][f] = (X[perm[i]][f] - mean[f]) * inv_std[f] for f < used, 0 up to ld_out
__global__ void standardise_kernel(const float* X, int ld, const int32_t* perm, long long rows_out, int used,
                                   const float* mean, const float* inv_std, float* out, int ld_out) {
  const long long total = rows_out * ld_out;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / ld_out;
    const int f = (int)(e % ld_out);
    const long long src = perm ? (long long)perm[i] : i;
    out[e] = (f < used) ? (X[src * ld + f] - mean[f]) * inv_std[f] : 0.0f;
  }
}

// k[c] = log2(n_sub / max(accepted[c], 1)): the log2 of a cell's mean accepted step
// relative to the uniform substep
__global__ void step_targets_kernel(const int32_t* accepted, int stride, int ncell, int n_sub, float* k) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int a = accepted[(size_t)c * stride];
    k[c] = (float)log2((double)n_sub / (double)(a > 1 ? a : 1));
  }
}

}  // namespace
}  // namespace mri

extern "C" size_t mri_learned_moments_workspace_size(int cols) {
  return cols < 1 ? 0 : (size_t)mri::kMomChunks * cols * 2 * sizeof(double);
}

extern "C" int mri_learned_moments(const float* X, long long rows, int cols, int ld, float floor_sd, float* mean,
                                   float* inv_std, float* sd, void* workspace, size_t workspace_bytes, void* stream) {
  if (rows < 1 || cols < 1 || ld < cols || !(floor_sd >= 0.0f) || !X || !mean || !inv_std) return MRI_EINVAL;
  if (!workspace || workspace_bytes < mri_learned_moments_workspace_size(cols)) return MRI_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* part = static_cast<double*>(workspace);
  mri::moments_part_kernel<<<dim3((cols + 31) / 32, mri::kMomChunks), dim3(32, 8), 0, st>>>(X, rows, cols, ld, part);
  mri::moments_final_kernel<<<(cols + 127) / 128, 128, 0, st>>>(part, rows, cols, floor_sd, mean, inv_std, sd);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_learned_standardise(const float* X, int ld, const int32_t* perm, long long rows_out, int used,
                                       const float* mean, const float* inv_std, float* out, int ld_out, void* stream) {
  if (rows_out < 0 || used < 0 || used > ld || used > ld_out || !X || !mean || !inv_std || !out) return MRI_EINVAL;
  if (rows_out == 0) return MRI_OK;
  mri::standardise_kernel<<<grid_for(rows_out * ld_out), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      X, ld, perm, rows_out, used, mean, inv_std, out, ld_out);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_learned_step_targets(const int32_t* accepted, int stride, int ncell, int n_sub, float* k,
                                        void* stream) {
  if (ncell < 0 || stride < 1 || n_sub < 1) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  if (!accepted || !k) return MRI_EINVAL;
  mri::step_targets_kernel<<<grid_for(ncell), 256, 0, static_cast<cudaStream_t>(stream)>>>(accepted, stride, ncell,
                                                                                         n_sub, k);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_learned_step_exp(const float* yhat, int ld_yhat, int col, int ncell, float tmean, float tstd,
                                    int kmin, int kmax, int8_t* step_exp, void* stream) {
  if (ncell < 0 || col < 0 || ld_yhat <= col || kmin > kmax || kmin < -128 || kmax > 127) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  if (!yhat || !step_exp) return MRI_EINVAL;
  mri::step_exp_kernel<<<grid_for(ncell), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      yhat, ld_yhat, col, ncell, tmean, tstd, kmin, kmax, step_exp);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_learned_features(const double* y, const double* p, const double* phi, int K, int ncell, int n,
                                    double Hstage, const float* mean, const float* inv_std, float* x, int ld_x,
                                    void* stream) {
  if (ncell < 0 || n < 2 || K < 0 || K > 4 || ld_x < 2 * n + 2 || !(Hstage > 0)) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  if (!y || !p || !mean || !inv_std || !x || (K > 0 && !phi)) return MRI_EINVAL;
  mri::features_kernel<<<grid_for((long long)ncell * ld_x), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      y, p, phi, K, ncell, n, Hstage, mean, inv_std, x, ld_x);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_learned_targets(const double* y_in, const double* y_seq, int G, int ncell, int n,
                                   const float* tmean, const float* tinv_std, float* t, int ld_t, void* stream) {
  if (ncell < 0 || n < 1 || G < 1 || ld_t < G * n) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  if (!y_in || !y_seq || !tmean || !tinv_std || !t) return MRI_EINVAL;
  mri::targets_kernel<<<grid_for((long long)ncell * ld_t), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      y_in, y_seq, G, ncell, n, tmean, tinv_std, t, ld_t);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_learned_guess(const double* y_in, const float* yhat, int ld_yhat, int G, int ncell, int n,
                                 const float* tmean, const float* tstd, double* guess, void* stream) {
  if (ncell < 0 || n < 1 || G < 1 || ld_yhat < G * n) return MRI_EINVAL;
  if (ncell == 0) return MRI_OK;
  if (!y_in || !yhat || !tmean || !tstd || !guess) return MRI_EINVAL;
  mri::guess_kernel<<<grid_for((long long)ncell * G * n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      y_in, yhat, ld_yhat, G, ncell, n, tmean, tstd, guess);
  return cudaGetLastError() == cudaSuccess ? MRI_OK : MRI_ECUDA;
}

extern "C" int mri_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* C, int ldc,
                             int* err, void* stream) {
  if (!A || !B || !C || !err || M < 1 || N < 16 || N > 256 || N % 16 != 0 || K < 1 || K % 8 != 0 || lda < K ||
      ldb < K || lda % 8 != 0 || ldb % 8 != 0 || ldc < N)
    return MRI_EINVAL;
  const int used = gemm(static_cast<const __nv_bfloat16*>(A), lda, static_cast<const __nv_bfloat16*>(B), ldb, M, N,
                        K, EPI_F32, nullptr, C, ldc, nullptr, 0, 1, 0, err, static_cast<cudaStream_t>(stream));
  return used < 0 ? MRI_ECUDA : MRI_OK;
}
