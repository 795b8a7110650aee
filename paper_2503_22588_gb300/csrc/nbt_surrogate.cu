// nbt_surrogate.cu -- tensor-core kernels of the learned IG surrogate.
//
// This file holds the operand loaders and epilogues that turn the tcgen05
// GEMM of nbt_tc.cuh into the surrogate's layers, and their C-ABI entry
// points.  The paper has no learned component; the surrogate prunes
// candidate perspectives before exact raycasting (the exact IG of Section
// III re-scores the survivors).

#include <cuda_bf16.h>

#include <algorithm>

#include "nbt_internal.cuh"
#include "nbt_tc.cuh"

namespace nbt {
namespace {

using bf16 = __nv_bfloat16;

// Row-major K-major BF16 matrix [rows, K] with row stride ld elements
// (ld % 8 == 0, base 16-byte aligned, K % 8 == 0).
struct MatLoader {
  const bf16 *p;
  int rows, K, ld;
  __device__ __forceinline__ uint4 chunk(int r, int kc) const {
    const int k = kc * 8;
    if (r >= rows || k >= K) return make_uint4(0u, 0u, 0u, 0u);
    return __ldg((const uint4 *)(p + (size_t)r * ld + k));
  }
};

// FP32 row-major store of C[m, n] for n < N.
struct StoreF32 {
  float *c;
  int N, ldc;
  __device__ __forceinline__ void row(int m, int n0, const float v[16]) const {
    float *dst = c + (size_t)m * ldc + n0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (n0 + i < N) dst[i] = v[i];
  }
};

int *g_err[64] = {nullptr};

int dev_err_word(int **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return NBT_ECUDA;
  if (!g_err[dev]) {
    int *p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return NBT_ENOMEM;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return NBT_ECUDA;
    g_err[dev] = p;
  }
  *out = g_err[dev];
  return NBT_OK;
}

template <int BN, class LA, class LB, class EP>
int launch_gemm(const LA &la, const LB &lb, const EP &ep, int M, int K, cudaStream_t stream) {
  int *err = nullptr;
  int rc = dev_err_word(&err);
  if (rc != NBT_OK) return rc;
  const size_t smem = tc::gemm_smem_bytes(BN);
  auto kern = tc::gemm_kernel<BN, LA, LB, EP>;
  NBT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)((M + tc::kBM - 1) / tc::kBM);
  kern<<<grid, tc::kThreads, smem, stream>>>(la, lb, ep, M, K, err);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

}  // namespace
}  // namespace nbt

using namespace nbt;

extern "C" {

// Test entry point: C[M, N] (FP32, row stride N) = A[M, K] * B[N, K]^T with
// BF16 row-major A and B (row strides K).  N in [1, 256]; K % 8 == 0.
int nbt_tc_gemm(const void *a, const void *b, float *c, int32_t m, int32_t n, int32_t k, void *stream) {
  if (!a || !b || !c || m < 1 || n < 1 || n > 256 || k < 8 || (k % 8) != 0) return NBT_EINVAL;
  if (((uintptr_t)a & 15u) || ((uintptr_t)b & 15u)) return NBT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const MatLoader la{(const bf16 *)a, m, k, k};
  const MatLoader lb{(const bf16 *)b, n, k, k};
  const StoreF32 ep{c, n, n};
  if (n <= 16) return launch_gemm<16>(la, lb, ep, m, k, s);
  if (n <= 32) return launch_gemm<32>(la, lb, ep, m, k, s);
  if (n <= 64) return launch_gemm<64>(la, lb, ep, m, k, s);
  if (n <= 128) return launch_gemm<128>(la, lb, ep, m, k, s);
  return launch_gemm<256>(la, lb, ep, m, k, s);
}

// Device error word of the tensor-core kernels on the current device: 1
// after a bounded wait gave up.  Reading clears it.
int nbt_tc_error(int32_t *flag) {
  if (!flag) return NBT_EINVAL;
  int *err = nullptr;
  int rc = dev_err_word(&err);
  if (rc != NBT_OK) return rc;
  int v = 0;
  NBT_CUDA_TRY(cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) NBT_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
  *flag = v;
  return NBT_OK;
}

}  // extern "C"
