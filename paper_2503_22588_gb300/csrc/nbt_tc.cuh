// nbt_tc.cuh -- 5th-generation tensor-core (tcgen05) GEMM for the IG surrogate.
//
// C[M, N] = A[M, K] * B[N, K]^T with BF16 operands and FP32 accumulation in
// tensor memory (TMEM), written directly in PTX for sm_103a:
//   - a CTA of 128 threads owns one 128-row x BN-column tile of C (BN <=
//     256, one TMEM accumulator of BN FP32 columns) and one split of K;
//   - K advances in stages of 64: all threads gather the A and B stage
//     (through loader functors: a plain matrix, or an implicit-GEMM view of
//     a convolution) into shared memory in the canonical no-swizzle K-major
//     layout, then one thread issues four tcgen05.mma (K = 16 each) and
//     commits them to the stage's mbarrier; two stages alternate, so the
//     gather of stage k+1 overlaps the MMAs of stage k (gemm_kernel, for
//     loaders that must transpose); loaders that can name a 16-byte source
//     per chunk get four stages filled by cp.async (gemm_async_kernel);
//   - the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w .. 32w+31 = rows of the tile) and hands each row's values
//     to an epilogue functor.
// Every mbarrier wait is bounded (%globaltimer, c_wait_ns); on timeout the
// kernel sets an error word, waits once more (bounded) for its MMAs and
// frees its TMEM.
// The helpers below (descriptors, MMAs with A in shared or tensor memory,
// TMEM loads and stores, bounded waits) also serve the fused surrogate
// kernels.
//
// Shared-memory layout of one operand stage (rows R = 128 for A, BN for B):
// four K16 blocks of R x 16 BF16; inside a block, 8-row x 16-byte core
// matrices, the two K-halves of an 8-row group adjacent (128 B apart, the
// descriptor's leading byte offset) and 8-row groups 256 B apart (stride
// byte offset).

#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace nbt {
namespace tc {

constexpr int kBM = 128;        // tile rows (UMMA M)
constexpr int kBK = 64;         // K per stage (4 MMAs of K = 16)
constexpr int kThreads = 128;
constexpr uint64_t kDefaultWaitNs = 2000000000ull;  // default bound on any mbarrier wait: 2 s

// The bound in use (nanoseconds of %globaltimer), per device; set by
// nbt_tc_set_wait_limit.  This header is compiled into one translation unit.
__constant__ uint64_t c_wait_ns = kDefaultWaitNs;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor: start address, leading byte offset (K
// direction), stride byte offset (M/N direction), descriptor version 1, no
// swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = FP32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Bounded wait for the completion of phase `parity`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer() - t0 > c_wait_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Make this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy).
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The same with A in tensor memory (lane m = row m, BF16 element k of the
// row in 32-bit column k / 2, even k in the low half).
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Four consecutive 32-bit columns of this thread's TMEM lane (warp-collective;
// the address names the warp's lane quarter).  Completion: tmem_wait_st().
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Arrive on `bar` once every tcgen05.mma this thread issued so far is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 4 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float v[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__host__ __device__ constexpr int tmem_cols(int bn) { return bn <= 32 ? 32 : (bn <= 64 ? 64 : (bn <= 128 ? 128 : 256)); }

// Byte offset of 16-byte chunk (row r, chunk kc of the stage) in an operand
// stage with R rows: K16 block kc / 2, 8-row group r / 8, K-half kc % 2.
__device__ __forceinline__ uint32_t stage_off(int r, int kc, int rows) {
  return (uint32_t)((kc >> 1) * (rows * 32) + (r >> 3) * 256 + (kc & 1) * 128 + (r & 7) * 16);
}

__host__ __device__ constexpr size_t stage_bytes(int bn) { return (size_t)(kBM + bn) * kBK * 2; }
__host__ __device__ constexpr size_t gemm_smem_bytes(int bn) { return 2 * stage_bytes(bn) + 1024; }

// The GEMM kernel.  Grid: x over 128-row tiles of M, y over BN-column tiles
// of N, z over splits of K (kt_split stages of 64 each).
// LoadA / LoadB: `template <int ROWS> void fill(uint8_t *stage, int row0,
// int kc0, int tid) const` writes rows row0 .. row0+ROWS-1, K chunks
// kc0 .. kc0+7 (8 BF16 each, zero outside the operand) into the stage.
// Epi: `void row(int m, int n, const float v[16], int z) const` receives
// columns n .. n+15 of row m < M (columns past the real N are the loader's
// zeros' products; the epilogue skips them).
template <int BN, class LoadA, class LoadB, class Epi>
__global__ void __launch_bounds__(kThreads) gemm_kernel(LoadA la, LoadB lb, Epi epi, int M, int K, int kt_split,
                                                        int *err) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN, z = blockIdx.z;
  constexpr uint32_t NCOLS = (uint32_t)tmem_cols(BN);
  if (warp == 0) tmem_alloc(&tmem_base, NCOLS);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_bf16(kBM, BN);
  const int kt_all = (K + kBK - 1) / kBK;
  const int kt_begin = z * kt_split;
  const int kt_end = min(kt_all, kt_begin + kt_split);
  bool ok = true;
  int issued = 0;
  for (int kt = kt_begin; kt < kt_end; ++kt) {
    const int it = kt - kt_begin, s = it & 1;
    if (it >= 2) ok = mbar_wait(&mbar[s], (uint32_t)((it - 2) >> 1) & 1u);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    uint8_t *sa = smem + s * stage_bytes(BN);
    uint8_t *sb = sa + kBM * kBK * 2;
    const int kc0 = kt * (kBK / 8);
    la.template fill<kBM>(sa, m0, kc0, tid);
    lb.template fill<BN>(sb, n0, kc0, tid);
    fence_smem_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = sdesc(a0 + kk * (kBM * 32), 128, 256);
        const uint64_t bd = sdesc(b0 + kk * (BN * 32), 128, 256);
        mma_bf16(tmem, ad, bd, idesc, (it | kk) != 0 ? 1u : 0u);
      }
      mma_commit(&mbar[s]);
    }
    ++issued;
  }
  if (ok && issued > 0) {
    const int kl = issued - 1;
    ok = mbar_wait(&mbar[kl & 1], (uint32_t)(kl >> 1) & 1u);
  }
  ok = __syncthreads_and(ok) != 0;
  fence_after_sync();
  if (ok) {
    const int row = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int nn = 0; nn < BN; nn += 16) {
      float v[16];
      if (issued > 0) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)nn, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.0f;  // empty K split: contributes zeros
      }
      if (row < M) epi.row(row, n0 + nn, v, z);
    }
  } else {
    if (tid == 0) atomicExch(err, 1);
    // wait (bounded) for every committed stage before freeing the accumulator
    for (int k = (issued > 2 ? issued - 2 : 0); k < issued; ++k) (void)mbar_wait(&mbar[k & 1], (uint32_t)(k >> 1) & 1u);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------------------
// Asynchronous variant for loaders whose chunks are plain 16-byte copies
// (`const void *src(int row, int kchunk)`, nullptr where the operand is
// zero, and `const void *base()`, any valid address of the operand): the
// stages are filled with cp.async, kAsyncStages deep, so the gathers of the
// next stages are in flight while the tensor core works on the current one.
// A stage is refilled only after the mbarrier of the MMAs that read it has
// completed.
// ---------------------------------------------------------------------------
constexpr int kAsyncStages = 4;

__host__ __device__ constexpr size_t gemm_async_smem_bytes(int bn) { return kAsyncStages * stage_bytes(bn) + 1024; }

// 16-byte global -> shared copy; zero-fills when !valid (no bytes are read).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int ROWS, class L>
__device__ __forceinline__ void fill_async(const L &l, uint8_t *stage, int row0, int kc0, int tid) {
  const uint32_t base = smem_u32(stage);
  for (int c = tid; c < ROWS * 8; c += kThreads) {
    const int r = c % ROWS, kc = c / ROWS;
    const void *p = l.src(row0 + r, kc0 + kc);
    cp_async16(base + stage_off(r, kc, ROWS), p ? p : l.base(), p != nullptr);
  }
}

template <int BN, class LoadA, class LoadB, class Epi>
__global__ void __launch_bounds__(kThreads) gemm_async_kernel(LoadA la, LoadB lb, Epi epi, int M, int K,
                                                              int kt_split, int *err) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N");
  constexpr int S = kAsyncStages;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t mbar[S];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN, z = blockIdx.z;
  constexpr uint32_t NCOLS = (uint32_t)tmem_cols(BN);
  if (warp == 0) tmem_alloc(&tmem_base, NCOLS);
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < S; ++i) mbar_init(&mbar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = idesc_bf16(kBM, BN);
  const int kt_all = (K + kBK - 1) / kBK;
  const int kt_begin = z * kt_split;
  const int nk = max(0, min(kt_all, kt_begin + kt_split) - kt_begin);
  auto load_stage = [&](int it) {
    uint8_t *sa = smem + (it % S) * stage_bytes(BN);
    const int kc0 = (kt_begin + it) * (kBK / 8);
    fill_async<kBM>(la, sa, m0, kc0, tid);
    fill_async<BN>(lb, sa + kBM * kBK * 2, n0, kc0, tid);
  };
#pragma unroll
  for (int it = 0; it < S - 1; ++it) {
    if (it < nk) load_stage(it);
    cp_async_commit();
  }
  bool ok = true;
  int issued = 0;
  for (int it = 0; it < nk; ++it) {
    cp_async_wait<S - 2>();   // this thread's copies of k-tile `it` have landed
    fence_smem_async();
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if (tid == 0) {
      fence_after_sync();
      const uint32_t a0 = smem_u32(smem + (it % S) * stage_bytes(BN));
      const uint32_t b0 = a0 + kBM * kBK * 2;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = sdesc(a0 + kk * (kBM * 32), 128, 256);
        const uint64_t bd = sdesc(b0 + kk * (BN * 32), 128, 256);
        mma_bf16(tmem, ad, bd, idesc, (it | kk) != 0 ? 1u : 0u);
      }
      mma_commit(&mbar[it % S]);
    }
    ++issued;
    // refill the stage the MMAs of k-tile it - 1 read, once they are done
    const int nxt = it + S - 1;
    if (nxt < nk) {
      if (it >= 1) ok = mbar_wait(&mbar[(it - 1) % S], (uint32_t)((it - 1) / S) & 1u);
      if (ok) load_stage(nxt);
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  if (ok && issued > 0) {
    const int kl = issued - 1;
    ok = mbar_wait(&mbar[kl % S], (uint32_t)(kl / S) & 1u);
  }
  ok = __syncthreads_and(ok) != 0;
  fence_after_sync();
  if (ok) {
    const int row = m0 + warp * 32 + (tid & 31);
#pragma unroll 1
    for (int nn = 0; nn < BN; nn += 16) {
      float v[16];
      if (issued > 0) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)nn, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.0f;  // empty K split: contributes zeros
      }
      if (row < M) epi.row(row, n0 + nn, v, z);
    }
  } else {
    if (tid == 0) atomicExch(err, 1);
    // wait (bounded) for every committed stage before freeing the accumulator
    for (int k = (issued > S ? issued - S : 0); k < issued; ++k) (void)mbar_wait(&mbar[k % S], (uint32_t)(k / S) & 1u);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

}  // namespace tc
}  // namespace nbt
