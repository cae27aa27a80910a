// BF16 GEMM on the fifth-generation tensor cores (tcgen05) for the learned
// warm start:  C[M x N] = A[M x K] * B[N x K]^T  (+ bias[N], optional GELU),
// A and B bf16 row-major (both K-major), accumulation in FP32 in tensor
// memory (TMEM).
//
// One CTA of 128 threads computes a 128 x 128 tile.  Per K step of 64 the
// threads stage the A and B tiles in shared memory in the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices, K-adjacent core
// matrices 128 B apart, 8-row groups 1024 B apart), one elected thread
// issues four tcgen05.mma (K = 16 each) into the TMEM accumulator and
// commits them to an mbarrier; thread 0 waits (bounded) for the commit and
// the block follows it before the shared tiles are rewritten.  The epilogue reads the
// accumulator with tcgen05.ld (each warp its 32 TMEM lanes = rows), applies
// bias and GELU and stores FP32 and/or BF16.  A wait that runs out sets the
// error word, and the CTA still frees its TMEM before returning.
#include <cuda_bf16.h>

#include "qfs_kernels.h"

namespace qfs {

namespace {

constexpr int kTM = 128, kTN = 128, kTK = 64;
constexpr long long kGemmWaitLimit = 1LL << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension
// (K) byte offset and stride (8-row group) byte offset, all >> 4; descriptor
// version 1; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = kTN, M = kTM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (long long i = 0; i < kGemmWaitLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ float gelu_tanh(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  return 0.5f * x * (1.f + tanhf(k0 * (x + k1 * x * x * x)));
}

}  // namespace

__global__ void __launch_bounds__(128, 1) k_gemm_bf16_tc(GemmArgs g) {
  __shared__ __align__(128) unsigned char sa[kTM * kTK * 2];
  __shared__ __align__(128) unsigned char sb[kTN * kTK * 2];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(kTN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const __nv_bfloat16* A = g.A;
  const __nv_bfloat16* B = g.B;
  unsigned phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < g.K; k0 += kTK) {
    // Stage A rows m0.., B rows n0.., columns k0..k0+63 as core matrices.
    for (int c = tid; c < kTM * (kTK / 8); c += 128) {
      const int r = c >> 3, kc = c & 7;
      const uint4 va = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * g.lda + k0 + kc * 8);
      *reinterpret_cast<uint4*>(sa + ((r >> 3) * 8 + kc) * 128 + (r & 7) * 16) = va;
      const uint4 vb = *reinterpret_cast<const uint4*>(B + (size_t)(n0 + r) * g.ldb + k0 + kc * 8);
      *reinterpret_cast<uint4*>(sb + ((r >> 3) * 8 + kc) * 128 + (r & 7) * 16) = vb;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int i = 0; i < kTK / 16; ++i) {
        const uint64_t ad = smem_desc(su32(sa) + i * 256, 128, 1024);
        const uint64_t bd = smem_desc(su32(sb) + i * 256, 128, 1024);
        const uint32_t acc = (k0 > 0 || i > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&mbar))
                   : "memory");
    }
    // Thread 0 waits (bounded) for the MMAs; the block follows its verdict,
    // so every thread leaves the loop at the same step.
    int mine = 1;
    if (tid == 0) mine = mbar_wait_bounded(&mbar, phase) ? 1 : 0;
    ok = __syncthreads_and(mine) != 0;
    if (!ok) {
      if (tid == 0) {
        atomicOr(g.err, 1);
        mbar_wait_bounded(&mbar, phase);  // give in-flight MMAs a second bounded chance
      }
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (ok) {
    // Epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31.
    const int row = m0 + warp * 32 + lane;
    for (int cb = 0; cb < kTN; cb += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
            "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
            "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
            "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < g.M_valid) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + cb + j;
          float x = __uint_as_float(v[j]);
          if (g.bias) x += g.bias[col];
          if (g.C32) g.C32[(size_t)row * g.ldc + col] = x;
          if (g.C16) g.C16[(size_t)row * g.ldc + col] = __float2bfloat16(g.gelu ? gelu_tanh(x) : x);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN) : "memory");
  }
}

void launch_gemm_bf16_tc(const GemmArgs& g, cudaStream_t st) {
  dim3 grid(g.N / kTN, g.M / kTM);
  k_gemm_bf16_tc<<<grid, 128, 0, st>>>(g);
}

}  // namespace qfs
