// BF16 GEMMs on the fifth-generation tensor cores (tcgen05) for the learned
// warm start:  C[M x N] = A[M x K] * B[N x K]^T  (+ bias[N], optional GELU),
// A and B bf16 row-major (both K-major), accumulation in FP32 in tensor
// memory (TMEM).
//
// k_gemm_bf16_tma: a warp-specialised pipeline.  Warp 0
// issues TMA tile loads (128-byte swizzle) into a ring of kStages shared
// stages, each tracked by a "full" mbarrier (transaction bytes) and an
// "empty" mbarrier; warp 1 owns the TMEM accumulator (128 x BN fp32
// columns) and one of its threads issues the tcgen05.mma chain, releasing
// each stage with tcgen05.commit; warps 2-9 wait for the final commit and
// run the epilogue (tcgen05.ld, bias, GELU, stores in whole 128-byte lines
// through shared memory).  With split-K (grid z) each CTA reduces a K range
// and adds its tile into C32 with vector atomics (the first split adds the
// bias).

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <mutex>

#include "qfs_kernels.h"

namespace qfs {

namespace {

constexpr long long kGemmWaitLimit = 1LL << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

// The tanh form of GELU, 0.5 x (1 + tanh u) with u = sqrt(2/pi) (x +
// 0.044715 x^3), evaluated as the equal x / (1 + exp(-2u)): one exponential
// and one division instead of tanhf, ~1e-6 relative, far below the bf16
// rounding of the result.  exp(-2u) = inf for u < -44 gives -0.
__device__ __forceinline__ float gelu_tanh(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * fmaf(k1 * x, x * x, x);
  return __fdividef(x, 1.f + __expf(-2.f * u));
}

}  // namespace

// ------------------------------------------------------------ TMA pipeline

namespace {

// Warp 0: TMA producer; warp 1: MMA issuer; warps 2-9: epilogue (two per
// TMEM lane quadrant, each with half of the tile's columns).
constexpr int kBM = 128, kBK = 64, kStages = 4, kTmaThreads = 320;
// Row stride (floats) of an epilogue warp's 32 x 32 staging block: 16-byte
// aligned rows whose float4 accesses by 8 lanes cover all 32 banks.
constexpr int kTileStride = 36;
static_assert(8 * 32 * kTileStride * 4 <= kStages * kBM * kBK * 2, "epilogue blocks fit the operand stages");

template <int BN>
struct TmaCfg {
  static constexpr int kABytes = kBM * kBK * 2;
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kStageBytes = kABytes + kBBytes;
  // stages, 1024-byte alignment slack, barriers (256 B), the tile's bias
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 256 + BN * 4;
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                     ((uint32_t)(kBM >> 4) << 24);
};

// K-major operand with the 128-byte swizzle: rows of 64 bf16 (128 B), 8-row
// groups 1024 B apart (stride byte offset); the leading byte offset is not
// used by swizzled K-major layouts.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}

}  // namespace

template <int BN>
__global__ void __launch_bounds__(kTmaThreads, 1)
    k_gemm_bf16_tma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, GemmArgs g) {
  using Cfg = TmaCfg<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = su32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sb = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(sb + kStages * Cfg::kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* accf = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int KT = g.K / kBK;
  const int splitk = gridDim.z;
  const int kb = (int)((long long)blockIdx.z * KT / splitk), ke = (int)((long long)(blockIdx.z + 1) * KT / splitk);
  const int nk = ke - kb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init1(&full[s]);
      mbar_init1(&empty[s]);
    }
    mbar_init1(accf);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // Launched as a programmatic dependent of the previous kernel on the
  // stream: the set-up above may overlap its tail; no global memory is read
  // or written before that kernel has completed and its writes are visible.
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == 0) {
    // Producer: one thread issues the TMA loads of both operands per stage.
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % kStages;
        const unsigned ph = (unsigned)(i / kStages) & 1u;
        if (!mbar_wait_bounded(&empty[s], ph ^ 1u) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[s])),
                     "r"(Cfg::kStageBytes)
                     : "memory");
        const uint32_t dst = base + (uint32_t)(s * Cfg::kStageBytes);
        tma_load_2d(dst, &mapA, &full[s], (kb + i) * kBK, m0);
        tma_load_2d(dst + Cfg::kABytes, &mapB, &full[s], (kb + i) * kBK, n0);
        ++issued;
      }
      if (*abort_flag) {
        // Wait (bounded) for every copy this CTA issued before leaving.
        for (int i = 0; i < issued; ++i) mbar_wait_bounded(&full[i % kStages], (unsigned)(i / kStages) & 1u);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // MMA issuer.
    if (lane == 0) {
      for (int i = 0; i < nk; ++i) {
        const int s = i % kStages;
        const unsigned ph = (unsigned)(i / kStages) & 1u;
        if (!mbar_wait_bounded(&full[s], ph) || *abort_flag) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = base + (uint32_t)(s * Cfg::kStageBytes), b0 = a0 + Cfg::kABytes;
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          const uint64_t ad = desc_sw128(a0 + kk * 32), bd = desc_sw128(b0 + kk * 32);
          const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(Cfg::kIdesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&empty[s]))
                     : "memory");
      }
      // Arrives once every MMA issued above has completed.
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(accf))
                   : "memory");
      // Every operand load of this CTA is issued: the next kernel on the
      // stream may start its set-up (it waits for this grid to complete
      // before touching memory).
      asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    __syncwarp();
  } else {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the
    // tile) and columns half * BN/2 .. + BN/2 - 1.  The bias (added by the
    // first K split only) is staged in shared memory while the MMAs run.
    const int q = warp & 3, half = (warp - 2) >> 2;
    float* stile = reinterpret_cast<float*>(sb) + (warp - 2) * 32 * kTileStride;
    float* sbias = reinterpret_cast<float*>(sb + kStages * Cfg::kStageBytes + 256);
    const bool add_bias = g.bias != nullptr && blockIdx.z == 0;
    if (add_bias)
      for (int j = threadIdx.x - 64; j < BN; j += kTmaThreads - 64) sbias[j] = g.bias[n0 + j];
    asm volatile("bar.sync 1, %0;" ::"n"(kTmaThreads - 64) : "memory");
    const bool ok = mbar_wait_bounded(accf, 0) && !*abort_flag;
    if (!ok) {
      *abort_flag = 1;
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr int HC = BN / 2;
      for (int cb = half * HC; cb < (half + 1) * HC; cb += 64) {
        uint32_t v[64];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cb;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t* w = v + 32 * hh;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
              "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
                "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]),
                "=r"(w[15]), "=r"(w[16]), "=r"(w[17]), "=r"(w[18]), "=r"(w[19]), "=r"(w[20]), "=r"(w[21]),
                "=r"(w[22]), "=r"(w[23]), "=r"(w[24]), "=r"(w[25]), "=r"(w[26]), "=r"(w[27]), "=r"(w[28]),
                "=r"(w[29]), "=r"(w[30]), "=r"(w[31])
              : "r"(taddr + 32u * hh)
              : "memory");
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // Each 32 x 32 block goes through this warp's slice of the (now idle)
        // operand stages: lane l writes its row, then eight lanes cover one
        // row's 128 bytes per store, so every store writes whole lines.
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int lc = cb + 32 * hh, col = n0 + lc;
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4) {
            float4 f = make_float4(__uint_as_float(v[32 * hh + 4 * j4]), __uint_as_float(v[32 * hh + 4 * j4 + 1]),
                                   __uint_as_float(v[32 * hh + 4 * j4 + 2]), __uint_as_float(v[32 * hh + 4 * j4 + 3]));
            if (add_bias) {
              f.x += sbias[lc + 4 * j4];
              f.y += sbias[lc + 4 * j4 + 1];
              f.z += sbias[lc + 4 * j4 + 2];
              f.w += sbias[lc + 4 * j4 + 3];
            }
            *reinterpret_cast<float4*>(stile + lane * kTileStride + 4 * j4) = f;
          }
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int r = 4 * it + (lane >> 3), c4 = lane & 7;
            const int grow = m0 + q * 32 + r;
            const float4 f = *reinterpret_cast<const float4*>(stile + r * kTileStride + 4 * c4);
            if (grow < g.M_valid) {
              float* d32 = g.C32 ? g.C32 + (size_t)grow * g.ldc + col + 4 * c4 : nullptr;
              if (splitk > 1) {
                atomicAdd(reinterpret_cast<float4*>(d32), f);
              } else {
                if (d32) *reinterpret_cast<float4*>(d32) = f;
                if (g.C16) {
                  float a0 = f.x, a1 = f.y, a2 = f.z, a3 = f.w;
                  if (g.gelu) {
                    a0 = gelu_tanh(a0);
                    a1 = gelu_tanh(a1);
                    a2 = gelu_tanh(a2);
                    a3 = gelu_tanh(a3);
                  }
                  const __nv_bfloat162 p0 = __floats2bfloat162_rn(a0, a1), p1 = __floats2bfloat162_rn(a2, a3);
                  *reinterpret_cast<uint2*>(g.C16 + (size_t)grow * g.ldc + col + 4 * c4) =
                      make_uint2(*reinterpret_cast<const uint32_t*>(&p0), *reinterpret_cast<const uint32_t*>(&p1));
                }
              }
            }
          }
          __syncwarp();
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) atomicOr(g.err, 1);
  if (warp == 1) {
    // After a give-up, let the MMAs already issued finish (bounded) before
    // the accumulator is released.
    if (lane == 0 && *abort_flag) mbar_wait_bounded(accf, 0);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Row-major bf16 matrix (rows x K, leading dimension ld) as TMA tiles of
// box_rows x 64 with the 128-byte swizzle.
bool encode_kmajor(CUtensorMap* map, const void* ptr, int rows, int K, int ld, int box_rows) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Encoded maps of recent operands (the training loop reuses the same
// buffers every step; encoding is host work on every launch otherwise).
// Keyed by everything the encoding reads; small, round-robin replacement.
struct MapKey {
  const void* ptr;
  int rows, K, ld, box_rows;
  bool operator==(const MapKey& o) const {
    return ptr == o.ptr && rows == o.rows && K == o.K && ld == o.ld && box_rows == o.box_rows;
  }
};
bool cached_kmajor(CUtensorMap* map, const void* ptr, int rows, int K, int ld, int box_rows) {
  constexpr int kSlots = 64;
  static std::mutex mu;
  static MapKey keys[kSlots];
  static CUtensorMap maps[kSlots];
  static int used = 0, next = 0;
  const MapKey k{ptr, rows, K, ld, box_rows};
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
      if (keys[i] == k) {
        *map = maps[i];
        return true;
      }
  }
  if (!encode_kmajor(map, ptr, rows, K, ld, box_rows)) return false;
  std::lock_guard<std::mutex> lock(mu);
  const int slot = used < kSlots ? used++ : (next++ % kSlots);
  keys[slot] = k;
  maps[slot] = *map;
  return true;
}

template <int BN>
cudaError_t launch_tma(const GemmArgs& g, int splitk, cudaStream_t st) {
  static const cudaError_t attr = cudaFuncSetAttribute(k_gemm_bf16_tma<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       TmaCfg<BN>::kSmem);
  if (attr != cudaSuccess) return attr;
  CUtensorMap ma, mb;
  if (!cached_kmajor(&ma, g.A, g.M, g.K, g.lda, kBM) || !cached_kmajor(&mb, g.B, g.N, g.K, g.ldb, BN))
    return cudaErrorInvalidValue;
  dim3 grid(g.N / BN, g.M / kBM, splitk);
  // Programmatic dependent launch: this GEMM's set-up may overlap the tail
  // of the previous kernel on the stream (the kernel waits for it before
  // any memory access).
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kTmaThreads);
  cfg.dynamicSmemBytes = TmaCfg<BN>::kSmem;
  cfg.stream = st;
  cudaLaunchAttribute pdl[1];
  pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  pdl[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_gemm_bf16_tma<BN>, ma, mb, g);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

int gemm_splitk_for(const GemmArgs& g, int num_sms) {
  if (g.C16 || g.gelu || !g.C32) return 1;  // (the bias is added by the first split)
  const int BN = g.N % 256 == 0 ? 256 : 128;
  const int tiles = (g.N / BN) * (g.M / kBM);
  const int KT = g.K / kBK;
  int s = 1;
  while (tiles * s * 2 <= num_sms && KT / (s * 2) >= 4) s *= 2;
  return s;
}

cudaError_t launch_gemm_bf16_tc(const GemmArgs& g, cudaStream_t st) {
  const int splitk = g.splitk > 1 ? g.splitk : 1;
  if (splitk > 1) {
    // The split CTAs add into C32, which starts from zero.
    const cudaError_t e = cudaMemset2DAsync(g.C32, (size_t)g.ldc * 4, 0, (size_t)g.N * 4, g.M_valid, st);
    if (e != cudaSuccess) return e;
  }
  return g.N % 256 == 0 ? launch_tma<256>(g, splitk, st) : launch_tma<128>(g, splitk, st);
}

}  // namespace qfs
