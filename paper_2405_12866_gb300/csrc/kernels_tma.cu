// Backward step of the sweep (Section 3 of the paper) with the state rows
// staged in shared memory by the bulk-copy (TMA) engine.
//
// Each unit of work is the 2^U rows (all M samples each) spanned by the
// qubits of gate k+1 (whose new value is carried into Phi) and gate k (whose
// environment is reduced).  A row is M contiguous samples, so it moves as one
// cp.async.bulk of M * sizeof(complex) bytes.  One producer warp fills a ring
// of shared-memory stages (Phi rows and B_{k-1} rows of several units per
// stage), tracked by mbarriers with transaction counts; four consumer warps
// compute from shared memory: every consumer thread owns one sample of one
// unit and so holds all 2^U rows of its sample - no shuffles, no register
// staging of loads, and the bytes in flight are limited by shared memory,
// not registers.
//
// Every mbarrier wait is bounded.  A wait that runs out sets the run's error
// word (the host turns it into QFS_ETIMEOUT), the producer then waits, again
// with a bound, for the copies it issued, and the block returns.
#include "polar4.cuh"
#include "qfs_common.cuh"
#include "qfs_kernels.h"

#include <algorithm>
#include <cstdlib>

namespace qfs {

namespace {

constexpr int kStages = 3;
constexpr int kConsumerWarps = 4;
constexpr int kThreads = 32 * (kConsumerWarps + 1);
constexpr long long kWaitLimit = 1LL << 22;  // try_wait rounds before giving up
constexpr int kStageBytes = 32 * 1024;       // target bytes (Phi + B) per stage

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Global -> shared bulk copy completing on `bar` (16-byte aligned, size a
// multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace

struct TmaBwdArgs {
  BwdArgs b;
  int ups;        // units per stage
  int row_bytes;  // M * sizeof(complex)
  int* err;       // run error word: bit 0 = a bounded wait ran out
};

template <typename T, int U, int EA, int EB>
__global__ void __launch_bounds__(kThreads, 1) k_backward_tma(TmaBwdArgs ta) {
  using T2 = typename C2<T>::t;
  constexpr int ROWS = 1 << U;
  const BwdArgs& a = ta.b;
  const int s = blockIdx.y;
  if (a.active && !a.active[s]) return;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ uint64_t full[kStages], empty[kStages];
  __shared__ T2 gs[16];
  __shared__ double red[kConsumerWarps][32];
  __shared__ double2 sm_polar[32];
  __shared__ int is_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M = a.g.M, UPS = ta.ups;
  const size_t stage_elems = (size_t)UPS * 2 * ROWS * M;
  T2* stage_base = reinterpret_cast<T2*>(dsm);
  auto srow = [&](int st, int uu, int arr, int t) {  // row t of array arr (0 Phi, 1 B) of unit uu
    return stage_base + (size_t)st * stage_elems + ((size_t)(uu * 2 + arr) * ROWS + t) * M;
  };
  const bool has_gate = a.gates != nullptr;
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 16)
    gs[tid] = has_gate ? reinterpret_cast<const T2*>(a.gates)[s * a.gate_stride + tid] : T2{};
  __syncthreads();

  const T2* B = reinterpret_cast<const T2*>(a.bprev) + s * a.bprev_stride;
  const T2* P = reinterpret_cast<const T2*>(a.phi_in) + s * a.phi_in_stride;
  T2* Po = a.phi_out ? reinterpret_cast<T2*>(a.phi_out) + s * a.g.sN : nullptr;
  auto row_of = [&](int r, int t) {
    uint32_t base = (uint32_t)r;
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int p = a.g.ins[i];
      base = ((base >> p) << (p + 1)) | (base & ((1u << p) - 1u));
    }
#pragma unroll
    for (int i = 0; i < U; ++i)
      if ((t >> i) & 1) base |= 1u << a.g.pos[i];
    return base;
  };
  const int u0 = blockIdx.x * a.chunk;
  const int u1 = min(u0 + a.chunk, a.units_per_start);
  const int nsteps = u1 > u0 ? (u1 - u0 + UPS - 1) / UPS : 0;

  T acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = T(0);

  if (warp == kConsumerWarps) {
    // Producer warp: lane 0 manages the barriers, all lanes issue copies.
    int issued = 0;
    for (int i = 0; i < nsteps; ++i) {
      const int st = i % kStages;
      int ok = 1;
      if (lane == 0) {
        if (i >= kStages && !mbar_wait(&empty[st], ((i / kStages) - 1) & 1)) ok = 0;
        if (ok) {
          const int nu = min(UPS, u1 - (u0 + i * UPS));
          mbar_arrive_expect_tx(&full[st], (unsigned)(nu * ROWS * 2 * ta.row_bytes));
        }
      }
      ok = __shfl_sync(FULL, ok, 0);
      if (!ok) {
        if (lane == 0) atomicOr(ta.err, 1);
        break;
      }
      const int ub = u0 + i * UPS;
      const int nu = min(UPS, u1 - ub);
      for (int c = lane; c < nu * ROWS * 2; c += 32) {
        const int uu = c / (ROWS * 2), rem = c - uu * ROWS * 2, arr = rem / ROWS, t = rem - arr * ROWS;
        const size_t row = row_of(ub + uu, t);
        const T2* src = (arr == 0 ? P : B) + row * M;
        bulk_g2s(srow(st, uu, arr, t), src, (unsigned)ta.row_bytes, &full[st]);
      }
      issued = i + 1;
    }
    // Wait (bounded) for copies still landing in this block's shared memory
    // before the block may exit: the last min(issued, kStages) stages.
    if (lane == 0) {
      for (int i = max(0, issued - kStages); i < issued; ++i)
        if (!mbar_wait(&full[i % kStages], (i / kStages) & 1)) atomicOr(ta.err, 1);
    }
    __syncwarp();
  } else {
    // Consumers: thread tid handles (unit uu, sample j) pairs of each stage.
    const T2* gsp = gs;
    for (int i = 0; i < nsteps; ++i) {
      const int st = i % kStages;
      if (!mbar_wait(&full[st], (i / kStages) & 1)) {
        if (lane == 0) atomicOr(ta.err, 1);
        break;
      }
      const int ub = u0 + i * UPS;
      const int nu = min(UPS, u1 - ub);
      for (int w = tid; w < nu * M; w += 32 * kConsumerWarps) {
        const int uu = w / M, j = w - uu * M;
        T2* ph = srow(st, uu, 0, 0) + j;
        const T2* bb = srow(st, uu, 1, 0) + j;
        if (has_gate) {
          // Phi_k = g_{k+1}^dagger Phi_{k+1} on local bits U-1, U-2.
#pragma unroll
          for (int t0 = 0; t0 < ROWS / 4; ++t0) {
            T2 x[4], y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = ph[(size_t)((q << (U - 2)) | t0) * M];
#pragma unroll
            for (int yy = 0; yy < 4; ++yy) {
              T2 t{T(0), T(0)};
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const T2 g = gsp[4 * q + yy];  // conj(g[q][yy]) = g^dagger[yy][q]
                t.x += g.x * x[q].x + g.y * x[q].y;
                t.y += g.x * x[q].y - g.y * x[q].x;
              }
              y[yy] = t;
            }
#pragma unroll
            for (int yy = 0; yy < 4; ++yy) {
              const int t = (yy << (U - 2)) | t0;
              ph[(size_t)t * M] = y[yy];
              if (Po) Po[(size_t)row_of(ub + uu, t) * M + j] = y[yy];
            }
          }
        }
        // E_k[x][y] += B[x] conj(Phi_k[y]) over the groups of gate k.
#pragma unroll
        for (int jg = 0; jg < ROWS / 4; ++jg) {
          int rest = 0, bit = 0;
#pragma unroll
          for (int i2 = 0; i2 < U; ++i2) {
            if (i2 == EA || i2 == EB) continue;
            rest |= ((jg >> bit) & 1) << i2;
            ++bit;
          }
          T2 bx[4], py[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int t = rest | ((q >> 1) << EA) | ((q & 1) << EB);
            bx[q] = bb[(size_t)t * M];
            py[q] = ph[(size_t)t * M];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              cfma_conj(acc[2 * (4 * x + y)], acc[2 * (4 * x + y) + 1], bx[x], py[y]);
            }
        }
      }
      // Shared-memory writes of this stage (Phi_k) must be ordered before the
      // bulk copies that will refill it.
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
  }

  // Block reduction of the environment partials (consumer warps only).
  if (warp < kConsumerWarps) red[warp][lane] = (double)warp_reduce_scatter32<T>(acc, lane);
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
    for (int w = 0; w < kConsumerWarps; ++w) t += red[w][lane];
    reinterpret_cast<T*>(a.partials)[((long long)s * a.nblk + blockIdx.x) * 32 + lane] = (T)t;
  }
  if (a.fuse) {
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(a.counters + s, 1u) == (unsigned)(a.nblk - 1);
    __syncthreads();
    if (is_last && warp == 0) {
      __threadfence();
      update_one_start<T, sizeof(T) == 4 ? 1 : 2, true>(a.upd, s, sm_polar);
      if (lane == 0) a.counters[s] = 0u;
    }
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The same backward step with the rows staged by per-thread 16-byte
// asynchronous copies (cp.async) in a kStages-deep pipeline: every thread
// issues copies for the stage kStages-1 ahead of the one it computes, so
// many kilobytes per SM are in flight without holding registers, and no
// thread ever waits on a flag.
template <typename T, int U, int EA, int EB>
__global__ void __launch_bounds__(128, 1) k_backward_cpa(TmaBwdArgs ta) {
  using T2 = typename C2<T>::t;
  constexpr int ROWS = 1 << U;
  constexpr int NT = 128;
  const BwdArgs& a = ta.b;
  const int s = blockIdx.y;
  if (a.active && !a.active[s]) return;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ T2 gs[16];
  __shared__ double red[4][32];
  __shared__ double2 sm_polar[32];
  __shared__ int is_last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M = a.g.M, UPS = ta.ups;
  const int chunks_per_row = ta.row_bytes / 16;
  const size_t stage_elems = (size_t)UPS * 2 * ROWS * M;
  T2* stage_base = reinterpret_cast<T2*>(dsm);
  auto srow = [&](int st, int uu, int arr, int t) {
    return stage_base + (size_t)st * stage_elems + ((size_t)(uu * 2 + arr) * ROWS + t) * M;
  };
  const bool has_gate = a.gates != nullptr;
  if (tid < 16)
    gs[tid] = has_gate ? reinterpret_cast<const T2*>(a.gates)[s * a.gate_stride + tid] : T2{};
  const T2* B = reinterpret_cast<const T2*>(a.bprev) + s * a.bprev_stride;
  const T2* P = reinterpret_cast<const T2*>(a.phi_in) + s * a.phi_in_stride;
  T2* Po = a.phi_out ? reinterpret_cast<T2*>(a.phi_out) + s * a.g.sN : nullptr;
  auto row_of = [&](int r, int t) {
    uint32_t base = (uint32_t)r;
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int p = a.g.ins[i];
      base = ((base >> p) << (p + 1)) | (base & ((1u << p) - 1u));
    }
#pragma unroll
    for (int i = 0; i < U; ++i)
      if ((t >> i) & 1) base |= 1u << a.g.pos[i];
    return base;
  };
  const int u0 = blockIdx.x * a.chunk;
  const int u1 = min(u0 + a.chunk, a.units_per_start);
  const int nsteps = u1 > u0 ? (u1 - u0 + UPS - 1) / UPS : 0;
  auto issue = [&](int i) {
    if (i < nsteps) {
      const int st = i % kStages;
      const int ub = u0 + i * UPS;
      const int nu = min(UPS, u1 - ub);
      const int total = nu * 2 * ROWS * chunks_per_row;
      for (int c = tid; c < total; c += NT) {
        const int rowi = c / chunks_per_row, ch = c - rowi * chunks_per_row;
        const int uu = rowi / (2 * ROWS), rem = rowi - uu * 2 * ROWS, arr = rem / ROWS, t = rem - arr * ROWS;
        const size_t row = row_of(ub + uu, t);
        const T2* src = (arr == 0 ? P : B) + row * M;
        cp_async16(reinterpret_cast<char*>(srow(st, uu, arr, t)) + ch * 16,
                   reinterpret_cast<const char*>(src) + ch * 16);
      }
    }
    cp_async_commit();  // one group per stage (possibly empty) keeps the count aligned
  };

  T acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = T(0);
#pragma unroll
  for (int i = 0; i < kStages - 1; ++i) issue(i);
  __syncthreads();  // gs visible
  for (int i = 0; i < nsteps; ++i) {
    cp_async_wait<kStages - 2>();  // stage i has landed (this thread's copies)
    __syncthreads();               // ... and every thread's
    const int st = i % kStages;
    const int ub = u0 + i * UPS;
    const int nu = min(UPS, u1 - ub);
    for (int w = tid; w < nu * M; w += NT) {
      const int uu = w / M, j = w - uu * M;
      T2* ph = srow(st, uu, 0, 0) + j;
      const T2* bb = srow(st, uu, 1, 0) + j;
      if (has_gate) {
#pragma unroll
        for (int t0 = 0; t0 < ROWS / 4; ++t0) {
          T2 x[4], y[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) x[q] = ph[(size_t)((q << (U - 2)) | t0) * M];
#pragma unroll
          for (int yy = 0; yy < 4; ++yy) {
            T2 t{T(0), T(0)};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const T2 g = gs[4 * q + yy];  // conj(g[q][yy]) = g^dagger[yy][q]
              t.x += g.x * x[q].x + g.y * x[q].y;
              t.y += g.x * x[q].y - g.y * x[q].x;
            }
            y[yy] = t;
          }
#pragma unroll
          for (int yy = 0; yy < 4; ++yy) {
            const int t = (yy << (U - 2)) | t0;
            ph[(size_t)t * M] = y[yy];
            if (Po) Po[(size_t)row_of(ub + uu, t) * M + j] = y[yy];
          }
        }
      }
#pragma unroll
      for (int jg = 0; jg < ROWS / 4; ++jg) {
        int rest = 0, bit = 0;
#pragma unroll
        for (int i2 = 0; i2 < U; ++i2) {
          if (i2 == EA || i2 == EB) continue;
          rest |= ((jg >> bit) & 1) << i2;
          ++bit;
        }
        T2 bx[4], py[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int t = rest | ((q >> 1) << EA) | ((q & 1) << EB);
          bx[q] = bb[(size_t)t * M];
          py[q] = ph[(size_t)t * M];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            cfma_conj(acc[2 * (4 * x + y)], acc[2 * (4 * x + y) + 1], bx[x], py[y]);
          }
      }
    }
    __syncthreads();  // stage i fully consumed before it is refilled
    issue(i + kStages - 1);
  }
  cp_async_wait<0>();

  red[warp][lane] = (double)warp_reduce_scatter32<T>(acc, lane);
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
    for (int w = 0; w < 4; ++w) t += red[w][lane];
    reinterpret_cast<T*>(a.partials)[((long long)s * a.nblk + blockIdx.x) * 32 + lane] = (T)t;
  }
  if (a.fuse) {
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(a.counters + s, 1u) == (unsigned)(a.nblk - 1);
    __syncthreads();
    if (is_last && warp == 0) {
      __threadfence();
      update_one_start<T, sizeof(T) == 4 ? 1 : 2, true>(a.upd, s, sm_polar);
      if (lane == 0) a.counters[s] = 0u;
    }
  }
}

namespace {

constexpr int kMaxDynSmem = kStages * kStageBytes;

bool g_use_bulk = false;  // true: one producer warp with cp.async.bulk; false: cp.async by all threads

template <typename T, int U, int EA, int EB>
void launch_tma_instance(const TmaBwdArgs& ta, dim3 grid, size_t smem, cudaStream_t st) {
  if (g_use_bulk) k_backward_tma<T, U, EA, EB><<<grid, kThreads, smem, st>>>(ta);
  else k_backward_cpa<T, U, EA, EB><<<grid, 128, smem, st>>>(ta);
}

template <typename T, int U, int EA, int EB>
void configure_instance() {
  cudaFuncSetAttribute(k_backward_tma<T, U, EA, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaxDynSmem);
  cudaFuncSetAttribute(k_backward_cpa<T, U, EA, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaxDynSmem);
}

template <typename T>
void configure_type() {
  configure_instance<T, 4, 1, 0>();
  configure_instance<T, 3, 2, 0>();
  configure_instance<T, 3, 0, 2>();
  configure_instance<T, 3, 1, 0>();
  configure_instance<T, 3, 0, 1>();
  configure_instance<T, 2, 1, 0>();
  configure_instance<T, 2, 0, 1>();
}

template <typename T>
void dispatch_tma(const TmaBwdArgs& ta, dim3 grid, size_t smem, cudaStream_t st) {
  const int U = ta.b.g.U, ea = ta.b.g.ea, eb = ta.b.g.eb;
  if (U == 4) launch_tma_instance<T, 4, 1, 0>(ta, grid, smem, st);
  else if (U == 3) {
    if (ea == 2 && eb == 0) launch_tma_instance<T, 3, 2, 0>(ta, grid, smem, st);
    else if (ea == 0 && eb == 2) launch_tma_instance<T, 3, 0, 2>(ta, grid, smem, st);
    else if (ea == 1 && eb == 0) launch_tma_instance<T, 3, 1, 0>(ta, grid, smem, st);
    else launch_tma_instance<T, 3, 0, 1>(ta, grid, smem, st);
  } else {
    if (ea == 1) launch_tma_instance<T, 2, 1, 0>(ta, grid, smem, st);
    else launch_tma_instance<T, 2, 0, 1>(ta, grid, smem, st);
  }
}

}  // namespace

void configure_tma_kernels() {
  if (const char* f = std::getenv("QFS_BULK_COPY")) g_use_bulk = std::atoi(f) != 0;
  configure_type<float>();
  configure_type<double>();
}

bool tma_backward_supported(Real r, int M, int U) {
  const int row_bytes = M * (r == R32 ? 8 : 16);
  const int unit_bytes = 2 * (1 << U) * row_bytes;
  return row_bytes % 16 == 0 && unit_bytes <= kStageBytes;
}

Shape make_tma_shape(int n, int M, int S, Real r, int num_sms, int U) {
  Shape sh;
  const int row_bytes = M * (r == R32 ? 8 : 16);
  const int unit_bytes = 2 * (1 << U) * row_bytes;
  sh.vec = kStageBytes / unit_bytes;  // units per stage (held in `vec`)
  sh.units_per_start = 1 << (n - U);
  sh.threads = kThreads;
  // About two blocks per SM (each holds kStages stages) over all starts.
  const long long want_blocks = 2LL * num_sms;
  const long long per_start = std::max(1LL, want_blocks / std::max(S, 1));
  long long chunk = (sh.units_per_start + per_start - 1) / per_start;
  if (chunk < 1) chunk = 1;
  sh.chunk = (int)chunk;
  sh.nblk = (sh.units_per_start + sh.chunk - 1) / sh.chunk;
  return sh;
}

void launch_backward_tma(Real r, const BwdGeom& g, const Shape& sh, int S, const void* bprev,
                         long long bprev_stride, const void* phi_in, long long phi_in_stride,
                         void* phi_out, const void* gates, long long gate_stride, void* partials,
                         int stream_b, const int* active, cudaStream_t st, const UpdateArgs* fuse,
                         unsigned* counters, int* err) {
  TmaBwdArgs ta;
  ta.b = BwdArgs{bprev, bprev_stride, phi_in, phi_in_stride, phi_out, gates, gate_stride,
                 partials, sh.nblk, g, sh.units_per_start, sh.chunk, stream_b, active,
                 fuse ? 1 : 0, counters, fuse ? *fuse : UpdateArgs{}};
  ta.ups = sh.vec;
  ta.row_bytes = g.M * (r == R32 ? 8 : 16);
  ta.err = err;
  const size_t smem = (size_t)kStages * ta.ups * 2 * (1 << g.U) * ta.row_bytes;
  dim3 grid(sh.nblk, S);
  if (r == R32) dispatch_tma<float>(ta, grid, smem, st);
  else dispatch_tma<double>(ta, grid, smem, st);
}

}  // namespace qfs
