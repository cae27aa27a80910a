// One whole sweep (Section 3 of the paper) of every multistart as a single
// persistent, cooperative launch: a dataflow schedule instead of one launch
// per gate step.
//
// The sweep is a chain of steps per start: L-1 forward steps (B_k = g_k
// B_{k-1}), L backward steps (Phi_k = g_{k+1}^dagger Phi_{k+1}, environment of
// gate k from B_{k-1} and Phi_k, then the polar update of gate k) and, in
// complex64, the residual pass that gives the sample cost.  Steps of
// different starts are independent.  Every (step, start, chunk of rows) is a
// work item; items are numbered step-major, then start, then chunk, and
// handed out by one atomic counter.  An item waits (bounded) until its start
// has finished all earlier steps; the CTA that completes the last chunk of a
// backward step runs the gate update (one warp) and then publishes the step.
// Because items are taken in an order in which every dependency comes first
// and all CTAs are co-resident (cooperative launch), the smallest unfinished
// item can always proceed.  While one start waits for its update, the other
// starts' items keep the memory system busy, and no launch boundary, tail
// wave or idle update kernel sits between gate steps.
//
// Data written inside the launch (B list, Phi, gates, partial sums) is read
// back through L2 (ld.global.cg), never from a possibly stale L1 line.
// Every wait is bounded: when one runs out the CTA sets the run's error word
// and every CTA stops taking items; the host reports QFS_ETIMEOUT.
#include "polar4.cuh"
#include "qfs_common.cuh"
#include "qfs_kernels.h"

#include <algorithm>

namespace qfs {

namespace {

constexpr long long kDfSpinLimit = 1LL << 25;  // polls of 32+ ns before giving up (> 1 s)
constexpr int kDfThreads = 128;

template <typename T, int VEC> struct DfV;
template <> struct DfV<float, 2> { using t = float4; };
template <> struct DfV<float, 1> { using t = float2; };
template <> struct DfV<double, 1> { using t = double2; };

template <typename T, int VEC>
__device__ __forceinline__ void ldg(const typename C2<T>::t* p, typename C2<T>::t (&o)[VEC]) {
  using V = typename DfV<T, VEC>::t;
  const V v = __ldcg(reinterpret_cast<const V*>(p));
  if constexpr (VEC == 2) {
    o[0] = float2{v.x, v.y};
    o[1] = float2{v.z, v.w};
  } else {
    o[0] = v;
  }
}
template <typename T, int VEC>
__device__ __forceinline__ void stg(typename C2<T>::t* p, const typename C2<T>::t (&o)[VEC]) {
  using V = typename DfV<T, VEC>::t;
  if constexpr (VEC == 2) {
    __stcg(reinterpret_cast<V*>(p), V{o[0].x, o[0].y, o[1].x, o[1].y});
  } else {
    __stcg(reinterpret_cast<V*>(p), o[0]);
  }
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
struct DfShared {
  typename C2<T>::t gs[16];
  double red[4][32];
  double2 polar[32];
  long long item;
  int flag;
};

// Block-wide sum of 32 per-thread values (one per lane slot) into
// partials[slot * 32 + lane] by warp 0.
template <typename T, typename PT>
__device__ __forceinline__ void block_partials32(double mine, DfShared<T>& sh, PT* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  sh.red[warp][lane] = mine;
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kDfThreads / 32; ++w) t += sh.red[w][lane];
    __stcg(out + lane, (PT)t);
  }
}

// Gate of this start (16 complex) into shared memory.
template <typename T>
__device__ __forceinline__ void load_gate(const DfStep& st, int s, DfShared<T>& sh) {
  using T2 = typename C2<T>::t;
  if (threadIdx.x < 16)
    sh.gs[threadIdx.x] = st.gate ? __ldcg(reinterpret_cast<const T2*>(st.gate) + s * st.gate_stride + threadIdx.x)
                                 : T2{};
  __syncthreads();
}

// Forward rows of one chunk: Y = (g (x) I) X on the pair of st.fg.
template <typename T, int VEC>
__device__ void df_forward(const DfStep& st, int s, int c, DfShared<T>& sh) {
  using T2 = typename C2<T>::t;
  load_gate<T>(st, s, sh);
  T2 gr[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) gr[i] = sh.gs[i];
  const T2* X = reinterpret_cast<const T2*>(st.in) + s * st.in_stride;
  T2* Y = reinterpret_cast<T2*>(st.out) + s * st.fg.sN;
  const int MV = st.fg.M / VEC;
  const int u0 = c * st.chunk, u1 = min(u0 + st.chunk, st.units);
  for (int u = u0 + threadIdx.x; u < u1; u += kDfThreads) {
    const int r = u / MV, jv = u - r * MV;
    const uint32_t base = insert_two_zero_bits((uint32_t)r, st.fg.lo, st.fg.hi);
    uint32_t off[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const uint32_t row = base | ((uint32_t)(x >> 1) << st.fg.pos_a) | ((uint32_t)(x & 1) << st.fg.pos_b);
      off[x] = row * (uint32_t)st.fg.M + (uint32_t)jv * VEC;
    }
    T2 v[4][VEC];
#pragma unroll
    for (int x = 0; x < 4; ++x) ldg<T, VEC>(X + off[x], v[x]);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      T2 o[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        T2 acc = cmul(gr[4 * x], v[0][q]);
#pragma unroll
        for (int xp = 1; xp < 4; ++xp) {
          const T2 t = cmul(gr[4 * x + xp], v[xp][q]);
          acc.x += t.x;
          acc.y += t.y;
        }
        o[q] = acc;
      }
      stg<T, VEC>(Y + off[x], o);
    }
  }
}

// Backward step on 16-row units (gate k+1 and gate k on four distinct
// qubits): four lanes share a unit as in the per-step kernel; the partial
// sums of E_k go to partials slot (s, c).
template <typename T, int VEC>
__device__ void df_backward_q4(const DfStep& st, int s, int c, DfShared<T>& sh, T* part) {
  using T2 = typename C2<T>::t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qx = lane >> 3, v = lane & 7;
  load_gate<T>(st, s, sh);
  T2 gd[16];
#pragma unroll
  for (int y = 0; y < 4; ++y)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T2 t = sh.gs[4 * j + y];
      gd[4 * y + j] = T2{t.x, -t.y};
    }
  const T2* B = reinterpret_cast<const T2*>(st.in) + s * st.in_stride;
  const T2* P = reinterpret_cast<const T2*>(st.phi_in) + s * st.phi_in_stride;
  T2* Po = reinterpret_cast<T2*>(st.phi_out) + s * st.bg.sN;
  const uint32_t M = (uint32_t)st.bg.M;
  const uint32_t d0 = (1u << st.bg.pos[0]) * M, d1 = (1u << st.bg.pos[1]) * M;
  const uint32_t d2 = (1u << st.bg.pos[2]) * M, d3 = (1u << st.bg.pos[3]) * M;
  const uint32_t xoff = ((qx >> 1) ? d1 : 0u) + ((qx & 1) ? d0 : 0u);
  const uint32_t joff[4] = {0u, d2, d3, d3 + d2};
  T acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = T(0);
  const int MV = st.bg.M / VEC;
  const int u0 = c * st.chunk, u1 = min(u0 + st.chunk, st.units);
  auto unit_off = [&](int u) {
    const int r = u / MV, jv = u - r * MV;
    uint32_t base = (uint32_t)r;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = st.bg.ins[i];
      base = ((base >> p) << (p + 1)) | (base & ((1u << p) - 1u));
    }
    return base * M + (uint32_t)jv * VEC + xoff;
  };
  auto load_unit = [&](int u, T2 (&ph)[4][VEC], T2 (&b)[4][VEC]) {
    if (u < u1) {
      const uint32_t o = unit_off(u);
#pragma unroll
      for (int j = 0; j < 4; ++j) ldg<T, VEC>(P + o + joff[j], ph[j]);
#pragma unroll
      for (int j = 0; j < 4; ++j) ldg<T, VEC>(B + o + joff[j], b[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < VEC; ++q) ph[j][q] = b[j][q] = T2{T(0), T(0)};
    }
  };
  T2 phn[4][VEC], bn[4][VEC];
  int ub = u0 + warp * 8;
  if (ub < u1) load_unit(ub + v, phn, bn);
  for (; ub < u1; ub += 32) {
    const int u = ub + v;
    const bool valid = u < u1;
    T2 ph[4][VEC], b[4][VEC];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        ph[j][q] = phn[j][q];
        b[j][q] = bn[j][q];
      }
    if (ub + 32 < u1) load_unit(ub + 32 + v, phn, bn);
    const uint32_t base_off = valid ? unit_off(u) : 0u;
    {
      T2 nw[4][VEC];
#pragma unroll
      for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          T2 t = cmul(gd[4 * y], ph[0][q]);
#pragma unroll
          for (int j = 1; j < 4; ++j) {
            const T2 w = cmul(gd[4 * y + j], ph[j][q]);
            t.x += w.x;
            t.y += w.y;
          }
          nw[y][q] = t;
        }
#pragma unroll
      for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int q = 0; q < VEC; ++q) ph[y][q] = nw[y][q];
      if (valid) {
#pragma unroll
        for (int y = 0; y < 4; ++y) stg<T, VEC>(Po + base_off + joff[y], ph[y]);
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          T2 pp = ph[j][q];
          if (m) {
            pp.x = __shfl_xor_sync(FULL, pp.x, 8 * m);
            pp.y = __shfl_xor_sync(FULL, pp.y, 8 * m);
          }
          const T2 bb = b[j][q];
          acc[2 * m] += bb.x * pp.x + bb.y * pp.y;
          acc[2 * m + 1] += bb.y * pp.x - bb.x * pp.y;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    acc[i] += __shfl_xor_sync(FULL, acc[i], 1);
    acc[i] += __shfl_xor_sync(FULL, acc[i], 2);
    acc[i] += __shfl_xor_sync(FULL, acc[i], 4);
  }
  // Lane (x, 0) holds E[x][x^m]; gather them into lane slots 2(4x+y)+{0,1}.
  if (v == 0) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int e = 4 * qx + (qx ^ m);
      sh.red[warp][2 * e] = (double)acc[2 * m];
      sh.red[warp][2 * e + 1] = (double)acc[2 * m + 1];
    }
  }
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kDfThreads / 32; ++w) t += sh.red[w][lane];
    __stcg(part + lane, (T)t);
  }
}

template <int U, int EA, int EB>
__device__ __forceinline__ constexpr int df_spread_rest(int j) {
  int t = 0, bit = 0;
  for (int i = 0; i < U; ++i) {
    if (i == EA || i == EB) continue;
    t |= ((j >> bit) & 1) << i;
    ++bit;
  }
  return t;
}

// Backward step on 2^U-row units, one unit per thread (U = 2 or 3), or the
// residual pass (MODE 1: sum |g^dagger Phi - B|^2 into a double partial).
template <typename T, int VEC, int MODE, int U, int EA, int EB>
__device__ void df_backward_gen(const DfStep& st, int s, int c, DfShared<T>& sh, void* part) {
  using T2 = typename C2<T>::t;
  constexpr int ROWS = 1 << U;
  const int lane = threadIdx.x & 31;
  load_gate<T>(st, s, sh);
  const bool has_gate = st.gate != nullptr;
  auto gd = [&](int y, int yp) {
    const T2 t = sh.gs[4 * yp + y];
    return T2{t.x, -t.y};
  };
  const T2* B = reinterpret_cast<const T2*>(st.in) + s * st.in_stride;
  const T2* P = reinterpret_cast<const T2*>(st.phi_in) + s * st.phi_in_stride;
  T2* Po = st.phi_out ? reinterpret_cast<T2*>(st.phi_out) + s * st.bg.sN : nullptr;
  const uint32_t M = (uint32_t)st.bg.M;
  uint32_t dpos[U];
#pragma unroll
  for (int i = 0; i < U; ++i) dpos[i] = (1u << st.bg.pos[i]) * M;
  T acc[MODE == 0 ? 32 : 1];
#pragma unroll
  for (int i = 0; i < (MODE == 0 ? 32 : 1); ++i) acc[i] = T(0);
  const int MV = st.bg.M / VEC;
  const int u0 = c * st.chunk, u1 = min(u0 + st.chunk, st.units);
  for (int u = u0 + threadIdx.x; u < u1; u += kDfThreads) {
    const int r = u / MV, jv = u - r * MV;
    uint32_t base = (uint32_t)r;
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int p = st.bg.ins[i];
      base = ((base >> p) << (p + 1)) | (base & ((1u << p) - 1u));
    }
    const uint32_t base_off = base * M + (uint32_t)jv * VEC;
    auto off = [&](int t) {
      uint32_t o = base_off;
#pragma unroll
      for (int i = 0; i < U; ++i)
        if ((t >> i) & 1) o += dpos[i];
      return o;
    };
    T2 ph[ROWS][VEC];
#pragma unroll
    for (int t = 0; t < ROWS; ++t) ldg<T, VEC>(P + off(t), ph[t]);
    if (has_gate) {
#pragma unroll
      for (int t0 = 0; t0 < ROWS / 4; ++t0) {
        T2 nw[4][VEC];
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            T2 a2 = cmul(gd(y, 0), ph[(0 << (U - 2)) | t0][q]);
#pragma unroll
            for (int yp = 1; yp < 4; ++yp) {
              const T2 w = cmul(gd(y, yp), ph[(yp << (U - 2)) | t0][q]);
              a2.x += w.x;
              a2.y += w.y;
            }
            nw[y][q] = a2;
          }
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
          for (int q = 0; q < VEC; ++q) ph[(y << (U - 2)) | t0][q] = nw[y][q];
      }
      if (Po) {
#pragma unroll
        for (int t = 0; t < ROWS; ++t) stg<T, VEC>(Po + off(t), ph[t]);
      }
    }
    if constexpr (MODE == 0) {
#pragma unroll
      for (int j = 0; j < ROWS / 4; ++j) {
        const int rest = df_spread_rest<U, EA, EB>(j);
        T2 b[4][VEC];
#pragma unroll
        for (int x = 0; x < 4; ++x) ldg<T, VEC>(B + off(rest | ((x >> 1) << EA) | ((x & 1) << EB)), b[x]);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int ty = rest | ((y >> 1) << EA) | ((y & 1) << EB);
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
              const T2 bb = b[x][q], pp = ph[ty][q];
              acc[2 * (4 * x + y)] += bb.x * pp.x + bb.y * pp.y;
              acc[2 * (4 * x + y) + 1] += bb.y * pp.x - bb.x * pp.y;
            }
          }
      }
    } else {
#pragma unroll
      for (int t = 0; t < ROWS; ++t) {
        T2 b[VEC];
        ldg<T, VEC>(B + off(t), b);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          const T dx = ph[t][q].x - b[q].x, dy = ph[t][q].y - b[q].y;
          acc[0] += dx * dx + dy * dy;
        }
      }
    }
  }
  if constexpr (MODE == 0) {
    const double mine = (double)warp_reduce_scatter32<T>(acc, lane);
    block_partials32<T, T>(mine, sh, reinterpret_cast<T*>(part));
  } else {
    double v = (double)acc[0];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(FULL, v, m);
    block_partials32<T, double>(lane == 0 ? v : 0.0, sh, reinterpret_cast<double*>(part));
  }
}

template <typename T>
__device__ void df_process(const DfStep& st, int s, int c, DfShared<T>& sh, void* partials, double* resid) {
  constexpr int V2 = sizeof(T) == 4 ? 2 : 1;  // samples per thread for 4- and 16-row units
  T* part = reinterpret_cast<T*>(partials) + ((long long)s * st.nchunk + c) * 32;
  double* part64 = resid + ((long long)s * st.nchunk + c) * 32;
  switch (st.kind) {
    case DF_FWD: df_forward<T, V2>(st, s, c, sh); break;
    case DF_BWD4: df_backward_q4<T, V2>(st, s, c, sh, part); break;
    case DF_BWD2_10: df_backward_gen<T, V2, 0, 2, 1, 0>(st, s, c, sh, part); break;
    case DF_BWD2_01: df_backward_gen<T, V2, 0, 2, 0, 1>(st, s, c, sh, part); break;
    case DF_BWD3_20: df_backward_gen<T, 1, 0, 3, 2, 0>(st, s, c, sh, part); break;
    case DF_BWD3_02: df_backward_gen<T, 1, 0, 3, 0, 2>(st, s, c, sh, part); break;
    case DF_BWD3_10: df_backward_gen<T, 1, 0, 3, 1, 0>(st, s, c, sh, part); break;
    case DF_BWD3_01: df_backward_gen<T, 1, 0, 3, 0, 1>(st, s, c, sh, part); break;
    case DF_RESID: df_backward_gen<T, V2, 1, 2, 1, 0>(st, s, c, sh, part64); break;
    default: break;
  }
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(kDfThreads, sizeof(T) == 4 ? 3 : 2) k_sweep_df(DfArgs a) {
  __shared__ DfShared<T> sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) {
      long long w = -1;
      if (!ld_volatile_i32(a.err)) {
        const unsigned x = atomicAdd(a.queue, 1u);
        if ((long long)x < a.total_items) w = x;
      }
      sh.item = w;
    }
    __syncthreads();
    const long long w = sh.item;
    if (w < 0) return;
    int i = 0;
    while (i + 1 < a.nsteps && a.steps[i + 1].item0 <= w) ++i;
    const DfStep& st = a.steps[i];
    const int rel = (int)(w - st.item0);
    const int s = rel / st.nchunk, c = rel - s * st.nchunk;
    // Wait until start s has completed steps 0 .. i-1.
    if (threadIdx.x == 0) {
      int ok = 1;
      long long polls = 0;
      while (ld_acquire_u32(a.done + s) < (unsigned)i) {
        if (++polls > kDfSpinLimit || ld_volatile_i32(a.err)) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
      if (!ok) atomicOr(a.err, 1);
      sh.flag = ok;
    }
    __syncthreads();
    if (!sh.flag) return;
    const bool act = a.active == nullptr || a.active[s] != 0;
    if (a.trace && threadIdx.x == 0 && c == 0) a.trace[((long long)i * a.S + s) * 4] = globaltimer_ns();
    if (act) df_process<T>(st, s, c, sh, a.partials, a.resid_partials);
    // Publish this chunk; the last chunk of (step, start) finishes the step.
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned old = atomicAdd(a.chunk_cnt + (long long)i * a.S + s, 1u);
      sh.flag = old == (unsigned)(st.nchunk - 1);
    }
    __syncthreads();
    if (sh.flag) {
      unsigned long long* tr = a.trace ? a.trace + ((long long)i * a.S + s) * 4 : nullptr;
      if (tr && threadIdx.x == 0) tr[1] = globaltimer_ns();
      if (act && st.kind != DF_FWD) {
        __threadfence();
        if (st.kind == DF_RESID) {
          if (warp == 0) {
            const double* pp = a.resid_partials + (long long)s * st.nchunk * 32;
            double t = 0.0;
            for (int b = lane; b < st.nchunk; b += 32) t += __ldcg(pp + (long long)b * 32);
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) t += __shfl_xor_sync(FULL, t, m);
            if (lane == 0) a.resid_cost[s] = t * a.inv_M;
          }
        } else {
          // Sum the chunk partials with all four warps (warp w takes chunks
          // w, w+4, ...; fixed order), then one warp runs the update.
          const T* pp = reinterpret_cast<const T*>(a.partials) + (long long)s * st.nchunk * 32;
          T acc[4] = {T(0), T(0), T(0), T(0)};
          int b = warp;
          for (; b + 12 < st.nchunk; b += 16) {
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += __ldcg(pp + (long long)(b + 4 * q) * 32 + lane);
          }
          for (; b < st.nchunk; b += 4) acc[0] += __ldcg(pp + (long long)b * 32 + lane);
          sh.red[warp][lane] = (double)((acc[0] + acc[1]) + (acc[2] + acc[3]));
          __syncthreads();
          if (tr && threadIdx.x == 0) tr[2] = globaltimer_ns();
          if (warp == 0) {
            const double v = ((sh.red[0][lane] + sh.red[1][lane]) + (sh.red[2][lane] + sh.red[3][lane]));
            update_from_sum<sizeof(T) == 4 ? 1 : 2>(st.upd, s, v, sh.polar);
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        if (tr) tr[3] = globaltimer_ns();
        st_release_u32(a.done + s, (unsigned)(i + 1));
      }
    }
    __syncthreads();
  }
}

int df_blocks_per_sm(Real r) {
  static int cache[2] = {0, 0};
  int& c = cache[r == R32 ? 0 : 1];
  if (c) return c;
  int b = 0;
  const cudaError_t e = r == R32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_df<float>, kDfThreads, 0)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_df<double>, kDfThreads, 0);
  if (e != cudaSuccess || b < 1) {
    cudaGetLastError();
    return 0;
  }
  c = b;
  return c;
}

cudaError_t launch_sweep_df(Real r, const DfArgs& a, int num_sms, cudaStream_t st) {
  const int bps = df_blocks_per_sm(r);
  if (bps < 1) return cudaErrorLaunchOutOfResources;
  const int grid = (int)std::min<long long>((long long)bps * num_sms, std::max<long long>(a.total_items, 1));
  DfArgs args = a;
  void* params[] = {&args};
  return r == R32 ? cudaLaunchCooperativeKernel((const void*)k_sweep_df<float>, dim3(grid), dim3(kDfThreads), params,
                                                0, st)
                  : cudaLaunchCooperativeKernel((const void*)k_sweep_df<double>, dim3(grid), dim3(kDfThreads),
                                                params, 0, st);
}

// Chunking of one step: about `target` bytes of streaming per item, a
// multiple of 32 units per chunk.
void df_chunking(DfStep& st, double bytes_per_unit, double target) {
  long long nchunk = (long long)((st.units * bytes_per_unit + target - 1) / target);
  nchunk = std::max<long long>(1, std::min<long long>(nchunk, (st.units + 31) / 32));
  long long chunk = (st.units + nchunk - 1) / nchunk;
  chunk = (chunk + 31) / 32 * 32;
  st.chunk = (int)chunk;
  st.nchunk = (int)((st.units + chunk - 1) / chunk);
}

}  // namespace qfs
