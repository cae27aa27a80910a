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

// One CTA per SM holding all the warps the registers allow (12 for complex64,
// 8 for complex128): an item is streamed by the whole SM, so the chunks of
// one start finish sooner than with several smaller CTAs sharing the SM.
template <typename T>
__host__ __device__ constexpr int df_threads() {
  return sizeof(T) == 4 ? 512 : 256;
}
constexpr int kDfMaxWarps = 16;

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

// Scratch of the CTA-wide gate update (4x4 matrices in the lane layout
// M[r][c] at 4c + r).
struct DfUpd {
  double2 A[16];             // A = E^dagger scaled by a power of two
  double2 Q[2][16];          // iterate (double buffer)
  double2 T[16];             // products
  double2 X[16];             // the correction factor of the polish step
  float2 V[16];              // right singular vectors (FP32 Jacobi)
  float sig[16];             // singular value of column (lane >> 2)
  int ok;
};

template <typename T>
struct DfShared {
  typename C2<T>::t gs[16];
  typename C2<T>::t gs2[16];  // the second gate of a two-gate forward step
  double red[kDfMaxWarps][32];
  double2 polar[32];
  DfUpd u;
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
    for (int w = 0; w < df_threads<T>() / 32; ++w) t += sh.red[w][lane];
    __stcg(out + lane, (PT)t);
  }
}

// Start s's input and Phi input: per-start stride, plus a per-target stride
// for the arrays one per target (Psi, U Psi) when several targets share the
// launch (start s belongs to target s / spt).
template <typename T2>
__device__ __forceinline__ const T2* df_in(const DfStep& st, int s) {
  return reinterpret_cast<const T2*>(st.in) + s * st.in_stride + (long long)(s / st.spt) * st.in_gstride;
}
template <typename T2>
__device__ __forceinline__ const T2* df_phi_in(const DfStep& st, int s) {
  return reinterpret_cast<const T2*>(st.phi_in) + s * st.phi_in_stride + (long long)(s / st.spt) * st.phi_in_gstride;
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
  const T2* X = df_in<T2>(st, s);
  T2* Y = reinterpret_cast<T2*>(st.out) + s * st.fg.sN;
  const int MV = st.fg.M / VEC;
  const int u0 = c * st.chunk, u1 = min(u0 + st.chunk, st.units);
  auto offsets = [&](int u, uint32_t (&off)[4]) {
    const int r = u / MV, jv = u - r * MV;
    const uint32_t base = insert_two_zero_bits((uint32_t)r, st.fg.lo, st.fg.hi);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const uint32_t row = base | ((uint32_t)(x >> 1) << st.fg.pos_a) | ((uint32_t)(x & 1) << st.fg.pos_b);
      off[x] = row * (uint32_t)st.fg.M + (uint32_t)jv * VEC;
    }
  };
  auto apply = [&](const T2 (&v)[4][VEC], const uint32_t (&off)[4]) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      T2 o[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        T2 acc = cmul(gr[4 * x], v[0][q]);
#pragma unroll
        for (int xp = 1; xp < 4; ++xp) acc = cfma(gr[4 * x + xp], v[xp][q], acc);
        o[q] = acc;
      }
      stg<T, VEC>(Y + off[x], o);
    }
  };
  // Two units per thread per round: eight loads in flight.
  constexpr int NT = df_threads<T>();
  int u = u0 + threadIdx.x;
  for (; u + NT < u1; u += 2 * NT) {
    uint32_t oa[4], ob[4];
    offsets(u, oa);
    offsets(u + NT, ob);
    T2 va[4][VEC], vb[4][VEC];
#pragma unroll
    for (int x = 0; x < 4; ++x) ldg<T, VEC>(X + oa[x], va[x]);
#pragma unroll
    for (int x = 0; x < 4; ++x) ldg<T, VEC>(X + ob[x], vb[x]);
    apply(va, oa);
    apply(vb, ob);
  }
  if (u < u1) {
    uint32_t oa[4];
    offsets(u, oa);
    T2 va[4][VEC];
#pragma unroll
    for (int x = 0; x < 4; ++x) ldg<T, VEC>(X + oa[x], va[x]);
    apply(va, oa);
  }
}

// Asynchronous 16-byte copies global -> shared (L2 only), in groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stages of the backward step's copy pipeline.  Each thread copies the
// sixteen bytes it will itself consume (eight rows of its unit: four of Phi,
// four of B) into its own slots of a stage, so completion needs only the
// thread's own cp.async.wait_group, never a block barrier; with kDfStages
// stages, kDfStages - 1 rounds of loads are in flight per thread while one
// round is computed, held in shared memory instead of registers.  Slot
// (stage, row j, thread t) sits at ((stage * 8 + j) * threads + t) * 16
// bytes: a warp reads 512 contiguous bytes, free of bank conflicts.
constexpr int kDfStages = 3;
template <typename T>
__host__ __device__ constexpr int df_stage_bytes() {
  return kDfStages * 8 * df_threads<T>() * 16;
}

// Two forward steps in one pass over 16-row units (gates k and k+1 on four
// distinct qubits; geometry bg with gate k's pair on local bits 3, 2 and
// gate k+1's on local bits 1, 0): B_k = g_k B_{k-1} and B_{k+1} = g_{k+1}
// B_k, both stored, B_k never read back.  Four lanes share a unit: lane
// quarter qx holds the four rows of one value of gate k+1's bits and applies
// g_k to them; g_{k+1} then mixes the four quarters through shuffles.  Rows
// are staged by cp.async into the thread's own slots (kDfFwd2Stages - 1
// rounds in flight).
constexpr int kDfFwd2Stages = 4;
template <typename T, int VEC>
__device__ void df_forward2(const DfStep& st, int s, int c, DfShared<T>& sh, uint4* stage) {
  using T2 = typename C2<T>::t;
  static_assert(sizeof(T2) * VEC == 16, "one 16-byte slot per row");
  static_assert(kDfFwd2Stages * 4 <= kDfStages * 8, "forward stages fit the stage buffer");
  constexpr int NT = df_threads<T>();
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qx = lane >> 3, v = lane & 7;
  if (threadIdx.x < 16)
    sh.gs[threadIdx.x] = __ldcg(reinterpret_cast<const T2*>(st.gate) + s * st.gate_stride + threadIdx.x);
  else if (threadIdx.x < 32)
    sh.gs2[threadIdx.x - 16] =
        __ldcg(reinterpret_cast<const T2*>(st.gate2) + s * st.gate_stride + (threadIdx.x - 16));
  __syncthreads();
  T2 g1[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) g1[i] = sh.gs[i];
  T2 g2[4];  // row qx of g_{k+1}
#pragma unroll
  for (int m = 0; m < 4; ++m) g2[m] = sh.gs2[4 * qx + m];
  const T2* X = df_in<T2>(st, s);
  T2* Y1 = reinterpret_cast<T2*>(st.out) + s * st.bg.sN;
  T2* Y2 = reinterpret_cast<T2*>(st.out2) + s * st.bg.sN;
  const uint32_t M = (uint32_t)st.bg.M;
  const uint32_t d0 = (1u << st.bg.pos[0]) * M, d1 = (1u << st.bg.pos[1]) * M;
  const uint32_t d2 = (1u << st.bg.pos[2]) * M, d3 = (1u << st.bg.pos[3]) * M;
  const uint32_t xoff = ((qx >> 1) ? d1 : 0u) + ((qx & 1) ? d0 : 0u);
  const uint32_t joff[4] = {0u, d2, d3, d3 + d2};  // j = 2 bit(local 3) + bit(local 2): gate k's index
  const int MV = st.bg.M / VEC;
  const int u0 = c * st.chunk, u1 = min(u0 + st.chunk, st.units);
  constexpr int per_round = 8 * NW;
  const int rounds = (u1 - u0 + per_round - 1) / per_round;
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
  auto issue = [&](int rd) {
    const int u = u0 + rd * per_round + warp * 8 + v;
    if (rd < rounds && u < u1) {
      uint4* slot = stage + (size_t)((rd % kDfFwd2Stages) * 4) * NT + threadIdx.x;
      const uint32_t o = unit_off(u);
#pragma unroll
      for (int j = 0; j < 4; ++j) cp_async16(slot + (size_t)j * NT, X + o + joff[j]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int rd = 0; rd < kDfFwd2Stages - 1; ++rd) issue(rd);
  for (int rd = 0; rd < rounds; ++rd) {
    issue(rd + kDfFwd2Stages - 1);
    cp_async_wait<kDfFwd2Stages - 1>();
    const int u = u0 + rd * per_round + warp * 8 + v;
    const bool valid = u < u1;  // (all four lanes of a unit agree)
    T2 b[4][VEC];
    {
      const uint4* slot = stage + (size_t)((rd % kDfFwd2Stages) * 4) * NT + threadIdx.x;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint4 w4 = valid ? slot[(size_t)j * NT] : make_uint4(0u, 0u, 0u, 0u);
        const T2* e = reinterpret_cast<const T2*>(&w4);
#pragma unroll
        for (int q = 0; q < VEC; ++q) b[j][q] = e[q];
      }
    }
    const uint32_t o = valid ? unit_off(u) : 0u;
    T2 y[4][VEC];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        T2 acc = cmul(g1[4 * x], b[0][q]);
#pragma unroll
        for (int xp = 1; xp < 4; ++xp) acc = cfma(g1[4 * x + xp], b[xp][q], acc);
        y[x][q] = acc;
      }
    if (valid) {
#pragma unroll
      for (int x = 0; x < 4; ++x) stg<T, VEC>(Y1 + o + joff[x], y[x]);
    }
    // z = g_{k+1} y over the quarters, summed in the order of the one-gate
    // forward step (quarter 0 first); quarter xp sits xor 8 (qx ^ xp) away.
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      T2 z[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        T2 w[4];
#pragma unroll
        for (int xp = 0; xp < 4; ++xp) {
          w[xp].x = __shfl_xor_sync(FULL, y[x][q].x, 8 * (qx ^ xp));
          w[xp].y = __shfl_xor_sync(FULL, y[x][q].y, 8 * (qx ^ xp));
        }
        T2 acc = cmul(g2[0], w[0]);
#pragma unroll
        for (int xp = 1; xp < 4; ++xp) acc = cfma(g2[xp], w[xp], acc);
        z[q] = acc;
      }
      if (valid) stg<T, VEC>(Y2 + o + joff[x], z);
    }
  }
  cp_async_wait<0>();
}

// Backward step on 16-row units (gate k+1 and gate k on four distinct
// qubits): four lanes share a unit as in the per-step kernel; the partial
// sums of E_k go to partials slot (s, c).
template <typename T, int VEC>
__device__ void df_backward_q4(const DfStep& st, int s, int c, DfShared<T>& sh, T* part, uint4* stage) {
  using T2 = typename C2<T>::t;
  static_assert(sizeof(T2) * VEC == 16, "one 16-byte slot per row");
  constexpr int NT = df_threads<T>();
  constexpr int NW = NT / 32;
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
  const T2* B = df_in<T2>(st, s);
  const T2* P = df_phi_in<T2>(st, s);
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
  constexpr int per_round = 8 * NW;  // units of one round (eight per warp)
  const int rounds = (u1 - u0 + per_round - 1) / per_round;
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
  auto issue = [&](int rd) {
    const int u = u0 + rd * per_round + warp * 8 + v;
    if (rd < rounds && u < u1) {
      uint4* slot = stage + (size_t)((rd % kDfStages) * 8) * NT + threadIdx.x;
      const uint32_t o = unit_off(u);
#pragma unroll
      for (int j = 0; j < 4; ++j) cp_async16(slot + (size_t)j * NT, P + o + joff[j]);
#pragma unroll
      for (int j = 0; j < 4; ++j) cp_async16(slot + (size_t)(4 + j) * NT, B + o + joff[j]);
    }
    cp_async_commit();  // (an empty group keeps the group count uniform)
  };
#pragma unroll
  for (int rd = 0; rd < kDfStages - 1; ++rd) issue(rd);
  for (int rd = 0; rd < rounds; ++rd) {
    issue(rd + kDfStages - 1);
    cp_async_wait<kDfStages - 1>();  // this thread's copies of round rd have landed
    const int u = u0 + rd * per_round + warp * 8 + v;
    const bool valid = u < u1;
    T2 ph[4][VEC], b[4][VEC];
    {
      const uint4* slot = stage + (size_t)((rd % kDfStages) * 8) * NT + threadIdx.x;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint4 w4 = valid ? slot[(size_t)j * NT] : make_uint4(0u, 0u, 0u, 0u);
        const T2* e = reinterpret_cast<const T2*>(&w4);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          if (j < 4) ph[j][q] = e[q];
          else b[j - 4][q] = e[q];
        }
      }
    }
    const uint32_t base_off = valid ? unit_off(u) : 0u;
    {
      T2 nw[4][VEC];
#pragma unroll
      for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          T2 t = cmul(gd[4 * y], ph[0][q]);
#pragma unroll
          for (int j = 1; j < 4; ++j) t = cfma(gd[4 * y + j], ph[j][q], t);
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
          cfma_conj(acc[2 * m], acc[2 * m + 1], b[j][q], pp);
        }
    }
  }
  cp_async_wait<0>();
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
    for (int w = 0; w < NW; ++w) t += sh.red[w][lane];
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
  const T2* B = df_in<T2>(st, s);
  const T2* P = df_phi_in<T2>(st, s);
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
  for (int u = u0 + threadIdx.x; u < u1; u += df_threads<T>()) {
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
            for (int yp = 1; yp < 4; ++yp) a2 = cfma(gd(y, yp), ph[(yp << (U - 2)) | t0][q], a2);
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
              cfma_conj(acc[2 * (4 * x + y)], acc[2 * (4 * x + y) + 1], b[x][q], ph[ty][q]);
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
          acc[0] = fmat(dx, dx, fmat(dy, dy, acc[0]));
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

// C = op(X) Y for 4x4 complex matrices in shared memory (lane layout),
// op(X) = X^dagger when AH, by all 128 threads of the CTA.  FP64 arithmetic
// issues at a fixed cost per warp instruction on this GPU whatever the
// number of active lanes, so the 256 real products are packed two per
// thread over four warps (one per SM sub-partition): thread t forms the real
// (t even) or imaginary part of X[r][k] Y[k][c] for entry t/8, k = (t/2)%4,
// and the k terms are summed by two shuffles.  POST = 1 stores
// 1.5 I - 0.5 C instead (the Newton-Schulz factor).  The caller
// synchronises before and after.
template <bool AH, int POST>
__device__ __forceinline__ void mm64_cta(const double2* X, const double2* Y, double2* C) {
  const int t = threadIdx.x;
  if (t >= 128) return;  // four warps take part
  const int e = t >> 3, k = (t >> 1) & 3, part = t & 1;
  const int r = e & 3, c = e >> 2;
  double2 x = AH ? X[4 * r + k] : X[4 * k + r];
  if (AH) x.y = -x.y;
  const double2 y = Y[4 * c + k];
  double v = part ? fma(x.x, y.y, x.y * y.x) : fma(x.x, y.x, -(x.y * y.y));
  v += __shfl_xor_sync(FULL, v, 2);
  v += __shfl_xor_sync(FULL, v, 4);
  if (k == 0) {
    if (POST == 1) v = fma(-0.5, v, (part == 0 && r == c) ? 1.5 : 0.0);
    reinterpret_cast<double*>(C + e)[part] = v;
  }
}

// FP32 part of the update on warp 0 (as in warp_polar4_fast): scale A by an
// exact power of two, one-sided Jacobi on A V0, Q0 = W V^H.  Leaves the
// scaled A, Q0 (promoted), V and the singular values in u; returns false
// when A is zero or too ill-conditioned for the fast path.
__device__ __forceinline__ bool df_polar_begin(double2 a, double2 v0, DfUpd& u) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, row = l16 & 3, col = l16 >> 2;
  const bool isV = lane >= 16;
  int e = 0;
  if (!isV) {
    const int ex = (__double2hiint(a.x) >> 20) & 0x7ff, ey = (__double2hiint(a.y) >> 20) & 0x7ff;
    e = max(ex, ey);
  }
  e = __reduce_max_sync(FULL, e);
  if (e == 0) return false;
  const double sc = __hiloint2double((2046 - e) << 20, 0);
  const double2 as{a.x * sc, a.y * sc};
  if (!isV) u.A[l16] = as;
  const float2 a32{(float)as.x, (float)as.y};
  const float2 v032{(float)v0.x, (float)v0.y};
  float2 x;
  {
    float2 acc{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 ak = shfl_c(a32, 4 * k + row), vk = shfl_c(v032, 16 + 4 * col + k);
      acc = cfma(ak, vk, acc);
    }
    x = isV ? v032 : acc;
  }
  x = jacobi32_sweeps(x);
  float2 w = shfl_c(x, l16);
  const float2 v = shfl_c(x, 16 + l16);
  float nrm = w.x * w.x + w.y * w.y;
  nrm += __shfl_xor_sync(FULL, nrm, 1);
  nrm += __shfl_xor_sync(FULL, nrm, 2);
  float smax = nrm, smin = nrm;
  smax = fmaxf(smax, __shfl_xor_sync(FULL, smax, 4));
  smax = fmaxf(smax, __shfl_xor_sync(FULL, smax, 8));
  smin = fminf(smin, __shfl_xor_sync(FULL, smin, 4));
  smin = fminf(smin, __shfl_xor_sync(FULL, smin, 8));
  if (!(smin > 1e-6f * smax)) return false;
  const float inv = rsqrtf(nrm);
  const float sig = nrm * inv;
  w = float2{w.x * inv, w.y * inv};
  const float2 q32 = mm_bh(w, v, row, col);
  if (!isV) {
    u.Q[0][l16] = double2{(double)q32.x, (double)q32.y};
    u.V[l16] = v;
    u.sig[l16] = sig;
  }
  return true;
}

// The update of gate k for start s by the whole CTA: the same mathematics as
// polar_update_warp / update_from_sum (FP32 Jacobi, two FP64 Newton-Schulz
// steps, POLISH skew-Hermitian corrections), with the FP64 products spread
// over the four warps.  Warp 0 holds the summed environment value v (lane j
// = value j of E) and, in lanes 16..31, the Jacobi start v0 (the gate's V
// from its previous update, or the identity), loaded by the caller before
// the partial sums so that its latency is off the chain.  All threads call
// it.
template <typename T, int POLISH>
__device__ void df_update(const UpdateArgs& ua, int s, DfShared<T>& sh, double v, double2 v0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l16 = lane & 15, row = l16 & 3, col = l16 >> 2;
  DfUpd& u = sh.u;
  double2* vio = ua.vprev ? ua.vprev + s * ua.g_stride : nullptr;
  double2* g64 = ua.g64 + s * ua.g_stride;
  double2 e{0.0, 0.0}, a{0.0, 0.0};
  if (warp == 0) {
    e = double2{__shfl_sync(FULL, v, 2 * l16), __shfl_sync(FULL, v, 2 * l16 + 1)};
    if (ua.env_out && lane < 16) ua.env_out[s * ua.env_stride + l16] = e;
    double2 m = e;
    if (ua.beta != 0.0 && lane < 16) {
      const double2 go = g64[4 * row + col];
      m = double2{(1.0 - ua.beta) * m.x + ua.beta * go.x, (1.0 - ua.beta) * m.y - ua.beta * go.y};
    }
    a = double2{m.x, -m.y};
    const bool ok = df_polar_begin(a, v0, u);
    if (lane == 0) u.ok = ok ? 1 : 0;
  }
  __syncthreads();
  bool ok = u.ok != 0;
  int cur = 0;
  if (ok) {
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
      mm64_cta<true, 1>(u.Q[cur], u.Q[cur], u.T);  // T = (3I - Q^H Q) / 2
      __syncthreads();
      mm64_cta<false, 0>(u.Q[cur], u.T, u.Q[cur ^ 1]);
      __syncthreads();
      cur ^= 1;
    }
#pragma unroll 1
    for (int it = 0; it < POLISH; ++it) {
      mm64_cta<true, 0>(u.Q[cur], u.A, u.T);  // B = Q^H A
      __syncthreads();
      if (warp == 0) {
        const double2 bm = u.T[l16];
        const double2 bt = u.T[4 * row + col];  // B[col][row]
        const float2 k32{0.5f * (float)(bm.x - bt.x), 0.5f * (float)(bm.y + bt.y)};
        const float2 om = skew_correction(k32, u.V[l16], u.sig[l16], row, col);
        const float big = max_abs16(om);
        const int good = it > 0 || big < 1e-3f ? 1 : 0;
        const double2 xc = exp_skew3(om, big, row, col);
        if (lane < 16) u.X[l16] = xc;
        if (lane == 0) u.ok = good;
      }
      __syncthreads();
      if (!u.ok) {
        ok = false;
        break;
      }
      mm64_cta<false, 0>(u.Q[cur], u.X, u.Q[cur ^ 1]);
      __syncthreads();
      cur ^= 1;
    }
  }
  if (warp == 0) {
    double2 p;
    if (ok) {
      p = u.Q[cur][l16];
      if (vio && lane < 16) vio[l16] = double2{(double)u.V[l16].x, (double)u.V[l16].y};
    } else {
      // Zero, ill-conditioned or not converging: the FP64 Jacobi (which
      // also completes rank-deficient cases), from the identity.
      p = warp_polar4(a, double2{row == col ? 1.0 : 0.0, 0.0}, sh.polar, vio);
    }
    if (lane < 16) {
      g64[4 * row + col] = p;
      if (ua.g32) (ua.g32 + s * ua.g_stride)[4 * row + col] = float2{(float)p.x, (float)p.y};
    }
    if (ua.cost_out) {
      double t = lane < 16 ? (p.x * e.x - p.y * e.y) : 0.0;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
      if (lane == 0) ua.cost_out[s] = 2.0 - 2.0 * ua.inv_M * t;
    }
  }
}

// Partial-sum slots: start s owns slots s * stride .. s * stride + stride - 1
// (stride = the most chunks of any step), so starts that are at different
// steps, with different chunk counts, never share a slot.
template <typename T>
__device__ void df_process(const DfStep& st, int s, int c, DfShared<T>& sh, void* partials, double* resid,
                           int stride, uint4* stage) {
  constexpr int V2 = sizeof(T) == 4 ? 2 : 1;  // samples per thread for 4- and 16-row units
  T* part = reinterpret_cast<T*>(partials) + ((long long)s * stride + c) * 32;
  double* part64 = resid + ((long long)s * stride + c) * 32;
  switch (st.kind) {
    case DF_FWD: df_forward<T, V2>(st, s, c, sh); break;
    case DF_FWD2: df_forward2<T, V2>(st, s, c, sh, stage); break;
    case DF_BWD4: df_backward_q4<T, V2>(st, s, c, sh, part, stage); break;
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
__global__ void __launch_bounds__(df_threads<T>(), 1) k_sweep_df(DfArgs a) {
  __shared__ DfShared<T> sh;
  extern __shared__ __align__(16) uint4 df_stage[];  // df_stage_bytes<T>() of copy stages
  constexpr int NW = df_threads<T>() / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // Thread 0 takes the next item when the CTA is free (a reservation held
  // while the current item runs would delay that item by a whole item).
  // A CTA's items increase, so the step search resumes where it stopped.
  // The next sweep's control words (a slot this sweep does not use).
  if (a.zero_next != nullptr)
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.zero_count; k += gridDim.x * blockDim.x)
      a.zero_next[k] = 0u;
  // A sweep queued behind one that met the tolerance does nothing.
  if (a.stop != nullptr && ld_volatile_i32(a.stop)) return;
  int i = 0;
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
    while (i + 1 < a.nsteps && a.steps[i + 1].item0 <= w) ++i;
    const DfStep& st = a.steps[i];
    const int rel = (int)(w - st.item0);
    const int s = rel / st.nchunk, c = rel - s * st.nchunk;
    unsigned long long* itr = a.item_trace ? a.item_trace + w * 4 : nullptr;
    if (itr && threadIdx.x == 0) {
      itr[0] = globaltimer_ns();
      itr[3] = ((unsigned long long)blockIdx.x << 40) | ((unsigned long long)i << 20) | (unsigned)s;
    }
    // Wait until start s has completed steps 0 .. i-1.
    if (threadIdx.x == 0) {
      int ok = 1;
      long long polls = 0;
      while (ld_acquire_u32(a.done + s) < (unsigned)i) {
        if (++polls > a.wait_limit || ld_volatile_i32(a.err)) {
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
    // The residual pass of a start whose cost estimate from the gate-1
    // update is far above the tolerance is skipped: it could not decide
    // anything (the estimate, accurate to ~1e-7 absolute, stands).
    const bool act = (a.active == nullptr || a.active[s] != 0) &&
                     !(st.kind == DF_RESID && a.resid_skip > 0.0 && __ldcg(a.resid_cost + s) > a.resid_skip);
    if (a.trace && threadIdx.x == 0 && c == 0) a.trace[((long long)i * a.S + s) * 4] = globaltimer_ns();
    if (itr && threadIdx.x == 0) itr[1] = globaltimer_ns();
    if (act) df_process<T>(st, s, c, sh, a.partials, a.resid_partials, a.part_stride, df_stage);
    // Publish this chunk; the last chunk of (step, start) finishes the step.
    __syncthreads();
    if (threadIdx.x == 0) {
      if (itr) itr[2] = globaltimer_ns();
      __threadfence();
      const unsigned old = atomicAdd(a.chunk_cnt + (long long)i * a.S + s, 1u);
      sh.flag = old == (unsigned)(st.nchunk - 1);
    }
    __syncthreads();
    if (sh.flag) {
      unsigned long long* tr = a.trace ? a.trace + ((long long)i * a.S + s) * 4 : nullptr;
      if (tr && threadIdx.x == 0) tr[1] = globaltimer_ns();
      if (act && st.kind != DF_FWD && st.kind != DF_FWD2) {
        __threadfence();
        if (st.kind == DF_RESID) {
          if (warp == 0) {
            const double* pp = a.resid_partials + (long long)s * a.part_stride * 32;
            double t = 0.0;
            for (int b = lane; b < st.nchunk; b += 32) t += __ldcg(pp + (long long)b * 32);
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) t += __shfl_xor_sync(FULL, t, m);
            if (lane == 0) {
              a.resid_cost[s] = t * a.inv_M;
              if (a.cost_row != nullptr) a.cost_row[s] = t * a.inv_M;
              if (a.stop != nullptr && t * a.inv_M <= a.stop_tol) atomicExch(a.stop, 1);
            }
          }
        } else {
          // The Jacobi start of the update, then the chunk partials summed
          // by all warps (warp w takes chunks w, w + NW, ...; fixed order).
          double2 v0{(lane & 3) == ((lane & 15) >> 2) ? 1.0 : 0.0, 0.0};
          if (warp == 0 && lane >= 16 && st.upd.vprev) v0 = (st.upd.vprev + s * st.upd.g_stride)[lane & 15];
          const T* pp = reinterpret_cast<const T*>(a.partials) + (long long)s * a.part_stride * 32;
          T acc[4] = {T(0), T(0), T(0), T(0)};
          int b = warp;
          for (; b + 3 * NW < st.nchunk; b += 4 * NW) {
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += __ldcg(pp + (long long)(b + q * NW) * 32 + lane);
          }
          for (; b < st.nchunk; b += NW) acc[0] += __ldcg(pp + (long long)b * 32 + lane);
          sh.red[warp][lane] = (double)((acc[0] + acc[1]) + (acc[2] + acc[3]));
          __syncthreads();
          if (tr && threadIdx.x == 0) tr[2] = globaltimer_ns();
          double v = 0.0;
          if (warp == 0) {
#pragma unroll
            for (int w = 0; w < NW; ++w) v += sh.red[w][lane];
          }
          // complex64 sweeps: the polar factor to FP32 accuracy, the
          // accuracy of their environments (no skew-Hermitian correction);
          // FP64 sweeps: polar to FP64 rounding (two corrections).
          df_update<T, sizeof(T) == 4 ? 0 : 2>(st.upd, s, sh, v, v0);
          if (st.upd.cost_out != nullptr && threadIdx.x == 0) {
            const double cost = st.upd.cost_out[s];
            if (a.cost_row != nullptr) a.cost_row[s] = cost;
            if (a.stop != nullptr && a.stop_from_update && cost <= a.stop_tol) atomicExch(a.stop, 1);
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
  cudaError_t e;
  if (r == R32) {
    e = cudaFuncSetAttribute(k_sweep_df<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, df_stage_bytes<float>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_df<float>, df_threads<float>(),
                                                        df_stage_bytes<float>());
  } else {
    e = cudaFuncSetAttribute(k_sweep_df<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             df_stage_bytes<double>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sweep_df<double>, df_threads<double>(),
                                                        df_stage_bytes<double>());
  }
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
  return r == R32 ? cudaLaunchCooperativeKernel((const void*)k_sweep_df<float>, dim3(grid),
                                                dim3(df_threads<float>()), params, df_stage_bytes<float>(), st)
                  : cudaLaunchCooperativeKernel((const void*)k_sweep_df<double>, dim3(grid),
                                                dim3(df_threads<double>()), params, df_stage_bytes<double>(), st);
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
