// Streaming kernels of the QFactor-Sample sweep (Section 3 of the paper):
// gate application to the stored list B of intermediate states, and the
// fused backward step that carries the updated gate into Phi and reduces the
// 4x4 environment of the next gate over the 2^(n-2)*M untouched amplitudes.
//
// These kernels are HBM-bound K=4 contractions: one 16-byte vector per row
// per thread, four rows per group, coalesced because the M samples of a row
// are contiguous.  No tensor cores: a 4x4 complex mat-vec per 64 bytes read
// is far below any tensor-core ridge point.
#include "polar4.cuh"
#include "qfs_common.cuh"
#include "qfs_kernels.h"

#include <algorithm>

namespace qfs {

Geom make_geom(int n, int M, int a, int b) {
  Geom g;
  g.n = n;
  g.M = M;
  g.pos_a = n - 1 - a;
  g.pos_b = n - 1 - b;
  g.lo = std::min(g.pos_a, g.pos_b);
  g.hi = std::max(g.pos_a, g.pos_b);
  g.sN = (long long)M << n;
  return g;
}

Shape make_shape(int n, int M, int S, Real r, int num_sms) {
  Shape sh;
  sh.vec = (r == R32 && (M % 2) == 0) ? 2 : 1;
  sh.units_per_start = (1 << (n - 2)) * (M / sh.vec);
  const long long total = (long long)sh.units_per_start * S;
  // Small problems use 128-thread blocks so more SMs take part.
  sh.threads = total >= (long long)num_sms * 512 ? 256 : 128;
  // Aim for about four blocks per SM over all starts.
  long long want_blocks = (long long)num_sms * 4;
  long long chunk = (total + want_blocks - 1) / want_blocks;
  chunk = ((chunk + sh.threads - 1) / sh.threads) * sh.threads;
  if (chunk < sh.threads) chunk = sh.threads;
  if (chunk > sh.units_per_start) chunk = ((sh.units_per_start + 31) / 32) * 32;
  sh.chunk = (int)chunk;
  sh.nblk = (sh.units_per_start + sh.chunk - 1) / sh.chunk;
  return sh;
}

template <typename T, int VEC> struct VecT;
template <> struct VecT<float, 2> { using t = float4; };
template <> struct VecT<float, 1> { using t = float2; };
template <> struct VecT<double, 1> { using t = double2; };

// Evict-first load for data read once per sweep.
template <typename T, int VEC>
__device__ __forceinline__ void ld(const typename C2<T>::t* p, typename C2<T>::t (&o)[VEC]) {
  using V = typename VecT<T, VEC>::t;
  V v = __ldcs(reinterpret_cast<const V*>(p));
  if constexpr (VEC == 2) {
    o[0] = float2{v.x, v.y};
    o[1] = float2{v.z, v.w};
  } else {
    o[0] = v;
  }
}
// Loads of data that a later kernel reads again (Phi, and the B list when it
// fits in L2) use the default caching policy.
template <typename T, int VEC>
__device__ __forceinline__ void ld_keep(const typename C2<T>::t* p, typename C2<T>::t (&o)[VEC]) {
  using V = typename VecT<T, VEC>::t;
  V v = *reinterpret_cast<const V*>(p);
  if constexpr (VEC == 2) {
    o[0] = float2{v.x, v.y};
    o[1] = float2{v.z, v.w};
  } else {
    o[0] = v;
  }
}
template <typename T, int VEC>
__device__ __forceinline__ void st(typename C2<T>::t* p, const typename C2<T>::t (&o)[VEC]) {
  using V = typename VecT<T, VEC>::t;
  if constexpr (VEC == 2) {
    *reinterpret_cast<V*>(p) = V{o[0].x, o[0].y, o[1].x, o[1].y};
  } else {
    *reinterpret_cast<V*>(p) = o[0];
  }
}

struct FwdArgs {
  const void* in; long long in_stride;
  void* out;
  const void* gates; long long gate_stride;
  Geom g; int units_per_start; int chunk;
  const int* active;  // per-start flag, nullable (all active)
};

template <typename T, int VEC>
__global__ void k_forward(FwdArgs a) {
  using T2 = typename C2<T>::t;
  const int s = blockIdx.y;
  if (a.active && !a.active[s]) return;
  __shared__ T2 gs[16];
  if (threadIdx.x < 16) gs[threadIdx.x] = reinterpret_cast<const T2*>(a.gates)[s * a.gate_stride + threadIdx.x];
  __syncthreads();
  T2 gr[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) gr[i] = gs[i];
  const T2* X = reinterpret_cast<const T2*>(a.in) + s * a.in_stride;
  T2* Y = reinterpret_cast<T2*>(a.out) + s * a.g.sN;
  const int MV = a.g.M / VEC;
  const int u0 = blockIdx.x * a.chunk;
  const int u1 = min(u0 + a.chunk, a.units_per_start);
  for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    const int r = u / MV, jv = u - r * MV;
    const uint32_t base = insert_two_zero_bits((uint32_t)r, a.g.lo, a.g.hi);
    long long off[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const uint32_t row = base | ((uint32_t)(x >> 1) << a.g.pos_a) | ((uint32_t)(x & 1) << a.g.pos_b);
      off[x] = (long long)row * a.g.M + (long long)jv * VEC;
    }
    T2 v[4][VEC];
#pragma unroll
    for (int x = 0; x < 4; ++x) ld_keep<T, VEC>(X + off[x], v[x]);
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
      st<T, VEC>(Y + off[x], o);
    }
  }
}

BwdGeom make_bwd_geom(int n, int M, int ua, int ub, int qa, int qb) {
  BwdGeom g;
  g.n = n;
  g.M = M;
  g.sN = (long long)M << n;
  // Local bits U-1, U-2 carry the gate applied to Phi; the environment pair
  // takes local bits of its own qubits, new qubits going to the low bits.
  int q[4] = {ua, ub, -1, -1};
  int U = 2;
  for (int x : {qa, qb})
    if (x != ua && x != ub) q[U++] = x;
  g.U = U;
  int local_of[4];
  for (int i = 0; i < U; ++i) local_of[i] = U - 1 - i;  // q[0] -> U-1, q[1] -> U-2, q[2] -> U-3, ...
  for (int i = 0; i < 4; ++i) g.pos[i] = 0;
  for (int i = 0; i < U; ++i) g.pos[local_of[i]] = n - 1 - q[i];
  auto local = [&](int qubit) {
    for (int i = 0; i < U; ++i)
      if (q[i] == qubit) return local_of[i];
    return -1;
  };
  g.ea = local(qa);
  g.eb = local(qb);
  int srt[4];
  for (int i = 0; i < U; ++i) srt[i] = g.pos[i];
  std::sort(srt, srt + U);
  for (int i = 0; i < 4; ++i) g.ins[i] = i < U ? srt[i] : 31;
  return g;
}

int bwd_resident_blocks(Real r, int vec, int U);  // defined after the kernels

Shape make_bwd_shape(int n, int M, int S, Real r, int num_sms, int U) {
  Shape sh;
  // 8-row units hold one complex64 sample per thread (registers); 4- and
  // 16-row units (the latter shared by four lanes) hold two.
  sh.vec = (r == R32 && (M % 2) == 0 && U != 3) ? 2 : 1;
  sh.units_per_start = (1 << (n - U)) * (M / sh.vec);
  sh.threads = 128;
  // One full wave: as many blocks as can be resident, split evenly over the
  // starts; a block's chunk is a multiple of 32 units.
  const long long slots = (long long)num_sms * std::max(1, bwd_resident_blocks(r, sh.vec, U));
  const long long per_start = std::max(1LL, slots / std::max(S, 1));
  long long chunk = (sh.units_per_start + per_start - 1) / per_start;
  chunk = ((chunk + 31) / 32) * 32;
  if (chunk < 32) chunk = 32;
  sh.chunk = (int)chunk;
  sh.nblk = (sh.units_per_start + sh.chunk - 1) / sh.chunk;
  return sh;
}



// Row t (0 <= t < 2^U) of a unit with the bits of j placed on the local
// bits other than EA and EB.
template <int U, int EA, int EB>
__device__ __forceinline__ constexpr int spread_rest(int j) {
  int t = 0, bit = 0;
  for (int i = 0; i < U; ++i) {
    if (i == EA || i == EB) continue;
    t |= ((j >> bit) & 1) << i;
    ++bit;
  }
  return t;
}

// One backward step.  A thread unit owns the 2^U rows spanned by the qubits
// of gate k+1 (local bits U-1, U-2) and gate k (local bits EA, EB) for VEC
// consecutive samples.  It carries the new gate k+1 into Phi
// (Phi_k = g_{k+1}^dagger Phi_{k+1}), stores Phi_k, and accumulates
// E_k[x][y] += B_{k-1}[x] conj(Phi_k[y]) over the groups of gate k.
// MODE 1 accumulates sum |Phi_k - B|^2 instead (the residual cost).
template <typename T, int VEC, int MODE, int U, int EA, int EB>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (U == 4 ? 3 : 4) : 2) k_backward(BwdArgs a) {
  using T2 = typename C2<T>::t;
  constexpr int ROWS = 1 << U;
  const int s = blockIdx.y;
  if (a.active && !a.active[s]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ T2 gs[16];
  __shared__ double red[4][32];
  __shared__ double2 sm_polar[32];
  __shared__ int is_last;
  const bool has_gate = a.gates != nullptr;
  if (threadIdx.x < 16)
    gs[threadIdx.x] = has_gate ? reinterpret_cast<const T2*>(a.gates)[s * a.gate_stride + threadIdx.x] : T2{};
  __syncthreads();
  // g^dagger[y][y'] = conj(g[y'][y]), read from shared memory (broadcast).
  auto gd = [&](int y, int yp) {
    const T2 t = gs[4 * yp + y];
    return T2{t.x, -t.y};
  };
  const T2* B = reinterpret_cast<const T2*>(a.bprev) + s * a.bprev_stride;
  const T2* P = reinterpret_cast<const T2*>(a.phi_in) + s * a.phi_in_stride;
  T2* Po = a.phi_out ? reinterpret_cast<T2*>(a.phi_out) + s * a.g.sN : nullptr;
  const uint32_t M = (uint32_t)a.g.M;
  uint32_t dpos[U];
#pragma unroll
  for (int i = 0; i < U; ++i) dpos[i] = (1u << a.g.pos[i]) * M;

  T acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = T(0);

  const int MV = a.g.M / VEC;
  const int u0 = blockIdx.x * a.chunk;
  const int u1 = min(u0 + a.chunk, a.units_per_start);
  for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    const int r = u / MV, jv = u - r * MV;
    uint32_t base = (uint32_t)r;
#pragma unroll
    for (int i = 0; i < U; ++i) {
      const int p = a.g.ins[i];
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
    for (int t = 0; t < ROWS; ++t) ld_keep<T, VEC>(P + off(t), ph[t]);
    if (has_gate) {
#pragma unroll
      for (int t0 = 0; t0 < ROWS / 4; ++t0) {
        T2 nw[4][VEC];
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            T2 acc2 = cmul(gd(y, 0), ph[(0 << (U - 2)) | t0][q]);
#pragma unroll
            for (int yp = 1; yp < 4; ++yp) acc2 = cfma(gd(y, yp), ph[(yp << (U - 2)) | t0][q], acc2);
            nw[y][q] = acc2;
          }
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
          for (int q = 0; q < VEC; ++q) ph[(y << (U - 2)) | t0][q] = nw[y][q];
      }
      if (Po) {
#pragma unroll
        for (int t = 0; t < ROWS; ++t) st<T, VEC>(Po + off(t), ph[t]);
      }
    }
    if constexpr (MODE == 0) {
#pragma unroll
      for (int j = 0; j < ROWS / 4; ++j) {
        const int rest = spread_rest<U, EA, EB>(j);
        T2 b[4][VEC];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int t = rest | ((x >> 1) << EA) | ((x & 1) << EB);
          if (a.stream_b) ld<T, VEC>(B + off(t), b[x]);
          else ld_keep<T, VEC>(B + off(t), b[x]);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int ty = rest | ((y >> 1) << EA) | ((y & 1) << EB);
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
              const T2 bb = b[x][q], pp = ph[ty][q];
              cfma_conj(acc[2 * (4 * x + y)], acc[2 * (4 * x + y) + 1], bb, pp);
            }
          }
      }
    } else {
#pragma unroll
      for (int t = 0; t < ROWS; ++t) {
        T2 b[VEC];
        ld_keep<T, VEC>(B + off(t), b);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          const T dx = ph[t][q].x - b[q].x, dy = ph[t][q].y - b[q].y;
          acc[0] = fmat(dx, dx, fmat(dy, dy, acc[0]));
        }
      }
    }
  }

  double mine;
  if constexpr (MODE == 0) {
    mine = (double)warp_reduce_scatter32<T>(acc, lane);
  } else {
    double v = (double)acc[0];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(FULL, v, m);
    mine = lane == 0 ? v : 0.0;
  }
  red[warp][lane] = mine;
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) t += red[w][lane];
    const long long slot = ((long long)s * a.nblk + blockIdx.x) * 32 + lane;
    if (MODE == 0) reinterpret_cast<T*>(a.partials)[slot] = (T)t;
    else reinterpret_cast<double*>(a.partials)[slot] = t;
  }
  if constexpr (MODE == 0) {
    if (a.fuse) {
      // Last block done: publish the partials, count the block, and let the
      // last one of this start run the update (no block ever waits).
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) is_last = atomicAdd(a.counters + s, 1u) == (unsigned)(a.nblk - 1);
      __syncthreads();
      if (is_last && warp == 0) {
        __threadfence();
        update_one_start<T, sizeof(T) == 4 ? 1 : 2, true>(a.upd, s, sm_polar);
        if (lane == 0) a.counters[s] = 0u;
      }
    }
  }
}

// Backward step for 16-row units (gate k+1 and gate k on four distinct
// qubits, the common case in brick walls).  Four lanes share a unit: lane
// quad index x (lane bits 3..4) owns the rows with gate k's local index x
// and all four values j of gate k+1's local index, for VEC samples.  It
// applies g_{k+1}^dagger to its own four Phi rows, stores them, and
// accumulates E_k[x][x^m] += sum_j B[(j, x)] conj(Phi_k[(j, x^m)]) with the
// partner's rows fetched by shuffle (lane ^ 8m).  Registers stay low (all
// eight loads of a lane are in flight together) and each unit's 16 rows are
// read once.  Local bits: 3, 2 = gate k+1, 1, 0 = gate k.
template <typename T, int VEC>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 3 : 2) k_backward_q4(BwdArgs a) {
  using T2 = typename C2<T>::t;
  const int s = blockIdx.y;
  if (a.active && !a.active[s]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int qx = lane >> 3, v = lane & 7;
  __shared__ T2 gs[16];
  __shared__ double red[4][32];
  __shared__ double2 sm_polar[32];
  __shared__ int is_last;
  const bool has_gate = a.gates != nullptr;
  if (threadIdx.x < 16)
    gs[threadIdx.x] = has_gate ? reinterpret_cast<const T2*>(a.gates)[s * a.gate_stride + threadIdx.x] : T2{};
  __syncthreads();
  T2 gd[16];  // g^dagger[y][j] = conj(g[j][y])
#pragma unroll
  for (int y = 0; y < 4; ++y)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T2 t = gs[4 * j + y];
      gd[4 * y + j] = T2{t.x, -t.y};
    }
  const T2* B = reinterpret_cast<const T2*>(a.bprev) + s * a.bprev_stride;
  const T2* P = reinterpret_cast<const T2*>(a.phi_in) + s * a.phi_in_stride;
  T2* Po = a.phi_out ? reinterpret_cast<T2*>(a.phi_out) + s * a.g.sN : nullptr;
  const uint32_t M = (uint32_t)a.g.M;
  const uint32_t d0 = (1u << a.g.pos[0]) * M, d1 = (1u << a.g.pos[1]) * M;
  const uint32_t d2 = (1u << a.g.pos[2]) * M, d3 = (1u << a.g.pos[3]) * M;
  const uint32_t xoff = ((qx >> 1) ? d1 : 0u) + ((qx & 1) ? d0 : 0u);
  const uint32_t joff[4] = {0u, d2, d3, d3 + d2};

  T acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = T(0);

  const int MV = a.g.M / VEC;
  const int u0 = blockIdx.x * a.chunk;
  const int u1 = min(u0 + a.chunk, a.units_per_start);
  // Loads of unit u: four Phi rows and four B rows of this lane.
  auto unit_off = [&](int u) {
    const int r = u / MV, jv = u - r * MV;
    uint32_t base = (uint32_t)r;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = a.g.ins[i];
      base = ((base >> p) << (p + 1)) | (base & ((1u << p) - 1u));
    }
    return base * M + (uint32_t)jv * VEC + xoff;
  };
  auto load_unit = [&](int u, T2 (&ph)[4][VEC], T2 (&b)[4][VEC]) {
    if (u < u1) {
      const uint32_t o = unit_off(u);
#pragma unroll
      for (int j = 0; j < 4; ++j) ld_keep<T, VEC>(P + o + joff[j], ph[j]);
      if (a.stream_b) {
#pragma unroll
        for (int j = 0; j < 4; ++j) ld<T, VEC>(B + o + joff[j], b[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) ld_keep<T, VEC>(B + o + joff[j], b[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < VEC; ++q) ph[j][q] = b[j][q] = T2{T(0), T(0)};
    }
  };
  // Software pipeline: the next unit's eight loads are in flight while the
  // current unit is computed.
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
    if (has_gate) {
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
      if (Po && valid) {
#pragma unroll
        for (int y = 0; y < 4; ++y) st<T, VEC>(Po + base_off + joff[y], ph[y]);
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
          cfma_conj(acc[2 * m], acc[2 * m + 1], bb, pp);
        }
    }
  }
  // Sum over the eight lanes of each quad index; lane (x, 0) holds E[x][x^m].
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    acc[i] += __shfl_xor_sync(FULL, acc[i], 1);
    acc[i] += __shfl_xor_sync(FULL, acc[i], 2);
    acc[i] += __shfl_xor_sync(FULL, acc[i], 4);
  }
  if (v == 0) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int e = 4 * qx + (qx ^ m);
      red[warp][2 * e] = (double)acc[2 * m];
      red[warp][2 * e + 1] = (double)acc[2 * m + 1];
    }
  }
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) t += red[w][lane];
    reinterpret_cast<T*>(a.partials)[((long long)s * a.nblk + blockIdx.x) * 32 + lane] = (T)t;
  }
  if (a.fuse) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(a.counters + s, 1u) == (unsigned)(a.nblk - 1);
    __syncthreads();
    if (is_last && warp == 0) {
      __threadfence();
      update_one_start<T, sizeof(T) == 4 ? 1 : 2, true>(a.upd, s, sm_polar);
      if (lane == 0) a.counters[s] = 0u;
    }
  }
}

void launch_forward(Real r, const Geom& g, const Shape& sh, int S, const void* in,
                    long long in_stride, void* out, const void* gates, long long gate_stride,
                    const int* active, cudaStream_t st) {
  FwdArgs a{in, in_stride, out, gates, gate_stride, g, sh.units_per_start, sh.chunk, active};
  dim3 grid(sh.nblk, S);
  if (r == R32) {
    if (sh.vec == 2) k_forward<float, 2><<<grid, sh.threads, 0, st>>>(a);
    else k_forward<float, 1><<<grid, sh.threads, 0, st>>>(a);
  } else {
    k_forward<double, 1><<<grid, sh.threads, 0, st>>>(a);
  }
}

template <typename T, int VEC, int MODE>
static void bwd_dispatch(const BwdArgs& a, dim3 grid, int threads, cudaStream_t st) {
  const int U = a.g.U, ea = a.g.ea, eb = a.g.eb;
  if constexpr (MODE == 1) {
    k_backward<T, VEC, 1, 2, 1, 0><<<grid, threads, 0, st>>>(a);
  } else {
    if (U == 4) k_backward_q4<T, VEC><<<grid, threads, 0, st>>>(a);
    else if (U == 3) {
      if (ea == 2 && eb == 0) k_backward<T, VEC, 0, 3, 2, 0><<<grid, threads, 0, st>>>(a);
      else if (ea == 0 && eb == 2) k_backward<T, VEC, 0, 3, 0, 2><<<grid, threads, 0, st>>>(a);
      else if (ea == 1 && eb == 0) k_backward<T, VEC, 0, 3, 1, 0><<<grid, threads, 0, st>>>(a);
      else k_backward<T, VEC, 0, 3, 0, 1><<<grid, threads, 0, st>>>(a);
    } else {
      if (ea == 1) k_backward<T, VEC, 0, 2, 1, 0><<<grid, threads, 0, st>>>(a);
      else k_backward<T, VEC, 0, 2, 0, 1><<<grid, threads, 0, st>>>(a);
    }
  }
}

// Resident 128-thread blocks per SM of the backward kernel a shape uses
// (cached per instance; the unit shape decides the instance).
int bwd_resident_blocks(Real r, int vec, int U) {
  static int cache[2][3][5] = {};
  const int ri = r == R32 ? 0 : 1;
  int& c = cache[ri][vec][U];
  if (c) return c;
  int b = 0;
  cudaError_t e = cudaSuccess;
  if (r == R32) {
    if (U == 4) e = vec == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward_q4<float, 2>, 128, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward_q4<float, 1>, 128, 0);
    else if (U == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward<float, 1, 0, 3, 1, 0>, 128, 0);
    else e = vec == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward<float, 2, 0, 2, 1, 0>, 128, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward<float, 1, 0, 2, 1, 0>, 128, 0);
  } else {
    if (U == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward_q4<double, 1>, 128, 0);
    else if (U == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward<double, 1, 0, 3, 1, 0>, 128, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward<double, 1, 0, 2, 1, 0>, 128, 0);
  }
  if (e != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 2;
  }
  c = b;
  return c;
}

void launch_backward(Real r, int mode, const BwdGeom& g, const Shape& sh, int S,
                     const void* bprev, long long bprev_stride, const void* phi_in,
                     long long phi_in_stride, void* phi_out, const void* gates,
                     long long gate_stride, void* partials, int stream_b, const int* active,
                     cudaStream_t st, const UpdateArgs* fuse, unsigned* counters) {
  BwdArgs a{bprev, bprev_stride, phi_in, phi_in_stride, phi_out, gates, gate_stride,
            partials, sh.nblk, g, sh.units_per_start, sh.chunk, stream_b, active,
            fuse ? 1 : 0, counters, fuse ? *fuse : UpdateArgs{}};
  dim3 grid(sh.nblk, S);
  if (r == R32) {
    if (sh.vec == 2) {
      if (mode == 0) bwd_dispatch<float, 2, 0>(a, grid, sh.threads, st);
      else bwd_dispatch<float, 2, 1>(a, grid, sh.threads, st);
    } else {
      if (mode == 0) bwd_dispatch<float, 1, 0>(a, grid, sh.threads, st);
      else bwd_dispatch<float, 1, 1>(a, grid, sh.threads, st);
    }
  } else {
    if (mode == 0) bwd_dispatch<double, 1, 0>(a, grid, sh.threads, st);
    else bwd_dispatch<double, 1, 1>(a, grid, sh.threads, st);
  }
}

// ------------------------------------------------------------ U * Psi (FP64)

// Each block computes 16 rows x 32 columns; each thread two rows of one column.
__global__ void k_gemm_upsi(const double2* __restrict__ U, const double2* __restrict__ Psi,
                            double2* __restrict__ out, int N, int M) {
  __shared__ double2 Us[16][33];
  __shared__ double2 Ps[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int row0 = blockIdx.x * 16;
  const int col = blockIdx.y * 32 + tx;
  double2 acc0{0.0, 0.0}, acc1{0.0, 0.0};
  for (int k0 = 0; k0 < N; k0 += 32) {
    for (int i = ty; i < 16; i += 8) {
      const int row = row0 + i, k = k0 + tx;
      Us[i][tx] = (row < N && k < N) ? U[(long long)row * N + k] : double2{0.0, 0.0};
    }
    for (int i = ty; i < 32; i += 8) {
      const int k = k0 + i;
      Ps[i][tx] = (k < N && col < M) ? Psi[(long long)k * M + col] : double2{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const double2 p = Ps[k][tx];
      const double2 u0 = Us[2 * ty][k], u1 = Us[2 * ty + 1][k];
      acc0.x = fma(u0.x, p.x, fma(-u0.y, p.y, acc0.x));
      acc0.y = fma(u0.x, p.y, fma(u0.y, p.x, acc0.y));
      acc1.x = fma(u1.x, p.x, fma(-u1.y, p.y, acc1.x));
      acc1.y = fma(u1.x, p.y, fma(u1.y, p.x, acc1.y));
    }
    __syncthreads();
  }
  if (col < M) {
    const int r0 = row0 + 2 * ty;
    if (r0 < N) out[(long long)r0 * M + col] = acc0;
    if (r0 + 1 < N) out[(long long)(r0 + 1) * M + col] = acc1;
  }
}

void launch_gemm_upsi(const double2* U, const double2* Psi, double2* out, int N, int M,
                      cudaStream_t st) {
  dim3 grid((N + 15) / 16, (M + 31) / 32);
  k_gemm_upsi<<<grid, dim3(32, 8), 0, st>>>(U, Psi, out, N, M);
}

// ------------------------------------------- U * Psi in FP32 pair arithmetic
//
// The same product to FP64-class accuracy on the FP32 pipe, which issues 64x
// the FP64 rate on this GPU.  Every FP64 operand x is split into two floats,
// x = x_h + x_l (x_h = fl32(x), x_l = fl32(x - x_h)), and every real product
// u psi is formed as u_h psi_h exactly (Dekker's product through an FMA: the
// rounded product plus its exact error) plus the cross terms u_h psi_l and
// u_l psi_h (u_l psi_l, below 2^-48 relative, is dropped).  The rounded
// products enter a float accumulator S through Knuth's two-sum, whose exact
// rounding error goes, with the small terms, into a second float s (the
// pair is renormalised every 32 terms).  A pair carries about 48 bits: the
// result is within ~2^-44 of the exact sum in the worst case at K = 4096.
//
// Work: tiles of 16 rows x 32 columns x one K slab; four warps, warp w owns
// rows 4w..4w+3 of its tile, lane c column c.  Slab partials (as doubles)
// go to a scratch buffer and a second kernel adds them in FP64.

__global__ void k_split_psi(const double2* __restrict__ psi, float4* __restrict__ out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = psi[i];
    const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
    out[i] = float4{hx, hy, __double2float_rn(v.x - (double)hx), __double2float_rn(v.y - (double)hy)};
  }
}

namespace {
// The _rn intrinsics keep every rounding where it is written: the compiler
// never contracts them into an FMA, which would void the error identities.
__device__ __forceinline__ void pair_add(float& S, float& s, float p) {
  const float t = __fadd_rn(S, p);
  const float bp = __fsub_rn(t, S);
  s = __fadd_rn(s, __fadd_rn(__fsub_rn(S, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
  S = t;
}
__device__ __forceinline__ void pair_norm(float& S, float& s) {
  const float t = __fadd_rn(S, s);
  const float bp = __fsub_rn(t, S);
  s = __fadd_rn(__fsub_rn(S, __fsub_rn(t, bp)), __fsub_rn(s, bp));
  S = t;
}
// acc (Sr, sr, Si, si) += u * p, u = (hr, hi, lr, li) likewise p.
__device__ __forceinline__ void pair_cmac(float4& acc, const float4 u, const float4 p) {
  const float a = __fmul_rn(u.x, p.x), b = __fmul_rn(-u.y, p.y), c = __fmul_rn(u.x, p.y), d = __fmul_rn(u.y, p.x);
  const float ea = fmaf(u.x, p.x, -a), eb = fmaf(-u.y, p.y, -b);
  const float ec = fmaf(u.x, p.y, -c), ed = fmaf(u.y, p.x, -d);
  const float smr = fmaf(u.x, p.z, fmaf(u.z, p.x, fmaf(-u.y, p.w, fmaf(-u.w, p.y, ea + eb))));
  const float smi = fmaf(u.x, p.w, fmaf(u.z, p.y, fmaf(u.y, p.z, fmaf(u.w, p.x, ec + ed))));
  pair_add(acc.x, acc.y, a);
  pair_add(acc.x, acc.y, b);
  acc.y = __fadd_rn(acc.y, smr);
  pair_add(acc.z, acc.w, c);
  pair_add(acc.z, acc.w, d);
  acc.w = __fadd_rn(acc.w, smi);
}
}  // namespace

constexpr int kPairRows = 16, kPairCols = 32, kPairK = 32;

__global__ void __launch_bounds__(128) k_gemm_upsi_pair(const double2* __restrict__ U, const float4* __restrict__ P,
                                                        double2* __restrict__ part, int N, int M, int slab,
                                                        int row_tiles, int col_tiles, int splits) {
  __shared__ float4 Us[kPairRows][kPairK + 1];
  __shared__ float4 Ps[kPairK][kPairCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long tiles = (long long)row_tiles * col_tiles * splits;
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int sp = (int)(t % splits);
    const long long rc = t / splits;
    const int ct = (int)(rc % col_tiles), rt = (int)(rc / col_tiles);
    const int row0 = rt * kPairRows, col = ct * kPairCols + lane;
    const int k0 = sp * slab, k1 = min(N, k0 + slab);
    float4 acc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] = float4{0.f, 0.f, 0.f, 0.f};
    for (int kc = k0; kc < k1; kc += kPairK) {
      // U chunk: 16 rows x 32 k, split on the way into shared memory.
#pragma unroll
      for (int i = 0; i < (kPairRows * kPairK) / 128; ++i) {
        const int e = i * 128 + threadIdx.x;
        const int r = e / kPairK, k = e % kPairK;
        const int row = row0 + r, kk = kc + k;
        float4 v{0.f, 0.f, 0.f, 0.f};
        if (row < N && kk < k1) {
          const double2 x = U[(long long)row * N + kk];
          const float hx = __double2float_rn(x.x), hy = __double2float_rn(x.y);
          v = float4{hx, hy, __double2float_rn(x.x - (double)hx), __double2float_rn(x.y - (double)hy)};
        }
        Us[r][k] = v;
      }
#pragma unroll
      for (int i = 0; i < (kPairK * kPairCols) / 128; ++i) {
        const int e = i * 128 + threadIdx.x;
        const int k = e / kPairCols, c = e % kPairCols;
        const int kk = kc + k, cc = ct * kPairCols + c;
        Ps[k][c] = (kk < k1 && cc < M) ? P[(long long)kk * M + cc] : float4{0.f, 0.f, 0.f, 0.f};
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < kPairK; ++k) {
        const float4 p = Ps[k][lane];
#pragma unroll
        for (int r = 0; r < 4; ++r) pair_cmac(acc[r], Us[4 * warp + r][k], p);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        pair_norm(acc[r].x, acc[r].y);
        pair_norm(acc[r].z, acc[r].w);
      }
      __syncthreads();
    }
    if (col < M) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = row0 + 4 * warp + r;
        if (row < N)
          part[((long long)sp * N + row) * M + col] =
              double2{(double)acc[r].x + (double)acc[r].y, (double)acc[r].z + (double)acc[r].w};
      }
    }
  }
}

__global__ void k_sum_slabs(const double2* __restrict__ part, double2* __restrict__ out, long long count,
                            int splits) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    double2 a = part[i];
    for (int s = 1; s < splits; ++s) {
      const double2 b = part[(long long)s * count + i];
      a.x += b.x;
      a.y += b.y;
    }
    out[i] = a;
  }
}

int upsi_pair_splits(int N, int M, int num_sms, size_t scratch_bytes) {
  const long long base = (long long)((N + kPairRows - 1) / kPairRows) * ((M + kPairCols - 1) / kPairCols);
  const long long want_tiles = 12LL * std::max(num_sms, 1);
  int splits = (int)std::min<long long>(16, std::max<long long>(1, (want_tiles + base - 1) / base));
  // Each slab is a whole number of K chunks; the scratch holds every slab.
  while (splits > 1 && ((size_t)splits * N * M * sizeof(double2) > scratch_bytes || N / splits < kPairK)) --splits;
  return splits;
}

void launch_gemm_upsi_pair(const double2* U, const double2* Psi, double2* out, int N, int M, float4* psi_split,
                           double2* scratch, int splits, int num_sms, cudaStream_t st) {
  const long long count = (long long)N * M;
  k_split_psi<<<(unsigned)std::min<long long>((count + 255) / 256, 4096), 256, 0, st>>>(Psi, psi_split, count);
  int slab = (N + splits - 1) / splits;
  slab = (slab + kPairK - 1) / kPairK * kPairK;
  const int row_tiles = (N + kPairRows - 1) / kPairRows, col_tiles = (M + kPairCols - 1) / kPairCols;
  const long long tiles = (long long)row_tiles * col_tiles * splits;
  static int per_sm = 0;  // resident CTAs per SM: the grid is one full wave
  if (per_sm == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm_upsi_pair, 128, 0) != cudaSuccess)
    per_sm = 4;
  const long long grid = std::min<long long>(tiles, (long long)std::max(per_sm, 1) * std::max(num_sms, 1));
  double2* dst = splits == 1 ? out : scratch;
  k_gemm_upsi_pair<<<(unsigned)grid, 128, 0, st>>>(U, psi_split, dst, N, M, slab, row_tiles, col_tiles, splits);
  if (splits > 1)
    k_sum_slabs<<<(unsigned)std::min<long long>((count + 255) / 256, 4096), 256, 0, st>>>(scratch, out, count,
                                                                                             splits);
}

__global__ void k_cast(const double2* in, float2* out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = float2{(float)v.x, (float)v.y};
  }
}

void launch_cast_c128_to_c64(const double2* in, float2* out, long long count, cudaStream_t st) {
  if (count <= 0) return;
  long long blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_cast<<<(int)blocks, 256, 0, st>>>(in, out, count);
}

__global__ void k_nonfinite(const double* x, long long count, int* flag) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    bad |= !isfinite(v);
  }
  if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

void launch_nonfinite_check(const double* x, long long count, int* flag, cudaStream_t st) {
  if (count <= 0) return;
  long long blocks = (count + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_nonfinite<<<(int)blocks, 256, 0, st>>>(x, count, flag);
}

}  // namespace qfs
