// Batched QFactor-Sample: many small instantiation problems (3-5 qubits,
// 2-10 two-qubit gates each) and their multistarts in one persistent launch.
//
// Each warp runs whole instantiations of one (problem, start) pair taken from
// an atomic work queue ordered largest problem first.  A warp keeps its
// running state B and Phi (N x M complex, N <= 32, M <= 16) and its gates in
// its own slice of shared memory and sweeps as in Section 3 of the paper;
// the list of intermediate states is replaced by walking B back with the
// old gate (B_{k-1} = g_k^dagger B_k), so nothing leaves the SM between
// sweeps.  Environments are reduced with one warp reduce-scatter; the update
// (Eq. 2) is the FP32 Jacobi polar factor with a Newton-Schulz step (FP64
// Jacobi for ill-conditioned environments).  The run's stop rule is kept
// without any waiting: a start stops when it converges or once its sweep
// passes the earliest converged sweep of its problem (an atomicMin); the
// lowest-cost start among those that converged at that sweep is the
// problem's answer, which is what lock-step multistarts would return.
// A finishing kernel then makes the selected gates unitary in FP64, checks
// the cost in FP64 and, if needed, refines with FP64 sweeps.
#include "polar4.cuh"
#include "qfs_common.cuh"
#include "qfs_kernels.h"

#include <climits>

namespace qfs {

namespace {

template <typename T> struct BT;
template <> struct BT<float> { using t2 = float2; };
template <> struct BT<double> { using t2 = double2; };

__device__ __forceinline__ uint32_t ins2(uint32_t r, int lo, int hi) {
  r = ((r >> lo) << (lo + 1)) | (r & ((1u << lo) - 1u));
  r = ((r >> hi) << (hi + 1)) | (r & ((1u << hi) - 1u));
  return r;
}

// X <- g X (dag = false) or X <- g^dagger X (dag = true) on qubits (qa, qb),
// X an N x M state in this warp's shared memory.
template <typename T2>
__device__ void warp_apply(T2* X, const T2* g, int n, int M, int qa, int qb, bool dag) {
  const int lane = threadIdx.x & 31;
  const int pa = n - 1 - qa, pb = n - 1 - qb;
  const int lo = min(pa, pb), hi = max(pa, pb);
  const int groups = (1 << (n - 2)) * M;
  // The operator in registers (the state writes below could alias it for
  // the compiler): gg[4y + x] = (g or g^dagger)[y][x].
  T2 gg[16];
#pragma unroll
  for (int y = 0; y < 4; ++y)
#pragma unroll
    for (int x = 0; x < 4; ++x) gg[4 * y + x] = dag ? T2{g[4 * x + y].x, -g[4 * x + y].y} : g[4 * y + x];
  __syncwarp();
  for (int w = lane; w < groups; w += 32) {
    const int r = w / M, j = w - r * M;
    const uint32_t base = ins2((uint32_t)r, lo, hi);
    int off[4];
    T2 v[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      off[x] = (int)((base | ((uint32_t)(x >> 1) << pa) | ((uint32_t)(x & 1) << pb)) * M + j);
      v[x] = X[off[x]];
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      T2 t{0, 0};
#pragma unroll
      for (int x = 0; x < 4; ++x) t = cfma(gg[4 * y + x], v[x], t);
      X[off[y]] = t;
    }
  }
  __syncwarp();
}

// E[x][y] = sum B[x] conj(Phi[y]) over the groups of (qa, qb); on return
// lane l16 < 16 holds the complex entry E[c][r] with l16 = 4c + r, the
// layout the polar routines take (as A[r][c] after conjugation).
template <typename T, typename T2>
__device__ T2 warp_env(const T2* Bs, const T2* Ph, int n, int M, int qa, int qb) {
  const int lane = threadIdx.x & 31;
  const int pa = n - 1 - qa, pb = n - 1 - qb;
  const int lo = min(pa, pb), hi = max(pa, pb);
  const int groups = (1 << (n - 2)) * M;
  T acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = T(0);
  for (int w = lane; w < groups; w += 32) {
    const int r = w / M, j = w - r * M;
    const uint32_t base = ins2((uint32_t)r, lo, hi);
    T2 b[4], p[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int off = (int)((base | ((uint32_t)(x >> 1) << pa) | ((uint32_t)(x & 1) << pb)) * M + j);
      b[x] = Bs[off];
      p[x] = Ph[off];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        cfma_conj(acc[2 * (4 * x + y)], acc[2 * (4 * x + y) + 1], b[x], p[y]);
      }
  }
  const T v = warp_reduce_scatter32<T>(acc, lane);
  const int l16 = lane & 15;
  return T2{__shfl_sync(FULL, v, 2 * l16), __shfl_sync(FULL, v, 2 * l16 + 1)};
}

// New gate from E (E[c][r] in lane 4c + r): the polar factor of E^dagger.
template <typename T2>
__device__ void warp_update(T2 e, T2* g, double2* sm, float2* v);

// v: the gate's right singular vectors from its previous update (the Jacobi
// start; identity at the first sweep), updated in place.
template <>
__device__ void warp_update<float2>(float2 e, float2* g, double2* sm, float2* v) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, r = l16 & 3, c = l16 >> 2;
  const float2 a32{e.x, -e.y};  // A[r][c] = conj(E[c][r])
  float2 q;
  if (!warp_polar4_f32_warm(a32, v, &q)) {
    const double2 p =
        warp_polar4(double2{(double)e.x, -(double)e.y}, double2{r == c ? 1.0 : 0.0, 0.0}, sm, nullptr);
    q = float2{(float)p.x, (float)p.y};
    if (lane < 16) v[l16] = float2{r == c ? 1.f : 0.f, 0.f};  // restart from the identity
  }
  if (lane < 16) g[4 * r + c] = q;
  __syncwarp();
}

template <>
__device__ void warp_update<double2>(double2 e, double2* g, double2* sm, float2* v) {
  (void)v;
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, r = l16 & 3, c = l16 >> 2;
  double2 p;
  polar_update_warp<2>(e, nullptr, 0.0, sm, g, nullptr, &p, nullptr);
  (void)r;
  (void)c;
  __syncwarp();
}

// (1/M) sum |g_1^dagger Phi_1 - Psi|^2 after the sweep (Phi_1 in Ph, which
// is overwritten).
template <typename T, typename T2>
__device__ T warp_residual(T2* Ph, const T2* g1, const T2* psi, int n, int M, int qa, int qb) {
  warp_apply<T2>(Ph, g1, n, M, qa, qb, true);
  const int lane = threadIdx.x & 31;
  const int E = M << n;
  // A sum of squares in the sweep's own precision: no cancellation, so its
  // relative error stays ~1e-6 even for the largest states, far below what
  // the FP64 check at dist_tol needs (FP64 on this GPU would cost a
  // 64-cycle warp instruction per operation).
  T acc = T(0);
  for (int i = lane; i < E; i += 32) {
    const T2 p = Ph[i], q = psi[i];
    const T dx = p.x - q.x, dy = p.y - q.y;
    acc = fmat(dx, dx, fmat(dy, dy, acc));
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
  if constexpr (sizeof(T) == 4) return acc * (1.f / (float)M);
  else return acc / M;
}

// One sweep of one start (Section 3): forward to B_{L-1} with the current
// gates, then k = L..1: environment from (B_{k-1}, Phi_k), update gate k,
// B_{k-2} = g_{k-1}^dagger B_{k-1} (old gate), Phi_{k-1} = g_k^dagger Phi_k
// (new gate).  Returns the residual cost of the swept gates.
template <typename T, typename T2>
__device__ T warp_sweep(T2* Bs, T2* Ph, T2* G, const T2* psi, const T2* phil, const int* pairs,
                             int n, int M, int L, double2* sm, float2* V = nullptr) {
  const int lane = threadIdx.x & 31;
  const int E = M << n;
  for (int i = lane; i < E; i += 32) Bs[i] = psi[i];
  __syncwarp();
  for (int k = 1; k <= L - 1; ++k) warp_apply<T2>(Bs, G + 16 * (k - 1), n, M, pairs[2 * (k - 1)], pairs[2 * (k - 1) + 1], false);
  for (int i = lane; i < E; i += 32) Ph[i] = phil[i];
  __syncwarp();
  for (int k = L; k >= 1; --k) {
    const int qa = pairs[2 * (k - 1)], qb = pairs[2 * (k - 1) + 1];
    const T2 e = warp_env<T, T2>(Bs, Ph, n, M, qa, qb);
    warp_update<T2>(e, G + 16 * (k - 1), sm, V ? V + 16 * (k - 1) : nullptr);
    if (k > 1) {
      warp_apply<T2>(Bs, G + 16 * (k - 2), n, M, pairs[2 * (k - 2)], pairs[2 * (k - 2) + 1], true);
      warp_apply<T2>(Ph, G + 16 * (k - 1), n, M, qa, qb, true);
    }
  }
  return warp_residual<T, T2>(Ph, G, psi, n, M, pairs[0], pairs[1]);
}

}  // namespace

// Per-problem set-up: Phi_L = U Psi in FP64 and complex64 copies of Psi and
// Phi_L.  One block per problem.
__global__ void k_batch_prep(BatchArgs a) {
  const int p = blockIdx.x;
  if (p >= a.P) return;
  const BatchProblem pr = a.probs[p];
  const int N = 1 << pr.n, M = pr.M;
  const double2* U = a.targets + pr.target_off;
  const double2* psi = a.psi64 + pr.state_off;
  for (int e = threadIdx.x; e < N * M; e += blockDim.x) {
    const int i = e / M, j = e - i * M;
    double2 acc{0.0, 0.0};
    for (int k = 0; k < N; ++k) {
      const double2 u = U[(size_t)i * N + k], s = psi[(size_t)k * M + j];
      acc.x = fma(u.x, s.x, fma(-u.y, s.y, acc.x));
      acc.y = fma(u.x, s.y, fma(u.y, s.x, acc.y));
    }
    a.phil64[pr.state_off + e] = acc;
    a.phil32[pr.state_off + e] = float2{(float)acc.x, (float)acc.y};
    const double2 s = psi[e];
    a.psi32[pr.state_off + e] = float2{(float)s.x, (float)s.y};
  }
  if (threadIdx.x == 0) a.s_star[p] = INT_MAX;
}

// Persistent sweep kernel: warps take (problem, start) items until the queue
// is empty.
__global__ void k_batch_sweep(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double2 sm_polar[kBatchMaxWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int E = a.max_elems;
  float2* base = reinterpret_cast<float2*>(dsm) + (size_t)warp * (2 * E + 32 * a.max_L);
  float2* Bs = base;
  float2* Ph = base + E;
  float2* G = base + 2 * E;
  float2* V = G + 16 * a.max_L;  // per gate: right singular vectors of its last update
  const int total = a.P * a.S;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= total) break;
    const int p = a.order[item / a.S], s = item % a.S;
    const BatchProblem pr = a.probs[p];
    const int* pairs = a.pairs + pr.pair_off;
    const size_t goff = pr.gate_off + (size_t)s * pr.L * 16;
    for (int i = lane; i < 16 * pr.L; i += 32) {
      const double2 g = a.init_gates[goff + i];
      G[i] = float2{(float)g.x, (float)g.y};
      const int e = i & 15;
      V[i] = float2{(e & 3) == (e >> 2) ? 1.f : 0.f, 0.f};
    }
    __syncwarp();
    const float2* psi = a.psi32 + pr.state_off;
    const float2* phil = a.phil32 + pr.state_off;
    int conv = INT_MAX, sweeps = 0, stall = 0;
    // The sweep's cost and the plateau test stay in FP32 (the FP64 pipe
    // costs 64 cycles per warp instruction); only the tolerance test is FP64.
    float cost = 4.f, prev = -1.f;
    const float dtr = (float)a.diff_tol_r;
    for (int sw = 1; sw <= a.max_sweeps; ++sw) {
      // A start that has not converged by its problem's earliest converged
      // sweep can no longer be selected.
      if (sw > *(volatile int*)(a.s_star + p)) break;
      cost = warp_sweep<float, float2>(Bs, Ph, G, psi, phil, pairs, pr.n, pr.M, pr.L, sm_polar[warp], V);
      sweeps = sw;
      if ((double)cost <= a.tol) {
        conv = sw;
        if (lane == 0) atomicMin(a.s_star + p, sw);
        break;
      }
      // Plateau (App. A): no relative improvement > diff_tol_r for
      // plateau_window sweeps in a row stops this start.
      if (a.plateau_window > 0 && prev >= 0.f) {
        stall = fabsf(prev) - fabsf(cost) > dtr * fabsf(cost) ? 0 : stall + 1;
        if (stall >= a.plateau_window && sw >= a.min_sweeps) break;
      }
      prev = cost;
    }
    const size_t ri = (size_t)p * a.S + s;
    if (lane == 0) {
      a.conv_sweep[ri] = conv;
      a.final_cost[ri] = (double)cost;
      a.sweeps_run[ri] = sweeps;
    }
    for (int i = lane; i < 16 * pr.L; i += 32) a.gates32[goff + i] = G[i];
    __syncwarp();
  }
}

// One warp per problem: pick the start, make its gates unitary in FP64, FP64
// cost check, FP64 refinement sweeps while the cost is above tol.
__global__ void k_batch_finalize(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double2 sm_polar[32];
  const int p = blockIdx.x;
  if (p >= a.P) return;
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, row = l16 & 3, col = l16 >> 2;
  const BatchProblem pr = a.probs[p];
  const int E = pr.M << pr.n;
  double2* Bs = reinterpret_cast<double2*>(dsm);
  double2* Ph = Bs + a.max_elems;
  double2* G = Ph + a.max_elems;
  // Selection: among starts converged at the earliest converged sweep, the
  // lowest cost (lowest index on ties); if none converged, the lowest cost.
  int best = 0;
  const int sst = a.s_star[p];
  double bc = 1e300;
  for (int s = 0; s < a.S; ++s) {
    const size_t ri = (size_t)p * a.S + s;
    const bool eligible = sst == INT_MAX || a.conv_sweep[ri] == sst;
    const double c = a.final_cost[ri];
    if (eligible && c < bc) {
      bc = c;
      best = s;
    }
  }
  int sweeps = sst == INT_MAX ? a.sweeps_run[(size_t)p * a.S + best] : sst;
  const size_t goff = pr.gate_off + (size_t)best * pr.L * 16;
  // FP64 copy of the gates, made unitary by two Newton-Schulz steps.
  for (int k = 0; k < pr.L; ++k) {
    const float2 g32 = a.gates32[goff + 16 * k + (4 * row + col)];  // lane 4col+row holds g[row][col]
    double2 q{(double)g32.x, (double)g32.y};
    for (int it = 0; it < 2; ++it) {
      const double2 gq = mm64_ah(q, q, row, col, lane < 16);
      const double2 t{(row == col ? 1.5 : 0.0) - 0.5 * gq.x, -0.5 * gq.y};
      q = mm64(q, t, row, col, lane < 16);
    }
    if (lane < 16) G[16 * k + 4 * row + col] = q;
  }
  __syncwarp();
  const int* pairs = a.pairs + pr.pair_off;
  const double2* psi = a.psi64 + pr.state_off;
  const double2* phil = a.phil64 + pr.state_off;
  // FP64 cost: (1/M) || Phi_L - C Psi ||^2.
  auto cost64 = [&]() {
    for (int i = lane; i < E; i += 32) Bs[i] = psi[i];
    __syncwarp();
    for (int k = 1; k <= pr.L; ++k) warp_apply<double2>(Bs, G + 16 * (k - 1), pr.n, pr.M, pairs[2 * (k - 1)], pairs[2 * (k - 1) + 1], false);
    double acc = 0.0;
    for (int i = lane; i < E; i += 32) {
      const double dx = phil[i].x - Bs[i].x, dy = phil[i].y - Bs[i].y;
      acc += dx * dx + dy * dy;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    return acc / pr.M;
  };
  double c = cost64();
  int refine = 0;
  while (c > a.tol && refine < a.refine_max && (sst != INT_MAX || a.refine_unconverged)) {
    warp_sweep<double, double2>(Bs, Ph, G, psi, phil, pairs, pr.n, pr.M, pr.L, sm_polar);
    ++refine;
    c = cost64();
  }
  for (int i = lane; i < 16 * pr.L; i += 32) a.gates_out[pr.gate_out_off + i] = G[i];
  if (lane == 0) {
    a.res_cost[p] = c;
    a.res_sweeps[p] = sweeps;
    a.res_best[p] = best;
    a.res_refine[p] = refine;
  }
}

void launch_batch_prep(const BatchArgs& a, cudaStream_t st) {
  k_batch_prep<<<a.P, 128, 0, st>>>(a);
}

size_t batch_sweep_smem(int warps, int max_elems, int max_L) {
  return (size_t)warps * (2 * max_elems + 32 * max_L) * sizeof(float2);
}

int batch_sweep_blocks_per_sm(int warps, size_t smem) {
  cudaFuncSetAttribute(k_batch_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_sweep, 32 * warps, smem) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  return b < 1 ? 1 : b;
}

void launch_batch_sweep(const BatchArgs& a, int blocks, int warps, size_t smem, cudaStream_t st) {
  k_batch_sweep<<<blocks, 32 * warps, smem, st>>>(a);
}

void launch_batch_finalize(const BatchArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(2 * a.max_elems + 16 * a.max_L) * sizeof(double2);
  cudaFuncSetAttribute(k_batch_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_batch_finalize<<<a.P, 32, smem, st>>>(a);
}

}  // namespace qfs
