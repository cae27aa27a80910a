// Batched QFactor-Sample: many small instantiation problems (3-5 qubits,
// 2-10 two-qubit gates each) and their multistarts in one persistent launch.
//
// Work is handed out in units: a unit is one problem and 32/G of its starts,
// run by one warp with G lanes per start (G = 32: a warp per start; G = 16,
// 8 or 4: two, four or eight starts share a warp).  Each start keeps its
// running state B and Phi (N x M complex, N <= 32, M <= 16), its gates and
// the right singular vectors of their last updates in its own slice of
// shared memory and sweeps as in Section 3 of the paper; the list of
// intermediate states is replaced by walking B back with the old gate
// (B_{k-1} = g_k^dagger B_k), so nothing leaves the SM between sweeps.  The
// starts' state arithmetic (gate applications, environment sums) runs side
// by side in their lane groups; each group reduces its environment over its
// own lanes, and the warp then updates the unit's gates one after another
// (Eq. 2: the FP32 Jacobi polar factor, FP64 Jacobi for ill-conditioned
// environments).  Units come from an atomic work
// queue ordered largest problem first; the schedule G (and the warps per
// block) of each class of problems (n, L, M) is chosen by the host's
// autotuner.  The run's stop rule is kept without any waiting: a start stops
// when it converges or once its sweep passes the earliest converged sweep of
// its problem (an atomicMin); the lowest-cost start among those that
// converged at that sweep is the problem's answer, which is what lock-step
// multistarts would return.  A finishing kernel then makes the selected
// gates unitary in FP64, checks the cost in FP64 and, if needed, refines
// with FP64 sweeps.
#include "polar4.cuh"
#include "qfs_common.cuh"
#include "qfs_kernels.h"

#include <climits>

namespace qfs {

namespace {

// Polar factor in FP32 (batched complex64 sweeps) of A (lanes 0..15, A[r][c]
// at 4c + r): one-sided Jacobi on X = A V0, V0 the right singular vectors of
// the gate's previous update (16 complex at v_io, V[r][c] at 4c + r), whose
// columns are already nearly orthogonal once the sweeps settle, so few
// rotation sweeps are needed.  The new V, made unitary to FP32 rounding by
// one Newton-Schulz step (so that no drift accumulates over sweeps), is
// written back to v_io.  Returns false when sigma_min < 1e-3 sigma_max (the
// caller then takes the FP64 Jacobi, which also completes rank-deficient
// cases).
__device__ __forceinline__ bool warp_polar4_f32_warm(float2 a, float2* v_io, float2* q_out) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, row = l16 & 3, col = l16 >> 2;
  const bool isV = lane >= 16;
  const float2 v0 = v_io[l16];  // every lane: V0[row][col]
  float2 x;
  {
    float2 acc{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 ak = shfl_c(a, 4 * k + row), vk = shfl_c(v0, 4 * col + k);
      acc = cfma(ak, vk, acc);
    }
    x = isV ? v0 : acc;
  }
  bool rotated = false;
  x = jacobi32_sweeps(x, &rotated);
  float2 w = shfl_c(x, l16);
  float2 v = shfl_c(x, 16 + l16);
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
  w = float2{w.x * inv, w.y * inv};
  // Q = W V^H, unitary to the Jacobi tolerance (~1e-6), with no
  // Newton-Schulz step: the batched sweeps see that deviation only
  // quadratically in their residual cost, each update starts afresh, and the
  // finishing kernel makes the answer unitary in FP64.  V carries over
  // between sweeps, so it is renormalised.
  *q_out = mm_bh(w, v, row, col);
  if (rotated) {  // an unrotated V is the stored one: nothing to renormalise
    const float2 gv = mm_ah(v, v, row, col);
    const float2 tv{(row == col ? 1.5f : 0.f) - 0.5f * gv.x, -0.5f * gv.y};
    v = mm(v, tv, row, col);
    __syncwarp();
    if (lane < 16) v_io[l16] = v;
  }
  __syncwarp();
  return true;
}

template <typename T> struct BT;
template <> struct BT<float> { using t2 = float2; };
template <> struct BT<double> { using t2 = double2; };

__device__ __forceinline__ uint32_t ins2(uint32_t r, int lo, int hi) {
  r = ((r >> lo) << (lo + 1)) | (r & ((1u << lo) - 1u));
  r = ((r >> hi) << (hi + 1)) | (r & ((1u << hi) - 1u));
  return r;
}

// X <- g X (dag = false) or X <- g^dagger X (dag = true) on qubits (qa, qb),
// X an N x M state in shared memory, by the G lanes of one group (gl = lane
// within the group).  The caller synchronises the warp.
template <int G, typename T2>
__device__ void group_apply(T2* X, const T2* g, int n, int M, int qa, int qb, bool dag, int gl) {
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
  for (int w = gl; w < groups; w += G) {
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
}

// Reduce-scatter of 32 per-lane values over the G lanes of a group: on
// return lane gl holds, in v[0 .. 32/G - 1], the group's sums of the values
// base .. base + 32/G - 1, base returned.
template <int G, typename T>
__device__ __forceinline__ int group_reduce_scatter(T (&v)[32], int gl) {
  int base = 0;
  int cnt = 32;
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1) {
    cnt >>= 1;
    const bool upper = (gl & o) != 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (i < cnt) {
        const T send = upper ? v[i] : v[i + cnt];
        const T keep = upper ? v[i + cnt] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, o);
      }
    }
    if (upper) base += cnt;
  }
  return base;
}

// Environment partial sums of one start over its group's lanes:
// acc[2(4x+y)+{0,1}] += B[x] conj(Phi[y]) over the groups of (qa, qb).
template <int G, typename T, typename T2>
__device__ void group_env_acc(const T2* Bs, const T2* Ph, int n, int M, int qa, int qb, int gl, T (&acc)[32]) {
  const int pa = n - 1 - qa, pb = n - 1 - qb;
  const int lo = min(pa, pb), hi = max(pa, pb);
  const int groups = (1 << (n - 2)) * M;
  for (int w = gl; w < groups; w += G) {
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
  double2 p;
  polar_update_warp<2>(e, nullptr, 0.0, sm, g, nullptr, &p, nullptr);
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Two updates side by side, one per 16-lane half of the warp (the schedule
// with 16 lanes per start).  Each lane of a half holds one entry of X = A V
// and the same entry of V (M[row][col] at lane 4 col + row of the half), so
// a Jacobi round needs no exchange between an X lane and a V lane; every
// shuffle stays inside its half (width 16).

__device__ __forceinline__ float2 shfl16(float2 v, int src) {
  return float2{__shfl_sync(FULL, v.x, src, 16), __shfl_sync(FULL, v.y, src, 16)};
}
__device__ __forceinline__ float2 mm16(float2 a, float2 b, int row, int col) {
  float2 acc{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 4; ++k) acc = cfma(shfl16(a, 4 * k + row), shfl16(b, 4 * col + k), acc);
  return acc;
}
__device__ __forceinline__ float2 mm16_ah(float2 a, float2 b, int row, int col) {
  float2 acc{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 ak = shfl16(a, 4 * row + k), bk = shfl16(b, 4 * col + k);
    acc = cfma(float2{ak.x, -ak.y}, bk, acc);
  }
  return acc;
}
__device__ __forceinline__ float2 mm16_bh(float2 a, float2 b, int row, int col) {
  float2 acc{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 ak = shfl16(a, 4 * k + row), bk = shfl16(b, 4 * k + col);
    acc = cfma(ak, float2{bk.x, -bk.y}, acc);
  }
  return acc;
}
// Whether every column pair of this half's X has |gamma|^2 <= kJac32Tol
// alpha beta (the Gram-matrix test of jacobi32_converged), as a
// warp-uniform two-bit mask (bit h: half h).
__device__ __forceinline__ unsigned half_converged(float2 x, int row, int col) {
  const float2 g = mm16_ah(x, x, row, col);
  const float dr = __shfl_sync(FULL, g.x, 5 * row, 16), dc = __shfl_sync(FULL, g.x, 5 * col, 16);
  const bool ok = row == col || (g.x * g.x + g.y * g.y) <= kJac32Tol * dr * dc;
  const unsigned b = __ballot_sync(FULL, ok);
  return ((b & 0xffffu) == 0xffffu ? 1u : 0u) | ((b >> 16) == 0xffffu ? 2u : 0u);
}

// The polar factor of A (A[row][col] at lane 4 col + row of each half), the
// Jacobi started from V0 = v_io (that half's gate's right singular vectors
// from its previous update) and the new V written back, as
// warp_polar4_f32_warm does for one matrix.  Returns, warp-uniformly, a
// two-bit mask of the halves whose fast path succeeded; a half that failed
// (zero or too ill-conditioned) has not written v_io and its *q_out is
// undefined.  `act` (per half): whether this half's result is wanted.
__device__ unsigned halfwarp_polar4_f32_warm(float2 a, float2* v_io, bool act, float2* q_out) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, row = l16 & 3, col = l16 >> 2, h = lane >> 4;
  const float2 v0 = act ? v_io[l16] : float2{row == col ? 1.f : 0.f, 0.f};
  if (!act) a = float2{row == col ? 1.f : 0.f, 0.f};
  float2 x = mm16(a, v0, row, col);
  float2 v = v0;
  unsigned done = half_converged(x, row, col);
  bool rotated = false;
  for (int sweep = 0; sweep < 12 && done != 3u; ++sweep) {
    const bool mine_done = (done >> h) & 1u;
    bool any = false;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const float2 y = shfl16(x, l16 ^ (4 * m)), yv = shfl16(v, l16 ^ (4 * m));
      const bool isP = col < (col ^ m);
      float nown = x.x * x.x + x.y * x.y;
      float npar = y.x * y.x + y.y * y.y;
      float2 g = isP ? float2{x.x * y.x + x.y * y.y, x.x * y.y - x.y * y.x}
                     : float2{y.x * x.x + y.y * x.y, y.x * x.y - y.y * x.x};
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        nown += __shfl_xor_sync(FULL, nown, o);
        npar += __shfl_xor_sync(FULL, npar, o);
        g.x += __shfl_xor_sync(FULL, g.x, o);
        g.y += __shfl_xor_sync(FULL, g.y, o);
      }
      const float alpha = isP ? nown : npar, beta = isP ? npar : nown;
      const float ag2 = g.x * g.x + g.y * g.y;
      float cs = 1.f, sn = 0.f, px = 1.f, py = 0.f;
      if (!mine_done && ag2 > kJac32Tol * alpha * beta && ag2 > 1e-36f) {
        const float rg = rsqrtf(ag2);
        const float zeta = 0.5f * (beta - alpha) * rg;
        const float q = fmaf(zeta, zeta, 1.f);
        const float t = fabsf(zeta) > 1e18f ? __fdividef(0.5f, zeta)
                                             : copysignf(__fdividef(1.f, fabsf(zeta) + q * rsqrtf(q)), zeta);
        cs = rsqrtf(fmaf(t, t, 1.f));
        sn = t * cs;
        px = g.x * rg;
        py = -g.y * rg;
        any = true;
      }
      if (isP) {
        const float tx = px * y.x - py * y.y, ty = px * y.y + py * y.x;
        const float ux = px * yv.x - py * yv.y, uy = px * yv.y + py * yv.x;
        x = float2{cs * x.x - sn * tx, cs * x.y - sn * ty};
        v = float2{cs * v.x - sn * ux, cs * v.y - sn * uy};
      } else {
        const float tx = px * x.x - py * x.y, ty = px * x.y + py * x.x;
        const float ux = px * v.x - py * v.y, uy = px * v.y + py * v.x;
        x = float2{sn * y.x + cs * tx, sn * y.y + cs * ty};
        v = float2{sn * yv.x + cs * ux, sn * yv.y + cs * uy};
      }
    }
    // A half with no rotation in a whole sweep is done; else the Gram test.
    const unsigned b = __ballot_sync(FULL, any);
    rotated |= ((b >> (16 * h)) & 0xffffu) != 0u;
    const unsigned none = ((b & 0xffffu) == 0u ? 1u : 0u) | ((b >> 16) == 0u ? 2u : 0u);
    done |= none;
    if (done != 3u) done |= half_converged(x, row, col);
  }
  float nrm = x.x * x.x + x.y * x.y;
  nrm += __shfl_xor_sync(FULL, nrm, 1);
  nrm += __shfl_xor_sync(FULL, nrm, 2);
  float smax = nrm, smin = nrm;
  smax = fmaxf(smax, __shfl_xor_sync(FULL, smax, 4));
  smax = fmaxf(smax, __shfl_xor_sync(FULL, smax, 8));
  smin = fminf(smin, __shfl_xor_sync(FULL, smin, 4));
  smin = fminf(smin, __shfl_xor_sync(FULL, smin, 8));
  const bool good = smin > 1e-6f * smax;
  const unsigned gb = __ballot_sync(FULL, good);
  const unsigned okmask = ((gb & 0xffffu) == 0xffffu ? 1u : 0u) | ((gb >> 16) == 0xffffu ? 2u : 0u);
  const float inv = rsqrtf(good ? nrm : 1.f);
  const float2 w{x.x * inv, x.y * inv};
  // Q = W V^H, unitary to the Jacobi tolerance (~1e-6): the batched sweeps'
  // residual cost sees that deviation only quadratically, every update
  // starts afresh from its environment, and the finishing kernel makes the
  // answer unitary in FP64 before the FP64 cost check.
  *q_out = mm16_bh(w, v, row, col);
  // Renormalise a rotated V (one Newton-Schulz step) so no drift
  // accumulates over sweeps; an unrotated V is the stored one.
  if (__any_sync(FULL, rotated)) {
    const float2 gv = mm16_ah(v, v, row, col);
    const float2 tv{(row == col ? 1.5f : 0.f) - 0.5f * gv.x, -0.5f * gv.y};
    v = mm16(v, tv, row, col);
    __syncwarp();
    if (act && ((okmask >> h) & 1u) && rotated) v_io[l16] = v;
  }
  __syncwarp();
  return okmask;
}

// The unit's two gate updates at once (16 lanes per start): half h updates
// the gate of start h from its environment e (E[c][r] at lane 4c + r of the
// half).  A half whose fast path fails takes the FP64 Jacobi (warp-wide, one
// half after the other), as warp_update does.
__device__ void halfwarp_update(float2 e, float2* g, double2* sm, float2* v, bool act) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, r = l16 & 3, c = l16 >> 2, h = lane >> 4;
  const float2 a32{e.x, -e.y};  // A[r][c] = conj(E[c][r])
  float2 q;
  const unsigned act_mask = __ballot_sync(FULL, act);
  const unsigned acts = ((act_mask & 0xffffu) ? 1u : 0u) | ((act_mask >> 16) ? 2u : 0u);
  const unsigned ok = halfwarp_polar4_f32_warm(a32, v, act, &q);
  for (int hh = 0; hh < 2; ++hh) {
    if (!((acts >> hh) & 1u) || ((ok >> hh) & 1u)) continue;
    // The FP64 Jacobi of half hh's matrix on the whole warp: A in lanes 0..15.
    const float2 ah{__shfl_sync(FULL, a32.x, 16 * hh + l16), __shfl_sync(FULL, a32.y, 16 * hh + l16)};
    const double2 p = warp_polar4(double2{(double)ah.x, (double)ah.y}, double2{r == c ? 1.0 : 0.0, 0.0}, sm, nullptr);
    const float2 pf{(float)p.x, (float)p.y};
    const float2 pq{__shfl_sync(FULL, pf.x, l16), __shfl_sync(FULL, pf.y, l16)};
    if (h == hh) {
      q = pq;
      v[l16] = float2{r == c ? 1.f : 0.f, 0.f};  // restart from the identity
    }
  }
  if (act) g[4 * r + c] = q;
  __syncwarp();
}

// Per-start smem slice (complex64): B (E_max), Phi (E_max), gates (16 L_max),
// right singular vectors (16 L_max), environment (16).
__host__ __device__ __forceinline__ int batch_slice_f2(int max_elems, int max_L) {
  return 2 * max_elems + 32 * max_L + 16;
}

// One sweep (Section 3) of every active start of a unit: forward to B_{L-1}
// with the current gates, then k = L..1: environment from (B_{k-1}, Phi_k),
// update gate k, B_{k-2} = g_{k-1}^dagger B_{k-1} (old gate), Phi_{k-1} =
// g_k^dagger Phi_k (new gate).  Returns, in every lane of a group, the
// residual (1/M) sum |g_1^dagger Phi_1 - Psi|^2 of its start's swept gates,
// as an FP32 sum of squares (no cancellation; relative error ~1e-6, far
// below what the FP64 check at dist_tol needs).  `act` is this group's
// start being active; `act_mask` has bit j set when group j is active.
template <int G>
__device__ float group_sweep(float2* slice, int slice_f2, int E_max, int L_max, const float2* psi,
                             const float2* phil, const int* pairs, int n, int M, int L, double2* sm, bool act,
                             unsigned act_mask) {
  constexpr int NG = 32 / G;
  const int lane = threadIdx.x & 31;
  const int gi = lane / G, gl = lane % G;
  float2* Bs = slice + gi * slice_f2;
  float2* Ph = Bs + E_max;
  float2* Gt = Ph + E_max;
  float2* V = Gt + 16 * L_max;
  float* Env = reinterpret_cast<float*>(V + 16 * L_max);
  const int E = M << n;
  if (act) {
    for (int i = gl; i < E; i += G) {
      Bs[i] = psi[i];
      Ph[i] = phil[i];
    }
  }
  __syncwarp();
  for (int k = 1; k <= L - 1; ++k) {
    if (act) group_apply<G, float2>(Bs, Gt + 16 * (k - 1), n, M, pairs[2 * (k - 1)], pairs[2 * (k - 1) + 1], false, gl);
    __syncwarp();
  }
  for (int k = L; k >= 1; --k) {
    const int qa = pairs[2 * (k - 1)], qb = pairs[2 * (k - 1) + 1];
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    if (act) group_env_acc<G, float, float2>(Bs, Ph, n, M, qa, qb, gl, acc);
    if constexpr (G == 32) {
      const float v = warp_reduce_scatter32<float>(acc, lane);
      const int l16 = lane & 15;
      const float2 e{__shfl_sync(FULL, v, 2 * l16), __shfl_sync(FULL, v, 2 * l16 + 1)};
      if (act) warp_update<float2>(e, Gt + 16 * (k - 1), sm, V + 16 * (k - 1));
    } else if constexpr (G == 16) {
      // After the reduce-scatter lane gl holds two of its start's 32
      // environment floats; gather E[c][r] to lane 4c + r of each half
      // through shared memory, then both starts' updates run side by side.
      const int base = group_reduce_scatter<G, float>(acc, gl);
      Env[base] = acc[0];
      Env[base + 1] = acc[1];
      __syncwarp();
      const float2 e{Env[2 * gl], Env[2 * gl + 1]};
      halfwarp_update(e, Gt + 16 * (k - 1), sm, V + 16 * (k - 1), act);
    } else {
      const int base = group_reduce_scatter<G, float>(acc, gl);
#pragma unroll
      for (int i = 0; i < 32 / G; ++i) Env[base + i] = acc[i];
      __syncwarp();
      // The warp updates the unit's gates one start after another.
      const int l16 = lane & 15;
#pragma unroll 1
      for (int j = 0; j < NG; ++j) {
        if (!((act_mask >> j) & 1u)) continue;
        float2* sj = slice + j * slice_f2;
        const float* envj = reinterpret_cast<const float*>(sj + 2 * E_max + 32 * L_max);
        const float2 e{envj[2 * l16], envj[2 * l16 + 1]};
        warp_update<float2>(e, sj + 2 * E_max + 16 * (k - 1), sm, sj + 2 * E_max + 16 * L_max + 16 * (k - 1));
      }
    }
    __syncwarp();
    if (k > 1 && act) {
      group_apply<G, float2>(Bs, Gt + 16 * (k - 2), n, M, pairs[2 * (k - 2)], pairs[2 * (k - 2) + 1], true, gl);
      group_apply<G, float2>(Ph, Gt + 16 * (k - 1), n, M, qa, qb, true, gl);
    }
    __syncwarp();
  }
  float r = 0.f;
  if (act) group_apply<G, float2>(Ph, Gt, n, M, pairs[0], pairs[1], true, gl);
  __syncwarp();
  if (act) {
    for (int i = gl; i < E; i += G) {
      const float2 p = Ph[i], q = psi[i];
      const float dx = p.x - q.x, dy = p.y - q.y;
      r = fmaf(dx, dx, fmaf(dy, dy, r));
    }
  }
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1) r += __shfl_xor_sync(FULL, r, o);
  __syncwarp();
  return r * (1.f / (float)M);
}

// One FP64 sweep of one start by a whole warp (the refinement sweeps of the
// finishing kernel), as group_sweep with G = 32, B and Phi in Bs and Ph.
__device__ void warp_sweep64(double2* Bs, double2* Ph, double2* G, const double2* psi, const double2* phil,
                             const int* pairs, int n, int M, int L, double2* sm) {
  const int lane = threadIdx.x & 31;
  const int E = M << n;
  for (int i = lane; i < E; i += 32) {
    Bs[i] = psi[i];
    Ph[i] = phil[i];
  }
  __syncwarp();
  for (int k = 1; k <= L - 1; ++k) {
    group_apply<32, double2>(Bs, G + 16 * (k - 1), n, M, pairs[2 * (k - 1)], pairs[2 * (k - 1) + 1], false, lane);
    __syncwarp();
  }
  for (int k = L; k >= 1; --k) {
    const int qa = pairs[2 * (k - 1)], qb = pairs[2 * (k - 1) + 1];
    double acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.0;
    group_env_acc<32, double, double2>(Bs, Ph, n, M, qa, qb, lane, acc);
    const double v = warp_reduce_scatter32<double>(acc, lane);
    const int l16 = lane & 15;
    const double2 e{__shfl_sync(FULL, v, 2 * l16), __shfl_sync(FULL, v, 2 * l16 + 1)};
    warp_update<double2>(e, G + 16 * (k - 1), sm, nullptr);
    if (k > 1) {
      group_apply<32, double2>(Bs, G + 16 * (k - 2), n, M, pairs[2 * (k - 2)], pairs[2 * (k - 2) + 1], true, lane);
      group_apply<32, double2>(Ph, G + 16 * (k - 1), n, M, qa, qb, true, lane);
    }
    __syncwarp();
  }
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

// One unit (a problem and up to 32/G of its starts) swept by the warp to
// its end, in `region` (the warp's shared memory, laid out for this
// problem: a slice of batch_slice_f2(N M, L) float2 per start).
template <int G>
__device__ __forceinline__ void batch_run_unit(const BatchArgs& a, const BatchUnit& u, float2* region,
                                               double2* sm_polar) {
  constexpr int NG = 32 / G;
  const int lane = threadIdx.x & 31;
  const int gi = lane / G, gl = lane % G;
  const int p = u.p;
  const BatchProblem pr = a.probs[p];
  const int* pairs = a.pairs + pr.pair_off;
  const int E = pr.M << pr.n, L = pr.L;
  const int sf = batch_slice_f2(E, L);
  const int s = u.s0 + gi;
  bool act = gi < u.ns;
  float2* mine = region + gi * sf;
  float2* Gt = mine + 2 * E;
  float2* V = Gt + 16 * L;
  const size_t goff = pr.gate_off + (size_t)s * L * 16;
  if (act) {
    for (int i = gl; i < 16 * L; i += G) {
      const double2 g = a.init_gates[goff + i];
      Gt[i] = float2{(float)g.x, (float)g.y};
      const int e = i & 15;
      V[i] = float2{(e & 3) == (e >> 2) ? 1.f : 0.f, 0.f};
    }
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
    if (sw > *(volatile int*)(a.s_star + p)) act = false;
    const unsigned ballot = __ballot_sync(FULL, act && gl == 0);
    unsigned mask = 0;
#pragma unroll
    for (int j = 0; j < NG; ++j) mask |= ((ballot >> (j * G)) & 1u) << j;
    if (!mask) break;
    const float c = group_sweep<G>(region, sf, E, L, psi, phil, pairs, pr.n, pr.M, L, sm_polar, act, mask);
    if (act) {
      cost = c;
      sweeps = sw;
      if ((double)cost <= a.tol) {
        conv = sw;
        if (gl == 0) atomicMin(a.s_star + p, sw);
        act = false;
      } else if (a.plateau_window > 0 && prev >= 0.f) {
        // Plateau (App. A): no relative improvement > diff_tol_r for
        // plateau_window sweeps in a row stops this start.
        stall = fabsf(prev) - fabsf(cost) > dtr * fabsf(cost) ? 0 : stall + 1;
        if (stall >= a.plateau_window && sw >= a.min_sweeps) act = false;
      }
      prev = cost;
    }
  }
  if (gi < u.ns) {
    const size_t ri = (size_t)p * a.S + s;
    if (gl == 0) {
      a.conv_sweep[ri] = conv;
      a.final_cost[ri] = (double)cost;
      a.sweeps_run[ri] = sweeps;
    }
    for (int i = gl; i < 16 * L; i += G) a.gates32[goff + i] = Gt[i];
  }
  __syncwarp();
}

// Persistent sweep kernel with G lanes per start: warps take units until
// the queue is empty.  region_f2: each warp's shared memory in float2 (at
// least (32/G) batch_slice_f2(N M, L) for every unit it may take).
template <int G>
__global__ void k_batch_sweep(BatchArgs a, const BatchUnit* units, int nunits, int* queue, int region_f2) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double2 sm_polar[kBatchMaxWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* region = reinterpret_cast<float2*>(dsm) + (size_t)warp * region_f2;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(queue, 1);
    item = __shfl_sync(FULL, item, 0);
    if (item >= nunits) break;
    const unsigned long long t0 = a.unit_trace ? globaltimer_ns() : 0ull;
    batch_run_unit<G>(a, units[item], region, sm_polar[warp]);
    if (a.unit_trace && lane == 0) {
      const BatchUnit u = units[item];
      unsigned sm;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
      unsigned long long* r = a.unit_trace + 4 * (size_t)item;
      r[0] = t0;
      r[1] = globaltimer_ns();
      r[2] = (unsigned long long)u.p;
      r[3] = ((unsigned long long)sm << 32) | ((unsigned long long)u.s0 << 16) | ((unsigned)u.ns << 8) | G;
    }
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
    for (int k = 1; k <= pr.L; ++k) {
      group_apply<32, double2>(Bs, G + 16 * (k - 1), pr.n, pr.M, pairs[2 * (k - 1)], pairs[2 * (k - 1) + 1], false,
                               lane);
      __syncwarp();
    }
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
    warp_sweep64(Bs, Ph, G, psi, phil, pairs, pr.n, pr.M, pr.L, sm_polar);
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

int batch_region_f2(int G, int max_elems, int max_L) { return (32 / G) * batch_slice_f2(max_elems, max_L); }

size_t batch_sweep_smem(int G, int warps, int max_elems, int max_L) {
  return (size_t)warps * batch_region_f2(G, max_elems, max_L) * sizeof(float2);
}

namespace {
template <int G>
int blocks_per_sm_g(int warps, size_t smem) {
  cudaFuncSetAttribute(k_batch_sweep<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_sweep<G>, 32 * warps, smem) != cudaSuccess) {
    cudaGetLastError();
    b = 0;
  }
  return b;
}
}  // namespace

int batch_sweep_blocks_per_sm(int G, int warps, size_t smem) {
  switch (G) {
    case 4: return blocks_per_sm_g<4>(warps, smem);
    case 8: return blocks_per_sm_g<8>(warps, smem);
    case 16: return blocks_per_sm_g<16>(warps, smem);
    case 32: return blocks_per_sm_g<32>(warps, smem);
    default: return 0;
  }
}

void launch_batch_sweep(int G, const BatchArgs& a, const BatchUnit* units, int nunits, int* queue, int blocks,
                        int warps, int region_f2, cudaStream_t st) {
  const size_t smem = (size_t)warps * region_f2 * sizeof(float2);
  switch (G) {
    case 4: k_batch_sweep<4><<<blocks, 32 * warps, smem, st>>>(a, units, nunits, queue, region_f2); break;
    case 8: k_batch_sweep<8><<<blocks, 32 * warps, smem, st>>>(a, units, nunits, queue, region_f2); break;
    case 16: k_batch_sweep<16><<<blocks, 32 * warps, smem, st>>>(a, units, nunits, queue, region_f2); break;
    default: k_batch_sweep<32><<<blocks, 32 * warps, smem, st>>>(a, units, nunits, queue, region_f2); break;
  }
}

void launch_batch_finalize(const BatchArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(2 * a.max_elems + 16 * a.max_L) * sizeof(double2);
  cudaFuncSetAttribute(k_batch_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_batch_finalize<<<a.P, 32, smem, st>>>(a);
}

}  // namespace qfs
