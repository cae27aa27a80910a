// The gate update of QFactor-Sample (Eq. 2 of the paper): given the 4x4
// environment E = X D Y^dagger, the new gate is u = Y X^dagger, the unitary
// polar factor of E^dagger.  With the damping of the paper's Appendix A the
// SVD is taken of (1 - beta) E + beta u_old^dagger instead.
//
// One warp per gate, in FP64: a one-sided (Hestenes) Jacobi SVD of
// A = E^dagger.  Lanes 0..15 hold A[r][c] (lane = 4c + r), lanes 16..31 the
// accumulated right rotations V[r][c].  Each round rotates the two disjoint
// column pairs (c, c^m), m = 1, 2, 3, so a sweep is three rounds.  When the
// columns are orthogonal, A V = W Sigma and the polar factor is W V^dagger.
#include "qfs_common.cuh"
#include "qfs_kernels.h"

namespace qfs {

// Returns, in lanes 0..15, P[r][c] of the polar factor of A, lane = 4c + r.
// `a` is A[r][c] in lanes 0..15 (ignored in 16..31).  `sm` is 32 double2 of
// shared memory private to this warp.
//
// FP64 instructions are scarce on this GPU (a warp-wide FP64 instruction
// occupies the SM's FP64 pipe for many cycles), so the rotation uses no FP64
// division or square root, only rsqrt, and the convergence test
// |gamma|^2 <= 1e-30 alpha beta needs no square root.
__device__ double2 warp_polar4(double2 a, double2* sm) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, r = l16 & 3, c = l16 >> 2;
  const bool isV = lane >= 16;
  double2 x = isV ? double2{r == c ? 1.0 : 0.0, 0.0} : a;

  for (int sweep = 0; sweep < 20; ++sweep) {
    int rotated = 0;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const double2 y = shfl_xor2(x, 4 * m);  // same row, partner column c^m
      const bool isP = c < (c ^ m);
      double nown = x.x * x.x + x.y * x.y;
      double npar = y.x * y.x + y.y * y.y;
      double2 g = isP ? cmulc(x, y) : cmulc(y, x);  // conj(a_p) a_q
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        nown += __shfl_xor_sync(FULL, nown, o);
        npar += __shfl_xor_sync(FULL, npar, o);
        g.x += __shfl_xor_sync(FULL, g.x, o);
        g.y += __shfl_xor_sync(FULL, g.y, o);
      }
      // The A half decides; the V half applies the same rotation.
      nown = __shfl_sync(FULL, nown, l16);
      npar = __shfl_sync(FULL, npar, l16);
      g = shfl2(g, l16);
      const double alpha = isP ? nown : npar;  // ||a_p||^2
      const double beta = isP ? npar : nown;   // ||a_q||^2
      const double ag2 = g.x * g.x + g.y * g.y;
      double cs = 1.0, sn = 0.0;
      double2 ph{1.0, 0.0};  // e^{-i phi}, gamma = |gamma| e^{i phi}
      if (ag2 > 1e-30 * alpha * beta && ag2 > 1e-300) {
        // Symmetric Schur rotation (Golub & Van Loan, Alg. 8.4.1) built from
        // reciprocal square roots only: 1/|gamma|, sqrt(q) = q rsqrt(q),
        // 1/D = rsqrt(D)^2.  c^2 + s^2 and |e^{-i phi}| are 1 to rounding.
        const double ri = rsqrt(ag2);
        const double zeta = 0.5 * (beta - alpha) * ri;
        double t;
        if (fabs(zeta) > 1e150) {
          t = 0.5 / zeta;
        } else {
          const double q = fma(zeta, zeta, 1.0);
          const double D = fabs(zeta) + q * rsqrt(q);
          const double rD = rsqrt(D);
          t = copysign(rD * rD, zeta);
        }
        cs = rsqrt(fma(t, t, 1.0));
        sn = t * cs;
        ph = double2{g.x * ri, -g.y * ri};
        rotated = 1;
      }
      // [a_p', a_q'] = [a_p, a_q] [[cs, sn], [-sn e^{-i phi}, cs e^{-i phi}]]
      if (isP) {
        const double2 t2 = cmul(ph, y);
        x = double2{cs * x.x - sn * t2.x, cs * x.y - sn * t2.y};
      } else {
        const double2 t2 = cmul(ph, x);
        x = double2{sn * y.x + cs * t2.x, sn * y.y + cs * t2.y};
      }
    }
    if (!__any_sync(FULL, rotated)) break;
  }

  // Column norms sigma_c^2 (A half), normalise W = A Sigma^{-1}.
  double nrm = x.x * x.x + x.y * x.y;
  nrm += __shfl_xor_sync(FULL, nrm, 1);
  nrm += __shfl_xor_sync(FULL, nrm, 2);
  double nmax = nrm;
  nmax = fmax(nmax, __shfl_xor_sync(FULL, nmax, 4));
  nmax = fmax(nmax, __shfl_xor_sync(FULL, nmax, 8));
  const bool null_col = !isV && !(nrm > 1e-28 * nmax && nrm > 1e-300);
  if (!isV) {
    const double inv = null_col ? 0.0 : rsqrt(nrm);
    x = double2{x.x * inv, x.y * inv};
  }
  sm[lane] = x;  // W at [4c + r], V at [16 + 4c + r]
  const unsigned any_null = __ballot_sync(FULL, null_col);
  __syncwarp();
  if (any_null && lane == 0) {
    // Rank-deficient environment: any completion of W to a unitary is an
    // optimal update.  Gram-Schmidt of unit vectors against the kept columns.
    for (int cc = 0; cc < 4; ++cc) {
      if (!((any_null >> (4 * cc)) & 1u)) continue;
      for (int e = 0; e < 4; ++e) {
        double2 v[4];
        for (int rr = 0; rr < 4; ++rr) v[rr] = double2{rr == e ? 1.0 : 0.0, 0.0};
        for (int k = 0; k < 4; ++k) {
          if (k == cc) continue;
          const bool kept = !((any_null >> (4 * k)) & 1u) || k < cc;
          if (!kept) continue;
          double2 d{0.0, 0.0};
          for (int rr = 0; rr < 4; ++rr) {
            const double2 t = cmulc(sm[4 * k + rr], v[rr]);
            d.x += t.x;
            d.y += t.y;
          }
          for (int rr = 0; rr < 4; ++rr) {
            const double2 t = cmul(sm[4 * k + rr], d);
            v[rr].x -= t.x;
            v[rr].y -= t.y;
          }
        }
        double nn = 0.0;
        for (int rr = 0; rr < 4; ++rr) nn += v[rr].x * v[rr].x + v[rr].y * v[rr].y;
        if (nn > 0.2) {
          const double inv = 1.0 / sqrt(nn);
          for (int rr = 0; rr < 4; ++rr) sm[4 * cc + rr] = double2{v[rr].x * inv, v[rr].y * inv};
          break;
        }
      }
    }
  }
  __syncwarp();
  // P[r][c'] = sum_c W[r][c] conj(V[c'][c]); lane 4c' + r.
  double2 p{0.0, 0.0};
  if (!isV) {
    const int cp = c;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 w = sm[4 * k + r];
      const double2 v = sm[16 + 4 * k + cp];
      p.x += w.x * v.x + w.y * v.y;
      p.y += w.y * v.x - w.x * v.y;
    }
  }
  __syncwarp();
  return p;
}

// Shared by the sweep update and the batched a4 entry point: lanes 0..15 hold
// the complex entry E[c][r] at lane 4c + r (the entry whose adjoint is A[r][c]).
__device__ void polar_update_warp(double2 e_cr, const double2* g_old, double beta,
                                  double2* sm, double2* g_out, float2* g32_out,
                                  double2* p_out) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, r = l16 & 3, c = l16 >> 2;
  double2 m = e_cr;
  if (beta != 0.0 && lane < 16) {
    // (1 - beta) E[c][r] + beta conj(g_old[r][c])
    const double2 go = g_old[4 * r + c];
    m = double2{(1.0 - beta) * m.x + beta * go.x, (1.0 - beta) * m.y - beta * go.y};
  }
  const double2 a = double2{m.x, -m.y};  // A = M^dagger: A[r][c] = conj(M[c][r])
  const double2 p = warp_polar4(a, sm);
  if (lane < 16) {
    // p is P[r][c] with lane = 4c + r; store row-major [4r + c].
    g_out[4 * r + c] = p;
    if (g32_out) g32_out[4 * r + c] = float2{(float)p.x, (float)p.y};
  }
  *p_out = p;
}

// One warp per block: the FP64 pipe of each SM serves one gate at a time.
__global__ void k_update(UpdateArgs a) {
  __shared__ double2 sm_all[1][32];
  const int warp = 0, lane = threadIdx.x & 31;
  const int s = blockIdx.x;
  if (s >= a.S) return;
  if (a.active && !a.active[s]) return;
  double2* sm = sm_all[warp];
  // Lane j sums value j over blocks in a fixed order (deterministic).
  const double* pp = a.partials + (long long)s * a.nblk * 32;
  double v = 0.0;
  for (int b = 0; b < a.nblk; ++b) v += pp[b * 32 + lane];
  // value j = 2*(4x+y) + {re, im} of E[x][y]; lane 4c + r needs E[c][r],
  // i.e. entry e = 4c + r = l16: real part at 2*l16, imaginary at 2*l16 + 1.
  const int l16 = lane & 15;
  const double re = __shfl_sync(FULL, v, 2 * l16);
  const double im = __shfl_sync(FULL, v, 2 * l16 + 1);
  const double2 e{re, im};
  if (a.env_out && lane < 16) a.env_out[s * a.env_stride + l16] = e;  // row-major E[x][y] at 4x+y
  double2* g64 = a.g64 + s * a.g_stride;
  float2* g32 = a.g32 ? a.g32 + s * a.g_stride : nullptr;
  double2 p;
  polar_update_warp(e, g64, a.beta, sm, g64, g32, &p);
  if (a.cost_out) {
    // Re Tr(g E) = sum_{r,c} Re(g[r][c] E[c][r]); lane 4c + r has both.
    double t = lane < 16 ? (p.x * e.x - p.y * e.y) : 0.0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) a.cost_out[s] = 2.0 - 2.0 * a.inv_M * t;
  }
}

void launch_update(const UpdateArgs& a, cudaStream_t st) {
  k_update<<<a.S, 32, 0, st>>>(a);
}

__global__ void k_residual_finish(const double* partials, int nblk, int S, double inv_M,
                                  double* cost_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += partials[((long long)s * nblk + b) * 32];
  cost_out[s] = t * inv_M;
}

void launch_residual_finish(const double* partials, int nblk, int S, double inv_M,
                            double* cost_out, cudaStream_t st) {
  k_residual_finish<<<(S + 127) / 128, 128, 0, st>>>(partials, nblk, S, inv_M, cost_out);
}

__global__ void k_gate_update_batch(int count, const double2* envs, const double2* g_old,
                                    double beta, double2* g_out) {
  __shared__ double2 sm_all[4][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 4 + warp;
  if (i >= count) return;
  const int l16 = lane & 15;
  // envs row-major E[x][y] at 4x + y; lane 4c + r needs E[c][r] = entry l16.
  const double2 e = envs[(long long)i * 16 + l16];
  double2 p;
  polar_update_warp(e, g_old ? g_old + (long long)i * 16 : nullptr, g_old ? beta : 0.0,
                    sm_all[warp], g_out + (long long)i * 16, nullptr, &p);
}

void launch_gate_update_batch(int count, const double2* envs, const double2* g_old, double beta,
                              double2* g_out, cudaStream_t st) {
  if (count <= 0) return;
  k_gate_update_batch<<<(count + 3) / 4, 128, 0, st>>>(count, envs, g_old, beta, g_out);
}

}  // namespace qfs
