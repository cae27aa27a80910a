// Device code of the gate update (Eq. 2 of the paper), shared by the update
// kernel and the fused backward kernel: the unitary polar factor u = Y X^dagger
// of E^dagger for E = X D Y^dagger, with the damping of the paper's Appendix A.
#pragma once
#include "qfs_common.cuh"
#include "qfs_kernels.h"

namespace qfs {

// 2^-e for the binary exponent e of a positive normal double (exact).
__device__ __forceinline__ double pow2_neg_exponent(double x) {
  const int ebits = (__double2hiint(x) >> 20) & 0x7ff;
  return __hiloint2double((2046 - ebits) << 20, 0);
}

// Rescale a 2-vector whose norm is 1 + O(1e-7) to norm 1 to rounding:
// 1/sqrt(1 + d) = 1 - d/2 + 3d^2/8 + O(d^3).
__device__ __forceinline__ double unit_fix(double n2) {
  const double d = n2 - 1.0;
  return fma(d, fma(d, 0.375, -0.5), 1.0);
}

// Returns, in lanes 0..15, P[r][c] of the polar factor of A, lane = 4c + r.
// `a` is A[r][c] in lanes 0..15; `v0` is a unitary V0[r][c] in lanes 16..31
// (a start for the right singular vectors, e.g. those of the previous sweep;
// the identity when nothing better is known).  On return lanes 16..31 hold
// the final V (written to *v_out).  `sm` is 32 double2 of shared memory
// private to this warp.
//
// One-sided Jacobi on X = A V0: rounds rotate the two disjoint column pairs
// (c, c^m), m = 1, 2, 3, until |gamma|^2 <= 1e-30 alpha beta for every pair,
// with gamma = x_p^H x_q, alpha = |x_p|^2, beta = |x_q|^2 in FP64.  FP64
// instructions are scarce on this GPU, so the rotation angle is computed in
// FP32 from the FP64 difference beta - alpha and |gamma| (scaled by an exact
// power of two), then renormalised in FP64 so that every rotation, and hence
// V, stays unitary to rounding; an FP32 angle reduces gamma by ~1e-7 per
// rotation, so the FP64 test is still met within a few rounds.  Extreme
// ratios that FP32 cannot represent take an FP64 angle built from rsqrt.
__device__ __forceinline__ double2 warp_polar4(double2 a, double2 v0, double2* sm, double2* v_out) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, r = l16 & 3, c = l16 >> 2;
  const bool isV = lane >= 16;
  // X[r][c] = sum_k A[r][k] V0[k][c]: A[r][k] sits in lane 4k + r,
  // V0[k][c] in lane 16 + 4c + k.
  double2 x;
  {
    double2 acc{0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 ak = shfl2(a, 4 * k + r);
      const double2 vk = shfl2(v0, 16 + 4 * c + k);
      acc = cfma(ak, vk, acc);
    }
    x = isV ? v0 : acc;
  }

  for (int sweep = 0; sweep < 24; ++sweep) {
    int rotated = 0;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const double2 y = shfl_xor2(x, 4 * m);  // same row, partner column c^m
      const bool isP = c < (c ^ m);
      double nown = x.x * x.x + x.y * x.y;
      double npar = y.x * y.x + y.y * y.y;
      double2 g = isP ? cmulc(x, y) : cmulc(y, x);  // conj(x_p) x_q
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
      const double alpha = isP ? nown : npar;  // ||x_p||^2
      const double beta = isP ? npar : nown;   // ||x_q||^2
      const double ag2 = g.x * g.x + g.y * g.y;
      double cs = 1.0, sn = 0.0;
      double2 ph{1.0, 0.0};  // e^{-i phi}, gamma = |gamma| e^{i phi}
      if (ag2 > 1e-30 * alpha * beta && ag2 > 1e-300) {
        const double sc = pow2_neg_exponent(fmax(alpha, beta));
        const float g2 = (float)(ag2 * sc * sc);
        if (g2 > 1e-30f) {
          // Symmetric Schur rotation (Golub & Van Loan, Alg. 8.4.1) in FP32.
          const float dif = (float)((beta - alpha) * sc);
          const float rg = rsqrtf(g2);
          const float zeta = 0.5f * dif * rg;
          const float t = fabsf(zeta) > 1e18f ? 0.5f / zeta
                                               : copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
          const float cf = rsqrtf(fmaf(t, t, 1.0f));
          cs = (double)cf;
          sn = (double)(t * cf);
          const double f = unit_fix(cs * cs + sn * sn);
          cs *= f;
          sn *= f;
          ph = double2{(double)((float)(g.x * sc) * rg), (double)(-(float)(g.y * sc) * rg)};
          const double fp = unit_fix(ph.x * ph.x + ph.y * ph.y);
          ph.x *= fp;
          ph.y *= fp;
        } else {
          // |gamma| below FP32 range relative to the columns: FP64 angle.
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
        }
        rotated = 1;
      }
      // [x_p', x_q'] = [x_p, x_q] [[cs, sn], [-sn e^{-i phi}, cs e^{-i phi}]]
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
  if (isV && v_out) v_out[l16] = x;

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

// ---------------------------------------------------------------------------
// Fast path: FP32 Jacobi SVD + FP64 polish.
//
// All 4x4 matrices below live in lanes 0..15 as M[row][col] at lane
// 4*col + row (lanes 16..31 hold a copy of the same layout).

template <typename T2>
__device__ __forceinline__ T2 shfl_c(T2 v, int src);
template <>
__device__ __forceinline__ float2 shfl_c<float2>(float2 v, int src) {
  return float2{__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src)};
}
template <>
__device__ __forceinline__ double2 shfl_c<double2>(double2 v, int src) {
  return shfl2(v, src);
}

// C = A B, C = A^H B, C = A B^H in the lane layout above.
template <typename T2>
__device__ __forceinline__ T2 mm(T2 a, T2 b, int row, int col) {
  T2 acc{0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) acc = cfma(shfl_c(a, 4 * k + row), shfl_c(b, 4 * col + k), acc);
  return acc;
}
template <typename T2>
__device__ __forceinline__ T2 mm_ah(T2 a, T2 b, int row, int col) {
  T2 acc{0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T2 ak = shfl_c(a, 4 * row + k), bk = shfl_c(b, 4 * col + k);  // conj(A[k][row]) B[k][col]
    acc = cfma(T2{ak.x, -ak.y}, bk, acc);
  }
  return acc;
}
template <typename T2>
__device__ __forceinline__ T2 mm_bh(T2 a, T2 b, int row, int col) {
  T2 acc{0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const T2 ak = shfl_c(a, 4 * k + row), bk = shfl_c(b, 4 * k + col);  // A[row][k] conj(B[col][k])
    acc = cfma(ak, T2{bk.x, -bk.y}, acc);
  }
  return acc;
}

// FP64 products: the shuffles involve the whole warp, the arithmetic only
// lanes 0..15 (the FP64 pipe is the scarce resource); lanes 16..31 get 0.
__device__ __forceinline__ double2 mm64(double2 a, double2 b, int row, int col, bool act) {
  double2 ak[4], bk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ak[k] = shfl2(a, 4 * k + row);
    bk[k] = shfl2(b, 4 * col + k);
  }
  double2 acc{0.0, 0.0};
  if (act) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc.x = fma(ak[k].x, bk[k].x, fma(-ak[k].y, bk[k].y, acc.x));
      acc.y = fma(ak[k].x, bk[k].y, fma(ak[k].y, bk[k].x, acc.y));
    }
  }
  return acc;
}
__device__ __forceinline__ double2 mm64_ah(double2 a, double2 b, int row, int col, bool act) {
  double2 ak[4], bk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ak[k] = shfl2(a, 4 * row + k);  // conj(A[k][row]) B[k][col]
    bk[k] = shfl2(b, 4 * col + k);
  }
  double2 acc{0.0, 0.0};
  if (act) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc.x = fma(ak[k].x, bk[k].x, fma(ak[k].y, bk[k].y, acc.x));
      acc.y = fma(ak[k].x, bk[k].y, fma(-ak[k].y, bk[k].x, acc.y));
    }
  }
  return acc;
}

// Skew-Hermitian correction Omega (FP32) from K = skew part of Q^H A:
// solve Omega H + H Omega = 2K in the basis V of H's eigenvectors.
__device__ __forceinline__ float2 skew_correction(float2 k32, float2 v, float sig, int row, int col) {
  const float2 kv = mm(mm_ah(v, k32, row, col), v, row, col);
  const float si = __shfl_sync(FULL, sig, 4 * row);  // sigma_row; sig is sigma_col
  const float den = 2.f / (si + sig);
  const float2 ot{kv.x * den, kv.y * den};
  float2 om = mm_bh(mm(v, ot, row, col), v, row, col);
  const float2 omt = shfl_c(om, 4 * row + col);  // Om[col][row]
  return float2{0.5f * (om.x - omt.x), 0.5f * (om.y + omt.y)};  // exactly skew-Hermitian
}

// FP32 Jacobi tolerance: a column pair counts as orthogonal when |gamma|^2
// <= kJac32Tol alpha beta, i.e. |gamma| <= 1e-6 sqrt(alpha beta).  The Gram
// entries of X = A V0 carry FP32 rounding of 2-5e-7 of sqrt(alpha beta), so a
// tighter test keeps rotating rounding noise.  Columns orthogonal to 1e-6
// leave the polar factor within ~1e-6 of the exact one; the polar factor
// maximises Re tr(g E) over unitary g, so that error changes the objective
// only at second order (1e-12).  The FP64 updates follow with Newton-Schulz
// steps that make the factor unitary to FP64 precision; the batched form
// keeps the FP32 factor and makes its answer unitary in FP64 at the end.
constexpr float kJac32Tol = 1e-12f;

// True when every column pair of X (lanes 0..15) has |gamma|^2 <= kJac32Tol
// alpha beta, from the Gram matrix X^H X in one product: cheaper than a
// sweep that finds nothing to rotate.
__device__ __forceinline__ bool jacobi32_converged(float2 x) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, row = l16 & 3, col = l16 >> 2;
  const float2 g = mm_ah(x, x, row, col);  // G[row][col] = <x_row, x_col>
  const float dr = __shfl_sync(FULL, g.x, 5 * row), dc = __shfl_sync(FULL, g.x, 5 * col);
  const bool ok = row == col || (g.x * g.x + g.y * g.y) <= kJac32Tol * dr * dc;
  return __all_sync(FULL, ok);
}

// FP32 one-sided Jacobi sweeps on X (lanes 0..15, X[r][c] at 4c + r) with
// the accumulated right rotations V in lanes 16..31, until every column pair
// has |gamma|^2 <= kJac32Tol alpha beta or 12 sweeps.
// *rotated_out (optional): whether any rotation was applied.
__device__ __forceinline__ float2 jacobi32_sweeps(float2 x, bool* rotated_out = nullptr) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, col = l16 >> 2;
  const int c = col;
  bool any = false;
  if (rotated_out) *rotated_out = false;
  if (jacobi32_converged(x)) return x;  // a warm start that is already orthogonal
  for (int sweep = 0; sweep < 12; ++sweep) {
    int rotated = 0;
#pragma unroll
    for (int m = 1; m <= 3; ++m) {
      const float2 y = shfl_c(x, lane ^ (4 * m));
      const bool isP = c < (c ^ m);
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
      nown = __shfl_sync(FULL, nown, l16);
      npar = __shfl_sync(FULL, npar, l16);
      g = shfl_c(g, l16);
      const float alpha = isP ? nown : npar, beta = isP ? npar : nown;
      const float ag2 = g.x * g.x + g.y * g.y;
      float cs = 1.f, sn = 0.f, px = 1.f, py = 0.f;
      if (ag2 > kJac32Tol * alpha * beta && ag2 > 1e-36f) {
        const float rg = rsqrtf(ag2);
        const float zeta = 0.5f * (beta - alpha) * rg;
        // t = sign(zeta) / (|zeta| + sqrt(zeta^2 + 1)) with the hardware
        // reciprocal and square root: the angle only has to shrink gamma,
        // the convergence test below decides, and V is renormalised.
        const float q = fmaf(zeta, zeta, 1.f);
        const float t = fabsf(zeta) > 1e18f ? __fdividef(0.5f, zeta)
                                             : copysignf(__fdividef(1.f, fabsf(zeta) + q * rsqrtf(q)), zeta);
        cs = rsqrtf(fmaf(t, t, 1.f));
        sn = t * cs;
        px = g.x * rg;
        py = -g.y * rg;
        rotated = 1;
      }
      if (isP) {
        const float tx = px * y.x - py * y.y, ty = px * y.y + py * y.x;
        x = float2{cs * x.x - sn * tx, cs * x.y - sn * ty};
      } else {
        const float tx = px * x.x - py * x.y, ty = px * x.y + py * x.x;
        x = float2{sn * y.x + cs * tx, sn * y.y + cs * ty};
      }
    }
    const bool r = __any_sync(FULL, rotated) != 0;
    any |= r;
    if (!r || jacobi32_converged(x)) break;
  }
  if (rotated_out) *rotated_out = any;
  return x;
}

// exp(Omega) to third order for a small skew-Hermitian Omega (lanes 0..15,
// FP32; big = max_ij |Re| + |Im| of its entries), as the FP64 entry of lane
// l16.  The first-order term enters exactly (FP32 -> FP64 is exact), so X
// keeps Omega's exact skew-Hermitian structure; the O(|Omega|^2) terms are
// summed in FP32 (relative error 6e-8).  Omega^2 is skipped below 1e-8 and
// Omega^3 below 2e-6 (their norms are then under 1e-15 and 1e-16).
__device__ __forceinline__ double2 exp_skew3(float2 om, float big, int row, int col) {
  float2 hot{0.f, 0.f};
  if (big >= 1e-8f) {
    const float2 om2 = mm(om, om, row, col);
    hot = float2{0.5f * om2.x, 0.5f * om2.y};
    if (big >= 2e-6f) {
      const float2 om3 = mm(om2, om, row, col);
      hot.x = fmaf(om3.x, 1.f / 6.f, hot.x);
      hot.y = fmaf(om3.y, 1.f / 6.f, hot.y);
    }
  }
  return double2{(row == col ? 1.0 : 0.0) + ((double)om.x + (double)hot.x), (double)om.y + (double)hot.y};
}

// max over lanes 0..15 of |Re| + |Im| (every lane gets it).
__device__ __forceinline__ float max_abs16(float2 v) {
  float big = fabsf(v.x) + fabsf(v.y);
  big = fmaxf(big, __shfl_xor_sync(FULL, big, 1));
  big = fmaxf(big, __shfl_xor_sync(FULL, big, 2));
  big = fmaxf(big, __shfl_xor_sync(FULL, big, 4));
  big = fmaxf(big, __shfl_xor_sync(FULL, big, 8));
  return big;
}

// POLISH = 2 (FP64 sweeps): two polish steps, accurate to FP64 rounding.
// POLISH = 1 (complex64 sweeps, whose environments are accurate to ~1e-7
// anyway): one polish step, ~1e-12.  Both are unitary to rounding.
//
// Polar factor of A (FP64, lanes 0..15, A[r][c] at 4c + r).  v0: a unitary
// start for the right singular vectors in lanes 16..31 (identity if none).
// Returns P in lanes 0..15 (P[r][c] at 4c + r), writes the right singular
// vectors to v_out (16 complex, V[r][c] at 4c + r) when non-null.
//
//  1. One-sided Jacobi in FP32 on X = A V0 (A scaled by an exact power of
//     two): A V = W Sigma, Q0 = W V^H, all to FP32 accuracy.
//  2. FP64: one Newton-Schulz step Q0 <- Q0 (3I - Q0^H Q0) / 2 makes Q0
//     unitary to ~1e-14.
//  3. FP64: B = Q0^H A = exp(Omega0) H exactly when A = Q H, so the polar
//     factor is Q0 exp(Omega0).  The skew part K = (B - B^H)/2 satisfies
//     Omega0 H + H Omega0 = 2K to first order; in the basis of V this is
//     Omega~_ij = 2 K~_ij / (sigma_i + sigma_j), solved in FP32 (Omega0 is
//     ~1e-7, so FP32 leaves ~1e-14 absolute error).
//  4. FP64: P = Q0 (I + Omega + Omega^2/2), unitary to ~1e-14.
// Returns false (and leaves P undefined) when A is too ill-conditioned for
// this path (sigma_min < 1e-3 sigma_max) or the correction is not small;
// the caller then takes the FP64 Jacobi.
template <int POLISH>
__device__ __forceinline__ bool warp_polar4_fast(double2 a, double2 v0, double2* p_out, double2* v_out) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, row = l16 & 3, col = l16 >> 2;
  const bool isV = lane >= 16;
  // Exact power-of-two scale from the largest exponent of A's entries.
  int e = 0;
  if (!isV) {
    const int ex = (__double2hiint(a.x) >> 20) & 0x7ff, ey = (__double2hiint(a.y) >> 20) & 0x7ff;
    e = max(ex, ey);
  }
  e = __reduce_max_sync(FULL, e);
  if (e == 0) return false;  // A == 0 (or denormal): leave it to the FP64 path
  const double sc = __hiloint2double((2046 - e) << 20, 0);
  const double2 as{a.x * sc, a.y * sc};
  const float2 a32{(float)as.x, (float)as.y};
  const float2 v032{(float)v0.x, (float)v0.y};
  // X = A V0 (A lanes), V0 (V lanes).
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
  // Every lane: W[row][col] and V[row][col] at index l16; sigma per column.
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
  if (!(smin > 1e-6f * smax)) return false;  // sigma_min < 1e-3 sigma_max
  const float inv = rsqrtf(nrm);
  const float sig = nrm * inv;                // sigma of column `col` (scaled)
  w = float2{w.x * inv, w.y * inv};
  // Q0 = W V^H (FP32, unitary to ~1e-6), promoted; two Newton-Schulz steps
  // in FP64 make it unitary to rounding.
  const bool act = !isV;
  const float2 q32 = mm_bh(w, v, row, col);
  double2 q{(double)q32.x, (double)q32.y};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double2 gq = mm64_ah(q, q, row, col, act);  // Q^H Q
    const double2 t{(row == col ? 1.5 : 0.0) - 0.5 * gq.x, -0.5 * gq.y};
    q = mm64(q, t, row, col, act);
  }
  // POLISH steps: B = Q^H A, K = (B - B^H)/2, Q <- Q exp(Omega).  The first
  // leaves O(|Omega0|^2) ~ 1e-12, the second FP64 rounding.
#pragma unroll
  for (int it = 0; it < POLISH; ++it) {
    const double2 bm = mm64_ah(q, as, row, col, act);
    const double2 bt = shfl2(bm, 4 * row + col);  // B[col][row]
    const float2 k32{0.5f * (float)(bm.x - bt.x), 0.5f * (float)(bm.y + bt.y)};
    const float2 om = skew_correction(k32, v, sig, row, col);
    const float big = max_abs16(om);
    if (it == 0 && !(big < 1e-3f)) return false;
    // exp(Omega) to third order (|Omega|^4 < 1e-12 after the first check).
    q = mm64(q, exp_skew3(om, big, row, col), row, col, act);
  }
  *p_out = q;
  if (v_out && lane < 16) v_out[l16] = double2{(double)v.x, (double)v.y};
  return true;
}

// Shared by the sweep update and the batched a4 entry point: lanes 0..15 hold
// the complex entry E[c][r] at lane 4c + r (the entry whose adjoint is A[r][c]).
// v_io: the gate's V from its previous update (16 complex, V[r][c] at
// 4c + r), read as the Jacobi start and overwritten with the new V; NULL
// starts from the identity.
template <int POLISH>
__device__ __forceinline__ void polar_update_warp(double2 e_cr, const double2* g_old, double beta,
                                  double2* sm, double2* g_out, float2* g32_out,
                                  double2* p_out, double2* v_io) {
  const int lane = threadIdx.x & 31;
  const int l16 = lane & 15, r = l16 & 3, c = l16 >> 2;
  double2 v0 = double2{r == c ? 1.0 : 0.0, 0.0};
  if (v_io && lane >= 16) v0 = v_io[l16];
  double2 m = e_cr;
  if (beta != 0.0 && lane < 16) {
    // (1 - beta) E[c][r] + beta conj(g_old[r][c])
    const double2 go = g_old[4 * r + c];
    m = double2{(1.0 - beta) * m.x + beta * go.x, (1.0 - beta) * m.y - beta * go.y};
  }
  const double2 a = double2{m.x, -m.y};  // A = M^dagger: A[r][c] = conj(M[c][r])
  double2 p;
  if (!warp_polar4_fast<POLISH>(a, v0, &p, v_io)) {
    // The stored V is unitary only to FP32 accuracy; the FP64 Jacobi needs
    // an exactly unitary start.
    p = warp_polar4(a, double2{r == c ? 1.0 : 0.0, 0.0}, sm, v_io);
  }
  if (lane < 16) {
    // p is P[r][c] with lane = 4c + r; store row-major [4r + c].
    g_out[4 * r + c] = p;
    if (g32_out) g32_out[4 * r + c] = float2{(float)p.x, (float)p.y};
  }
  *p_out = p;
}


// The update of gate k for start s once the environment is summed (one
// warp; lane j holds value j = 2(4x+y) + {re, im} of E[x][y]): form
// (1 - beta) E + beta g_old^dagger, replace the gate with the polar factor
// of its adjoint, and optionally write E, the cost 2 - (2/M) Re Tr(g E) and
// the new V.
template <int POLISH>
__device__ __forceinline__ void update_from_sum(const UpdateArgs& a, int s, double v, double2* sm) {
  const int lane = threadIdx.x & 31;
  // Lane 4c + r needs E[c][r], i.e. entry e = 4c + r = l16: real part at
  // 2*l16, imaginary at 2*l16 + 1.
  const int l16 = lane & 15;
  const double re = __shfl_sync(FULL, v, 2 * l16);
  const double im = __shfl_sync(FULL, v, 2 * l16 + 1);
  const double2 e{re, im};
  if (a.env_out && lane < 16) a.env_out[s * a.env_stride + l16] = e;  // row-major E[x][y] at 4x+y
  double2* g64 = a.g64 + s * a.g_stride;
  float2* g32 = a.g32 ? a.g32 + s * a.g_stride : nullptr;
  double2 p;
  polar_update_warp<POLISH>(e, g64, a.beta, sm, g64, g32, &p, a.vprev ? a.vprev + s * a.g_stride : nullptr);
  if (a.cost_out) {
    // Re Tr(g E) = sum_{r,c} Re(g[r][c] E[c][r]); lane 4c + r has both.
    double t = lane < 16 ? (p.x * e.x - p.y * e.y) : 0.0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) a.cost_out[s] = 2.0 - 2.0 * a.inv_M * t;
  }
}

// The update of gate k for start s from the backward step's block partials
// (one warp): the partials are summed in a fixed order, then as above.
// PT is the partials' type (float after complex64 steps, double after FP64).
template <typename PT, int POLISH, bool COHERENT>
__device__ __forceinline__ void update_one_start(const UpdateArgs& a, int s, double2* sm) {
  const int lane = threadIdx.x & 31;
  const PT* pp = reinterpret_cast<const PT*>(a.partials) + (long long)s * a.nblk * 32;
  PT acc = PT(0);
  for (int b = 0; b < a.nblk; ++b) acc += COHERENT ? __ldcg(pp + b * 32 + lane) : pp[b * 32 + lane];
  update_from_sum<POLISH>(a, s, (double)acc, sm);
}

}  // namespace qfs
