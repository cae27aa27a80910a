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
#include "polar4.cuh"

namespace qfs {

// One warp per block: the FP64 pipe of each SM serves one gate at a time.
__global__ void k_update(UpdateArgs a) {
  __shared__ double2 sm[32];
  const int s = blockIdx.x;
  if (s >= a.S) return;
  if (a.active && !a.active[s]) return;
  if (a.partials_f32) update_one_start<float, 1, false>(a, s, sm);
  else update_one_start<double, 2, false>(a, s, sm);
}

__global__ void k_set_identity4(double2* v, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count * 16;
       i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i & 15);
    v[i] = double2{(e & 3) == (e >> 2) ? 1.0 : 0.0, 0.0};
  }
}

void launch_set_identity4(double2* v, long long count, cudaStream_t st) {
  if (count <= 0) return;
  long long blocks = (count * 16 + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_set_identity4<<<(int)blocks, 256, 0, st>>>(v, count);
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
  polar_update_warp<2>(e, g_old ? g_old + (long long)i * 16 : nullptr, g_old ? beta : 0.0,
                       sm_all[warp], g_out + (long long)i * 16, nullptr, &p, nullptr);
}

void launch_gate_update_batch(int count, const double2* envs, const double2* g_old, double beta,
                              double2* g_out, cudaStream_t st) {
  if (count <= 0) return;
  k_gate_update_batch<<<(count + 3) / 4, 128, 0, st>>>(count, envs, g_old, beta, g_out);
}

}  // namespace qfs
