// Elementwise and reduction kernels of the learned warm start (the network
// proposes initial gates; the sweep judges them).  The matrix products run
// on the tensor cores (mlp_gemm.cu); these kernels build the features, cast
// and transpose operands, form the loss gradient, back-propagate GELU, sum
// bias gradients and apply Adam.
#include <cuda_bf16.h>

#include "qfs_common.cuh"
#include "qfs_kernels.h"

#include <algorithm>

namespace qfs {

namespace {
// Derivative of the tanh form of GELU, 0.5 x (1 + tanh u) with u =
// k0 (x + k1 x^3): with s = 1 / (1 + exp(-2u)) = (1 + tanh u) / 2 it is
// s + 2 x s (1 - s) k0 (1 + 3 k1 x^2) (1 - tanh^2 u = 4 s (1 - s), free of
// the cancellation of 1 - t^2); ~1e-6 relative.  exp(-2u) = inf gives s = 0.
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * fmaf(k1 * x, x * x, x);
  const float s = __fdividef(1.f, 1.f + __expf(-2.f * u));
  return fmaf(2.f * x * s * (1.f - s), k0 * fmaf(3.f * k1, x * x, 1.f), s);
}
}  // namespace

// Features of target t: the 16 x 8 complex matrix U_t Phi_fix as 256 reals
// (row-major, re/im interleaved), bf16, row t of X (ld = 256).  Rows
// count..rows-1 are zero.
__global__ void k_ws_features(const double2* __restrict__ U, const double2* __restrict__ phif, int count,
                              int rows, __nv_bfloat16* __restrict__ X) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // one complex output
  if (e >= (long long)rows * 128) return;
  const int t = (int)(e / 128), k = (int)(e % 128), i = k / 8, j = k % 8;
  float re = 0.f, im = 0.f;
  if (t < count) {
    const double2* u = U + (size_t)t * 256 + i * 16;
    for (int q = 0; q < 16; ++q) {
      const double2 a = u[q], b = phif[q * 8 + j];
      re += (float)(a.x * b.x - a.y * b.y);
      im += (float)(a.x * b.y + a.y * b.x);
    }
  }
  // Scaled by sqrt(16) = 4 so that the features have unit variance per
  // complex entry (the columns of U Phi_fix are unit vectors of length 16).
  X[(size_t)t * 256 + 2 * k] = __float2bfloat16(4.f * re);
  X[(size_t)t * 256 + 2 * k + 1] = __float2bfloat16(4.f * im);
}

// dst[c][r] = src[r][c] (bf16), 32 x 32 tiles; R, C multiples of 32.
// dst (C x R) = src (R x C)^T, both bf16 row-major, R and C multiples of 64:
// 64 x 64 tiles, two elements per access (128-byte rows per warp on both
// sides); the shared tile's rows are padded by one word.
__global__ void k_transpose_bf16_64(const __nv_bfloat16* __restrict__ src, int R, int C,
                                    __nv_bfloat16* __restrict__ dst) {
  __shared__ __nv_bfloat16 tile[64][66];
  const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int y = ty; y < 64; y += 8) {
    const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(src + (size_t)(r0 + y) * C + c0 + 2 * tx);
    tile[y][2 * tx] = v.x;
    tile[y][2 * tx + 1] = v.y;
  }
  __syncthreads();
  for (int y = ty; y < 64; y += 8) {
    __nv_bfloat162 v;
    v.x = tile[2 * tx][y];
    v.y = tile[2 * tx + 1][y];
    *reinterpret_cast<__nv_bfloat162*>(dst + (size_t)(c0 + y) * R + r0 + 2 * tx) = v;
  }
}

__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ src, int R, int C,
                                 __nv_bfloat16* __restrict__ dst) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) tile[y][threadIdx.x] = src[(size_t)(r0 + y) * C + c0 + threadIdx.x];
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) dst[(size_t)(c0 + y) * R + r0 + threadIdx.x] = tile[threadIdx.x][y];
}

__global__ void k_cast_f32_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// Output gradient of the mean squared error over the first n_out columns of
// the first B_valid rows: dY = 2 (Y - T) / (B_valid n_out) (fp32 and bf16),
// zero elsewhere; loss partial sums per block into loss_part[blockIdx.x].
__global__ void k_ws_loss_grad(const float* __restrict__ Y, int ldy, const float* __restrict__ T, int n_out,
                               int rows, int B_valid, float* __restrict__ dY32, __nv_bfloat16* __restrict__ dY16,
                               double* __restrict__ loss_part) {
  __shared__ double red[256];
  double acc = 0.0;
  const double scale = 2.0 / ((double)B_valid * n_out);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * ldy; e += gridDim.x * blockDim.x) {
    const int r = e / ldy, c = e - r * ldy;
    float g = 0.f;
    if (r < B_valid && c < n_out) {
      const double d = (double)Y[e] - (double)T[(size_t)r * n_out + c];
      acc += d * d;
      g = (float)(scale * d);
    }
    dY32[e] = g;
    dY16[e] = __float2bfloat16(g);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// dZ = dH * gelu'(Z) (fp32 and bf16), rows >= B_valid zeroed.
// Four elements per thread (n and ld multiples of 4); row-major, so the
// first B_valid rows are exactly the elements below B_valid * ld.  dZ32 may
// be dH (in place: each thread reads its four elements before writing them).
__global__ void k_gelu_back(const float* dH, const float* __restrict__ Z, long long n, int ld, int B_valid,
                            float* dZ32, __nv_bfloat16* __restrict__ dZ16) {
  const long long nvalid = (long long)B_valid * ld;
  for (long long i = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x); i < n;
       i += 4LL * gridDim.x * blockDim.x) {
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < nvalid) {
      const float4 h = *reinterpret_cast<const float4*>(dH + i), z = *reinterpret_cast<const float4*>(Z + i);
      g = make_float4(h.x * gelu_grad_f(z.x), h.y * gelu_grad_f(z.y), h.z * gelu_grad_f(z.z), h.w * gelu_grad_f(z.w));
    }
    *reinterpret_cast<float4*>(dZ32 + i) = g;
    const __nv_bfloat162 a = __floats2bfloat162_rn(g.x, g.y), b = __floats2bfloat162_rn(g.z, g.w);
    *reinterpret_cast<uint2*>(dZ16 + i) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
  }
}

// db[c] += sum over rows of G[r][c]: block (32 columns x 8 row lanes) over a
// slice of the rows, reduced in shared memory, one atomic per column and
// block (db is zeroed by the launcher).
__global__ void k_colsum(const float* __restrict__ G, int rows, int cols, float* __restrict__ db) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (c < cols)
    for (int r = blockIdx.y * 8 + threadIdx.y; r < rows; r += 8 * gridDim.y) s += G[(size_t)r * cols + c];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    float t = 0.f;
#pragma unroll
    for (int y = 0; y < 8; ++y) t += red[y][threadIdx.x];
    atomicAdd(db + c, t);
  }
}

// acc += (sum of parts[0..n)) * scale (one block).
__global__ void k_loss_accumulate(const double* __restrict__ parts, int n, double scale, double* __restrict__ acc) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += parts[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += red[0] * scale;
}

// Adam (Kingma & Ba 2015) on fp32 master parameters with a bf16 copy.
// With `sched` (device, 3 floats per step: lr, bc1, bc2) the step's values
// are read at index *sched_step, so that one captured graph serves every
// step; otherwise the arguments are used.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, __nv_bfloat16* __restrict__ w16, const float* __restrict__ sched,
                       const int* __restrict__ sched_step) {
  if (sched) {
    const int s = *sched_step;
    lr = sched[3 * s];
    bc1 = sched[3 * s + 1];
    bc2 = sched[3 * s + 2];
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16(wi);
  }
}

// Network outputs -> 6 gates per row (G[r][c] from outputs 2(16g + 4r + c),
// +1) -> E = G^dagger, so that the polar update (which returns the polar
// factor of E^dagger) projects G onto U(4).
__global__ void k_ws_gates_adjoint(const float* __restrict__ Y, int ldy, int count, double2* __restrict__ E) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)count * 96) return;
  const int t = (int)(e / 96), q = (int)(e % 96), g = q / 16, x = (q % 16) / 4, y = q % 4;
  const float* row = Y + (size_t)t * ldy + 32 * g;
  // E[x][y] = conj(G[y][x])
  E[e] = double2{(double)row[2 * (4 * y + x)], -(double)row[2 * (4 * y + x) + 1]};
}

// Mini-batch gather: rows idx[0..bv) of the device training set into the
// batch buffers; rows bv..B-1 of X are zeroed.
// Rows idx[0 .. bv) of the training set, after advancing idx by
// *jstep * batch when jstep is given (the step within the epoch, read on the
// device so that one captured graph serves every step).
__global__ void k_ws_gather(const __nv_bfloat16* __restrict__ Xall, const float* __restrict__ Tall,
                            const int* __restrict__ idx, int bv, int B, __nv_bfloat16* __restrict__ X,
                            float* __restrict__ T, const int* __restrict__ jstep, int batch) {
  if (jstep) idx += (long long)*jstep * batch;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < (long long)B * 256) {
    const int r = (int)(e / 256), c = (int)(e % 256);
    X[e] = r < bv ? Xall[(size_t)idx[r] * 256 + c] : __float2bfloat16(0.f);
  }
  if (e < (long long)bv * 192) {
    const int r = (int)(e / 192), c = (int)(e % 192);
    T[e] = Tall[(size_t)idx[r] * 192 + c];
  }
}

// The end of a training step: the step within the epoch and the step of
// the call advance.
__global__ void k_ws_step_advance(int* jstep, int* gstep) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *jstep += 1;
    *gstep += 1;
  }
}

static int blocks_for(long long n, int threads = 256, int cap = 4096) {
  long long b = (n + threads - 1) / threads;
  return (int)(b > cap ? cap : (b < 1 ? 1 : b));
}

void launch_ws_features(const double2* U, const double2* phif, int count, int rows, __nv_bfloat16* X,
                        cudaStream_t st) {
  const long long n = (long long)rows * 128;
  k_ws_features<<<(int)((n + 255) / 256), 256, 0, st>>>(U, phif, count, rows, X);
}
void launch_ws_gates_adjoint(const float* Y, int ldy, int count, double2* E, cudaStream_t st) {
  const long long n = (long long)count * 96;
  k_ws_gates_adjoint<<<(int)((n + 255) / 256), 256, 0, st>>>(Y, ldy, count, E);
}
void launch_ws_gather(const __nv_bfloat16* Xall, const float* Tall, const int* idx, int bv, int B,
                      __nv_bfloat16* X, float* T, cudaStream_t st, const int* jstep, int batch) {
  const long long n = (long long)B * 256;
  k_ws_gather<<<(int)((n + 255) / 256), 256, 0, st>>>(Xall, Tall, idx, bv, B, X, T, jstep, batch);
}
void launch_ws_step_advance(int* jstep, int* gstep, cudaStream_t st) { k_ws_step_advance<<<1, 32, 0, st>>>(jstep, gstep); }
void launch_transpose_bf16(const __nv_bfloat16* src, int R, int C, __nv_bfloat16* dst, cudaStream_t st) {
  if (R % 64 == 0 && C % 64 == 0)
    k_transpose_bf16_64<<<dim3(C / 64, R / 64), dim3(32, 8), 0, st>>>(src, R, C, dst);
  else
    k_transpose_bf16<<<dim3(C / 32, R / 32), dim3(32, 8), 0, st>>>(src, R, C, dst);
}
void launch_cast_f32_bf16(const float* a, __nv_bfloat16* b, long long n, cudaStream_t st) {
  k_cast_f32_bf16<<<blocks_for(n), 256, 0, st>>>(a, b, n);
}
int launch_ws_loss_grad(const float* Y, int ldy, const float* T, int n_out, int rows, int B_valid, float* dY32,
                        __nv_bfloat16* dY16, double* loss_part, cudaStream_t st) {
  const int blocks = blocks_for((long long)rows * ldy, 256, 1024);
  k_ws_loss_grad<<<blocks, 256, 0, st>>>(Y, ldy, T, n_out, rows, B_valid, dY32, dY16, loss_part);
  return blocks;
}
void launch_gelu_back(const float* dH, const float* Z, long long n, int ld, int B_valid, float* dZ32,
                      __nv_bfloat16* dZ16, cudaStream_t st) {
  k_gelu_back<<<blocks_for(n / 4), 256, 0, st>>>(dH, Z, n, ld, B_valid, dZ32, dZ16);
}
void launch_colsum(const float* G, int rows, int cols, float* db, cudaStream_t st) {
  cudaMemsetAsync(db, 0, sizeof(float) * (size_t)cols, st);
  const int ychunks = std::max(1, std::min(64, rows / 64));
  k_colsum<<<dim3((cols + 31) / 32, ychunks), dim3(32, 8), 0, st>>>(G, rows, cols, db);
}
void launch_loss_accumulate(const double* parts, int n, double scale, double* acc, cudaStream_t st) {
  k_loss_accumulate<<<1, 256, 0, st>>>(parts, n, scale, acc);
}
void launch_adam(float* w, float* m, float* v, const float* g, long long n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, __nv_bfloat16* w16, cudaStream_t st, const float* sched,
                 const int* sched_step) {
  k_adam<<<blocks_for(n), 256, 0, st>>>(w, m, v, g, n, lr, b1, b2, eps, bc1, bc2, w16, sched, sched_step);
}

}  // namespace qfs
