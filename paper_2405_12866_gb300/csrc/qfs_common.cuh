// Device helpers shared by the QFactor-Sample kernels (sm_103a).
//
// Layout conventions (the C-ABI header states them for callers):
//   * a state is N x M complex, row-major, sample index fastest;
//   * qubit q is bit (n-1-q) of the row index;
//   * a gate on (a, b) is a row-major 4x4 complex matrix indexed by the local
//     index 2*bit_a + bit_b.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qfs {

constexpr unsigned FULL = 0xffffffffu;

template <typename T> struct C2;
template <> struct C2<float>  { using t = float2;  };
template <> struct C2<double> { using t = double2; };

// The device's global timer (ns), for the trace stamps.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// acc + a * b as four FMAs (two per component, no rounded product in between).
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
template <typename T2> __device__ __forceinline__ T2 cfma(T2 a, T2 b, T2 acc) {
  acc.x = fmat(a.x, b.x, acc.x);
  acc.x = fmat(-a.y, b.y, acc.x);
  acc.y = fmat(a.x, b.y, acc.y);
  acc.y = fmat(a.y, b.x, acc.y);
  return acc;
}
// acc (re, im) + b * conj(p) as four FMAs.
template <typename T, typename T2> __device__ __forceinline__ void cfma_conj(T& re, T& im, T2 b, T2 p) {
  re = fmat(b.x, p.x, re);
  re = fmat(b.y, p.y, re);
  im = fmat(b.y, p.x, im);
  im = fmat(-b.x, p.y, im);
}
// conj(a) * b
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
  return T2{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

__device__ __forceinline__ double2 shfl_xor2(double2 v, int m) {
  return double2{__shfl_xor_sync(FULL, v.x, m), __shfl_xor_sync(FULL, v.y, m)};
}
__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return double2{__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src)};
}

// Insert zero bits at positions lo < hi into r (r counts the N/4 groups).
__device__ __forceinline__ uint32_t insert_two_zero_bits(uint32_t r, int lo, int hi) {
  r = ((r >> lo) << (lo + 1)) | (r & ((1u << lo) - 1u));
  r = ((r >> hi) << (hi + 1)) | (r & ((1u << hi) - 1u));
  return r;
}

// Warp reduce-scatter of 32 per-lane values: on return lane l holds the sum
// over the warp of value l.  31 shuffles instead of 32 x 5.
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter32(T (&v)[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      T send = upper ? v[i] : v[i + w];
      T keep = upper ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, w);
    }
  }
  return v[0];
}

}  // namespace qfs
