// FMA throughput of the FP64 and FP32 pipes: independent FMA chains in
// registers, one store per thread at the end (out has grid*block elements).
// Prints TFLOP/s (2 flops per FMA) for each type.
#include <cstdio>
#include <cuda_runtime.h>

template <typename T, int CHAINS>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
double run(int sms, int iters) {
  const int block = 256, grid = sms * 8;
  T* out;
  cudaMalloc(&out, sizeof(T) * grid * block);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_loop<T, 8><<<grid, block>>>(out, 16, (T)0.999, (T)0.001);
  cudaEventRecord(e0);
  fma_loop<T, 8><<<grid, block>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaFree(out);
  const double flops = 2.0 * 8 * (double)iters * grid * block;
  return flops / (ms * 1e-3) / 1e12;
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const double f64 = run<double>(sms, 2000);
  const double f32 = run<float>(sms, 20000);
  printf("{\"sms\": %d, \"fp64_fma_tflops\": %.3f, \"fp32_fma_tflops\": %.3f, \"err\": \"%s\"}\n", sms, f64, f32,
         cudaGetErrorString(cudaGetLastError()));
  return 0;
}
