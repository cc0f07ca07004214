// FP64 / FP32 FMA throughput microbenchmark (test helper): 8 independent FMA
// chains per thread, 1216 CTAs x 256 threads, no memory traffic, CUDA events.
// Prints one line per precision.
#include <cstdio>
#include <cuda_runtime.h>
template <class T>
__global__ void k(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
    x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <class T> void run(const char* name, int iters) {
  int blocks = 152 * 8, threads = 256;
  T* out; cudaMalloc(&out, sizeof(T) * blocks * threads);
  k<T><<<blocks, threads>>>(out, 100, (T)0.999, (T)0.001);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0);
  k<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  double flops = 2.0 * 8 * (double)iters * blocks * threads;
  printf("%s: %.3f TFLOP/s (%.3f ms) err=%s\n", name, flops / ms / 1e9, ms, cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
}
int main() { run<double>("fp64 fma", 20000); run<float>("fp32 fma", 200000); return 0; }
