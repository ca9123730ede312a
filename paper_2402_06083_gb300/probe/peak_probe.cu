// peak_probe.cu -- binary64 / binary32 FMA issue rate of this GPU.
//
// Each thread runs CH independent FMA chains (x <- x a + b) for 'iters'
// rounds; 2 flops per FMA.  With enough independent chains and warps the
// result is the FMA pipe's throughput, the denominator of the ALU roofline
// of the Newton kernels (the path is FP64-FMA-bound, not a contraction).
// Standalone: not part of libmtsplit.so.
#include <cstdio>
#include <cuda_runtime.h>

template <class T, int CH>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T, int CH>
double tflops(int sms, int blocks_per_sm, int bs, int iters) {
  T* out = nullptr;
  const int nthr = sms * blocks_per_sm * bs;
  if (cudaMalloc(&out, sizeof(T) * nthr) != cudaSuccess) return -1.0;
  k_fma_chains<T, CH><<<sms * blocks_per_sm, bs>>>(out, 16, (T)0.999, (T)0.001);  // warm-up
  cudaDeviceSynchronize();
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  k_fma_chains<T, CH><<<sms * blocks_per_sm, bs>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return 2.0 * (double)nthr * iters * CH / (ms * 1e-3) / 1e12;
}

int main() {
  int sms = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("SMs %d, max clock %d kHz\n", sms, clk);
  for (int bpsm : {1, 2, 4, 8})
    printf("fp64 chains8 blocks/SM %d x 256: %.3f TFLOP/s\n", bpsm, tflops<double, 8>(sms, bpsm, 256, 1 << 14));
  printf("fp64 chains2 blocks/SM 4 x 256: %.3f TFLOP/s\n", tflops<double, 2>(sms, 4, 256, 1 << 14));
  printf("fp64 chains1 blocks/SM 1 x 32: %.3f TFLOP/s\n", tflops<double, 1>(sms, 1, 32, 1 << 14));
  printf("fp64 chains1 blocks/SM 4 x 128: %.3f TFLOP/s\n", tflops<double, 1>(sms, 4, 128, 1 << 14));
  for (int bpsm : {2, 4, 8})
    printf("fp32 chains8 blocks/SM %d x 256: %.3f TFLOP/s\n", bpsm, tflops<float, 8>(sms, bpsm, 256, 1 << 16));
  const cudaError_t e = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}
