// mt_peak.cu -- the FMA issue rate of the GPU in binary64 and binary32, the
// denominator of the ALU roofline that the benchmark reports for each Newton
// kernel against the pipe of its own precision.  The Newton kernels are
// bound by that pipe: they are neither a dense contraction nor HBM-bound
// (a root writes at most 32 bytes against ~10^4 flops).
//
// Each thread runs CH independent chains x <- x a + b (a, b fixed, |a| < 1,
// so the chains stay bounded) for 'iters' rounds; enough chains and warps
// hide the FMA latency, so the rate is the pipe's throughput.  2 flops per
// FMA.  The grid fills every SM with 4 blocks of 256 threads.
#include <cuda_runtime.h>

#include "mt_internal.h"
#include "mtsplit.h"

namespace mt {

constexpr int PEAK_CH = 8;
constexpr int PEAK_BLOCKS_PER_SM = 4;
constexpr int PEAK_BS = 256;

template <class T>
__global__ void __launch_bounds__(PEAK_BS) k_fma_chains(T* __restrict__ out, int iters, T a, T b) {
  T x[PEAK_CH];
#pragma unroll
  for (int c = 0; c < PEAK_CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PEAK_CH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PEAK_CH; ++c) s += x[c];
  out[(size_t)blockIdx.x * PEAK_BS + threadIdx.x] = s;  // keeps the chains alive
}

size_t fma_peak_bytes() {
  return (size_t)device_sm_count() * PEAK_BLOCKS_PER_SM * PEAK_BS * sizeof(double);
}

template <class T>
cudaError_t fma_rate(void* work, int iters, cudaStream_t s, double* tflops) {
  const int grid = device_sm_count() * PEAK_BLOCKS_PER_SM;
  T* out = (T*)work;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    MT_COUNT_LAUNCH(2);
    k_fma_chains<T><<<grid, PEAK_BS, 0, s>>>(out, 64, (T)0.999, (T)0.001);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    k_fma_chains<T><<<grid, PEAK_BS, 0, s>>>(out, iters, (T)0.999, (T)0.001);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess)
    *tflops = 2.0 * (double)grid * PEAK_BS * (double)iters * PEAK_CH / ((double)ms * 1e-3) / 1e12;
  return e;
}

}  // namespace mt

extern "C" MT_API size_t mt_fma_peak_workspace_bytes(void) { return mt::fma_peak_bytes(); }

namespace {
mt_status peak_fail(mt_status st, const char* msg) {
  mt::set_error_message(msg);  // reported by mt_last_error()
  return st;
}
}  // namespace

extern "C" MT_API mt_status mt_fma_peak(int prec, void* d_work, size_t work_bytes, double* tflops, void* stream) {
  mt::set_error_message("");
  if (!tflops || (prec != MT_FP64 && prec != MT_MIXED))
    return peak_fail(MT_EINVAL, "mt_fma_peak: prec must be MT_FP64 or MT_MIXED");
  if (!d_work || work_bytes < mt::fma_peak_bytes()) return peak_fail(MT_ENOMEM, "mt_fma_peak: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  // about 30 ms of work at the rates of a GB300 (binary64 ~1.2, binary32 ~74 TFLOP/s)
  const cudaError_t e = prec == MT_FP64 ? mt::fma_rate<double>(d_work, 1 << 14, s, tflops)
                                        : mt::fma_rate<float>(d_work, 1 << 19, s, tflops);
  if (e != cudaSuccess) return peak_fail(MT_ECUDA, cudaGetErrorString(e));
  return MT_OK;
}

extern "C" MT_API mt_status mt_check_sqrt_up(unsigned long long* n_fail, double* max_rel, void* stream) {
  mt::set_error_message("");
  if (!n_fail || !max_rel) return peak_fail(MT_EINVAL, "mt_check_sqrt_up: null output");
  const cudaError_t e = mt::check_sqrt_up(n_fail, max_rel, (cudaStream_t)stream);
  if (e != cudaSuccess) return peak_fail(MT_ECUDA, cudaGetErrorString(e));
  return MT_OK;
}
