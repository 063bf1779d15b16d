// Measured arithmetic ceilings for the rooflines of the ALU-bound kernels: the
// FP32 and FP64 fused multiply-add rates of this GPU.  Every thread runs CH
// independent FMA recurrences a <- a * b + c (b just below 1, so the values
// stay bounded and no operand is a constant the compiler could fold), enough
// of them per SM sub-partition to cover the pipe latency; one FMA counts two
// flops.  The grid holds BLOCKS_PER_SM blocks of 256 threads per SM.
#include <cuda_runtime.h>

#include "ibm.h"

extern "C" ibm_status ibm__noalloc_fail(ibm_status s, const char *msg);

namespace {

constexpr int CH = 8;
constexpr int THREADS = 256;
constexpr int BLOCKS_PER_SM = 4;

template <typename T>
__global__ void __launch_bounds__(THREADS) k_fma_peak(long long iters, T b, T c, T *__restrict__ out) {
  T a[CH];
#pragma unroll
  for (int i = 0; i < CH; i++) a[i] = (T)(threadIdx.x + 37 * i) * (T)1e-4;
#pragma unroll 8
  for (long long it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < CH; i++) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < CH; i++) s += a[i];
  out[(size_t)blockIdx.x * THREADS + threadIdx.x] = s;
}

template <typename T>
ibm_status run(long long iters, double *flops_per_s, double *ms) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ibm__noalloc_fail(IBM_ECUDA, "ibm_fma_peak: no CUDA device");
  const int blocks = nsm * BLOCKS_PER_SM;
  T *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ibm_status st = IBM_OK;
  float t = 0.f;
  if (cudaMalloc(&out, (size_t)blocks * THREADS * sizeof(T)) != cudaSuccess)
    return ibm__noalloc_fail(IBM_ENOMEM, "ibm_fma_peak: output allocation failed");
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = ibm__noalloc_fail(IBM_ECUDA, "ibm_fma_peak: event creation failed");
  } else {
    const T b = (T)0.9999999, c = (T)1e-7;
    k_fma_peak<T><<<blocks, THREADS>>>(iters / 16 + 1, b, c, out);  // warm-up (clocks, instruction cache)
    cudaEventRecord(e0);
    k_fma_peak<T><<<blocks, THREADS>>>(iters, b, c, out);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || t <= 0.f)
      st = ibm__noalloc_fail(IBM_ECUDA, "ibm_fma_peak: kernel or timing failed");
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (st != IBM_OK) return st;
  *ms = (double)t;
  *flops_per_s = 2.0 * CH * (double)iters * (double)blocks * THREADS / ((double)t * 1e-3);
  return IBM_OK;
}

}  // namespace

extern "C" ibm_status ibm_fma_peak(int fp64, long long iters, double *flops_per_s, double *ms) {
  if (!flops_per_s || !ms || iters <= 0) return ibm__noalloc_fail(IBM_EINVAL, "ibm_fma_peak: bad argument");
  return fp64 ? run<double>(iters, flops_per_s, ms) : run<float>(iters, flops_per_s, ms);
}
