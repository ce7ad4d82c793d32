// Diagnostics of the device arithmetic the propagation kernels rely on; not
// part of the method.
//  - mg_probe_fma_rate: the GPU's FP64 (or FP32) fused multiply-add rate,
//    measured with CUDA events on independent FMA chains.  The FP64
//    configurations of the propagator are bound by the FP64 units, so their
//    roofline is stated against this measured rate.
//  - mg_probe_expi: the kernels' table-driven e^{i theta} (expi_tab, Tang's
//    method) evaluated on the GPU at caller-given arguments, so that its
//    accuracy can be checked against the host's sin and cos.
// Neither allocates device memory: the sink of the rate kernel and the
// 256-entry table of expi_tab are file-scope device arrays, and the caller
// passes the argument and result buffers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "mg_device.cuh"
#include "mgrid.h"

namespace mgk {
void fill_sincos_table(double* t);  // mg_capi.cu: the contexts' table

namespace {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_ITERS = 4096;

static __device__ double g_fma_sink[2];
static __device__ double2 g_expi_table[256];

// FMA_CHAINS independent chains per thread, FMA_ITERS FMAs each; a and b are
// kernel arguments, so nothing folds at compile time.  One thread stores the
// combined chains so that none of them is dead code.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T a, T b, int out) {
  T x[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < FMA_ITERS; i += 16) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
  if (s == (T)-12345.0) g_fma_sink[out] = (double)s;  // never true for these inputs
}

__global__ void k_expi(const double* __restrict__ th, double* __restrict__ s, double* __restrict__ c, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double sn, cs;
    expi_tab(th[i], g_expi_table, sn, cs);
    s[i] = sn;
    c[i] = cs;
  }
}

}  // namespace
}  // namespace mgk

using namespace mgk;

extern "C" mg_status mg_probe_fma_rate(int precision, void* cuda_stream, double* tflops) {
  if (!tflops || (precision != MG_FP64 && precision != MG_FP32_MIXED)) return MG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MG_ERR_CUDA;
  void* fn = precision == MG_FP64 ? (void*)k_fma_rate<double> : (void*)k_fma_rate<float>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0) != cudaSuccess || occ < 1) return MG_ERR_CUDA;
  // FP64: enough blocks for a few waves; FP32 issues 64x faster, so more work
  const int blocks = sms * occ * (precision == MG_FP64 ? 2 : 64);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MG_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MG_ERR_CUDA;
  }
  float best = 0;
  bool ok = true;
  for (int rep = 0; rep < 4 && ok; ++rep) {  // first repetition: warm-up
    ok = cudaEventRecord(e0, st) == cudaSuccess;
    if (precision == MG_FP64)
      k_fma_rate<double><<<blocks, 256, 0, st>>>(0.999999, 1e-9, 0);
    else
      k_fma_rate<float><<<blocks, 256, 0, st>>>(0.999999f, 1e-9f, 1);
    ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0;
    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    if (ok && rep > 0 && (best == 0 || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || !(best > 0)) return MG_ERR_CUDA;
  const double flops = 2.0 * (double)blocks * 256.0 * FMA_CHAINS * FMA_ITERS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return MG_OK;
}

extern "C" mg_status mg_probe_expi(const double* d_theta, double* d_sin, double* d_cos, int64_t n,
                                   void* cuda_stream) {
  if (n < 0 || (n > 0 && (!d_theta || !d_sin || !d_cos))) return MG_ERR_ARG;
  if (n == 0) return MG_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // e^{i k pi/128}, k = 0..255, exactly as the contexts build it
  double2 tab[256];
  fill_sincos_table(reinterpret_cast<double*>(tab));
  if (cudaMemcpyToSymbolAsync(g_expi_table, tab, sizeof(tab), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MG_ERR_CUDA;
  k_expi<<<1024, 256, 0, st>>>(d_theta, d_sin, d_cos, n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return MG_ERR_CUDA;
  return MG_OK;
}
