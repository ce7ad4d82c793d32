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
#include "mg_tc.cuh"
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

// ---- tensor-core DFT of 16-point lines, standalone -----------------------
// The split-product DFT-GEMM of mg_tc.cuh on caller-given lines: every block
// builds the B operand of M = diag(post) F diag(pre) once, then transforms
// 256 lines per round (two warpgroups of 128 rows, one issuing thread, one
// commit per round, bounded waits).
static __device__ float2 g_tc_mult[32];  // pre[16], post[16]
static __device__ int g_tc_status;

template <int TC, bool INV>
__global__ void __launch_bounds__(256, 1)
    k_tc_dft16(const float2* __restrict__ x, float2* __restrict__ y, int64_t nlines, int has_post, int* status) {
  using TS = TcShape<TC>;
  extern __shared__ __align__(1024) unsigned char dyn[];
  unsigned char* tcb = dyn;
  unsigned char* tca = dyn + TS::NSPLIT * TS::B_BYTES;
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tslot;
  __shared__ float2 mult[32];
  if (threadIdx.x < 32) mult[threadIdx.x] = g_tc_mult[threadIdx.x];
  __syncthreads();
  tc_build_b<TC, INV>(tcb, mult, has_post ? mult + 16 : nullptr);
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    fence_mbar_init();
  }
  fence_proxy_async();
  tc_alloc(&tslot);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tslot;
  const int wg = threadIdx.x >> 7, row = threadIdx.x & 127;
  unsigned par = 0;
  bool failed = false;
  for (int64_t base = (int64_t)blockIdx.x * 256; base < nlines; base += (int64_t)gridDim.x * 256) {
    const int64_t line = base + threadIdx.x;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = line < nlines ? x[line * 16 + r] : make_float2(0.f, 0.f);
    tc_stage_line<TC>(tca + wg * TS::NSPLIT * TS::A_BYTES, row, v);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      tc_issue_products<TC>(tmem, tca, tcb);
      tc_issue_products<TC>(tmem + 32, tca + TS::NSPLIT * TS::A_BYTES, tcb);
      tc_commit(&bar);
    }
    bool ok = failed;
    const uint64_t t0 = global_ns();
    for (unsigned sp = 0; !ok; ++sp) {
      ok = mbar_try_wait(&bar, par);
      if (!ok && (sp & 255u) == 0 && global_ns() - t0 > 1000000000ull) {
        failed = true;
        atomicExch(status, 1);
        break;
      }
    }
    par ^= 1u;
    tc_fence_after();
    float d[32];
    tc_ld32(tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + wg * 32, d);
    tc_fence_before();
    if (line < nlines) {
#pragma unroll
      for (int r = 0; r < 16; ++r) y[line * 16 + r] = make_float2(d[2 * r], d[2 * r + 1]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc_dealloc(tmem);
}

template <int TC, bool INV> void* tc_kernel() { return (void*)k_tc_dft16<TC, INV>; }

// The same lines through the FP32 register DFT (16 = 4 x 4 with twiddles, the
// short-axis kernel's codelet form): the comparison for the tensor-core forms.
static __device__ float2 g_tw16[16];  // e^{-2 pi i m / 16}, rounded to FP32

template <bool INV>
__global__ void __launch_bounds__(256)
    k_reg_dft16(const float2* __restrict__ x, float2* __restrict__ y, int64_t nlines, int has_post) {
  __shared__ float2 tw[16], mult[32];
  if (threadIdx.x < 16) tw[threadIdx.x] = g_tw16[threadIdx.x];
  if (threadIdx.x < 32) mult[threadIdx.x] = g_tc_mult[threadIdx.x];
  __syncthreads();
  for (int64_t line = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; line < nlines;
       line += (int64_t)gridDim.x * blockDim.x) {
    float2 v[16], w[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(x[line * 16 + r], mult[r]);
    // first stage: 4-point DFTs over n1 (input index 4 n1 + n2), twiddle W^(n2 k1)
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      float2 t[4];
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) t[n1] = v[4 * n1 + n2];
      Dft<INV, 4, float2>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) {
        const int m = n2 * k1;
        w[n2 * 4 + k1] = m == 0 ? t[k1] : (INV ? cmulc(t[k1], tw[m]) : cmul(t[k1], tw[m]));
      }
    }
    // second stage: 4-point DFTs over n2, output index k1 + 4 k2
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 t[4];
#pragma unroll
      for (int n2 = 0; n2 < 4; ++n2) t[n2] = w[n2 * 4 + k1];
      Dft<INV, 4, float2>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) y[line * 16 + r] = has_post ? cmul(v[r], mult[16 + r]) : v[r];
  }
}

}  // namespace
}  // namespace mgk

using namespace mgk;

extern "C" mg_status mg_probe_tc_dft16(int split, int inverse, const void* d_x, void* d_y, int64_t nlines,
                                       const double* pre, const double* post, void* cuda_stream) {
  if (nlines < 0 || (nlines > 0 && (!d_x || !d_y)) || !pre || split < 0 || split > 2) return MG_ERR_ARG;
  if (nlines == 0) return MG_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float2 m[32];
  for (int i = 0; i < 16; ++i) {
    m[i] = make_float2((float)pre[2 * i], (float)pre[2 * i + 1]);
    m[16 + i] = post ? make_float2((float)post[2 * i], (float)post[2 * i + 1]) : make_float2(1.f, 0.f);
  }
  if (split == 0) {
    float2 tw[16];
    for (int i = 0; i < 16; ++i) {
      const double a = -2.0 * M_PI * i / 16.0;
      tw[i] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    int dev = 0, sms = 0;
    if (cudaMemcpyToSymbolAsync(g_tc_mult, m, sizeof(m), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyToSymbolAsync(g_tw16, tw, sizeof(tw), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return MG_ERR_CUDA;
    const int64_t want = (nlines + 255) / 256;
    const int blocks = (int)(want < 8 * sms ? want : 8 * sms);
    const float2* xp = (const float2*)d_x;
    float2* yp = (float2*)d_y;
    if (inverse)
      k_reg_dft16<true><<<blocks, 256, 0, st>>>(xp, yp, nlines, post ? 1 : 0);
    else
      k_reg_dft16<false><<<blocks, 256, 0, st>>>(xp, yp, nlines, post ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return MG_ERR_CUDA;
    return MG_OK;
  }
  void* fn = split == 1 ? (inverse ? tc_kernel<TC_TF32X3, true>() : tc_kernel<TC_TF32X3, false>())
                        : (inverse ? tc_kernel<TC_BF16X3, true>() : tc_kernel<TC_BF16X3, false>());
  const int smem = split == 1 ? TcShape<TC_TF32X3>::NSPLIT * (TcShape<TC_TF32X3>::B_BYTES + 2 * TcShape<TC_TF32X3>::A_BYTES)
                              : TcShape<TC_BF16X3>::NSPLIT * (TcShape<TC_BF16X3>::B_BYTES + 2 * TcShape<TC_BF16X3>::A_BYTES);
  int* status = nullptr;
  if (cudaGetSymbolAddress((void**)&status, g_tc_status) != cudaSuccess) return MG_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_tc_mult, m, sizeof(m), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return MG_ERR_CUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MG_ERR_CUDA;
  const int64_t want = (nlines + 255) / 256;
  const int blocks = (int)(want < sms ? want : sms);
  int has_post = post ? 1 : 0;
  void* args[] = {(void*)&d_x, (void*)&d_y, (void*)&nlines, (void*)&has_post, (void*)&status};
  if (cudaLaunchKernel(fn, dim3(blocks), dim3(256), args, smem, st) != cudaSuccess) return MG_ERR_CUDA;
  int hs = 0;
  if (cudaMemcpyFromSymbolAsync(&hs, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MG_ERR_CUDA;
  return hs ? MG_ERR_TIMEOUT : MG_OK;
}

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
