// Re-representation of the state on another grid (sm_103a): the exact
// trigonometric interpolation u' = f~(q', p') f(q, p') u between the grid
// centred at (q, p) and the grid centred at (q', p') (eq:F_defintion,
// eq:F_inv_definition).  It is the last step of every time step of the naive
// adaptive grid of Sec. II.F, and maps a state onto another grid for
// comparisons (the interpolation used for the error norms of Sec. III).
//
// In the kernels' factorisation, f(q, p') u = F(A(p') u) up to a constant
// phase, and f~(q', p') f(q, p') is the diagonal factor e^{i delta . p^K / hbar}
// in momentum space, delta = q' - q: the kinetic substep of k_propagate with
// tau = 0 and a prescribed shift.  One cooperative launch runs the D forward
// and D inverse axis passes with grid barriers in between.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_device.cuh"
#include "mg_regrid.h"

namespace mgk {

namespace {

template <typename T, int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    k_regrid(const __grid_constant__ Plan P, const __grid_constant__ Bufs B, const __grid_constant__ RegridArgs R) {
  using V = typename VT<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sflag;
  const Smem<V> S = carve<V>(P, B, smem_raw);
  const int D = P.D;
  if (__ldcg(B.status) != ST_OK) return;
  double* sc = S.sc;
  if (threadIdx.x < SC_N) sc[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x < D) {
    const int a = threadIdx.x;
    const double q0 = __ldcg(R.src_ctrl + a);
    sc[SC_Q + a] = q0;
    sc[SC_QN + a] = R.qt[a];
    sc[SC_P + a] = R.keep_p ? __ldcg(R.src_ctrl + 8 + a) : R.pt[a];
    sc[SC_DELTA + a] = R.qt[a] - q0;
  }
  if (threadIdx.x == 0) sc[SC_TAU] = 0.0;
  load_tables(P, B, S, LT_TW | LT_SCT);
  __syncthreads();
  // A(p'), conj(A(p'))/N and K = e^{i delta p^K / hbar} on the p' grid
  build_tables(P, B, S, TB_A | TB_K);
  if (!grid_sync(B, &sflag)) return;
  load_tables(P, B, S, LT_A | LT_K | LT_C);
  init_mbarriers(S);
  __syncthreads();
  for (int i = 0; i < D; ++i) {
    PassArgs a{};
    a.l = D - 1 - i; a.fft = 1; a.pre = PRE_A;
    a.src = R.buf; a.dst = R.buf;
    axis_pass<T, false, KIND>(P, B, a, S, -1);
    if (!grid_sync(B, &sflag)) return;
  }
  for (int i = 0; i < D; ++i) {
    PassArgs a{};
    a.l = i; a.fft = 1; a.pre = PRE_K; a.post = 1;
    a.src = R.buf; a.dst = R.buf;
    axis_pass<T, true, KIND>(P, B, a, S, -1);
    if (i + 1 < D && !grid_sync(B, &sflag)) return;
  }
  if (R.commit && blockIdx.x == 0 && threadIdx.x < D) {
    B.ctrl[threadIdx.x] = sc[SC_QN + threadIdx.x];
    B.ctrl[8 + threadIdx.x] = sc[SC_P + threadIdx.x];
  }
}

// Inner product sum_J conj(a_J) b_J of two states on the same grid: FP64
// per-thread sums, then per-CTA sums in a fixed order into part[cta][0..1]
// (real, imaginary); the host adds the CTA records in order.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_inner(const __grid_constant__ Plan P, const void* a_, const void* b_,
                                                    double* part) {
  using V = typename VT<T>::v;
  __shared__ double red[2][THREADS / 32];
  const V* a = (const V*)a_;
  const V* b = (const V*)b_;
  double re = 0, im = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.npts; j += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = to_d2(a[j]), y = to_d2(b[j]);
    re = fma(x.x, y.x, fma(x.y, y.y, re));
    im = fma(x.x, y.y, fma(-x.y, y.x, im));
  }
  re = warp_sum(re);
  im = warp_sum(im);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = re;
    red[1][warp] = im;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    part[(size_t)blockIdx.x * PSTRIDE + threadIdx.x] = s;
  }
}

template <typename T, int KIND> static void* regrid_fn() { return (void*)k_regrid<T, KIND>; }

}  // namespace

// The regrid kernel for FP64 (prec 0) or FP32 (prec 1) storage; the
// potential kind only selects the axis-pass instantiation (no potential
// work is done).
void* regrid_kernel(int prec, int kind) {
  switch (kind * 2 + prec) {
    case POT_HARMONIC * 2: return regrid_fn<double, POT_HARMONIC>();
    case POT_ATOM_DIATOM * 2: return regrid_fn<double, POT_ATOM_DIATOM>();
    case POT_HENON_HEILES * 2: return regrid_fn<double, POT_HENON_HEILES>();
    case POT_SECREST_JOHNSON * 2: return regrid_fn<double, POT_SECREST_JOHNSON>();
    case POT_HARMONIC * 2 + 1: return regrid_fn<float, POT_HARMONIC>();
    case POT_ATOM_DIATOM * 2 + 1: return regrid_fn<float, POT_ATOM_DIATOM>();
    case POT_HENON_HEILES * 2 + 1: return regrid_fn<float, POT_HENON_HEILES>();
    case POT_SECREST_JOHNSON * 2 + 1: return regrid_fn<float, POT_SECREST_JOHNSON>();
  }
  return nullptr;
}

void* inner_kernel(int prec) { return prec ? (void*)k_inner<float> : (void*)k_inner<double>; }

}  // namespace mgk
