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

namespace mgk {
namespace {

// Target centres in the workspace's control block: q' at ctrl[48..56), p' at
// ctrl[56..64).
constexpr int CTRL_TARGET_Q = 48, CTRL_TARGET_P = 56;

template <typename T, int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    k_regrid(const __grid_constant__ Plan P, const __grid_constant__ Bufs B) {
  using V = typename VT<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sflag;
  const Smem<V> S = carve<V>(P, smem_raw);
  const int D = P.D;
  if (__ldcg(B.status) != ST_OK) return;
  double* sc = S.sc;
  if (threadIdx.x < SC_N) sc[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x < D) {
    const int a = threadIdx.x;
    const double q0 = __ldcg(B.ctrl + a), q1 = __ldcg(B.ctrl + CTRL_TARGET_Q + a);
    sc[SC_Q + a] = q0;
    sc[SC_QN + a] = q1;
    sc[SC_P + a] = __ldcg(B.ctrl + CTRL_TARGET_P + a);
    sc[SC_DELTA + a] = q1 - q0;
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
    a.src = B.psi; a.dst = B.psi;
    axis_pass<T, false, KIND>(P, B, a, S, -1);
    if (!grid_sync(B, &sflag)) return;
  }
  for (int i = 0; i < D; ++i) {
    PassArgs a{};
    a.l = i; a.fft = 1; a.pre = PRE_K; a.post = 1;
    a.src = B.psi; a.dst = B.psi;
    axis_pass<T, true, KIND>(P, B, a, S, -1);
    if (i + 1 < D && !grid_sync(B, &sflag)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x < D) {
    B.ctrl[threadIdx.x] = sc[SC_QN + threadIdx.x];
    B.ctrl[8 + threadIdx.x] = sc[SC_P + threadIdx.x];
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

}  // namespace mgk
