// Device side of the moving-grid split-operator propagator (sm_103a).
//
// One persistent cooperative kernel runs a whole mg_propagate call: every
// kinetic substep U_T,adpt (eq:T_split_substep_adaptive) and potential
// substep U_V,adpt (Sec. II.G.1) of every step, with the grid centres (q, p)
// updated in between from grid-wide reductions (the Ehrenfest averages of
// eq:eom_qt_case_III_T and eq:eom_pt_solution_case_III_V).
//
// Work decomposition.  The state is a row-major D-dimensional array.  A
// "pass" applies 1D transforms along one axis l: tiles of W adjacent lines are
// staged in shared memory (coalesced global access), transformed with a
// mixed-radix Stockham FFT (radix 2/3/4/8) in shared memory, and written
// back.  The diagonal multipliers of the method are fused into the passes:
//   forward pass along l:   u * A_l[j_l]                then FFT_l
//   inverse pass along l:   phi * K_l[k_l]  then IFFT_l then * conj(A_l[j_l]) / N_l
// where A_l[j] = (-1)^j e^{-i p_l (j - N_l/2) dq_l / hbar} is the j-dependent
// part of e^{-i t_KJ/hbar} (eq:t_definition) and
// K_l[k] = e^{(i/hbar)(delta_l p_l^K - tau minv_l (p_l^K)^2 / 2)} combines the
// kinetic phase of eq:U_T_tensor with f~(q + delta, p) f(q, p), which for a
// grid shift delta is exactly the diagonal factor e^{i delta . p^K / hbar}.
// The last forward pass also accumulates the kinetic moments (|phi|^2 and
// (k - N/2)|phi|^2); the last inverse pass also applies the potential phase
// e^{-i sigma V(x^J)/hbar} (eq:U_V_tensor) and accumulates |u|^2 dV/dq.
// Grid-wide dependencies (the reductions, and the per-axis tables that depend
// on their result) are separated by a capped-spin grid barrier.  When the
// whole state fits in the CTAs' shared memory, the tiles of the first and
// last axes stay resident across those barriers.
//
// Every wait in this file is bounded: a barrier that does not complete
// within the time limit records MG_ERR_TIMEOUT and the kernel returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_device.cuh"

namespace mgk {
namespace {

// ---------------------------------------------------------------------------
// The persistent propagation kernel
// ---------------------------------------------------------------------------

template <typename T, int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    k_propagate(const __grid_constant__ Plan P, const __grid_constant__ Bufs B, const __grid_constant__ Run RN) {
  using V = typename VT<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sflag;
  const Smem<V> S = carve<V>(P, B, smem_raw);
  const int D = P.D;
  // an unreported error from an earlier launch makes every later launch a no-op
  if (__ldcg(B.status) != ST_OK) return;
  double* sc = S.sc;
  if (threadIdx.x < SC_N) sc[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x < D) {
    sc[SC_Q + threadIdx.x] = __ldcg(B.ctrl + threadIdx.x);
    sc[SC_P + threadIdx.x] = __ldcg(B.ctrl + 8 + threadIdx.x);
  }
  load_tables(P, B, S, LT_TW | LT_A | LT_C | LT_SCT);
  init_mbarriers(S);
  const double* gam = B.gamma;
  int res = -1;
  bool kept = false;

  if (RN.lead_v) {
    if (threadIdx.x == 0) {
      const double sig = (RN.split == SPLIT_VTV ? 0.5 : 1.0) * gam[0] * RN.dt;
      sc[SC_SIG] = sig;
      sc[SC_SGH] = -sig / P.hbar;
    }
    if (threadIdx.x < D) sc[SC_QN + threadIdx.x] = sc[SC_Q + threadIdx.x];
    __syncthreads();
    build_tables(P, B, S, TB_V);
    if (!grid_sync(B, &sflag)) return;
    load_tables(P, B, S, LT_V);
    __syncthreads();
    PassArgs a{};
    a.l = D - 1; a.fft = 0; a.red = RED_V; a.slot = 1;
    a.keep = P.resident; a.src = B.psi; a.dst = B.psi;
    res = axis_pass<T, false, KIND>(P, B, a, S, -1);
    kept = P.resident;
    if (!grid_sync(B, &sflag)) return;
    finish(B, S, 1, D + 1);
    centre_after_potential(P, S, RN.motion);
    if (sc[SC_ERR] != 0.0) goto done;
    build_tables(P, B, S, TB_A);
    if (!grid_sync(B, &sflag)) return;
    load_tables(P, B, S, LT_A);
    __syncthreads();
  }

  for (int64_t u = 0; u < RN.n_units; ++u) {
    if (threadIdx.x == 0) {
      double tau, sig;
      bool hasv;
      unit_coeffs(RN, gam, u, tau, sig, hasv);
      sc[SC_TAU] = tau;
      sc[SC_SIG] = sig;
      sc[SC_SGH] = -sig / P.hbar;
      sc[SC_HASV] = hasv ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool hasv = sc[SC_HASV] != 0.0;
    // forward transform, kinetic moments on the last pass
    for (int i = 0; i < D; ++i) {
      const bool last = (i == D - 1);
      PassArgs a{};
      a.l = D - 1 - i; a.fft = 1; a.pre = PRE_A;
      a.from_smem = (i == 0 && kept);
      a.keep = last && P.resident;
      a.red = last ? RED_KIN : RED_NONE; a.slot = 0;
      a.src = B.psi; a.dst = B.psi;
      res = axis_pass<T, false, KIND>(P, B, a, S, res);
      kept = a.keep;
      if (!last && !grid_sync(B, &sflag)) return;
    }
    if (!grid_sync(B, &sflag)) return;
    finish(B, S, 0, D + 1);
    centre_after_kinetic(P, S, RN.motion);
    if (sc[SC_ERR] != 0.0) goto done;
    build_tables(P, B, S, TB_K | (hasv ? TB_V : 0));
    if (!grid_sync(B, &sflag)) return;
    load_tables(P, B, S, LT_K | (hasv ? LT_V : 0));
    if (threadIdx.x < D) sc[SC_Q + threadIdx.x] = sc[SC_QN + threadIdx.x];
    __syncthreads();
    // inverse transform, potential substep fused into the last pass
    for (int i = 0; i < D; ++i) {
      const bool last = (i == D - 1);
      PassArgs a{};
      a.l = i; a.fft = 1; a.pre = PRE_K; a.post = 1;
      a.from_smem = (i == 0 && kept);
      a.keep = last && hasv && P.resident;
      a.red = (last && hasv) ? RED_V : RED_NONE; a.slot = 1;
      a.src = B.psi; a.dst = B.psi;
      res = axis_pass<T, true, KIND>(P, B, a, S, res);
      kept = a.keep;
      if (!last && !grid_sync(B, &sflag)) return;
    }
    if (hasv) {
      if (!grid_sync(B, &sflag)) return;
      finish(B, S, 1, D + 1);
      centre_after_potential(P, S, RN.motion);
      if (sc[SC_ERR] != 0.0) goto done;
      build_tables(P, B, S, TB_A);
      if (!grid_sync(B, &sflag)) return;
      load_tables(P, B, S, LT_A);
      __syncthreads();
    }
  }
  if (kept) flush_resident<T>(P, B, S, res);
done:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int a = 0; a < D; ++a) {
      B.ctrl[a] = sc[SC_Q + a];
      B.ctrl[8 + a] = sc[SC_P + a];
    }
    if (sc[SC_ERR] != 0.0) atomicExch(B.status, (int)sc[SC_ERR]);
  }
}

// Tables A/Ainv for the current p-centre (after a state upload).  The
// shared-memory layout is the plan's own (element type of its precision).
template <typename T>
__global__ void __launch_bounds__(THREADS) k_init_tables(const __grid_constant__ Plan P,
                                                          const __grid_constant__ Bufs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<typename VT<T>::v> S = carve<typename VT<T>::v>(P, B, smem_raw);
  if (threadIdx.x < SC_N) S.sc[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x < P.D) {
    S.sc[SC_P + threadIdx.x] = B.ctrl[8 + threadIdx.x];
    S.sc[SC_Q + threadIdx.x] = B.ctrl[threadIdx.x];
  }
  load_tables(P, B, S, LT_SCT);
  __syncthreads();
  build_tables(P, B, S, TB_A);
}

// Observables: tables of V (unscaled) and of the kinetic energy.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_obs_tables(const __grid_constant__ Plan P,
                                                         const __grid_constant__ Bufs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<typename VT<T>::v> S = carve<typename VT<T>::v>(P, B, smem_raw);
  if (threadIdx.x < SC_N) S.sc[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x < P.D) {
    S.sc[SC_P + threadIdx.x] = B.ctrl[8 + threadIdx.x];
    S.sc[SC_QN + threadIdx.x] = B.ctrl[threadIdx.x];
  }
  if (threadIdx.x == 0) S.sc[SC_SGH] = 1.0;
  __syncthreads();
  build_tables(P, B, S, TB_V | TB_E);
}

// Observables: one forward pass (out of place into scratch) or the V pass.
template <typename T, int KIND>
__global__ void __launch_bounds__(THREADS)
    k_obs_pass(const __grid_constant__ Plan P, const __grid_constant__ Bufs B, int l, int mode) {
  using V = typename VT<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<V> S = carve<V>(P, B, smem_raw);
  if (threadIdx.x < SC_N) S.sc[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x < P.D) {
    S.sc[SC_Q + threadIdx.x] = B.ctrl[threadIdx.x];
    S.sc[SC_P + threadIdx.x] = B.ctrl[8 + threadIdx.x];  // p^K of the kinetic cross terms
  }
  if (threadIdx.x == 0) S.sc[SC_SGH] = 1.0;
  load_tables(P, B, S, LT_TW | LT_A | LT_C | LT_V | LT_E | LT_SCT);
  init_mbarriers(S);
  PassArgs a{};
  a.l = l;
  if (mode == 0) {  // forward transform pass; kinetic moments on axis 0
    a.fft = 1; a.pre = PRE_A;
    a.red = (l == 0) ? RED_OBS_KIN : RED_NONE; a.slot = 0;
    a.src = (l == P.D - 1) ? B.psi : (const void*)B.scratch;
    a.dst = B.scratch;
  } else {  // <V>, <x>, norm over psi (read only)
    a.red = RED_OBS_V; a.slot = 1;
    a.src = B.psi; a.dst = nullptr;
  }
  axis_pass<T, false, KIND>(P, B, a, S, -1);
}

// Separable state u^J = prod_l f_l[j_l] from per-axis factors staged in
// B.tabK (FP64 products, stored in the context's precision).  One row of the
// contiguous axis per thread at a time.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_set_product(const __grid_constant__ Plan P,
                                                          const __grid_constant__ Bufs B) {
  using V = typename VT<T>::v;
  const int D = P.D;
  const int nl = P.ax[D - 1].n;
  const int64_t rows = P.npts / nl;
  const double2* f = B.tabK;
  V* u = (V*)B.psi;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = make_double2(1.0, 0.0);
    uint64_t rem = (uint64_t)r;
    for (int a = D - 2; a >= 0; --a) {
      const uint64_t n = (uint64_t)P.N[a];
      const double2 v = f[P.ax[a].toff + (int)(rem % n)];
      rem /= n;
      acc = cmul(acc, v);
    }
    for (int j = 0; j < nl; ++j) {
      const double2 v = cmul(acc, f[P.ax[D - 1].toff + j]);
      u[r * nl + j] = from_d2<V>(v);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side launchers (C++ linkage, used by mg_capi.cu)
// ---------------------------------------------------------------------------

template <typename T, int KIND> static void* prop_fn() { return (void*)k_propagate<T, KIND>; }
template <typename T, int KIND> static void* obs_fn() { return (void*)k_obs_pass<T, KIND>; }

// prec 0: FP64 storage and arithmetic; prec 1: FP32 storage and transforms
// with FP64 phase arguments, reductions and grid centres.
void* propagate_kernel(int prec, int kind) {
  switch (kind * 2 + prec) {
    case POT_HARMONIC * 2: return prop_fn<double, POT_HARMONIC>();
    case POT_ATOM_DIATOM * 2: return prop_fn<double, POT_ATOM_DIATOM>();
    case POT_HENON_HEILES * 2: return prop_fn<double, POT_HENON_HEILES>();
    case POT_SECREST_JOHNSON * 2: return prop_fn<double, POT_SECREST_JOHNSON>();
    case POT_HARMONIC * 2 + 1: return prop_fn<float, POT_HARMONIC>();
    case POT_ATOM_DIATOM * 2 + 1: return prop_fn<float, POT_ATOM_DIATOM>();
    case POT_HENON_HEILES * 2 + 1: return prop_fn<float, POT_HENON_HEILES>();
    case POT_SECREST_JOHNSON * 2 + 1: return prop_fn<float, POT_SECREST_JOHNSON>();
  }
  return nullptr;
}

void* obs_kernel(int prec, int kind) {
  switch (kind * 2 + prec) {
    case POT_HARMONIC * 2: return obs_fn<double, POT_HARMONIC>();
    case POT_ATOM_DIATOM * 2: return obs_fn<double, POT_ATOM_DIATOM>();
    case POT_HENON_HEILES * 2: return obs_fn<double, POT_HENON_HEILES>();
    case POT_SECREST_JOHNSON * 2: return obs_fn<double, POT_SECREST_JOHNSON>();
    case POT_HARMONIC * 2 + 1: return obs_fn<float, POT_HARMONIC>();
    case POT_ATOM_DIATOM * 2 + 1: return obs_fn<float, POT_ATOM_DIATOM>();
    case POT_HENON_HEILES * 2 + 1: return obs_fn<float, POT_HENON_HEILES>();
    case POT_SECREST_JOHNSON * 2 + 1: return obs_fn<float, POT_SECREST_JOHNSON>();
  }
  return nullptr;
}

void* init_tables_kernel(int prec) { return prec ? (void*)k_init_tables<float> : (void*)k_init_tables<double>; }
void* set_product_kernel(int prec) { return prec ? (void*)k_set_product<float> : (void*)k_set_product<double>; }
void* obs_tables_kernel(int prec) { return prec ? (void*)k_obs_tables<float> : (void*)k_obs_tables<double>; }

}  // namespace mgk
