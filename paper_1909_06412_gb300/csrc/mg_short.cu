// Short-axis propagation kernel (sm_103a): the moving-grid split-operator
// integrator of mg_kernels.cu specialised to tensor grids whose D >= 3 axes
// all have n = 8, 12 or 16 points (the 8D Henon-Heiles grids of Sec. III.C).
//
// Same method and same persistent structure as k_propagate: kinetic substeps
// U_T,adpt (eq:T_split_substep_adaptive) and potential substeps U_V,adpt
// (Sec. II.G.1) with the grid centres updated from grid-wide reductions
// (eq:eom_qt_case_III_T, eq:eom_pt_solution_case_III_V), composed as in
// eq:comp_TVT, all in one cooperative launch.  What differs is how a
// transform moves through memory:
//  - A pass transforms a group of up to SHORT_MAXG consecutive axes (mg_short.h),
//    so a full transform of an 8D grid takes 3-4 passes over the state
//    instead of 8.
//  - Chunks are copied between global and shared memory with cp.async
//    (16 B per FP64 element, 8 B per FP32 element), nreg-1 chunks ahead of the
//    one being transformed.
//  - Each thread transforms whole lines held in registers: an n-point DFT of
//    compile-time length (8: radix-8 codelet; 12 = 4 x 3 and 16 = 4 x 4 as two
//    codelet stages with the twiddles in between).
//  - The multipliers of the method are applied per line: A_l before the
//    forward DFT along l, K_l before and conj(A_l)/N_l after the inverse DFT.
//  - The potential phase e^{-i sigma V(x^J)/hbar} (eq:U_V_tensor) is a product
//    of per-axis factors e^{-i sigma f_a(x_a)/hbar} and nearest-neighbour pair
//    factors e^{-i sigma h_a(x_a) g_{a+1}(x_{a+1})/hbar}, each tabulated from
//    an FP64 phase argument once per substep; V = sum_a f_a + sum_a h_a g_{a+1}
//    covers the Henon-Heiles and the diagonal harmonic potentials.  Its
//    gradient, needed for <dV/dq>, is accumulated from tabulated f', g, g', h,
//    h' with the line structure: the terms that do not depend on the line's
//    own coordinate are weighted by the line's norm once per line.
//  - FP32 storage: the sums over points are per-line FP32 sums accumulated
//    per thread with an error-free two-sum, then in FP64 across threads and
//    CTAs, like the FP32 kinetic moments of the general kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_device.cuh"
#include "mg_short.h"

namespace mgk {
namespace {

constexpr int short_threads(int n) { return n % 3 == 0 ? 288 : 256; }

enum { SM_NONE = 0, SM_KIN = 1, SM_V = 2, SM_VONLY = 3 };

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies of one element
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async_el(double2* s, const double2* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_el(float2* s, const float2* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// ---------------------------------------------------------------------------
// n-point DFT of a line held in registers (natural order in and out)
// ---------------------------------------------------------------------------

// x[k] *= W_n^m (W_n = e^{-2 pi i / n}; conjugate for the inverse); m is a
// compile-time constant after unrolling, quarter turns are exact.
template <bool INV, int N, typename V>
__device__ __forceinline__ V twiddle(V t, int m, const V* __restrict__ tw) {
  if (m == 0) return t;
  if (4 * m == N) return mul_si<INV>(t);
  if (2 * m == N) return V{-t.x, -t.y};
  if (4 * m == 3 * N) return mul_si<!INV>(t);
  return INV ? cmulc(t, tw[m]) : cmul(t, tw[m]);
}

// N = R1 * R2 by one decimation step: input index R2 n1 + n2, output k1 + R1 k2.
template <bool INV, int R1, int R2, typename V>
__device__ __forceinline__ void dft2(V* x, const V* __restrict__ tw) {
  constexpr int N = R1 * R2;
  V y[N];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    V t[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) t[n1] = x[R2 * n1 + n2];
    Dft<INV, R1, V>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = twiddle<INV, N>(t[k1], (n2 * k1) % N, tw);
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    V t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
    Dft<INV, R2, V>::run(t);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = t[k2];
  }
}

template <bool INV, int N, typename V> struct LineDft;
template <bool INV, typename V> struct LineDft<INV, 8, V> {
  static __device__ __forceinline__ void run(V* x, const V*) { Dft<INV, 8, V>::run(x); }
};
template <bool INV, typename V> struct LineDft<INV, 12, V> {
  static __device__ __forceinline__ void run(V* x, const V* tw) { dft2<INV, 4, 3>(x, tw); }
};
template <bool INV, typename V> struct LineDft<INV, 16, V> {
  static __device__ __forceinline__ void run(V* x, const V* tw) { dft2<INV, 4, 4>(x, tw); }
};

// ---------------------------------------------------------------------------
// Per-thread accumulators of the fused reductions
// ---------------------------------------------------------------------------

template <typename T> struct LineAcc;
template <> struct LineAcc<double> {
  double a[MAXD + 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < MAXD + 1; ++i) a[i] = 0.0;
  }
  __device__ __forceinline__ void add(int i, double x) { a[i] += x; }
  __device__ __forceinline__ double get(int i) const { return a[i]; }
  // i known only at run time: predicated adds keep the array in registers
  __device__ __forceinline__ void add_rt(int i, double x) {
#pragma unroll
    for (int k = 0; k < MAXD + 1; ++k)
      if (k == i) a[k] += x;
  }
};
template <> struct LineAcc<float> {
  float s[MAXD + 1], c[MAXD + 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < MAXD + 1; ++i) s[i] = c[i] = 0.f;
  }
  __device__ __forceinline__ void add(int i, float x) { two_sum_acc(s[i], c[i], x); }
  __device__ __forceinline__ double get(int i) const { return (double)s[i] + (double)c[i]; }
  __device__ __forceinline__ void add_rt(int i, float x) {
#pragma unroll
    for (int k = 0; k < MAXD + 1; ++k)
      if (k == i) two_sum_acc(s[k], c[k], x);
  }
};

// Sum of acc[0 .. nv-1] over the CTA in a fixed order (warp trees, then warp
// order) into the CTA's record of `slot`, read back by finish().
template <typename T>
__device__ void block_record(const Bufs& B, double* red, int slot, const LineAcc<T>& acc, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < MAXD + 1; ++v)
    if (v < nv) {
      const double s = warp_sum(acc.get(v));
      if (lane == 0) red[warp * 16 + v] = s;
    }
  __syncthreads();
  if (warp == 0 && lane < nv) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += red[w * 16 + lane];
    __stcg(B.part + ((size_t)slot * gridDim.x + blockIdx.x) * PSTRIDE + lane, s);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Shared memory of the short-axis kernel
// ---------------------------------------------------------------------------

template <typename V, typename T> struct SSm {
  Smem<V> s;  // tw, tA, tAi, tK, sct, fin, sc, red (the fields the shared helpers use)
  V* F;       // [D*n] per-axis potential factors
  V* Pt;      // [(D-1)*n*n] pair factors
  T* col;     // [5][D*n] f', g, g', h, h'
  V* reg[3];
};

template <typename V, typename T>
__device__ SSm<V, T> carve_short(const Plan& P, const ShortPlan& SP, unsigned char* base) {
  SSm<V, T> m;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += (bytes + 15) & ~size_t(15);
    return p;
  };
  const int TT = P.tab_total, n = SP.n;
  Smem<V>& s = m.s;
  s.tw = (V*)take(sizeof(V) * TT);
  s.tA = (V*)take(sizeof(V) * TT);
  s.tAi = (V*)take(sizeof(V) * TT);
  s.tK = (V*)take(sizeof(V) * TT);
  s.tv = nullptr;
  s.tc = nullptr;
  s.te = nullptr;
  s.sct = (double2*)take(sizeof(double2) * 256);
  s.red = (double*)take(sizeof(double) * 16 * 32);
  s.fin = (double*)take(sizeof(double) * PSTRIDE);
  s.sc = (double*)take(sizeof(double) * SC_N);
  s.mbar = nullptr;
  s.mphase = nullptr;
  s.tb = nullptr;
  s.li = nullptr;
  m.F = (V*)take(sizeof(V) * TT);
  m.Pt = (V*)take(sizeof(V) * (P.D - 1) * n * n);
  m.col = (T*)take(sizeof(T) * 5 * TT);
  for (int r = 0; r < 3; ++r) m.reg[r] = r < SP.nreg ? (V*)take(sizeof(V) * SP.region_elems) : nullptr;
  s.reg[0] = m.reg[0];
  s.reg[1] = m.reg[1];
  s.reg[2] = m.reg[2];
  s.end = off;
  return m;
}

// ---------------------------------------------------------------------------
// Potential tables: V = sum_a f_a(x_a) + sum_{a<D-1} h_a(x_a) g_{a+1}(x_{a+1})
// ---------------------------------------------------------------------------

// f, f', g, g', h, h' of axis a at x.
__device__ __forceinline__ void chain_terms(const Plan& P, int a, double x, double* t) {
  const int D = P.D;
  if (P.pot_kind == POT_HENON_HEILES) {
    const double lam = P.pot[0];
    t[0] = 0.5 * x * x - (a >= 1 ? lam * x * x * x / 3.0 : 0.0);
    t[1] = x - (a >= 1 ? lam * x * x : 0.0);
    t[2] = a >= 1 ? x : 0.0;
    t[3] = a >= 1 ? 1.0 : 0.0;
    t[4] = a <= D - 2 ? lam * x * x : 0.0;
    t[5] = a <= D - 2 ? 2.0 * lam * x : 0.0;
  } else {  // harmonic with a diagonal force-constant matrix
    const double k = P.pot[a * D + a];
    const double d = x - P.pot[D * D + a];
    t[0] = 0.5 * k * d * d;
    t[1] = k * d;
    t[2] = t[3] = t[4] = t[5] = 0.0;
  }
}

// Build the per-axis factors F, the gradient columns (in B.tabV) and the pair
// factors for the grid centred at q_new (scalars SC_QN, SC_SGH of the CTA).
// Tasks of 32 entries, dealt to warp 0 of every CTA first.  A grid barrier
// must follow.
template <typename V>
__device__ void build_v_short(const Plan& P, const ShortPlan& SP, const Bufs& B, const Smem<V>& S) {
  const int TT = P.tab_total, n = SP.n;
  const int nP = SP.pairs ? (P.D - 1) * n * n : 0;
  const int nchF = (TT + 31) / 32, nchP = (nP + 31) / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const double* sc = S.sc;
  const double sgh = sc[SC_SGH];
  for (int t = warp * gridDim.x + blockIdx.x; t < nchF + nchP; t += nwarps * gridDim.x) {
    if (t < nchF) {
      const int e = t * 32 + lane;
      if (e >= TT) continue;
      const int a = e / n, j = e - a * n;
      const double x = fma((double)(j - n / 2), P.dq[a], sc[SC_QN + a]);
      double c[6];
      chain_terms(P, a, x, c);
      double sn, cs;
      expi_prec(P.prec, sgh * c[0], S.sct, sn, cs);
      __stcg(SP.tabF + e, P.prec ? round_unit_f32(cs, sn, 1.0) : make_double2(cs, sn));
#pragma unroll
      for (int k = 0; k < 5; ++k) __stcg(B.tabV + k * TT + e, c[1 + k]);
    } else {
      const int e = (t - nchF) * 32 + lane;
      if (e >= nP) continue;
      const int a = e / (n * n), rem = e - a * n * n;
      const int j = rem / n, j2 = rem - j * n;
      const double x = fma((double)(j - n / 2), P.dq[a], sc[SC_QN + a]);
      const double y = fma((double)(j2 - n / 2), P.dq[a + 1], sc[SC_QN + a + 1]);
      double ca[6], cb[6];
      chain_terms(P, a, x, ca);
      chain_terms(P, a + 1, y, cb);
      double sn, cs;
      expi_prec(P.prec, sgh * ca[4] * cb[2], S.sct, sn, cs);
      __stcg(SP.tabP + e, P.prec ? round_unit_f32(cs, sn, 1.0) : make_double2(cs, sn));
    }
  }
}

template <typename V, typename T>
__device__ void load_v_short(const Plan& P, const ShortPlan& SP, const Bufs& B, const SSm<V, T>& S) {
  const int TT = P.tab_total, n = SP.n;
  const int nP = SP.pairs ? (P.D - 1) * n * n : 0;
  for (int e = threadIdx.x; e < TT; e += blockDim.x) {
    S.F[e] = from_d2<V>(__ldcg(SP.tabF + e));
#pragma unroll
    for (int k = 0; k < 5; ++k) S.col[k * TT + e] = (T)__ldcg(B.tabV + k * TT + e);
  }
  for (int e = threadIdx.x; e < nP; e += blockDim.x) S.Pt[e] = from_d2<V>(__ldcg(SP.tabP + e));
}

// ---------------------------------------------------------------------------
// Index helpers
// ---------------------------------------------------------------------------

template <int N> __device__ __forceinline__ int ipow(int k) {
  int r = 1;
#pragma unroll
  for (int i = 0; i < SHORT_MAXG; ++i)
    if (i < k) r *= N;
  return r;
}

// Base-N digits of x into j[a] for lo <= a <= hi (j[hi] least significant).
template <int N> __device__ __forceinline__ void digits(unsigned x, int lo, int hi, int (&j)[MAXD]) {
#pragma unroll
  for (int a = MAXD - 1; a >= 0; --a)
    if (a >= lo && a <= hi) {
      const unsigned q = x / N;
      j[a] = (int)(x - q * N);
      x = q;
    }
}

// j[i] for an index known only at run time, without moving j to local memory.
__device__ __forceinline__ int pick(const int (&j)[MAXD], int i) {
  int v = 0;
#pragma unroll
  for (int k = 0; k < MAXD; ++k)
    if (k == i) v = j[k];
  return v;
}

// ---------------------------------------------------------------------------
// Chunk copies
// ---------------------------------------------------------------------------

// Global offset of chunk c (first element) and its number of planes.
__device__ __forceinline__ void chunk_geom(const GroupPlan& G, int64_t c, int64_t& gbase, int& nwt) {
  if (G.contig) {
    const int64_t b0 = c * G.WT;
    gbase = b0 * G.ng;
    nwt = (int)(G.nblk - b0 < G.WT ? G.nblk - b0 : G.WT);
  } else {
    const int64_t o = c / G.nb, b = c - o * G.nb;
    gbase = o * (int64_t)G.ng * G.inner + b * G.WT;
    nwt = G.WT;
  }
}

template <int N, typename V>
__device__ __forceinline__ void issue_load(const GroupPlan& G, const V* __restrict__ src, int64_t c, V* reg) {
  int64_t gb;
  int nwt;
  chunk_geom(G, c, gb, nwt);
  const int cnt = nwt * G.ng;
  if (G.contig) {
    const Div16 dng((unsigned)G.ng);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int wt = (int)dng((unsigned)e), row = e - wt * G.ng;
      cp_async_el(reg + wt * G.PS + (row / N) * (N + 1) + row % N, src + gb + e);
    }
  } else {
    const Div16 dw((unsigned)G.WT);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int row = (int)dw((unsigned)e), wt = e - row * G.WT;
      cp_async_el(reg + wt * G.PS + (row / N) * (N + 1) + row % N, src + gb + row * G.inner + wt);
    }
  }
}

template <int N, typename V>
__device__ __forceinline__ void store_chunk(const GroupPlan& G, V* __restrict__ dst, int64_t c, const V* reg) {
  int64_t gb;
  int nwt;
  chunk_geom(G, c, gb, nwt);
  const int cnt = nwt * G.ng;
  if (G.contig) {
    const Div16 dng((unsigned)G.ng);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int wt = (int)dng((unsigned)e), row = e - wt * G.ng;
      __stcs(dst + gb + e, reg[wt * G.PS + (row / N) * (N + 1) + row % N]);
    }
  } else {
    const Div16 dw((unsigned)G.WT);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int row = (int)dw((unsigned)e), wt = e - row * G.WT;
      __stcs(dst + gb + row * G.inner + wt, reg[wt * G.PS + (row / N) * (N + 1) + row % N]);
    }
  }
}

// ---------------------------------------------------------------------------
// One group pass
// ---------------------------------------------------------------------------

template <typename T, int N, bool INV>
__device__ void short_pass(const Plan& P, const ShortPlan& SP, const Bufs& B, const SSm<typename VT<T>::v, T>& S,
                           int gi, int mode, int slot) {
  using V = typename VT<T>::v;
  const GroupPlan& G = SP.grp[gi];
  const int D = P.D, g = G.g, l0 = G.l0;
  const int TT = P.tab_total;
  V* psi = (V*)B.psi;
  const V* tw = S.s.tw;  // forward twiddles of axis 0 (all axes have n points)
  const int nreg = SP.nreg;
  const int64_t mine = blockIdx.x < G.nchunks ? (G.nchunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  LineAcc<T> acc;
  acc.zero();

  for (int s = 0; s < nreg - 1; ++s) {
    if (s < mine) issue_load<N>(G, psi, blockIdx.x + (int64_t)s * gridDim.x, S.reg[s]);
    cp_commit();
  }
  for (int64_t i = 0; i < mine; ++i) {
    const int64_t c = blockIdx.x + i * gridDim.x;
    {
      const int64_t i2 = i + nreg - 1;
      if (i2 < mine) issue_load<N>(G, psi, blockIdx.x + i2 * gridDim.x, S.reg[i2 % nreg]);
      cp_commit();
    }
    if (nreg == 3) cp_wait<2>();
    else cp_wait<1>();
    __syncthreads();
    V* reg = S.reg[i % nreg];
    int64_t gb;
    int nwt;
    chunk_geom(G, c, gb, nwt);
    const int nl = nwt * ipow<N>(g - 1);  // lines along any group axis
    // first block (contig) or first trailing index (strided) of the chunk
    const unsigned cbase = G.contig ? (unsigned)(c * G.WT) : (unsigned)((c % G.nb) * G.WT);
    const int kfirst = mode == SM_VONLY ? g - 1 : 0;
    for (int kk = kfirst; kk < g; ++kk) {
      // forward: last axis of the group first; inverse: first axis first
      const int k = mode == SM_VONLY ? g - 1 : (INV ? kk : g - 1 - kk);
      const int a = l0 + k;
      const bool last = (kk == g - 1);
      const int nlo = ipow<N>(g - 1 - k), nhi = ipow<N>(k);
      const int stride = (k == g - 1) ? 1 : ipow<N>(g - 2 - k) * (N + 1);
      const Div16 dlo((unsigned)nlo), dhi((unsigned)nhi);
      const V* pre = mode == SM_VONLY ? nullptr : (INV ? S.s.tK : S.s.tA) + a * N;
      const V* post = (mode != SM_VONLY && INV) ? S.s.tAi + a * N : nullptr;
      for (int L = threadIdx.x; L < nl; L += blockDim.x) {
        const int t = (int)dlo((unsigned)L), lo = L - t * nlo;
        const int wt = (int)dhi((unsigned)t), hi = t - wt * nhi;
        const int base = wt * G.PS +
                         (k == g - 1 ? hi * (N + 1) : (hi * nlo + lo / N) * (N + 1) + lo % N);
        V x[N];
#pragma unroll
        for (int r = 0; r < N; ++r) x[r] = reg[base + r * stride];
        if (pre) {
#pragma unroll
          for (int r = 0; r < N; ++r) x[r] = cmul(x[r], pre[r]);
          LineDft<INV, N, V>::run(x, tw);
        }
        if (post) {
#pragma unroll
          for (int r = 0; r < N; ++r) x[r] = cmul(x[r], post[r]);
        }
        if (last && mode == SM_KIN) {
          // kinetic moments; the line runs along axis 0 (k = 0, l0 = 0)
          int j[MAXD];
          digits<N>((unsigned)lo, 1, g - 1, j);
          if (!G.contig) digits<N>(cbase + wt, g, D - 1, j);
          T s0 = 0, s1 = 0;
#pragma unroll
          for (int r = 0; r < N; ++r) {
            const T w = x[r].x * x[r].x + x[r].y * x[r].y;
            s0 += w;
            s1 += (T)(r - N / 2) * w;
          }
          acc.add(0, s0);
          acc.add(1, s1);
#pragma unroll
          for (int b = 1; b < MAXD; ++b)
            if (b < D) acc.add(1 + b, (T)(j[b] - N / 2) * s0);
        } else if (last && (mode == SM_V || mode == SM_VONLY)) {
          // potential phase and gradient moments; the line runs along axis D-1
          int j[MAXD];
          if (g >= 2) digits<N>((unsigned)hi, l0, D - 2, j);
          if (l0 > 0) digits<N>(cbase + wt, 0, l0 - 1, j);
          const int jm = pick(j, D - 2), jm2 = pick(j, D - 3 < 0 ? 0 : D - 3);
          const T* cfp = S.col;
          const T* cg = S.col + TT;
          const T* cgp = S.col + 2 * TT;
          const T* ch = S.col + 3 * TT;
          const T* chp = S.col + 4 * TT;
          V lf = S.F[j[0]];
#pragma unroll
          for (int b = 1; b < MAXD - 1; ++b)
            if (b < D - 1) lf = cmul(lf, S.F[b * N + j[b]]);
          const V* prow = nullptr;
          if (SP.pairs) {
#pragma unroll
            for (int b = 0; b < MAXD - 2; ++b)
              if (b < D - 2) lf = cmul(lf, S.Pt[(b * N + j[b]) * N + j[b + 1]]);
            prow = S.Pt + ((D - 2) * N + jm) * N;
          }
          const V* fl = S.F + (D - 1) * N;
          T s0 = 0, sg = 0, sfp = 0, sgp = 0;
#pragma unroll
          for (int r = 0; r < N; ++r) {
            const T w = x[r].x * x[r].x + x[r].y * x[r].y;
            s0 += w;
            sg += cg[(D - 1) * N + r] * w;
            sfp += cfp[(D - 1) * N + r] * w;
            sgp += cgp[(D - 1) * N + r] * w;
            V f = cmul(lf, fl[r]);
            if (prow) f = cmul(f, prow[r]);
            x[r] = cmul(x[r], f);
          }
          acc.add(0, s0);
          // axes whose derivative does not involve the line's coordinate
#pragma unroll
          for (int b = 0; b < MAXD - 2; ++b)
            if (b < D - 2) {
              T gb2 = cfp[b * N + j[b]] + chp[b * N + j[b]] * cg[(b + 1) * N + j[b + 1]];
              if (b > 0) gb2 += ch[(b - 1) * N + j[b - 1]] * cgp[b * N + j[b]];
              acc.add(1 + b, gb2 * s0);
            }
          {
            const int b = D - 2;  // D >= 3
            const T gb2 = (cfp[b * N + jm] + ch[(b - 1) * N + jm2] * cgp[b * N + jm]) * s0 + chp[b * N + jm] * sg;
            acc.add_rt(1 + b, gb2);
            acc.add_rt(D, sfp + ch[b * N + jm] * sgp);
          }
        }
#pragma unroll
        for (int r = 0; r < N; ++r) reg[base + r * stride] = x[r];
      }
      __syncthreads();
    }
    store_chunk<N>(G, psi, c, reg);
    __syncthreads();
  }
  cp_wait<0>();
  if (mode != SM_NONE) block_record<T>(B, S.s.red, slot, acc, D + 1);
}

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------

template <typename T, int N>
__global__ void __launch_bounds__(short_threads(N), 1)
    k_propagate_short(const __grid_constant__ Plan P, const __grid_constant__ Bufs B,
                      const __grid_constant__ Run RN, const __grid_constant__ ShortPlan SP) {
  using V = typename VT<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sflag;
  const SSm<V, T> S = carve_short<V, T>(P, SP, smem_raw);
  const int D = P.D, ng = SP.ngroups;
  if (__ldcg(B.status) != ST_OK) return;
  double* sc = S.s.sc;
  if (threadIdx.x < SC_N) sc[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x < D) {
    sc[SC_Q + threadIdx.x] = __ldcg(B.ctrl + threadIdx.x);
    sc[SC_P + threadIdx.x] = __ldcg(B.ctrl + 8 + threadIdx.x);
  }
  load_tables(P, B, S.s, LT_TW | LT_A | LT_SCT);
  __syncthreads();
  const double* gam = B.gamma;

  if (RN.lead_v) {
    if (threadIdx.x == 0) {
      const double sig = (RN.split == SPLIT_VTV ? 0.5 : 1.0) * gam[0] * RN.dt;
      sc[SC_SIG] = sig;
      sc[SC_SGH] = -sig / P.hbar;
    }
    if (threadIdx.x < D) sc[SC_QN + threadIdx.x] = sc[SC_Q + threadIdx.x];
    __syncthreads();
    build_v_short(P, SP, B, S.s);
    if (!grid_sync(B, &sflag)) return;
    load_v_short(P, SP, B, S);
    __syncthreads();
    short_pass<T, N, false>(P, SP, B, S, 0, SM_VONLY, 1);
    if (!grid_sync(B, &sflag)) return;
    finish(B, S.s, 1, D + 1);
    centre_after_potential(P, S.s, RN.motion);
    if (sc[SC_ERR] != 0.0) goto done;
    build_tables(P, B, S.s, TB_A);
    if (!grid_sync(B, &sflag)) return;
    load_tables(P, B, S.s, LT_A);
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
    // forward transform, group by group from the last axis; kinetic moments
    // in the pass over the group that holds axis 0
    for (int gi = 0; gi < ng; ++gi) {
      short_pass<T, N, false>(P, SP, B, S, gi, gi == ng - 1 ? SM_KIN : SM_NONE, 0);
      if (!grid_sync(B, &sflag)) return;
    }
    finish(B, S.s, 0, D + 1);
    centre_after_kinetic(P, S.s, RN.motion);
    if (sc[SC_ERR] != 0.0) goto done;
    build_tables(P, B, S.s, TB_K);
    if (hasv) build_v_short(P, SP, B, S.s);
    if (!grid_sync(B, &sflag)) return;
    load_tables(P, B, S.s, LT_K);
    if (hasv) load_v_short(P, SP, B, S);
    if (threadIdx.x < D) sc[SC_Q + threadIdx.x] = sc[SC_QN + threadIdx.x];
    __syncthreads();
    // inverse transform from the group of axis 0; the potential substep is
    // fused into the pass over the group that holds the last axis
    for (int gi = ng - 1; gi >= 0; --gi) {
      short_pass<T, N, true>(P, SP, B, S, gi, (gi == 0 && hasv) ? SM_V : SM_NONE, 1);
      if (gi > 0 && !grid_sync(B, &sflag)) return;
    }
    if (hasv) {
      if (!grid_sync(B, &sflag)) return;
      finish(B, S.s, 1, D + 1);
      centre_after_potential(P, S.s, RN.motion);
      if (sc[SC_ERR] != 0.0) goto done;
      build_tables(P, B, S.s, TB_A);
      if (!grid_sync(B, &sflag)) return;
      load_tables(P, B, S.s, LT_A);
      __syncthreads();
    }
  }
done:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int a = 0; a < D; ++a) {
      B.ctrl[a] = sc[SC_Q + a];
      B.ctrl[8 + a] = sc[SC_P + a];
    }
    if (sc[SC_ERR] != 0.0) atomicExch(B.status, (int)sc[SC_ERR]);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side lookup (C++ linkage, used by mg_capi.cu)
// ---------------------------------------------------------------------------

// The kernel for FP64 (prec 0) or FP32 (prec 1) storage and axis length n.
void* short_kernel(int prec, int n) {
  switch (n * 2 + prec) {
    case 16: return (void*)k_propagate_short<double, 8>;
    case 17: return (void*)k_propagate_short<float, 8>;
    case 24: return (void*)k_propagate_short<double, 12>;
    case 25: return (void*)k_propagate_short<float, 12>;
    case 32: return (void*)k_propagate_short<double, 16>;
    case 33: return (void*)k_propagate_short<float, 16>;
  }
  return nullptr;
}

int short_threads_for(int n) { return short_threads(n); }

}  // namespace mgk
