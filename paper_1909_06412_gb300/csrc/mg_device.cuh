// Device building blocks shared by the propagation kernels (mg_kernels.cu)
// and the reversible adjoint (mg_adjoint.cu): DFT codelets and the Stockham
// FFT in shared memory, bulk copies, the capped grid barrier, shared-memory
// layout, per-axis tables, potentials, reductions and the axis pass.  Every
// definition has internal linkage (one copy per translation unit).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_plan.h"

namespace mgk {
namespace {

template <typename T> struct VT;
template <> struct VT<double> { using v = double2; };
template <> struct VT<float> { using v = float2; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return V{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) { return V{a.x * s, a.y * s}; }
// multiply by s*i with s = +1 for the inverse and -1 for the forward transform
template <bool INV, typename V> __device__ __forceinline__ V mul_si(V a) {
  return INV ? V{-a.y, a.x} : V{a.y, -a.x};
}
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
template <typename V> __device__ __forceinline__ V from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

// ---------------------------------------------------------------------------
// DFT codelets of radix 2, 3, 4, 8; exponent sign -1 (forward) or +1 (inverse)
// ---------------------------------------------------------------------------

template <bool INV, int R, typename V> struct Dft;

template <bool INV, typename V> struct Dft<INV, 2, V> {
  static __device__ __forceinline__ void run(V* v) {
    V a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  }
};

// Irrational codelet constants are applied as hi + lo pairs: a rounded
// constant alone makes every butterfly non-unitary by the same ~1e-16, a bias
// that builds up linearly over thousands of transforms.
template <typename T> struct Split;
template <> struct Split<double> {
  static constexpr double r2h = 0.70710678118654757, r2l = -4.833646656726457e-17;  // 1/sqrt(2)
  static constexpr double r3h = 0.8660254037844386, r3l = 5.0175421109034514e-17;    // sqrt(3)/2
};
template <> struct Split<float> {
  static constexpr float r2h = 0.70710677f, r2l = 1.21016175e-08f;
  static constexpr float r3h = 0.86602539f, r3l = 1.55436251e-08f;
};
template <typename V, typename T> __device__ __forceinline__ V cscale2(V a, T hi, T lo) {
  return V{fma(a.x, hi, a.x * lo), fma(a.y, hi, a.y * lo)};
}

template <bool INV, typename V> struct Dft<INV, 3, V> {
  static __device__ __forceinline__ void run(V* v) {
    using T = decltype(v[0].x);
    V t = cadd(v[1], v[2]);
    V d = csub(v[1], v[2]);
    V m = V{v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y};
    V e = cscale2(mul_si<INV>(d), Split<T>::r3h, Split<T>::r3l);
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, e);
    v[2] = csub(m, e);
  }
};

template <bool INV, typename V> struct Dft<INV, 4, V> {
  static __device__ __forceinline__ void run(V* v) {
    V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    V t2 = cadd(v[1], v[3]), t3 = mul_si<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

// Radix 8 by one decimation-in-frequency split into two 4-point DFTs.
template <bool INV, typename V> struct Dft<INV, 8, V> {
  static __device__ __forceinline__ void run(V* v) {
    using T = decltype(v[0].x);
    V a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      a[r] = cadd(v[r], v[r + 4]);
      b[r] = csub(v[r], v[r + 4]);
    }
    b[1] = cscale2(cadd(b[1], mul_si<INV>(b[1])), Split<T>::r2h, Split<T>::r2l);  // * e^{s i pi/4}
    b[2] = mul_si<INV>(b[2]);                                                       // * e^{s i pi/2}
    b[3] = cscale2(csub(mul_si<INV>(b[3]), b[3]), Split<T>::r2h, Split<T>::r2l);  // * e^{3 s i pi/4}
    Dft<INV, 4, V>::run(a);
    Dft<INV, 4, V>::run(b);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      v[2 * r] = a[r];
      v[2 * r + 1] = b[r];
    }
  }
};

// ---------------------------------------------------------------------------
// Stockham FFT in shared memory
// ---------------------------------------------------------------------------

// Exact quotient x / d for 0 <= x < 2^16 and 1 <= d < 2^16 from m = ceil(2^32/d):
// floor(x m / 2^32) = floor(x/d + x e) with 0 <= x e < 2^-16 < 1/d, so the
// result never crosses the next integer.  Replaces runtime integer division
// in the index arithmetic of the passes.
struct Div16 {
  unsigned m;  // 0 encodes d = 1 (2^32 does not fit)
  __device__ __forceinline__ explicit Div16(unsigned d) : m(d > 1 ? 0xFFFFFFFFu / d + 1u : 0u) {}
  __device__ __forceinline__ unsigned operator()(unsigned x) const { return m ? __umulhi(x, m) : x; }
};

// One Stockham autosort pass of radix R over L lines of length n (in -> out).
// The first pass (Ns == 1) has no twiddles; it applies the diagonal
// pre-multiplier `pre` (A_l or K_l) to its inputs instead, if given.
// Tile layout: with wsh = 0 a line is n contiguous elements; with wsh > 0 the
// lines come in tiles of W = 2^wsh lines stored point-major (element p of line
// w of a tile at p*W + w), so a warp works on adjacent lines and adjacent
// shared-memory words.
template <bool INV, int R, typename V>
__device__ __forceinline__ void stockham_pass(const V* __restrict__ in, V* __restrict__ out, int n, int L,
                                              int Ns, const V* __restrict__ tw, const V* __restrict__ pre,
                                              int wsh) {
  const int nR = n / R;
  const int total = L * nR;
  const int ts = n / (Ns * R);
  const int W = 1 << wsh;
  const Div16 divL((unsigned)L), divnR((unsigned)nR), divNs((unsigned)Ns);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    int line, j, lbase, ps;
    if (wsh) {
      j = (int)divL((unsigned)b);
      line = b - j * L;
      lbase = (line >> wsh) * W * n + (line & (W - 1));
      ps = W;
    } else {
      line = (int)divnR((unsigned)b);
      j = b - line * nR;
      lbase = line * n;
      ps = 1;
    }
    const V* src = in + lbase;
    V* dst = out + lbase;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * nR) * ps];
    const int k = j - (int)divNs((unsigned)j) * Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const V w = tw[k * r * ts];
        v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
      }
    } else if (pre) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = cmul(v[r], pre[j + r * nR]);
    }
    Dft<INV, R, V>::run(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * ps] = v[r];
  }
}

// Full 1D transform of L lines; returns the buffer that holds the result.
template <bool INV, typename V>
__device__ V* stockham(V* in, V* out, int L, const AxisPlan& ax, const V* tw, const V* pre, int wsh) {
  int Ns = 1;
  for (int pi = 0; pi < ax.nrad; ++pi) {
    const int R = ax.rad[pi];
    const V* pm = pi == 0 ? pre : nullptr;
    if (R == 8) stockham_pass<INV, 8>(in, out, ax.n, L, Ns, tw, pm, wsh);
    else if (R == 4) stockham_pass<INV, 4>(in, out, ax.n, L, Ns, tw, pm, wsh);
    else if (R == 3) stockham_pass<INV, 3>(in, out, ax.n, L, Ns, tw, pm, wsh);
    else stockham_pass<INV, 2>(in, out, ax.n, L, Ns, tw, pm, wsh);
    __syncthreads();
    V* t = in;
    in = out;
    out = t;
    Ns *= R;
  }
  return in;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine) into shared memory with an mbarrier
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// global -> shared bulk copy; 16-byte aligned addresses, size a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// ---------------------------------------------------------------------------
// e^{i theta} by the table-driven method (Tang 1990): theta = k pi/128 + r with
// a Cody-Waite reduction (pi/128 split in three words), e^{i k pi/128} from a
// 256-entry table, and Taylor series of sin r, cos r for |r| <= pi/256
// (truncation below 1e-17).  About 17 FP64 instructions instead of ~27.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void expi_tab(double th, const double2* __restrict__ tab, double& s, double& c) {
  if (!(fabs(th) < 1e15)) {  // huge or non-finite argument: library routine
    sincos(th, &s, &c);
    return;
  }
  const long long ki = __double2ll_rn(th * 40.74366543152521);  // 128/pi
  const double k = (double)ki;
  double r = fma(-k, 0.02454369260617026, th);
  r = fma(-k, 9.567553118338697e-19, r);
  r = fma(-k, -2.3396639138424529e-35, r);
  const double2 t = tab[ki & 255];
  const double r2 = r * r;
  const double sr = fma(r2 * r, fma(r2, 1.0 / 120.0, -1.0 / 6.0), r);
  const double cr = fma(r2, fma(r2, fma(r2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  c = fma(t.x, cr, -t.y * sr);
  s = fma(t.y, cr, t.x * sr);
}

// ---------------------------------------------------------------------------
// Grid barrier with a time limit
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t BARRIER_LIMIT_NS = 5000000000ull;  // 5 s
constexpr unsigned BARRIER_MAX_SPINS = 400000000u;

// All CTAs of the (cooperative) grid must call this.  Returns false after a
// timeout (B.bar_limit_ns, else BARRIER_LIMIT_NS, or BARRIER_MAX_SPINS
// spins); the status word then holds ST_TIMEOUT.
//
// One 64-bit word holds the generation (high half) and the arrivals of the
// current generation (low half).  An arriving CTA adds 1 and learns the
// generation it arrived in from the returned value; the last arrival adds
// 2^32 - gridDim.x, which starts the next generation and zeroes the count in
// one atomic, and the others wait for the generation to change.  The count
// is back at zero after every completed barrier, so the word needs no reset
// between launches of any grid size.
__device__ bool grid_sync(const Bufs& B, int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* word = reinterpret_cast<unsigned long long*>(B.bar);
    __threadfence();
    const unsigned long long old = atomicAdd(word, 1ull);
    const unsigned g0 = (unsigned)(old >> 32);
    int ok = 1;
    if ((unsigned)old == gridDim.x - 1) {
      atomicAdd(word, (1ull << 32) - gridDim.x);
    } else {
      const uint64_t t0 = global_ns();
      const uint64_t limit = B.bar_limit_ns ? B.bar_limit_ns : BARRIER_LIMIT_NS;
      unsigned spins = 0;
      while ((unsigned)(ld_acquire_u64(word) >> 32) == g0) {
        if (spins > 64) __nanosleep(20);
        ++spins;
        if ((spins & 127u) == 0 && (global_ns() - t0 > limit || spins > BARRIER_MAX_SPINS)) {
          ok = 0;
          atomicExch(B.status, ST_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// ---------------------------------------------------------------------------
// Shared memory: every per-axis table of all axes, the scalar state of the
// grid centres, reduction scratch and two data regions.
// ---------------------------------------------------------------------------

// scalar slots (doubles) in Smem::sc
enum { SC_Q = 0, SC_P = 8, SC_QN = 16, SC_DELTA = 24, SC_TAU = 32, SC_SIG = 33, SC_SGH = 34, SC_HASV = 35,
       SC_ERR = 36, SC_MOM = 64, SC_N = SCALARS };

template <typename V> struct Smem {
  V* tw;        // twiddles, all axes (tab_total)
  V* tA;        // A_l
  V* tAi;       // conj(A_l)/N_l
  V* tK;        // kinetic multiplier
  double* tv;   // NVCOL * tab_total potential columns
  double* tc;   // k - N/2
  double* te;   // kinetic energy per axis entry
  double2* sct; // 256-entry e^{i k pi/128}
  double* red;  // THREADS * (D+2) per-thread partials
  double* fin;  // PSTRIDE finished sums
  double* sc;   // SC_N scalars
  V* reg[3];    // data regions (the third only for HBM-streamed passes)
  uint64_t* mbar; // one mbarrier per data region
  unsigned* mphase; // their phase bits, carried from one streamed pass to the next
  int64_t* tb;  // element offset of each tile of the current chunk
  uint16_t* li; // multi-index of each line of the current chunk (D per line)
  size_t end;   // bytes used
};

template <typename V> __device__ Smem<V> carve(const Plan& P, const Bufs& B, unsigned char* base) {
  Smem<V> s;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += (bytes + 15) & ~size_t(15);
    return p;
  };
  const int TT = P.tab_total;
  s.tw = (V*)take(sizeof(V) * TT);
  if (P.tab_global & TG_MULT) {
    // FP64 only (V = double2): the workspace tables themselves
    s.tA = (V*)B.tabA;
    s.tAi = (V*)B.tabAi;
    s.tK = (V*)B.tabK;
  } else {
    s.tA = (V*)take(sizeof(V) * TT);
    s.tAi = (V*)take(sizeof(V) * TT);
    s.tK = (V*)take(sizeof(V) * TT);
  }
  if (P.tab_global & TG_COLS) {
    s.tv = B.tabV;
    s.tc = B.tabC;
    s.te = B.tabE;
  } else {
    s.tv = (double*)take(sizeof(double) * NVCOL * TT);
    s.tc = (double*)take(sizeof(double) * TT);
    s.te = (double*)take(sizeof(double) * TT);
  }
  s.sct = (double2*)take(sizeof(double2) * 256);
  s.red = (double*)take(sizeof(double) * THREADS * (3 * P.D + 5));
  s.fin = (double*)take(sizeof(double) * PSTRIDE);
  s.sc = (double*)take(sizeof(double) * SC_N);
  s.reg[0] = (V*)take(P.region_bytes);
  s.reg[1] = (V*)take(P.region_bytes);
  s.reg[2] = P.resident ? nullptr : (V*)take(P.region_bytes);
  s.mbar = (uint64_t*)take(sizeof(uint64_t) * 3);
  s.mphase = (unsigned*)take(sizeof(unsigned) * 4);
  s.tb = (int64_t*)take(sizeof(int64_t) * P.max_tiles);
  s.li = (uint16_t*)take(sizeof(uint16_t) * P.max_lines * P.D);
  s.end = off;
  return s;
}

enum { LT_TW = 1, LT_A = 2, LT_K = 4, LT_V = 8, LT_C = 16, LT_E = 32, LT_SCT = 64 };

// Copy tables from global memory (written by other CTAs) into shared memory.
template <typename V> __device__ void load_tables(const Plan& P, const Bufs& B, const Smem<V>& S, int what) {
  const int TT = P.tab_total;
  // tables kept in the workspace are read there (after the grid barrier that
  // follows their build, like every other global value)
  if (P.tab_global & TG_MULT) what &= ~(LT_A | LT_K);
  if (P.tab_global & TG_COLS) what &= ~(LT_V | LT_C | LT_E);
  // every load of an entry is issued before its shared-memory stores, so that
  // the L2 round trips of an entry overlap instead of following one another
  for (int e = threadIdx.x; e < TT; e += blockDim.x) {
    double2 tw, a, ai, k;
    double v[NVCOL], cc, ee;
    if (what & LT_TW) tw = __ldcg(B.tw + e);
    if (what & LT_A) {
      a = __ldcg(B.tabA + e);
      ai = __ldcg(B.tabAi + e);
    }
    if (what & LT_K) k = __ldcg(B.tabK + e);
    if (what & LT_V) {
#pragma unroll
      for (int c = 0; c < NVCOL; ++c) v[c] = __ldcg(B.tabV + c * TT + e);
    }
    if (what & LT_C) cc = __ldcg(B.tabC + e);
    if (what & LT_E) ee = __ldcg(B.tabE + e);
    if (what & LT_TW) S.tw[e] = from_d2<V>(tw);
    if (what & LT_A) {
      S.tA[e] = from_d2<V>(a);
      S.tAi[e] = from_d2<V>(ai);
    }
    if (what & LT_K) S.tK[e] = from_d2<V>(k);
    if (what & LT_V) {
#pragma unroll
      for (int c = 0; c < NVCOL; ++c) S.tv[c * TT + e] = v[c];
    }
    if (what & LT_C) S.tc[e] = cc;
    if (what & LT_E) S.te[e] = ee;
  }
  if (what & LT_SCT)
    for (int e = threadIdx.x; e < 256; e += blockDim.x) S.sct[e] = __ldcg(B.sct + e);
}

// ---------------------------------------------------------------------------
// Potentials: V (as a phase -sigma V / hbar, folded into the tables) and grad V
// ---------------------------------------------------------------------------

// Per-point evaluation from per-axis tables.  th = -sigma V / hbar (or V
// itself when the tables were built with scale 1), g = grad V.
template <int KIND, int DM = MAXD>
__device__ __forceinline__ void vpoint(const Plan& P, const double* tv, const int* idx, double sgh,
                                       double& th, double* g) {
  const int TT = P.tab_total;
  const int D = P.D;
#define COL(c, a) tv[(c) * TT + P.ax[a].toff + idx[a]]
  if (KIND == POT_HARMONIC) {
    if (!P.pot_general) {
      th = 0;
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < D) {
          th += COL(0, a);
          g[a] = COL(1, a);
        }
    } else {
      double d[DM];
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < D) d[a] = COL(0, a);
      double v = 0;
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < D) {
          double s = 0;
#pragma unroll
          for (int b = 0; b < DM; ++b)
            if (b < D) s += P.pot[a * D + b] * d[b];
          g[a] = s;
          v += d[a] * s;
        }
      th = 0.5 * sgh * v;
    }
  } else if (KIND == POT_ATOM_DIATOM) {
    const double gR = COL(0, 0), dgR = COL(1, 0), sgR = COL(2, 0);
    const double sf = COL(0, 1), df = COL(1, 1), h = COL(2, 1), dh = COL(3, 1);
    th = fma(sgR, h, sf);
    g[0] = dgR * h;
    g[1] = fma(gR, dh, df);
  } else if (KIND == POT_HENON_HEILES) {
    const double lam = P.pot[0];
    double x[DM], x2[DM];
    double s1 = 0, cpl = 0;
#pragma unroll
    for (int a = 0; a < DM; ++a)
      if (a < D) {
        x[a] = COL(0, a);
        x2[a] = COL(2, a);
        s1 += COL(1, a);
        g[a] = COL(3, a);
      }
#pragma unroll
    for (int a = 0; a + 1 < DM; ++a)
      if (a + 1 < D) {
        cpl = fma(x2[a], x[a + 1], cpl);
        g[a] = fma(2.0 * lam * x[a], x[a + 1], g[a]);
        g[a + 1] = fma(lam, x2[a], g[a + 1]);
      }
    th = fma(sgh * lam, cpl, s1);
  } else {  // POT_SECREST_JOHNSON
    const double c = COL(0, 1);
    th = fma(COL(2, 0), c, COL(0, 0));
    const double e = COL(3, 0) * c;
    g[0] = COL(1, 0) + e;
    g[1] = -e;
  }
#undef COL
}

// Potential columns of one table entry (axis a, coordinate x).
// Part 0 of the columns (0, 1 and 4) or part 1 (2 and 3): the two halves
// of the evaluation, each with at most half of the exponentials, so that the
// distributed table build can give them to different warps.
__device__ void vcolumns_part(const Plan& P, int a, double x, double sgh, int part, double* c) {
  if (part == 0) {
    c[0] = c[1] = c[4] = 0.0;
  } else {
    c[2] = c[3] = 0.0;
  }
  if (P.pot_kind == POT_HARMONIC) {
    if (part) return;
    const double d = x - P.pot[P.D * P.D + a];
    if (!P.pot_general) {
      const double k = P.pot[a * P.D + a];
      c[0] = sgh * 0.5 * k * d * d;
      c[1] = k * d;
    } else {
      c[0] = d;
    }
  } else if (P.pot_kind == POT_ATOM_DIATOM) {
    const double Dm = P.pot[0], aa = P.pot[1], re = P.pot[2], A = P.pot[3], be = P.pot[4];
    if (a == 0) {
      const double g = A * exp(-be * x);
      if (part == 0) {
        c[0] = g;
        c[1] = -be * g;
      } else {
        c[2] = sgh * g;
      }
    } else if (part == 0) {
      const double em = exp(-aa * (x - re));
      c[0] = sgh * Dm * (1.0 - em) * (1.0 - em);
      c[1] = 2.0 * Dm * (1.0 - em) * aa * em;
    } else {
      const double ep = exp(0.5 * be * x), en = exp(-0.5 * be * x);
      c[2] = ep + en;
      c[3] = 0.5 * be * (ep - en);
    }
  } else if (P.pot_kind == POT_HENON_HEILES) {
    const double lam = P.pot[0];
    if (part == 0) {
      c[0] = x;
      c[1] = sgh * (0.5 * x * x - (a >= 1 ? lam * x * x * x / 3.0 : 0.0));
    } else {
      c[2] = x * x;
      c[3] = x - (a >= 1 ? lam * x * x : 0.0);
    }
  } else {  // SECREST_JOHNSON
    const double Dm = P.pot[0], be = P.pot[1], al = P.pot[2];
    if (a == 0) {
      if (part == 0) {
        const double e1 = exp(-be * x);
        c[0] = sgh * Dm * (1.0 - e1) * (1.0 - e1);
        c[1] = 2.0 * Dm * (1.0 - e1) * be * e1;
      } else {
        const double ea = exp(al * x);
        c[2] = sgh * ea;
        c[3] = al * ea;
      }
    } else if (part == 0) {
      c[0] = exp(-al * x);
    }
  }
}
__device__ void vcolumns_eval(const Plan& P, int a, double x, double sgh, double* c) {
  vcolumns_part(P, a, x, sgh, 0, c);
  vcolumns_part(P, a, x, sgh, 1, c);
}
__device__ void vcolumns(const Plan& P, const Bufs& B, int e, int a, double x, double sgh, int part) {
  const int TT = P.tab_total;
  double c[NVCOL];
  vcolumns_part(P, a, x, sgh, part, c);
  if (part == 0) {
    __stcg(B.tabV + e, c[0]);
    __stcg(B.tabV + TT + e, c[1]);
    __stcg(B.tabV + 4 * TT + e, c[4]);
  } else {
    __stcg(B.tabV + 2 * TT + e, c[2]);
    __stcg(B.tabV + 3 * TT + e, c[3]);
  }
}

enum { TB_K = 1, TB_V = 2, TB_A = 4, TB_E = 8, TB_V1 = 16 /* second half of TB_V, build_tables only */ };

// e^{i theta} for a table entry: FP64 for FP64 storage; for FP32 storage the
// FP64 argument is reduced modulo 2 pi in FP64 and the sine and cosine are
// taken in FP32 (the entry is rounded to FP32 anyway).
__device__ __forceinline__ void expi_prec(int prec, double th, const double2* tab, double& s, double& c) {
  if (!prec) {
    expi_tab(th, tab, s, c);
    return;
  }
  const double kk = rint(th * 0.15915494309189535);
  double r = fma(-kk, 6.283185307179586, th);
  r = fma(-kk, 2.4492935982947064e-16, r);
  float sf, cf;
  sincosf((float)r, &sf, &cf);
  s = sf;
  c = cf;
}

// For FP32 storage: of the four float pairs that bracket (x, y), the one whose
// squared modulus is closest to m2.  Plain rounding leaves |w|^2 - 1 at ~1e-7
// with a fixed sign per entry, a bias that a table reused by every transform
// turns into a steady norm drift; this choice keeps each multiplier unitary to
// ~1e-9 while staying within one float ulp of the exact value.
__device__ double2 round_unit_f32(double x, double y, double m2) {
  const float xf = (float)x, yf = (float)y;
  const float xs[2] = {xf, (double)xf < x ? nextafterf(xf, INFINITY) : nextafterf(xf, -INFINITY)};
  const float ys[2] = {yf, (double)yf < y ? nextafterf(yf, INFINITY) : nextafterf(yf, -INFINITY)};
  double best = INFINITY;
  double2 r = make_double2(xf, yf);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const double e = fabs(fma((double)xs[a], (double)xs[a], (double)ys[b] * (double)ys[b]) - m2);
      if (e < best) {
        best = e;
        r = make_double2(xs[a], ys[b]);
      }
    }
  return r;
}

// Distributed construction of the per-axis tables.  The work is cut into
// tasks of 32 consecutive entries of one table, one task per warp with every
// lane busy (an FP64 warp instruction costs the same with 1 or 32 lanes), and
// the tasks are dealt out first to warp 0 of every CTA, then to warp 1, ...
// so that they run on as many SM sub-partitions as possible at once.  Inputs
// (tau, delta, p, q, sgh) come from the CTA's scalar slots.  A grid barrier
// must follow before the tables are used.
// Table entries of axis a, index j (c = j - N_a/2), from the CTA's scalars.
// Kinetic factor K_a[j] = e^{(i/hbar)(delta_a p^K - tau minv_a (p^K)^2 / 2)}.
// Exact 2^-k for n = 2^k (else 0): built from the exponent bits, no division.
__device__ __forceinline__ double exact_inv_pow2(int n) {
  if (n <= 0 || (n & (n - 1))) return 0.0;
  return __hiloint2double((1023 - (31 - __clz(n))) << 20, 0);
}
// x / hbar, skipping the division (an FP64 subroutine on the critical path of
// the table builds) when hbar = 1, where it is the identity.
__device__ __forceinline__ double over_hbar(const Plan& P, double x) { return P.hbar == 1.0 ? x : x / P.hbar; }

__device__ __forceinline__ double2 kin_entry(const Plan& P, const double* sc, const double2* sct, int a, double c) {
  const double pk = fma(c, P.dp[a], sc[SC_P + a]);
  const double th = over_hbar(P, sc[SC_DELTA + a] * pk - 0.5 * sc[SC_TAU] * P.minv[a] * pk * pk);
  double sn, cs;
  expi_prec(P.prec, th, sct, sn, cs);
  return P.prec ? round_unit_f32(cs, sn, 1.0) : make_double2(cs, sn);
}
// Demodulation A_a[j] = (-1)^j e^{-i p_a c dq_a / hbar} and conj(A_a[j]) / N_a.
__device__ __forceinline__ void demod_entry(const Plan& P, const double* sc, const double2* sct, int a, int j,
                                            double c, double2& A, double2& Ai) {
  const int n = P.ax[a].n;
  const double th = over_hbar(P, -sc[SC_P + a] * c * P.dq[a]);
  double sn, cs;
  expi_prec(P.prec, th, sct, sn, cs);
  const double sg = (j & 1) ? -1.0 : 1.0;
  // conj(A)/N by division: a rounded 1/N would bias every inverse transform.
  // For N = 2^k the product with the exact 2^-k is the same number.
  const double r = exact_inv_pow2(n);
  double ax, ay;
  if (r != 0.0) {
    ax = sg * cs * r;
    ay = -sg * sn * r;
  } else {
    ax = sg * cs / (double)n;
    ay = -sg * sn / (double)n;
  }
  if (P.prec) {
    A = round_unit_f32(sg * cs, sg * sn, 1.0);
    const double inv = 1.0 / ((double)n * (double)n);
    Ai = round_unit_f32(ax, ay, inv);
  } else {
    A = make_double2(sg * cs, sg * sn);
    Ai = make_double2(ax, ay);
  }
}

template <typename V> __device__ void build_tables(const Plan& P, const Bufs& B, const Smem<V>& S, int what) {
  const int TT = P.tab_total, D = P.D;
  const int nch = (TT + 31) / 32;
  int kinds[5], nk = 0;
  if (what & TB_V) {  // the longest tasks first
    kinds[nk++] = TB_V;
    kinds[nk++] = TB_V1;
  }
  if (what & TB_K) kinds[nk++] = TB_K;
  if (what & TB_A) kinds[nk++] = TB_A;
  if (what & TB_E) kinds[nk++] = TB_E;
  const int ntask = nk * nch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int t = warp * gridDim.x + blockIdx.x; t < ntask; t += nwarps * gridDim.x) {
    const int kind = kinds[t / nch];
    const int e = (t % nch) * 32 + lane;
    if (e >= TT) continue;
    int a = 0;
    while (a + 1 < D && e >= P.ax[a + 1].toff) ++a;
    const int j = e - P.ax[a].toff;
    const int n = P.ax[a].n;
    const double c = (double)(j - n / 2);
    const double* sc = S.sc;
    if (kind == TB_K) {
      __stcg(B.tabK + e, kin_entry(P, sc, S.sct, a, c));
    } else if (kind == TB_A) {
      double2 A, Ai;
      demod_entry(P, sc, S.sct, a, j, c, A, Ai);
      __stcg(B.tabA + e, A);
      __stcg(B.tabAi + e, Ai);
    } else if (kind == TB_V || kind == TB_V1) {
      vcolumns(P, B, e, a, fma(c, P.dq[a], sc[SC_QN + a]), sc[SC_SGH], kind == TB_V1);
    } else {
      const double pk = fma(c, P.dp[a], sc[SC_P + a]);
      __stcg(B.tabE + e, 0.5 * P.minv[a] * pk * pk);
    }
  }
}

// The same tables built by one CTA for itself, straight into its shared
// memory (grids small enough for a few CTAs; no barrier needed across CTAs).
// Tasks of 32 entries are dealt out over the CTA's warps.
template <typename V> __device__ void build_tables_local(const Plan& P, const Smem<V>& S, int what) {
  const int TT = P.tab_total, D = P.D;
  const int nch = (TT + 31) / 32;
  int kinds[3], nk = 0;
  if (what & TB_K) kinds[nk++] = TB_K;
  if (what & TB_V) kinds[nk++] = TB_V;
  if (what & TB_A) kinds[nk++] = TB_A;
  const int ntask = nk * nch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int t = warp; t < ntask; t += nwarps) {
    const int kind = kinds[t / nch];
    const int e = (t % nch) * 32 + lane;
    if (e >= TT) continue;
    int a = 0;
    while (a + 1 < D && e >= P.ax[a + 1].toff) ++a;
    const int j = e - P.ax[a].toff;
    const double c = (double)(j - P.ax[a].n / 2);
    const double* sc = S.sc;
    if (kind == TB_K) {
      S.tK[e] = from_d2<V>(kin_entry(P, sc, S.sct, a, c));
    } else if (kind == TB_A) {
      double2 A, Ai;
      demod_entry(P, sc, S.sct, a, j, c, A, Ai);
      S.tA[e] = from_d2<V>(A);
      S.tAi[e] = from_d2<V>(Ai);
    } else {
      double cv[NVCOL];
      vcolumns_eval(P, a, fma(c, P.dq[a], sc[SC_QN + a]), sc[SC_SGH], cv);
#pragma unroll
      for (int k = 0; k < NVCOL; ++k) S.tv[k * TT + e] = cv[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Reductions: deterministic per-CTA partials, then a fixed-order finish
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Per-thread partials -> one record per CTA.  The per-thread values go
// through shared memory so that warp v sums value v (8 partials per lane, then
// a shuffle tree): nv short FP64 chains on different sub-partitions instead of
// nv * 8 warps of shuffle trees.
// The record goes to `rec` (shared memory, read by the other CTAs of a
// cluster) or, when rec is null, to the grid's per-CTA slot in global memory.
template <typename V, int DM = MAXD>
__device__ void block_partials(const Bufs& B, const Smem<V>& S, int slot, const double* acc, int nv,
                               double* rec = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nt = blockDim.x;
#pragma unroll
  for (int v = 0; v < DM + 2; ++v)
    if (v < nv) S.red[v * nt + threadIdx.x] = acc[v];
  __syncthreads();
  for (int v = warp; v < nv; v += nt >> 5) {
    double s = 0;
    for (int k = lane; k < nt; k += 32) s += S.red[v * nt + k];
    s = warp_sum(s);
    if (lane == 0) {
      if (rec) rec[v] = s;
      else __stcg(B.part + ((size_t)slot * gridDim.x + blockIdx.x) * PSTRIDE + v, s);
    }
  }
  __syncthreads();
}

// Sum the per-CTA partials of `slot` in a fixed order; result in S.fin.
template <typename V> __device__ void finish(const Bufs& B, const Smem<V>& S, int slot, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = (int)gridDim.x;
  for (int v = warp; v < nv; v += blockDim.x >> 5) {
    const double* pv = B.part + (size_t)slot * G * PSTRIDE + v;
    double s = 0;
    int b = lane;
    // four loads in flight, added in the same (increasing b) order
    for (; b + 96 < G; b += 128) {
      const double x0 = __ldcg(pv + (size_t)b * PSTRIDE), x1 = __ldcg(pv + (size_t)(b + 32) * PSTRIDE);
      const double x2 = __ldcg(pv + (size_t)(b + 64) * PSTRIDE), x3 = __ldcg(pv + (size_t)(b + 96) * PSTRIDE);
      s += x0;
      s += x1;
      s += x2;
      s += x3;
    }
    for (; b < G; b += 32) s += __ldcg(pv + (size_t)b * PSTRIDE);
    s = warp_sum(s);
    if (lane == 0) S.fin[v] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One pass along one axis
// ---------------------------------------------------------------------------

enum { PRE_NONE = 0, PRE_A = 1, PRE_K = 2 };
enum { RED_NONE = 0, RED_KIN = 1, RED_V = 2, RED_OBS_KIN = 3, RED_OBS_V = 4 };

struct PassArgs {
  int l;
  int from_smem;  // input already in smem region `res_in` (single chunk)
  int keep;       // leave the result in smem (single chunk), no global store
  int fft;        // apply the 1D transform
  int pre, post;  // multipliers (post: conj(A)/N)
  int red;        // fused reduction / potential phase
  int slot;       // partial-sum slot
  const void* src;
  void* dst;
  // position in the team of CTAs sharing the grid (default: the whole launch)
  // and, for teams smaller than the launch, the shared-memory reduction record
  int64_t bid = 0, nb = 0;
  double* rec = nullptr;
};

// sum_{a<b} minv_ab p_a p_b at the p-grid point of multi-index idx (the
// off-diagonal part of T(p^K) = p^T m^-1 p / 2, eq:KE_operator).
template <int DM>
__device__ __forceinline__ double kinetic_cross(const Plan& P, const double* tc, const double* sc, const int* idx) {
  double pk[DM];
#pragma unroll
  for (int a = 0; a < DM; ++a)
    if (a < P.D) pk[a] = fma(tc[P.ax[a].toff + idx[a]], P.dp[a], sc[SC_P + a]);
  double e = 0.0;
#pragma unroll
  for (int a = 0; a < DM; ++a)
#pragma unroll
    for (int b = a + 1; b < DM; ++b)
      if (b < P.D) e = fma(P.minvf[a * P.D + b] * pk[a], pk[b], e);
  return e;
}

// s + c += x with Knuth's error-free two-sum (FP32).
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// Multi-index of element j of line (o, i) of axis l.
__device__ __forceinline__ void decode(const Plan& P, int l, unsigned o, unsigned i, int j, int* idx) {
  for (int a = l - 1; a >= 0; --a) {
    const unsigned n = (unsigned)P.N[a];
    idx[a] = (int)(o % n);
    o /= n;
  }
  for (int a = P.D - 1; a > l; --a) {
    const unsigned n = (unsigned)P.N[a];
    idx[a] = (int)(i % n);
    i /= n;
  }
  idx[l] = j;
}

// Queue the bulk copies of chunk (tiles c0 .. c0+nt-1 of this CTA) into region
// `reg`, completing on `bar`.  Called by warp 0 only.  A strided tile is n
// rows of W contiguous elements (one copy per row); a contiguous-axis tile is
// one line of n elements (one copy).
template <typename V>
__device__ void issue_chunk(const AxisPlan& ax, bool contig, const V* src, int64_t c0, int nt, V* reg,
                            uint64_t* bar, int64_t bid, int64_t nb) {
  const int lane = threadIdx.x & 31;
  const int n = ax.n, W = ax.W;
  const int64_t s = ax.stride, tpo = contig ? 1 : ax.stride / W;
  const unsigned rowbytes = (unsigned)((contig ? W * n : W) * sizeof(V));
  const int rows = contig ? nt : nt * n;
  fence_proxy_async();  // earlier generic accesses to `reg` before the async writes
  if (lane == 0) mbar_expect_tx(bar, (unsigned)rows * rowbytes);
  __syncwarp();
  for (int r = lane; r < rows; r += 32) {
    const int ti = contig ? r : r / n;
    const int j = contig ? 0 : r - ti * n;
    const int64_t t = bid + (c0 + ti) * nb;
    const int64_t o = t / tpo;
    const int64_t base = contig ? t * W * n : o * n * s + (t - o * tpo) * W + (int64_t)j * s;
    bulk_load(reg + (contig ? ti * W * n : ti * W * n + j * W), src + base, rowbytes, bar);
  }
}

// Wait for a region's bulk copies (every thread).  Bounded by time (the
// barrier limit) and by a spin count; a timeout is recorded in the status word.
__device__ __forceinline__ void wait_region(const Bufs& B, uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return;
  const uint64_t t0 = global_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++spins;
    if ((spins & 63u) == 0 && (global_ns() - t0 > BARRIER_LIMIT_NS || spins > BARRIER_MAX_SPINS)) {
      if (threadIdx.x == 0) atomicExch(B.status, ST_TIMEOUT);
      break;
    }
  }
}

template <typename T, bool INV, int KIND, int DM = MAXD>
__device__ int axis_pass(const Plan& P, const Bufs& B, const PassArgs& A, const Smem<typename VT<T>::v>& S,
                         int res_in) {
  using V = typename VT<T>::v;
  const AxisPlan& ax = P.ax[A.l];
  const int n = ax.n, W = ax.W, D = P.D;
  const bool contig = (A.l == D - 1);
  const int wsh = contig ? 0 : __ffs(W) - 1;   // W is a power of two
  const int64_t s = ax.stride;
  const int64_t tpo = contig ? 1 : s / W;  // tiles per outer index
  const int64_t ws = contig ? n : 1;       // element step between lines of a tile
  const int64_t es = contig ? 1 : s;       // element step along the axis
  const V* tw = S.tw + ax.toff;
  const V* pre = A.pre == PRE_A ? S.tA + ax.toff : (A.pre == PRE_K ? S.tK + ax.toff : nullptr);
  const V* post = A.post ? S.tAi + ax.toff : nullptr;
  const double sgh = S.sc[SC_SGH];

  double acc[DM + 2];
#pragma unroll
  for (int v = 0; v < DM + 2; ++v) acc[v] = 0;
  // FP32 storage: the kinetic moments are summed per thread in FP32 with an
  // error-free two-sum (sum + compensation), so the per-thread partials are
  // accurate to ~1e-14 without an FP64 instruction per point.
  float ks[DM + 1], kc[DM + 1];
#pragma unroll
  for (int v = 0; v < DM + 1; ++v) ks[v] = kc[v] = 0.f;

  const int64_t bid = A.nb ? A.bid : (int64_t)blockIdx.x, nb = A.nb ? A.nb : (int64_t)gridDim.x;
  const int64_t mine = bid < ax.ntiles ? (ax.ntiles - bid + nb - 1) / nb : 0;
  const V* src = (const V*)A.src;
  V* dst = (V*)A.dst;
  int res = -1;
  const int chunk = A.from_smem || A.keep ? (int)mine : ax.tpc;
  // HBM-streamed passes: chunk k+1 is copied by the TMA engine into a third
  // region while chunk k is transformed and written back.
  const bool stream = !P.resident && !A.from_smem && !A.keep && mine > 0;
  int rd = 0, rt = 1, rf = 2;  // data, temporary and prefetch regions
  unsigned parity = 0;          // one phase bit per region
  if (stream) {
    parity = *S.mphase;
    if (threadIdx.x < 32)
      issue_chunk(ax, contig, src, 0, (int)(mine < chunk ? mine : chunk), S.reg[rd], S.mbar + rd, bid, nb);
  }
  for (int64_t c0 = 0; c0 < mine; c0 += chunk) {
    const int nt = (int)(mine - c0 < chunk ? mine - c0 : chunk);
    const int cnt = nt * W * n;
    if (stream && c0 + chunk < mine && threadIdx.x < 32) {
      const int64_t c1 = c0 + chunk;
      issue_chunk(ax, contig, src, c1, (int)(mine - c1 < chunk ? mine - c1 : chunk), S.reg[rf], S.mbar + rf, bid,
                  nb);
    }
    // per-tile offsets (one 64-bit division per tile, not per element) and,
    // for the fused reductions, the multi-index of every line of the chunk
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      const int64_t t = bid + (c0 + k) * nb;
      const int64_t o = t / tpo;
      S.tb[k] = contig ? t * W * n : o * n * s + (t - o * tpo) * W;
    }
    if (A.red != RED_NONE) {
      for (int kw = threadIdx.x; kw < nt * W; kw += blockDim.x) {
        const int k = kw / W, w = kw - k * W;
        const int64_t t = bid + (c0 + k) * nb;
        const int64_t o = t / tpo;
        int idx[DM];
        const unsigned lo = contig ? (unsigned)(t * W + w) : (unsigned)o;
        const unsigned li = contig ? 0u : (unsigned)((t - o * tpo) * W + w);
        decode(P, A.l, lo, li, 0, idx);
        for (int a = 0; a < D; ++a) S.li[kw * D + a] = (uint16_t)idx[a];
      }
    }
    V* cur;
    V* oth;
    if (A.from_smem) {
      cur = S.reg[res_in];
      oth = S.reg[res_in ^ 1];
    } else if (stream) {
      wait_region(B, S.mbar + rd, (parity >> rd) & 1u);
      parity ^= 1u << rd;
      cur = S.reg[rd];
      oth = S.reg[rt];
    } else {
      // up to LOADS independent global loads in flight per thread before the
      // shared-memory stores (one L2 round trip instead of one per element)
      constexpr int LOADS = 8;
      __syncthreads();  // S.tb ready
      cur = S.reg[0];
      oth = S.reg[1];
      const Div16 divWn((unsigned)(W * n)), divn((unsigned)n);
      for (int e0 = threadIdx.x; e0 < cnt; e0 += LOADS * blockDim.x) {
        V vals[LOADS];
#pragma unroll
        for (int u = 0; u < LOADS; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < cnt) {
            const int ti = (int)divWn((unsigned)e);
            const int rem = e - ti * W * n;
            const int w = contig ? (int)divn((unsigned)rem) : rem & (W - 1);
            const int j = contig ? rem - w * n : rem >> wsh;
            vals[u] = __ldcg(src + S.tb[ti] + j * es + w * ws);
          }
        }
#pragma unroll
        for (int u = 0; u < LOADS; ++u) {
          const int e = e0 + u * blockDim.x;
          if (e < cnt) cur[e] = vals[u];
        }
      }
    }
    __syncthreads();
    if (A.fft) {
      cur = stockham<INV>(cur, oth, nt * W, ax, tw, pre, wsh);
    } else if (pre) {
      for (int e = threadIdx.x; e < cnt; e += blockDim.x)
        cur[e] = cmul(cur[e], pre[contig ? e % n : (e % (W * n)) >> wsh]);
      __syncthreads();
    }

    // epilogue: element e of the chunk is tile ti, point j, line w
    const Div16 divWn((unsigned)(W * n)), divn((unsigned)n);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int ti = (int)divWn((unsigned)e);
      const int rem = e - ti * W * n;
      const int w = contig ? (int)divn((unsigned)rem) : rem & (W - 1);
      const int j = contig ? rem - w * n : rem >> wsh;
      V v = cur[e];
      if (post) v = cmul(v, post[j]);
      if (A.red != RED_NONE) {
        int idx[DM];
#pragma unroll
        for (int a = 0; a < DM; ++a)
          if (a < D) idx[a] = S.li[(ti * W + w) * D + a];
        idx[A.l] = j;
        // |value|^2: FP64 for FP64 storage; FP32 product, FP64 accumulation otherwise
        bool handled = false;
        if constexpr (sizeof(T) == 4) {
          if (A.red == RED_KIN) {
            const float w2f = fmaf(v.x, v.x, v.y * v.y);
            two_sum_acc(ks[0], kc[0], w2f);
#pragma unroll
            for (int a = 0; a < DM; ++a)
              if (a < D) two_sum_acc(ks[1 + a], kc[1 + a], (float)(idx[a] - (P.ax[a].n >> 1)) * w2f);
            handled = true;
          }
        }
        if (!handled) {
          double w2;
          if constexpr (sizeof(T) == 8) w2 = fma((double)v.x, (double)v.x, (double)v.y * (double)v.y);
          else w2 = (double)fmaf(v.x, v.x, v.y * v.y);
          acc[0] += w2;
          if (A.red == RED_KIN || A.red == RED_OBS_KIN) {
            double te = 0;
#pragma unroll
            for (int a = 0; a < DM; ++a)
              if (a < D) {
                acc[1 + a] = fma(S.tc[P.ax[a].toff + idx[a]], w2, acc[1 + a]);
                if (A.red == RED_OBS_KIN) te += S.te[P.ax[a].toff + idx[a]];
              }
            if (A.red == RED_OBS_KIN && P.minv_general) te += kinetic_cross<DM>(P, S.tc, S.sc, idx);
            if (A.red == RED_OBS_KIN) acc[D + 1] = fma(te, w2, acc[D + 1]);
          } else {
            double th, g[DM];
            vpoint<KIND, DM>(P, S.tv, idx, sgh, th, g);
            if (A.red == RED_V) {
#pragma unroll
              for (int a = 0; a < DM; ++a)
                if (a < D) acc[1 + a] = fma(g[a], w2, acc[1 + a]);
              if constexpr (sizeof(T) == 8) {
                double sn, cs;
                expi_tab(th, S.sct, sn, cs);
                v = V{fma(v.x, cs, -v.y * sn), fma(v.x, sn, v.y * cs)};
              } else {
                // FP64 phase argument reduced modulo 2 pi (two-word 2 pi), then
                // FP32 sine and cosine of the reduced angle (|r| <= pi)
                const double kk = rint(th * 0.15915494309189535);
                double r = fma(-kk, 6.283185307179586, th);
                r = fma(-kk, 2.4492935982947064e-16, r);
                float sn, cs;
                sincosf((float)r, &sn, &cs);
                v = V{fmaf(v.x, cs, -v.y * sn), fmaf(v.x, sn, v.y * cs)};
              }
            } else {  // observables: <x> and <V>
#pragma unroll
              for (int a = 0; a < DM; ++a)
                if (a < D)
                  acc[1 + a] = fma(fma(S.tc[P.ax[a].toff + idx[a]], P.dq[a], S.sc[SC_Q + a]), w2, acc[1 + a]);
              acc[D + 1] = fma(th, w2, acc[D + 1]);
            }
          }
        }
      }
      if (A.red == RED_KIN && P.minv_general) {
        // the non-separable part of the kinetic phase e^{-i tau T(p^K)/hbar}
        // (eq:U_T_tensor, T = p^T m^-1 p / 2): e^{-i tau sum_{a<b} minv_ab p_a p_b / hbar},
        // applied while the state is in p-representation; the separable part
        // and the grid shift are in the per-axis tables of the inverse passes
        int idx[DM];
#pragma unroll
        for (int a = 0; a < DM; ++a)
          if (a < D) idx[a] = S.li[(ti * W + w) * D + a];
        idx[A.l] = j;
        const double th = over_hbar(P, -S.sc[SC_TAU] * kinetic_cross<DM>(P, S.tc, S.sc, idx));
        if constexpr (sizeof(T) == 8) {
          double sn, cs;
          expi_tab(th, S.sct, sn, cs);
          v = V{fma(v.x, cs, -v.y * sn), fma(v.x, sn, v.y * cs)};
        } else {
          const double kk = rint(th * 0.15915494309189535);
          double r = fma(-kk, 6.283185307179586, th);
          r = fma(-kk, 2.4492935982947064e-16, r);
          float sn, cs;
          sincosf((float)r, &sn, &cs);
          v = V{fmaf(v.x, cs, -v.y * sn), fmaf(v.x, sn, v.y * cs)};
        }
      }
      if (A.keep) cur[e] = v;
      else if (dst) __stcg(dst + S.tb[ti] + j * es + w * ws, v);
    }
    __syncthreads();
    if (stream) {
      // the prefetched region holds the next chunk; the other two are free
      const int nd = rf;
      rf = rd;
      rd = nd;
    } else {
      res = cur == S.reg[0] ? 0 : (cur == S.reg[1] ? 1 : 2);
    }
  }
  if (stream) {
    if (threadIdx.x == 0) *S.mphase = parity;
    __syncthreads();
  }
  if (A.red != RED_NONE) {
    if constexpr (sizeof(T) == 4) {
      if (A.red == RED_KIN) {
#pragma unroll
        for (int v = 0; v < DM + 1; ++v) acc[v] = (double)ks[v] + (double)kc[v];
      }
    }
    const int nv = (A.red == RED_OBS_KIN || A.red == RED_OBS_V) ? D + 2 : D + 1;
    block_partials<V, DM>(B, S, A.slot, acc, nv, A.rec ? A.rec + A.slot * PSTRIDE : nullptr);
  }
  return res;
}

// One-time set-up of the streamed-pass mbarriers (kernel start, before use).
template <typename V> __device__ void init_mbarriers(const Smem<V>& S) {
  if (threadIdx.x == 0) {
    for (int r = 0; r < 3; ++r) mbar_init(S.mbar + r);
    *S.mphase = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// Store tiles of axis D-1 that are resident in smem region `res` to psi.
template <typename T> __device__ void flush_resident(const Plan& P, const Bufs& B,
                                                      const Smem<typename VT<T>::v>& S, int res) {
  using V = typename VT<T>::v;
  const AxisPlan& ax = P.ax[P.D - 1];
  const int n = ax.n, W = ax.W;
  const int64_t bid = blockIdx.x, nb = gridDim.x;
  const int64_t mine = bid < ax.ntiles ? (ax.ntiles - bid + nb - 1) / nb : 0;
  V* dst = (V*)B.psi;
  const int cnt = (int)mine * W * n;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int ti = e / (W * n);
    const int rem = e - ti * W * n;
    const int64_t t = bid + (int64_t)ti * nb;
    __stcg(dst + t * W * n + rem, S.reg[res][e]);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Scalar bookkeeping of the grid centres.  Runs in warp 0 only, lane a for
// axis a, results in shared memory (every extra warp running scalar FP64
// code would cost another 64 cycles per instruction on its sub-partition).
// ---------------------------------------------------------------------------

// Substep sizes of kinetic unit u (a kinetic substep, optionally followed by a
// fused potential substep), with the half-steps of neighbouring symmetric
// stages merged (U_T(a) U_T(b) = U_T(a+b) also for the moving grid, because
// <p> is invariant under the kinetic substep).
__device__ __forceinline__ void unit_coeffs(const Run& R, const double* gam, int64_t u, double& tau,
                                            double& sig, bool& hasv) {
  const int S = R.S;
  const int64_t nS = R.n_steps * S;
  const double dt = R.dt;
  const int k = (int)(u % S);
  if (R.split == SPLIT_TVT) {
    if (u == 0) tau = 0.5 * gam[0] * dt;
    else if (u == nS) tau = 0.5 * gam[S - 1] * dt;
    else tau = 0.5 * (gam[(k + S - 1) % S] + gam[k]) * dt;
    hasv = u < nS;
    sig = gam[k] * dt;
  } else if (R.split == SPLIT_VTV) {
    tau = gam[k] * dt;
    hasv = true;
    sig = (u == nS - 1) ? 0.5 * gam[S - 1] * dt : 0.5 * (gam[k] + gam[(k + 1) % S]) * dt;
  } else {  // first-order TV: V(g_k dt) T(g_k dt) per stage
    tau = gam[k] * dt;
    hasv = u < nS - 1;
    sig = gam[(k + 1) % S] * dt;
  }
}

// After the kinetic moments: delta = tau m^-1 <p> (or m^-1 p, or 0), q_new.
template <typename V> __device__ void centre_after_kinetic(const Plan& P, const Smem<V>& S, int motion) {
  if (threadIdx.x < 32) {
    const int a = threadIdx.x;
    double* sc = S.sc;
    int bad = 0;
    double pi = 0.0, n = 0.0;
    if (a < P.D) {
      n = S.fin[0];
      pi = fma(P.dp[a], S.fin[1 + a] / n, sc[SC_P + a]);
      sc[SC_MOM + a] = motion == GRID_ADAPTIVE ? pi : sc[SC_P + a];
    }
    __syncwarp();
    if (a < P.D) {
      // delta = tau m^-1 <p> (eq:eom_qt_solution_case_III_T) with the full
      // symmetric inverse mass matrix of eq:KE_operator when it has
      // off-diagonal entries
      double mdot = P.minv[a] * sc[SC_MOM + a];
      if (P.minv_general) {
        mdot = 0.0;
        for (int b = 0; b < P.D; ++b) mdot = fma(P.minvf[a * P.D + b], sc[SC_MOM + b], mdot);
      }
      const double delta = motion == GRID_FIXED ? 0.0 : sc[SC_TAU] * mdot;
      if (!(n > 0) || !isfinite(n) || !isfinite(pi)) bad = ST_NONFINITE;
      else if (fabs(delta) > 10.0 * P.N[a] * P.dq[a]) bad = ST_UNSTABLE;
      sc[SC_DELTA + a] = delta;
      sc[SC_QN + a] = sc[SC_Q + a] + delta;
    }
    bad = __reduce_min_sync(0xffffffffu, bad);
    if (a == 0) sc[SC_ERR] = (double)bad;
  }
  __syncthreads();
}

// After the potential moments: p <- p - sigma <dV/dq>.
template <typename V> __device__ void centre_after_potential(const Plan& P, const Smem<V>& S, int motion) {
  if (threadIdx.x < 32) {
    const int a = threadIdx.x;
    double* sc = S.sc;
    int bad = 0;
    if (a < P.D) {
      const double n = S.fin[0];
      const double g = S.fin[1 + a] / n;
      if (!(n > 0) || !isfinite(n) || !isfinite(g)) bad = ST_NONFINITE;
      if (motion != GRID_FIXED) {
        const double dpn = sc[SC_SIG] * g;
        if (fabs(dpn) > 10.0 * P.N[a] * P.dp[a]) bad = bad ? bad : ST_UNSTABLE;
        sc[SC_P + a] -= dpn;
      }
    }
    bad = __reduce_min_sync(0xffffffffu, bad);
    if (a == 0) sc[SC_ERR] = (double)bad;
  }
  __syncthreads();
}


}  // namespace
}  // namespace mgk
