// Host side of the C-ABI declared in include/mgrid.h: validation, planning of
// the axis passes, workspace layout, host-side state preparation (initial
// wavepackets, composition coefficients) and kernel launches.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "mg_plan.h"
#include "mg_regrid.h"
#include "mg_short.h"
#include "mgrid.h"

namespace mgk {
void* propagate_kernel(int prec, int kind);
void* obs_kernel(int prec, int kind);
void* init_tables_kernel(int prec);
void* obs_tables_kernel(int prec);
void* set_product_kernel(int prec);
void* adjoint_kernel(int kind);
void* short_kernel(int prec, int n, int tma, int tc);
void* regrid_kernel(int prec, int kind);
void* inner_kernel(int prec);
int short_threads_for(int prec, int n);
int short_lpc_for(int prec, int n, int tc);
int short_tc_smem_bytes(int tc);
}  // namespace mgk

using namespace mgk;

namespace {

constexpr int MAXBLOCKS = 2048;
constexpr int RESIDENT_CAP = 96 * 1024;  // bytes per smem region when tiles stay resident
constexpr int CHUNK_REGION = 64 * 1024;  // bytes per smem region otherwise

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t ctrl, bar, status, part, tw, tabA, tabAi, tabK, tabV, tabC, tabE, gamma, sct, tabF, tabP, tabB, scratch, total;
};

// Axis length of a grid the short-axis kernel can take (D >= 3 axes, all of
// one length 8, 12 or 16), else 0.
int short_shape(int D, const int64_t* N) {
  if (D < 3 || D > MAXD) return 0;
  const int64_t n = N[0];
  if (n != 8 && n != 12 && n != 16) return 0;
  for (int l = 1; l < D; ++l)
    if (N[l] != n) return 0;
  return (int)n;
}

Layout layout_for(int D, const int64_t* N, int precision) {
  int64_t npts = 1, tt = 0;
  for (int l = 0; l < D; ++l) {
    npts *= N[l];
    tt += N[l];
  }
  Layout L{};
  size_t o = 0;
  auto put = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.ctrl = put(CTRL * sizeof(double));
  L.bar = put(64 * sizeof(unsigned));
  L.status = put(sizeof(int));
  // two slots of per-CTA records; the adjoint's records are 32 doubles
  L.part = put(2ull * MAXBLOCKS * 32 * sizeof(double));
  L.tw = put(tt * sizeof(double2));
  L.tabA = put(tt * sizeof(double2));
  L.tabAi = put(tt * sizeof(double2));
  L.tabK = put(tt * sizeof(double2));
  L.tabV = put((size_t)NVCOL * tt * sizeof(double));
  L.tabC = put(tt * sizeof(double));
  L.tabE = put(tt * sizeof(double));
  L.gamma = put(MAX_STAGES * sizeof(double));
  L.sct = put(256 * sizeof(double2));
  // per-axis and pair potential factors of the short-axis kernel
  const int sn = short_shape(D, N);
  L.tabF = put(sn ? tt * sizeof(double2) : 0);
  L.tabP = put(sn ? (size_t)(D - 1) * sn * sn * sizeof(double2) : 0);
  L.tabB = put(sn ? 2 * tt * sizeof(double2) : 0);
  L.scratch = put((size_t)npts * (precision == 0 ? sizeof(double2) : sizeof(float2)));
  L.total = o;
  return L;
}

// Axis length check: even, 2..MAXN, only prime factors 2 and 3.
bool axis_supported(int64_t n) {
  if (n < 2 || n > MAXN || n % 2) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// Radix passes for length n using powers of two no larger than rmax (8, 4 or 2)
// and radix 3.  A smaller rmax gives more butterflies per pass: on GB300 an
// FP64 warp instruction costs a sub-partition 64 cycles whatever its number of
// active lanes, so a CTA with few lines is faster with radix 4 or 2 spread over
// all four sub-partitions than with radix 8 on one or two.
void radix_plan(int n, AxisPlan& ax, int rmax = 8) {
  int c2 = 0, c3 = 0;
  while (n % 2 == 0) { n /= 2; ++c2; }
  while (n % 3 == 0) { n /= 3; ++c3; }
  ax.nrad = 0;
  if (rmax >= 8)
    while (c2 >= 3) { ax.rad[ax.nrad++] = 8; c2 -= 3; }
  if (rmax >= 4)
    while (c2 >= 2) { ax.rad[ax.nrad++] = 4; c2 -= 2; }
  while (c2 >= 1) { ax.rad[ax.nrad++] = 2; c2 -= 1; }
  for (int i = 0; i < c3; ++i) ax.rad[ax.nrad++] = 3;
}

size_t smem_for(const Plan& P) {
  // must match carve() in mg_device.cuh
  const size_t vs = P.prec == 0 ? sizeof(double2) : sizeof(float2);
  auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t TT = (size_t)P.tab_total;
  const int nmult = (P.tab_global & TG_MULT) ? 0 : 3;
  const int ncols = (P.tab_global & TG_COLS) ? 0 : 1;
  size_t s = (1 + nmult) * r16(vs * TT) + ncols * (r16(sizeof(double) * NVCOL * TT) + 2 * r16(sizeof(double) * TT)) +
             r16(sizeof(double2) * 256) + r16(sizeof(double) * THREADS * (3 * P.D + 5)) +
             r16(sizeof(double) * PSTRIDE) + r16(sizeof(double) * SCALARS) +
             (P.resident ? 2 : 3) * r16((size_t)P.region_bytes) + r16(sizeof(uint64_t) * 3) +
             r16(sizeof(unsigned) * 4) + r16(sizeof(int64_t) * P.max_tiles) +
             r16(sizeof(uint16_t) * P.max_lines * P.D);
  return s;
}

// Tile and chunk sizes for a given grid size of the persistent kernel.
constexpr int64_t SMEM_CAP = 227 * 1024;  // dynamic shared memory a CTA may use

void chunk_plan(Plan& P, int64_t region) {
  const size_t vs = P.prec == 0 ? sizeof(double2) : sizeof(float2);
  const int D = P.D;
  P.region_bytes = (int)((region + 15) & ~int64_t(15));
  for (int l = 0; l < D; ++l) {
    AxisPlan& ax = P.ax[l];
    const int64_t tile_bytes = (int64_t)ax.W * ax.n * vs;
    ax.tpc = (int)std::max<int64_t>(1, P.region_bytes / tile_bytes);
    // butterflies a CTA has per pass; aim for at least one warp per sub-partition
    const int64_t mine = (ax.ntiles + P.nblocks - 1) / P.nblocks;
    const int64_t lines = std::min<int64_t>(mine, ax.tpc) * ax.W;
    const int rmax = lines * ax.n / 8 >= 128 ? 8 : (lines * ax.n / 4 >= 128 ? 4 : 2);
    radix_plan(ax.n, ax, rmax);
  }
  // per-chunk tile offsets and line indices live in shared memory
  P.max_tiles = 1;
  P.max_lines = 1;
  for (int l = 0; l < D; ++l) {
    const AxisPlan& ax = P.ax[l];
    const int64_t mine = std::max<int64_t>((ax.ntiles + P.nblocks - 1) / P.nblocks, 1);
    const int64_t tiles = (P.resident && (l == 0 || l == D - 1)) ? mine : std::min<int64_t>(ax.tpc, mine);
    P.max_tiles = (int)std::max<int64_t>(P.max_tiles, tiles);
    P.max_lines = (int)std::max<int64_t>(P.max_lines, tiles * ax.W);
  }
  P.smem_bytes = (int)smem_for(P);
}

void tile_plan_tables(Plan& P) {
  const size_t vs = P.prec == 0 ? sizeof(double2) : sizeof(float2);
  const int D = P.D;
  int64_t need_res = 0, need_min = 0;
  for (int l = 0; l < D; ++l) {
    AxisPlan& ax = P.ax[l];
    const bool contig = (l == D - 1);
    ax.W = contig ? 1 : (P.prec == 0 ? 2 : (ax.stride % 4 == 0 ? 4 : 2));
    if (!contig && ax.W > ax.stride) ax.W = (int)ax.stride;
    const int64_t lines = P.npts / ax.n;
    ax.ntiles = lines / ax.W;
    const int64_t tile_bytes = (int64_t)ax.W * ax.n * vs;
    need_min = std::max(need_min, tile_bytes);
    if (l == 0 || l == D - 1) {
      const int64_t mine = (ax.ntiles + P.nblocks - 1) / P.nblocks;
      need_res = std::max(need_res, mine * tile_bytes);
    }
  }
  P.resident = need_res <= RESIDENT_CAP;
  if (P.resident) {
    chunk_plan(P, std::max(need_res, need_min));
    return;
  }
  // HBM-streamed passes: three chunk regions (load, transform, prefetch).  A
  // tile is as large as a region allows, so that the TMA engine moves it in a
  // few large copies: on the contiguous axis W consecutive lines (one copy), on
  // a strided axis n rows of W adjacent elements (one copy per row).
  int64_t region = CHUNK_REGION;
  for (;;) {
    for (int l = 0; l < D; ++l) {
      AxisPlan& ax = P.ax[l];
      const int64_t lim = std::max<int64_t>(1, region / ((int64_t)ax.n * vs));
      const int64_t lines = P.npts / ax.n;
      const int64_t mult = (l == D - 1) ? lines : ax.stride;  // W must divide this
      int64_t W = 1;
      while (W * 2 <= lim && mult % (W * 2) == 0) W *= 2;
      if (l < D - 1 && W * vs < 16) W = std::min<int64_t>(ax.stride, 16 / (int64_t)vs);  // 16-byte rows
      ax.W = (int)W;
      ax.ntiles = lines / W;
    }
    need_min = 0;
    for (int l = 0; l < D; ++l) need_min = std::max<int64_t>(need_min, (int64_t)P.ax[l].W * P.ax[l].n * vs);
    chunk_plan(P, std::max(region, need_min));
    if (P.smem_bytes <= SMEM_CAP || region <= 4096) break;
    region = region - region / 8 - 16;
  }
}

// Tiles and chunks, with the per-axis tables in shared memory when they fit
// beside the data regions; long axes (sum of lengths in the thousands) keep
// their potential columns, and for FP64 their multipliers too, in the
// workspace.
void tile_plan(Plan& P) {
  P.tab_global = 0;
  tile_plan_tables(P);
  if (P.smem_bytes <= SMEM_CAP) return;
  P.tab_global = TG_COLS;
  tile_plan_tables(P);
  if (P.smem_bytes <= SMEM_CAP || P.prec != 0) return;
  P.tab_global = TG_COLS | TG_MULT;
  tile_plan_tables(P);
}

// Shared memory of the short-axis kernel for regions of `re` elements: sets
// region_elems, nreg (3 if it fits, else 2) and smem_bytes.  Must match
// carve_short() in mg_short.cu.
bool short_smem(const Plan& P, ShortPlan& SP, int re) {
  auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t tcb = (size_t)short_tc_smem_bytes(SP.tc);
  const size_t vs = P.prec == 0 ? sizeof(double2) : sizeof(float2);
  const size_t ts = P.prec == 0 ? sizeof(double) : sizeof(float);
  const size_t TT = (size_t)P.tab_total, n = (size_t)SP.n;
  // the sincos table only for FP64 (the FP32 phases use sincosf); one
  // 16-value record per warp
  const size_t tabs = 5 * r16(vs * TT) + (P.prec == 0 ? r16(sizeof(double2) * 256) : 0) +
                      r16(sizeof(double) * 16 * (size_t)(SP.threads / 32)) + r16(sizeof(double) * PSTRIDE) +
                      r16(sizeof(double) * SCALARS) + r16(sizeof(uint64_t) * 3) + r16(sizeof(unsigned) * 4) +
                      r16(vs * (size_t)(P.D - 1) * n * (n + 1)) + r16(ts * 5 * TT) +
                      r16(vs * (size_t)SP.ngroups * n * (n + 1));
  const size_t cap = 227 * 1024 - 1024;  // dynamic shared memory, with room for the static part
  const size_t rb = r16(vs * (size_t)re);
  for (int nreg = 3; nreg >= 2; --nreg) {
    // + up to 1008 bytes per region to start it on a 1024-byte boundary;
    // regions of whole kilobytes need that only before the first
    const size_t total = tabs + (rb % 1024 == 0 ? 1008 + (size_t)nreg * rb : (size_t)nreg * (rb + 1008)) + tcb;
    if (total <= cap) {
      SP.region_elems = re;
      SP.nreg = nreg;
      SP.smem_bytes = (int)total;
      return true;
    }
  }
  return false;
}

// Groups, chunking and shared memory of the short-axis kernel (mg_short.h).
// A chunk holds lpc lines along any axis of its group (one line per thread
// for FP64, two for FP32).  The group that ends at the last axis takes the
// most axes whose blocks tile a chunk; the other groups, from the back, the
// most axes (up to SHORT_MAXG) whose chunk rows of WT adjacent elements are
// at least 32 bytes (one DRAM sector) and divide the trailing index range.
bool short_plan(const Plan& P, ShortPlan& SP, int tc = 0) {
  std::memset(&SP, 0, sizeof(ShortPlan));
  SP.tc = tc;
  const int D = P.D;
  const int n = short_shape(D, P.N);
  if (!n || P.minv_general) return false;  // per-axis kinetic tables only
  const size_t vs = P.prec == 0 ? sizeof(double2) : sizeof(float2);
  const int threads = short_threads_for(P.prec, n);
  const int lpc = short_lpc_for(P.prec, n, tc);
  auto pw = [&](int k) {
    int64_t r = 1;
    for (int i = 0; i < k; ++i) r *= n;
    return r;
  };
  int gc = 0;
  for (int g = 1; g <= std::min(D, SHORT_MAXG); ++g)
    if (lpc % pw(g - 1) == 0) gc = g;
  int ngr = 0;
  {
    GroupPlan& G = SP.grp[ngr++];
    G.l0 = D - gc;
    G.g = gc;
    G.contig = 1;
    G.WT = (int)(lpc / pw(gc - 1));
    G.ng = (int)pw(gc);
    G.inner = 1;
    G.nb = 1;
    G.nblk = P.npts / G.ng;
    G.nchunks = (G.nblk + G.WT - 1) / G.WT;
    G.PS = (int)(pw(gc - 1) * (n + 1) + (gc >= 2 ? 1 : 0));
  }
  for (int l1 = D - gc - 1; l1 >= 0;) {
    bool ok = false;
    for (int g = std::min(SHORT_MAXG, l1 + 1); g >= 1 && !ok; --g) {
      if (lpc % pw(g - 1)) continue;
      const int64_t W = lpc / pw(g - 1);
      const int64_t inner = pw(D - 1 - l1);
      if (inner % W) continue;
      if (g > 1 && (size_t)W * vs < 32) continue;
      GroupPlan& G = SP.grp[ngr++];
      G.l0 = l1 - g + 1;
      G.g = g;
      G.contig = 0;
      G.WT = (int)W;
      G.ng = (int)pw(g);
      G.inner = inner;
      G.nb = inner / W;
      G.nblk = 0;
      G.nchunks = P.npts / ((int64_t)G.ng * inner) * G.nb;
      G.PS = (int)(pw(g - 1) * (n + 1) + (g >= 2 ? 1 : 0));
      l1 -= g;
      ok = true;
    }
    if (!ok) return false;
  }
  SP.n = n;
  SP.ngroups = ngr;
  SP.threads = threads;
  int re = 0;
  for (int i = 0; i < ngr; ++i) re = std::max(re, SP.grp[i].WT * SP.grp[i].PS);
  if (!short_smem(P, SP, re)) return false;
  // FP64 12-point lines run two chunks at a time: three regions needed
  return !(P.prec == 0 && n == 12 && SP.nreg != 3);
}

// TMA tensor maps of the short-axis kernel's chunks (FP32 storage, 16-point
// axes, a three-axis group at the end and groups of one or two axes before
// it).  cuTensorMapEncodeTiled comes from the driver through the runtime's
// entry-point query, so the library links no driver stub.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool short_tma_maps(const Plan& P, ShortPlan& SP, void* psi) {
  static_assert(sizeof(TensorMapBytes) == sizeof(CUtensorMap), "tensor map size");
  if (P.prec != 1 || SP.n != 16) return false;
  const int D = P.D;
  const GroupPlan& G0 = SP.grp[0];
  if (!G0.contig || G0.g != 3 || ((uintptr_t)psi & 15)) return false;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const int n = 16;
  const size_t es = sizeof(float2);
  for (int gi = 0; gi < SP.ngroups; ++gi) {
    const GroupPlan& G = SP.grp[gi];
    cuuint64_t dim[5], str[4];
    cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    int rank;
    CUtensorMapSwizzle sw;
    if (gi == 0) {
      rank = 4;
      dim[0] = dim[1] = dim[2] = n;
      dim[3] = (cuuint64_t)G.nblk;
      str[0] = n * es;
      str[1] = n * n * es;
      str[2] = (cuuint64_t)n * n * n * es;
      box[0] = box[1] = box[2] = n;
      box[3] = (cuuint32_t)G.WT;
      sw = CU_TENSOR_MAP_SWIZZLE_128B;
    } else {
      if (G.contig || G.g > 2) return false;
      const int64_t WP = std::min<int64_t>(G.WT, 256);
      if (G.WT % WP || (WP * es) % 16) return false;
      rank = 0;
      dim[rank] = (cuuint64_t)G.inner;
      box[rank++] = (cuuint32_t)WP;
      int64_t s = G.inner;
      for (int k = 0; k < G.g; ++k) {  // the group's axes, last first
        str[rank - 1] = (cuuint64_t)(s * es);
        dim[rank] = n;
        box[rank++] = n;
        s *= n;
      }
      if (G.l0 > 0) {
        str[rank - 1] = (cuuint64_t)(s * es);
        dim[rank] = (cuuint64_t)(P.npts / s);
        box[rank++] = 1;
      }
      sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    }
    for (int r = 0; r < rank; ++r)
      if (dim[r] > (1ull << 32)) return false;
    CUresult r = enc((CUtensorMap*)&SP.tmap[gi], CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)rank, psi, dim, str, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    SP.trank[gi] = rank;
  }
  (void)D;
  return true;
}

// Regions of the TMA layouts are unpadded: WT blocks of n^g, or n^g rows of
// WT elements.  Recomputes region size, depth and shared memory for them.
bool short_tma_smem(const Plan& P, ShortPlan& SP) {
  int re = 0;
  for (int i = 0; i < SP.ngroups; ++i) re = std::max(re, SP.grp[i].WT * SP.grp[i].ng);
  return short_smem(P, SP, re);
}

// ---- composition coefficients (eq:comp_TVT; Yoshida 1990 triple jump,
// ---- Suzuki 1990 fractal), built by recursion on the order -----------------

// Stage coefficients of a named scheme into g[0 .. cap-1]; returns the number
// of stages S, or -1 for an unknown name or S > cap.  No heap use: the
// allocation-free entry point shares this generator.
int scheme_fill(const char* name, double* g, int cap) {
  if (!name || cap < 1) return -1;
  int family = -1, order = 0;
  if (std::strcmp(name, "strang") == 0) { family = 0; order = 2; }
  else if (std::strncmp(name, "yoshida", 7) == 0) { family = 1; order = std::atoi(name + 7); }
  else if (std::strncmp(name, "suzuki", 6) == 0) { family = 2; order = std::atoi(name + 6); }
  if (family < 0 || order < 2 || order > 10 || order % 2) return -1;
  double tmp[MAX_STAGES];
  int s = 1;
  g[0] = 1.0;
  for (int k = 1; 2 * k < order; ++k) {
    // raise the order from 2k to 2k+2
    const double e = 1.0 / (2 * k + 1);
    double w[5];
    int nw;
    if (family == 1) {
      const double a = 1.0 / (2.0 - std::pow(2.0, e));
      w[0] = a; w[1] = 1.0 - 2.0 * a; w[2] = a; nw = 3;
    } else {
      const double a = 1.0 / (4.0 - std::pow(4.0, e));
      w[0] = a; w[1] = a; w[2] = 1.0 - 4.0 * a; w[3] = a; w[4] = a; nw = 5;
    }
    if (s * nw > cap || s * nw > MAX_STAGES) return -1;
    for (int b = 0; b < nw; ++b)
      for (int i = 0; i < s; ++i) tmp[b * s + i] = w[b] * g[i];
    s *= nw;
    std::memcpy(g, tmp, sizeof(double) * s);
  }
  return s;
}

bool scheme_coeffs(const char* name, std::vector<double>& g) {
  g.assign(MAX_STAGES, 0.0);
  const int s = scheme_fill(name, g.data(), MAX_STAGES);
  if (s < 1) return false;
  g.resize(s);
  return true;
}

// Host twin of the kernels' round_unit_f32: the float pair bracketing (x, y)
// whose squared modulus is closest to 1 (FP32 twiddles without a norm bias).
void round_unit_f32_host(double x, double y, double* ox, double* oy) {
  const float xf = (float)x, yf = (float)y;
  const float xs[2] = {xf, (double)xf < x ? std::nextafterf(xf, INFINITY) : std::nextafterf(xf, -INFINITY)};
  const float ys[2] = {yf, (double)yf < y ? std::nextafterf(yf, INFINITY) : std::nextafterf(yf, -INFINITY)};
  double best = INFINITY;
  *ox = xf;
  *oy = yf;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const double e = std::fabs((double)xs[a] * xs[a] + (double)ys[b] * ys[b] - 1.0);
      if (e < best) {
        best = e;
        *ox = xs[a];
        *oy = ys[b];
      }
    }
}

}  // namespace

namespace mgk {

// e^{i k pi/128}, k = 0..255, for the table-driven sincos of the kernels:
// cosine and sine of the extended-precision angle, each correctly rounded.
// (Constants chosen to make |w| = 1 to the last bit instead move their
// angles by up to an ulp; on the 256 x 256 atom-diatom run to t = 2000 a.u.
// that took the p-centre 1e-12 further from an extended-precision run of the
// method, while fixing only a norm drift of the same size.)
void fill_sincos_table(double* t) {
  for (int k = 0; k < 256; ++k) {
    const long double a = 3.14159265358979323846264338327950288L * (long double)k / 128.0L;
    t[2 * k] = (double)std::cos(a);
    t[2 * k + 1] = (double)std::sin(a);
  }
}

// Forward twiddles e^{-2 pi i m / n}, m = 0 .. n-1, into t (2 n doubles):
// correctly rounded FP64 pairs, or for FP32 storage the float pairs of
// round_unit_f32_host.
void fill_twiddles(int n, int prec, double* t);

}  // namespace mgk

void mgk::fill_twiddles(int n, int prec, double* t) {
  for (int m = 0; m < n; ++m) {
    const long double ang = 2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)n;
    const double c = (double)std::cos(ang), s = (double)std::sin(ang);
    t[2 * m] = c;
    t[2 * m + 1] = -s;
    if (prec) round_unit_f32_host(c, -s, &t[2 * m], &t[2 * m + 1]);
  }
}

namespace {

// ---- digamma by recurrence + asymptotic series (Abramowitz & Stegun 6.3.5,
// ---- 6.3.18) for the Morse-state mean ------------------------------------------

double digamma(double x) {
  double r = 0;
  while (x < 12.0) {
    r -= 1.0 / x;
    x += 1.0;
  }
  const double i2 = 1.0 / (x * x);
  return r + std::log(x) - 0.5 / x -
         i2 * (1.0 / 12 - i2 * (1.0 / 120 - i2 * (1.0 / 252 - i2 * (1.0 / 240 - i2 / 132))));
}

}  // namespace

struct mg_ctx {
  Plan P;
  ShortPlan SP;  // short-axis kernel plan (SP.on = 0 when the grid does not qualify)
  Bufs B;
  Layout L;
  cudaStream_t stream;
  void* d_work;
  size_t work_bytes;
  double q[MAXD], p[MAXD], t;
  bool pot_set, state_set;
  bool tables_stale;  // the grid centre moved in a batched launch; A tables to rebuild
  double stuck_barrier_s;  // test hook: > 0 arms a barrier that cannot complete (mg_test_stuck_barrier)
  int64_t launches;
  std::vector<double> host;  // staging for psi
  std::vector<double> gam;
  double ctrl[32];
};

namespace {

mg_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? MG_OK : MG_ERR_CUDA; }

// Potentials of the form sum_a f_a(x_a) + sum_a h_a(x_a) g_{a+1}(x_{a+1}),
// the ones the short-axis kernel evaluates from per-axis and pair tables.
bool uses_short_kernel(const Plan& P) {
  return P.pot_kind == MG_POT_HENON_HEILES || (P.pot_kind == MG_POT_HARMONIC && !P.pot_general);
}

mg_status upload_ctrl(mg_ctx* c) {
  for (int a = 0; a < MAXD; ++a) {
    c->ctrl[a] = a < c->P.D ? c->q[a] : 0.0;
    c->ctrl[8 + a] = a < c->P.D ? c->p[a] : 0.0;
  }
  c->ctrl[16] = c->t;
  return cuda_ok(cudaMemcpyAsync(c->B.ctrl, c->ctrl, 17 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
}

mg_status launch_plain(mg_ctx* c, void* fn, void** args, size_t smem) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return MG_ERR_CUDA;
  }
  cudaError_t e = cudaLaunchKernel(fn, dim3(c->P.nblocks), dim3(THREADS), args, smem, c->stream);
  c->launches++;
  return cuda_ok(e);
}

mg_status init_tables(mg_ctx* c) {
  void* args[] = {&c->P, &c->B};
  c->tables_stale = false;
  return launch_plain(c, init_tables_kernel(c->P.prec), args, c->P.smem_bytes);
}

mg_status refresh_tables(mg_ctx* c) { return c->tables_stale ? init_tables(c) : MG_OK; }

mg_status read_status(mg_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return MG_ERR_CUDA;
  int st = 0;
  e = cudaMemcpy(&st, c->B.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return MG_ERR_CUDA;
  if (st != 0) {
    int zero = 0;
    cudaMemcpy(c->B.status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    return (mg_status)st;
  }
  return MG_OK;
}

double sqrt_cell(const Plan& P) {
  double v = 1;
  for (int l = 0; l < P.D; ++l) v *= P.dq[l];
  return std::sqrt(v);
}

// Copy the host FP64 scaled state into d_psi (converting to the storage type).
mg_status upload_u(mg_ctx* c) {
  const size_t n = (size_t)c->P.npts;
  if (c->P.prec == 0)
    return cuda_ok(cudaMemcpyAsync(c->B.psi, c->host.data(), n * sizeof(double2), cudaMemcpyHostToDevice,
                                   c->stream));
  std::vector<float> f(2 * n);
  for (size_t i = 0; i < 2 * n; ++i) f[i] = (float)c->host[i];
  mg_status s = cuda_ok(cudaMemcpyAsync(c->B.psi, f.data(), n * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK) s = cuda_ok(cudaStreamSynchronize(c->stream));
  return s;
}

}  // namespace

extern "C" {

size_t mg_workspace_bytes(int D, const int64_t* N, int precision) {
  if (D < 1 || D > MAXD || !N || (precision != MG_FP64 && precision != MG_FP32_MIXED)) return 0;
  for (int l = 0; l < D; ++l)
    if (!axis_supported(N[l])) return 0;
  return layout_for(D, N, precision).total;
}

mg_status mg_create(mg_ctx** out, int D, const int64_t* N, const double* dq, const double* minv, double hbar,
                    int precision, void* d_psi, void* d_work, size_t work_bytes, void* cuda_stream) {
  return mg_create_ex(out, D, N, dq, minv, hbar, precision, d_psi, d_work, work_bytes, cuda_stream, 0);
}

mg_status mg_create_ex(mg_ctx** out, int D, const int64_t* N, const double* dq, const double* minv, double hbar,
                       int precision, void* d_psi, void* d_work, size_t work_bytes, void* cuda_stream, int flags) {
  if (!out || !N || !dq || !minv || !d_psi || !d_work) return MG_ERR_ARG;
  if (flags & ~(MG_CREATE_GENERAL_KERNEL | MG_CREATE_NO_TMA | MG_CREATE_TC_TF32X3 | MG_CREATE_TC_BF16X3))
    return MG_ERR_ARG;
  if ((flags & MG_CREATE_TC_TF32X3) && (flags & MG_CREATE_TC_BF16X3)) return MG_ERR_ARG;
  const int want_tc = (flags & MG_CREATE_TC_TF32X3) ? 1 : ((flags & MG_CREATE_TC_BF16X3) ? 2 : 0);
  if (want_tc && (flags & (MG_CREATE_GENERAL_KERNEL | MG_CREATE_NO_TMA))) return MG_ERR_ARG;
  // the tensor-core variant of the short-axis kernel is not enabled (mgrid.h)
  if (want_tc) return MG_ERR_UNSUPPORTED;
  *out = nullptr;
  if (D < 1 || D > MAXD || !(hbar > 0) || !std::isfinite(hbar)) return MG_ERR_ARG;
  if (precision != MG_FP64 && precision != MG_FP32_MIXED) return MG_ERR_ARG;
  for (int l = 0; l < D; ++l) {
    if (N[l] < 2 || N[l] % 2) return MG_ERR_ARG;
    if (!(dq[l] > 0) || !std::isfinite(dq[l])) return MG_ERR_ARG;
    if (!axis_supported(N[l])) return MG_ERR_UNSUPPORTED;
  }
  // the inverse mass matrix of eq:KE_operator: symmetric positive definite
  // (Cholesky factorisation succeeds)
  {
    double L[MAXD * MAXD] = {0};
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        const double v = minv[a * D + b];
        if (!std::isfinite(v) || v != minv[b * D + a]) return MG_ERR_ARG;
      }
    for (int a = 0; a < D; ++a)
      for (int b = 0; b <= a; ++b) {
        double s = minv[a * D + b];
        for (int k = 0; k < b; ++k) s -= L[a * MAXD + k] * L[b * MAXD + k];
        if (a == b) {
          if (!(s > 0)) return MG_ERR_ARG;
          L[a * MAXD + a] = std::sqrt(s);
        } else {
          L[a * MAXD + b] = s / L[b * MAXD + b];
        }
      }
  }
  if (((uintptr_t)d_work & 255) || ((uintptr_t)d_psi & 15)) return MG_ERR_ARG;
  Layout L = layout_for(D, N, precision);
  if (work_bytes < L.total) return MG_ERR_ARG;

  mg_ctx* c = new mg_ctx();
  std::memset(&c->P, 0, sizeof(Plan));
  Plan& P = c->P;
  P.D = D;
  P.prec = precision;
  P.hbar = hbar;
  P.npts = 1;
  P.maxn = 0;
  P.tab_total = 0;
  P.pot_kind = -1;
  for (int l = 0; l < D; ++l) P.npts *= N[l];
  for (int l = D - 1; l >= 0; --l) {
    AxisPlan& ax = P.ax[l];
    ax.n = (int)N[l];
    ax.stride = (l == D - 1) ? 1 : P.ax[l + 1].stride * N[l + 1];
  }
  for (int l = 0; l < D; ++l) {
    AxisPlan& ax = P.ax[l];
    P.N[l] = N[l];
    P.dq[l] = dq[l];
    P.dp[l] = 2.0 * M_PI * hbar / ((double)N[l] * dq[l]);
    P.minv[l] = minv[l * D + l];
    ax.outer = P.npts / (ax.n * ax.stride);
    ax.toff = P.tab_total;
    P.tab_total += ax.n;
    P.maxn = std::max(P.maxn, ax.n);
    radix_plan(ax.n, ax);
  }
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      P.minvf[a * D + b] = minv[a * D + b];
      if (a != b && minv[a * D + b] != 0.0) P.minv_general = 1;
    }
  // grid of the persistent kernel: one CTA per SM (all co-resident)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return MG_ERR_CUDA;
  }
  P.nblocks = std::min(MAXBLOCKS, sms);
  tile_plan(P);
  for (int kind = 0; kind < 4; ++kind) {
    void* fn = propagate_kernel(P.prec, kind);
    if (P.smem_bytes > 48 * 1024)
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, THREADS, P.smem_bytes) != cudaSuccess || occ < 1) {
      delete c;
      return MG_ERR_UNSUPPORTED;
    }
    if (occ * sms < P.nblocks) {
      P.nblocks = occ * sms;
      tile_plan(P);
    }
  }

  c->L = L;
  c->stream = (cudaStream_t)cuda_stream;
  c->d_work = d_work;
  c->work_bytes = work_bytes;
  char* w = (char*)d_work;
  Bufs& B = c->B;
  B.psi = d_psi;
  B.ctrl = (double*)(w + L.ctrl);
  B.bar = (unsigned*)(w + L.bar);
  B.status = (int*)(w + L.status);
  B.part = (double*)(w + L.part);
  B.tw = (double2*)(w + L.tw);
  B.tabA = (double2*)(w + L.tabA);
  B.tabAi = (double2*)(w + L.tabAi);
  B.tabK = (double2*)(w + L.tabK);
  B.tabV = (double*)(w + L.tabV);
  B.tabC = (double*)(w + L.tabC);
  B.tabE = (double*)(w + L.tabE);
  B.gamma = (const double*)(w + L.gamma);
  B.sct = (double2*)(w + L.sct);
  B.scratch = (double2*)(w + L.scratch);

  // short-axis kernel: one CTA per SM, all co-resident
  if (!(flags & MG_CREATE_GENERAL_KERNEL) && short_plan(P, c->SP, want_tc)) {
    c->SP.tma = !(flags & MG_CREATE_NO_TMA) && short_tma_maps(P, c->SP, d_psi) ? 1 : 0;
    if (c->SP.tma && !short_tma_smem(P, c->SP)) c->SP.tma = 0;
    void* fn = short_kernel(P.prec, c->SP.n, c->SP.tma, c->SP.tc);
    int occ = 0;
    // the tensor-core variant holds 64 TMEM columns per CTA (512 per SM)
    if (fn && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, c->SP.smem_bytes) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, c->SP.threads, c->SP.smem_bytes) == cudaSuccess &&
        occ >= 1 && (!c->SP.tc || occ * 64 <= 512)) {
      c->SP.nblocks = std::min(MAXBLOCKS, occ * sms);
      c->SP.tabF = (double2*)(w + L.tabF);
      c->SP.tabP = (double2*)(w + L.tabP);
      c->SP.tabB = (double2*)(w + L.tabB);
      c->SP.tabC = c->SP.tabB + P.tab_total;
      c->SP.on = 1;
    } else {
      cudaGetLastError();
      c->SP.on = 0;
    }
  }
  if (want_tc && !(c->SP.on && c->SP.tma && c->SP.tc)) {
    // the tensor-core line DFTs exist for FP32 grids of 16-point axes whose
    // chunks move by TMA copies only
    delete c;
    return MG_ERR_UNSUPPORTED;
  }

  // static tables: twiddles e^{-2 pi i m/N_l} and k - N_l/2
  std::vector<double> tw(2 * P.tab_total), kc(P.tab_total);
  for (int l = 0; l < D; ++l) {
    const int n = P.ax[l].n;
    fill_twiddles(n, P.prec, &tw[2 * P.ax[l].toff]);
    for (int m = 0; m < n; ++m) kc[P.ax[l].toff + m] = (double)(m - n / 2);
  }
  std::vector<double> sct(512);
  fill_sincos_table(sct.data());
  mg_status s = cuda_ok(cudaMemsetAsync(d_work, 0, L.scratch, c->stream));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(B.sct, sct.data(), 512 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(B.tw, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(B.tabC, kc.data(), kc.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK) s = cuda_ok(cudaStreamSynchronize(c->stream));
  if (s != MG_OK) {
    delete c;
    return s;
  }
  for (int a = 0; a < MAXD; ++a) c->q[a] = c->p[a] = 0.0;
  c->t = 0;
  c->pot_set = c->state_set = false;
  c->launches = 0;
  *out = c;
  return MG_OK;
}

mg_status mg_destroy(mg_ctx* ctx) {
  if (!ctx) return MG_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
  return MG_OK;
}

mg_status mg_set_potential(mg_ctx* c, int kind, const double* params, int nparams) {
  if (!c || (!params && nparams > 0)) return MG_ERR_ARG;
  const int D = c->P.D;
  int need;
  switch (kind) {
    case MG_POT_HARMONIC: need = D * D + D; break;
    case MG_POT_ATOM_DIATOM: need = 5; if (D != 2) return MG_ERR_ARG; break;
    case MG_POT_HENON_HEILES: need = 1; break;
    case MG_POT_SECREST_JOHNSON: need = 3; if (D != 2) return MG_ERR_ARG; break;
    default: return MG_ERR_ARG;
  }
  if (nparams != need) return MG_ERR_ARG;
  for (int i = 0; i < nparams; ++i)
    if (!std::isfinite(params[i])) return MG_ERR_ARG;
  c->P.pot_kind = kind;
  c->P.pot_general = 0;
  std::memset(c->P.pot, 0, sizeof(c->P.pot));
  std::memcpy(c->P.pot, params, sizeof(double) * nparams);
  if (kind == MG_POT_HARMONIC)
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        if (params[a * D + b] != params[b * D + a]) return MG_ERR_ARG;
        if (a != b && params[a * D + b] != 0.0) c->P.pot_general = 1;
      }
  c->pot_set = true;
  return MG_OK;
}

mg_status mg_set_state(mg_ctx* c, const double* psi, const double* q, const double* p, double t) {
  if (!c || !q || !p || !std::isfinite(t)) return MG_ERR_ARG;
  for (int a = 0; a < c->P.D; ++a)
    if (!std::isfinite(q[a]) || !std::isfinite(p[a])) return MG_ERR_ARG;
  mg_status s = cuda_ok(cudaStreamSynchronize(c->stream));
  if (s != MG_OK) return s;
  if (psi) {
    const size_t n = (size_t)c->P.npts;
    const double sc = sqrt_cell(c->P);
    c->host.resize(2 * n);
    for (size_t i = 0; i < 2 * n; ++i) c->host[i] = psi[i] * sc;
    s = upload_u(c);
    if (s != MG_OK) return s;
  } else if (!c->state_set) {
    return MG_ERR_STATE;
  }
  for (int a = 0; a < c->P.D; ++a) {
    c->q[a] = q[a];
    c->p[a] = p[a];
  }
  c->t = t;
  s = upload_ctrl(c);
  if (s == MG_OK) s = init_tables(c);
  if (s == MG_OK) s = cuda_ok(cudaStreamSynchronize(c->stream));
  if (s == MG_OK) c->state_set = true;
  return s;
}

mg_status mg_upload_u(mg_ctx* c, const void* host_u, const double* q, const double* p, double t) {
  if (!c || !host_u || !q || !p || !std::isfinite(t)) return MG_ERR_ARG;
  for (int a = 0; a < c->P.D; ++a)
    if (!std::isfinite(q[a]) || !std::isfinite(p[a])) return MG_ERR_ARG;
  const size_t bytes = (size_t)c->P.npts * (c->P.prec == 0 ? sizeof(double2) : sizeof(float2));
  mg_status s = cuda_ok(cudaMemcpyAsync(c->B.psi, host_u, bytes, cudaMemcpyHostToDevice, c->stream));
  if (s != MG_OK) return s;
  for (int a = 0; a < c->P.D; ++a) {
    c->q[a] = q[a];
    c->p[a] = p[a];
  }
  c->t = t;
  s = upload_ctrl(c);
  if (s == MG_OK) s = init_tables(c);
  if (s == MG_OK) c->state_set = true;
  return s;
}

mg_status mg_download_u(mg_ctx* c, void* host_u, double* q, double* p, double* t) {
  if (!c || !host_u) return MG_ERR_ARG;
  if (!c->state_set) return MG_ERR_STATE;
  const size_t bytes = (size_t)c->P.npts * (c->P.prec == 0 ? sizeof(double2) : sizeof(float2));
  mg_status s = cuda_ok(cudaMemcpyAsync(host_u, c->B.psi, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (s == MG_OK) s = mg_get_state(c, nullptr, q, p, t);  // synchronises, reports the status
  return s;
}

double mg_morse_mean(double Dm, double a, double re, double mass, double hbar) {
  // <x> = re - (digamma(2 lam - 1) - ln(2 lam)) / a: z = 2 lam e^{-a(x - re)}
  // is Gamma(2 lam - 1)-distributed under |phi0|^2.
  const double lam = std::sqrt(2.0 * mass * Dm) / (a * hbar);
  if (!(lam > 0.5)) return NAN;
  return re - (digamma(2.0 * lam - 1.0) - std::log(2.0 * lam)) / a;
}

mg_status mg_set_separable(mg_ctx* c, const int* kinds, const double* params, const double* q_ctr,
                           const double* p_ctr) {
  if (!c || !kinds || !params || !q_ctr || !p_ctr) return MG_ERR_ARG;
  const Plan& P = c->P;
  const int D = P.D;
  std::vector<std::vector<double>> fac(D);  // per-axis complex samples (re, im)
  for (int l = 0; l < D; ++l) {
    const double* w = params + 4 * l;
    const int n = (int)P.N[l];
    fac[l].resize(2 * n);
    for (int j = 0; j < n; ++j) {
      const double x = q_ctr[l] + (j - n / 2) * P.dq[l];
      double re, im;
      if (kinds[l] == 0) {
        const double q0 = w[0], p0 = w[1], sg = w[2];
        if (!(sg > 0)) return MG_ERR_ARG;
        const double d = x - q0;
        const double amp = std::pow(M_PI * sg * sg, -0.25) * std::exp(-d * d / (2.0 * sg * sg));
        const double ph = p0 * d / P.hbar;
        re = amp * std::cos(ph);
        im = amp * std::sin(ph);
      } else if (kinds[l] == 1) {
        const double Dm = w[0], aa = w[1], re0 = w[2], mass = w[3];
        const double lam = std::sqrt(2.0 * mass * Dm) / (aa * P.hbar);
        if (!(lam > 0.5) || !(aa > 0)) return MG_ERR_ARG;
        const double z = 2.0 * lam * std::exp(-aa * (x - re0));
        const double lg = (lam - 0.5) * std::log(z) - 0.5 * z + 0.5 * (std::log(aa) - std::lgamma(2.0 * lam - 1.0));
        re = std::exp(lg);
        im = 0.0;
      } else {
        return MG_ERR_ARG;
      }
      fac[l][2 * j] = re;
      fac[l][2 * j + 1] = im;
    }
  }
  // The outer product is formed on the device from the per-axis factors
  // (first axis scaled by sqrt(prod dq)), staged in the kinetic table, which
  // every propagation rebuilds before use.
  const double sc = sqrt_cell(P);
  std::vector<double> f(2 * (size_t)P.tab_total);
  for (int l = 0; l < D; ++l)
    for (int j = 0; j < (int)P.N[l]; ++j) {
      const double m = l == 0 ? sc : 1.0;
      f[2 * (P.ax[l].toff + j)] = fac[l][2 * j] * m;
      f[2 * (P.ax[l].toff + j) + 1] = fac[l][2 * j + 1] * m;
    }
  mg_status s = cuda_ok(cudaStreamSynchronize(c->stream));
  if (s == MG_OK)
    s = cuda_ok(cudaMemcpyAsync(c->B.tabK, f.data(), f.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK) {
    void* args[] = {&c->P, &c->B};
    s = launch_plain(c, set_product_kernel(P.prec), args, 0);
  }
  if (s != MG_OK) return s;
  for (int a = 0; a < D; ++a) {
    c->q[a] = q_ctr[a];
    c->p[a] = p_ctr[a];
  }
  c->t = 0;
  s = upload_ctrl(c);
  if (s == MG_OK) s = init_tables(c);
  if (s == MG_OK) s = cuda_ok(cudaStreamSynchronize(c->stream));
  if (s == MG_OK) c->state_set = true;
  return s;
}

mg_status mg_propagate(mg_ctx* c, int64_t n_steps, double dt, const char* scheme, int split, int grid_motion) {
  if (!c || n_steps < 0 || !std::isfinite(dt)) return MG_ERR_ARG;
  if (split != MG_TVT && split != MG_VTV && split != MG_TV) return MG_ERR_ARG;
  if (grid_motion == MG_GRID_NAIVE) {
    // Sec. II.F: each step on the fixed grid, then the grid moved to the
    // new <q>, <p> by f~(<q>, <p>) f(q, <p>); host-sequenced, one step at a time
    if (!scheme_coeffs(scheme, c->gam)) return MG_ERR_ARG;
    for (int64_t s = 0; s < n_steps; ++s) {
      mg_status st = mg_propagate(c, 1, dt, scheme, split, MG_GRID_FIXED);
      double mq[MAXD], mp[MAXD];
      if (st == MG_OK) st = mg_get_observables(c, nullptr, nullptr, mq, mp);
      if (st == MG_OK) st = mg_regrid(c, mq, mp);
      if (st != MG_OK) return st;
    }
    return MG_OK;
  }
  if (grid_motion != MG_GRID_ADAPTIVE && grid_motion != MG_GRID_ADAPTIVE_CENTRE_P && grid_motion != MG_GRID_FIXED)
    return MG_ERR_ARG;
  if (!scheme_coeffs(scheme, c->gam)) return MG_ERR_ARG;
  if (!c->pot_set || !c->state_set) return MG_ERR_STATE;
  if (n_steps == 0) return MG_OK;
  if (refresh_tables(c) != MG_OK) return MG_ERR_CUDA;
  Run R{};
  R.n_steps = n_steps;
  R.S = (int)c->gam.size();
  R.dt = dt;
  R.split = split;
  R.motion = grid_motion;
  R.lead_v = split != MG_TVT;
  R.n_units = (split == MG_TVT) ? n_steps * R.S + 1 : n_steps * R.S;
  mg_status s = cuda_ok(cudaMemcpyAsync((void*)c->B.gamma, c->gam.data(), c->gam.size() * sizeof(double),
                                        cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK) s = cuda_ok(cudaMemsetAsync(c->B.bar, 0, 64 * sizeof(unsigned), c->stream));
  if (s != MG_OK) return s;
  const bool short_path = c->SP.on && uses_short_kernel(c->P);
  Bufs B = c->B;
  if (c->stuck_barrier_s > 0) {
    // test hook: the barrier word starts with gridDim.x arrivals of the
    // current generation, so no arrival is ever the last one; every CTA's
    // wait runs out after the short limit and the kernel returns
    const unsigned long long word = (unsigned long long)(short_path ? c->SP.nblocks : c->P.nblocks);
    s = cuda_ok(cudaMemcpyAsync(c->B.bar, &word, sizeof(word), cudaMemcpyHostToDevice, c->stream));
    if (s == MG_OK) s = cuda_ok(cudaStreamSynchronize(c->stream));
    if (s != MG_OK) return s;
    B.bar_limit_ns = (uint64_t)(c->stuck_barrier_s * 1e9);
    c->stuck_barrier_s = 0;
  }
  if (short_path) {
    ShortPlan SP = c->SP;
    SP.pairs = c->P.pot_kind == MG_POT_HENON_HEILES;
    void* sfn = short_kernel(c->P.prec, SP.n, SP.tma, SP.tc);
    void* sargs[] = {&c->P, &B, &R, &SP};
    cudaError_t e = cudaLaunchCooperativeKernel(sfn, dim3(SP.nblocks), dim3(SP.threads), sargs, SP.smem_bytes,
                                                c->stream);
    c->launches++;
    if (e != cudaSuccess) return MG_ERR_CUDA;
    c->t += (double)n_steps * dt;
    return MG_OK;
  }
  void* fn = propagate_kernel(c->P.prec, c->P.pot_kind);
  if (!fn) return MG_ERR_UNSUPPORTED;
  if (c->P.smem_bytes > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, c->P.smem_bytes) != cudaSuccess)
    return MG_ERR_CUDA;
  void* args[] = {&c->P, &B, &R};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(c->P.nblocks), dim3(THREADS), args, c->P.smem_bytes, c->stream);
  c->launches++;
  if (e != cudaSuccess) return MG_ERR_CUDA;
  c->t += (double)n_steps * dt;
  return MG_OK;
}

mg_status mg_test_stuck_barrier(mg_ctx* c, double limit_s) {
  if (!c || !(limit_s > 0) || !(limit_s <= 5.0)) return MG_ERR_ARG;
  c->stuck_barrier_s = limit_s;
  return MG_OK;
}

namespace {

// One regrid launch on context c (tables and barrier of c).
mg_status launch_regrid(mg_ctx* c, const RegridArgs& R) {
  mg_status s = cuda_ok(cudaMemsetAsync(c->B.bar, 0, 64 * sizeof(unsigned), c->stream));
  if (s != MG_OK) return s;
  void* fn = regrid_kernel(c->P.prec, c->pot_set ? c->P.pot_kind : MG_POT_HARMONIC);
  if (!fn) return MG_ERR_UNSUPPORTED;
  if (c->P.smem_bytes > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, c->P.smem_bytes) != cudaSuccess)
    return MG_ERR_CUDA;
  RegridArgs r = R;
  void* args[] = {&c->P, &c->B, &r};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(c->P.nblocks), dim3(THREADS), args, c->P.smem_bytes, c->stream);
  c->launches++;
  return cuda_ok(e);
}

}  // namespace

mg_status mg_regrid(mg_ctx* c, const double* q, const double* p) {
  if (!c || !q || !p) return MG_ERR_ARG;
  if (!c->state_set) return MG_ERR_STATE;
  const int D = c->P.D;
  for (int a = 0; a < D; ++a)
    if (!std::isfinite(q[a]) || !std::isfinite(p[a])) return MG_ERR_ARG;
  mg_status s = refresh_tables(c);
  if (s != MG_OK) return s;
  RegridArgs R{};
  for (int a = 0; a < D; ++a) {
    R.qt[a] = q[a];
    R.pt[a] = p[a];
  }
  R.src_ctrl = c->B.ctrl;
  R.buf = c->B.psi;
  R.keep_p = 0;
  R.commit = 1;
  s = launch_regrid(c, R);
  if (s != MG_OK) return s;
  for (int a = 0; a < D; ++a) {
    c->q[a] = q[a];
    c->p[a] = p[a];
  }
  return read_status(c);
}

mg_status mg_inner_product(mg_ctx* a, const mg_ctx* b, double* re, double* im) {
  if (!a || !b || !re || !im) return MG_ERR_ARG;
  if (!a->state_set || !b->state_set) return MG_ERR_STATE;
  const Plan &Pa = a->P, &Pb = b->P;
  if (Pa.D != Pb.D || Pa.prec != Pb.prec || Pa.hbar != Pb.hbar) return MG_ERR_ARG;
  for (int l = 0; l < Pa.D; ++l)
    if (Pa.N[l] != Pb.N[l] || Pa.dq[l] != Pb.dq[l]) return MG_ERR_ARG;
  // b's state, final on its stream, copied into a's scratch and carried onto
  // a's positions with b's own momentum window
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MG_ERR_CUDA;
  mg_status s = read_status(a);
  if (s != MG_OK) return s;
  const size_t bytes = (size_t)Pa.npts * (Pa.prec == 0 ? sizeof(double2) : sizeof(float2));
  s = cuda_ok(cudaMemcpyAsync(a->B.scratch, b->B.psi, bytes, cudaMemcpyDeviceToDevice, a->stream));
  if (s != MG_OK) return s;
  double qa[16];
  if (cudaMemcpy(qa, a->B.ctrl, sizeof(qa), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
  RegridArgs R{};
  for (int l = 0; l < Pa.D; ++l) R.qt[l] = qa[l];
  R.src_ctrl = b->B.ctrl;
  R.buf = a->B.scratch;
  R.keep_p = 1;
  R.commit = 0;
  s = launch_regrid(a, R);
  a->tables_stale = true;  // the launch rebuilt a's tables for b's momentum window
  if (s != MG_OK) return s;
  void* args[] = {&a->P, &a->B.psi, &a->B.scratch, &a->B.part};
  if (cudaLaunchKernel(inner_kernel(Pa.prec), dim3(Pa.nblocks), dim3(THREADS), args, 0, a->stream) != cudaSuccess)
    return MG_ERR_CUDA;
  a->launches++;
  s = read_status(a);
  if (s != MG_OK) return s;
  std::vector<double> part((size_t)Pa.nblocks * PSTRIDE);
  if (cudaMemcpy(part.data(), a->B.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MG_ERR_CUDA;
  double sr = 0, si = 0;
  for (int k = 0; k < Pa.nblocks; ++k) {
    sr += part[(size_t)k * PSTRIDE];
    si += part[(size_t)k * PSTRIDE + 1];
  }
  *re = sr;
  *im = si;
  return MG_OK;
}

mg_status mg_sync(mg_ctx* c) {
  if (!c) return MG_ERR_ARG;
  return read_status(c);
}

mg_status mg_get_state(mg_ctx* c, double* psi, double* q, double* p, double* t) {
  if (!c) return MG_ERR_ARG;
  if (!c->state_set) return MG_ERR_STATE;
  mg_status s = read_status(c);
  if (s != MG_OK) return s;
  const int D = c->P.D;
  double ctrl[17];
  if (cudaMemcpy(ctrl, c->B.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
  for (int a = 0; a < D; ++a) {
    c->q[a] = ctrl[a];
    c->p[a] = ctrl[8 + a];
    if (q) q[a] = ctrl[a];
    if (p) p[a] = ctrl[8 + a];
  }
  if (t) *t = c->t;
  if (psi) {
    const size_t n = (size_t)c->P.npts;
    const double sc = 1.0 / sqrt_cell(c->P);
    if (c->P.prec == 0) {
      if (cudaMemcpy(psi, c->B.psi, n * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
      for (size_t i = 0; i < 2 * n; ++i) psi[i] *= sc;
    } else {
      std::vector<float> f(2 * n);
      if (cudaMemcpy(f.data(), c->B.psi, n * sizeof(float2), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
      for (size_t i = 0; i < 2 * n; ++i) psi[i] = (double)f[i] * sc;
    }
  }
  return MG_OK;
}

mg_status mg_get_observables(mg_ctx* c, double* norm, double* energy, double* mean_q, double* mean_p) {
  if (!c) return MG_ERR_ARG;
  if (!c->state_set || !c->pot_set) return MG_ERR_STATE;
  mg_status s = read_status(c);
  if (s != MG_OK) return s;
  const Plan& P = c->P;
  void* targs[] = {&c->P, &c->B};
  s = refresh_tables(c);
  if (s == MG_OK) s = launch_plain(c, obs_tables_kernel(P.prec), targs, P.smem_bytes);
  void* fn = obs_kernel(P.prec, P.pot_kind);
  for (int l = P.D - 1; l >= 0 && s == MG_OK; --l) {
    int mode = 0;
    void* args[] = {&c->P, &c->B, &l, &mode};
    s = launch_plain(c, fn, args, P.smem_bytes);
  }
  if (s == MG_OK) {
    int l = P.D - 1, mode = 1;
    void* args[] = {&c->P, &c->B, &l, &mode};
    s = launch_plain(c, fn, args, P.smem_bytes);
  }
  if (s != MG_OK) return s;
  s = read_status(c);
  if (s != MG_OK) return s;
  const int nb = P.nblocks;
  std::vector<double> part(2ull * nb * PSTRIDE);
  if (cudaMemcpy(part.data(), c->B.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MG_ERR_CUDA;
  double ctrl[17];
  if (cudaMemcpy(ctrl, c->B.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
  const int D = P.D;
  double k[PSTRIDE] = {0}, v[PSTRIDE] = {0};
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < D + 2; ++i) {
      k[i] += part[(size_t)b * PSTRIDE + i];
      v[i] += part[((size_t)nb + b) * PSTRIDE + i];
    }
  if (norm) *norm = v[0];
  if (energy) *energy = k[D + 1] / k[0] + v[D + 1] / v[0];
  for (int a = 0; a < D; ++a) {
    if (mean_q) mean_q[a] = v[1 + a] / v[0];
    if (mean_p) mean_p[a] = ctrl[8 + a] + P.dp[a] * k[1 + a] / k[0];
  }
  return MG_OK;
}

mg_status mg_adjoint(mg_ctx* c, int64_t n_steps, double dt, const char* scheme, int split, int grid_motion,
                     void* d_ubar, double* qbar, double* pbar, double* theta_bar, int ntheta) {
  if (!c || !d_ubar || !qbar || !pbar || n_steps < 0 || !std::isfinite(dt)) return MG_ERR_ARG;
  if (split != MG_TVT && split != MG_VTV && split != MG_TV) return MG_ERR_ARG;
  if (grid_motion != MG_GRID_ADAPTIVE && grid_motion != MG_GRID_ADAPTIVE_CENTRE_P && grid_motion != MG_GRID_FIXED)
    return MG_ERR_ARG;
  if (((uintptr_t)d_ubar & 15)) return MG_ERR_ARG;
  if (!scheme_coeffs(scheme, c->gam)) return MG_ERR_ARG;
  if (!c->pot_set || !c->state_set) return MG_ERR_STATE;
  const Plan& P = c->P;
  const int nth = P.pot_kind == MG_POT_ATOM_DIATOM ? 4 : 0;
  if (P.prec != MG_FP64 || !P.resident || P.minv_general) return MG_ERR_UNSUPPORTED;
  if (P.pot_kind != MG_POT_HARMONIC && P.pot_kind != MG_POT_ATOM_DIATOM) return MG_ERR_UNSUPPORTED;
  if (ntheta != nth || (nth > 0 && !theta_bar)) return MG_ERR_ARG;
  for (int a = 0; a < P.D; ++a)
    if (!std::isfinite(qbar[a]) || !std::isfinite(pbar[a])) return MG_ERR_ARG;
  if (n_steps == 0) {
    for (int k = 0; k < nth; ++k) theta_bar[k] = 0.0;
    return MG_OK;
  }
  // the dual (state + cotangent) passes need two more shared-memory regions
  const size_t smem = (size_t)P.smem_bytes + 2 * (((size_t)P.region_bytes + 15) & ~size_t(15));
  void* fn = adjoint_kernel(P.pot_kind);
  if (!fn || smem > 227 * 1024) return MG_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MG_ERR_CUDA;
  int occ = 0, dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, THREADS, smem) != cudaSuccess)
    return MG_ERR_CUDA;
  if (occ * sms < P.nblocks) return MG_ERR_UNSUPPORTED;
  double norm = 0;
  mg_status s = mg_get_observables(c, &norm, nullptr, nullptr, nullptr);
  if (s != MG_OK) return s;
  AdjRun AR{};
  AR.R.n_steps = n_steps;
  AR.R.S = (int)c->gam.size();
  AR.R.dt = dt;
  AR.R.split = split;
  AR.R.motion = grid_motion;
  AR.R.lead_v = split != MG_TVT;
  AR.R.n_units = (split == MG_TVT) ? n_steps * AR.R.S + 1 : n_steps * AR.R.S;
  AR.ubar = d_ubar;
  AR.ntheta = nth;
  AR.norm = norm;
  double cb[16] = {0};
  for (int a = 0; a < P.D; ++a) {
    cb[a] = qbar[a];
    cb[8 + a] = pbar[a];
  }
  s = cuda_ok(cudaMemcpyAsync(c->B.ctrl + 20, cb, sizeof(cb), cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK)
    s = cuda_ok(cudaMemcpyAsync((void*)c->B.gamma, c->gam.data(), c->gam.size() * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
  if (s == MG_OK) s = cuda_ok(cudaMemsetAsync(c->B.bar, 0, 64 * sizeof(unsigned), c->stream));
  if (s != MG_OK) return s;
  void* args[] = {&c->P, &c->B, &AR};
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(P.nblocks), dim3(THREADS), args, smem, c->stream);
  c->launches++;
  if (e != cudaSuccess) return MG_ERR_CUDA;
  s = read_status(c);
  if (s != MG_OK) return s;
  double ctrl[CTRL];
  if (cudaMemcpy(ctrl, c->B.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
  for (int a = 0; a < P.D; ++a) {
    c->q[a] = ctrl[a];
    c->p[a] = ctrl[8 + a];
    qbar[a] = ctrl[20 + a];
    pbar[a] = ctrl[28 + a];
  }
  for (int k = 0; k < nth; ++k) theta_bar[k] = ctrl[36 + k];
  c->t -= (double)n_steps * dt;
  return MG_OK;
}

int64_t mg_kernel_launches(const mg_ctx* c) { return c ? c->launches : -1; }

int mg_propagate_path(const mg_ctx* c) {
  if (!c || !c->pot_set) return -1;
  if (!c->SP.on || !uses_short_kernel(c->P)) return 0;
  return c->SP.tma ? 2 : 1;
}

int mg_tables_in_workspace(const mg_ctx* c) { return c ? c->P.tab_global : -1; }

int mg_scheme_coefficients(const char* scheme, double* gamma, int max) {
  std::vector<double> g;
  if (!scheme_coeffs(scheme, g)) return -1;
  if (gamma)
    for (int i = 0; i < (int)g.size() && i < max; ++i) gamma[i] = g[i];
  return (int)g.size();
}

int mg_short_axis_plan(int D, const int64_t* N, int precision, int* first_axis, int* naxes, int* threads,
                       int* smem_bytes) {
  if (!N || D < 1 || D > MAXD || (precision != MG_FP64 && precision != MG_FP32_MIXED)) return -1;
  for (int l = 0; l < D; ++l)
    if (!axis_supported(N[l])) return -1;
  // the parts of the grid plan that the short-axis planner reads (as mg_create
  // fills them)
  Plan P;
  std::memset(&P, 0, sizeof(Plan));
  P.D = D;
  P.prec = precision;
  P.hbar = 1.0;
  P.npts = 1;
  for (int l = 0; l < D; ++l) P.npts *= N[l];
  for (int l = D - 1; l >= 0; --l) {
    P.ax[l].n = (int)N[l];
    P.ax[l].stride = (l == D - 1) ? 1 : P.ax[l + 1].stride * N[l + 1];
  }
  for (int l = 0; l < D; ++l) {
    P.N[l] = N[l];
    P.dq[l] = 1.0;
    P.ax[l].outer = P.npts / (P.ax[l].n * P.ax[l].stride);
    P.ax[l].toff = P.tab_total;
    P.tab_total += P.ax[l].n;
    P.maxn = std::max(P.maxn, P.ax[l].n);
  }
  ShortPlan SP;
  if (!short_plan(P, SP)) return 0;
  for (int g = 0; g < SP.ngroups; ++g) {
    if (first_axis) first_axis[g] = SP.grp[g].l0;
    if (naxes) naxes[g] = SP.grp[g].g;
  }
  if (threads) *threads = SP.threads;
  if (smem_bytes) *smem_bytes = SP.smem_bytes;
  return SP.ngroups;
}

const char* mg_status_string(int s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_UNSUPPORTED: return "unsupported configuration";
    case MG_ERR_CUDA: return "CUDA runtime error";
    case MG_ERR_TIMEOUT: return "grid barrier timed out";
    case MG_ERR_NONFINITE: return "non-finite norm or reduction";
    case MG_ERR_UNSTABLE: return "grid centre diverged (time step beyond the Verlet stability limit)";
    case MG_ERR_STATE: return "potential or state not set";
  }
  return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// mg_propagate_noalloc: the propagation kernel for callers that cannot
// allocate device memory.  Its scratch (per-axis tables, per-CTA partial
// sums, barrier words, composition coefficients, grid centres) lives in one
// file-scope __device__ array instead of a caller-provided workspace.
// ---------------------------------------------------------------------------

#include <mutex>

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 768 * 1024;  // held by every GPU that loads the library
constexpr int NOALLOC_MAXTAB = 4096;                  // largest sum of the axis lengths
constexpr int NOALLOC_MAXBLOCKS = 1024;               // largest persistent grid
constexpr int NOALLOC_MAXDEV = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Offsets inside g_noalloc_scratch (fixed, independent of the grid), each
// aligned to 256 bytes (the kernels load double2 values: 16-byte alignment
// is required).
constexpr size_t na_al(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t NA_CTRL = 0;
constexpr size_t NA_BAR = 256;
constexpr size_t NA_STATUS = 512;
constexpr size_t NA_PART = 768;
constexpr size_t NA_TW = na_al(NA_PART + 2ull * NOALLOC_MAXBLOCKS * PSTRIDE * sizeof(double));
constexpr size_t NA_TABA = na_al(NA_TW + NOALLOC_MAXTAB * sizeof(double2));
constexpr size_t NA_TABAI = na_al(NA_TABA + NOALLOC_MAXTAB * sizeof(double2));
constexpr size_t NA_TABK = na_al(NA_TABAI + NOALLOC_MAXTAB * sizeof(double2));
constexpr size_t NA_TABV = na_al(NA_TABK + NOALLOC_MAXTAB * sizeof(double2));
constexpr size_t NA_TABC = na_al(NA_TABV + (size_t)NVCOL * NOALLOC_MAXTAB * sizeof(double));
constexpr size_t NA_TABE = na_al(NA_TABC + NOALLOC_MAXTAB * sizeof(double));
constexpr size_t NA_GAMMA = na_al(NA_TABE + NOALLOC_MAXTAB * sizeof(double));
constexpr size_t NA_SCT = na_al(NA_GAMMA + MAX_STAGES * sizeof(double));
constexpr size_t NA_END = NA_SCT + 256 * sizeof(double2);
static_assert(NA_END <= NOALLOC_SCRATCH_BYTES, "static scratch too small for its layout");
static_assert(NA_TW % 256 == 0 && NA_TABA % 256 == 0 && NA_TABAI % 256 == 0 && NA_TABK % 256 == 0 &&
                  NA_TABV % 256 == 0 && NA_TABC % 256 == 0 && NA_TABE % 256 == 0 && NA_GAMMA % 256 == 0 &&
                  NA_SCT % 256 == 0,
              "static scratch regions must be 256-byte aligned");

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAXDEV];

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a stand-in, so the address is looked up once per device
// (with that device current) and cached.
mg_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAXDEV) return MG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MG_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_propagate_noalloc(int D, const int64_t* N, const double* dq, const double* minv,
                                          double hbar, int pot_kind, const double* pot_params, int npot,
                                          void* d_psi, double* q, double* p, int64_t n_steps, double dt,
                                          const char* scheme, int split, int grid_motion, void* cuda_stream) {
  // ---- arguments (nothing touches the device before they pass) ----
  if (!N || !dq || !minv || !d_psi || !q || !p || (!pot_params && npot > 0)) return MG_ERR_ARG;
  if (D < 1 || D > MAXD || !(hbar > 0) || !std::isfinite(hbar) || n_steps < 0 || !std::isfinite(dt))
    return MG_ERR_ARG;
  if (split != MG_TVT && split != MG_VTV && split != MG_TV) return MG_ERR_ARG;
  // the naive grid (one host round trip and regrid per step) needs the
  // context's scratch state buffer: not offered here
  if (grid_motion == MG_GRID_NAIVE) return MG_ERR_UNSUPPORTED;
  if (grid_motion != MG_GRID_ADAPTIVE && grid_motion != MG_GRID_ADAPTIVE_CENTRE_P && grid_motion != MG_GRID_FIXED)
    return MG_ERR_ARG;
  if ((uintptr_t)d_psi & 15) return MG_ERR_ARG;
  int tab_total = 0;
  for (int l = 0; l < D; ++l) {
    if (N[l] < 2 || N[l] % 2 || !(dq[l] > 0) || !std::isfinite(dq[l])) return MG_ERR_ARG;
    if (!axis_supported(N[l])) return MG_ERR_UNSUPPORTED;
    tab_total += (int)N[l];
    if (!std::isfinite(q[l]) || !std::isfinite(p[l])) return MG_ERR_ARG;
  }
  if (tab_total > NOALLOC_MAXTAB) return MG_ERR_UNSUPPORTED;  // beyond the static scratch
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) {
      const double v = minv[a * D + b];
      if (!std::isfinite(v)) return MG_ERR_ARG;
      if (a != b && v != 0.0) return MG_ERR_UNSUPPORTED;
      if (a == b && !(v > 0)) return MG_ERR_ARG;
    }
  int need;
  switch (pot_kind) {
    case MG_POT_HARMONIC: need = D * D + D; break;
    case MG_POT_ATOM_DIATOM: need = 5; if (D != 2) return MG_ERR_ARG; break;
    case MG_POT_HENON_HEILES: need = 1; break;
    case MG_POT_SECREST_JOHNSON: need = 3; if (D != 2) return MG_ERR_ARG; break;
    default: return MG_ERR_ARG;
  }
  if (npot != need) return MG_ERR_ARG;
  for (int i = 0; i < npot; ++i)
    if (!std::isfinite(pot_params[i])) return MG_ERR_ARG;
  double gam[MAX_STAGES];
  const int S = scheme_fill(scheme, gam, MAX_STAGES);
  if (S <= 0) return MG_ERR_ARG;
  if (n_steps == 0) return MG_OK;

  // ---- plan (same tiling rules as a context) ----
  Plan P;
  std::memset(&P, 0, sizeof(Plan));
  P.D = D;
  P.prec = MG_FP64;
  P.hbar = hbar;
  P.npts = 1;
  for (int l = 0; l < D; ++l) P.npts *= N[l];
  for (int l = D - 1; l >= 0; --l) {
    P.ax[l].n = (int)N[l];
    P.ax[l].stride = (l == D - 1) ? 1 : P.ax[l + 1].stride * N[l + 1];
  }
  for (int l = 0; l < D; ++l) {
    AxisPlan& ax = P.ax[l];
    P.N[l] = N[l];
    P.dq[l] = dq[l];
    P.dp[l] = 2.0 * M_PI * hbar / ((double)N[l] * dq[l]);
    P.minv[l] = minv[l * D + l];
    ax.outer = P.npts / (ax.n * ax.stride);
    ax.toff = P.tab_total;
    P.tab_total += ax.n;
    P.maxn = std::max(P.maxn, ax.n);
    radix_plan(ax.n, ax);
  }
  P.pot_kind = pot_kind;
  std::memcpy(P.pot, pot_params, sizeof(double) * npot);
  if (pot_kind == MG_POT_HARMONIC)
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        if (pot_params[a * D + b] != pot_params[b * D + a]) return MG_ERR_ARG;
        if (a != b && pot_params[a * D + b] != 0.0) P.pot_general = 1;
      }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MG_ERR_CUDA;
  P.nblocks = std::min(NOALLOC_MAXBLOCKS, sms);
  tile_plan(P);
  void* fn = propagate_kernel(P.prec, pot_kind);
  if (!fn) return MG_ERR_UNSUPPORTED;
  if (P.smem_bytes > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes) != cudaSuccess)
    return MG_ERR_CUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, THREADS, P.smem_bytes) != cudaSuccess || occ < 1)
    return MG_ERR_UNSUPPORTED;
  if (occ * sms < P.nblocks) {
    P.nblocks = occ * sms;
    tile_plan(P);
  }

  // ---- scratch inside the static array ----
  void* base = nullptr;
  mg_status s = noalloc_scratch(&base);
  if (s != MG_OK) return s;
  char* w = (char*)base;
  Bufs B;
  std::memset(&B, 0, sizeof(Bufs));
  B.psi = d_psi;
  B.ctrl = (double*)(w + NA_CTRL);
  B.bar = (unsigned*)(w + NA_BAR);
  B.status = (int*)(w + NA_STATUS);
  B.part = (double*)(w + NA_PART);
  B.tw = (double2*)(w + NA_TW);
  B.tabA = (double2*)(w + NA_TABA);
  B.tabAi = (double2*)(w + NA_TABAI);
  B.tabK = (double2*)(w + NA_TABK);
  B.tabV = (double*)(w + NA_TABV);
  B.tabC = (double*)(w + NA_TABC);
  B.tabE = (double*)(w + NA_TABE);
  B.gamma = (const double*)(w + NA_GAMMA);
  B.sct = (double2*)(w + NA_SCT);
  B.scratch = nullptr;  // only the observables use it

  // The array keeps the previous call's contents: the barrier words and the
  // status word must start at zero; every other table is rewritten before use.
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double tw[2 * NOALLOC_MAXTAB], kc[NOALLOC_MAXTAB], ctrl[17], sct[512];
  fill_sincos_table(sct);
  for (int l = 0; l < D; ++l) {
    const int n = P.ax[l].n;
    fill_twiddles(n, MG_FP64, &tw[2 * P.ax[l].toff]);
    for (int m = 0; m < n; ++m) kc[P.ax[l].toff + m] = (double)(m - n / 2);
  }
  for (int a = 0; a < 8; ++a) {
    ctrl[a] = a < D ? q[a] : 0.0;
    ctrl[8 + a] = a < D ? p[a] : 0.0;
  }
  ctrl[16] = 0.0;
  s = cuda_ok(cudaMemsetAsync(w + NA_BAR, 0, 512, st));  // barrier words and status
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(B.tw, tw, sizeof(double) * 2 * P.tab_total, cudaMemcpyHostToDevice, st));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(B.tabC, kc, sizeof(double) * P.tab_total, cudaMemcpyHostToDevice, st));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(B.ctrl, ctrl, sizeof(ctrl), cudaMemcpyHostToDevice, st));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync((void*)B.gamma, gam, sizeof(double) * S, cudaMemcpyHostToDevice, st));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(B.sct, sct, sizeof(sct), cudaMemcpyHostToDevice, st));
  if (s != MG_OK) return s;

  // ---- launches: A tables for the starting p-centre, then the propagation ----
  void* targs[] = {&P, &B};
  if (P.smem_bytes > 48 * 1024 &&
      cudaFuncSetAttribute(init_tables_kernel(P.prec), cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes) != cudaSuccess)
    return MG_ERR_CUDA;
  if (cudaLaunchKernel(init_tables_kernel(P.prec), dim3(P.nblocks), dim3(THREADS), targs, P.smem_bytes, st) != cudaSuccess)
    return MG_ERR_CUDA;
  Run R;
  std::memset(&R, 0, sizeof(Run));
  R.n_steps = n_steps;
  R.S = S;
  R.dt = dt;
  R.split = split;
  R.motion = grid_motion;
  R.lead_v = split != MG_TVT;
  R.n_units = (split == MG_TVT) ? n_steps * S + 1 : n_steps * S;
  void* args[] = {&P, &B, &R};
  if (cudaLaunchCooperativeKernel(fn, dim3(P.nblocks), dim3(THREADS), args, P.smem_bytes, st) != cudaSuccess)
    return MG_ERR_CUDA;

  // ---- read back the grid centres and the status (synchronises the stream) ----
  int status = 0;
  s = cuda_ok(cudaMemcpyAsync(ctrl, B.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, st));
  if (s == MG_OK) s = cuda_ok(cudaMemcpyAsync(&status, B.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (s == MG_OK) s = cuda_ok(cudaStreamSynchronize(st));
  if (s != MG_OK) return s;
  if (status != 0) return (mg_status)status;
  for (int a = 0; a < D; ++a) {
    q[a] = ctrl[a];
    p[a] = ctrl[8 + a];
  }
  return MG_OK;
}

// ---------------------------------------------------------------------------
// Batched propagation: many grid contexts advanced by one persistent launch
// of thread-block clusters, replayed from a CUDA graph.
// ---------------------------------------------------------------------------

namespace mgk {
void* batch_kernel(int prec);
}

namespace {

constexpr int BATCH_MAXD = 3;
constexpr int BATCH_SMEM_CAP = 227 * 1024;

// Must match batch_carve() in mg_batch.cu.
size_t batch_smem_bytes(const BatchArgs& A, int prec) {
  const size_t vs = prec == 0 ? sizeof(double2) : sizeof(float2);
  auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t TT = (size_t)A.tab_total;
  return 4 * r16(vs * TT) + r16(sizeof(double) * NVCOL * TT) + r16(sizeof(double) * TT) +
         r16(sizeof(double2) * 256) + r16(sizeof(double) * THREADS * (A.D + 2)) + r16(sizeof(double) * PSTRIDE) +
         r16(sizeof(double) * SCALARS) + 3 * r16((size_t)A.region_bytes) + r16(sizeof(uint64_t) * 3) +
         r16(sizeof(unsigned) * 4) + r16(sizeof(int64_t) * A.max_tiles) +
         r16(sizeof(uint16_t) * A.max_lines * A.D);
}

// Tiles of one problem for a team of C CTAs: on each axis W lines per tile,
// the largest power of two whose tile stays within `target` bytes (at least
// 16-byte rows on strided axes, for the bulk copies).  Returns the largest
// tile in bytes.
int64_t batch_tiles(Plan& P, int C, int64_t target) {
  const int64_t vs = P.prec == 0 ? 16 : 8;
  int64_t big = 0;
  P.nblocks = C;
  P.resident = 0;
  for (int l = 0; l < P.D; ++l) {
    AxisPlan& ax = P.ax[l];
    const bool contig = (l == P.D - 1);
    const int64_t lines = P.npts / ax.n;
    const int64_t lim = std::max<int64_t>(1, target / ((int64_t)ax.n * vs));
    const int64_t mult = contig ? lines : ax.stride;
    int64_t W = 1;
    while (W * 2 <= lim && mult % (W * 2) == 0) W *= 2;
    if (!contig && W * vs < 16) W = std::min<int64_t>(ax.stride, 16 / vs);
    ax.W = (int)W;
    ax.ntiles = lines / W;
    big = std::max<int64_t>(big, W * ax.n * vs);
  }
  return big;
}

// Chunks and radix plans of one problem once the region size is known.
void batch_chunks(Plan& P, int64_t region, int rmax_req, int& max_tiles, int& max_lines) {
  const int64_t vs = P.prec == 0 ? 16 : 8;
  for (int l = 0; l < P.D; ++l) {
    AxisPlan& ax = P.ax[l];
    const int64_t tile = (int64_t)ax.W * ax.n * vs;
    ax.tpc = (int)std::max<int64_t>(1, region / tile);
    const int64_t mine = std::max<int64_t>(1, (ax.ntiles + P.nblocks - 1) / P.nblocks);
    const int64_t tiles = std::min<int64_t>(mine, ax.tpc);
    const int64_t lines = tiles * ax.W;
    const int rmax = rmax_req ? rmax_req : (lines * ax.n / 8 >= 128 ? 8 : (lines * ax.n / 4 >= 128 ? 4 : 2));
    radix_plan(ax.n, ax, rmax);
    max_tiles = (int)std::max<int64_t>(max_tiles, tiles);
    max_lines = (int)std::max<int64_t>(max_lines, lines);
  }
}

// Relative cost of one stage of a problem (transform work per point grows
// with the log of the axis lengths; the multipliers and reductions add a
// per-point constant).
double batch_cost(const Plan& P) {
  double lg = 0;
  for (int l = 0; l < P.D; ++l) lg += std::log2((double)P.ax[l].n);
  return (double)P.npts * (lg + 2.0 * P.D + 4.0);
}

struct BatchLayout {
  size_t probs, team_start, team_items, run, bstatus, sct, total;
};

BatchLayout batch_layout(int nprob) {
  BatchLayout L{};
  size_t o = 0;
  auto put = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.probs = put((size_t)nprob * sizeof(BatchProb));
  L.team_start = put((size_t)(MAXTEAMS + 1) * sizeof(int));
  L.team_items = put((size_t)nprob * sizeof(int));
  L.run = put(sizeof(BatchRun) + (size_t)nprob * sizeof(double));
  L.bstatus = put((size_t)nprob * sizeof(int));
  L.sct = put(256 * sizeof(double2));
  L.total = o;
  return L;
}

bool same_potential(const Plan& a, const Plan& b) {
  return a.pot_kind == b.pot_kind && a.pot_general == b.pot_general &&
         std::memcmp(a.pot, b.pot, sizeof(a.pot)) == 0;
}

}  // namespace

struct mg_batch {
  int nprob, prec, C, nteams, smem;
  std::vector<mg_ctx*> ctx;
  std::vector<BatchProb> hprob;
  BatchLayout L;
  BatchArgs A;
  char* d_work;
  cudaStream_t stream;  // the contexts' stream
  cudaStream_t cap;     // private stream the launch was captured on
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaEvent_t done;
  bool pending;
  unsigned char* h_run;  // pinned: BatchRun then one dt per problem
  size_t run_bytes;
  int64_t launches;
};

extern "C" {

size_t mg_batch_workspace_bytes(int nprob) {
  if (nprob < 1) return 0;
  return batch_layout(nprob).total;
}

mg_status mg_batch_destroy(mg_batch* b) {
  if (!b) return MG_ERR_ARG;
  if (b->pending) cudaEventSynchronize(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->h_run) cudaFreeHost(b->h_run);
  delete b;
  return MG_OK;
}

mg_status mg_batch_create(mg_batch** out, int nprob, mg_ctx* const* ctxs, int cluster, const int* tile_bytes,
                          const int* radix_max, void* d_work, size_t work_bytes) {
  if (!out || !ctxs || nprob < 1 || !d_work) return MG_ERR_ARG;
  *out = nullptr;
  if (cluster == 0) cluster = 2;
  if (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) return MG_ERR_ARG;
  if (((uintptr_t)d_work & 255)) return MG_ERR_ARG;
  const BatchLayout L = batch_layout(nprob);
  if (work_bytes < L.total) return MG_ERR_ARG;
  const int prec = ctxs[0] ? ctxs[0]->P.prec : 0;
  for (int i = 0; i < nprob; ++i) {
    const mg_ctx* c = ctxs[i];
    if (!c) return MG_ERR_ARG;
    if (!c->pot_set || !c->state_set) return MG_ERR_STATE;
    if (c->P.prec != prec || c->stream != ctxs[0]->stream) return MG_ERR_ARG;
    if (c->P.D > BATCH_MAXD || c->P.minv_general) return MG_ERR_UNSUPPORTED;
    if (tile_bytes && tile_bytes[i] < 0) return MG_ERR_ARG;
    if (radix_max && radix_max[i] != 0 && radix_max[i] != 2 && radix_max[i] != 4 && radix_max[i] != 8)
      return MG_ERR_ARG;
  }
  mg_batch* b = new mg_batch();
  b->nprob = nprob;
  b->prec = prec;
  b->C = cluster;
  b->L = L;
  b->d_work = (char*)d_work;
  b->stream = ctxs[0]->stream;
  b->ctx.assign(ctxs, ctxs + nprob);
  b->hprob.resize(nprob);
  std::memset(b->hprob.data(), 0, sizeof(BatchProb) * nprob);

  // ---- tiles, chunk region and shared-memory layout --------------------------
  const int64_t def_target = prec == 0 ? 32768 : 16384;
  int64_t scale_num = 1, scale_den = 1;  // shrinks every target while the layout is too large
  BatchArgs& A = b->A;
  std::memset(&A, 0, sizeof(BatchArgs));
  for (;;) {
    int64_t big = 0;
    A.D = 1;
    A.tab_total = 1;
    for (int i = 0; i < nprob; ++i) {
      Plan& P = b->hprob[i].P;
      P = ctxs[i]->P;
      P.tab_global = 0;  // the batched kernel keeps every table in shared memory
      const int64_t t = (tile_bytes && tile_bytes[i] ? tile_bytes[i] : def_target) * scale_num / scale_den;
      big = std::max(big, batch_tiles(P, cluster, std::max<int64_t>(t, 1)));
      A.D = std::max(A.D, P.D);
      A.tab_total = std::max(A.tab_total, P.tab_total);
    }
    const int64_t region = ((std::max(big, def_target * scale_num / scale_den) + 15) / 16) * 16;
    A.region_bytes = (int)region;
    A.max_tiles = 1;
    A.max_lines = 1;
    for (int i = 0; i < nprob; ++i)
      batch_chunks(b->hprob[i].P, region, radix_max ? radix_max[i] : 0, A.max_tiles, A.max_lines);
    A.smem_bytes = (int)batch_smem_bytes(A, prec);
    for (int i = 0; i < nprob; ++i) {
      Plan& P = b->hprob[i].P;
      P.region_bytes = A.region_bytes;
      P.max_tiles = A.max_tiles;
      P.max_lines = A.max_lines;
      P.smem_bytes = A.smem_bytes;
    }
    if (A.smem_bytes <= BATCH_SMEM_CAP) break;
    if (scale_den >= 64) {
      delete b;
      return MG_ERR_UNSUPPORTED;
    }
    scale_den *= 2;
  }
  b->smem = A.smem_bytes;

  void* fn = batch_kernel(prec);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, A.smem_bytes) != cudaSuccess) {
    delete b;
    return MG_ERR_CUDA;
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = A.smem_bytes;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) != cudaSuccess || ncl < 1) {
    delete b;
    return MG_ERR_UNSUPPORTED;
  }
  b->nteams = std::min(std::min(ncl, nprob), MAXTEAMS);
  A.nteams = b->nteams;

  // ---- longest-processing-time assignment of problems to teams ----------------
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::vector<double> cost(nprob);
  for (int i = 0; i < nprob; ++i) cost[i] = batch_cost(b->hprob[i].P);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> load(b->nteams, 0.0);
  std::vector<std::vector<int>> lists(b->nteams);
  for (int i : order) {
    int best = 0;
    for (int t = 1; t < b->nteams; ++t)
      if (load[t] < load[best]) best = t;
    load[best] += cost[i];
    lists[best].push_back(i);
  }
  std::vector<int> start(b->nteams + 1, 0), items;
  items.reserve(nprob);
  for (int t = 0; t < b->nteams; ++t) {
    start[t] = (int)items.size();
    items.insert(items.end(), lists[t].begin(), lists[t].end());
  }
  start[b->nteams] = (int)items.size();

  // ---- device descriptors ------------------------------------------------------
  for (int i = 0; i < nprob; ++i) {
    BatchProb& Q = b->hprob[i];
    const mg_ctx* c = ctxs[i];
    Q.psi = c->B.psi;
    Q.ctrl = c->B.ctrl;
    Q.status = c->B.status;
    Q.tw = c->B.tw;
    Q.tc = c->B.tabC;
  }
  char* w = b->d_work;
  A.probs = (const BatchProb*)(w + L.probs);
  A.team_start = (const int*)(w + L.team_start);
  A.team_items = (const int*)(w + L.team_items);
  A.run = (const BatchRun*)(w + L.run);
  A.dt = (const double*)(w + L.run + sizeof(BatchRun));
  A.bstatus = (int*)(w + L.bstatus);
  A.sct = (const double2*)(w + L.sct);
  std::vector<double> sct(512);
  fill_sincos_table(sct.data());
  b->run_bytes = sizeof(BatchRun) + (size_t)nprob * sizeof(double);
  mg_status s = cuda_ok(cudaMemcpy(w + L.probs, b->hprob.data(), sizeof(BatchProb) * nprob, cudaMemcpyHostToDevice));
  if (s == MG_OK) s = cuda_ok(cudaMemcpy(w + L.team_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (s == MG_OK) s = cuda_ok(cudaMemcpy(w + L.team_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (s == MG_OK) s = cuda_ok(cudaMemset(w + L.bstatus, 0, (size_t)nprob * sizeof(int)));
  if (s == MG_OK) s = cuda_ok(cudaMemcpy(w + L.sct, sct.data(), 512 * sizeof(double), cudaMemcpyHostToDevice));
  if (s == MG_OK) s = cuda_ok(cudaHostAlloc((void**)&b->h_run, b->run_bytes, cudaHostAllocDefault));
  if (s == MG_OK) std::memset(b->h_run, 0, b->run_bytes);
  if (s == MG_OK) s = cuda_ok(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
  if (s == MG_OK) s = cuda_ok(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));

  // ---- the launch as a graph: upload of the run parameters, then the kernel ----
  if (s == MG_OK) s = cuda_ok(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  if (s == MG_OK) {
    cudaError_t e = cudaMemcpyAsync(w + L.run, b->h_run, b->run_bytes, cudaMemcpyHostToDevice, b->cap);
    cfg.gridDim = dim3(b->nteams * cluster);
    cfg.stream = b->cap;
    void* args[] = {&A};
    if (e == cudaSuccess) e = cudaLaunchKernelExC(&cfg, fn, args);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &b->graph);
    s = cuda_ok(e != cudaSuccess ? e : e2);
  }
  if (s == MG_OK) s = cuda_ok(cudaGraphInstantiate(&b->exec, b->graph, 0));
  if (s != MG_OK) {
    mg_batch_destroy(b);
    return s;
  }
  *out = b;
  return MG_OK;
}

mg_status mg_batch_propagate(mg_batch* b, int64_t n_steps, const double* dt, const char* scheme, int split,
                             int grid_motion) {
  if (!b || !dt || n_steps < 0) return MG_ERR_ARG;
  if (split != MG_TVT && split != MG_VTV && split != MG_TV) return MG_ERR_ARG;
  if (grid_motion != MG_GRID_ADAPTIVE && grid_motion != MG_GRID_ADAPTIVE_CENTRE_P && grid_motion != MG_GRID_FIXED)
    return MG_ERR_ARG;
  for (int i = 0; i < b->nprob; ++i)
    if (!std::isfinite(dt[i])) return MG_ERR_ARG;
  std::vector<double> gam;
  if (!scheme_coeffs(scheme, gam) || (int)gam.size() > MAX_STAGES) return MG_ERR_ARG;
  if (n_steps == 0) return MG_OK;
  // potentials changed through the contexts since the last launch
  bool dirty = false;
  for (int i = 0; i < b->nprob; ++i) {
    const mg_ctx* c = b->ctx[i];
    if (!c->pot_set || !c->state_set) return MG_ERR_STATE;
    Plan& P = b->hprob[i].P;
    if (!same_potential(P, c->P)) {
      P.pot_kind = c->P.pot_kind;
      P.pot_general = c->P.pot_general;
      std::memcpy(P.pot, c->P.pot, sizeof(P.pot));
      dirty = true;
    }
  }
  if (b->pending) {
    if (cudaEventSynchronize(b->done) != cudaSuccess) return MG_ERR_CUDA;
    b->pending = false;
  }
  if (dirty &&
      cudaMemcpyAsync(b->d_work + b->L.probs, b->hprob.data(), sizeof(BatchProb) * b->nprob, cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess)
    return MG_ERR_CUDA;
  BatchRun* R = (BatchRun*)b->h_run;
  R->n_steps = n_steps;
  R->S = (int)gam.size();
  R->split = split;
  R->motion = grid_motion;
  for (size_t k = 0; k < gam.size(); ++k) R->gamma[k] = gam[k];
  std::memcpy(b->h_run + sizeof(BatchRun), dt, sizeof(double) * b->nprob);
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return MG_ERR_CUDA;
  if (cudaEventRecord(b->done, b->stream) != cudaSuccess) return MG_ERR_CUDA;
  b->pending = true;
  b->launches++;
  for (int i = 0; i < b->nprob; ++i) {
    b->ctx[i]->t += (double)n_steps * dt[i];
    b->ctx[i]->tables_stale = true;
  }
  return MG_OK;
}

mg_status mg_batch_sync(mg_batch* b, int* first_failed) {
  if (!b) return MG_ERR_ARG;
  if (first_failed) *first_failed = -1;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MG_ERR_CUDA;
  b->pending = false;
  std::vector<int> st(b->nprob);
  if (cudaMemcpy(st.data(), b->d_work + b->L.bstatus, sizeof(int) * b->nprob, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MG_ERR_CUDA;
  for (int i = 0; i < b->nprob; ++i)
    if (st[i] != 0) {
      if (first_failed) *first_failed = i;
      cudaMemset(b->d_work + b->L.bstatus, 0, sizeof(int) * b->nprob);
      return (mg_status)st[i];
    }
  return MG_OK;
}

mg_status mg_batch_info(const mg_batch* b, int* cluster, int* nteams, int* smem_bytes, int64_t* launches) {
  if (!b) return MG_ERR_ARG;
  if (cluster) *cluster = b->C;
  if (nteams) *nteams = b->nteams;
  if (smem_bytes) *smem_bytes = b->smem;
  if (launches) *launches = b->launches;
  return MG_OK;
}

}  // extern "C"
