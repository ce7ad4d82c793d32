// Plain-old-data descriptors shared by the host planner (mg_capi.cu) and the
// device kernels.  No CUDA types beyond double2.
#pragma once
#include <stdint.h>
#include <vector_types.h>

namespace mgk {

constexpr int MAXD = 8;        // axes
constexpr int MAXRAD = 12;     // Stockham passes per axis
constexpr int MAXN = 2048;     // longest axis
constexpr int PSTRIDE = 16;    // doubles per CTA partial-sum record
constexpr int NVCOL = 5;       // potential-table columns per axis
constexpr int MAX_STAGES = 625;
constexpr int THREADS = 256;   // threads per CTA of every kernel
constexpr int SCALARS = 112;   // double slots of per-CTA scalar state in shared memory
constexpr int CTRL = 64;       // doubles of the control block in the workspace

enum { POT_HARMONIC = 0, POT_ATOM_DIATOM = 1, POT_HENON_HEILES = 2, POT_SECREST_JOHNSON = 3 };
enum { SPLIT_TVT = 0, SPLIT_VTV = 1, SPLIT_TV = 2 };
enum { GRID_ADAPTIVE = 0, GRID_CENTRE_P = 1, GRID_FIXED = 2 };
// Per-axis tables too large for shared memory (long axes) stay in the workspace:
// TG_COLS the potential columns, k - N/2 and the kinetic energies; TG_MULT
// (FP64 only) the multipliers A, conj(A)/N and K.
enum { TG_COLS = 1, TG_MULT = 2 };
enum { ST_OK = 0, ST_TIMEOUT = -4, ST_NONFINITE = -5, ST_UNSTABLE = -6 };

// One axis of the tensor-product grid and how its 1D transforms are tiled.
struct AxisPlan {
  int n;                 // points on the axis (N_l)
  int nrad;              // Stockham passes
  int rad[MAXRAD];       // radix of each pass (2, 3, 4 or 8)
  int W;                 // lines per tile (adjacent in the contiguous index)
  int tpc;               // tiles a CTA processes per smem chunk
  int toff;              // offset of this axis in the per-axis tables
  int64_t stride;        // element stride of the axis (prod of N_m, m > l)
  int64_t outer;         // prod of N_m, m < l
  int64_t ntiles;        // tiles in one pass over the whole grid
};

struct Plan {
  int D;
  int prec;              // 0 = FP64, 1 = FP32 storage
  int nblocks;           // CTAs of the persistent kernel (all co-resident)
  int resident;          // tiles of axes 0 and D-1 stay in smem across barriers
  int maxn;              // longest axis
  int tab_total;         // sum of N_l
  int region_bytes;      // bytes of each of the two smem data regions
  int smem_bytes;        // dynamic smem per CTA
  int max_tiles;         // most tiles in one smem chunk (any axis)
  int max_lines;         // most lines in one smem chunk (any axis)
  int tab_global;        // TG_* bits: per-axis tables read from the workspace, not shared memory
  int64_t npts;
  int64_t N[MAXD];
  double dq[MAXD], dp[MAXD], minv[MAXD], hbar;  // minv: diagonal of the inverse mass matrix
  double minvf[MAXD * MAXD];  // the full symmetric inverse mass matrix, row-major D x D
  int minv_general;           // minvf has nonzero off-diagonal entries (general kernel only)
  AxisPlan ax[MAXD];
  int pot_kind;
  int pot_general;       // harmonic potential with a non-diagonal K
  double pot[MAXD * MAXD + MAXD];
};

// Device buffers, all inside the caller's workspace except psi.
struct Bufs {
  void* psi;             // scaled state u (complex128 or complex64)
  double* ctrl;          // [0,8) q, [8,16) p, [16] t
  unsigned* bar;         // grid barrier: one 64-bit word (generation, arrivals)
  int* status;
  double* part;          // [2][nblocks][PSTRIDE] per-CTA partial sums
  double2* tw;           // forward twiddles e^{-2 pi i m / N_l}, per axis
  double2* tabA;         // A_l[j] = (-1)^j e^{-i p_l (j - N_l/2) dq_l / hbar}
  double2* tabAi;        // conj(A_l[j]) / N_l
  double2* tabK;         // kinetic multiplier per axis (Sec. II.G.2, with the grid shift)
  double* tabV;          // [NVCOL][tab_total] potential columns
  double* tabC;          // k - N_l/2 as double
  double* tabE;          // per-axis kinetic energy minv_l (p_l^K)^2 / 2
  const double* gamma;   // composition coefficients
  double2* sct;          // 256 entries e^{i k pi / 128}
  double2* scratch;      // npts complex128 (observables, host staging)
  uint64_t bar_limit_ns; // time limit of a grid-barrier wait (0 = the default 5 s)
};

// One persistent launch.
struct Run {
  int64_t n_units;       // kinetic units (each optionally followed by a fused V)
  int64_t n_steps;
  int split, motion, S, lead_v;
  double dt;
};

// One adjoint launch (the propagation it reverses, and the cotangent buffer).
struct AdjRun {
  Run R;
  void* ubar;            // device complex128 cotangent of psi (in: at t_end; out: at t_start)
  int ntheta;            // potential parameters differentiated (4 for atom-diatom)
  double norm;           // sum |u|^2, an invariant of the propagation
};

// ---- batched launch: many independent grids, one cluster of CTAs per grid ----

constexpr int MAXTEAMS = 4096;  // clusters of one batched launch

// One problem of a batch: its plan tiled for a team of CTAs, and the buffers
// of the grid context that owns it.
struct BatchProb {
  Plan P;
  void* psi;
  double* ctrl;
  int* status;
  const double2* tw;
  const double* tc;
};

// Parameters of one batched propagation (uploaded by the launch itself).
struct BatchRun {
  int64_t n_steps;
  int S, split, motion, pad;
  double gamma[MAX_STAGES];
};

struct BatchArgs {
  const BatchProb* probs;
  const int* team_start;   // [nteams + 1] offsets into team_items
  const int* team_items;   // problem indices, each team's in processing order
  const BatchRun* run;
  const double* dt;        // per problem
  int* bstatus;            // per problem: 0 or the failure status
  const double2* sct;      // 256 entries e^{i k pi / 128}
  int nteams;
  // shared-memory layout (maxima over the problems)
  int D, tab_total, region_bytes, max_tiles, max_lines, smem_bytes;
};

}  // namespace mgk
