// Plain-old-data plan of the short-axis propagation kernel (mg_short.cu),
// shared by the host planner (mg_capi.cu) and the device code.
//
// The short-axis kernel serves tensor grids whose D >= 3 axes all have the
// same short length n (8, 12 or 16 points), the shape of the 8D Henon-Heiles
// grids of Sec. III.C.  Instead of one pass over the state per axis it
// transforms a group of g consecutive axes per pass: a chunk of the state
// (whole n^g blocks of the group's axes, for several adjacent values of the
// remaining index) is staged in shared memory, and every 1D transform of the
// group is done there with one thread per line and the line held in
// registers.
#pragma once
#include <stdint.h>
#include <vector_types.h>

#include "mg_plan.h"

namespace mgk {

constexpr int SHORT_MAXG = 4;     // axes per group
constexpr int SHORT_TC_MAXG = 3;  // axes per group of the tensor-core variant (TMA plans)

// One group of consecutive axes l0 .. l0+g-1 and how its passes are chunked.
//  - contig = 1: the group ends at the last (contiguous) axis; a chunk is WT
//    consecutive blocks of n^g elements.
//  - contig = 0: a chunk is one n^g block of the group's axes for WT adjacent
//    values of the index of the axes after the group (rows of WT contiguous
//    elements, `inner` elements apart).
// Shared-memory layout of a chunk (both kinds): plane wt (a block, or one
// value of the trailing index) starts at wt * PS; inside a plane the group's
// points are stored with their last-axis lines padded to n + 1 elements, and
// PS = n^(g-1) (n + 1) (+1 for g >= 2) is odd, so that the lines one warp
// touches fall into different shared-memory banks.
struct GroupPlan {
  int l0, g;
  int contig;
  int WT;           // blocks (contig) or adjacent trailing indices (strided) per chunk
  int PS;           // elements per plane in shared memory
  int ng;           // n^g
  int64_t inner;    // element stride of axis l0+g-1
  int64_t nb;       // chunks per value of the leading index (strided)
  int64_t nblk;     // blocks of n^g in the grid (contig)
  int64_t nchunks;  // chunks in one pass
};

// An encoded TMA tensor map (CUtensorMap, 128 bytes, 64-byte aligned): opaque
// here; the device code only passes its address to cp.async.bulk.tensor.
struct alignas(64) TensorMapBytes {
  unsigned char b[128];
};

struct ShortPlan {
  int on;            // the grid has the short-axis shape and the kernel fits
  int tma;           // chunks move by TMA tensor copies (FP32, n = 16); else cp.async
  int tc;            // line DFTs on the tensor cores: 0 none, 1 3xTF32, 2 BF16x3 (FP32, n = 16, TMA)
  int trank[MAXD];   // rank of each group's tensor map
  int n;             // axis length
  int ngroups;       // grp[0] ends at the last axis, grp[ngroups-1] starts at axis 0
  int threads;       // threads per CTA
  int nblocks;       // CTAs (all co-resident, one per SM)
  int nreg;          // shared-memory chunk regions (2 or 3: prefetch depth nreg-1)
  int region_elems;  // elements of one region
  int smem_bytes;    // dynamic shared memory per CTA
  int pairs;         // potential has nearest-neighbour pair terms (Henon-Heiles)
  GroupPlan grp[MAXD];
  double2* tabB;     // [D*n] forward multiplier (A/N or A conj(A_old)/N)
  double2* tabC;     // [D*n] post-multiplier conj(A) of a launch's last inverse passes
  double2* tabF;     // [D*n] e^{-i sigma f_a(x)/hbar} per axis entry
  double2* tabP;     // [(D-1)*n*n] e^{-i sigma h_a(x_a) g_{a+1}(x_{a+1})/hbar}
  // TMA (tma = 1): one tensor map per group over psi.  The group that ends at
  // the last axis is a rank-4 view {n, n, n, blocks} (innermost first) copied
  // in boxes of {n, n, n, WT} with the 128-byte swizzle; a strided group is a
  // view {trailing index, its axes from the last, leading index} copied in
  // boxes of {WP, n, .., 1}, WP = min(WT, 256), WT / WP boxes per chunk.
  TensorMapBytes tmap[MAXD];
};

}  // namespace mgk
