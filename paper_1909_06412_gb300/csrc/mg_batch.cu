// Batched propagation: many independent moving grids of uneven sizes and
// potentials in one persistent launch.
//
// The launch is a set of thread-block clusters ("teams").  Each team works
// through its own list of whole problems (balanced by the host,
// longest-processing-time first).  A problem is propagated exactly as the
// single-grid kernel propagates it (same passes, same fused multipliers and
// reductions, same centre updates, Sec. II.G), with three differences that
// come from the smaller team:
//   - the tiles of a pass are dealt out over the team's CTAs, and the passes
//     are separated by a cluster barrier instead of a grid barrier;
//   - the per-CTA reduction records live in shared memory and every CTA sums
//     the team's records itself, in rank order, through distributed shared
//     memory (identical results in every CTA, so every branch on them is
//     uniform across the team);
//   - every CTA builds the per-axis multiplier tables for itself, straight
//     into shared memory, so a table needs no barrier between CTAs.
// The grids stay in global memory (for a batch of small grids, in L2) and are
// streamed through shared memory by the TMA engine pass by pass.
//
// The cluster barrier is a hardware barrier that every CTA of a team reaches
// the same number of times: the problem lists, the run parameters and every
// reduction result are identical across a team.  The copy waits of the
// streamed passes are bounded as in the single-grid kernel.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_device.cuh"

namespace cg = cooperative_groups;

namespace mgk {
namespace {

// Problems of a batch have at most this many axes (per-thread arrays of the
// passes are sized by it).
constexpr int BATCH_MAXD = 3;

// Shared-memory layout of the batched kernel (matches batch_smem_bytes on the host).
template <typename V> __device__ Smem<V> batch_carve(const BatchArgs& BA, unsigned char* base) {
  Smem<V> s;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += (bytes + 15) & ~size_t(15);
    return p;
  };
  const int TT = BA.tab_total;
  s.tw = (V*)take(sizeof(V) * TT);
  s.tA = (V*)take(sizeof(V) * TT);
  s.tAi = (V*)take(sizeof(V) * TT);
  s.tK = (V*)take(sizeof(V) * TT);
  s.tv = (double*)take(sizeof(double) * NVCOL * TT);
  s.tc = (double*)take(sizeof(double) * TT);
  s.te = nullptr;
  s.sct = (double2*)take(sizeof(double2) * 256);
  s.red = (double*)take(sizeof(double) * THREADS * (BA.D + 2));
  s.fin = (double*)take(sizeof(double) * PSTRIDE);
  s.sc = (double*)take(sizeof(double) * SC_N);
  s.reg[0] = (V*)take(BA.region_bytes);
  s.reg[1] = (V*)take(BA.region_bytes);
  s.reg[2] = (V*)take(BA.region_bytes);
  s.mbar = (uint64_t*)take(sizeof(uint64_t) * 3);
  s.mphase = (unsigned*)take(sizeof(unsigned) * 4);
  s.tb = (int64_t*)take(sizeof(int64_t) * BA.max_tiles);
  s.li = (uint16_t*)take(sizeof(uint16_t) * BA.max_lines * BA.D);
  s.end = off;
  return s;
}

__device__ __forceinline__ void team_sync(const cg::cluster_group& cl, int C) {
  if (C > 1) cl.sync();
  else __syncthreads();
}

// Team-wide sum of the records of `slot` (written by the passes into `rec`),
// in rank order, into S.fin.  Includes the team barrier that orders the
// records (and the pass's global stores) before their use.
template <typename V>
__device__ void team_finish(const cg::cluster_group& cl, int C, const Smem<V>& S, double* rec, int slot, int nv) {
  team_sync(cl, C);
  if (threadIdx.x < nv) {
    double s = 0;
    for (int r = 0; r < C; ++r) {
      const double* rr = C > 1 ? cl.map_shared_rank(rec, r) : rec;
      s += rr[slot * PSTRIDE + threadIdx.x];
    }
    S.fin[threadIdx.x] = s;
  }
  __syncthreads();
}

// One problem from its current centre for the batch's run parameters.
template <typename T, int KIND>
__device__ __noinline__ void run_problem(const Plan& P, const BatchProb& Q, const BatchArgs& BA, int pi,
                            const Smem<typename VT<T>::v>& S, const cg::cluster_group& cl, int C, int rank,
                            double* rec) {
  using V = typename VT<T>::v;
  const int D = P.D, TT = P.tab_total;
  double* sc = S.sc;
  Bufs B{};
  B.psi = Q.psi;
  B.status = Q.status;
  for (int i = threadIdx.x; i < SC_N; i += blockDim.x) sc[i] = 0.0;
  __syncthreads();
  if (threadIdx.x < D) {
    sc[SC_Q + threadIdx.x] = __ldcg(Q.ctrl + threadIdx.x);
    sc[SC_P + threadIdx.x] = __ldcg(Q.ctrl + 8 + threadIdx.x);
  }
  for (int e = threadIdx.x; e < TT; e += blockDim.x) {
    S.tw[e] = from_d2<V>(__ldg(Q.tw + e));
    S.tc[e] = __ldg(Q.tc + e);
  }
  __syncthreads();
  build_tables_local(P, S, TB_A);
  __syncthreads();

  Run RN{};
  RN.n_steps = BA.run->n_steps;
  RN.S = BA.run->S;
  RN.split = BA.run->split;
  RN.motion = BA.run->motion;
  RN.lead_v = RN.split != SPLIT_TVT;
  RN.n_units = RN.split == SPLIT_TVT ? RN.n_steps * RN.S + 1 : RN.n_steps * RN.S;
  RN.dt = BA.dt[pi];
  const double* gam = BA.run->gamma;

  PassArgs base{};
  base.bid = rank;
  base.nb = C;
  base.rec = rec;
  base.src = Q.psi;
  base.dst = Q.psi;
  int res = -1;

  if (RN.lead_v) {
    if (threadIdx.x == 0) {
      const double sig = (RN.split == SPLIT_VTV ? 0.5 : 1.0) * gam[0] * RN.dt;
      sc[SC_SIG] = sig;
      sc[SC_SGH] = -sig / P.hbar;
    }
    if (threadIdx.x < D) sc[SC_QN + threadIdx.x] = sc[SC_Q + threadIdx.x];
    __syncthreads();
    build_tables_local(P, S, TB_V);
    __syncthreads();
    PassArgs a = base;
    a.l = D - 1; a.fft = 0; a.red = RED_V; a.slot = 1;
    res = axis_pass<T, false, KIND, BATCH_MAXD>(P, B, a, S, res);
    team_finish(cl, C, S, rec, 1, D + 1);
    centre_after_potential(P, S, RN.motion);
    if (sc[SC_ERR] != 0.0) goto done;
    build_tables_local(P, S, TB_A);
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
      PassArgs a = base;
      a.l = D - 1 - i; a.fft = 1; a.pre = PRE_A;
      a.red = last ? RED_KIN : RED_NONE; a.slot = 0;
      res = axis_pass<T, false, KIND, BATCH_MAXD>(P, B, a, S, res);
      if (!last) team_sync(cl, C);
    }
    team_finish(cl, C, S, rec, 0, D + 1);
    centre_after_kinetic(P, S, RN.motion);
    if (sc[SC_ERR] != 0.0) goto done;
    build_tables_local(P, S, TB_K | (hasv ? TB_V : 0));
    if (threadIdx.x < D) sc[SC_Q + threadIdx.x] = sc[SC_QN + threadIdx.x];
    __syncthreads();
    // inverse transform, potential substep fused into the last pass
    for (int i = 0; i < D; ++i) {
      const bool last = (i == D - 1);
      PassArgs a = base;
      a.l = i; a.fft = 1; a.pre = PRE_K; a.post = 1;
      a.red = (last && hasv) ? RED_V : RED_NONE; a.slot = 1;
      res = axis_pass<T, true, KIND, BATCH_MAXD>(P, B, a, S, res);
      if (!last) team_sync(cl, C);
    }
    if (hasv) {
      team_finish(cl, C, S, rec, 1, D + 1);
      centre_after_potential(P, S, RN.motion);
      if (sc[SC_ERR] != 0.0) goto done;
      build_tables_local(P, S, TB_A);
      __syncthreads();
    }
  }
done:
  if (rank == 0 && threadIdx.x == 0) {
    for (int a = 0; a < D; ++a) {
      Q.ctrl[a] = sc[SC_Q + a];
      Q.ctrl[8 + a] = sc[SC_P + a];
    }
    const int st = (int)sc[SC_ERR];
    if (st != 0) {
      atomicExch(Q.status, st);
      BA.bstatus[pi] = st;
    } else {
      // a bounded copy wait that gave up recorded its timeout in the context
      const int ws = *(volatile int*)Q.status;
      if (ws != 0) BA.bstatus[pi] = ws;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(THREADS, 1) k_batch(const __grid_constant__ BatchArgs BA) {
  using V = typename VT<T>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Plan sP;
  __shared__ __align__(16) double rec[2 * PSTRIDE];
  const cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int team = (int)(blockIdx.x / C);
  const Smem<V> S = batch_carve<V>(BA, smem_raw);
  for (int e = threadIdx.x; e < 256; e += blockDim.x) S.sct[e] = __ldg(BA.sct + e);
  init_mbarriers(S);
  if (team >= BA.nteams) return;  // the whole cluster leaves together
  const int i0 = BA.team_start[team], i1 = BA.team_start[team + 1];
  for (int it = i0; it < i1; ++it) {
    const int pi = BA.team_items[it];
    const BatchProb& Q = BA.probs[pi];
    {
      const int* src = (const int*)&Q.P;
      int* dst = (int*)&sP;
      for (int w = threadIdx.x; w < (int)(sizeof(Plan) / sizeof(int)); w += blockDim.x) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    switch (sP.pot_kind) {
      case POT_HARMONIC: run_problem<T, POT_HARMONIC>(sP, Q, BA, pi, S, cl, C, rank, rec); break;
      case POT_ATOM_DIATOM: run_problem<T, POT_ATOM_DIATOM>(sP, Q, BA, pi, S, cl, C, rank, rec); break;
      case POT_HENON_HEILES: run_problem<T, POT_HENON_HEILES>(sP, Q, BA, pi, S, cl, C, rank, rec); break;
      default: run_problem<T, POT_SECREST_JOHNSON>(sP, Q, BA, pi, S, cl, C, rank, rec); break;
    }
    // no CTA rewrites its tables, records or plan copy while a peer may still read them
    team_sync(cl, C);
  }
}

}  // namespace

void* batch_kernel(int prec) { return prec ? (void*)k_batch<float> : (void*)k_batch<double>; }

}  // namespace mgk
