// Reversible adjoint of the moving-grid propagation (FP64, shared-memory
// resident grids).
//
// One persistent cooperative kernel walks the kinetic units of a finished
// mg_propagate call backwards.  It carries the state (u, q, p) and its
// cotangent (ubar, qbar, pbar) through every substep, where
// dJ = Re sum conj(ubar) du + qbar.dq + pbar.dp.  There is no tape: each
// substep is undone with the same substep at the negated time, which is exact
// because the integrator is time-reversible (Sec. II.G).  The same passes
// apply the substep's vector-Jacobian product.
//
// Potential substep u' = e^{-i s V/hbar} u, p' = p - s g
// (eq:eom_pt_solution_case_III_V), with gbar = -s pbar':
//   ubar = e^{+i s V/hbar} ubar' + 2 [gbar.(grad V - g)/n] u,
//   Vbar = (s/hbar) Im(conj(ubar') u'),
//   qbar += sum [Vbar grad V + (Hess V gbar) |u|^2/n],
//   thetabar += sum [Vbar dV/dtheta + (d grad V/dtheta . gbar) |u|^2/n].
// The term -2 (gbar.g/n) u is a real multiple of u.  It changes no later
// reduction (each involves Im of conj(ubar) times u-like terms), and substeps
// map it linearly onto the regenerated u.  So it accumulates in one scalar
// beta and is added at t = 0.
// Kinetic substep (eq:T_split_substep_adaptive) in the transform frame
// phi = F(A u), phi' = K phi, u' = conj(A)/N F^-1 phi', with phibar' =
// F(A ubar'):
//   deltabar = qbar' - (1/hbar) sum p^K Im(conj(phibar') phi') / N,
//   pibar = tau m^-1 deltabar,
//   ubar = conj(A)/N F^-1 conj(K) [phibar' + 2 s_K phi'],
//     with s_K = pibar.(p^K - pi)/n,
//   pbar += pibar - (1/hbar) sum (delta - tau m^-1 p^K) Im(conj(phibar') phi') / N
//           + (1/hbar) sum y Im(conj(ubar) u) - (1/hbar) sum y Im(conj(ubar') u'),
//     where y_J = (j - N/2) dq comes from dA/dp.
// The oracle's taped gradient (oracle/adjoint.py) derives the same products
// from the literal operators.  It is checked against finite differences.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_device.cuh"

namespace mgk {

namespace {

constexpr int ASTRIDE = 32;  // doubles per CTA record of the adjoint
enum { AD_FWD = 0, AD_INV = 1, AD_VREV = 2, AD_FLUSH = 3 };

// adjoint scalar slots (doubles) following the forward ones
enum { SA_QB = 40, SA_PB = 48, SA_PI = 56, SA_DB = 64, SA_PIB = 72, SA_GB = 80, SA_S1 = 88, SA_S0 = 96,
       SA_BETA = 97, SA_TH = 98, SA_N = 104 };

// V, grad V, Hessian, dV/dtheta and d(grad V)/dtheta at one point x, directly
// from the potential's formula.  Theta for the atom-diatom model is
// (Dm, a, beta, A); the harmonic potential has no differentiated parameters.
template <int KIND>
__device__ void vderiv(const Plan& P, const double* x, double& V, double* G, double* H, double* dV,
                       double* dG) {
  const int D = P.D;
  if (KIND == POT_HARMONIC) {
    double d[MAXD];
    for (int a = 0; a < D; ++a) d[a] = x[a] - P.pot[D * D + a];
    V = 0;
    for (int a = 0; a < D; ++a) {
      double s = 0;
      for (int b = 0; b < D; ++b) {
        s += P.pot[a * D + b] * d[b];
        H[a * D + b] = P.pot[a * D + b];
      }
      G[a] = s;
      V += 0.5 * d[a] * s;
    }
  } else {  // POT_ATOM_DIATOM, axes (R, r)
    const double Dm = P.pot[0], aa = P.pot[1], re = P.pot[2], A = P.pot[3], be = P.pot[4];
    const double R = x[0], r = x[1];
    const double E = exp(-aa * (r - re));
    const double ep = exp(0.5 * be * r), en = exp(-0.5 * be * r);
    const double h = ep + en, sh = ep - en, hp = 0.5 * be * sh;
    const double gR = A * exp(-be * R);
    const double f = Dm * (1.0 - E) * (1.0 - E);
    const double fp = 2.0 * Dm * aa * (E - E * E);
    const double fpp = 2.0 * Dm * aa * aa * E * (2.0 * E - 1.0);
    V = f + gR * h;
    G[0] = -be * gR * h;
    G[1] = fp + gR * hp;
    H[0] = be * be * gR * h;
    H[1] = H[2] = -be * gR * hp;
    H[3] = fpp + 0.25 * be * be * gR * h;
    dV[0] = (1.0 - E) * (1.0 - E);
    dV[1] = 2.0 * Dm * (1.0 - E) * E * (r - re);
    dV[2] = -R * gR * h + 0.5 * gR * r * sh;
    dV[3] = gR * h / A;
    dG[0] = 0.0;
    dG[1] = fp / Dm;
    dG[2] = 0.0;
    dG[3] = 2.0 * Dm * ((E - E * E) - aa * (r - re) * E * (1.0 - 2.0 * E));
    dG[4] = -gR * h + be * R * gR * h - 0.5 * be * gR * r * sh;
    dG[5] = -R * gR * hp + gR * (0.5 * sh + 0.25 * be * r * h);
    dG[6] = -be * gR * h / A;
    dG[7] = gR * hp / A;
  }
}

// Per-CTA records of reduction `slot` (two slots alternate, so that a CTA
// writing the next reduction never overtakes one still reading the last).
template <typename V>
__device__ void adj_partials(const Bufs& B, const Smem<V>& S, int slot, const double* acc, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nt = blockDim.x;
  for (int v = 0; v < nv; ++v) S.red[v * nt + threadIdx.x] = acc[v];
  __syncthreads();
  for (int v = warp; v < nv; v += nt >> 5) {
    double s = 0;
    for (int k = lane; k < nt; k += 32) s += S.red[v * nt + k];
    s = warp_sum(s);
    if (lane == 0) __stcg(B.part + ((size_t)slot * gridDim.x + blockIdx.x) * ASTRIDE + v, s);
  }
  __syncthreads();
}
// Fixed-order sum of the records of `slot` over CTAs into out (shared memory).
__device__ void adj_finish(const Bufs& B, int slot, double* out, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = warp; v < nv; v += blockDim.x >> 5) {
    double s = 0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(B.part + ((size_t)slot * gridDim.x + b) * ASTRIDE + v);
    s = warp_sum(s);
    if (lane == 0) out[v] = s;
  }
  __syncthreads();
}

struct AdjPass {
  int l, mode, first, last, from_smem, keep;
};

// One dual pass along axis l over (u, ubar); acc accumulates this phase's
// reductions across its passes.  Returns the smem region holding the result.
template <int KIND>
__device__ int adj_pass(const Plan& P, const Bufs& B, const AdjRun& AR, const AdjPass& A, const Smem<double2>& S,
                        double2* const* breg, int res_in, double* acc) {
  using V = double2;
  const AxisPlan& ax = P.ax[A.l];
  const int n = ax.n, W = ax.W, D = P.D;
  const bool contig = (A.l == D - 1);
  const int wsh = contig ? 0 : __ffs(W) - 1;
  const int64_t s = ax.stride;
  const int64_t tpo = contig ? 1 : s / W;
  const int64_t ws = contig ? n : 1, es = contig ? 1 : s;
  const double* sc = S.sc;
  const double hb = P.hbar;
  const V* tw = S.tw + ax.toff;
  const V* pre = A.mode == AD_FWD ? S.tA + ax.toff : (A.mode == AD_INV ? S.tK + ax.toff : nullptr);
  const V* post = A.mode == AD_INV ? S.tAi + ax.toff : nullptr;
  V* ug = (V*)B.psi;
  V* bg = (V*)AR.ubar;
  const int64_t bid = blockIdx.x, nb = gridDim.x;
  const int64_t mine = bid < ax.ntiles ? (ax.ntiles - bid + nb - 1) / nb : 0;
  const int chunk = A.from_smem || A.keep ? (int)mine : ax.tpc;
  int res = -1;
  for (int64_t c0 = 0; c0 < mine; c0 += chunk) {
    const int nt = (int)(mine - c0 < chunk ? mine - c0 : chunk);
    const int cnt = nt * W * n;
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      const int64_t t = bid + (c0 + k) * nb;
      const int64_t o = t / tpo;
      S.tb[k] = contig ? t * W * n : o * n * s + (t - o * tpo) * W;
    }
    for (int kw = threadIdx.x; kw < nt * W; kw += blockDim.x) {
      const int k = kw / W, w = kw - k * W;
      const int64_t t = bid + (c0 + k) * nb;
      const int64_t o = t / tpo;
      int idx[MAXD];
      decode(P, A.l, contig ? (unsigned)(t * W + w) : (unsigned)o,
             contig ? 0u : (unsigned)((t - o * tpo) * W + w), 0, idx);
      for (int a = 0; a < D; ++a) S.li[kw * D + a] = (uint16_t)idx[a];
    }
    __syncthreads();
    V *cu, *ou, *cb, *ob;
    if (A.from_smem) {
      cu = S.reg[res_in];
      ou = S.reg[res_in ^ 1];
      cb = breg[res_in];
      ob = breg[res_in ^ 1];
    } else {
      cu = S.reg[0];
      ou = S.reg[1];
      cb = breg[0];
      ob = breg[1];
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int ti = e / (W * n);
        const int rem = e - ti * W * n;
        const int w = contig ? rem / n : rem & (W - 1);
        const int j = contig ? rem - w * n : rem >> wsh;
        const int64_t gi = S.tb[ti] + j * es + w * ws;
        cu[e] = __ldcg(ug + gi);
        cb[e] = __ldcg(bg + gi);
      }
      __syncthreads();
    }
    // per-element index helper
    auto coords = [&](int e, int* idx, int& j) {
      const int ti = e / (W * n);
      const int rem = e - ti * W * n;
      const int w = contig ? rem / n : rem & (W - 1);
      j = contig ? rem - w * n : rem >> wsh;
      for (int a = 0; a < D; ++a) idx[a] = S.li[(ti * W + w) * D + a];
      idx[A.l] = j;
      return ti;
    };
    // prologues
    if (A.mode == AD_FWD && A.first) {  // q-space: sum y Im(conj(ubar') u')
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int idx[MAXD], j;
        coords(e, idx, j);
        const double im = cb[e].x * cu[e].y - cb[e].y * cu[e].x;  // Im(conj(ub) u)
        for (int a = 0; a < D; ++a) acc[a] += S.tc[P.ax[a].toff + idx[a]] * P.dq[a] * im;
      }
    }
    if (A.mode == AD_INV && A.first) {  // p-space: phibar += 2 s_K phi'
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int idx[MAXD], j;
        coords(e, idx, j);
        double sk = sc[SA_S0];
        for (int a = 0; a < D; ++a) sk = fma(sc[SA_S1 + a], S.tc[P.ax[a].toff + idx[a]], sk);
        cb[e] = V{fma(2.0 * sk, cu[e].x, cb[e].x), fma(2.0 * sk, cu[e].y, cb[e].y)};
      }
      __syncthreads();
    }
    if (A.mode == AD_FWD || A.mode == AD_INV) {
      V* ru = (A.mode == AD_FWD) ? stockham<false>(cu, ou, nt * W, ax, tw, pre, wsh)
                                 : stockham<true>(cu, ou, nt * W, ax, tw, pre, wsh);
      V* rb = (A.mode == AD_FWD) ? stockham<false>(cb, ob, nt * W, ax, tw, pre, wsh)
                                 : stockham<true>(cb, ob, nt * W, ax, tw, pre, wsh);
      cu = ru;
      cb = rb;
    }
    // epilogue
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      int idx[MAXD], j;
      const int ti = coords(e, idx, j);
      const int rem = e - ti * W * n;
      const int w = contig ? rem / n : rem & (W - 1);
      V u = cu[e], b = cb[e];
      if (post) {
        u = cmul(u, post[j]);
        b = cmul(b, post[j]);
      }
      if (A.mode == AD_FWD && A.last) {  // p-space moments
        const double rho = u.x * u.x + u.y * u.y;
        const double im = b.x * u.y - b.y * u.x;  // Im(conj(phibar') phi')
        acc[D] += rho;
        acc[2 * D + 1] += im;
        for (int a = 0; a < D; ++a) {
          const double c = S.tc[P.ax[a].toff + idx[a]];
          acc[D + 1 + a] += c * rho;
          acc[2 * D + 2 + a] += c * im;
        }
      } else if (A.mode == AD_INV && A.last) {  // q-space: sum y Im(conj(ubar) u)
        const double im = b.x * u.y - b.y * u.x;
        for (int a = 0; a < D; ++a) acc[a] += S.tc[P.ax[a].toff + idx[a]] * P.dq[a] * im;
      } else if (A.mode == AD_VREV) {
        const double sig = sc[SC_SIG];
        double x[MAXD], Vv, G[MAXD], H[MAXD * MAXD], dV[4] = {0, 0, 0, 0}, dG[4 * MAXD];
        for (int a = 0; a < D; ++a) x[a] = fma(S.tc[P.ax[a].toff + idx[a]], P.dq[a], sc[SC_Q + a]);
        vderiv<KIND>(P, x, Vv, G, H, dV, dG);
        const double w2 = u.x * u.x + u.y * u.y;
        const double im = b.x * u.y - b.y * u.x;  // Im(conj(ubar') u')
        const double Vb = sig / hb * im;
        double sn, cs;
        expi_tab(sig * Vv / hb, S.sct, sn, cs);  // e^{+i s V / hbar}
        const V ur = V{u.x * cs - u.y * sn, u.x * sn + u.y * cs};
        const V br = V{b.x * cs - b.y * sn, b.x * sn + b.y * cs};
        double gdot = 0;
        for (int a = 0; a < D; ++a) gdot += sc[SA_GB + a] * G[a];
        const double k2 = 2.0 * gdot / AR.norm;
        u = ur;
        b = V{fma(k2, ur.x, br.x), fma(k2, ur.y, br.y)};
        acc[0] += w2;
        for (int a = 0; a < D; ++a) {
          double hg = 0;
          for (int c = 0; c < D; ++c) hg += H[a * D + c] * sc[SA_GB + c];
          acc[1 + a] += G[a] * w2;
          acc[1 + D + a] += Vb * G[a] + hg * w2 / AR.norm;
        }
        for (int k = 0; k < AR.ntheta; ++k) {
          double dgg = 0;
          for (int a = 0; a < D; ++a) dgg += dG[k * D + a] * sc[SA_GB + a];
          acc[1 + 2 * D + k] += Vb * dV[k] + dgg * w2 / AR.norm;
        }
      } else if (A.mode == AD_FLUSH) {  // ubar_0 = stored ubar + beta u_0
        const double beta = sc[SA_BETA];
        b = V{fma(beta, u.x, b.x), fma(beta, u.y, b.y)};
      }
      if (A.keep) {
        cu[e] = u;
        cb[e] = b;
      } else {
        const int64_t gi = S.tb[ti] + j * es + w * ws;
        __stcg(ug + gi, u);
        __stcg(bg + gi, b);
      }
    }
    __syncthreads();
    res = cu == S.reg[0] ? 0 : 1;
  }
  return res;
}

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1)
    k_adjoint(const __grid_constant__ Plan P, const __grid_constant__ Bufs B, const __grid_constant__ AdjRun AR) {
  using V = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sflag;
  const Smem<V> S = carve<V>(P, B, smem_raw);
  // two more data regions for ubar, after the forward layout
  double2* breg[2];
  {
    size_t off = S.end;
    breg[0] = (double2*)(smem_raw + off);
    breg[1] = (double2*)(smem_raw + off + (((size_t)P.region_bytes + 15) & ~size_t(15)));
  }
  const int D = P.D;
  const Run& RN = AR.R;
  if (__ldcg(B.status) != ST_OK) return;
  double* sc = S.sc;
  for (int i = threadIdx.x; i < SA_N; i += blockDim.x) sc[i] = 0.0;
  __syncthreads();
  if (threadIdx.x < D) {
    sc[SC_Q + threadIdx.x] = __ldcg(B.ctrl + threadIdx.x);
    sc[SC_P + threadIdx.x] = __ldcg(B.ctrl + 8 + threadIdx.x);
    sc[SA_QB + threadIdx.x] = __ldcg(B.ctrl + 20 + threadIdx.x);
    sc[SA_PB + threadIdx.x] = __ldcg(B.ctrl + 28 + threadIdx.x);
  }
  load_tables(P, B, S, LT_TW | LT_A | LT_C | LT_SCT);
  __syncthreads();
  const double* gam = B.gamma;
  double acc[ASTRIDE];
  // finished sums: the reduction scratch is free once the records are written
  double* const fin = S.red;
  int slot = 0;
  int res = -1;
  bool kept = false;
  const double hb = P.hbar;
  const double Ntot = (double)P.npts;

  auto vrev = [&](double sig) -> bool {
    // potential substep backwards: regenerate u, p; cotangents; beta
    if (threadIdx.x == 0) sc[SC_SIG] = sig;
    if (threadIdx.x < D) sc[SA_GB + threadIdx.x] = RN.motion == GRID_FIXED ? 0.0 : -sig * sc[SA_PB + threadIdx.x];
    __syncthreads();
    for (int v = 0; v < ASTRIDE; ++v) acc[v] = 0;
    AdjPass a{D - 1, AD_VREV, 1, 1, kept ? 1 : 0, 1};
    res = adj_pass<KIND>(P, B, AR, a, S, breg, res, acc);
    kept = true;
    adj_partials(B, S, slot, acc, 1 + 2 * D + AR.ntheta);
    if (!grid_sync(B, &sflag)) return false;
    adj_finish(B, slot, fin, 1 + 2 * D + AR.ntheta);
    slot ^= 1;
    if (threadIdx.x == 0) {
      const double n = fin[0];
      double gg = 0;
      for (int b = 0; b < D; ++b) {
        const double g = fin[1 + b] / n;
        gg += sc[SA_GB + b] * g;
        if (RN.motion != GRID_FIXED) sc[SC_P + b] += sig * g;
        sc[SA_QB + b] += fin[1 + D + b];
      }
      for (int k = 0; k < AR.ntheta; ++k) sc[SA_TH + k] += fin[1 + 2 * D + k];
      sc[SA_BETA] += -2.0 * gg / AR.norm;
    }
    __syncthreads();
    build_tables(P, B, S, TB_A);
    if (!grid_sync(B, &sflag)) return false;
    load_tables(P, B, S, LT_A);
    __syncthreads();
    return true;
  };

  auto trev = [&](double tau) -> bool {
    // forward transforms of (u', ubar') with the moments of the p-space pass
    for (int v = 0; v < ASTRIDE; ++v) acc[v] = 0;
    for (int i = 0; i < D; ++i) {
      const bool last = (i == D - 1);
      AdjPass a{D - 1 - i, AD_FWD, i == 0, last, (i == 0 && kept) ? 1 : 0, last ? 1 : 0};
      res = adj_pass<KIND>(P, B, AR, a, S, breg, res, acc);
      kept = a.keep;
      if (!last && !grid_sync(B, &sflag)) return false;
    }
    adj_partials(B, S, slot, acc, 3 * D + 2);
    if (!grid_sync(B, &sflag)) return false;
    adj_finish(B, slot, fin, 3 * D + 2);
    slot ^= 1;
    if (threadIdx.x == 0) {
      const double np = fin[D], sim = fin[2 * D + 1];
      const double nu = np / Ntot;
      double s0 = 0;
      for (int b = 0; b < D; ++b) {
        const double p = sc[SC_P + b];
        const double pi = p + P.dp[b] * fin[D + 1 + b] / np;
        const double mom = RN.motion == GRID_ADAPTIVE ? pi : p;
        const double delta = RN.motion == GRID_FIXED ? 0.0 : tau * P.minv[b] * mom;
        const double spim = p * sim + P.dp[b] * fin[2 * D + 2 + b];  // sum p^K im
        const double deltab = sc[SA_QB + b] - spim / (hb * Ntot);
        const double pib = RN.motion == GRID_ADAPTIVE ? tau * P.minv[b] * deltab : 0.0;
        double pbn = sc[SA_PB + b] + pib;
        if (RN.motion == GRID_CENTRE_P) pbn += tau * P.minv[b] * deltab;
        pbn -= (delta * sim - tau * P.minv[b] * spim) / (hb * Ntot);
        pbn -= fin[b] / hb;  // - (1/hbar) sum y Im(conj(ubar') u')
        sc[SA_PB + b] = pbn;
        sc[SC_DELTA + b] = -delta;  // regeneration: K with -tau, -delta
        sc[SC_Q + b] -= delta;
        s0 += pib * (p - pi);
        sc[SA_S1 + b] = pib * P.dp[b] / nu;
      }
      sc[SA_S0] = s0 / nu;
      sc[SC_TAU] = -tau;
    }
    __syncthreads();
    build_tables(P, B, S, TB_K);
    if (!grid_sync(B, &sflag)) return false;
    load_tables(P, B, S, LT_K);
    __syncthreads();
    // inverse transforms; q-space moment of (ubar, u) on the last pass
    for (int v = 0; v < ASTRIDE; ++v) acc[v] = 0;
    for (int i = 0; i < D; ++i) {
      const bool last = (i == D - 1);
      AdjPass a{i, AD_INV, i == 0, last, (i == 0 && kept) ? 1 : 0, last ? 1 : 0};
      res = adj_pass<KIND>(P, B, AR, a, S, breg, res, acc);
      kept = a.keep;
      if (!last && !grid_sync(B, &sflag)) return false;
    }
    adj_partials(B, S, slot, acc, D);
    if (!grid_sync(B, &sflag)) return false;
    adj_finish(B, slot, fin, D);
    slot ^= 1;
    if (threadIdx.x == 0)
      for (int b = 0; b < D; ++b) sc[SA_PB + b] += fin[b] / hb;
    __syncthreads();
    return true;
  };

  for (int64_t u = RN.n_units - 1; u >= 0; --u) {
    double tau, sig;
    bool hasv;
    unit_coeffs(RN, gam, u, tau, sig, hasv);
    if (hasv && !vrev(sig)) return;
    if (!trev(tau)) return;
  }
  if (RN.lead_v) {
    const double sig = (RN.split == SPLIT_VTV ? 0.5 : 1.0) * gam[0] * RN.dt;
    if (!vrev(sig)) return;
  }
  // ubar_0 = stored ubar + beta u_0; write both arrays back
  {
    for (int v = 0; v < ASTRIDE; ++v) acc[v] = 0;
    AdjPass a{D - 1, AD_FLUSH, 1, 1, kept ? 1 : 0, 0};
    adj_pass<KIND>(P, B, AR, a, S, breg, res, acc);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int a = 0; a < D; ++a) {
      B.ctrl[a] = sc[SC_Q + a];
      B.ctrl[8 + a] = sc[SC_P + a];
      B.ctrl[20 + a] = sc[SA_QB + a];
      B.ctrl[28 + a] = sc[SA_PB + a];
    }
    for (int k = 0; k < 4; ++k) B.ctrl[36 + k] = sc[SA_TH + k];
  }
}

}  // namespace

void* adjoint_kernel(int kind) {
  if (kind == POT_HARMONIC) return (void*)k_adjoint<POT_HARMONIC>;
  if (kind == POT_ATOM_DIATOM) return (void*)k_adjoint<POT_ATOM_DIATOM>;
  return nullptr;
}

}  // namespace mgk
