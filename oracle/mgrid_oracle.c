/* Plain FP64 CPU oracle of the moving-grid split-operator integrator of
 * Choi & Vanicek (arXiv:1909.06412).  TEST INFRASTRUCTURE ONLY: the GPU
 * library is checked against it; it shares no code with that library and the
 * product path never calls it.
 *
 * Written for clarity, not speed: every operator is applied as the paper
 * states it, with no merging of substeps, no fusion and no reordering.
 * Section and equation names below are the paper's.
 */
#include "mgrid_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

struct orc_ctx {
  int D;
  int64_t N[ORC_MAXD];
  double dq[ORC_MAXD];
  double dp[ORC_MAXD];
  double minv[ORC_MAXD * ORC_MAXD];
  double hbar;
  int64_t npts;
  int pot_kind;
  double pot[ORC_MAXD * ORC_MAXD + ORC_MAXD];
  int npot;
  cplx* u;         /* scaled state u^J = psi(x^J) sqrt(prod dq) */
  double q[ORC_MAXD], p[ORC_MAXD], t;
};

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* 1D transforms (the discrete Fourier transform of Sec. II.B)              */
/* ------------------------------------------------------------------------ */

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* ------------------------------------------------------------------------ */
/* Accurate phase factors                                                   */
/* ------------------------------------------------------------------------ */
/* The phases of eq:t_definition reach tens to hundreds of radians; a plain
 * FP64 product loses ~1e-14 rad on such arguments, and those errors build up
 * over thousands of substeps.  Phase arguments are therefore accumulated as
 * unevaluated sums hi + lo (error-free products by fma, Dekker/Knuth
 * two-sum) and reduced modulo 2 pi with a two-word 2 pi before cos/sin, so
 * every factor e^{i theta} is correct to a few 1e-16 whatever |theta|. */
typedef struct { double hi, lo; } dd;

static const double TWO_PI_HI = 6.283185307179586232;      /* fl(2 pi)       */
static const double TWO_PI_LO = 2.4492935982947064e-16;    /* 2 pi - fl(2 pi) */

static dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return (dd){s, (a - (s - bb)) + (b - bb)};
}
static dd fast_two_sum(double a, double b) {
  double s = a + b;
  return (dd){s, b - (s - a)};
}
static dd dd_of_prod(double a, double b) {
  double p = a * b;
  return (dd){p, fma(a, b, -p)};
}
static dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
static dd dd_mul(dd x, dd y) {
  dd p = dd_of_prod(x.hi, y.hi);
  p.lo += x.hi * y.lo + x.lo * y.hi;
  return fast_two_sum(p.hi, p.lo);
}
static dd dd_mul_d(dd x, double b) {
  dd p = dd_of_prod(x.hi, b);
  p.lo += x.lo * b;
  return fast_two_sum(p.hi, p.lo);
}
static dd dd_div_d(dd x, double b) {
  double q1 = x.hi / b;
  dd p = dd_of_prod(q1, b);
  double r = ((x.hi - p.hi) - p.lo) + x.lo;
  return fast_two_sum(q1, r / b);
}
/* e^{i theta} for theta = hi + lo. */
static cplx expi(dd th) {
  double k = nearbyint(th.hi / TWO_PI_HI);
  dd kp = dd_of_prod(k, TWO_PI_HI);
  double r = ((th.hi - kp.hi) - kp.lo) + th.lo - k * TWO_PI_LO;
  return cos(r) + I * sin(r);
}

/* e^{sign 2 pi i m / n} with the integer m reduced modulo n first. */
static cplx root_of_unity(int64_t m, int64_t n, int sign) {
  int64_t r = m % n;
  if (r < 0) r += n;
  dd a = dd_add(dd_of_prod(TWO_PI_HI, (double)r), dd_of_prod(TWO_PI_LO, (double)r));
  a = dd_div_d(a, (double)n);
  if (sign < 0) { a.hi = -a.hi; a.lo = -a.lo; }
  return expi(a);
}

int orc_dft1d_direct(int64_t n, const double* in, double* out, int sign) {
  if (n <= 0 || (sign != 1 && sign != -1)) return -1;
  const cplx* x = (const cplx*)in;
  cplx* y = (cplx*)out;
  double s = 1.0 / sqrt((double)n);
  for (int64_t k = 0; k < n; ++k) {
    cplx acc = 0;
    for (int64_t j = 0; j < n; ++j) acc += root_of_unity(k * j, n, sign) * x[j];
    y[k] = acc * s;
  }
  return 0;
}

/* The roots of unity of the DFTs as two-word constants w = hi + lo: hi the
 * correctly rounded value, lo the rest (from extended-precision cosine and
 * sine).  A rounded twiddle is the same error in every transform; over the
 * thousands of transforms of a long run those errors add up coherently
 * (about 5e-12 on the grid centre of the 256 x 256 atom-diatom run to
 * t = 2000 a.u.), while with the lo parts the transform's rounding is that
 * of its additions and products only. */
typedef struct { cplx hi, lo; } root2;

static root2 root2_of(int64_t m, int64_t n, int sign) {
  int64_t r = m % n;
  if (r < 0) r += n;
  const long double a = (long double)sign * 6.283185307179586476925286766559L * (long double)r / (long double)n;
  const long double cl = cosl(a), sl = sinl(a);
  const double ch = (double)cl, sh = (double)sl;
  root2 w = {ch + I * sh, (double)(cl - (long double)ch) + I * (double)(sl - (long double)sh)};
  return w;
}

/* x * (w.hi + w.lo), the two products added last */
static cplx mul_root2(cplx x, root2 w) {
  const double xr = creal(x), xi = cimag(x);
  const double hr = creal(w.hi), hi = cimag(w.hi), lr = creal(w.lo), li = cimag(w.lo);
  return ((xr * hr - xi * hi) + (xr * lr - xi * li)) + I * ((xr * hi + xi * hr) + (xr * li + xi * lr));
}

/* table[m] = e^{sign 2 pi i m / n}, m = 0 .. n-1 */
static root2* root2_table(int64_t n, int sign) {
  root2* t = malloc(sizeof(root2) * (size_t)n);
  if (!t) return NULL;
  for (int64_t m = 0; m < n; ++m) t[m] = root2_of(m, n, sign);
  return t;
}

/* Iterative radix-2 Cooley-Tukey: bit-reversal permutation, then log2(n)
 * levels of butterflies; tw = root2_table(n, sign) (level len uses
 * tw[k n / len]). */
static void fft_radix2(int64_t n, cplx* x, const root2* tw) {
  for (int64_t i = 1, j = 0; i < n; ++i) {
    int64_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) { cplx tmp = x[i]; x[i] = x[j]; x[j] = tmp; }
  }
  for (int64_t len = 2; len <= n; len <<= 1) {
    int64_t half = len / 2;
    for (int64_t start = 0; start < n; start += len) {
      for (int64_t k = 0; k < half; ++k) {
        cplx a = x[start + k];
        cplx b = mul_root2(x[start + k + half], tw[k * (n / len)]);
        x[start + k] = a + b;
        x[start + k + half] = a - b;
      }
    }
  }
}

/* Unnormalised DFT of one line: radix-2 FFT or direct sum, with the roots
 * of unity tw = root2_table(n, sign). */
static int dft_line(int64_t n, cplx* x, const root2* tw) {
  if (is_pow2(n)) {
    fft_radix2(n, x, tw);
    return 0;
  }
  cplx* tmp = malloc(sizeof(cplx) * (size_t)n);
  if (!tmp) return -2;
  for (int64_t k = 0; k < n; ++k) {
    cplx acc = 0;
    for (int64_t j = 0; j < n; ++j) acc += mul_root2(x[j], tw[(k * j) % n]);
    tmp[k] = acc;
  }
  memcpy(x, tmp, sizeof(cplx) * (size_t)n);
  free(tmp);
  return 0;
}

int orc_dft1d(int64_t n, double* xin, int sign) {
  if (n <= 0 || (sign != 1 && sign != -1)) return -1;
  cplx* x = (cplx*)xin;
  root2* tw = root2_table(n, sign);
  if (!tw) return -2;
  int rc = dft_line(n, x, tw);
  free(tw);
  double s = 1.0 / sqrt((double)n);
  for (int64_t i = 0; i < n; ++i) x[i] *= s;
  return rc;
}

/* Unnormalised DFT along every axis of a D-dimensional row-major array. */
static int dft_all_axes(const orc_ctx* c, cplx* a, int sign) {
  int64_t maxn = 0;
  for (int l = 0; l < c->D; ++l) maxn = c->N[l] > maxn ? c->N[l] : maxn;
  cplx* line = malloc(sizeof(cplx) * (size_t)maxn);
  if (!line) return -2;
  for (int l = 0; l < c->D; ++l) {
    int64_t n = c->N[l], stride = 1, outer = 1;
    for (int m = l + 1; m < c->D; ++m) stride *= c->N[m];
    for (int m = 0; m < l; ++m) outer *= c->N[m];
    root2* tw = root2_table(n, sign);
    if (!tw) {
      free(line);
      return -2;
    }
    for (int64_t o = 0; o < outer; ++o) {
      for (int64_t i = 0; i < stride; ++i) {
        cplx* base = a + o * n * stride + i;
        for (int64_t j = 0; j < n; ++j) line[j] = base[j * stride];
        dft_line(n, line, tw);
        for (int64_t j = 0; j < n; ++j) base[j * stride] = line[j];
      }
    }
    free(tw);
  }
  free(line);
  return 0;
}

/* Multi-index of flat position J (last axis fastest). */
static void unflatten(const orc_ctx* c, int64_t J, int64_t* idx) {
  for (int l = c->D - 1; l >= 0; --l) {
    idx[l] = J % c->N[l];
    J /= c->N[l];
  }
}

/* ------------------------------------------------------------------------ */
/* Composition coefficients (eq:comp_TVT; Yoshida 1990 and Suzuki 1990)     */
/* ------------------------------------------------------------------------ */

int orc_scheme(const char* name, double* gamma, int cap) {
  int family, order;
  if (strcmp(name, "strang") == 0 || strcmp(name, "tvt") == 0 || strcmp(name, "vtv") == 0 ||
      strcmp(name, "tv") == 0) {
    family = 0;
    order = 2;
  } else if (strncmp(name, "yoshida", 7) == 0) {
    family = 1;
    order = atoi(name + 7);
  } else if (strncmp(name, "suzuki", 6) == 0) {
    family = 2;
    order = atoi(name + 6);
  } else {
    return -1;
  }
  if (order < 2 || order > 10 || order % 2) return -1;
  /* Work arrays big enough for Suzuki order 10 (5^4 = 625 stages). */
  double cur[625], nxt[625];
  int s = 1;
  cur[0] = 1.0;
  for (int o = 2; o < order && family != 0; o += 2) {
    int n = o / 2;
    double e = 1.0 / (2.0 * n + 1.0);
    if (family == 1) {
      /* triple jump: S_{2n+2}(h) = S_{2n}(g1 h) S_{2n}(g2 h) S_{2n}(g1 h) */
      double g1 = 1.0 / (2.0 - pow(2.0, e)), g2 = 1.0 - 2.0 * g1;
      double g[3] = {g1, g2, g1};
      for (int b = 0; b < 3; ++b)
        for (int k = 0; k < s; ++k) nxt[b * s + k] = g[b] * cur[k];
      s *= 3;
    } else {
      /* fractal: S_{2n+2}(h) = S_{2n}(g1 h)^2 S_{2n}(g2 h) S_{2n}(g1 h)^2 */
      double g1 = 1.0 / (4.0 - pow(4.0, e)), g2 = 1.0 - 4.0 * g1;
      double g[5] = {g1, g1, g2, g1, g1};
      for (int b = 0; b < 5; ++b)
        for (int k = 0; k < s; ++k) nxt[b * s + k] = g[b] * cur[k];
      s *= 5;
    }
    memcpy(cur, nxt, sizeof(double) * (size_t)s);
  }
  for (int k = 0; k < s && k < cap; ++k) gamma[k] = cur[k];
  return s;
}

/* ------------------------------------------------------------------------ */
/* Context, grid and potential (eq:x_I_definition, eq:hamiltonian)          */
/* ------------------------------------------------------------------------ */

orc_ctx* orc_create(int D, const int64_t* N, const double* dq, const double* minv, double hbar) {
  if (D < 1 || D > ORC_MAXD || !(hbar > 0)) return NULL;
  orc_ctx* c = calloc(1, sizeof(orc_ctx));
  if (!c) return NULL;
  c->D = D;
  c->hbar = hbar;
  c->npts = 1;
  for (int l = 0; l < D; ++l) {
    if (N[l] < 2 || N[l] % 2 || !(dq[l] > 0)) { free(c); return NULL; }
    c->N[l] = N[l];
    c->dq[l] = dq[l];
    c->dp[l] = TWO_PI * hbar / ((double)N[l] * dq[l]);
    c->npts *= N[l];
  }
  memcpy(c->minv, minv, sizeof(double) * (size_t)(D * D));
  c->u = calloc((size_t)c->npts, sizeof(cplx));
  if (!c->u) { free(c); return NULL; }
  c->pot_kind = -1;
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  free(c->u);
  free(c);
}

int64_t orc_npoints(const orc_ctx* c) { return c ? c->npts : -1; }

int orc_set_potential(orc_ctx* c, int kind, const double* params, int nparams) {
  int need;
  switch (kind) {
    case ORC_POT_HARMONIC: need = c->D * c->D + c->D; break;
    case ORC_POT_ATOM_DIATOM: need = 5; if (c->D != 2) return -1; break;
    case ORC_POT_HENON_HEILES: need = 1; break;
    case ORC_POT_SECREST_JOHNSON: need = 3; if (c->D != 2) return -1; break;
    default: return -1;
  }
  if (nparams != need) return -1;
  c->pot_kind = kind;
  c->npot = nparams;
  memcpy(c->pot, params, sizeof(double) * (size_t)nparams);
  return 0;
}

/* V(x) and its gradient at one point, straight from the formulas. */
static void potential_at(const orc_ctx* c, const double* x, double* V, double* g) {
  const int D = c->D;
  const double* P = c->pot;
  switch (c->pot_kind) {
    case ORC_POT_HARMONIC: {
      const double* K = P;
      const double* ctr = P + D * D;
      double v = 0;
      for (int a = 0; a < D; ++a) {
        double ga = 0;
        for (int b = 0; b < D; ++b) ga += K[a * D + b] * (x[b] - ctr[b]);
        g[a] = ga;
        v += 0.5 * (x[a] - ctr[a]) * ga;
      }
      *V = v;
      break;
    }
    case ORC_POT_ATOM_DIATOM: {
      double Dm = P[0], a = P[1], re = P[2], A = P[3], be = P[4];
      double R = x[0], r = x[1];
      double em = exp(-a * (r - re));
      double e1 = A * exp(-be * (R - 0.5 * r));
      double e2 = A * exp(-be * (R + 0.5 * r));
      *V = Dm * (1.0 - em) * (1.0 - em) + e1 + e2;
      g[0] = -be * e1 - be * e2;
      g[1] = 2.0 * Dm * (1.0 - em) * a * em + 0.5 * be * e1 - 0.5 * be * e2;
      break;
    }
    case ORC_POT_HENON_HEILES: {
      double lam = P[0], v = 0;
      for (int l = 0; l < D; ++l) {
        v += 0.5 * x[l] * x[l];
        g[l] = x[l];
      }
      for (int l = 0; l + 1 < D; ++l) {
        v += lam * (x[l] * x[l] * x[l + 1] - x[l + 1] * x[l + 1] * x[l + 1] / 3.0);
        g[l] += 2.0 * lam * x[l] * x[l + 1];
        g[l + 1] += lam * (x[l] * x[l] - x[l + 1] * x[l + 1]);
      }
      *V = v;
      break;
    }
    case ORC_POT_SECREST_JOHNSON: {
      double Dm = P[0], be = P[1], al = P[2];
      double e1 = exp(-be * x[0]);
      double e2 = exp(-al * (x[1] - x[0]));
      *V = Dm * (1.0 - e1) * (1.0 - e1) + e2;
      g[0] = 2.0 * Dm * (1.0 - e1) * be * e1 + al * e2;
      g[1] = -al * e2;
      break;
    }
    default:
      *V = 0;
      for (int a = 0; a < D; ++a) g[a] = 0;
  }
}

int orc_potential_eval(const orc_ctx* c, int64_t npts, const double* x, double* V, double* grad) {
  if (c->pot_kind < 0) return -1;
  double g[ORC_MAXD];
  for (int64_t i = 0; i < npts; ++i) {
    potential_at(c, x + i * c->D, &V[i], g);
    if (grad)
      for (int a = 0; a < c->D; ++a) grad[i * c->D + a] = g[a];
  }
  return 0;
}

/* q-grid point x^J for the grid centred at q (eq:x_I_definition). */
static void qpoint(const orc_ctx* c, const double* q, const int64_t* j, double* x) {
  for (int l = 0; l < c->D; ++l) x[l] = q[l] + ((double)j[l] - 0.5 * (double)c->N[l]) * c->dq[l];
}
/* p-grid point p^K for the grid centred at p. */
static void ppoint(const orc_ctx* c, const double* p, const int64_t* k, double* x) {
  for (int l = 0; l < c->D; ++l) x[l] = p[l] + ((double)k[l] - 0.5 * (double)c->N[l]) * c->dp[l];
}

static double kinetic(const orc_ctx* c, const double* pk) {
  double T = 0;
  for (int a = 0; a < c->D; ++a)
    for (int b = 0; b < c->D; ++b) T += 0.5 * pk[a] * c->minv[a * c->D + b] * pk[b];
  return T;
}

static double sqrt_cell(const orc_ctx* c) {
  double v = 1;
  for (int l = 0; l < c->D; ++l) v *= c->dq[l];
  return sqrt(v);
}

/* ------------------------------------------------------------------------ */
/* States                                                                   */
/* ------------------------------------------------------------------------ */

int orc_set_state(orc_ctx* c, const double* psi, const double* q, const double* p, double t) {
  double s = sqrt_cell(c);
  const cplx* src = (const cplx*)psi;
  for (int64_t J = 0; J < c->npts; ++J) c->u[J] = src[J] * s;
  memcpy(c->q, q, sizeof(double) * (size_t)c->D);
  memcpy(c->p, p, sizeof(double) * (size_t)c->D);
  c->t = t;
  return 0;
}

int orc_get_state(const orc_ctx* c, double* psi, double* q, double* p, double* t) {
  double s = 1.0 / sqrt_cell(c);
  if (psi) {
    cplx* dst = (cplx*)psi;
    for (int64_t J = 0; J < c->npts; ++J) dst[J] = c->u[J] * s;
  }
  if (q) memcpy(q, c->q, sizeof(double) * (size_t)c->D);
  if (p) memcpy(p, c->p, sizeof(double) * (size_t)c->D);
  if (t) *t = c->t;
  return 0;
}

int orc_set_u(orc_ctx* c, const double* u) {
  memcpy(c->u, u, sizeof(cplx) * (size_t)c->npts);
  return 0;
}

int orc_get_u(const orc_ctx* c, double* u) {
  memcpy(u, c->u, sizeof(cplx) * (size_t)c->npts);
  return 0;
}

/* Morse ground state phi0(x) = Nrm z^{lam-1/2} e^{-z/2}, z = 2 lam e^{-a(x-re)},
 * lam = sqrt(2 m Dm)/(a hbar); |Nrm|^2 = a / Gamma(2 lam - 1). */
static double morse_ground(double x, double Dm, double a, double re, double m, double hbar) {
  double lam = sqrt(2.0 * m * Dm) / (a * hbar);
  double z = 2.0 * lam * exp(-a * (x - re));
  double lg = (lam - 0.5) * log(z) - 0.5 * z + 0.5 * (log(a) - lgamma(2.0 * lam - 1.0));
  return exp(lg);
}

double orc_morse_mean(double Dm, double a, double re, double m, double hbar) {
  /* Trapezoid rule on a fine uniform grid that covers the whole density. */
  double lam = sqrt(2.0 * m * Dm) / (a * hbar);
  double xpk = re - log((2.0 * lam - 1.0) / (2.0 * lam)) / a;
  double half = 60.0 / (a * sqrt(lam)) + 40.0 / (a * (2.0 * lam - 1.0)) + 5.0 / a;
  int64_t n = 400000;
  double h = 2.0 * half / (double)n, s0 = 0, s1 = 0;
  for (int64_t i = 0; i <= n; ++i) {
    double x = xpk - half + h * (double)i;
    double f = morse_ground(x, Dm, a, re, m, hbar);
    double w = (i == 0 || i == n) ? 0.5 : 1.0;
    s0 += w * f * f;
    s1 += w * x * f * f;
  }
  return s1 / s0;
}

int orc_set_separable(orc_ctx* c, const int* kinds, const double* params, const double* q_ctr,
                      const double* p_ctr) {
  memcpy(c->q, q_ctr, sizeof(double) * (size_t)c->D);
  memcpy(c->p, p_ctr, sizeof(double) * (size_t)c->D);
  c->t = 0;
  double s = sqrt_cell(c);
  int64_t j[ORC_MAXD];
  double x[ORC_MAXD];
  for (int64_t J = 0; J < c->npts; ++J) {
    unflatten(c, J, j);
    qpoint(c, c->q, j, x);
    cplx v = 1;
    for (int l = 0; l < c->D; ++l) {
      const double* P = params + 4 * l;
      if (kinds[l] == 0) {
        double q0 = P[0], p0 = P[1], sg = P[2];
        double d = x[l] - q0;
        v *= pow(M_PI * sg * sg, -0.25) * cexp(-d * d / (2.0 * sg * sg) + I * p0 * d / c->hbar);
      } else if (kinds[l] == 1) {
        v *= morse_ground(x[l], P[0], P[1], P[2], P[3], c->hbar);
      } else {
        return -1;
      }
    }
    c->u[J] = v * s;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The shifted transform f(q,p) (eq:F_defintion, eq:t_definition)           */
/* ------------------------------------------------------------------------ */

/* f(q,p) = N^{-1/2} e^{-2 pi i <K,J>} e^{-i t_KJ/hbar} with
 * t_KJ = sum_l [(p_l - dp_l N_l/2)(q_l - dq_l N_l/2) + p_l j_l dq_l + q_l k_l dp_l
 *               - pi hbar (j_l + k_l)].
 * The J-dependent part of t is applied before the DFT, the K-dependent and
 * constant parts after it; f~ = f^dagger reverses this. */
/* scale: 0 = N^{-1/2} (the unitary f of eq:F_defintion), 1 = none, 2 = 1/N.
 * Inside a kinetic substep the forward transform is left unscaled and the
 * inverse divided by N: the two N^{-1/2} factors of f~ f applied as one exact
 * (power-of-two N) or correctly rounded division, so that f~ f = 1
 * (eq:F_inv_definition) holds without a systematic rounding bias. */
static int apply_f_scaled(const orc_ctx* c, const double* q, const double* p, const double* in,
                          double* out, int sign, int scale);

int orc_apply_f(const orc_ctx* c, const double* q, const double* p, const double* in, double* out,
                int sign) {
  return apply_f_scaled(c, q, p, in, out, sign, 0);
}

static int apply_f_scaled(const orc_ctx* c, const double* q, const double* p, const double* in,
                          double* out, int sign, int scale) {
  if (sign != 1 && sign != -1) return -1;
  const int D = c->D;
  const double hb = c->hbar;
  cplx* a = (cplx*)out;
  memcpy(a, in, sizeof(cplx) * (size_t)c->npts);
  int64_t idx[ORC_MAXD];
  /* constant part: sum_l (p_l - dp_l N_l/2)(q_l - dq_l N_l/2) */
  dd cst = {0, 0};
  for (int l = 0; l < D; ++l) {
    dd pa = dd_add((dd){p[l], 0}, dd_mul_d((dd){c->dp[l], 0}, -0.5 * (double)c->N[l]));
    dd qa = dd_add((dd){q[l], 0}, dd_mul_d((dd){c->dq[l], 0}, -0.5 * (double)c->N[l]));
    cst = dd_add(cst, dd_mul(pa, qa));
  }
  /* J part: sum_l p_l j_l dq_l;  K part: cst + sum_l q_l k_l dp_l (then / hbar) */
  for (int pass = 0; pass < 2; ++pass) {
    const int jpart = (sign == -1) == (pass == 0);
    if (pass == 1) {
      dft_all_axes(c, a, sign);
      const double nn = (double)c->npts, rs = 1.0 / sqrt(nn);
      for (int64_t K = 0; K < c->npts; ++K) {
        if (scale == 0) a[K] *= rs;
        else if (scale == 2) a[K] = creal(a[K]) / nn + I * (cimag(a[K]) / nn);
      }
    }
    for (int64_t I_ = 0; I_ < c->npts; ++I_) {
      unflatten(c, I_, idx);
      dd ph = jpart ? (dd){0, 0} : cst;
      double sg = 1;
      for (int l = 0; l < D; ++l) {
        dd f = jpart ? dd_of_prod(p[l], c->dq[l]) : dd_of_prod(q[l], c->dp[l]);
        ph = dd_add(ph, dd_mul_d(f, (double)idx[l]));
        if (idx[l] & 1) sg = -sg;
      }
      ph = dd_div_d(ph, hb);
      if (sign == -1) { ph.hi = -ph.hi; ph.lo = -ph.lo; }
      a[I_] *= sg * expi(ph);
    }
  }
  return 0;
}

int orc_apply_f_dense(const orc_ctx* c, const double* q, const double* p, const double* in,
                      double* out, int sign) {
  if (c->npts > 4096 || (sign != 1 && sign != -1)) return -1;
  const int D = c->D;
  const int64_t n = c->npts;
  const double hb = c->hbar;
  const cplx* x = (const cplx*)in;
  cplx* y = (cplx*)out;
  int64_t K[ORC_MAXD], J[ORC_MAXD];
  double rn = 1.0 / sqrt((double)n);
  for (int64_t r = 0; r < n; ++r) {
    cplx acc = 0;
    for (int64_t s = 0; s < n; ++s) {
      /* matrix element f_KJ with K = row, J = column for f; f^dagger_JK = conj(f_KJ) */
      int64_t kf = sign == -1 ? r : s, jf = sign == -1 ? s : r;
      unflatten(c, kf, K);
      unflatten(c, jf, J);
      double t = 0, frac = 0;
      for (int l = 0; l < D; ++l) {
        double Nl = (double)c->N[l];
        t += (p[l] - c->dp[l] * Nl / 2) * (q[l] - c->dq[l] * Nl / 2) + p[l] * (double)J[l] * c->dq[l] +
             q[l] * (double)K[l] * c->dp[l] - M_PI * hb * (double)(J[l] + K[l]);
        frac += (double)((K[l] * J[l]) % c->N[l]) / Nl;
      }
      cplx f = rn * cexp(-I * TWO_PI * frac) * cexp(-I * t / hb);
      acc += (sign == -1 ? f : conj(f)) * x[s];
    }
    y[r] = acc;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Substeps (Sec. II.G) and composition (eq:SO_TVT, eq:comp_TVT)            */
/* ------------------------------------------------------------------------ */

/* Potential propagation: psi <- U_V(tau, q) psi, q unchanged,
 * p <- p - tau <dV/dq> (eq:eom_pt_solution_case_III_V). */
int orc_substep_V(orc_ctx* c, double tau, int grid_motion) {
  if (c->pot_kind < 0) return -1;
  const int D = c->D;
  int64_t j[ORC_MAXD];
  double x[ORC_MAXD], g[ORC_MAXD], gs[ORC_MAXD] = {0}, n = 0, V;
  for (int64_t J = 0; J < c->npts; ++J) {
    unflatten(c, J, j);
    qpoint(c, c->q, j, x);
    potential_at(c, x, &V, g);
    double w = creal(c->u[J]) * creal(c->u[J]) + cimag(c->u[J]) * cimag(c->u[J]);
    n += w;
    for (int a = 0; a < D; ++a) gs[a] += g[a] * w;
    c->u[J] *= cexp(-I * tau * V / c->hbar);
  }
  if (grid_motion != ORC_GRID_FIXED)
    for (int a = 0; a < D; ++a) c->p[a] -= tau * gs[a] / n;
  return 0;
}

/* Kinetic propagation (eq:T_split_substep_adaptive):
 * phi = f(q0,p0) u, q_tau = q0 + tau m^-1 <p> (eq:eom_qt_case_III_T),
 * u <- f~(q_tau, p0) U~_T(tau, p0) phi. */
int orc_substep_T(orc_ctx* c, double tau, int grid_motion) {
  const int D = c->D;
  cplx* phi = malloc(sizeof(cplx) * (size_t)c->npts);
  if (!phi) return -2;
  apply_f_scaled(c, c->q, c->p, (const double*)c->u, (double*)phi, -1, 1);
  int64_t k[ORC_MAXD];
  double pk[ORC_MAXD], ps[ORC_MAXD] = {0}, n = 0;
  for (int64_t K = 0; K < c->npts; ++K) {
    unflatten(c, K, k);
    ppoint(c, c->p, k, pk);
    double w = creal(phi[K]) * creal(phi[K]) + cimag(phi[K]) * cimag(phi[K]);
    n += w;
    for (int a = 0; a < D; ++a) ps[a] += pk[a] * w;
  }
  double qn[ORC_MAXD];
  for (int a = 0; a < D; ++a) {
    double v = 0;
    for (int b = 0; b < D; ++b) {
      double mom = grid_motion == ORC_GRID_ADAPTIVE_CENTRE_P ? c->p[b] : ps[b] / n;
      v += c->minv[a * D + b] * mom;
    }
    qn[a] = c->q[a] + (grid_motion == ORC_GRID_FIXED ? 0.0 : tau * v);
  }
  for (int64_t K = 0; K < c->npts; ++K) {
    unflatten(c, K, k);
    ppoint(c, c->p, k, pk);
    phi[K] *= cexp(-I * tau * kinetic(c, pk) / c->hbar);
  }
  apply_f_scaled(c, qn, c->p, (const double*)phi, (double*)c->u, 1, 2);
  memcpy(c->q, qn, sizeof(double) * (size_t)D);
  free(phi);
  return 0;
}

int orc_propagate(orc_ctx* c, int64_t n_steps, double dt, const char* scheme, int split,
                  int grid_motion) {
  double gamma[625];
  int S = orc_scheme(scheme, gamma, 625);
  if (S <= 0) return -1;
  if (split != ORC_SPLIT_TVT && split != ORC_SPLIT_VTV && split != ORC_SPLIT_TV) return -1;
  if (c->pot_kind < 0) return -1;
  for (int64_t s = 0; s < n_steps; ++s) {
    for (int k = 0; k < S; ++k) {
      double h = gamma[k] * dt;
      if (split == ORC_SPLIT_TVT) {
        orc_substep_T(c, 0.5 * h, grid_motion);
        orc_substep_V(c, h, grid_motion);
        orc_substep_T(c, 0.5 * h, grid_motion);
      } else if (split == ORC_SPLIT_VTV) {
        orc_substep_V(c, 0.5 * h, grid_motion);
        orc_substep_T(c, h, grid_motion);
        orc_substep_V(c, 0.5 * h, grid_motion);
      } else { /* U_TV(h) = U_T(h) U_V(h): the potential acts first */
        orc_substep_V(c, h, grid_motion);
        orc_substep_T(c, h, grid_motion);
      }
    }
    c->t += dt;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables (eq:scalar_prod; energy of Sec. III.A)                       */
/* ------------------------------------------------------------------------ */

int orc_observables(const orc_ctx* c, double* norm, double* energy, double* mean_q,
                    double* mean_p) {
  const int D = c->D;
  int64_t j[ORC_MAXD];
  double x[ORC_MAXD], g[ORC_MAXD], n = 0, ev = 0, qs[ORC_MAXD] = {0}, V = 0;
  for (int64_t J = 0; J < c->npts; ++J) {
    unflatten(c, J, j);
    qpoint(c, c->q, j, x);
    double w = creal(c->u[J]) * creal(c->u[J]) + cimag(c->u[J]) * cimag(c->u[J]);
    n += w;
    for (int a = 0; a < D; ++a) qs[a] += x[a] * w;
    if (c->pot_kind >= 0) {
      potential_at(c, x, &V, g);
      ev += V * w;
    }
  }
  cplx* phi = malloc(sizeof(cplx) * (size_t)c->npts);
  if (!phi) return -2;
  orc_apply_f(c, c->q, c->p, (const double*)c->u, (double*)phi, -1);
  double et = 0, ps[ORC_MAXD] = {0}, pk[ORC_MAXD];
  for (int64_t K = 0; K < c->npts; ++K) {
    unflatten(c, K, j);
    ppoint(c, c->p, j, pk);
    double w = creal(phi[K]) * creal(phi[K]) + cimag(phi[K]) * cimag(phi[K]);
    et += kinetic(c, pk) * w;
    for (int a = 0; a < D; ++a) ps[a] += pk[a] * w;
  }
  free(phi);
  if (norm) *norm = n;
  if (energy) *energy = (et + ev) / n;
  for (int a = 0; a < D; ++a) {
    if (mean_q) mean_q[a] = qs[a] / n;
    if (mean_p) mean_p[a] = ps[a] / n;
  }
  return 0;
}

int orc_regrid(const orc_ctx* c, const double* u_b, const double* q_b, const double* p,
               const double* q_a, double* out) {
  cplx* phi = malloc(sizeof(cplx) * (size_t)c->npts);
  if (!phi) return -2;
  orc_apply_f(c, q_b, p, u_b, (double*)phi, -1);
  orc_apply_f(c, q_a, p, (const double*)phi, out, 1);
  free(phi);
  return 0;
}
