/* Plain FP64 CPU oracle of the moving-grid split-operator integrator
 * (Choi & Vanicek, "A time-reversible integrator for the time-dependent
 * Schroedinger equation on an adaptive grid", arXiv:1909.06412).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the checker the GPU path is
 * compared against.  It shares no code, header, table or helper with the
 * CUDA library; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It is deliberately slow and literal.
 *
 * Conventions (Sec. II.B-D of the paper):
 *   - D axes, axis l has N_l (even) points, spacing dq_l, dp_l = 2*pi*hbar/(N_l dq_l).
 *   - q-grid x_l^J = q_l + (j_l - N_l/2) dq_l, p-grid p_l^K = p_l + (k_l - N_l/2) dp_l.
 *   - State u: row-major, last axis contiguous, interleaved (re, im) doubles,
 *     u^J = psi(x^J) * sqrt(prod dq_l) so that sum |u|^2 is the grid norm
 *     of the scalar product (eq:scalar_prod).
 *
 * Every entry point returns 0 on success and a negative code on bad input.
 */
#ifndef MGRID_ORACLE_H
#define MGRID_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXD 8

enum { ORC_POT_HARMONIC = 0, ORC_POT_ATOM_DIATOM = 1, ORC_POT_HENON_HEILES = 2,
       ORC_POT_SECREST_JOHNSON = 3 };
enum { ORC_SPLIT_TVT = 0, ORC_SPLIT_VTV = 1, ORC_SPLIT_TV = 2 };
enum { ORC_GRID_ADAPTIVE = 0, ORC_GRID_ADAPTIVE_CENTRE_P = 1, ORC_GRID_FIXED = 2 };

typedef struct orc_ctx orc_ctx;

/* 1D unitary DFT of length n in place (interleaved complex).  Radix-2 FFT when
 * n is a power of two, direct O(n^2) sum otherwise.  sign=-1 forward
 * (e^{-2 pi i kj/n}), +1 inverse. */
int orc_dft1d(int64_t n, double* x, int sign);
/* Direct O(n^2) unitary DFT, out of place, for cross-checks. */
int orc_dft1d_direct(int64_t n, const double* in, double* out, int sign);

/* Composition coefficients gamma_1..gamma_S of a named symmetric scheme
 * ("strang", "yoshida4/6/8/10" triple jump, "suzuki4/6/8/10" fractal).
 * Returns S (>0), or a negative code; writes at most cap values. */
int orc_scheme(const char* name, double* gamma, int cap);

orc_ctx* orc_create(int D, const int64_t* N, const double* dq, const double* minv, double hbar);
void orc_destroy(orc_ctx* c);
int64_t orc_npoints(const orc_ctx* c);
/* Potential kinds and parameter layouts:
 *  HARMONIC:        params = [K (D*D row-major), c (D)]:  V = 1/2 (x-c)^T K (x-c)
 *  ATOM_DIATOM:     axes (R, r); params = [Dm, a, re, A, beta]:
 *                   V = Dm (1-e^{-a(r-re)})^2 + A e^{-beta(R-r/2)} + A e^{-beta(R+r/2)}
 *  HENON_HEILES:    params = [lambda]:  V = sum x_l^2/2 + lambda sum_{l<D} (x_l^2 x_{l+1} - x_{l+1}^3/3)
 *  SECREST_JOHNSON: axes (q1, q2); params = [Dm, beta, alpha]:
 *                   V = Dm (1-e^{-beta q1})^2 + e^{-alpha (q2-q1)}                        */
int orc_set_potential(orc_ctx* c, int kind, const double* params, int nparams);
/* Evaluate V and grad V at npts points x (npts*D row-major). grad may be NULL. */
int orc_potential_eval(const orc_ctx* c, int64_t npts, const double* x, double* V, double* grad);

/* State in/out: psi is the physical wavefunction psi(x^J) (interleaved). */
int orc_set_state(orc_ctx* c, const double* psi, const double* q, const double* p, double t);
int orc_get_state(const orc_ctx* c, double* psi, double* q, double* p, double* t);
/* Raw scaled state u (sum |u|^2 = norm). */
int orc_set_u(orc_ctx* c, const double* u);
int orc_get_u(const orc_ctx* c, double* u);

/* Separable product initial state.  Per axis a factor of kind 0 (Gaussian,
 * params [q0, p0, sigma]: (pi s^2)^{-1/4} exp[-(x-q0)^2/(2 s^2) + i p0 (x-q0)/hbar])
 * or kind 1 (Morse ground state, params [Dm, a, re, mass]).  The grid centre is
 * set to (q_ctr, p_ctr).  Samples are taken on that grid. */
int orc_set_separable(orc_ctx* c, const int* kinds, const double* params /* D*4 */,
                      const double* q_ctr, const double* p_ctr);
/* Mean of x under the Morse ground state, by quadrature on a fine grid. */
double orc_morse_mean(double Dm, double a, double re, double mass, double hbar);

/* The shifted transform f(q,p) of eq:F_defintion applied as pre-phase, unitary
 * DFT and post-phase (sign=-1), or its adjoint f~ = f^dagger (sign=+1). */
int orc_apply_f(const orc_ctx* c, const double* q, const double* p, const double* in,
                double* out, int sign);
/* Same operator built as a dense N x N matrix from eq:t_definition (N <= 4096). */
int orc_apply_f_dense(const orc_ctx* c, const double* q, const double* p, const double* in,
                      double* out, int sign);

/* One potential substep U_V,adpt(tau) (Sec. II.G.1) and one kinetic substep
 * U_T,adpt(tau) (Sec. II.G.2) on the context state. */
int orc_substep_V(orc_ctx* c, double tau, int grid_motion);
int orc_substep_T(orc_ctx* c, double tau, int grid_motion);

/* n_steps of the named composition with the named split (eq:comp_TVT). */
int orc_propagate(orc_ctx* c, int64_t n_steps, double dt, const char* scheme, int split,
                  int grid_motion);

/* Observables: norm = sum|u|^2, energy = <T> + <V>, mean q and mean p (both
 * normalised by the norm). */
int orc_observables(const orc_ctx* c, double* norm, double* energy, double* mean_q,
                    double* mean_p);

/* Trigonometric interpolation (regrid): the state (u_b on a grid centred at
 * q_b, p) resampled on the grid centred at q_a with the same p window. */
int orc_regrid(const orc_ctx* c, const double* u_b, const double* q_b, const double* p,
               const double* q_a, double* out);

#ifdef __cplusplus
}
#endif
#endif
