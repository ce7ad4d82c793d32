/* mgrid: GPU (sm_103a) moving-grid split-operator propagator for the
 * time-dependent Schroedinger equation, after Choi & Vanicek,
 * "A time-reversible integrator for the time-dependent Schroedinger
 * equation on an adaptive grid" (arXiv:1909.06412).
 *
 * One context = one D-dimensional tensor-product grid (Sec. II.B,
 * eq:multi_index_I, eq:x_I_definition) whose centre (q_t, p_t) moves with
 * the wavepacket: inside every kinetic substep the q-centre advances by
 * tau m^-1 <p> (eq:eom_qt_case_III_T), inside every potential substep the
 * p-centre advances by -tau <dV/dq> (eq:eom_pt_solution_case_III_V).
 * Substeps are composed symmetrically (eq:SO_TVT, eq:comp_TVT).
 *
 * Conventions shared by every entry point:
 *  - Grid: axis l has N_l points (even, 2 <= N_l <= 2048, only factors 2 and 3),
 *    spacing dq_l > 0 and momentum spacing dp_l = 2 pi hbar / (N_l dq_l);
 *    x_l^J = q_l + (j_l - N_l/2) dq_l and p_l^K = p_l + (k_l - N_l/2) dp_l.
 *  - Arrays: row-major, last axis contiguous; complex values interleaved
 *    (re, im); host arrays are always FP64.
 *  - Device memory is owned by the caller (a torch tensor, say): the library
 *    never allocates or frees device memory.  d_psi holds the scaled state
 *    u^J = psi(x^J) sqrt(prod dq_l) (so sum |u|^2 is the norm of
 *    eq:scalar_prod) as complex128 (MG_FP64) or complex64 (MG_FP32_MIXED).
 *  - Work runs on the stream given at creation.  Entry points that return
 *    data to the host synchronise that stream; the others only enqueue.
 *  - Errors: every call returns an mg_status.  Device-side failures (barrier
 *    timeout, non-finite norm, runaway grid centre) are recorded in a device
 *    word and reported by the next synchronising call (mg_sync, mg_get_*).
 *  - A context is not thread-safe; use one per stream.
 */
#ifndef MGRID_H
#define MGRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;

typedef enum {
  MG_OK = 0,
  MG_ERR_ARG = -1,         /* invalid argument (null pointer, bad size, unknown name) */
  MG_ERR_UNSUPPORTED = -2, /* valid but not supported by this build (axis length, D) */
  MG_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  MG_ERR_TIMEOUT = -4,     /* a grid-wide barrier in the persistent kernel timed out */
  MG_ERR_NONFINITE = -5,   /* the norm or a reduction became non-finite */
  MG_ERR_UNSTABLE = -6,    /* a grid centre jumped by more than 10 grid spans in one substep
                              (Verlet instability of Sec. II.H, eq:verlet_stability_cond) */
  MG_ERR_STATE = -7        /* call out of order (no potential or state set yet) */
} mg_status;

enum { MG_FP64 = 0, MG_FP32_MIXED = 1 };
/* eq:SO_TVT (T half-steps around V), its V<->T exchange, and first-order
 * eq:SO_TV (U_T U_V: the potential acts first). */
enum { MG_TVT = 0, MG_VTV = 1, MG_TV = 2 };
/* ADAPTIVE: q-centre moves with the <p> reduction (eq:eom_qt_case_III_T);
 * ADAPTIVE_CENTRE_P: moves with the p-centre itself (eq:eom_qt_solution_case_III_T);
 * FIXED: centres never move (the conventional split-operator method);
 * NAIVE: the naive adaptive grid of Sec. II.F (eq:naive_wf_solution): every
 * time step runs on the fixed grid, then the grid moves to the new <q>, <p>
 * by f~(<q>, <p>) f(q, <p>).  Norm-preserving but not time-reversible
 * (eq:naive_t_rev_fail); mg_propagate only, one host round trip per step. */
enum { MG_GRID_ADAPTIVE = 0, MG_GRID_ADAPTIVE_CENTRE_P = 1, MG_GRID_FIXED = 2, MG_GRID_NAIVE = 3 };
/* Potentials (params layout):
 *  HARMONIC        [K (D*D row-major, symmetric), c (D)]: V = 1/2 (x-c)^T K (x-c)
 *  ATOM_DIATOM     D=2, axes (R, r), [Dm, a, re, A, beta]:
 *                  V = Dm (1-e^{-a(r-re)})^2 + A e^{-beta(R-r/2)} + A e^{-beta(R+r/2)}
 *  HENON_HEILES    [lambda]: V = sum x_l^2/2 + lambda sum_{l<D} (x_l^2 x_{l+1} - x_{l+1}^3/3)
 *                  (Sec. III.C)
 *  SECREST_JOHNSON D=2, [Dm, beta, alpha]: V = Dm (1-e^{-beta q1})^2 + e^{-alpha(q2-q1)}
 *                  (eq:modified_secrest_johnson) */
enum { MG_POT_HARMONIC = 0, MG_POT_ATOM_DIATOM = 1, MG_POT_HENON_HEILES = 2,
       MG_POT_SECREST_JOHNSON = 3 };

/* Device workspace the caller must provide for a grid (bytes, 256-aligned
 * start required).  Returns 0 for an invalid or unsupported grid. */
size_t mg_workspace_bytes(int D, const int64_t* N, int precision);

/* Create a context (Sec. II.B grid; eq:KE_operator kinetic energy).
 * minv: D*D row-major inverse mass matrix, symmetric positive definite
 * (MG_ERR_ARG otherwise).  A matrix with off-diagonal entries runs on the
 * general kernel, whose kinetic substep applies the non-separable part of
 * e^{-i tau T(p^K)/hbar} point by point and moves the grid by
 * tau m^-1 <p> with the full matrix; mg_adjoint and mg_batch_create refuse
 * such contexts (MG_ERR_UNSUPPORTED).  d_psi: device buffer of
 * prod(N) complex elements of the chosen precision.  d_work: device buffer of
 * at least mg_workspace_bytes() bytes.  cuda_stream: a cudaStream_t (NULL =
 * legacy default stream).  The context keeps the pointers, not copies. */
mg_status mg_create(mg_ctx** out, int D, const int64_t* N, const double* dq, const double* minv,
                    double hbar, int precision, void* d_psi, void* d_work, size_t work_bytes,
                    void* cuda_stream);

/* mg_create with a choice of kernel (flags = 0 is mg_create).  The method is
 * the same whichever kernel runs; the flags select how the transforms move
 * through memory and which units compute them.
 *  MG_CREATE_GENERAL_KERNEL  never use the short-axis kernel (one pass per axis)
 *  MG_CREATE_NO_TMA          short-axis kernel with cp.async chunk copies only
 *  MG_CREATE_TC_TF32X3       reserved: the short-axis kernel with its 16-point
 *  MG_CREATE_TC_BF16X3       line DFTs on the tensor cores (3xTF32 / BF16x3
 *                            split products).  Not enabled in this build: both
 *                            return MG_ERR_UNSUPPORTED.  The tensor-core
 *                            16-point DFT itself is mg_probe_tc_dft16.
 * At most one tensor-core flag, and neither with the first two flags
 * (MG_ERR_ARG). */
enum { MG_CREATE_GENERAL_KERNEL = 1, MG_CREATE_NO_TMA = 2, MG_CREATE_TC_TF32X3 = 4, MG_CREATE_TC_BF16X3 = 8 };
mg_status mg_create_ex(mg_ctx** out, int D, const int64_t* N, const double* dq, const double* minv,
                       double hbar, int precision, void* d_psi, void* d_work, size_t work_bytes,
                       void* cuda_stream, int flags);
mg_status mg_destroy(mg_ctx* ctx);

/* Select the potential (eq:hamiltonian); layouts above. */
mg_status mg_set_potential(mg_ctx* ctx, int kind, const double* params, int nparams);

/* Upload a physical wavefunction psi(x^J) (host, interleaved FP64,
 * prod(N) complex values) sampled on the grid centred at (q, p), with time t.
 * psi == NULL keeps the device state and only sets (q, p, t). */
mg_status mg_set_state(mg_ctx* ctx, const double* psi, const double* q, const double* p, double t);

/* Host-buffer state transfer without conversion, for callers that keep the
 * state in host memory between calls (the scaled state u^J = psi(x^J)
 * sqrt(prod dq_l) in the storage precision: prod(N) interleaved complex128
 * values for MG_FP64, complex64 for MG_FP32_MIXED).
 * mg_upload_u: copy host_u into d_psi on the context's stream and set the
 *   grid centres (q, p) and time t; asynchronous: host_u must stay valid and
 *   unchanged until the stream has reached the copy.  Page-locked host_u
 *   (cudaHostAlloc, or a pinned torch tensor) copies at full link bandwidth.
 * mg_download_u: copy d_psi into host_u and return q, p, t (each may be
 *   NULL); synchronises the stream and reports any pending device status. */
mg_status mg_upload_u(mg_ctx* ctx, const void* host_u, const double* q, const double* p, double t);
mg_status mg_download_u(mg_ctx* ctx, void* host_u, double* q, double* p, double* t);

/* Build a separable initial state on the grid centred at (q_ctr, p_ctr), t=0.
 * Per axis l, kinds[l] and params[4*l .. 4*l+3]:
 *   0 Gaussian (eq:general_GWP): [q0, p0, sigma, -]:
 *     (pi sigma^2)^{-1/4} exp[-(x-q0)^2/(2 sigma^2) + i p0 (x-q0)/hbar]
 *   1 Morse ground state [Dm, a, re, mass]: N z^{lam-1/2} e^{-z/2},
 *     z = 2 lam e^{-a(x-re)}, lam = sqrt(2 mass Dm)/(a hbar). */
mg_status mg_set_separable(mg_ctx* ctx, const int* kinds, const double* params,
                           const double* q_ctr, const double* p_ctr);

/* Propagate n_steps time steps dt (negative dt propagates backward) with a
 * named symmetric composition (eq:comp_TVT): "strang" (second order),
 * "yoshida4|6|8|10" (triple jump) or "suzuki4|6|8|10" (Suzuki fractal),
 * applied to the split `split` with grid motion `grid_motion`.  All steps run
 * in one persistent kernel launch on the context's stream. */
mg_status mg_propagate(mg_ctx* ctx, int64_t n_steps, double dt, const char* scheme, int split,
                       int grid_motion);

/* Synchronise and read back: psi (physical psi(x^J), host FP64 interleaved,
 * may be NULL), grid centres q, p (D doubles each, may be NULL) and time t. */
mg_status mg_get_state(mg_ctx* ctx, double* psi, double* q, double* p, double* t);

/* Synchronise and compute norm = sum |u|^2 (eq:scalar_prod), energy
 * <T> + <V> (Sec. III.A), <q> and <p> (normalised by the norm).  Any output
 * pointer may be NULL. */
mg_status mg_get_observables(mg_ctx* ctx, double* norm, double* energy, double* mean_q,
                             double* mean_p);

/* Represent the current state on the grid centred at (q, p) instead (host,
 * D doubles each): u <- f~(q, p) f(q_t, p) u, the exact trigonometric
 * interpolation of the band-limited state between the two grids
 * (eq:F_defintion, eq:F_inv_definition; the regridding of Sec. II.F and of
 * the error norms of Sec. III).  Sets the context's centres to (q, p), leaves
 * t unchanged, synchronises the stream.  Norm-preserving; a regrid back to
 * the original centres restores the state to rounding. */
mg_status mg_regrid(mg_ctx* ctx, const double* q, const double* p);

/* Inner product <psi_a | psi_b> = prod dq_l sum_J conj(psi_a(x_a^J)) psi_b(x_a^J)
 * of the states of two contexts with the same axis lengths, spacings,
 * precision and hbar (eq:scalar_prod), each on its own moving grid: b's
 * state is carried onto a's grid positions by trigonometric interpolation
 * with b's own momentum window (eq:F_defintion), in a's workspace.  With a
 * context holding psi_0 it gives the autocorrelation <psi_0 | psi_t>; for
 * two propagated states it shows that the moving grid does not conserve
 * the inner product exactly (Sec. II.E).  Neither state changes; both
 * streams are synchronised.  MG_ERR_ARG for mismatched grids. */
mg_status mg_inner_product(mg_ctx* a, const mg_ctx* b, double* re, double* im);

/* Synchronise the context's stream and report any pending device status. */
mg_status mg_sync(mg_ctx* ctx);

/* Failure-detection test hook; the paper has no counterpart.  Arms the next
 * mg_propagate of this context so that its first grid-wide barrier cannot
 * complete (the barrier word starts with every CTA already counted in the
 * current generation, so no arrival is the last one) and each barrier wait
 * gives up after limit_s seconds (0 < limit_s <= 5) instead of 5 s.  Every
 * CTA then records MG_ERR_TIMEOUT and returns: the next synchronising call
 * reports it, the state is left partly propagated, and later calls run
 * normally (every launch starts from a cleared barrier word).  Nothing waits
 * without a limit.  MG_ERR_ARG for a NULL context or limit_s out of range. */
mg_status mg_test_stuck_barrier(mg_ctx* ctx, double limit_s);

/* Reverse-mode derivative of the last mg_propagate call, by the reversible
 * adjoint: the context's state must be the final state of that call (same
 * n_steps, dt, scheme, split, grid_motion).  Each substep of Sec. II.G is undone
 * by the same substep at the negated time (exact time reversibility), so no
 * trajectory is stored, and its vector-Jacobian product is applied to the
 * cotangent on the way.  Convention: for a real objective J,
 * ubar = dJ/dRe u + i dJ/dIm u (u the scaled state in d_psi), qbar = dJ/dq,
 * pbar = dJ/dp.
 *  - d_ubar: device complex128 buffer like d_psi; in: ubar at the final time,
 *    out: ubar at the initial time.  qbar, pbar: host, D doubles, in/out.
 *  - theta_bar: host, out, ntheta values dJ/d(Dm, a, beta, A) for
 *    MG_POT_ATOM_DIATOM (ntheta = 4); ntheta = 0 for MG_POT_HARMONIC.
 *  - On return the context holds the regenerated initial state and time.
 *  - FP64 contexts whose state and cotangent fit in the CTAs' shared memory;
 *    harmonic or atom-diatom potential.  MG_ERR_UNSUPPORTED otherwise.
 *  - Synchronises the context's stream. */
mg_status mg_adjoint(mg_ctx* ctx, int64_t n_steps, double dt, const char* scheme, int split, int grid_motion,
                     void* d_ubar, double* qbar, double* pbar, double* theta_bar, int ntheta);

/* Number of kernels this context has launched so far. */
int64_t mg_kernel_launches(const mg_ctx* ctx);

/* Which propagation kernel mg_propagate uses for this context with its
 * current potential: 1 = the short-axis kernel (D >= 3 axes, all of one
 * length 8, 12 or 16, and a Henon-Heiles or diagonal harmonic potential:
 * several axes transformed per pass over the state), 2 = the same kernel
 * moving its chunks with TMA tensor copies (FP32 storage, 16-point axes),
 * 0 = the general kernel (one pass per axis), -1 for a NULL context or no
 * potential yet.  The same method either way (Sec. II.G); only the memory
 * traffic differs.  mg_create_ex's flags choose. */
int mg_propagate_path(const mg_ctx* ctx);

/* Where the general kernel reads its per-axis tables (Sec. II.G: the
 * separable multipliers and potential columns, sum of N_l entries each):
 * 0 = all in shared memory; bit 1 = the potential columns, k - N_l/2 and the
 * kinetic energies stay in the workspace; bit 2 = the multipliers A, conj(A)/N
 * and K too (FP64 only).  Chosen by mg_create when the tables and the data
 * regions do not fit one CTA's shared memory (axis lengths summing to about
 * 2000 or more).  -1 for a NULL context.  Host-only. */
int mg_tables_in_workspace(const mg_ctx* ctx);

/* Host-only (no GPU): the stage coefficients gamma_1..gamma_S of a named
 * composition (eq:comp_TVT), each stage a second-order step of length
 * gamma_k dt.  Triple jump (Yoshida): S_{2k+2}(h) = S_{2k}(a h) S_{2k}((1-2a) h)
 * S_{2k}(a h), a = 1/(2 - 2^{1/(2k+1)}); Suzuki fractal: S_{2k}(a h)^2
 * S_{2k}((1-4a) h) S_{2k}(a h)^2, a = 1/(4 - 4^{1/(2k+1)}).  Writes at most
 * `max` values to gamma (may be NULL) and returns S, or -1 for an unknown
 * name. */
int mg_scheme_coefficients(const char* scheme, double* gamma, int max);

/* Host-only planning query (no GPU, no context): the axis groups the
 * short-axis kernel uses for a grid of D axes of lengths N in `precision`.
 * Each group is a run of naxes[g] consecutive axes starting at first_axis[g],
 * transformed together in one pass over the state (g = 0 is the group that
 * ends at the last axis; a transform takes one pass per group).  Returns the
 * number of groups, 0 if the grid does not take the short-axis kernel, -1 for
 * an invalid grid.  first_axis and naxes: caller arrays of 8 ints (or NULL);
 * threads, smem_bytes (or NULL): the CTA size and the dynamic shared memory
 * of the cp.async layout (the TMA layout, chosen at mg_create, may differ). */
int mg_short_axis_plan(int D, const int64_t* N, int precision, int* first_axis, int* naxes, int* threads,
                       int* smem_bytes);

/* ---- Diagnostics of the device arithmetic (no counterpart in the paper) ----
 * mg_probe_fma_rate: the measured fused multiply-add rate of the current GPU
 * in TFLOP/s (2 flop per FMA), FP64 (precision = MG_FP64) or FP32
 * (MG_FP32_MIXED): independent FMA chains on every SM, best of three timed
 * launches after a warm-up, on cuda_stream (synchronised).  The FP64
 * propagation is bound by the FP64 units, and its roofline is stated against
 * this rate.
 * mg_probe_expi: e^{i theta} as the kernels evaluate it for their phase
 * factors (table-driven sine and cosine after Tang, with a three-word
 * Cody-Waite reduction by pi/128), for n arguments d_theta (device FP64),
 * written to d_sin and d_cos (device FP64, n each); synchronises cuda_stream.
 * Neither allocates device memory. */
mg_status mg_probe_fma_rate(int precision, void* cuda_stream, double* tflops);

/* The n-point DFT of eq:F_defintion's discrete transform (n = 16) as a dense
 * GEMM on the tensor cores (tcgen05.mma, operands in shared memory,
 * accumulator in tensor memory), applied to nlines independent lines:
 *   y_l[j] = post[j] sum_i e^{s 2 pi i j i / 16} pre[i] x_l[i],
 * s = -1 (inverse = 0) or +1 (inverse = 1), unnormalised.  d_x, d_y: device
 * complex64 (interleaved FP32), 16 values per line, line-major.  pre, post:
 * host complex FP64 (16 values each; post may be NULL for 1).  split = 1:
 * 3xTF32 split products (x = xb + xs, M = Mb + Ms, Xb Mb + Xb Ms + Xs Mb);
 * split = 2: BF16x3 (three bfloat16 terms each, six products); FP32
 * accumulation either way.  split = 0: the same lines through an FP32
 * register DFT (4 x 4 with twiddles) on the FP32 units, the comparison for
 * the tensor-core forms.  Synchronises cuda_stream; MG_ERR_TIMEOUT if a
 * tensor-core completion wait ran out (every wait is bounded). */
mg_status mg_probe_tc_dft16(int split, int inverse, const void* d_x, void* d_y, int64_t nlines, const double* pre,
                            const double* post, void* cuda_stream);
mg_status mg_probe_expi(const double* d_theta, double* d_sin, double* d_cos, int64_t n, void* cuda_stream);

/* <x> under the Morse ground state above (host quadrature helper for
 * choosing an initial grid centre). */
double mg_morse_mean(double Dm, double a, double re, double mass, double hbar);

const char* mg_status_string(int status);

/* Propagation without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory -
 * code running inside a host application or framework that owns all device
 * memory through its own pool and forbids plug-ins to call cudaMalloc, or a
 * latency-critical loop in which an allocation (which may synchronise the
 * device) is not acceptable.  It does what mg_create + mg_set_potential +
 * mg_set_state(NULL, q, p, 0) + mg_propagate + mg_get_state(NULL, q, p, ...)
 * do, but its scratch lives in a 768 KiB array inside the library (held by
 * every GPU that loads the library until the process exits) instead of a
 * caller-provided workspace; it calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *  - d_psi: device buffer of prod(N) complex128 values holding the scaled
 *    state u^J = psi(x^J) sqrt(prod dq_l), updated in place.  FP64 only.
 *  - q, p: host arrays of D doubles, the grid centres on entry and on exit.
 *  - grid_motion: MG_GRID_ADAPTIVE, MG_GRID_ADAPTIVE_CENTRE_P or
 *    MG_GRID_FIXED; MG_GRID_NAIVE returns MG_ERR_UNSUPPORTED (it needs the
 *    context's state-sized scratch buffer).
 *  - Other arguments as in mg_create, mg_set_potential and mg_propagate.
 *  - Limits: sum of the axis lengths <= 4096 and at most 1024 CTAs; larger
 *    grids return MG_ERR_UNSUPPORTED before any device work.
 *  - The array's device address is looked up (cudaGetSymbolAddress, with
 *    the device current) by the first call on each device and kept for the
 *    process; that first call should come before any stream capture begins
 *    on the device.  The kept address does not survive cudaDeviceReset: do
 *    not call this entry point again in a process after a device reset.
 *  - All calls share the one array: calls that overlap on the GPU (other
 *    streams, other host threads) race and corrupt each other.  The call
 *    synchronises `cuda_stream` before it returns. */
mg_status mg_propagate_noalloc(int D, const int64_t* N, const double* dq, const double* minv, double hbar,
                               int pot_kind, const double* pot_params, int npot, void* d_psi, double* q,
                               double* p, int64_t n_steps, double dt, const char* scheme, int split,
                               int grid_motion, void* cuda_stream);

/* ---- Batched propagation ---------------------------------------------------
 * Many independent grids of uneven sizes and potentials advanced by one
 * persistent launch.  The paper propagates one wavepacket at a time; the
 * batch applies the same integrator (the substeps of Sec. II.G composed as in
 * eq:comp_TVT) to every problem independently, with results equal to
 * mg_propagate on each context up to the order of floating-point sums.
 *
 * Each problem is an existing context (mg_create + mg_set_potential + a
 * state), which keeps its own state buffer and workspace; the batch adds only
 * the launch.  A team of `cluster` CTAs (a thread-block cluster) propagates
 * one problem at a time; problems are dealt to teams longest first.  The
 * launch (upload of the run parameters + the kernel) is captured once into a
 * CUDA graph at mg_batch_create and replayed by every mg_batch_propagate. */
typedef struct mg_batch mg_batch;

/* Device workspace bytes a batch of `nprob` problems needs (0 if nprob < 1). */
size_t mg_batch_workspace_bytes(int nprob);

/* Create a batch over nprob contexts.
 *  - ctxs: nprob contexts, all of one precision, created on one CUDA stream
 *    (the batch runs on it), with a potential and a state set, and at most 3
 *    axes each.  A context may appear once only.  The contexts must outlive
 *    the batch.
 *  - cluster: CTAs per team, 1, 2, 4 or 8 (0 = 2).
 *  - tile_bytes: NULL or nprob targets for the bytes of one FFT tile of that
 *    problem (0 = default); radix_max: NULL or nprob largest Stockham radix
 *    (0 = default, else 2, 4 or 8).  These are the knobs the autotuner sets.
 *  - d_work: caller-owned device buffer of mg_batch_workspace_bytes(nprob)
 *    bytes, 256-byte aligned; the batch also allocates a small pinned host
 *    block for the run parameters.
 * Returns MG_ERR_STATE if a context lacks a potential or a state,
 * MG_ERR_UNSUPPORTED for contexts with more than 3 axes or a layout that does
 * not fit in shared memory. */
mg_status mg_batch_create(mg_batch** out, int nprob, mg_ctx* const* ctxs, int cluster, const int* tile_bytes,
                          const int* radix_max, void* d_work, size_t work_bytes);

/* Advance every problem by n_steps of the named scheme with its own time step
 * dt[i] (nprob host doubles); split and grid_motion as in mg_propagate, for
 * all problems.  Potentials changed through mg_set_potential since the last
 * call are picked up.  Asynchronous on the contexts' stream: per-problem
 * failures (non-finite reductions, diverging centres) are reported by
 * mg_batch_sync and by each context's next synchronising call. */
mg_status mg_batch_propagate(mg_batch* batch, int64_t n_steps, const double* dt, const char* scheme, int split,
                             int grid_motion);

/* Wait for the batch; returns the status of the first failed problem (its
 * index in *first_failed, else -1) or MG_OK. */
mg_status mg_batch_sync(mg_batch* batch, int* first_failed);

/* Launch shape: CTAs per team, teams, dynamic shared memory per CTA, and the
 * number of batched launches so far. */
mg_status mg_batch_info(const mg_batch* batch, int* cluster, int* nteams, int* smem_bytes, int64_t* launches);

mg_status mg_batch_destroy(mg_batch* batch);

#ifdef __cplusplus
}
#endif
#endif
