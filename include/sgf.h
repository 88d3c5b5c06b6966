/*
 * sgf.h -- C ABI of the GB300 library for the FFT-accelerated, shifted-Green-function Nystrom
 * operator of Bruno & Maas, "Shifted equivalent sources and FFT acceleration for periodic
 * scattering problems, including Wood anomalies" (arXiv:1707.04950).
 *
 * Conventions shared by every entry point
 *  - Profile f(x) = a[0] + sum_{m=1..M} a[m] cos(2 pi m x/d) + b[m] sin(2 pi m x/d), period d.
 *  - Nystrom nodes x_l = l d/N, l = 1..N (Section 4.2); vectors are length N, index l-1.
 *  - Complex vectors are interleaved (re, im) pairs of double (complex128) in DEVICE memory unless
 *    an entry point says "host". The caller owns every buffer it passes; the library never frees
 *    or retains caller pointers beyond the call.
 *  - All work is enqueued on the stream given to sgf_create; calls that return results to host
 *    memory synchronise that stream before returning. Device-output calls do not synchronise.
 *  - Every call returns sgf_status; SGF_OK is 0. On failure sgf_last_error() holds a message.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef SGF_H
#define SGF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgf_ctx sgf_ctx;

typedef enum {
  SGF_OK = 0,
  SGF_EINVAL = 1,          /* bad argument or parameter combination                          */
  SGF_ERESONANT_CELL = 2,  /* -k^2 is (close to) a Dirichlet eigenvalue of the cell (Remark non-resonant) */
  SGF_EPOLE_ON_GRID = 3,   /* a shifted pole (0, -m h) falls on a lag of an equivalent-source grid */
  SGF_EWINDOW = 4,         /* window constraints violated: a >= L, or h <= a max|f'| (Remark a_cond) */
  SGF_ENOCONV = 5,         /* GMRES did not reach the tolerance within maxit                  */
  SGF_EBREAKDOWN = 6,      /* Krylov breakdown                                                 */
  SGF_ENONFINITE = 7,      /* a non-finite value was produced                                   */
  SGF_ETIMEOUT = 8,        /* reserved: no kernel of this library waits on a device flag, so no
                              call returns it                                                   */
  SGF_ECUDA = 9,           /* a CUDA runtime call failed                                        */
  SGF_ESTATE = 10          /* call order violated (e.g. apply before build)                    */
} sgf_status;

/* Numerical parameters of one problem (Sections 3-5). Lengths in the units of d and 1/k. */
typedef struct {
  int N;            /* Nystrom nodes per period                                                 */
  int j;            /* number of shifts of the multipolar Green function (eq. shifted_green_function) */
  double h;         /* shift length h (poles at (0, -m h), 1 <= m <= j)                          */
  int n_per;        /* smooth truncation A = n_per d of the spatial lattice sum (eq. Gq_limit)      */
  double c_win;     /* flat fraction c of the window S_{cA,A}                                   */
  int Ma;           /* singular window a = Ma dx (eq. dsing_def); gamma = a/2                     */
  double eta;       /* mode-completion threshold (eq. M_eta)                                      */
  int nx, ny;       /* cells: d = nx L, cell box [hmin, hmin + ny L) (eq. L_constr)               */
  double hmin;      /* bottom of the reference periodicity domain                                 */
  int p, e;         /* equivalent sources: spacing L/p, e extra points per side end (eq. eq_mesh)  */
  int n_coll;       /* collocation points on the boundary of S_q (eq. eq_source_point)           */
  int n_fb;         /* order of the cell reconstruction basis, 2 n_fb + 1 functions (eq. planewave) */
  double delta_min; /* spectral series used where min_m |Y + m h| >= delta_min (Section 3.2)     */
  double spec_exp;  /* spectral series truncated where |e^{i beta_n delta}| < e^{-spec_exp}       */
  int precision;    /* 64: all stages FP64; 32: projection, FFT and interpolation in FP32 complex  */
  double ls_reg;    /* Tikhonov weight of the equivalent-source least squares: minimise
                       |A xi - psi|^2 + (ls_reg |A|_F)^2 |xi|^2 (0 = plain QR solution)           */
} sgf_params;

/* Suggested parameters for a problem (profile as for sgf_set_profile_fourier, wave as for
 * sgf_set_wave) and a target accuracy tol in [1e-14, 1e-2], following the parameter guidance of
 * Section 6.1 ("Computing costs"): cells of side L <= 0.45 lambda (n_x a power of two, the cell not
 * resonant); N from 6 log10(1/tol) points per wavelength of arc length (at least 16), a multiple
 * of n_x; the singular window a = 0.95 L; the cell box around the profile; j = 8 shifts near a
 * Wood anomaly (some |beta_n| < k/10), none otherwise; h/lambda from 1/3 (shallow) to 1 (deep:
 * 1/3 + 0.06 H/lambda), clear of the singular window (h > 1.2 a max|f'|) and off the grid lags;
 * n_per doubled from 8 until the
 * windowed lattice sum of G_j next to the shifted images changes by less than tol/10 (at most
 * 16384); the remaining fields at the library's defaults. Host only (no GPU, no context).
 * SGF_EINVAL for arguments out of range. SGF_ENOCONV when the lattice-sum check did not reach
 * tol/10 by n_per = 16384: *out is still filled (with n_per = 16384), but that accuracy is not
 * reached by the windowed sums. */
sgf_status sgf_suggest_params(double d, int M, const double* a, const double* b, double k, double theta_rad, int bc,
                              double tol, int precision, sgf_params* out);

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t (NULL = legacy default). */
sgf_status sgf_create(sgf_ctx** out, int device, void* cuda_stream);
void sgf_destroy(sgf_ctx* ctx);
const char* sgf_last_error(const sgf_ctx* ctx);

/* Surface profile (Section 2): period d, M+1 cosine coefficients a[0..M] and sine coefficients
 * b[0..M] (b[0] ignored), host arrays copied by the call. */
sgf_status sgf_set_profile_fourier(sgf_ctx* ctx, double d, int M, const double* a, const double* b);

/* Incidence e^{i(alpha x - beta y)}, alpha = k sin(theta), beta = k cos(theta) (eq. fist_eq);
 * bc = 0 Dirichlet (TE, double layer), 1 Neumann (TM, single layer). */
sgf_status sgf_set_wave(sgf_ctx* ctx, double k, double theta_rad, int bc);

/* Numerical parameters (copied). Validated by sgf_build_operator. */
sgf_status sgf_set_params(sgf_ctx* ctx, const sgf_params* p);

/* Algorithm 2 (initialisation) on the device: geometry and cells, least-squares factors, the
 * periodised kernel table on the lag grids (hybrid spectral/spatial, Remark large_FFT_eval) and its
 * spectra, per-cell projection and reconstruction matrices, the block-sparse near-field operator
 * (exact intersecting part, singular quadrature of eq. local_mat, local equivalent-source
 * subtraction folded in) and the mode factors of eq. D_M_deltax. Synchronises the stream. */
sgf_status sgf_build_operator(sgf_ctx* ctx);

/* Algorithm 3: out = A mu, A = (sigma/2 I + D^dx) in its accelerated form, for nrhs right-hand
 * sides stored one after another (column stride N). sigma = +1 Dirichlet, -1 Neumann.
 * transpose_conj = 1 applies the conjugate transpose A^H instead: the stages of Algorithm 3 run
 * backwards (reconstruction and sample gather transposed, grid convolution with conjugated spectra,
 * scatter and projection transposed, near-field blocks, mode factors conjugate-transposed), in
 * the same precision as the forward map. mu_dev/out_dev: device complex128, not overlapping.
 * Enqueued on the context stream. SGF_EINVAL for transpose_conj outside {0, 1}, or when the
 * adjoint near-field rows exceed the shared-memory limit (then only the forward map exists). */
sgf_status sgf_apply(sgf_ctx* ctx, const void* mu_dev, void* out_dev, int nrhs, int transpose_conj);

/* Same as sgf_apply with HOST complex128 buffers: copies mu to the device, applies, copies back,
 * synchronises. */
sgf_status sgf_apply_host(sgf_ctx* ctx, const void* mu_host, void* out_host, int nrhs);

/* Right-hand side of eq. discrete_eq at the nodes into out_dev (device complex128, length N). */
sgf_status sgf_rhs(sgf_ctx* ctx, void* out_dev);

/* Algorithm 1: GMRES (restarted after min(1000, maxit) vectors, fewer if the basis would exceed
 * 2 GiB; zero initial guess; CGS2 Arnoldi on FP64 vectors with float-float projections, about 48
 * significant bits; Givens rotations on the host every 1 to 8 steps) on the system with the
 * right-hand side of sgf_rhs; with precision 32 an FP64 residual-refinement loop wraps inner GMRES
 * solves on the mixed operator, the later ones deflated with the first one's Krylov space (GCRO
 * form, up to 256 vectors). Writes the solution to mu_dev; *iters = operator applications,
 * *relres = final ||b - A mu|| / ||b|| with the FP64 operator. Allocates its Krylov storage on the
 * device for the call. Synchronises. */
sgf_status sgf_solve(sgf_ctx* ctx, double tol, int maxit, void* mu_dev, int* iters, double* relres);

/* Algorithm 1 on a caller's right-hand side: GMRES (as in sgf_solve, same precision handling) on
 * A x = rhs (transpose_conj = 0) or A^H x = rhs (transpose_conj = 1, the adjoint system of a
 * gradient computation). rhs_dev, x_dev: device complex128 of length N. Synchronises. */
sgf_status sgf_solve_rhs(sgf_ctx* ctx, const void* rhs_dev, int transpose_conj, double tol, int maxit, void* x_dev,
                         int* iters, double* relres);

/* The unaccelerated Nystrom operator (Section 4: eq. discrete_eq with D^dx = D~_sing + D~_reg + D_M,
 * eqs. local_mat, D_ns, G_jq_s, D_M_deltax; G~ by the hybrid spectral/spatial evaluation of
 * Sections 3.2 and 4.2.3) assembled as a dense row-major N x N complex128 matrix in device memory
 * owned by the context (16 N^2 bytes; 8 <= N <= 32768, 2 <= Ma < N/2). It needs the profile, the
 * wave and the parameters (N, j, h, n_per, c_win, Ma, eta, delta_min, spec_exp; the accelerator's
 * cell parameters are not used) and works with or without sgf_build_operator; a later
 * sgf_build_operator discards it. Assembly evaluates G~ once per entry (a warp per entry, FP64):
 * about 5 s at N = 4096 on one GB300, growing as N^2. Errors: SGF_ESTATE before the setters, SGF_EINVAL for sizes out
 * of range, SGF_EWINDOW (j > 0 and h <= a max|f'|). Synchronises. */
sgf_status sgf_build_exact(sgf_ctx* ctx);

/* Which operator sgf_apply, sgf_apply_host, sgf_solve and sgf_solve_rhs use: 0 the accelerated
 * operator of sgf_build_operator (the default), 1 the dense operator of sgf_build_exact (FP64 GEMV,
 * forward and adjoint; solves skip the mixed-precision refinement). sgf_gradient, sgf_field and
 * batches always use the accelerated operator (sgf_gradient refuses while 1 is selected).
 * SGF_ESTATE when 1 is asked before sgf_build_exact. */
sgf_status sgf_select_operator(sgf_ctx* ctx, int exact);

/* Copy of the dense operator into A_dev (device complex128, N*N, row-major). Synchronises. */
sgf_status sgf_exact_matrix(const sgf_ctx* ctx, void* A_dev);

/* Scattered field off the surface (the remark after Algorithm 3; eq. int_eq_dirichlet discretised
 * with the operator's trapezoid weights: the double layer of mu for Dirichlet, the single layer for
 * Neumann, plus the completion modes M^eta) at n_targets points.
 *   mu_dev    device complex128 [N], a density (normally the solution of sgf_solve)
 *   xy        HOST double [2 n_targets], interleaved (x, y); any x (the field is alpha-quasi-
 *             periodic), y >= h_min (the bottom of the cell box)
 *   u_dev     device complex128 [n_targets], the field in the targets' order
 *   total     0: u^scat; 1: u^scat + u^inc
 * Targets inside the cell box (y < h_min + n_y L) take Algorithm 3 in FP64 with the target in
 * place of a node: the convolved equivalent-source grids, the Fourier-Bessel fit of phi^ni on the
 * target's cell, and the exact sum over the nodes of its local cells. Targets above the box take the
 * Rayleigh form of the same sum (every node lies below them). The trapezoid sum loses accuracy
 * within a few node spacings of the surface (near-singular integrand); the value below the surface
 * is that of the representation, not a physical field.
 * Errors: SGF_EINVAL for a non-finite target, a target below the box, a target on a node, or
 * targets above the box too close to the highest node for the Rayleigh form (fewer than ~2e5
 * modes); SGF_ESTATE before build. Synchronises. */
sgf_status sgf_field(sgf_ctx* ctx, const void* mu_dev, long n_targets, const double* xy, void* u_dev, int total);

/* Rayleigh coefficients B_n for n = n_lo..n_hi (eq. rayexp) from the solution mu (device), into
 * host B[2*(n_hi-n_lo+1)] (interleaved complex); host eff[n_hi-n_lo+1] gets e_n = beta_n/beta |B_n|^2
 * for propagating n (0 otherwise) and *energy_err = 1 - sum over propagating n in the range
 * (eq. energy_error). Synchronises. */
sgf_status sgf_rayleigh(sgf_ctx* ctx, const void* mu_dev, int n_lo, int n_hi, double* B, double* eff,
                        double* energy_err);

/* Same result as sgf_rayleigh, for callers that cannot allocate memory during the call: processes
 * working inside a device-memory budget fixed up front, and real-time loops that must stay out of
 * the allocator (cudaMalloc and cudaFree can synchronise the device and take unbounded time). (The
 * paper has no counterpart; this is a property of the library, not of the method.)
 * It calls no cudaMalloc, cudaFree or other allocating routine, on the device or the host: its
 * scratch (per-mode data and the B_n before they are copied back) lives in a static device array of
 * 1024 modes x 64 bytes that every GPU loading the library holds until the process exits. At most
 * 1024 modes (n_hi - n_lo + 1) per call; larger ranges return SGF_EINVAL with a message. The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress, with that device
 * current). All calls share the one array, which keeps the last call's contents; every entry a call
 * reads is written by that call first. Calls whose GPU work overlaps (other streams, other host
 * threads on the same device) race on the array: serialise them. The call copies through fixed host
 * stack buffers and synchronises the context stream after each copy, so it must not be made on a
 * stream that is being captured into a graph. Accepts the same context states as sgf_rayleigh (a
 * built operator, or the geometry set by sgf_build_exact); SGF_ESTATE otherwise. */
sgf_status sgf_rayleigh_noalloc(sgf_ctx* ctx, const void* mu_dev, int n_lo, int n_hi, double* B, double* eff,
                                double* energy_err);

/* Gradient of the efficiency e_n = (beta_n/beta)|B_n|^2 (eqs. rayexp, energy_error) with respect to
 * the profile's Fourier coefficients a_0..a_M, b_1..b_M (as set by sgf_set_profile_fourier), for the
 * accelerated discrete system. The paper solves forward problems only; this is its discrete adjoint:
 * dB_n = (dw)^T mu + lam^T (db - dA mu) with B_n = w^T mu and A^T lam = w, lam from one adjoint GMRES
 * solve (tol, maxit as sgf_solve_rhs). Every factor of A, b and w depends on one node's position
 * (f, f'), so their derivatives are built analytically, node by node, with the operator's own
 * kernels in derivative mode (Hessian of the shifted Green function for the projection and the near
 * operator, Fourier-Bessel recurrences for the reconstruction rows, derivatives of the window, of the
 * log-singular coefficient and of the mode, incidence and Rayleigh factors), and applied through
 * the forward and adjoint maps; the f'' term of the K_r diagonal is analytic; the chain rule maps
 * node sensitivities to the coefficients. mu_dev: the solution of sgf_solve (device complex128,
 * length N). Host outputs: grad_a[M+1], grad_b[M+1] (grad_b[0] = 0), B[2] = B_n (may be NULL), *e_n
 * (may be NULL; 0 with a zero gradient for an evanescent n), *adj_iters (may be NULL). The cell
 * assignment is that of the build: the gradient is that of the operator with this assignment.
 * Synchronises. */
sgf_status sgf_gradient(sgf_ctx* ctx, const void* mu_dev, int n, double tol, int maxit, double* B, double* e_n,
                        double* grad_a, double* grad_b, int* adj_iters);

/* The same gradient with the node derivatives taken as central differences of the factors rebuilt
 * at all target (or all source) positions moved by +-1e-6 max(1, max|v|), v = f, f' (each factor
 * depends on one node, so one pair of rebuilds gives every node's derivative): a cross-check of
 * sgf_gradient. Same arguments. */
sgf_status sgf_gradient_fd(sgf_ctx* ctx, const void* mu_dev, int n, double tol, int maxit, double* B, double* e_n,
                           double* grad_a, double* grad_b, int* adj_iters);

/* ------------------------------------------------------------------------------------------------
 * Batches of independent problems (different surfaces, wavenumbers or incidence angles, each in its
 * own built context). The paper solves one problem at a time; a batch launches the forward maps of
 * all its problems as independent branches of one CUDA graph so that problems too small to fill
 * the GPU alone share it, and runs GMRES on all of them in lockstep. */
typedef struct sgf_batch sgf_batch;

/* Create a batch over n built contexts (distinct, same device, each with its captured forward map:
 * the default unless the environment sets SGF_NO_GRAPH). The batch keeps the context pointers, not
 * ownership: destroy the batch before its contexts. Work is enqueued on cuda_stream (a
 * cudaStream_t, NULL = legacy default). While a batch call runs, the contexts' staging buffers and
 * grids are in use: do not apply or solve with those contexts on other streams at the same time.
 * On failure *out still receives a batch whose sgf_batch_last_error() explains it; destroy it. */
sgf_status sgf_batch_create(sgf_batch** out, int n, sgf_ctx* const* ctxs, void* cuda_stream);

/* Which form the batch runs: 0 every problem's own forward map (child graphs side by side); 1 the
 * same with one near operator shared among the problems; 2 the multi-column form. Forms 1 and 2
 * apply when all problems have the same profile, wavenumber, boundary condition and parameters
 * and differ only in the incidence angle (Algorithm 1 over several alpha on one surface): the
 * projection P_q and the cell reconstruction rows do not depend on alpha (the twists e^{-i alpha x}
 * of the scatter and e^{i alpha x} of the samples are applied per problem), and the near operators
 * differ only by the quasi-periodic phase e^{i alpha d w} of each block's period copy w. Form 1
 * makes one pass over the first problem's near blocks for every angle; form 2 runs the whole forward
 * map on up to 8 problems per pass: P, the near rows and the reconstruction rows read once for
 * all of them, each problem's spectra, twists and mode factors per column (the first problem's
 * precision for all). sgf_batch_create times the eligible forms and keeps the fastest; the
 * environment variables SGF_BATCH_SHARED=1 (or 0) and SGF_BATCH_MULTI=1 (or 0) force a form. */
int sgf_batch_shared_near(const sgf_batch* batch);
void sgf_batch_destroy(sgf_batch* batch);
const char* sgf_batch_last_error(const sgf_batch* batch);

/* out_devs[p] = A_p mu_devs[p] for every problem p (Algorithm 3 in each context's precision), one
 * graph launch for the whole batch. Host arrays of n device pointers (complex128, length N_p).
 * Enqueued on the batch stream; does not synchronise. */
sgf_status sgf_batch_apply(sgf_batch* batch, const void* const* mu_devs, void* const* out_devs);

/* Algorithm 1 for every problem on its incident-wave right-hand side (as sgf_solve): restarted GMRES
 * (restart length as sgf_solve, bases within 4 GiB for the batch; CGS2 as in sgf_solve) in
 * lockstep: one graph launch per Arnoldi step for all problems, one batched kernel per
 * Gram-Schmidt pass. If any context uses precision 32, every problem runs FP64 residual refinement
 * around inner solves (tolerance 1e-6) on its own operator, the later ones deflated with the first
 * one's Krylov spaces. Solutions go to mu_devs[p];
 * host iters[n] and relres[n] (may be NULL) receive operator applications and the final FP64
 * relative residual of each problem. SGF_ENOCONV names the first problem above tol. Synchronises. */
sgf_status sgf_batch_solve(sgf_batch* batch, double tol, int maxit, void* const* mu_devs, int* iters,
                           double* relres);

/* Copy of the parameters currently set (after sgf_autotune_cells: the ones chosen). */
sgf_status sgf_get_params(const sgf_ctx* ctx, sgf_params* out);

/* Cell-size autotuner (the paper leaves the cell side L to the user within the constraints of
 * Section 5.1: a < L, non-resonant cells). For the profile, wave and parameters set, tries each cell
 * count nx_list[i] (cells of side L = d/nx) with the quantities tied to L re-derived: box bottom
 * hmin = min f - L/2 and rows ny = floor((max f - hmin)/L) + 1, singular window
 * Ma = floor(0.75 L/dx); with shifts (j > 0) the shift follows the rule of sgf_suggest_params:
 * h0 = max(h set, 1.2 a max|f'|) (clear of the singular window, Section 5.1), then
 * h = (round(h0/dg) + 1/(j+1)) dg with dg = L/p (off the grid lags), one dg more if still inside
 * the window. Start from the parameters sgf_suggest_params gives for the problem.
 * Every candidate that builds is timed over `reps` applications; host ms[i] (may be NULL) receives
 * its time per application in milliseconds, or minus the build status for a candidate that does
 * not build. The context is left built with the fastest (*best_nx; sgf_get_params gives its
 * parameters). SGF_EINVAL if no candidate builds (the context is then unbuilt, parameters
 * restored). Rebuilds the operator several times: a set-up step, not for a hot loop. */
sgf_status sgf_autotune_cells(sgf_ctx* ctx, const int* nx_list, int n, int reps, int* best_nx, double* ms);

/* Accuracy-aware form of sgf_autotune_cells: each candidate that builds is also solved on the
 * incident-wave right-hand side (GMRES to 1e-12, at most 4000 applications) and its energy error
 * 1 - sum e_n over the propagating modes (eq. energy_error, the paper's accuracy measure) goes to
 * host eps[i] (may be NULL; 1e300 where no solution was obtained). The fastest candidate with
 * |energy error| < eps_tol is kept. If candidates build but none reaches eps_tol, the context is
 * built with the most accurate one and SGF_ENOCONV is returned with a message. SGF_EINVAL for
 * eps_tol <= 0 or when no candidate builds. A set-up step: it builds and solves once per candidate
 * (and allocates a solution buffer for the duration of the call). */
sgf_status sgf_autotune(sgf_ctx* ctx, const int* nx_list, int n, int reps, double eps_tol, int* best_nx, double* ms,
                        double* eps);

/* Introspection: fills host info[0..23] (the caller's buffer holds 24 doubles) with N, number of
 * occupied cells, near-field entries, P_x^H, rows^H, P_y^H, P_x^V, rows^V, P_y^V, n_eq (per
 * orientation), n_fit, n_fb basis size, |U^eta|, algorithmic bytes of one FP64 matvec, of one mixed
 * matvec, kernel launches per matvec, 1 if applications run as captured CUDA graphs, the longest
 * near-field row, the largest cell node count, log2 of the twiddle table length, then the wall
 * times (ms) of the last sgf_build_operator (Algorithm 2): total, kernel tables and their spectra
 * (the periodised Green function on the grids), least squares with the projection and
 * reconstruction factors, near operator. */
sgf_status sgf_info(const sgf_ctx* ctx, double* info);

/* Device time of the stages of the last sgf_apply when profiling is switched on with
 * sgf_set_profiling(ctx, 1) (the stages then run one after another on the context stream): host
 * times_ms[0..7] = project, forward X-FFT, Y convolution, inverse X-FFT, near field (block-sparse
 * rows, sigma/2 identity), interpolation of the far field + modes, total, unused. */
sgf_status sgf_set_profiling(sgf_ctx* ctx, int on);
sgf_status sgf_stage_times(const sgf_ctx* ctx, double* times_ms);

/* Testing hook: restrict sgf_apply to a subset of its terms. Bit 0 the FFT far field
 * (interpolated phi^all), bit 1 the block-sparse near operator, bit 2 the mode completion D_M,
 * bit 3 the sigma/2 identity. Default 15 (all). */
sgf_status sgf_debug_mask(sgf_ctx* ctx, int mask);

/* Testing hook: force the launch variants of the grid convolution for the following applications
 * (forward and adjoint, every orientation) instead of the per-launch choice: conv_variant 1 = the Y
 * convolution with 16 values per thread in registers, 2 = the same with its partial product in a
 * global scratch array (allocated here if the build did not need it), 3 = 8 values per thread, 0 =
 * chosen per launch; fftx_vpt 8 or 16 values per thread in the X passes, 0 = chosen per launch. The
 * captured forward maps are captured again. SGF_EINVAL if a forced variant does not fit the launch
 * limits (threads, shared memory, registers) of an orientation; SGF_ESTATE before build. A rebuild
 * clears the forcing. Synchronises. */
sgf_status sgf_debug_force_variants(sgf_ctx* ctx, int conv_variant, int fftx_vpt);

/* Copy of internal tables for testing: which = 0 twisted kernel table of orientation lam
 * (0 = H, 1 = V) before the Y transform, [P_x][P_y] complex128 with kind 0 monopole, 1 dipole.
 * Host buffer of P_x*P_y complex128. Synchronises. */
sgf_status sgf_debug_table(const sgf_ctx* ctx, int lam, int kind, void* host_out);

#ifdef __cplusplus
}
#endif
#endif /* SGF_H */
