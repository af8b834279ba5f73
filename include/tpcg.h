/*
 * tpcg.h -- C ABI of libtpcg: pseudoinverse-preconditioned CG for the
 * finite-difference Poisson problem  -Laplace(ups) = eta  on a 2D rectangle
 * or 3D cuboid (Chumchal, Marton, Plesinger, Simunkova, "Tensor-structured PCG
 * for finite difference solver of domain patterns in ferroelectric material").
 *
 * Operator (eq. ourproblem2, Sec. 3.3):
 *     L = I_t (x) I_q (x) L_n  +  I_t (x) L_q (x) I_n  +  L_t (x) I_q (x) I_n,
 * where L_l = L_l(alpha, beta, gamma) / h_l^2 is the 1D FD minus-Laplacian of
 * eq. (lap1d) (Sec. 3.1) with the corner entries fixed by the axis' boundary
 * condition.  Solver: PCG, Algorithm 1 (Sec. 4.1), with the Moore-Penrose
 * pseudoinverse preconditioner of Algorithms 5 and 7 (Sec. 4.3.3): project on
 * the 1D eigenvector bases by three mode products, multiply by the Hadamard
 * pseudoinverse of all eigenvalue sums (zero on the null space), project back.
 *
 * Data layout.  A grid function is a contiguous array of nz*ny*nx doubles with
 * x fastest, then y, then z -- the paper's vec() order (first index fastest,
 * Sec. 2.1); as a PyTorch tensor it has shape (nz, ny, nx).  nz == 1 selects
 * the 2D problem (Algorithms 4/6); bc[2] and h[2] are then ignored.
 *
 * Conventions.
 *  - Every function returns a status code (TPCG_OK == 0).  No C++ exception
 *    crosses this boundary.  tpcg_strerror() names a code.
 *  - "device pointer" means memory of the CUDA device that was current when
 *    the plan was created; "host pointer" means ordinary or pinned host memory.
 *  - Work is issued on the plan's CUDA stream (stream-ordered).  Functions that
 *    return a tpcg_info (or host data) synchronise that stream before they
 *    return; the others only enqueue work.
 *  - The caller owns eta/ups buffers; the plan owns its eigenbases and
 *    workspaces and frees them in tpcg_plan_destroy().
 *  - A plan is not thread-safe: one host thread at a time per plan.
 */
#ifndef TPCG_H
#define TPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TPCG_OK                 0
#define TPCG_ERR_INVALID_ARG    1  /* bad size, BC code, spacing, pointer or tolerance */
#define TPCG_ERR_OOM            2  /* device or host allocation failed */
#define TPCG_ERR_CUDA           3  /* a CUDA runtime/driver call failed */
#define TPCG_ERR_NOT_CONVERGED  4  /* maxit reached; ups holds the last iterate */
#define TPCG_ERR_BREAKDOWN      5  /* rho <= 0, <W,P> <= 0 or a non-finite scalar (e.g. NaN in eta) */
#define TPCG_ERR_TIMEOUT        6  /* a bounded device-side wait gave up */
#define TPCG_ERR_UNSUPPORTED    7  /* valid request this build cannot serve (e.g. axis > 256 for tensor-core forms) */
#define TPCG_ERR_EIGENBASIS     8  /* closed-form eigenbasis failed its accuracy check */
#define TPCG_ERR_ADMISSION      9  /* server: the request can never fit the device-memory budget */
#define TPCG_PENDING           10  /* server: the request has not finished yet */
#define TPCG_ERR_UNKNOWN_TICKET 11 /* server: no such (unreleased) request */
#define TPCG_ERR_CANCELLED     12  /* server: request still queued when the server was destroyed */

/* ---- boundary conditions per axis (list under eq. lap1d, Sec. 3.1) ---- */
#define TPCG_BC_P   0  /* periodic:          (alpha, beta, gamma) = (2, 2, -1) */
#define TPCG_BC_D   1  /* Dirichlet:                                (2, 2,  0) */
#define TPCG_BC_N   2  /* Neumann:                                  (1, 1,  0) */
#define TPCG_BC_DN  3  /* Dirichlet at index 1, Neumann at index n: (2, 1,  0) */
#define TPCG_BC_ND  4  /* Neumann at index 1, Dirichlet at index n: (1, 2,  0) */

/* ---- precision forms of the preconditioner (Algorithm 7) ---------------
 * In every form the residual r = eta - L ups, the CG inner products, alpha,
 * beta, the solution update and the null-space (mean) projection are FP64;
 * only the three forward and three backward mode products change.        */
#define TPCG_FP64         0  /* mode products in FP64 (CUDA cores)                   */
#define TPCG_MIXED_TF32   1  /* TF32 tensor-core mode products (FP32 containers rounded
                                to nearest even at the 10-bit TF32 mantissa), FP32
                                accumulation and FP32 intermediates: FP32's range,
                                no scaling; one launch per mode product, the
                                eigenbasis streamed with the data                   */
#define TPCG_MIXED_BF16   2  /* BF16 tensor-core mode products, FP32 accumulation    */
#define TPCG_MIXED_FP16   3  /* FP16 tensor-core mode products, FP32 accumulation;
                                R is scaled by a power of two to unit RMS before the
                                conversion and the Hadamard step by 2^-s so every
                                intermediate stays inside the FP16 range; the scale
                                is undone exactly on Z                              */
#define TPCG_MIXED_BF16X3 4  /* split BF16 tensor-core mode products: every operand x
                                (R, the eigenbases, each intermediate) is carried as
                                two BF16 words hi = bf16(x), lo = bf16(x - hi), and
                                each K step issues three MMAs, hi.hi + lo.hi + hi.lo,
                                into one FP32 accumulator (the lo.lo term, 2^-16
                                relative, is dropped): mode products accurate to
                                about 2^-16 instead of 2^-8, so CG needs fewer
                                refinement iterations; one launch per mode product
                                (the pair around G fused, TPCG_OPT_FUSE_G), the
                                eigenbasis streamed with the data, intermediates
                                4 B per point (hi and lo planes).  R enters scaled
                                by a power of two to unit RMS, split from its FP32
                                round-to-odd image (lo exact to one unit of its last
                                place); the scale is undone exactly on Z           */

/* ---- tpcg_solve flags ---------------------------------------------------- */
#define TPCG_ZERO_GUESS   1u  /* ignore ups on entry and start from ups = 0 */

typedef struct tpcg_plan tpcg_plan;

/* Per-solve report.  Residuals are relative to ||eta_hat||_2, where eta_hat is
 * eta after the null-space projection of eq. (centering) (Sec. 3.4.1) when
 * the operator is singular (every present axis P or N), else eta itself.   */
typedef struct {
  int    status;            /* same value the call returned                         */
  int    iters;             /* PCG iterations s performed (Algorithm 1)               */
  int    precond_applies;   /* applications of the preconditioner                  */
  int    prec;              /* precision form used                                  */
  double rel_res_true;      /* ||eta_hat - L ups||_2 / ||eta_hat||_2, FP64, at exit  */
  double rel_res_recur;     /* ||R_s||_2 / ||eta_hat||_2 of the CG recurrence        */
  double eta_norm;          /* ||eta_hat||_2                                        */
  double removed_mean;      /* mean removed from eta (singular operators), else 0   */
  double null_component;    /* mean removed from ups at exit (singular), else 0     */
  int    checks;            /* evaluations of the true residual (stop-test checks   */
                            /* behind Remark stoppincrit, plus the exit report)     */
} tpcg_info;

/* Create a plan for an nx x ny x nz grid (eq. lap1d requires n >= 3 on every
 * present axis; nz == 1 is the 2D problem).  bc[3] holds TPCG_BC_* codes for
 * x, y, z; h[3] the grid spacings (> 0; L_l is divided by h_l^2).  prec is a
 * TPCG_FP64 / TPCG_MIXED_* form.  stream is a cudaStream_t (NULL = the legacy
 * default stream) on which all of the plan's work is issued.
 * Plan setup (Algorithm 5): per axis the eigenpairs of L_l from the closed
 * forms of Lemmas spectrumP/D/N/M (Sec. 3.2), orthonormalised, checked
 * against L_l (||V^T V - I||_max and ||L - V Lambda V^T||_F), and copied to
 * the device with the workspaces.  On error *out is NULL.                   */
int tpcg_plan_create(int nx, int ny, int nz, const int bc[3], const double h[3], int prec, void* stream,
                     tpcg_plan** out);

/* Release all device and host memory of a plan (synchronises its stream).  */
int tpcg_plan_destroy(tpcg_plan* plan);

/* Change the stream on which the plan issues its work.                     */
int tpcg_plan_set_stream(tpcg_plan* plan, void* stream);

/* Bytes of device memory the plan holds (eigenbases + workspaces).         */
int tpcg_plan_device_bytes(const tpcg_plan* plan, size_t* bytes);

/* Solve L ups = eta by PCG (Algorithm 1) with the pseudoinverse
 * preconditioner (Algorithm 7).  eta, ups: device pointers, nz*ny*nx doubles
 * each, layout above; eta is read only; ups holds the initial guess on entry
 * (unless flags has TPCG_ZERO_GUESS) and the solution on exit.  Singular
 * operators: eta is centred (eq. centering), Z is centred every iteration
 * (Remark orthogonality) and ups is returned with zero mean (the minimum-norm
 * solution).  Stops when the recurrence residual is <= tol*||eta_hat||
 * and an FP64 evaluation of ||eta_hat - L ups|| confirms it (Remark
 * stoppincrit: the paper stops at a fixed count; the true residual is used
 * here).  tol in (0, 1), maxit >= 1.  info (host pointer, may be NULL)
 * receives the report.  Synchronises the plan's stream.
 * Returns TPCG_OK, TPCG_ERR_NOT_CONVERGED (ups = last iterate),
 * TPCG_ERR_BREAKDOWN, TPCG_ERR_TIMEOUT or an argument/CUDA error.           */
int tpcg_solve(tpcg_plan* plan, const double* eta, double* ups, double tol, int maxit, unsigned flags,
               tpcg_info* info);

/* As tpcg_solve, with eta and ups in HOST memory (pinned memory gives the
 * fastest copies).  The copies in and out run on the plan's stream through
 * plan-owned device buffers.                                               */
int tpcg_solve_host(tpcg_plan* plan, const double* eta_host, double* ups_host, double tol, int maxit,
                    unsigned flags, tpcg_info* info);

/* Solve L ups_host[i] = eta_host[i] for i = 0 .. nrhs-1 on one plan, every
 * vector in HOST memory (pinned memory lets the copies overlap): the
 * copy in of right-hand side i+1 and the copy out of solution i-1 run on
 * plan-owned copy streams while solve i runs, through two plan-owned pairs of
 * device buffers (allocated on first use; tpcg_plan_device_bytes counts
 * them).  Each solve is the one tpcg_solve_host performs (same arguments
 * tol, maxit, flags; Algorithm 1); ups_host[i] holds the initial guess unless
 * flags has TPCG_ZERO_GUESS.  infos (host array of nrhs, may be NULL)
 * receives one report per solve.  The solves have no counterpart in the
 * paper beyond Algorithm 1 itself: this call only schedules their copies.
 * Returns when every solution is in host memory: TPCG_OK, else the first
 * per-solve status that was not TPCG_OK (every solve still runs), or
 * TPCG_ERR_INVALID_ARG (nrhs < 0, a NULL array or entry, tol or maxit out of
 * range: nothing runs), TPCG_ERR_OOM, TPCG_ERR_CUDA.                        */
int tpcg_solve_host_stream(tpcg_plan* plan, int nrhs, const double* const* eta_host, double* const* ups_host,
                           double tol, int maxit, unsigned flags, tpcg_info* infos);

/* Plan options (no counterpart in the paper: they choose how the library
 * schedules the same arithmetic).
 * TPCG_OPT_DEFER_U (mixed forms; 0 = off, the default): instead of updating
 * U every iteration (Algorithm 1, U += alpha P), the update records alpha and
 * the direction, which stays in a ring of eight, and U is formed with the same
 * FP64 operations in the same order (bitwise the same U) before each
 * true-residual check, every seventh step and before an unconverged iterate is
 * returned.  It moves 16 bytes per grid point per iteration out of the
 * iteration and adds one formation pass bound by the FP64 pipe: slower for one
 * solve at a time, faster in total when several plans solve concurrently
 * (e.g. tpcg_solve_batched over several plans).  Setting it allocates the
 * ring (six more int32 words per grid point than a plan that updates in place;
 * TPCG_ERR_OOM if that fails, the plan unchanged).  Ignored for TPCG_FP64.
 * TPCG_OPT_FUSE_G (mixed forms; 1 = on, the default): the forward and the
 * backward mode product along the axis where the Hadamard step by G is
 * applied (Algorithm 7) run as one kernel that keeps the scaled
 * intermediate in shared memory: one launch and one round trip of the
 * intermediate through memory fewer per preconditioner application, the same
 * operations, bitwise the same Z.  0 runs one launch per mode product.  Used
 * when the axis has at most 128 points, a multiple of 16, and the pass
 * layouts allow it (TPCG_MIXED_BF16X3 with a kernel of its own: split
 * operands, the eigenbasis of that axis resident once, the intermediate's two
 * planes double-buffered); ignored otherwise and for TPCG_FP64 and
 * TPCG_MIXED_TF32 (one launch per mode product).
 * TPCG_OPT_SLICES (TPCG_MIXED_BF16 and TPCG_MIXED_FP16; 1 = on, the
 * default; ignored for the other forms): 3D grids with nx a
 * multiple of 16 and every axis at most 256 points group the six mode products
 * of Algorithm 7 by the data they touch: one launch applies the x and the y
 * product to every z-plane (frontal slice) with the intermediate kept in
 * shared memory, one launch applies the z products and the Hadamard step to
 * the mode-3 fibres (two launches when the z axis exceeds 128 points or
 * TPCG_OPT_FUSE_G is 0), one launch applies the backward x and y products
 * per z-plane.  Same products, same precision; the rounding points of the
 * intermediates differ (x before y in the backward products).  0 keeps one
 * launch per mode product.
 * TPCG_OPT_GRAPHS (0 = off, the default): a solve's launch sequences -- the
 * set-up and each chunk of iterations the host enqueues between reads of the
 * device state -- are captured as CUDA graphs the first time they occur on
 * the plan and replayed afterwards (one graph launch instead of some ten
 * kernel launches per iteration; the kernels read the solve's eta and ups
 * from the device state, so one graph serves every solve of the plan).
 * Same kernels, same order, bitwise the same results.  It pays where one
 * plan solves the same shape of chunk many times and the host's launches
 * are the limit; each new chunk length costs a capture and an instantiation
 * first.  Plans on the legacy default stream (stream NULL) and plans being
 * profiled launch directly.  Changing any option, the comparator
 * preconditioner or the autotuned launch sequence drops the plan's graphs.
 * TPCG_OPT_SWEEP_GRAIN (1..64; 4 = the default): the least work one block
 * of the persistent stencil and pointwise sweeps takes -- this many (32 x 8
 * tile, z-plane) pairs, or 256 x this many grid points -- below the grid of
 * every SM's resident blocks; the per-pass tensor-core launches take at
 * least grain / 8 row tiles of 128 per CTA (one per SM below grain 16).
 * Larger grains run the sweeps of a small grid
 * on fewer SMs, so that the kernels of other plans' streams share the GPU
 * (tpcg_solve_batched over many small grids: 16 measured faster than 4;
 * three concurrent 256 x 256 x 128 plans: 32 fastest of 4..64); a plan
 * solved alone keeps the smaller grain (lower latency).  Grids of
 * 256 x 256 x 128 points and more fill every SM at grains up to 8.  The
 * grain sets the reductions' block count, so results are bitwise
 * reproducible per grain, not across grains.
 * Returns TPCG_OK, TPCG_ERR_OOM (above), or TPCG_ERR_INVALID_ARG (NULL plan,
 * unknown option, value not 0 or 1, a grain outside 1..64).  Set options between solves only: not
 * while another host thread, tpcg_solve_batched or a server request is using
 * the plan.  Setting TPCG_OPT_DEFER_U first waits for the work already
 * enqueued on the plan's stream, then replaces the direction storage.      */
#define TPCG_OPT_DEFER_U 1
#define TPCG_OPT_FUSE_G 2
#define TPCG_OPT_SLICES 3
#define TPCG_OPT_GRAPHS 4
#define TPCG_OPT_SWEEP_GRAIN 5
int tpcg_plan_set_option(tpcg_plan* plan, int option, int value);

/* Autotuner of the preconditioner's launch sequence (no counterpart in the
 * paper: it chooses how the library schedules the same products of
 * Algorithm 7).  For a mixed-form plan it times every distinct sequence the
 * plan offers -- frontal-slice launches or one launch per mode product
 * (TPCG_OPT_SLICES), the products around G fused or not (TPCG_OPT_FUSE_G) --
 * with `applies` preconditioner applications each (CUDA events on the plan's
 * stream, a constant input in the plan's own buffers, nothing allocated),
 * sets the fastest as the plan's options and reports it.  cache_path (host
 * string, may be NULL): a text file of lines "nx ny nz prec slices fuse_g
 * us_per_apply"; a line for this grid and precision is used without timing
 * (from_cache = 1), a new result is appended.  The plan's workspace contents
 * (R, its 16-bit copy, Z) are overwritten: call between solves.  FP64 plans
 * have one sequence: TPCG_OK with candidates = 0.  Synchronises the plan's
 * stream.  TPCG_ERR_INVALID_ARG (NULL plan or out, applies outside 1..1000),
 * TPCG_ERR_CUDA.                                                            */
typedef struct {
  int slices;            /* TPCG_OPT_SLICES chosen                                 */
  int fuse_g;            /* TPCG_OPT_FUSE_G chosen                                 */
  double us_per_apply;   /* its time per preconditioner application (microseconds) */
  int candidates;        /* sequences timed (0 when read from the cache)           */
  int from_cache;        /* 1: taken from cache_path                               */
} tpcg_tune_result;
int tpcg_plan_autotune(tpcg_plan* plan, const char* cache_path, int applies, tpcg_tune_result* out);

/* Many independent solves in one call (the batched form of tpcg_solve).
 * Solve s uses plans[s] and has nrhs[s] right-hand sides (nrhs == NULL: one
 * each) stored back to back: right-hand side r is eta[s] + r*N_s and its
 * solution ups[s] + r*N_s, N_s = nx*ny*nz of plans[s] (device pointers).
 * tol[s] is the tolerance of solve s (tol == NULL: 1e-10); maxit and flags
 * apply to every solve.  infos (host, may be NULL) receives one tpcg_info per
 * right-hand side, in order.  The right-hand sides of one plan are solved one
 * after another (a plan's workspace serves one solve at a time; a plan may
 * appear more than once); different plans advance concurrently, one host
 * thread driving all of them, so plans created on distinct streams overlap
 * on the GPU.  Each result equals the result of tpcg_solve on the same input.
 * Returns TPCG_OK if every solve succeeded, else the first failing status
 * (per-solve statuses are in infos), or an argument/CUDA error.            */
int tpcg_solve_batched(tpcg_plan* const* plans, int nsolves, const int* nrhs, const double* const* eta,
                       double* const* ups, const double* tol, int maxit, unsigned flags, tpcg_info* infos);

/* z = M(r): one application of the plan's preconditioner (Algorithm 7 in the
 * plan's precision form, or the comparator chosen by tpcg_plan_set_precond),
 * without centring.  r, z: device pointers of nz*ny*nx doubles (may not
 * alias).  Enqueues only.                                                    */
int tpcg_precond_apply(tpcg_plan* plan, const double* r, double* z);

/* ---- comparator preconditioners (Sec. 4.3.1; Experiment 2, Sec. 5) ------ */
#define TPCG_PRECOND_PINV    0  /* Moore-Penrose pseudoinverse, Algorithms 5/7 (the default)        */
#define TPCG_PRECOND_NONE    1  /* M = I: unpreconditioned CG                                       */
#define TPCG_PRECOND_JACOBI  2  /* p steps of (weighted) Jacobi from X_0 = 0, Algorithms 2/3:
                                 * X_j = X_{j-1} + (R - L X_{j-1}) / (omega * d), d the Kronecker
                                 * sum of the 1D diagonals (corner entries of eq. lap1d included)  */

/* Select the preconditioner of an FP64 plan (TPCG_ERR_UNSUPPORTED for the
 * mixed forms, whose tensor-core path is the pseudoinverse).  p (1..64) and
 * omega (>= 1, the splitting parameter of Sec. 4.3.1) are used by
 * TPCG_PRECOND_JACOBI only.  Takes effect for the next solve.              */
int tpcg_plan_set_precond(tpcg_plan* plan, int kind, int p, double omega);

/* w = L x: the 7-point (5-point in 2D) Kronecker-sum stencil of eq.
 * (ourproblem), FP64, per-axis corners of eq. (lap1d).  x, w: device
 * pointers of nz*ny*nx doubles (may not alias).  Enqueues only.            */
int tpcg_apply_laplacian(tpcg_plan* plan, const double* x, double* w);

/* Fold constant nonhomogeneous boundary data into a right-hand side in place
 * (Sec. 3.4.2).  bval[2m] is the value on the start face of axis m (index 1),
 * bval[2m+1] on the end face (index n); periodic axes and the absent z axis
 * ignore theirs.  A Dirichlet face adds u_B / h^2 to its boundary layer, a
 * Neumann face adds e_B / h, where e_B is the outward normal derivative (the
 * sign reading of Problem 2, Sec. 5.1).  eta: device pointer (nz*ny*nx
 * doubles); bval: host pointer.  Enqueues only.                           */
int tpcg_rhs_add_bc(tpcg_plan* plan, double* eta, const double bval[6]);

/* The electric field of a potential, epsilon = -grad(ups) (Sec. 2; the text's
 * "nabla dot" of the scalar potential is read as the gradient), by central
 * differences  -(u_{i+1} - u_{i-1}) / (2 h)  per axis.  The neighbour across a
 * face is the ghost value of the plan's boundary condition (eq. lap1d) with
 * the face data of tpcg_rhs_add_bc: periodic faces wrap, a Dirichlet face
 * holds u_B, a Neumann face holds u_boundary + h e_B (e_B the outward normal
 * derivative).  bval: host pointer to 6 doubles laid out as for
 * tpcg_rhs_add_bc, or NULL for homogeneous data.  ups, ex, ey, ez: device
 * pointers of nz*ny*nx doubles (x, y, z components); ez is ignored (may be
 * NULL) for a 2D plan; outputs may not alias ups.  Enqueues only.           */
int tpcg_efield(tpcg_plan* plan, const double* ups, const double bval[6], double* ex, double* ey, double* ez);

/* ---- diagnostics of the CG recurrence (Algorithm 1, Sec. 4.1) ------------
 * The scalars of the plan's most recent iteration, as the device computed
 * them: for the last completed iteration s (0-based, iter = s + 1) alpha_s =
 * rho_s / <W_s, P_s> with W_s = L P_s, beta_s (the coefficient that formed
 * P_s = Z_s + beta_s P_{s-1}; 0 for the first direction), rho_s = <R_s, Z_s>
 * with Z_s centred (Remark orthogonality), the recurrence's ||R_{s+1}||^2 and
 * sum(R_{s+1}), and the mean of Z_s.  The mixed forms accumulate these per
 * thread in FP32 and combine them in FP64, and take rho from the FP16/BF16
 * copy of R the preconditioner read; the FP64 form computes them in FP64.
 * Valid after a solve that stopped (e.g. maxit reached) until the next call
 * that runs the plan.  Synchronises the plan's stream.                     */
typedef struct {
  int    iter;               /* iterations completed                                   */
  double alpha, beta, rho;   /* alpha_s, beta_s, rho_s                                 */
  double wp;                 /* <W_s, P_s> = <L P_s, P_s>                              */
  double rr, sum_r;          /* ||R_{s+1}||^2 and sum(R_{s+1}) of the recurrence       */
  double mean_z;             /* mean(Z_s) (singular operators; 0 otherwise)            */
  int    lp_shift;           /* FP16, split: R_s entered the preconditioner as R_s*2^k */
  int    direction_exponent; /* mixed forms: P_s = P_int * 2^-k (int32 fixed point)   */
} tpcg_cg_scalars;
int tpcg_plan_cg_scalars(tpcg_plan* plan, tpcg_cg_scalars* out);

/* FP64 copies of the plan's current CG vectors (device pointers of nz*ny*nx
 * doubles, each may be NULL): R (the residual the last update or check
 * wrote), Z (the last preconditioner output, exact conversion of the mixed
 * forms' FP32 Z) and P_s (the last direction; the mixed forms' fixed point
 * converted exactly).  Synchronises the plan's stream.                     */
int tpcg_plan_cg_vectors(tpcg_plan* plan, double* R, double* Z, double* P);

/* Copy the FP64 eigenpairs of axis (0 = x, 1 = y, 2 = z) to host memory:
 * lam[ell] (already divided by h^2) and V[ell*ell] row-major with column k
 * the eigenvector of lam[k] (eq. eig-svd-decomp).  ell is the axis length
 * (1 for the absent z axis of a 2D plan: lam = {0}, V = {1}).              */
int tpcg_plan_eigenpairs(const tpcg_plan* plan, int axis, double* lam, double* V);

/* ---- serving: continuous batching of independent solves -------------------
 * A domain-structure simulation issues a Poisson solve every time step (the
 * motivation of Sec. 1 and Sec. 6).  A server owns one worker thread on the
 * device that was current at tpcg_server_create.  Requests wait in arrival
 * order and are admitted as soon as a slot (at most max_slots solves run at
 * once) and device memory are free; each admitted solve runs on its own plan
 * and CUDA stream, so solves of different sizes overlap on the GPU while new
 * requests keep arriving.  Plans are cached by (grid, BCs, spacing,
 * precision), as many as the budget holds, and evicted least-recently-used
 * when idle and memory is needed.
 * A request with session != 0 starts from the previous solution of that
 * session (warm start), which stays on the device; the requests of one
 * session run in submission order, so every result equals the result the
 * same sequence of requests gives when run alone.                           */
typedef struct tpcg_server tpcg_server;

typedef struct {
  int nx, ny, nz;                /* grid; nz == 1: 2D                                     */
  int bc[3];                     /* TPCG_BC_* per axis                                    */
  double h[3];                   /* spacings                                              */
  int prec;                      /* TPCG_FP64 / TPCG_MIXED_*                              */
  unsigned long long session;    /* 0: start from zero; else warm start within the session */
  const double* eta;             /* HOST pointer, nz*ny*nx doubles, copied by submit      */
  double tol;                    /* relative residual tolerance, (0, 1)                   */
  int maxit;                     /* >= 1                                                  */
  unsigned flags;                /* TPCG_REQ_* below                                      */
} tpcg_request;

/* tpcg_request.flags: by default submit copies eta.  With a BORROW flag the
 * server reads eta from the caller's buffer when the request is admitted; the
 * buffer must stay valid and unchanged until the result has been taken.      */
#define TPCG_REQ_BORROW_HOST   1u  /* eta is host memory (pinned gives the fastest copy) */
#define TPCG_REQ_BORROW_DEVICE 2u  /* eta is device memory of the server's device        */

typedef struct {
  unsigned long long submitted, completed, failed, rejected;
  int queued, running;
  size_t device_bytes;           /* plans, session solutions and buffers now held         */
  double p50_ms, p99_ms, mean_ms; /* submit -> result-on-host latency of finished requests */
  double elapsed_s;              /* first submit -> last finished request                 */
} tpcg_server_stats;

/* hbm_budget: device bytes the server may hold (0: 90% of the free memory). */
int tpcg_server_create(size_t hbm_budget, int max_slots, tpcg_server** out);
/* Queue a request (eta is copied before the call returns); *ticket names it. */
int tpcg_server_submit(tpcg_server* server, const tpcg_request* req, unsigned long long* ticket);
/* Non-blocking: TPCG_PENDING, or the request's final status; the result
 * (ups_out: host, nz*ny*nx doubles, may be NULL; info may be NULL) is handed
 * out once and the ticket released.  TPCG_ERR_ADMISSION: the request alone
 * exceeds the budget.                                                        */
int tpcg_server_poll(tpcg_server* server, unsigned long long ticket, double* ups_out, tpcg_info* info);
/* As poll, blocking up to timeout_s seconds (< 0: no limit).                */
int tpcg_server_wait(tpcg_server* server, unsigned long long ticket, double timeout_s, double* ups_out,
                     tpcg_info* info);
int tpcg_server_get_stats(tpcg_server* server, tpcg_server_stats* stats);

/* Where each finished request spent its latency (submit -> result in host
 * memory), one record per request finished since the server was created or
 * its statistics were last reset (at most 2^20 kept), in finishing order.
 * queue_ms + build_ms + solve_ms + copy_ms = total_ms.  No counterpart in the
 * paper: it explains the serving latency of Sec. 1's time-stepping use.     */
typedef struct {
  unsigned long long ticket, session;
  int nx, ny, nz, prec;
  int status, iters;
  int plan_built;      /* 1: no idle cached plan of this key; one was created   */
  double queue_ms;     /* submit -> admitted (slot and device memory free)      */
  double build_ms;     /* admitted -> solve enqueued: plan creation (cache miss) */
  double solve_ms;     /* copy of eta in, the PCG iterations, exit work          */
  double copy_ms;      /* copy of the solution to host memory                    */
  double total_ms;
} tpcg_request_timing;
/* Copies up to max_records records to out (host array) and their count to
 * *n_records; max_records == 0 only reports how many are held.              */
int tpcg_server_get_timings(tpcg_server* server, tpcg_request_timing* out, int max_records, int* n_records);
/* Clear the counters and the latency record (e.g. after a warm-up phase).  */
int tpcg_server_reset_stats(tpcg_server* server);
/* Lets running requests finish, cancels queued ones, releases everything.  */
int tpcg_server_destroy(tpcg_server* server);

/* ---- instrumentation ------------------------------------------------------
 * Number of CUDA kernels the plan has launched since it was created.       */
int tpcg_plan_launch_count(const tpcg_plan* plan, unsigned long long* launches);

/* Tensor-core kernel launches per preconditioner application of a mixed-form
 * plan under its current options: one per mode product of Algorithm 7 (six
 * in 3D, four in 2D), one fewer with TPCG_OPT_FUSE_G where it applies; 0 for
 * TPCG_FP64.  TPCG_OK, or TPCG_ERR_INVALID_ARG for a NULL argument.         */
int tpcg_plan_precond_launches(const tpcg_plan* plan, int* launches);

/* Per-kernel-kind device time, measured with CUDA events recorded on the
 * plan's stream around every launch between tpcg_profile_begin() and
 * tpcg_profile_end().  Kinds: eta_sum, init_residual, direction, update,
 * true_residual, center, laplacian, modeprod_f64, modeprod_tc, convert.    */
typedef struct {
  char name[24];
  unsigned long long launches;  /* launches recorded while profiling          */
  double total_ms;              /* summed event-to-event time of those launches */
} tpcg_kernel_stat;

int tpcg_profile_begin(tpcg_plan* plan);
/* Synchronises the stream, stops recording, writes up to max_stats entries
 * (kinds with at least one launch) and their count to *n_stats.            */
int tpcg_profile_end(tpcg_plan* plan, tpcg_kernel_stat* stats, int max_stats, int* n_stats);

/* ---- allocation-free residual check ----------------------------------------
 * No counterpart in the paper.  For callers that must not allocate device
 * memory at the time they check a solution: time-stepping loops that cannot
 * afford the device synchronisation cudaMalloc/cudaFree may cause,
 * applications that hand this library a fixed budget at start-up and own
 * every allocation after it, or code running where allocating is not
 * allowed.  No plan is needed and nothing is allocated (no cudaMalloc, no
 * cudaFree, no allocating library call).
 *
 * Writes, on `stream`, out[0] = ||eta_hat - L ups||_2, out[1] = ||eta_hat||_2
 * and out[2] = the mean removed from eta (0 unless every present axis is P or
 * N), where L is the operator tpcg_plan_create(nx, ny, nz, bc, h, ...) would
 * build and eta_hat = eta - out[2].  eta, ups: device pointers of nz*ny*nx
 * doubles (layout as above); out: device pointer of 3 doubles.  Enqueues only.
 * Scratch: a static device array of the library (about 33 KB per GPU that
 * loads it, held until the process exits) for the partial sums of at most
 * 2048 reduction blocks.  Grids of more than 2^31 - 1 points are rejected with
 * TPCG_ERR_UNSUPPORTED.  The first call on a device looks the array's address
 * up (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  A new context on the device (after
 * cudaDeviceReset) moves the array; the next call notices the new context
 * and looks the address up again (make that call outside a capture too).
 * An error already pending in the calling thread (cudaPeekAtLastError) is
 * left in place and reported as TPCG_ERR_CUDA before anything is enqueued.
 * Every call uses the same array: calls that may run concurrently on the GPU
 * (different streams, no ordering between them) race and must not be issued.
 * Each call clears the array's arrival counters before use.               */
int tpcg_residual_norms_noalloc(int nx, int ny, int nz, const int bc[3], const double h[3], const double* eta,
                                const double* ups, double* out, void* stream);

/* Human-readable name of a status code (static string, never NULL).        */
const char* tpcg_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* TPCG_H */
