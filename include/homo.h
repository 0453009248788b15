/*
 * homo.h - C ABI of a GB300 (sm_103a) solver for the per-iteration hot path of
 * density-based inverse homogenization (Zhang et al., "An optimized, easy-to-use,
 * open-source GPU solver for large-scale inverse homogenization problems",
 * arXiv 2301.08911).
 *
 * One optimisation iteration (paper Sec. 3.3 "Solver for IHP", Sec. 5.2 main loop):
 *   homo_filter (rho -> rho~)          Sec. 5.2 / Sec. 6.4 periodic density filter
 *   homo_set_density (rho~ -> E)       SIMP, Sec. 3.2
 *   homo_solve_cases                   6 periodic cell problems K u_i = f_i (Eq. 4-5),
 *                                      multigrid-preconditioned CG (Sec. 3.3, Alg. 1)
 *   homo_CH                            homogenised tensor C^H (Eq. 7)
 *   homo_objective (host arithmetic)   f(C^H), df/dC^H (Eq. 19-22)
 *   homo_sensitivity                   df/d rho~ (Eq. 8-9)
 *   homo_filter (adjoint = itself)     df/d rho
 *   homo_update                        OC volume-constrained update (Sec. 3.3)
 *
 * Grid and layout conventions (every entry point):
 *   - n^3 voxel elements, periodic; n^3 vertices. Scalar element/vertex fields are
 *     float arrays of length N = n^3 with x fastest: index = x + n*(y + n*z).
 *   - Element local vertex j = a + 2b + 4c sits at offset (a,b,c) from the element
 *     origin; element (x,y,z) owns vertices (x..x+1, y..y+1, z..z+1) mod n.
 *   - Displacement / load fields of the 6 load cases are 18 planes of N floats:
 *     plane (3*case + comp), case in Voigt order 11,22,33,12,23,13 (Sec. 3.2),
 *     comp in x,y,z. Total 18*N floats.
 *   - Units: the library works in voxel units (element side 1, |Omega| = N).
 *     Against the paper's Omega = [0,1]^3 (h = 1/n): u_paper = h*u, f_paper = h^2*f,
 *     K_paper = h*K. C^H and sensitivities are unit-free and equal to the paper's.
 *
 * Memory and ownership: a context owns every device buffer it needs (filtered
 * density, moduli, the 6 displacement fields kept as warm starts, the multigrid
 * hierarchy, scratch). Pointers passed in are only read/written inside the call, on
 * the context's stream; "device" pointers must be device-accessible CUDA memory (for
 * example torch tensors' data_ptr()), "host" pointers ordinary host memory.
 *
 * Errors: every int-returning call returns HOMO_OK (0) or one of the HOMO_E* codes
 * below; no exception crosses the ABI. homo_last_error(ctx) returns a message for the
 * last failing call on that context (homo_last_error(NULL): last homo_create failure
 * on this thread). After HOMO_ECUDA the context should be destroyed.
 *
 * Threading: a context is not thread-safe; distinct contexts may be used from
 * distinct threads.
 */
#ifndef HOMO_H
#define HOMO_H

#ifdef __cplusplus
extern "C" {
#endif

#define HOMO_OK 0
#define HOMO_EINVAL 1      /* bad argument: size, pointer, parameter range            */
#define HOMO_ENOMEM 2      /* device or pinned-host allocation failed                  */
#define HOMO_ECUDA 3       /* a CUDA runtime call or kernel launch failed              */
#define HOMO_ENOCONV 4     /* max iterations reached; outputs valid, residuals given   */
#define HOMO_EDIVERGED 5   /* a residual norm became non-finite or blew up             */
#define HOMO_ESTATE 6      /* call out of order (e.g. homo_CH before a solve)          */

#define HOMO_NUM_CASES 6

/* Objective kinds for homo_objective (Sec. 5.2-5.3). */
#define HOMO_OBJ_BULK 0        /* Eq. 19: -(C00+C11+C22+2(C01+C02+C12))/9              */
#define HOMO_OBJ_SHEAR 1       /* Eq. 20: -(C33+C44+C55)/3                              */
#define HOMO_OBJ_POISSON 2     /* Eq. 21: C01+C02+C12 - beta^iter (C00+C11+C22)         */
#define HOMO_OBJ_LOGPOISSON 3  /* Eq. 22: log(1+eta(C01+C12+C20)/(C00+C11+C22))
                                            + tau (C00+C11+C22)^gamma, eta 0.6, gamma 0.5,
                                            tau = -1/E0^gamma                             */

typedef struct homo_ctx homo_ctx;

/* Optional solver settings. Zero-initialise and set struct_size = sizeof(homo_opts);
 * zero fields take the defaults. */
typedef struct homo_opts {
  int struct_size;
  int min_coarse;   /* coarsen by 2 while the next level keeps >= min_coarse cells per
                       axis (default 4, Sec. 3.3); the coarsest level is solved directly */
  int max_levels;   /* cap on the number of levels, 0 = no cap                           */
  int pre_sweeps;   /* smoothing sweeps before coarse correction (default 1)             */
  int post_sweeps;  /* smoothing sweeps after it (default 1; must equal pre_sweeps)      */
  int smoother;     /* HOMO_SMOOTH_GS8 (default) or HOMO_SMOOTH_CHEBYSHEV                */
  int cheb_degree;  /* Chebyshev polynomial degree per sweep, 2..4 (default 2)           */
  int precision;    /* HOMO_PRECISION_FP32 (default) or HOMO_PRECISION_MIXED             */
  int graphs;       /* 1: replay each CG iteration as a captured CUDA graph (needs a
                       non-NULL stream; not while profiling), 0 (default): plain launches */
  int coarse_sweeps; /* smoothing sweeps before and after the coarse correction on level 1,
                       the first level below the finest (0 = default 1)                   */
  int sweep_growth;  /* each further level smooths this many times as often as the level
                       above it, at most HOMO_MAX_LEVEL_SWEEPS (0 = default 3: 1, 3, 9,
                       27, 64, ... sweeps on levels 1, 2, 3, ...). The paper does not state
                       its sweep counts; a sweep costs 1/8 per level of one on the level
                       above, and the deeper smoothing cuts the CG iterations, whose cost
                       the finest level dominates (the finest level keeps pre_sweeps /
                       post_sweeps). */
} homo_opts;

#define HOMO_MAX_LEVEL_SWEEPS 64

/* Smoothers. GS8: 8-colour block Gauss-Seidel (Sec. 4.1-4.2, Eq. 15-16), colours 0..7
 * before and 7..0 after the coarse correction. CHEBYSHEV: Chebyshev polynomial in
 * D^-1 K (D the 3x3 block diagonal, the GS8 diagonal solve S_v of Eq. 16) on the
 * interval [lmax/10, lmax], lmax the element bound max eig(D_e^-1 K0) on the finest
 * level and a 12-step power-iteration estimate x1.15 on coarse levels; every step is
 * one data-parallel pass (not in the paper, which uses GS8). */
#define HOMO_SMOOTH_GS8 0
#define HOMO_SMOOTH_CHEBYSHEV 1

/* Storage precision of the preconditioner's coarse-level stencils (the paper's mixed
 * scheme keeps its numerical stencils in half precision and every vector in single
 * precision, Sec. 4.1 "Mixed floating-point precision representations", Sec. 6.3).
 * FP32: every stored stencil in FP32. MIXED: the stencils of the smoothed coarse levels
 * are also kept as BF16 (FP32 exponent range: an FP16 copy would flush the void-region
 * entries, ~E_min, to zero) and the coarse smoothers and residuals read that copy; each
 * block is stored as the BF16 rounding of (A_d(v) + A_-d(v+d)^T) / 2, so the rounded
 * coarse operators stay exactly symmetric. Arithmetic stays FP32, the Galerkin products
 * are formed from the FP32 stencils, and the CG iteration (u, r, p, q, the true residual)
 * is untouched: the solution meets the same tolerance; only the preconditioner changes. */
#define HOMO_PRECISION_FP32 0
#define HOMO_PRECISION_MIXED 1

/* Library version as 10000*major + 100*minor + patch. */
int homo_version(void);

/* Static text for a status code. */
const char* homo_status_string(int status);

/* Create a context for an n^3 periodic cell (Sec. 3.1-3.2).
 *   n     : cells per axis, 4 <= n <= 1024; every level that is smoothed must be even.
 *   E0    : Young's modulus of the solid (> 0); nu: Poisson's ratio in (-1, 0.5).
 *   p     : SIMP exponent (>= 1); Emin: floor modulus, 0 <= Emin < E0.
 *           Element modulus E_e = Emin + rho~_e^p (E0 - Emin).
 *   opts  : nullable.
 * Allocates every device buffer up front (about 450 bytes per element for n = 512).
 * Uses the current CUDA device. Returns HOMO_EINVAL / HOMO_ENOMEM / HOMO_ECUDA. */
int homo_create(homo_ctx** out, int n, double E0, double nu, double p, double Emin,
                const homo_opts* opts);

/* Free every resource of the context (synchronises its stream). NULL is accepted. */
int homo_destroy(homo_ctx* ctx);

/* Last error message of the context, or of the last failed homo_create on this
 * thread when ctx is NULL. Never NULL. */
const char* homo_last_error(const homo_ctx* ctx);

/* Run all further work of the context on this cudaStream_t (NULL = legacy default
 * stream). */
int homo_set_stream(homo_ctx* ctx, void* cuda_stream);

/* Number of multigrid levels and cells per axis of level l (0 = finest). */
int homo_num_levels(const homo_ctx* ctx);
int homo_level_size(const homo_ctx* ctx, int level);

/* Periodic linear-cone filter (Sec. 5.2 "conv", Sec. 6 radius 2, Sec. 6.4 periodic
 * kernel): out_e = sum_d w(d) in_(e+d) / sum_d w(d), w(d) = max(0, radius - |d|), d
 * integer offsets between element centres, wrapped periodically. The operator is
 * symmetric, so the same call applies its adjoint to sensitivities.
 *   in, out: device, N floats each; must not alias. 0 < radius <= 3.5. */
int homo_filter(homo_ctx* ctx, double radius, const float* in, float* out);

/* Sensitivity filter of the unfiltered variant (Sec. 5.3: the density is penalised
 * directly, E = Emin + rho^p (E0 - Emin), and the sensitivity is filtered before the OC
 * update). The paper names the step without its formula; this is the classic
 * density-weighted mesh-independence filter with the same periodic cone weights:
 *   out_e = sum_d w(d) rho_(e+d) dc_(e+d) / (max(gamma, rho_e) sum_d w(d)).
 *   rho, dc, out: device, N floats each; out must alias neither rho nor dc.
 *   0 < radius <= 3.5; 0 < gamma <= 1 (1e-3 is the usual choice). */
int homo_filter_sensitivity(homo_ctx* ctx, double radius, const float* rho, const float* dc,
                            double gamma, float* out);

/* Trigonometric density initialisation (Sec. 6.2). At the element centres x (unit cell),
 * with xb = R_q (x - (1/2, 1/2, 1/2)) and R_q the rotation of the quaternion q (scalar
 * first, normalised here), the basis T = {cos, sin}(2 pi k xb_i), k = 1..nb, i = 0..2, in
 * the order index 2 (3 (k-1) + i) + {0 cos, 1 sin}, is extended by the products T_a T_b,
 * a <= b (row by row after T); y = sum of weights[j] times member j. Then
 *   rho_e = clamp(rho_min + Vh / (1 + exp(-15 (y_e - mu))), rho_min, 1), Vh = min(1.5 V, 1),
 * with mu found so that the mean density is V (bisection, 32 shifts per pass).
 *   nb: 1..3; weights: host, nweights = 6 nb + 6 nb (6 nb + 1) / 2 (drawn in [-1, 1] by
 *   the caller); q: host, 4 doubles, not all zero; 0 <= rho_min < volfrac < 1;
 *   rho_out: device, N floats. Arithmetic in FP64 (a one-time setup step). Uses the
 *   context's CG scratch; synchronises the stream. */
int homo_trig_init(homo_ctx* ctx, int nb, const double q[4], const double* weights, int nweights,
                   double volfrac, double rho_min, float* rho_out);

/* Symmetry enforcement (Sec. 6.1): every element value becomes the average over its
 * orbit under the chosen group of the cube, as the paper's loop does to the sensitivity
 * before the OC update and to the density after it.
 *   kind: HOMO_SYM_REFLECT3 - reflections in the mid-planes x, y, z = 1/2 (8 maps);
 *         HOMO_SYM_ROTATE3  - rotations generated by quarter turns about the axes through
 *                             the centre (24 maps);
 *         HOMO_SYM_REFLECT6 - mid-plane reflections and reflections in the diagonal
 *                             planes x = y, y = z, z = x (all 48 signed permutations).
 *   in, out: device, N floats each; out may equal in (in-place).
 * Orbit members receive bitwise-equal values when the orbit's values lie within a factor
 * 2^29 of each other (FP64 sums of at most 48 FP32 values are then exact). */
#define HOMO_SYM_REFLECT3 1
#define HOMO_SYM_ROTATE3 2
#define HOMO_SYM_REFLECT6 3
int homo_symmetrize(homo_ctx* ctx, int kind, const float* in, float* out);

/* Set the physical (filtered) density rho~ and derive E_e (Sec. 3.2). Values are
 * clamped to [0, 1]. rho: N floats, device (on_device = 1) or host (on_device = 0).
 * Marks loads and the multigrid hierarchy stale; the 6 displacement fields are kept
 * as warm starts (Sec. 4.1 "Different GPU memory types"). */
int homo_set_density(homo_ctx* ctx, const float* rho, int on_device);

/* Solve K(E) u_i = f_i for the 6 unit macro strains (Eq. 4-5, Eq. 11-12) with CG
 * preconditioned by one multigrid V-cycle (Alg. 1): 8-colour block Gauss-Seidel
 * (Eq. 13-16), trilinear transfers, Galerkin coarse levels (Eq. 17-18), a direct
 * coarsest solve with the rigid-translation null space projected out (Sec. 4.2).
 *   rel_tol   : stop case i when ||f_i - K u_i||_2 / ||f_i||_2 <= rel_tol (> 0).
 *   max_iters : CG iteration cap (>= 1).
 *   warm_start: 1 = start from the fields of the previous solve, 0 = from zero.
 *   iters_out, relres_out: host arrays of 6 (nullable): CG iterations per case and
 *               final true relative residual per case.
 * The true residual is the rigid-translation-free part of f - K u (translations lie
 * outside the range of K). The result is certified in double-float arithmetic; for
 * rel_tol >= 1e-5 the starting residual is the FP32 one (see homo_residual).
 * Returns HOMO_ENOCONV if a case missed rel_tol within max_iters (fields valid),
 * HOMO_EDIVERGED on a non-finite residual. Synchronises the stream. */
int homo_solve_cases(homo_ctx* ctx, double rel_tol, int max_iters, int warm_start,
                     int iters_out[6], double relres_out[6]);

/* Solve the cell problems of several contexts (cells of any sizes) together: the contexts
 * advance their CG iterations in lockstep, each on its own stream, with one host
 * synchronisation per step for all of them, so small cells overlap on the GPU. Each
 * context's result is the one homo_solve_cases would give it (same kernels, same order).
 * With homo_opts.graphs = 1 and a non-NULL stream per context, every CG iteration is one
 * CUDA graph launch instead of about a hundred kernel launches. (The paper solves one
 * cell at a time; this entry point has no counterpart there.)
 *   ctxs: host array of count distinct contexts; rel_tol, max_iters, warm_start as in
 *   homo_solve_cases. iters_out, relres_out: host arrays of 6 * count (nullable), case
 *   results of context i at [6 i, 6 i + 6). status_out: host array of count (nullable),
 *   the status homo_solve_cases would return for context i.
 * Returns HOMO_EINVAL for bad arguments, otherwise the most severe per-context status
 * (HOMO_OK < HOMO_ENOCONV < others). */
int homo_solve_batch(homo_ctx* const* ctxs, int count, double rel_tol, int max_iters, int warm_start,
                     int* iters_out, double* relres_out, int* status_out);

/* Relative true residual ||f_i - K u_i||_2 / ||f_i||_2 (rigid translations removed) of
 * the context's current displacement fields, per case (0 where f_i = 0), by one of two
 * evaluations (the paper measures convergence with this quantity, Sec. 4.1 "Mixed
 * floating-point precision"; the two evaluations are this library's):
 *   method HOMO_RESIDUAL_FP32        : FP32 difference form, each neighbour difference
 *                                      formed from both parts of the double-float field;
 *   method HOMO_RESIDUAL_DOUBLE_FLOAT: double-float arithmetic throughout.
 *   relres_out: host, 6 doubles (output).
 * Needs loads (a homo_set_density); overwrites the context's residual scratch.
 * Returns HOMO_ESTATE before homo_set_density, HOMO_EINVAL on a bad method or NULL
 * output. Synchronises the stream. */
#define HOMO_RESIDUAL_FP32 0
#define HOMO_RESIDUAL_DOUBLE_FLOAT 1
int homo_residual(homo_ctx* ctx, int method, double relres_out[6]);

/* Residual fields, for parity tests of the finest-level residual kernels (the residual
 * of Eq. 5 evaluated in the vertex form of Eq. 13). out: device, 18 planes of n^3 floats
 * (plane = 3 case + component, x fastest), written by the call; nothing is removed from
 * it (rigid translations included).
 *   method HOMO_RESIDUAL_FP32 or HOMO_RESIDUAL_DOUBLE_FLOAT: the context's true residual
 *     f - K (u_hi + u_lo) of its own loads and displacement (the evaluations of
 *     homo_residual); b and u must be NULL.
 *   method HOMO_RESIDUAL_VCYCLE: b - K u for caller fields b and u (device, 18 n^3 floats
 *     each, neither aliasing out), the evaluation the V-cycle uses on the finest level.
 * Returns HOMO_ESTATE before homo_set_density, HOMO_EINVAL on a bad method or pointer
 * combination. Synchronises the stream. */
#define HOMO_RESIDUAL_VCYCLE 2
int homo_residual_field(homo_ctx* ctx, int method, const float* b, const float* u, float* out);

/* C^H without any device allocation (the paper has no counterpart to this entry point).
 * For callers that cannot call cudaMalloc while they run: an application that sets its
 * device-memory budget once at start-up, a framework whose own pooled allocator must
 * own every device byte, or a process whose device memory is already fully reserved.
 * Such callers hold the fields themselves and need no context (homo_create allocates).
 * Computes the same C^H as homo_CH (Eq. 7) from caller-owned buffers:
 *   n     : cells per axis, 4 <= n <= 1024 (larger n returns HOMO_EINVAL with a message
 *           in homo_last_error(NULL));
 *   nu    : Poisson's ratio of the unit-modulus element matrix;
 *   E     : device, N floats, element moduli E_e (as homo_set_density derives them);
 *   u, ulo: device, 18*N floats each (6-case layout above): displacement, optionally
 *           split into high and low parts; ulo may be NULL (treated as zero);
 *   CH    : host, 36 doubles, row-major 6x6 (output);
 *   cuda_stream: the stream to run on (NULL = legacy default stream).
 * Scratch: instead of allocating, the call uses one fixed array of about 200 KB that
 * every GPU which loads the library holds until the process exits. Its size does not
 * grow with n. The first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before any stream
 * capture. All calls share the array and it keeps the last call's contents (each call
 * overwrites every entry it later reads, so nothing needs clearing); calls that overlap
 * on the GPU, on any stream, race and must be serialised by the caller. Synchronises
 * the stream. Calls no cudaMalloc, cudaFree or allocating library routine. */
int homo_CH_noalloc(int n, double nu, const float* E, const float* u, const float* ulo,
                    double CH[36], void* cuda_stream);

/* Homogenised tensor C^H_ij = (1/|Omega|) sum_e E_e (chi_i - u_i)_e^T K0 (chi_j - u_j)_e
 * (Eq. 7) from the last solve. CH: host, 36 doubles, row-major 6x6, Voigt order
 * 11,22,33,12,23,13, engineering shear. Synchronises the stream. */
int homo_CH(homo_ctx* ctx, double CH[36]);

/* Element sensitivities of an objective with gradient dfdCH (host, 36 doubles, each
 * entry treated as an independent variable) with respect to the filtered density
 * (Eq. 8-9; the sum over e printed in Eq. 9 read as a per-element value):
 *   dfdrho_e = p rho~_e^(p-1) (E0 - Emin) sum_ij dfdCH_ij q_e,ij / |Omega|,
 *   q_e,ij = (chi_i - u_i)_e^T K0 (chi_j - u_j)_e.
 * dfdrho: device, N floats. */
int homo_sensitivity(homo_ctx* ctx, const double dfdCH[36], float* dfdrho);

/* Optimality-criteria update (Sec. 3.3; step limit, damping and minimum density of
 * Sec. 6): rho_new = clamp(rho (max(-dfdrho,0)/lambda)^damp, max(rho_min, rho-move),
 * min(1, rho+move)) with the multiplier lambda found on the device so that
 * mean(rho_new) equals volfrac (the side with mean <= volfrac is returned).
 *   dfdrho: device N floats (sensitivity w.r.t. rho); rho: device N floats, in/out.
 *   change_out: host, nullable: max |rho_new - rho|. */
int homo_update(homo_ctx* ctx, const float* dfdrho, float* rho, double volfrac,
                double move, double damp, double rho_min, double* change_out);

/* Objective value and gradient (host arithmetic only, Eq. 19-22).
 *   kind: HOMO_OBJ_*; iteration: loop counter l (HOMO_OBJ_POISSON uses beta^l);
 *   param: beta for HOMO_OBJ_POISSON, E0 for HOMO_OBJ_LOGPOISSON, ignored otherwise.
 *   CH: 36 doubles in; f_out: 1 double out; dfdCH: 36 doubles out. */
int homo_objective(int kind, const double CH[36], int iteration, double param,
                   double* f_out, double dfdCH[36]);

/* The 24x24 element matrix K0 the library uses (unit modulus, unit voxel, host
 * arithmetic only): the bilinear form of isotropic elasticity (Sec. 3.2) integrated in
 * closed form over a trilinear brick. Row/column 3j + comp, local vertex j = a+2b+4c.
 * Ke: host, 576 doubles, row-major. No GPU needed. */
int homo_element_matrix(double nu, double Ke[576]);

/* Largest eigenvalue of D_e^-1 K0 (D_e: the 3x3 block diagonal of K0), which bounds the
 * spectrum of D^-1 K on the finest level for any moduli; the Chebyshev smoother's upper
 * interval end there. Host arithmetic only; out: 1 double. */
int homo_element_jacobi_bound(double nu, double* out);

/* ---- Introspection and operator access (device pointers, 6-case layout above) ---- */

/* Copy the current 6 displacement fields out / in (18*N floats, device). */
int homo_get_displacement(homo_ctx* ctx, float* u);
int homo_set_displacement(homo_ctx* ctx, const float* u);

/* Exact copy of the displacement state that warm-starts the next solve: both FP32 parts
 * of the double-float fields u = hi + lo (18*N floats each, device, caller-owned).
 * Restoring a saved state makes the next warm-started solve repeat the one that followed
 * the save, iteration for iteration. Neither pointer may be NULL; enqueued on the
 * context's stream (no synchronisation). The paper has no counterpart (it keeps the
 * previous iterate in place, Sec. 4.1). */
int homo_save_displacement(homo_ctx* ctx, float* hi, float* lo);
int homo_restore_displacement(homo_ctx* ctx, const float* hi, const float* lo);

/* Assembled macro-strain loads f_i = sum_e E_e K0 chi_i,e for the current density
 * (Eq. 4 in the vertex form Eq. 11, element-relative chi of Eq. 12). f: 18*N floats. */
int homo_get_loads(homo_ctx* ctx, float* f);

/* out = K(E) u on the finest level, matrix-free (Eq. 13), for the 6 cases.
 * u, out: device, 18*N floats, must not alias. */
int homo_apply_K(homo_ctx* ctx, const float* u, float* out);

/* Galerkin stencil of level l >= 1 (Eq. 17-18): out[(v*27 + d)*9 + 3r + c], vertex v of
 * level l in x-fastest order, neighbour offset d = (dx+1) + 3(dy+1) + 9(dz+1), 3x3 block
 * row r, column c. out: device, 243 * n_l^3 floats. Builds the hierarchy if stale. */
int homo_get_stencil(homo_ctx* ctx, int level, float* out);

/* Restriction R = I^T from level l to l+1 and prolongation I from l+1 to l (trilinear,
 * periodic, Sec. 3.3). 6-case layouts on the respective level sizes. restrict: coarse =
 * R fine; prolong: fine = I coarse (overwrites). */
int homo_restrict(homo_ctx* ctx, int level, const float* fine, float* coarse);
int homo_prolong(homo_ctx* ctx, int level, const float* coarse, float* fine);
/* fine += I coarse (the same prolongation, accumulated). */
int homo_prolong_add(homo_ctx* ctx, int level, const float* coarse, float* fine);

/* ---- Tuning ----
 * The finest-level Gauss-Seidel pass (Eq. 15-16) is compiled in four variants: 3 or 6
 * load cases per thread (3: the cases are split over two thread groups, each rebuilding
 * the coupling blocks; 6: blocks built once, more registers) times 128 or 256 threads
 * per block. All four compute bitwise the same result; which is fastest depends on the
 * grid size. homo_set_tuning selects one (default 3, 256). homo_autotune times one
 * symmetric sweep pair of each on the context's own moduli and loads (needs a density;
 * uses the solver's scratch, so call it between solves), selects the fastest and caches
 * the choice per grid size for the process; flags HOMO_TUNE_RETIME ignores the cache.
 * Outputs (host, nullable): the chosen variant; ms: 4 times per sweep of the variants
 * (3,256), (3,128), (6,256), (6,128), -1 when the choice came from the cache. */
#define HOMO_TUNE_RETIME 1
int homo_set_tuning(homo_ctx* ctx, int gs_cases, int gs_block);
int homo_autotune(homo_ctx* ctx, int flags, int* gs_cases, int* gs_block, double* ms);

/* Coarse-level Gauss-Seidel kernels (Eq. 15-16 on levels >= 1). All four forms compute
 * bitwise the same iterates; they differ in how the work reaches the GPU:
 *  - levels with at most resident_max_n cells per axis (FP32 stencils, and only where the
 *    shared memory suffices: up to 16^3 with 16-CTA clusters): every sweep of one
 *    smoothing phase (the pre- or post-smoothing sweeps of a V-cycle, or the single sweep
 *    of homo_smooth) is one launch of six thread-block clusters, one per load case. Each
 *    CTA holds a copy of its case's displacement in shared memory, writes the updates of
 *    its own vertices into every copy of the cluster, and streams the stencil rows of its
 *    vertices for the next colour while the current one computes; the colour passes are
 *    separated by the cluster's hardware barrier (default 16);
 *  - other levels with at most cluster_max_n cells per axis: the same per-case cluster
 *    launch, reading the displacement and stencils through L2 (default 32);
 *  - larger levels with at most split_max_n cells per axis: one launch per colour pass with
 *    a thread per (vertex, load case), each loading a z-layer of 9 neighbours before its
 *    FMAs (default 32);
 *  - larger levels: one launch per colour pass with a thread per vertex and all 6 cases.
 * The small levels are bound by load latency and launch overhead, not by bytes: with the
 * default sweep counts a V-cycle of a 512^3 cell runs about 2,500 colour passes on levels
 * of 32^3 and below. Sizes in [0, 1024]; 0 disables a form. Changing them drops the
 * context's captured CUDA graphs. Where the device cannot launch the clusters, the next
 * form applies whatever the sizes say. homo_coarse_smoother reports the sizes and the
 * largest cluster of the L2 and of the resident form the device launches (-1: none);
 * outputs nullable. Both return HOMO_EINVAL for a NULL context or sizes out of range.
 * (The paper launches one kernel per colour pass; this setting has no counterpart there.) */
int homo_set_coarse_smoother(homo_ctx* ctx, int resident_max_n, int cluster_max_n, int split_max_n);
int homo_coarse_smoother(const homo_ctx* ctx, int* resident_max_n, int* cluster_max_n, int* split_max_n,
                         int* cluster, int* resident_cluster);

/* Autotuner of the coarse Gauss-Seidel forms. Times, on every smoothed coarse level of the
 * context's own hierarchy, the two smoothing phases of a V-cycle (the level's sweep count
 * from zero in colour order 0..7, then in order 7..0) in each form the level can take (the
 * thread-per-vertex form everywhere, the thread-per-(vertex, case) form up to 128^3, the
 * cluster forms up to 64^3 and where the device launches them), then sets the three sizes
 * of homo_set_coarse_smoother (each 0 or a level size) whose forms give the smallest sum
 * of those times, and caches them per (grid size, precision, sweep schedule) for the
 * process; flags HOMO_TUNE_RETIME ignores the cache. Needs a density; uses the coarse
 * levels' vectors, so call it between solves. The forms give bitwise the same iterates,
 * so the choice changes only the time. Outputs (host, nullable): the chosen sizes; ms:
 * 64 doubles, ms[4 l + k] the time of level l's two phases in form k (0 thread per
 * vertex, 1 thread per (vertex, case), 2 cluster through L2, 3 resident cluster), -1 where
 * not timed (all -1 when the choice came from the cache). (The paper has no counterpart.) */
int homo_autotune_coarse(homo_ctx* ctx, int flags, int* resident_max_n, int* cluster_max_n, int* split_max_n,
                         double* ms);

/* One 8-colour block Gauss-Seidel sweep (Eq. 15-16) on level l, in place on u, colours
 * 0..7 (reverse = 0) or 7..0 (reverse = 1). f, u: device, 6-case layout on level l. */
int homo_smooth(homo_ctx* ctx, int level, int reverse, const float* f, float* u);

/* z = M r with M one symmetric V-cycle from a zero initial guess (Alg. 1), the CG
 * preconditioner. r, z: device, 18*N floats, must not alias. */
int homo_vcycle(homo_ctx* ctx, const float* r, float* z);

/* ---- Measurement ---- */

/* Kernel classes for per-class device timing. */
#define HOMO_KC_FINE_MATVEC 0      /* CG product q = K p on the finest level (Eq. 13)      */
#define HOMO_KC_FINE_RESIDUAL 1    /* finest-level V-cycle residuals b - K u               */
#define HOMO_KC_FINE_GS 2          /* finest-level Gauss-Seidel colour passes (Eq. 15-16)  */
#define HOMO_KC_COARSE_GS 3        /* coarse-level Gauss-Seidel colour passes              */
#define HOMO_KC_COARSE_RESIDUAL 4  /* coarse-level residuals                               */
#define HOMO_KC_TRANSFER 5         /* restriction and prolongation                          */
#define HOMO_KC_COARSEST 6         /* coarsest direct solve                                 */
#define HOMO_KC_SETUP 7            /* loads, Galerkin assembly, coarsest factorisation      */
#define HOMO_KC_CG_VECTOR 8        /* CG vector updates, dot products, scalars              */
#define HOMO_KC_ELEMENT 9          /* C^H and sensitivity element kernels                   */
#define HOMO_KC_FILTER 10          /* density filter                                        */
#define HOMO_KC_OC 11              /* OC update                                             */
#define HOMO_KC_OTHER 12           /* SIMP moduli, field copies, stencil export             */
#define HOMO_KC_FINE_CHEB 13       /* finest-level Chebyshev smoothing steps                */
#define HOMO_KC_COARSE_CHEB 14     /* coarse-level Chebyshev smoothing steps                */
#define HOMO_KC_TRUE_RESIDUAL 15   /* true residuals f - K u (FP32 and double-float forms) */
#define HOMO_KC_COUNT 16

/* Start (enable = 1, counters reset) or stop (0) recording a CUDA event pair around
 * every kernel launch of the context, on its stream. */
int homo_profile_enable(homo_ctx* ctx, int enable);

/* Synchronise the stream and return, for kernel class kc, the number of kernels
 * launched and their summed device time in ms since profiling was enabled. */
int homo_profile_read(homo_ctx* ctx, int kc, long long* launches, double* total_ms);

/* Static name of a kernel class ("fine_matvec", ...), or "" for an unknown class. */
const char* homo_kernel_class_name(int kc);

/* Measured FP32 arithmetic peak of the current device, the denominator of the roofline of
 * the ALU-bound stencil kernels (the paper reports no such figure). A kernel of independent
 * FMA chains fills every SM (8 chains per thread, 1024 threads per SM); its CUDA-event
 * time gives TFLOP/s = 2 flops per FMA lane. packed = 0: scalar fma.rn.f32; packed = 1:
 * the two-lane fma.rn.f32x2 of sm_100 and later (4 flops per instruction).
 *   tflops_out: host, 1 double (output).
 * Allocates and frees a small device buffer; synchronises the device's legacy stream. */
int homo_probe_fp32_peak(int packed, double* tflops_out);

/* Total number of kernels this context has launched since it was created. */
long long homo_launch_count(const homo_ctx* ctx);

/* Residual history of the last homo_solve_cases: one row of 6 relative residuals
 * ||r_i||/||f_i|| per record (the initial true residual, every CG iteration, and the
 * true residual that closes every restart cycle). Copies min(rows, capacity) rows to out
 * (host, 6*capacity doubles) and returns the number of rows (negative on error). */
int homo_residual_history(const homo_ctx* ctx, double* out, int capacity);

/* ---- Learned warm start --------------------------------------------------------------
 * Not part of the paper's method, which starts each solve from the previous iterate
 * (Sec. 3.3). A fully convolutional network maps the filtered density of a cell to the
 * 18 displacement planes of its 6 load cases; a solve started from its prediction must
 * still meet the same tolerance, so the zero and previous-iterate starts remain the
 * reference it is measured against.
 *
 * Layouts (device memory; BF16 tensors are uint16 storage, 16-byte aligned):
 *   activation  x[v*C + c], voxel v = x + n*(y + n*z), C channels (C = 16 for the
 *               features, HOMO_NN_CHANNELS = 32 for every layer output).
 *   weights     W[t][o][i] of one layer, t = 9(dz+1) + 3(dy+1) + (dx+1) the tap of offset
 *               d = (dx,dy,dz) in {-1,0,1}^3, o output channel (32), i input channel.
 * A layer is the periodic cross-correlation
 *     y[v,o] = bias[o] + sum_t sum_i W[t,o,i] x[wrap(v + d_t), i]
 * with BF16 products and FP32 accumulation on the tensor cores.
 * Network with B residual blocks:
 *     h0 = relu(conv_in(features)),  t_b = relu(conv1_b(h_{b-1})),
 *     h_b = relu(conv2_b(t_b) + h_{b-1}),  y = conv_out(h_B),
 * prediction u[p*N + v] = scale[p/3] * y[v,p] for the 18 planes p (scale[c] = n s_c, s_c a
 * displacement scale of load case c chosen by the caller, e.g. the RMS of its training
 * displacements per unit cell size: it balances the 6 cases in the loss).
 * Features: (rho, rho^2, rho^3, 0, ..., 0).
 * Parameters (FP32, host order): per layer l = conv_in, conv1_1, conv2_1, ..., conv_out:
 * W_l (27 * 32 * c_in_l floats, c_in = 16 for conv_in, 32 otherwise) then bias_l (32). */
#define HOMO_NN_CHANNELS 32
#define HOMO_NN_FEATURES 16
#define HOMO_NN_RELU 0     /* out = bf16(relu(acc + bias + res))                         */
#define HOMO_NN_MASK 1     /* out = bf16((acc + res) * [mask > 0]); bias ignored         */
#define HOMO_NN_PLANES 2   /* out_planes[p*N + v] = scale[p/3] * (acc + bias), p < 18     */
#define HOMO_NN_PLANES_ADD 3  /* out_planes[p*N + v] += scale[p/3] * (acc + bias), p < 18 */
#define HOMO_NN_MSE_SCRATCH 1025   /* doubles of homo_nn_mse's loss buffer           */

/* One layer. x: n^3 x c_in BF16 (c_in 16 or 32; 32 for MASK / PLANES); w: packed BF16
 * weights [27][32][c_in]; bias: 32 floats or NULL; res, mask: n^3 x 32 BF16 or NULL
 * (mask required by MASK); out: n^3 x 32 BF16 (RELU, MASK) or out_planes: 18 n^3 floats
 * (PLANES, PLANES_ADD; then out, res and mask must be NULL); scale: host, 6 per-case
 * factors of the planes epilogues (NULL = 1). Outputs must not alias inputs.
 * Asynchronous on stream. HOMO_EINVAL on a bad size, combination or alignment. */
int homo_nn_conv3d(int n, int c_in, const void* x, const void* w, const float* bias, const void* res,
                   const void* mask, int epilogue, void* out, float* out_planes, const double* scale,
                   void* stream);

/* The layer runs on the tcgen05 tensor cores: one thread per CTA issues the MMAs and the
 * CTA waits for their completion on an mbarrier with a bounded number of polls. Returns
 * the number of tile waits that ran out since the last call (0 in normal operation; the
 * outputs of such a tile are not written) and resets it; -1 if it cannot be read.
 * Synchronous (reads a device counter). */
int homo_nn_tc_timeouts(void);

/* Exercises that bounded wait on its own: launches `blocks` CTAs (1..1024) that wait on an
 * mbarrier nothing arrives on, each giving up after the same poll limit and counting one
 * timeout (read with homo_nn_tc_timeouts). No tensor-core work is issued. For failure-
 * detection tests; takes about a second (each CTA polls 2^18 times). Synchronises the
 * device. */
int homo_nn_tc_wait_probe(int blocks);

/* Weight and bias gradients of one layer: dw[t][o][i] = sum_v dy[v,o] x[wrap(v + d_t), i],
 * db[o] = sum_v dy[v,o] (FP32, summed in a fixed order: deterministic). x: n^3 x c_in
 * BF16, dy: n^3 x 32 BF16; scratch: device floats, at least homo_nn_wgrad_scratch(n, c_in). */
size_t homo_nn_wgrad_scratch(int n, int c_in);
int homo_nn_wgrad(int n, int c_in, const void* x, const void* dy, float* dw, float* db, float* scratch,
                  size_t scratch_floats, void* stream);

/* Average pooling of a density: out[c] = mean of rho over the factor^3 voxels of coarse
 * voxel c; rho: n^3 floats, out: (n/factor)^3 floats (device); n divisible by factor. The
 * network is trained and evaluated on cells whose features span the same number of
 * voxels; pooling brings a larger cell to that scale. */
int homo_nn_pool(int n, int factor, const float* rho, float* out, void* stream);

/* Network input features of a filtered density rho (n^3 floats) into x (n^3 x 16 BF16). */
int homo_nn_features(int n, const float* rho, void* x, void* stream);

/* Loss sum_{v, p<18} (y[p][v] - u[p][v]/scale[p/3])^2 / (18 n^3) of the network output
 * planes y against solver displacements u (both 18 n^3 floats) into loss[0] (device; loss
 * holds HOMO_NN_MSE_SCRATCH doubles, the rest is scratch) and its gradient
 * dy[v][p] = bf16(2 (y - u/scale[p/3]) / (18 n^3)) (n^3 x 32 BF16, zero for p >= 18).
 * scale: host, 6 positive per-case factors. */
int homo_nn_mse(int n, const float* y, const float* u, const double* scale, void* dy, double* loss,
                void* stream);

/* Adam (Kingma and Ba 2015) on count FP32 parameters: m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, w -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps); step >= 1. */
int homo_nn_adam(size_t count, float* w, const float* g, float* m, float* v, int step, double lr, double beta1,
                 double beta2, double eps, void* stream);

/* BF16 copies of one layer's FP32 weights w[27][32][c_in]: w_fwd (same layout) and, when
 * c_in = 32 and w_bwd != NULL, w_bwd[t][i][o] = w[26 - t][o][i], the weights with which
 * homo_nn_conv3d propagates a gradient back through the layer. */
int homo_nn_pack(int c_in, const float* w, void* w_fwd, void* w_bwd, void* stream);

/* The network as one object: FP32 master parameters, Adam moments, packed BF16 weights
 * and activation buffers sized on first use for each grid size. Its calls return
 * HOMO_OK, HOMO_EINVAL, HOMO_ENOMEM or HOMO_ECUDA, with a message in
 * homo_net_last_error; they run on the stream of homo_net_set_stream (default: the
 * legacy default stream). A network is not thread-safe. */
typedef struct homo_net homo_net;

/* Number of FP32 parameters of a network with `blocks` residual blocks (1..16). */
size_t homo_net_param_count(int blocks);
/* params: host, homo_net_param_count(blocks) floats in the order above. */
int homo_net_create(homo_net** out, int blocks, const float* params);
int homo_net_destroy(homo_net* net);
const char* homo_net_last_error(const homo_net* net);
int homo_net_set_stream(homo_net* net, void* cuda_stream);
/* Copies (host, synchronous) of the parameters and of the gradients of the last train step. */
int homo_net_get_params(homo_net* net, float* params);
int homo_net_get_grads(homo_net* net, float* grads);
/* Predicted displacements for the filtered density rho (device, n^3 floats): u (device,
 * 18 n^3 floats) = scale[p/3] * y, or u += scale[p/3] * y when accumulate != 0 (scale: host,
 * 6 factors, any sign). Holds 224 n^3 bytes of activations until released. */
int homo_net_predict(homo_net* net, int n, const float* rho, const double* scale, float* u, int accumulate);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the loss of homo_nn_mse for the pair
 * (rho, u) (device); loss: host, nullable (non-NULL synchronises the stream). Holds
 * (424 + 128 blocks) n^3 bytes of activations plus the weight-gradient scratch until
 * released. */
int homo_net_train_step(homo_net* net, int n, const float* rho, const float* u, const double* scale, double lr,
                        double* loss);
/* Free the activation buffers. */
int homo_net_release(homo_net* net);
/* Kernels this network launched so far. */
long long homo_net_launch_count(const homo_net* net);

#ifdef __cplusplus
}
#endif

#endif /* HOMO_H */
