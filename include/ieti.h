/*
 * ieti.h -- C ABI of the GB300 library for the dual-primal isogeometric tearing
 * and interconnecting (IETI-DP / FETI-DP) method for 3D curl-curl magnetostatics
 * on multipatch spline discretisations (arXiv 2501.04340).
 *
 * Conventions shared by every entry point
 *   - Every function returns an ieti_status; IETI_OK = 0, errors are negative.
 *     After an error, ieti_last_error(ctx) returns a message owned by ctx.
 *   - Pointers named *_host are host memory owned by the caller; the library
 *     copies what it keeps before returning. Pointers named *_dev are device
 *     memory of the current CUDA device, owned by the caller.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Entry points
 *     that take a stream enqueue their work on it and may return before the
 *     work completes, unless stated otherwise.
 *   - Multi-column vectors are column-major with `nrhs` columns.
 *   - The context owns all device memory it allocates until ieti_destroy.
 *   - Global numbering (the data format of every index argument):
 *       node (i,j,k) of the glued control net -> i + N0 (j + N1 k);
 *       an edge of direction d joins node (i,j,k) to (i,j,k)+e_d (wrapping in a
 *       periodic direction 0) and is oriented along increasing parameter;
 *       edge ids: all direction-0 edges, then direction 1, then direction 2,
 *       each block lexicographic with i fastest.
 *     Multipliers (dual DOFs) are numbered by increasing edge id, as are the
 *     primal (coarse) DOFs.
 */
#ifndef IETI_H
#define IETI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IETI_OK = 0,
  IETI_ERR_INVALID_ARG = -1,
  IETI_ERR_NOT_SIMPLY_CONNECTED = -2,
  IETI_ERR_TREE_INCONSISTENT = -3,
  IETI_ERR_SINGULAR_LOCAL = -4,
  IETI_ERR_NO_CONVERGENCE = -5,
  IETI_ERR_TIMEOUT = -6,
  IETI_ERR_CUDA = -7,
  IETI_ERR_OOM = -8,
  IETI_ERR_STATE = -9
} ieti_status;

/* Precision of the local factorisations (Sec. 2.1: K_rr^(k) is factored per
 * subdomain).
 *   IETI_FP64:    FP64 Cholesky of every K_rr^(k); every operator in FP64.
 *   IETI_FP32_IR: FP32 Cholesky and FP32 local interface operators, used as an
 *                 approximate FETI-DP solver inside FP64 iterative refinement on
 *                 the assembled system (FP64 residuals, FP64 coarse matrix,
 *                 FP64 PCG vectors and inner products). */
typedef enum { IETI_FP64 = 0, IETI_FP32_IR = 1 } ieti_precision;

/* Source kinds of the right-hand side j of Eq. (3). */
typedef enum {
  IETI_SOURCE_SINE = 0,      /* J = s 2 pi^2 (sin pi y sin pi z, sin pi x sin pi z, sin pi x sin pi y);
                                params: one amplitude s per load case */
  IETI_SOURCE_FOURIER = 1,   /* J = sum_m Re(c_m exp(2 pi i k_m.x)); params per load case:
                                nmodes, then per mode k(3), Re c(3), Im c(3) */
  IETI_SOURCE_PATCHWISE = 2, /* J constant per patch; params: nrhs x npatch x 3 */
  IETI_SOURCE_TRIG = 3       /* the manufactured problem of Sec. 3 scaled by s: J = s 3 A_ana with
                                A_ana = (cos y cos z sin x, -2 cos x cos z sin y, cos x cos y sin z)
                                (curl curl A_ana = 3 A_ana) and the non-homogeneous tangential
                                Dirichlet data n x A = n x (s A_ana) on the boundary; params: one
                                amplitude s per load case. Axis-aligned affine box patches only
                                (affine = 1) and no periodic direction. The coefficients of the
                                edges in the boundary faces are s times the boundary L2
                                projection of the tangential trace of A_ana (computed once in
                                ieti_create, on the host), the loads are lifted by them
                                (j - K a_D, in ieti_assemble) and ieti_solve returns them in
                                the Dirichlet entries of the field. The reference flux of
                                ieti_eval_B is IETI_BREF_TRIG (exact for nu = 1). */
} ieti_source_kind;

/* Multipatch problem (Sec. 2): a structured P0 x P1 x P2 block grid of patches,
 * each the image of (0,1)^3 under a trivariate B-spline/NURBS map of degree p
 * with an open uniform knot vector; patch slab a of direction d has
 * nspan[d][a] knot spans. Neighbouring patches share full patch-facets and the
 * control points on them, so the geometry is one glued control net of
 * N0 x N1 x N2 points, N_d = sum_a (nspan[d][a] + p - 1) + 1 (no "+1" when
 * direction 0 is periodic). Patch (a,b,c) has index a + P0 (b + P1 c).
 * Subdomains (Sec. 2) are the groups of sub_of_patch; each must be connected
 * and simply connected. The edge space has degree p-1 along an edge and p
 * across it; homogeneous tangential Dirichlet data n x A = 0 on the boundary
 * except for IETI_SOURCE_TRIG, which brings its own data. The source
 * parameters are checked against the kind and nrhs (INVALID_ARG if too few). */
typedef struct {
  int degree;                  /* p >= 1 */
  int npatch[3];               /* P0, P1, P2 */
  const int* nspan_host[3];    /* nspan_host[d][a], a < npatch[d], each >= 1 */
  int periodic0;               /* 1: direction 0 is periodic (closed ring) */
  const double* ctrl_host;     /* N2 x N1 x N0 x 4: x, y, z, weight (i fastest) */
  const double* nu_host;       /* reluctivity per patch, > 0 */
  const int* sub_of_patch_host;/* subdomain id per patch, 0 .. nsub-1, all used */
  int source_kind;             /* ieti_source_kind */
  const double* source_params_host;
  int n_source_params;
  int nrhs;                    /* load cases, 1 .. 64 */
  int affine;                  /* 1 if every patch map is an axis-aligned affine
                                  map (enables the Kronecker assembly path; the
                                  library checks it: weights 1 and control points
                                  at the scaled Greville abscissae, else
                                  IETI_ERR_INVALID_ARG); 0 for any other map */
} ieti_problem_desc;

typedef struct ieti_ctx ieti_ctx;

typedef struct {
  int64_t nedge, nnode;        /* control mesh */
  int64_t n_dirichlet, n_tree; /* removed DOFs (Sec. 2, Sec. 2.2) */
  int64_t n_gauged;            /* unknowns of the gauged global system */
  int64_t m_r;                 /* multipliers lambda_r (Eq. (5)) */
  int64_t n_gp;                /* coarse primal DOFs */
  int64_t nsub, nrhs;
  int64_t max_nr, max_nI;      /* largest local r block / interface block */
  int64_t sum_nr2, sum_nI2;    /* sum_k n_r^2, sum_k n_I^2 (dense sizes) */
  int64_t bytes_device;        /* device memory held by the context */
  int tree_rerun;              /* 1 if Kruskal was rerun with boundary edges first */
} ieti_sizes;

typedef struct {
  int iterations;              /* PCG iterations (summed over refinement steps) */
  int refinement_steps;        /* FP64 refinement steps (IETI_FP32_IR), else 1 */
  double relres;               /* last ||b - F lambda|| / ||b|| (max over load cases) */
  double global_relres;        /* FP64 ||j - K a|| / ||j|| of the returned field */
  double kappa;                /* Lanczos estimate of kappa(M^-1 F) (first load case) */
  int converged;               /* 1 if every load case met the tolerance */
  double ms_total;             /* device time of the call */
  int fp64_fallback;           /* 1 if the FP32 factors were replaced by FP64 factors
                                  during the call (refinement stalled) */
} ieti_solve_info;

/* Builds the mesh, the 1D basis tables at the Gauss points (p+1 per span), the
 * facets, wire basket, edge weights (Fig. "weights"), the Kruskal spanning tree
 * (Sec. 2.2), primal (cotree weight-2) and dual DOFs, the signed jump operator
 * B_r (Eq. (4)/(5)) and C_p, and allocates every device buffer. Host-side and
 * one-off. Errors: INVALID_ARG (bad sizes), NOT_SIMPLY_CONNECTED (a subdomain
 * is not a contractible union of patches), TREE_INCONSISTENT (the spanning
 * tree is not a tree on the Dirichlet boundary even after the rerun, or a
 * multiplier would couple more than two subdomains), OOM, CUDA. */
ieti_status ieti_create(const ieti_problem_desc* desc, ieti_ctx** out);

/* Host-only variant of ieti_create: builds the mesh, tables, gauge and DOF maps
 * without touching the GPU, for inspection through ieti_query and
 * ieti_get_dofmap. Every other entry point returns IETI_ERR_STATE on such a
 * context. Same errors as ieti_create except CUDA and OOM. */
ieti_status ieti_create_host(const ieti_problem_desc* desc, ieti_ctx** out);

/* Replaces the per-patch reluctivities (npatch values) and/or the source
 * parameters (same layout as in the descriptor); either pointer may be NULL.
 * Takes effect at the next ieti_assemble. */
ieti_status ieti_set_params(ieti_ctx* ctx, const double* nu_host,
                            const double* source_params_host, int n_source_params);

/* Eq. (3), batched over all patches of all subdomains: assembles, per
 * subdomain k, the dense blocks K_rr^(k) (order [r_V, pad, r_I]), K_rp^(k),
 * K_pp^(k) and the loads j_r^(k), j_p^(k) in FP64 on the device. After the
 * first factorisation has found the nonzero 64 x 64 tiles of K_rr (a pattern
 * fixed by the mesh, not by the reluctivities), only those tiles are
 * generated again; the geometry at the Gauss points is kept from the first
 * assembly. */
ieti_status ieti_assemble(ieti_ctx* ctx, void* stream);

/* Sec. 2.1: batched Cholesky of every K_rr^(k) in the chosen precision, over
 * the nonzero 64 x 64 tiles of a tile-level symbolic factorisation (found on
 * the first call from the assembled K_rr and kept); the
 * interface Schur complement S_rIrI^(k) of Eq. (10) is taken from the factor
 * after the r_V columns; Phi^(k) = K_rr^-1 K_rp; the coarse matrix
 * S_Pi = -F (F of Eq. (7)) in FP64 and its Cholesky factor; the local
 * interface operators (K_rr^-1)_II = S_rIrI^-1. Under IETI_FP32_IR a
 * non-positive FP32 pivot (a local block too ill-conditioned for single
 * precision) makes the call factor in FP64 instead; the context then holds
 * FP64 factors as after IETI_FP64. Errors: SINGULAR_LOCAL (a non-positive
 * pivot in FP64; the subdomain id is in the message), STATE (not
 * assembled), TIMEOUT (a bounded device wait of the interface products or of
 * the W and Phi solves gave up), CUDA. Synchronises the stream. */
ieti_status ieti_factor(ieti_ctx* ctx, ieti_precision prec, void* stream);

/* Eq. (7): y = F_DP lam with F_DP = W - G F^-1 G^T = B_r K_rr^-1 B_r^T
 * + G S_Pi^-1 G^T (the SPD negation of the paper's S). lam_dev, y_dev: m_r x
 * nrhs FP64 device arrays (nrhs <= 64), not aliased. Uses the operators of the
 * last ieti_factor (FP64 or FP32 storage). Errors: STATE, INVALID_ARG. */
ieti_status ieti_apply_F(ieti_ctx* ctx, const double* lam_dev, double* y_dev, int nrhs,
                         void* stream);

/* Eq. (7), evaluated through the local factors instead of the explicit
 * W_k = S_rIrI^-1: the local part B_r K_rr^-1 B_r^T lam as triangular solves
 * with the r_I block of each Cholesky factor (K_rr^-1 restricted to the r_I
 * rows and columns is (L_II L_II^T)^-1), plus the same coarse part. The same
 * F_DP lam as ieti_apply_F up to rounding; kept to compare the two
 * evaluations. nrhs must equal the context's number of load cases (the
 * solves use its work buffers). Errors: STATE (not factored), INVALID_ARG,
 * TIMEOUT (a sweep wait gave up), CUDA. */
ieti_status ieti_apply_F_implicit(ieti_ctx* ctx, const double* lam_dev, double* y_dev, int nrhs,
                                  void* stream);

/* Eq. (10): z = M_D^-1 r = sum_k D^(k) B_rI^(k) S_rIrI^(k) B_rI^(k)T D^(k) r,
 * with D^(k) the rho-scaling weights nu_l / (nu_k + nu_l). r_dev, z_dev: m_r x
 * nrhs FP64 device arrays, not aliased. */
ieti_status ieti_apply_precond(ieti_ctx* ctx, const double* r_dev, double* z_dev, int nrhs,
                               void* stream);

/* Eqs. (7)-(9): right-hand side b = e - G F^-1 d, PCG with M_D^-1 on
 * F_DP lam = b until ||b - F_DP lam|| <= tol ||b|| per load case (or maxit),
 * coarse recovery a_p = C F^-1 (d - G^T lam) and local recovery
 * a_r = K_rr^-1 (j_r - K_rp a_p - B_r^T lam). Under IETI_FP32_IR this is the
 * inner solver of FP64 iterative refinement on the assembled system, repeated
 * until the FP64 relative residual of the field is <= tol_field (default 1e-10
 * when <= 0) or 16 refinement steps; if one of the first two correction
 * steps cuts the field residual by less than a factor 4 although its inner
 * PCG converged (FP32 factors outside their regime, kappa(K_rr) u_32 not
 * small), the context switches to FP64 factors for the remaining steps
 * (info->fp64_fallback). Each inner PCG stops at
 * max(tol, 1e-3) on the first step and max(tol, 3e-3) on the corrections,
 * since a refinement step with FP32 operators cannot reduce the error by much
 * more than that anyway. lam0_dev: m_r x nrhs initial multipliers or
 * NULL for zero (INVALID_ARG if it holds NaN or infinite values). a_dev: nedge x nrhs output field (tree DOFs
 * are zero; Dirichlet DOFs are zero, or the boundary coefficients of
 * IETI_SOURCE_TRIG). lam_dev: optional m_r x nrhs output of the final multipliers.
 * info: optional host struct. Synchronises the stream. Errors: STATE,
 * INVALID_ARG, NO_CONVERGENCE (info still filled, a_dev holds the last
 * iterate), TIMEOUT (a bounded wait of the triangular sweeps or of the
 * streamed products gave up; the context stays usable). */
ieti_status ieti_solve(ieti_ctx* ctx, const double* lam0_dev, double tol, int maxit,
                       double tol_field, double* a_dev, double* lam_dev,
                       ieti_solve_info* info, void* stream);

/* Reference fields of ieti_eval_B. */
typedef enum {
  IETI_BREF_NONE = 0,   /* no reference: only the norms of B */
  IETI_BREF_SINE = 1,   /* B_ref = s curl(sin pi y sin pi z, sin pi x sin pi z, sin pi x sin pi y)
                           = s pi (sin pi x (cos pi y - cos pi z), sin pi y (cos pi z - cos pi x),
                           sin pi z (cos pi x - cos pi y)), one amplitude s per load case: the
                           exact flux of IETI_SOURCE_SINE with amplitude s when nu = 1 */
  IETI_BREF_TRIG = 2    /* B_ref = s B_ana = s (-3 cos x sin y sin z, 0, 3 cos z sin x sin y) of
                           Sec. 3: the exact flux of IETI_SOURCE_TRIG with amplitude s when nu = 1 */
} ieti_bref_kind;

/* Sec. 3: the magnetic flux density B = curl a and the error
 * eps_B = sqrt(sum_k ||B_ref - B||^2_L2(Omega^(k))) of fields a, evaluated on
 * the device at the p+1 Gauss points per direction per knot span of every
 * element (the assembly's rule), with the covariant Piola map
 * B = DF curl_hat(a) / det DF and the measure |det DF| dxi.
 *   a_dev        nedge x nrhs FP64 device array in the global edge numbering;
 *                every entry is used (Dirichlet and tree edges included), so
 *                any field of the discrete space can be evaluated
 *   nrhs         1 .. 64 columns
 *   ref_kind     ieti_bref_kind; ref_amp_host: nrhs amplitudes (host), used
 *                unless ref_kind is IETI_BREF_NONE
 *   nB2_host     npatch x nrhs (patch fastest): ||B||^2_L2 over each patch
 *   err2_host    npatch x nrhs: ||B_ref - B||^2_L2 over each patch, or NULL
 *                (sum over the patches of subdomain k: the k-th term of eps_B^2)
 *   B_dev        optional (NULL): B at the Gauss points, nelem x (p+1)^3 x 3
 *                per column (elements patch by patch, spans with direction 0
 *                fastest; Gauss points x fastest; then the 3 components)
 * Synchronises the stream. Errors: STATE (host-only context), INVALID_ARG. */
ieti_status ieti_eval_B(ieti_ctx* ctx, const double* a_dev, int nrhs, int ref_kind,
                        const double* ref_amp_host, double* nB2_host, double* err2_host,
                        double* B_dev, void* stream);

/* Sizes of the problem and of the device data. */
ieti_status ieti_query(const ieti_ctx* ctx, ieti_sizes* out);

/* DOF maps for inspection (host copies). which:
 *   0 tree flag per edge (nedge, int64 0/1)
 *   1 edge weight 1..5 per edge (nedge)
 *   2 primal edge ids (n_gp)
 *   3 dual edge ids (m_r)
 *   4 r_V edge ids of subdomain `sub`, in the library's local order:
 *     lexicographic in the control index of the edge, the axis with the
 *     longest extent outermost, the direction last (a banded K_rr)
 *   5 r_I edge ids of subdomain `sub`
 *   6 primal edge ids of subdomain `sub`
 *   7 sign (+1/-1) of each r_I DOF of subdomain `sub`
 * Writes min(count, cap) values to out_host and the count to *count. */
ieti_status ieti_get_dofmap(const ieti_ctx* ctx, int which, int sub, int64_t* out_host,
                            int64_t cap, int64_t* count);

/* IETI_SOURCE_TRIG: the boundary coefficients a_D of the unit-amplitude field
 * (nedge FP64 values in the global edge numbering, zero off the Dirichlet
 * faces; host copy, also on a host-only context). Writes min(nedge, cap)
 * values to out_host and nedge to *count; *count = 0 for the other source
 * kinds (homogeneous data). */
ieti_status ieti_get_boundary_data(const ieti_ctx* ctx, double* out_host, int64_t cap, int64_t* count);

/* Copies a dense FP64 block of subdomain `sub` to the host, column-major with
 * leading dimension `rows` as returned in *rows_out, *cols_out. which:
 *   0 K_rr as assembled (rows/cols ordered [r_V, r_I], padding removed)
 *   1 K_rp, 2 K_pp, 3 j_r (n_r x nrhs), 4 j_p,
 *   5 S_rIrI (after ieti_factor), 6 (K_rr^-1)_II (after ieti_factor).
 * out_host may be NULL to query the shape. Synchronises the device. */
ieti_status ieti_get_block(ieti_ctx* ctx, int which, int sub, double* out_host, int64_t cap,
                           int64_t* rows_out, int64_t* cols_out);

/* The FP64 coarse matrix S_Pi = -F (n_gp x n_gp, host copy) after ieti_factor. */
ieti_status ieti_get_coarse(ieti_ctx* ctx, double* out_host, int64_t cap);

/* Interface right-hand side b = e - G F^-1 d (m_r x nrhs, device) for the
 * current loads, from the last factorisation. */
ieti_status ieti_interface_rhs(ieti_ctx* ctx, double* b_dev, void* stream);

/* Number of kernel launches this context has issued so far. */
int64_t ieti_launch_count(const ieti_ctx* ctx);

/* Testing aids for the failure paths and the experimental code paths (the
 * paper has no counterpart; faults are injected from the host, no device code
 * is made to fault):
 *   IETI_DEBUG_WAIT_POLLS   poll limit of the progress-counter waits of the
 *                           dependency-driven triangular sweeps (value >= 0
 *                           polls of about 0.1 us; < 0 restores the default
 *                           2^22). A wait that runs out sets the context's
 *                           error flag and lets the launch finish; the call
 *                           then returns IETI_ERR_TIMEOUT.
 *   IETI_DEBUG_PIVOT_FAULT  subdomain whose K_rr gets a negative first diagonal
 *                           entry in the factor buffer at every following
 *                           ieti_factor, which then returns
 *                           IETI_ERR_SINGULAR_LOCAL naming that subdomain
 *                           (value < 0 switches it off).
 *   IETI_DEBUG_FP64_FALLBACK value != 0: the next FP32 refinement treats its
 *                           first correction step as stalled and switches to
 *                           FP64 factors (the path taken when FP32 factors are
 *                           outside their regime).
 *   IETI_DEBUG_SYRK_TC      value != 0: the FP32 trailing updates run on the
 *                           tensor cores (tcgen05, split TF32 products); an
 *                           experimental path, slower than the default CUDA-core
 *                           update. Only before the first ieti_factor (STATE
 *                           after it).
 *   IETI_DEBUG_NO_AUTOTUNE  value != 0: the tile shapes of the streamed
 *                           products keep their defaults (no timing of
 *                           candidates at the first factorisation of each
 *                           precision).
 *   IETI_DEBUG_ELEMENT_LOADS value != 0: the loads of axis-aligned box patches
 *                           are integrated element by element like those of
 *                           curved patches, instead of from separable 1D
 *                           integrals (the same Gauss rule; kept to compare).
 *   IETI_DEBUG_SYRK_RESERVE SMs that the overlapped FP32 trailing update leaves
 *                           to the panel kernels of the next step (value 0 ..
 *                           SM count - 1; < 0 restores the default 24). Changes
 *                           only the time of ieti_factor.
 * Errors: INVALID_ARG (unknown setting, subdomain out of range), STATE. */
enum {
  IETI_DEBUG_WAIT_POLLS = 1,
  IETI_DEBUG_PIVOT_FAULT = 2,
  IETI_DEBUG_FP64_FALLBACK = 3,
  IETI_DEBUG_SYRK_TC = 4,
  IETI_DEBUG_NO_AUTOTUNE = 5,
  IETI_DEBUG_SYRK_RESERVE = 6,
  IETI_DEBUG_ELEMENT_LOADS = 7
};
ieti_status ieti_debug_set(ieti_ctx* ctx, int what, int64_t value);

/* Per-kernel-class device timing with CUDA events recorded around each launch
 * group on the launching stream (enable = 1), around the groups of some
 * classes only (enable > 1: class c is timed if bit c + 1 of enable is set),
 * or off (0); resets the totals.
 * Classes, in order: 0 assembly of K, 1 assembly of j, 2 diagonal-block
 * Cholesky, 3 panel triangular solve, 4 trailing symmetric update, 5 forward
 * substitution sweeps, 6 backward substitution sweeps, 7 local products with
 * W = S_rIrI^-1 (F-apply), 8 local products with S_rIrI (preconditioner),
 * 9 multiplier gathers, 10 coarse solves, 11 PCG vector kernels,
 * 12 FP64 field residual, 13 other. */
ieti_status ieti_profile(ieti_ctx* ctx, int enable);

/* Totals since the last ieti_profile call: milliseconds and number of timed
 * launch groups per class (first n classes). Synchronises the device. */
ieti_status ieti_profile_read(ieti_ctx* ctx, double* ms_host, int64_t* calls_host, int n);

void ieti_destroy(ieti_ctx* ctx);
const char* ieti_last_error(const ieti_ctx* ctx);

/* Batched interface product that allocates no device memory (the paper has no
 * counterpart; this is a library service).
 *
 * For callers that cannot call cudaMalloc when they need this product: an
 * outer solver or framework that owns the device memory pool and hands the
 * library only its own input and output buffers, where an allocation would fail
 * against that pool's budget or fragment it. The caller passes every input and
 * output; the scratch (per-subdomain descriptors and local products) lives in
 * one fixed 32 MiB array inside the library, which every GPU that loads the
 * library holds until the process exits.
 *
 * Computes y = sum_k B_k^T diag(w_k) M_k diag(w_k) B_k x, i.e. for each
 * subdomain k: u = w_k .* x[dual_k]; t = M_k u; y[dual_k] += w_k .* t.
 *   nsub        number of subdomains, 1..4096
 *   nI_host     host array: interface block size nI_k >= 0 of each subdomain
 *               (read during the call only)
 *   M_dev       device FP64: the symmetric blocks M_k, each nI_k x nI_k
 *               column-major, concatenated in subdomain order
 *   dual_dev    device int32: multiplier index (0 .. m-1) of every local
 *               interface DOF, concatenated in subdomain order; an index
 *               outside [0, m) is a caller error and its entry is skipped
 *   weight_dev  device FP64: weight w of every local interface DOF (same order)
 *   m, nrhs     multipliers and columns; x_dev, y_dev are m x nrhs FP64
 *               column-major, not aliased; y_dev is overwritten
 * Two uses: with M_k the interface Schur complement S_rIrI^(k) and w_k the
 * sign of each multiplier times its scaling weight this is the Dirichlet
 * preconditioner; with M_k = (K_rr^(k)^-1)_II (the inverse of S_rIrI^(k)) and
 * w_k the signs it is the local part of the F-apply, B_r K_rr^-1 B_r^T x.
 * Limits and errors: sum_k nI_k * nrhs must not exceed 4,177,920 (the scratch
 * minus the descriptor area); larger requests return IETI_ERR_INVALID_ARG with a
 * message on stderr, as do bad arguments. IETI_ERR_CUDA on a CUDA error.
 * The first call on each device looks up the device address of the scratch
 * array (one-time set-up with that device current); make that first call
 * before any stream capture. Every call shares the one scratch array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller. Enqueued on `stream`; returns before completion. */
ieti_status ieti_interface_product_noalloc(int nsub, const int* nI_host, const double* M_dev,
                                           const int* dual_dev, const double* weight_dev, int64_t m,
                                           const double* x_dev, double* y_dev, int nrhs, void* stream);

/* ---------------------------------------------------------------------------
 * Learned warm start for the interface multipliers (the paper has no learned
 * component; this is an extension). A 3-layer perceptron maps a parameter
 * vector of a problem instance (for example log nu per patch and the source
 * amplitudes) to an initial guess lambda0 for ieti_solve. PCG on Eq. (7) keeps
 * its own stopping test, so the guess changes iteration counts, not accuracy.
 *
 * Network: x' = (x - shift) .* scale; Z1 = x' W1^T + b1, A1 = relu(Z1);
 * Z2 = A1 W2^T + b2, A2 = relu(Z2); y = A2 W3^T + b3; lambda0 = out_scale * y.
 * GEMM operands are rounded to bfloat16 (round to nearest even), products are
 * accumulated in FP32 on the tensor cores; biases, master weights, gradients
 * and Adam moments are FP32. W_l is (out x in) row-major.
 * Parameter vector layout (FP32, host): W1 | b1 | W2 | b2 | W3 | b3, sizes
 * h*n_in, h, h*h, h, n_out*h, n_out.
 * Loss: mean over the batch and outputs of (y - t/out_scale)^2 (targets t in
 * multiplier units). Adam: beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.
 * Batches are row-major (batch x n_in / batch x n_out) FP32 device arrays.
 * ------------------------------------------------------------------------- */
typedef struct ieti_mlp ieti_mlp;

/* Allocates parameters (zero), moments, activations for up to max_batch rows.
 * IETI_ERR_INVALID_ARG on sizes < 1, IETI_ERR_OOM if allocation fails (the
 * handle is still returned and must be destroyed). Synchronous. */
ieti_status ieti_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, ieti_mlp** out);
/* sizes4 = {n_in, n_hidden, n_out, max_batch}; *nparam = parameter count. */
ieti_status ieti_mlp_query(const ieti_mlp* m, int* sizes4, int64_t* nparam);
/* Copies all parameters from the host (count must equal the parameter count),
 * resets the Adam moments and step counter. Synchronous. */
ieti_status ieti_mlp_set_params(ieti_mlp* m, const float* params_host, int64_t count);
/* Input normalisation (n_in entries each, host) and output scale (> 0). */
ieti_status ieti_mlp_set_scaling(ieti_mlp* m, const float* shift_host, const float* scale_host,
                                 float out_scale);
/* which = 0: parameters, 1: gradients of the last backward pass, 2: the input
 * shift (n_in), input scale (n_in) and out_scale (1). *count is set to the
 * number of values; with out_host == NULL nothing is copied, else cap must be
 * >= *count. IETI_ERR_INVALID_ARG for another `which`. Synchronous. */
ieti_status ieti_mlp_get(ieti_mlp* m, int which, float* out_host, int64_t cap, int64_t* count);
/* lambda0 (batch x n_out) for inputs x (batch x n_in); 1 <= batch <= max_batch.
 * Enqueued on `stream`. */
ieti_status ieti_mlp_forward(ieti_mlp* m, const float* x_dev, float* y_dev, int batch, void* stream);
/* As ieti_mlp_forward, but lambda0 is written in FP64: row b of lam_dev
 * (batch x n_out row-major) is the initial guess of load case / instance b, the
 * multi-column layout ieti_solve takes for lam0_dev. */
ieti_status ieti_mlp_forward_f64(ieti_mlp* m, const float* x_dev, double* lam_dev, int batch,
                                 void* stream);
/* Source-linear head: the outputs of a row are read as ncoef blocks of
 * m = n_out / ncoef values (the responses to ncoef unit sources, which the
 * solution depends on linearly) and combined with that row's coefficients:
 *   lam[b, j] = out_scale * sum_c coef[b, c] * y[b, c m + j]   (FP64 sum)
 * coef_dev: batch x ncoef FP64 row-major; lam_dev: batch x m FP64 row-major
 * (the lam0 layout of ieti_solve). IETI_ERR_INVALID_ARG unless ncoef divides
 * n_out. Enqueued on `stream`. */
ieti_status ieti_mlp_forward_combine(ieti_mlp* m, const float* x_dev, const double* coef_dev, int ncoef,
                                     double* lam_dev, int batch, void* stream);
/* Forward + loss + gradients of all parameters for targets t (batch x n_out).
 * If loss_host is not NULL, the loss is copied there and the stream is
 * synchronised; otherwise returns before completion. */
ieti_status ieti_mlp_backward(ieti_mlp* m, const float* x_dev, const float* t_dev, int batch,
                              float* loss_host, void* stream);
/* One Adam step with learning rate lr > 0 on the last gradients; refreshes the
 * bfloat16 weight copies. Enqueued on `stream`. */
ieti_status ieti_mlp_adam(ieti_mlp* m, float lr, void* stream);
/* Mini-batch training on n_samples pairs (X_dev: n_samples x n_in, T_dev:
 * n_samples x n_out, FP32 row-major, device). With normalise != 0 the input
 * shift/scale are first set to the per-feature mean and 1/std of X and
 * out_scale to the root mean square of T (1 if that is 0). Each epoch visits
 * the samples in an order drawn by a Fisher-Yates shuffle from splitmix64
 * seeded with (seed, epoch); batches of `batch` rows (the last one ragged),
 * one backward pass and one Adam step each, learning rate lr * decay^epoch
 * (0 < decay <= 1). loss_host (optional) receives the mean batch loss of the
 * last epoch. Synchronises the stream at the start (normalise) and at the end
 * (loss_host); IETI_ERR_INVALID_ARG on bad sizes. */
ieti_status ieti_mlp_fit(ieti_mlp* m, const float* X_dev, const float* T_dev, int n_samples, int batch,
                         int epochs, float lr, float decay, unsigned long long seed, int normalise,
                         float* loss_host, void* stream);
void ieti_mlp_destroy(ieti_mlp* m);
const char* ieti_mlp_last_error(const ieti_mlp* m);

#ifdef __cplusplus
}
#endif

#endif /* IETI_H */
