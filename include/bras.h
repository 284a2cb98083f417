/*
 * bras.h -- C ABI of the B300 BRAS mass-solve library (libbras.so).
 *
 * The library applies, on one GPU, the broken-space additive Schwarz (BRAS) approximation
 * of a conforming finite-element mass inverse,
 *
 *     M_bras^{-1} = D^{-1} P^T M_br^{-1} P D^{-1} = D^{-1} (sum_K P_K^T M_K^{-1} P_K) D^{-1}
 *
 * (Sec. 2.2, Eq. mhatinvbras_def and its element-sum form), together with the conforming
 * mass matrix M = P^T M_br P = sum_K P_K^T M_K P_K (Sec. 2.2, Eq. M_PMbrP), the diagonal
 * approximation diag(M)^{-1} (Sec. 2.1) and a preconditioned-CG mass solve with the
 * paper's stopping rule ||r_k||_2 / ||r_0||_2 <= rtol, u_0 = 0 (Sec. 3).
 *
 * Conventions shared by every call
 * --------------------------------
 *  * Pointers are DEVICE pointers unless a call says otherwise; the caller owns them.
 *    The context owns every table it builds, until bras_destroy.
 *  * Calls are ordered on the CUDA stream passed as `stream` (a cudaStream_t, may be
 *    NULL for the legacy default stream).  Apply calls are asynchronous; bras_setup and
 *    bras_pcg_solve synchronise the stream before they return.
 *  * Vectors with nrhs > 1 right-hand sides are RHS-interleaved: entry (i, r) is at
 *    i * nrhs + r.  Dof i is the global dof number used in `l2g`.
 *  * Element kinds (Sec. 3): BRAS_H1 = Lagrange (equispaced or GLL-based nodes, or Bernstein;
 *    bras_options.basis) P_p
 *    on triangles (dim 2) or tetrahedra (dim 3), p = 1..4; BRAS_HCURL = Nedelec first kind
 *    and BRAS_HDIV = Raviart-Thomas, order k = 1..4, or with bras_options.basis = 1 the
 *    second kinds N2curl and BDM (the full P_k^dim, k = 1..4; Tables 2-3), on triangles or
 *    tetrahedra, mapped by
 *    the covariant / contravariant Piola maps (Sec. 2.4, Eq. piola_mass_pullbacks) with
 *    |det J|.  Local dof order and dof functionals are the ones documented with the mesh
 *    generator and the reference elements (vertices of each tetrahedron listed in
 *    ascending global id for face moments of order >= 2).
 *  * Return codes: 0 = success, > 0 = non-fatal status, < 0 = error (nothing written
 *    to the outputs except where stated).  No call prints, throws or exits.
 *    bras_status_string() names a code; bras_last_error_detail() gives the element or
 *    dof index that caused the last error of this thread (-1 if none).
 *  * Determinism: every reduction (scatter-average, dot products) runs in a fixed order
 *    with no floating-point atomics, so two calls with the same inputs give bit-identical
 *    outputs.
 */
#ifndef BRAS_H
#define BRAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bras_ctx bras_ctx;

enum { BRAS_H1 = 0, BRAS_HCURL = 1, BRAS_HDIV = 2 };

/* Precision of an apply (the element data it streams and the arithmetic it runs in).
 * BRAS_FP64: double vectors, double element data, double arithmetic.
 * BRAS_FP32: float vectors, float element data, float arithmetic.
 * BRAS_BF16: float vectors and arithmetic; H(curl)/H(div) local inverses stored in
 *            bfloat16 (H1 has no per-element matrix: same as BRAS_FP32 there).       */
enum { BRAS_FP64 = 0, BRAS_FP32 = 1, BRAS_BF16 = 2, BRAS_FP64X = 3 };
/* BRAS_FP64X (bras_mass_apply only): double vectors and scatter sums; for H1 the local
 * products run in float-float arithmetic on the FP32 units (an error-free split of each
 * product into two floats and a compensated sum, about 2^-48 relative per term), the form
 * the mixed solve uses for its refinement residual b - M x; other spaces use FP64. */

/* Preconditioner of a solve: none, diag(M)^{-1} (Jacobi), or BRAS. */
enum { BRAS_PC_NONE = 0, BRAS_PC_JACOBI = 1, BRAS_PC_BRAS = 2 };

/* Solve modes: plain FP64 PCG, or FP32 inner PCG (FP64 dot products and scalars)
 * inside an FP64 iterative-refinement loop r = b - M x, x += d. */
enum { BRAS_SOLVE_FP64 = 0, BRAS_SOLVE_MIXED = 1 };

enum {
    BRAS_OK = 0,
    BRAS_NOT_CONVERGED = 1,       /* maxit reached; x, iters, relres are still written */
    BRAS_ERR_INVALID = -1,        /* bad argument (null pointer, size, enum, order)     */
    BRAS_ERR_L2G_RANGE = -2,      /* l2g entry outside [0, n_dof) (detail = flat index) */
    BRAS_ERR_NO_COPY = -3,        /* a dof no element references (detail = dof)        */
    BRAS_ERR_DEGENERATE = -4,     /* det J = 0 (detail = element)                        */
    BRAS_ERR_NOT_SPD = -5,        /* local Cholesky pivot <= 0 (detail = element)        */
    BRAS_ERR_CUDA = -6,           /* a CUDA call failed                                  */
    BRAS_ERR_OOM = -7,            /* device or host allocation failed                    */
    BRAS_ERR_BREAKDOWN = -8,      /* CG breakdown: p^T M p <= 0 or not finite            */
    BRAS_ERR_PRECISION = -9,      /* the context holds no tables for this precision      */
    BRAS_ERR_TOO_LARGE = -10,     /* a size exceeds a documented library limit           */
    BRAS_ERR_DEVICE = -11         /* a kernel's bounded wait ran out (detail = status bits) */
};

/* Options of bras_setup.  Zero-initialise, then set what you need. */
typedef struct {
    int precisions;      /* bit mask of (1 << BRAS_FP64 | 1 << BRAS_FP32 | 1 << BRAS_BF16);
                            0 means all three.  H(curl)/H(div) always keep the FP64 cell mass
                            matrices (refinement residual, diag); their FP64 inverses only with
                            the FP64 bit -- without it, FP64 BRAS applies and FP64 solves with
                            BRAS return BRAS_ERR_PRECISION (the mixed solve needs only FP32 or
                            bf16 inverses)                                                    */
    int block_elems;     /* elements per scatter block, 32..256 (H1 contexts without the
                            tensor-core kernel: 32..1024); 0 = 256                          */
    int max_nrhs;        /* largest nrhs the solve workspace is sized for; 0 = 1          */
    int simt_only;       /* 1: H1 FP32 applies on the FP32 units instead of the tensor-core
                            (3xTF32 tcgen05) local GEMM; 0 = tensor cores where supported  */
    int basis;           /* BRAS_H1: 0 = Lagrange (values at the equispaced nodes),
                            1 = Bernstein (B_alpha = p!/alpha! prod lambda_i^alpha_i, the
                            "Bernstein" family of Table 1), 2 = Lagrange at GLL-based nodes
                            (the recursive nodes of Isaac (2020) on the Gauss-Lobatto-Legendre
                            points: the "spectral" nodal variant of Sec. 3, Table 1's Lagrange
                            column; equal to 0 for p <= 2); same multi-indices, same l2g.
                            BRAS_HCURL / BRAS_HDIV: 0 = first kind (N1curl_k / RT_k),
                            1 = second kind (N2curl_k / BDM_k, k = 1..4)                  */
    int autotune;        /* 1: at setup, time the FP32 (else FP64) BRAS apply for eight cell
                            block sizes (H1 on the FP32 units: 64..1024; H1 with tensor
                            cores: 64..256; H(curl)/H(div): 32..256) whose kernels fit shared
                            memory and keep the fastest (one table build and twelve applies per
                            candidate, the mean of the last ten kept; ignored if block_elems is
                            set); 0 = the rule: the largest
                            size up to 256 whose FP32 kernel fits twice per SM              */
} bras_options;

/*
 * bras_setup -- build a context for one conforming space on one simplicial mesh.
 *
 * Computes, all on the device: J_K, |det J_K| and the Piola metric G_K of every cell
 * (Sec. 2.4); for H1 the single reference mass M_ref and its inverse (the affine
 * element inverse is M_K^{-1} = M_ref^{-1} / (rho_K |det J_K|)); for H(curl) and H(div)
 * every M_K = sum_ab G_K,ab R_ab and its FP64 Cholesky inverse (Sec. 2.2: M_K is SPD);
 * the multiplicities d_i = #{broken copies of dof i} (D = P^T P); diag(M); and the
 * deterministic scatter tables.  Not timed in solves (Sec. 3).
 *
 *   out      receives the new context (set to NULL on error).
 *   dim      2 (triangles) or 3 (tetrahedra).
 *   space    BRAS_H1, BRAS_HCURL or BRAS_HDIV;  order p or k (see above).
 *   coords   [n_vert * dim] double, vertex coordinates.
 *   cells    [n_cell * (dim+1)] int32, vertex ids of each simplex.
 *   l2g      [n_cell * n_loc] int32, local-to-global dof map (the map pi of Sec. 2.2).
 *   signs    [n_cell * n_loc] int8 in {+1, -1} (signed injection P), or NULL (all +1).
 *            Lagrange (H1) dofs have no orientation: for BRAS_H1 every sign must be +1
 *            (else BRAS_ERR_INVALID, the offending entry in bras_last_error_detail).
 *   rho      [n_cell] double > 0 element weights (mass density), or NULL (all 1).
 *   opt      options or NULL (defaults).
 * Limits: n_cell, n_dof < 2^31; n_cell * n_loc < 2^31.
 */
int bras_setup(bras_ctx** out, int dim, int space, int order,
               int64_t n_vert, const double* coords,
               int64_t n_cell, const int32_t* cells,
               int64_t n_dof, const int32_t* l2g, const int8_t* signs,
               const double* rho, const bras_options* opt, void* stream);

/* One mesh of a batch (all pointers host or device; same meaning as in bras_setup). */
typedef struct {
    int64_t n_vert;
    const double* coords;    /* [n_vert * dim]          */
    int64_t n_cell;
    const int32_t* cells;    /* [n_cell * (dim+1)]      */
    int64_t n_dof;
    const int32_t* l2g;      /* [n_cell * n_loc], dofs 0..n_dof-1 of this mesh */
    const int8_t* signs;     /* [n_cell * n_loc] or NULL */
    const double* rho;       /* [n_cell] or NULL          */
} bras_mesh_desc;

/*
 * bras_setup_batched -- one context for n_mesh independent meshes of the same space and
 * order (uneven sizes allowed).  The conforming systems stay independent: the context's
 * dof space is the concatenation of the meshes' dof spaces (mesh m owns the dofs
 * [off[m], off[m+1]) reported by bras_batch_offsets), every apply works on the whole
 * concatenation, and bras_pcg_solve with nrhs = 1 solves all meshes at once with
 * per-mesh CG scalars and per-mesh stopping tests (iters / relres then have n_mesh
 * entries).  Same limits as bras_setup on the totals.
 */
int bras_setup_batched(bras_ctx** out, int dim, int space, int order, int n_mesh,
                       const bras_mesh_desc* meshes, const bras_options* opt, void* stream);

/* Number of meshes of a context (1 unless batched) and, if dof_offsets is not NULL, the
 * n_mesh + 1 dof offsets (host array). */
int bras_batch_offsets(const bras_ctx* ctx, int* n_mesh, int64_t* dof_offsets);

/* Number of local dofs per cell for (dim, space, order, basis as in bras_options.basis), or
 * -1 if unsupported. */
int bras_n_local(int dim, int space, int order, int basis);

/* bras_mass_apply -- y = M x  (Eq. M_PMbrP, element by element).
 * x, y: [n_dof * nrhs] of double (BRAS_FP64) or float (BRAS_FP32 / BRAS_BF16); x and y
 * must not overlap.  nrhs >= 1. */
int bras_mass_apply(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs,
                    void* stream);

/* bras_apply -- y = M_bras^{-1} x = D^{-1} P^T M_br^{-1} P D^{-1} x  (Eq. mhatinvbras_def):
 * signed gather with D^{-1}, exact element-local inverse, multiplicity-weighted scatter.
 * Same argument rules as bras_mass_apply. */
int bras_apply(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs,
               void* stream);

/* bras_apply_noalloc -- the same y = M_bras^{-1} x as bras_apply, bit for bit (the paper has no
 * counterpart: this is a memory-management variant of this library), for callers that must
 * not have the library allocate device memory: code that owns all device memory through its
 * own pool or caching allocator, loops where the implicit synchronisation of cudaMalloc is not
 * acceptable, or a process with a device-memory budget fixed up front.  bras_apply may grow
 * its workspace on a call with a larger nrhs; this call never allocates or frees anything
 * (no cudaMalloc, no cudaFree, no allocating library routine).
 *   Scratch: the partial sums of cell-block boundary dofs go to one fixed 16 MiB array in
 *   device memory, part of the library image, which every GPU that loads the library keeps
 *   until the process exits.  A call whose partials (ctx's boundary partial count x nrhs x
 *   element size) exceed 16 MiB returns BRAS_ERR_TOO_LARGE (detail = bytes it would need)
 *   and launches nothing.
 *   The first call on a device looks the array's device address up (once per device, with
 *   that device current); make that first call before any stream capture on the device.
 *   All calls share the array and it keeps the last call's contents; nothing in it needs to
 *   start at zero.  Calls that may overlap on the GPU (on different streams, or different
 *   contexts at the same time) race on the array: order them on one stream.
 * Arguments, precisions and errors are those of bras_apply. */
int bras_apply_noalloc(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs,
                       void* stream);

/* bras_jacobi_apply -- y = diag(M)^{-1} x  (Sec. 2.1).  Same argument rules. */
int bras_jacobi_apply(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs,
                      void* stream);

/*
 * bras_pcg_solve -- solve M x = b by preconditioned CG (Sec. 3): u_0 = 0, stop when
 * ||r_k||_2 / ||r_0||_2 <= rtol for every right-hand side, or after maxit iterations.
 * On a batched context nrhs must be 1 and every mesh is its own system (iters and relres
 * have n_mesh entries).  A context's solve workspace serves one solve at a time.
 *   pc     BRAS_PC_NONE, BRAS_PC_JACOBI or BRAS_PC_BRAS.
 *   mode   BRAS_SOLVE_FP64: FP64 PCG, recurrence residual tested.
 *          BRAS_SOLVE_MIXED: FP32 (or BF16-inverse, if inner_precision = BRAS_BF16) inner
 *          PCG with FP64 dot products and scalars inside an FP64 refinement loop; the
 *          TRUE residual ||b - M x|| (FP64) is tested.
 *   inner_precision  BRAS_FP32 or BRAS_BF16 (mixed mode only; ignored in FP64 mode).
 *   b, x   [n_dof * nrhs] double; host OR device pointers (both on the same side).  With
 *          host pointers the copies in and out are part of the call.
 *   iters  [nrhs] int, host: CG iterations (mixed mode: total inner iterations).
 *   relres [nrhs] double, host: final ||r|| / ||b|| (recurrence residual in FP64 mode,
 *          true residual in mixed mode).
 * Returns BRAS_OK, BRAS_NOT_CONVERGED, or an error.  Synchronises `stream`.
 */
int bras_pcg_solve(const bras_ctx* ctx, int pc, int mode, int inner_precision,
                   const double* b, double* x, int nrhs, double rtol, int maxit,
                   int* iters, double* relres, void* stream);

/*
 * Stationary iterations (Sec. 3): linear in b, no inner products in the update, so they suit
 * settings where CG's global dot products cost (the stopping test still takes one norm per
 * iteration).  FP64 throughout; u_0 = 0; stop when ||r_k||_2 / ||r_0||_2 <= rtol (r_k the
 * recurrence residual) for every right-hand side, or after maxit iterations.  b, x, nrhs,
 * iters, relres, the batched-context rule and the return codes are those of bras_pcg_solve.
 * Scalar arrays (omega, lmin, lmax, lambda) are host arrays with one entry per right-hand
 * side (per mesh on a batched context).
 *
 * bras_lambda_max -- lambda_max(Mt^{-1} M) by the power iteration that the paper uses for
 * the fixed-point weights: v <- Mt^{-1} M v / ||.||_2, `iters` steps from v0, reporting the
 * Rayleigh quotient (M v, Mt^{-1} M v) / (M v, v) of the last step (a lower bound that
 * converges to lambda_max).  Mt = diag(M) for BRAS_PC_JACOBI, BRAS for BRAS_PC_BRAS.
 *   v0     [n_dof * nrhs] double, host or device, nonzero start vectors (not modified).
 *   lambda [nrhs] double, host (output).
 *
 * bras_fixed_point_solve -- damped fixed point u_{k+1} = u_k + omega Mt^{-1} (b - M u_k).
 * It converges for 0 < omega < 2 / lambda_max; the paper's weights are omega = 1 / lambda_max
 * (Jacobi) and omega = 2 / (1 + lambda_max) (BRAS, whose lambda_min >= 1, Sec. 2.3).
 *   omega  [nrhs] double > 0.
 *
 * bras_chebyshev_solve -- Chebyshev semi-iteration for the interval [lmin, lmax] that holds
 * the spectrum of Mt^{-1} M (for BRAS lmin = 1): with theta, delta the interval's centre and
 * half-width, d_k = c1_k d_{k-1} + c2_k Mt^{-1} r_k, u_{k+1} = u_k + d_k, r_{k+1} = r_k - M d_k,
 * where c1_0 = 0, c2_0 = 1/theta, rho_0 = delta/theta, rho_k = 1/(2 theta/delta - rho_{k-1}),
 * c1_k = rho_k rho_{k-1}, c2_k = 2 rho_k / delta.
 *   lmin, lmax  [nrhs] double, 0 < lmin < lmax.
 */
int bras_lambda_max(const bras_ctx* ctx, int pc, const double* v0, int nrhs, int iters, double* lambda,
                    void* stream);
int bras_fixed_point_solve(const bras_ctx* ctx, int pc, const double* omega, const double* b, double* x,
                           int nrhs, double rtol, int maxit, int* iters, double* relres, void* stream);
int bras_chebyshev_solve(const bras_ctx* ctx, int pc, const double* lmin, const double* lmax, const double* b,
                         double* x, int nrhs, double rtol, int maxit, int* iters, double* relres,
                         void* stream);

/*
 * bras_cg_lanczos -- estimates of lambda_min and lambda_max of Mt^{-1} M (Mt = diag(M) for
 * BRAS_PC_JACOBI, BRAS for BRAS_PC_BRAS, Mt = I for BRAS_PC_NONE), whose ratio is the spectral
 * condition number kappa_hat of Eq. spectral-kappa, on meshes too large for a dense
 * eigensolve: `steps` FP64 PCG iterations on M x = b (u_0 = 0, no stopping test) record their
 * coefficients alpha_k, beta_k, which define the tridiagonal matrix of the Lanczos process on
 * Mt^{-1} M (T[j][j] = 1/alpha_j + beta_j/alpha_{j-1}, T[j][j+1] = sqrt(beta_{j+1})/alpha_j);
 * its extreme eigenvalues (bisection on Sturm sequences) approach the extreme eigenvalues of
 * Mt^{-1} M from inside, lambda_max quickly, lambda_min more slowly.
 *   b          [n_dof] double, host or device, a start vector with components along the whole
 *              spectrum (e.g. N(0, 1) entries); one right-hand side; not on a batched context.
 *   steps      >= 1 iterations (fewer once ||r|| <= 1e-14 ||b||: beyond that the coefficients
 *              carry only rounding).
 *   lambda_min, lambda_max  host doubles (output); steps_done host int (output) or NULL.
 * Returns BRAS_OK, BRAS_ERR_BREAKDOWN, or an error.  Synchronises `stream`.
 */
int bras_cg_lanczos(const bras_ctx* ctx, int pc, const double* b, int steps, double* lambda_min,
                    double* lambda_max, int* steps_done, void* stream);

/*
 * bras_schur_apply -- y = -S~ x = B M_bras^{-1} B^T x, the BRAS approximation of the positive
 * Schur complement of the mixed Poisson saddle point [[M, B^T], [B, 0]] (Sec. 4,
 * Eq. approx_positive_schur_general with C = 0; Sec. 5.1), matrix-free: the divergence and its
 * transpose element by element, the BRAS apply in between.  Pair: RT_k or BDM_k (k = 1..4,
 * BDM with bras_options.basis = 1; the pair of Sec. 5.1) -- this context, H(div) on
 * tetrahedra -- with DG_{k-1}; B_ij = (div phi_j, chi_i), chi_i = chi^_i o F_K^{-1}, chi^_i the
 * polynomials of degree <= k - 1 orthonormal for the mean inner product on the reference
 * tetrahedron (Gram-Schmidt of the monomials by degree, then descending lexicographic
 * exponents), so cell K's block is sign(det J_K) B^.  (The spectrum of S~^{-1} S does not
 * depend on the DG basis.)
 *   x, y   [n_cell * n_q] of double (BRAS_FP64) or float (BRAS_FP32 / BRAS_BF16), cell K's
 *          n_q = k (k + 1) (k + 2) / 6 values at K * n_q, cells in the caller's order; one
 *          right-hand side; not on a batched context.
 * Returns BRAS_ERR_INVALID for other spaces.  The first call allocates its workspace
 * (8 bytes x (n_cell n_loc + 2 n_dof)).
 */
int bras_schur_apply(const bras_ctx* ctx, int precision, const void* x, void* y, void* stream);

/* bras_grad_rho -- rho_bar_K = -lambda_K^T M_K^1 x_K for the weighted mass M(rho) =
 * sum_K rho_K P_K^T M_K^1 P_K (M_K^1 = unit-density element matrix): the element part of
 * the adjoint gradient of x = M(rho)^{-1} b, with lambda = M^{-1} xbar (H1 only).
 * x, lam: [n_dof] double; rho_bar: [n_cell] double in the caller's cell order. */
int bras_grad_rho(const bras_ctx* ctx, const double* x, const double* lam, double* rho_bar,
                  void* stream);

/* bras_grad_log_rho -- the same element gradient with respect to log-densities: for rho_K =
 * exp(z_K) (the weights last set by bras_update_log_rho or bras_update_rho),
 * z_bar_K = rho_bar_K * rho_K = -rho_K lambda_K^T M_K^1 x_K, in one fused element kernel.
 * x, lam: [n_dof] double; z_bar: [n_cell] double in the caller's cell order (H1 only). */
int bras_grad_log_rho(const bras_ctx* ctx, const double* x, const double* lam, double* z_bar,
                      void* stream);

/* bras_update_rho -- replace the element weights (H1 only): rescales the per-element
 * factors and diag(M) without rebuilding the scatter tables.  rho: [n_cell] double > 0. */
int bras_update_rho(bras_ctx* ctx, const double* rho, void* stream);

/* bras_update_log_rho -- the same from log-densities: rho_K = exp(z_K), computed on the
 * device.  z: [n_cell] double, finite. */
int bras_update_log_rho(bras_ctx* ctx, const double* z, void* stream);

/* Sizes of a context: n_dof, n_cell, n_loc, number of scatter blocks. */
int bras_info(const bras_ctx* ctx, int64_t* n_dof, int64_t* n_cell, int* n_loc, int* n_blocks);

/* The cell block size in use and, after an autotuned setup, the sizes timed and their BRAS
 * apply times in microseconds (host arrays of at least 8 entries, or NULL; *count = 0 if the
 * setup was not tuned). */
int bras_block_tuning(const bras_ctx* ctx, int* block_elems, int* count, int* sizes, float* apply_us);

/* Bytes one apply moves by the algorithmic count: l2g map (4 B per local dof), the
 * per-element factor (H1) or packed local inverse (H(curl)/H(div)), x read and y written,
 * and one multiplicity byte per dof (BRAS apply only).  For roofline reporting. */
int64_t bras_algorithmic_bytes(const bras_ctx* ctx, int precision, int nrhs, int bras);

/* Device status of a context.  Every wait of the library's kernels on an mbarrier (a table
 * copy, a tensor-core GEMM) is bounded: it gives up after 0.5 s of the GPU's global timer,
 * lets the copies it issued land, releases its tensor memory, records a bit in the context's
 * status word (bit 0: a copy wait, bit 1: a GEMM or operand-tile wait) and leaves its outputs
 * unwritten.  The solvers (bras_pcg_solve, bras_fixed_point_solve, bras_chebyshev_solve,
 * bras_lambda_max, bras_cg_lanczos) read the word when they finish and return
 * BRAS_ERR_DEVICE (detail = the bits, the word cleared) if any bit is set; the stream-ordered
 * applies leave it to this call: it synchronises `stream`, returns BRAS_OK if the word is 0,
 * else BRAS_ERR_DEVICE with the bits as detail, and clears the word if `clear` != 0. */
int bras_device_status(bras_ctx* ctx, void* stream, int clear);

/* Self-test of the bounded wait: one CTA waits on an mbarrier that nothing completes, on the
 * legacy default stream, until the bound runs out.  *bits = the status bits it recorded
 * (1 expected), *elapsed_ms = the wait's duration by CUDA events (about 500 expected).  The
 * CUDA context stays usable.  Returns BRAS_OK, or BRAS_ERR_CUDA / BRAS_ERR_OOM. */
int bras_wait_selftest(int* bits, double* elapsed_ms);

void bras_destroy(bras_ctx* ctx);
const char* bras_status_string(int code);
int64_t bras_last_error_detail(void);

/* Number of CUDA kernels this library has launched since it was loaded (all contexts, all
 * threads); a host-side counter for launch accounting. */
int64_t bras_kernel_launches(void);

/* Number of CUDA graph launches this library has made since it was loaded (one per solve
 * that runs as a graph: bras_pcg_solve in either mode, the stationary solvers); the kernels
 * such a graph runs are counted by bras_kernel_launches. */
int64_t bras_graph_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* BRAS_H */
