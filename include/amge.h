/* libamge -- C ABI of the GB300 (sm_103a) AMGe solve path.
 *
 * Kalchev, Vassilevski, Villa, "Parallel Element-based Algebraic Multigrid for
 * H(curl) and H(div) Problems Using the ParELAG Library" (arXiv 2107.05613).
 * The library runs the solve phase of the paper's method on one GPU: conjugate
 * gradients preconditioned by one AMGe V-cycle (Algorithm 4.1, Section 4) per
 * iteration, with the hybrid smoother of eq. 4.1 (an l1-Jacobi sweep on A_l, then
 * an l1-Jacobi sweep on the auxiliary matrix G^T A_l G reached through the exterior
 * derivative G, corrected back through G) on every level and a dense direct solve
 * on the coarsest level.  The hierarchy itself (Sections 2-3: prolongators P_l,
 * coarse exterior derivatives, Galerkin A_l) is built on the host in FP64 from the
 * problem's coefficients (amge_setup_upload) or handed over as plain CSR arrays
 * (amge_upload_levels) or as a serialized blob (amge_upload_blob).
 *
 * Conventions
 *   - Every pointer argument documented as "device" must point to memory the
 *     calling context's current CUDA device can access; "host" pointers are
 *     ordinary CPU memory.  Sizes are element counts unless stated otherwise.
 *   - Levels are numbered from 0 (finest); the paper numbers them from 1.
 *   - Coefficient lettering: beta multiplies (Du, Dv), alpha multiplies (u, v)
 *     (eq. 2.2 of the paper letters them the other way round).
 *   - Multi-RHS vectors are row-major [n][nrhs] (right-hand sides contiguous).
 *   - All work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t
 *     passed as void*; NULL = the legacy default stream).  Functions that must read
 *     a scalar back (PCG convergence tests) synchronise that stream.
 *   - Errors are reported through the return code only; amge_last_error() returns
 *     a thread-local message describing the last failure.  No call traps or
 *     asserts on the device.
 */
#ifndef AMGE_H
#define AMGE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMGE_OK = 0,
  AMGE_EINVAL = 1,      /* invalid argument or malformed hierarchy */
  AMGE_ENOMEM = 2,      /* device allocation failed */
  AMGE_ECUDA = 3,       /* a CUDA runtime call failed */
  AMGE_ENOTCONV = 4,    /* PCG stopped at maxit; info holds the partial result */
  AMGE_ENONFINITE = 5,  /* a right-hand side or a PCG scalar is not finite */
  AMGE_EAGAIN = 6,
  AMGE_ETIMEOUT = 7,
  AMGE_ECANCELED = 8
} amge_status;

/* The problem's space, numbered by the exterior derivative that defines its
 * bilinear form: D_2 = curl (H(curl), Nedelec edge dofs, aux space H1 reached
 * through the discrete gradient) and D_3 = div (H(div), Raviart-Thomas face dofs,
 * aux space H(curl) reached through the discrete curl), Section 2 of the paper. */
typedef enum { AMGE_HCURL = 2, AMGE_HDIV = 3 } amge_form;

/* AMGE_FP64: every step in double precision.
 * AMGE_FP32_VCYCLE: the V-cycle's vectors are single precision, and so are its
 * prolongators, incidences, smoother data and the level products with single-
 * precision accumulation, except the residuals b - A_l x of iterates that carry a
 * correction through G or P: those use A_l's values to about 48 bits and sum to
 * about that precision (double-float pairs on the FP32 pipe by default, or FP64
 * values and sums, see amge_set_wide_arith), rounded once to single, because on
 * such iterates most of A_l x cancels and single-precision rounding would swamp the
 * residual's gradient (curl) part that the aux sweep and the coarse solve divide by
 * small mass-only diagonals.  The coarsest-level solve runs in the same ~48-bit
 * arithmetic (rounded to single); the outer PCG dot products, AXPYs and the
 * true-residual recomputation stay in double precision. */
typedef enum { AMGE_FP64 = 0, AMGE_FP32_VCYCLE = 1 } amge_precision;

/* A CSR matrix in host memory: row_ptr[n_rows+1], col[nnz] (0-based, each row's
 * columns strictly increasing), val[nnz]. */
typedef struct {
  int32_t n_rows;
  int32_t n_cols;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
} amge_csr;

/* A generated hierarchy (host memory, copied during amge_upload_levels).
 *   form        AMGE_HCURL (edge dofs; G_l = discrete gradient D_0 at level l) or
 *               AMGE_HDIV (face dofs; G_l = discrete curl D_1 at level l)
 *   num_levels  >= 1
 *   A[l]        problem matrix of level l (SPD), l = 0 .. num_levels-1
 *   P[l]        prolongator, level l+1 -> level l (n_l x n_{l+1}), l < num_levels-1
 *   G[l]        aux transition into level l's space (n_l x aux_l), l < num_levels-1
 *   nu_pre, nu_post  hybrid smoothing steps before / after the coarse correction (>= 1) */
typedef struct {
  int32_t form;
  int32_t num_levels;
  const amge_csr* A;
  const amge_csr* P;
  const amge_csr* G;
  int32_t nu_pre;
  int32_t nu_post;
} amge_hierarchy_desc;

typedef struct amge_hier amge_hier; /* opaque, device-resident hierarchy */

/* The problem the paper states (eq. 2.2, Section 5.1 setting), on the unit cube
 * split into n^3 cubes, each cut into the 6 Kuhn tetrahedra along its
 * (0,0,0)-(1,1,1) diagonal, lowest-order Whitney elements, natural boundary
 * conditions (every edge / face is a dof):
 *   H(curl): a(u, v) = (beta curl u, curl v) + (alpha u, v)
 *   H(div):  a(u, v) = (beta div u, div v) + (alpha u, v)
 *   form        AMGE_HCURL or AMGE_HDIV
 *   n           cubes per side, 1 .. 256
 *   num_levels  levels of the AMGe hierarchy, 1 .. 16, or 0 = agglomerate 2x2x2
 *               cells while the cell grid side m is even and > 8 (so n = 64 gives
 *               4 levels: 64^3 -> 32^3 -> 16^3 -> 8^3 cells)
 *   beta        host double [6 n^3], coefficient of the derivative term per
 *               tetrahedron (the paper's alpha), > 0 and finite; NULL = all ones
 *   alpha       host double [6 n^3], coefficient of the mass term (the paper's
 *               beta), > 0 and finite; NULL = all ones
 *   nu_pre, nu_post  hybrid smoothing steps before / after the coarse correction,
 *               1 .. 8
 *   flags       0, or AMGE_SETUP_TARGETS: the last coarsening's coarse space also
 *               takes the polynomial approximation targets (Sections 3.3.1-3.3.3: the
 *               interpolants of the vector monomials of degree <= 1 -- their traces on
 *               coarse edges / faces orthogonal to the PV traces, and their mass
 *               projections onto the D-free bubbles of coarse faces and cells --
 *               filtered of linear dependence, extended by eqs. 3.6 / 3.8, as extra
 *               columns of P after the coarse entities' ones); the coarsest space then
 *               reproduces every linear field, and the coarsest matrix is the Galerkin
 *               product P^T A P.  AMGE_SETUP_TARGETS2: the same with the monomials
 *               of degree <= 2 and the cross-space bubbles of eqs. 3.7 / 3.9; the
 *               coarsest space then reproduces every quadratic field.  Other bits:
 *               AMGE_EINVAL.
 * Tetrahedron t = 6 ((i n + j) n + k) + p lies in cube (i, j, k) (i, j, k the x, y, z
 * cube indices), p = 0 .. 5 the Kuhn permutation index in the order
 * (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x) of the monotone path from the
 * cube's (0,0,0) corner to its (1,1,1) corner. */
typedef struct {
  int32_t form;
  int32_t n;
  int32_t num_levels;
  const double* beta;
  const double* alpha;
  int32_t nu_pre;
  int32_t nu_post;
  int32_t flags;
} amge_problem;
#define AMGE_SETUP_TARGETS 1
#define AMGE_SETUP_TARGETS2 2

/* Options of a PCG solve.  rtol: stop when the true FP64 relative residual
 * ||b - A x||_2 / ||b||_2 <= rtol (x0 = 0); maxit >= 1; precision: amge_precision. */
typedef struct {
  double rtol;
  int32_t maxit;
  int32_t precision;
} amge_solve_opts;

/* Result of one right-hand side: iterations (number of products A p), status
 * (AMGE_OK, AMGE_ENOTCONV or AMGE_ENONFINITE), the true relative residual
 * recomputed in FP64 at exit, and the wall time of the whole solve call. */
typedef struct {
  int32_t iters;
  int32_t status;
  double true_relres;
  double time_ms;
} amge_info;

/* Build the problem's AMGe hierarchy on the host and upload it to the current
 * device (Sections 2-3 of the paper, then the preparation of amge_upload_levels).
 * The host FP64 setup forms the fine Whitney-form operator, agglomerates 2x2x2
 * cells per level, builds the coarse topology (Section 3.1), the PV traces
 * (eq. 3.5) and their local extensions (eqs. 3.6, 3.8) into the prolongators P_l,
 * the integer coarse exterior derivatives, and the Galerkin operators
 * A_{l+1} = P_l^T A_l P_l (Section 3.2.1), then hands them to amge_upload_levels.
 * Host memory of the setup is released before return; the caller's arrays are
 * only read.
 * Errors: AMGE_EINVAL for a NULL problem or out, a form, n, level count or
 * smoothing count out of range, a coefficient that is not positive and finite, or
 * a setup failure; AMGE_ECUDA if no CUDA device is current (checked first);
 * otherwise as amge_upload_levels.  On error *out is NULL. */
amge_status amge_setup_upload(const amge_problem* problem, void* stream, amge_hier** out);

/* New coefficients for a hierarchy made by amge_setup_upload, re-set up on the GPU.
 * The prolongators P_l and exterior derivatives G_l do not depend on the coefficients
 * (the local extensions of eqs. 3.6/3.8 use unweighted masses), so only the Galerkin
 * operators change: A_0 is re-assembled on the device from the per-tetrahedron beta
 * and alpha (host double [6 n^3] each as in amge_problem, NULL = ones), then
 * A_{l+1} = P_l^T A_l P_l (Section 3.2.1), the l1 diagonals of A_l and of
 * G_l^T A_l G_l, the stored A_l G_l, the FP32 copies and the sliced-ELL values are
 * recomputed on the device, and the coarsest Cholesky factor and inverse on the host
 * from the new A_L.  Kernel choices and captured graphs are kept; Gauss-Seidel data
 * (amge_set_smoother) are rebuilt; an auxiliary-space coarsest solver
 * (amge_set_coarse_solver) is dropped for the dense solve, to be set again.  Synchronises `stream`; no solve on h or on a
 * server slot of h may be in flight.  Results equal a fresh amge_setup_upload with
 * these coefficients up to the summation order of the products.
 * Errors: AMGE_EINVAL for NULL h, a hierarchy not made by amge_setup_upload (or with
 * fewer than two levels), a view, or a coefficient that is not positive and finite;
 * AMGE_EINVAL if the new coarsest matrix is not SPD; AMGE_ECUDA. */
amge_status amge_update_coefficients(amge_hier* h, const double* beta, const double* alpha, void* stream);

/* Upload a hierarchy serialized in the blob format below (the same bytes the CPU
 * oracle reads).  The blob is only read; it may be freed after return.  Little-
 * endian, every section starting at a multiple of 8 bytes from the blob's start:
 *   header, 32 bytes: char magic[8] = "AMGEBLOB"; uint32 version = 1; int32 form
 *     (amge_form); int32 num_levels L (1 .. 16); int32 nu_pre; int32 nu_post;
 *     int32 reserved = 0
 *   then 3L - 2 matrices in the order A_0 .. A_{L-1}, P_0 .. P_{L-2}, G_0 .. G_{L-2}
 *   (meanings as in amge_hierarchy_desc), each as
 *     int32 n_rows; int32 n_cols; int64 nnz;
 *     int32 row_ptr[n_rows + 1], zero-padded to a multiple of 8 bytes;
 *     int32 col[nnz], zero-padded to a multiple of 8 bytes;
 *     double val[nnz]
 *   and nothing after the last matrix (`bytes` must equal the layout's size).
 * Errors: AMGE_EINVAL for a NULL argument or a blob that does not follow the layout
 * (checked before any device work); otherwise as amge_upload_levels. */
amge_status amge_upload_blob(const void* blob, size_t bytes, void* stream, amge_hier** out);

/* Upload a generated hierarchy to the current device and prepare the solve data.
 * The host setup run here derives, in FP64, the l1-Jacobi diagonals m_l = sum_j
 * |(A_l)_ij| (Section 4.1 point smoother), the auxiliary diagonals m_aux,l = row
 * l1 sums of G_l^T A_l G_l (eq. 4.1, second line), the transposes P_l^T and G_l^T,
 * FP32 copies of every level operator, and the Cholesky factor of the dense
 * coarsest matrix together with its triangular inverse (the coarsest solve that
 * replaces the paper's AMS/ADS, Section 4.2).  Stored zeros of the input operators
 * are dropped.  For H(curl) with one pre- and one post-smoothing step it also forms
 * A_l G_l where that product is much sparser than A_l, dropping its cancellation
 * residue (entries at most 64 eps times the sum of their terms' magnitudes), and
 * times every candidate kernel of every operator (amge_autotune_report), for which
 * it allocates twice the GPU's L2 capacity for the duration of the call.  The
 * library owns the device memory until amge_hier_free.
 * Errors: AMGE_EINVAL for malformed CSR data, mismatched sizes, a coarsest matrix
 * that is not SPD, or a level too large for 32-bit indices; AMGE_ENOMEM;
 * AMGE_ECUDA.  On error *out is NULL. */
amge_status amge_upload_levels(const amge_hierarchy_desc* desc, void* stream, amge_hier** out);

/* Size of the finest level, number of levels and device bytes held. */
amge_status amge_hier_info(const amge_hier* h, int32_t* n_dofs, int32_t* levels, size_t* device_bytes);

/* One V-cycle (Algorithm 4.1 with x0 = 0, hybrid smoothing eq. 4.1, the
 * transposed smoother after the coarse correction): z = B^{-1} r.
 *   r_dev, z_dev  device, double [n][nrhs]; must not overlap
 *   nrhs          number of right-hand sides, 1 .. 32 (columns of a row-major block)
 *   precision     amge_precision of the internal arithmetic (the interface stays FP64)
 * Enqueued on `stream`; does not synchronise (the first call with nrhs > 1 allocates
 * the block workspace). */
amge_status amge_vcycle(amge_hier* h, const double* r_dev, double* z_dev, int32_t nrhs, int32_t precision,
                        void* stream);

/* PCG preconditioned by one V-cycle per iteration (Section 4), x0 = 0.
 *   b_dev, x_dev  device, double [n][nrhs]; x_dev is overwritten; 1 <= nrhs <= 32
 *   info          host, array of nrhs results
 * With nrhs > 1 the columns iterate together (one block V-cycle per iteration, one
 * read of every operator for all columns); a column stops moving once its true
 * residual meets the tolerance.  The first call with nrhs > 1 on a hierarchy
 * allocates the block workspace (sized for 32 columns) on the device.
 * Returns AMGE_OK when every right-hand side converged, AMGE_ENOTCONV when one
 * reached maxit (its info entry holds the iterations and the final true residual),
 * AMGE_ENONFINITE when a right-hand side or a PCG scalar is not finite.
 * Synchronises `stream` once per iteration to test convergence. */
amge_status amge_pcg_solve(amge_hier* h, const double* b_dev, double* x_dev, int32_t nrhs,
                           const amge_solve_opts* opts, amge_info* info, void* stream);

/* Same as amge_pcg_solve with host buffers: copies b_host (double [n][nrhs]) to
 * the device, solves, and copies the solution back into x_host before returning.
 * The device staging belongs to the hierarchy. */
amge_status amge_pcg_solve_host(amge_hier* h, const double* b_host, double* x_host, int32_t nrhs,
                                const amge_solve_opts* opts, amge_info* info, void* stream);

/* Single steps of the V-cycle, for step-by-step parity checks.  `level` selects
 * the level; x_dev / y_dev are device double vectors of the operator's column /
 * row count; `precision` selects the stored operator copy (FP32 mode converts
 * inputs and outputs through double).
 *   op AMGE_OP_A:  y = A_l x          AMGE_OP_P:  y = P_l x     AMGE_OP_PT: y = P_l^T x
 *      AMGE_OP_G:  y = G_l x          AMGE_OP_GT: y = G_l^T x
 *      AMGE_OP_SMOOTH_PRE:  y = one hybrid step (eq. 4.1) from x0 = 0 on b = x
 *      AMGE_OP_COARSE:      y = A_L^{-1} x on the coarsest level (level ignored)
 *      AMGE_OP_AG: y = (A_l G_l) x, where that product is stored (see
 *                  amge_autotune_report; AMGE_EINVAL elsewhere)
 *      AMGE_OP_A_WIDE (AMGE_FP32_VCYCLE only): y = A_l x with x rounded to FP32,
 *                  FP64 values and FP64 sums, the result rounded to FP32 -- the
 *                  product the FP32 V-cycle uses for residuals of iterates that
 *                  carry a correction through G or P (amge_vcycle)
 * Products run the kernel chosen for the operator (amge_autotune_report,
 * amge_set_kernel). */
enum {
  AMGE_OP_A = 0,
  AMGE_OP_P = 1,
  AMGE_OP_PT = 2,
  AMGE_OP_G = 3,
  AMGE_OP_GT = 4,
  AMGE_OP_SMOOTH_PRE = 5,
  AMGE_OP_COARSE = 6,
  AMGE_OP_AG = 7,
  AMGE_OP_A_WIDE = 8
};
amge_status amge_apply(amge_hier* h, int32_t op, int32_t level, const double* x_dev, double* y_dev,
                       int32_t precision, void* stream);

/* Deterministic FP64 dot product: *result_dev = sum_i x[i] y[i], reduced in a
 * fixed order independent of the launch (block partials in index order).
 *   x_dev, y_dev  device double [n];  result_dev  device double [1]
 * Uses the hierarchy's reduction scratch; calls on one hierarchy are stream-ordered. */
amge_status amge_dot(amge_hier* h, const double* x_dev, const double* y_dev, int64_t n, double* result_dev,
                     void* stream);

/* Hybrid-smoother choice (eq. 4.1 with either point smoother; Section 4.1):
 *   AMGE_SMOOTHER_L1_JACOBI  the default: one l1-Jacobi sweep, m_i = sum_j |a_ij|,
 *                            for the primary and for the auxiliary smoothing
 *   AMGE_SMOOTHER_SYM_GS     the smoother of the paper's runs (Section 5.1): `sweeps`
 *                            symmetric Gauss-Seidel steps (a forward then a backward
 *                            pass) for the primary and for the auxiliary smoothing,
 *                            on the gs_levels finest smoothing levels (l1-Jacobi on the
 *                            coarser ones); rows are visited in a multicolour order --
 *                            a greedy colouring of the pattern of A_l (of the symbolic
 *                            pattern of G^T A_l G for the aux matrix) in row order,
 *                            rows sorted by colour, one launch per colour.  The l1 term
 *                            of the paper's l1-scaled block variant couples a row to
 *                            rows outside its processor block and vanishes on one GPU.
 * The first selection of Gauss-Seidel on a level builds its data (a host pass over the
 * level's operators, the explicit G^T A_l G, device allocation) and synchronises; it
 * is kept for later selections.  Gauss-Seidel V-cycles run in FP64 on single vectors:
 * AMGE_FP32_VCYCLE solves and blocks of right-hand sides then fail with AMGE_EINVAL.
 * Errors: AMGE_EINVAL for an unknown smoother, sweeps outside [1, 8], gs_levels < 0,
 * or a workspace view; AMGE_ENOMEM, AMGE_ECUDA. */
enum { AMGE_SMOOTHER_L1_JACOBI = 0, AMGE_SMOOTHER_SYM_GS = 1 };
amge_status amge_set_smoother(amge_hier* h, int32_t smoother, int32_t sweeps, int32_t gs_levels);

/* Arithmetic of the FP32 V-cycle's residuals of corrected iterates (and of
 * AMGE_OP_A_WIDE):
 *   AMGE_WIDE_DF    the default: each value of A_l as the float pair hi + lo
 *                   (hi = fl32(a), lo = fl32(a - hi): 48 significant bits), each
 *                   product hi x formed exactly as a float pair (product and FMA
 *                   remainder), lo x added to the remainder, the row's sum kept as a
 *                   float pair (two-sum of the high parts); all on the FP32 pipe.
 *                   Error: a few multiples of 2^-48 |A_l| |x| per stored entry.
 *   AMGE_WIDE_FP64  FP64 values and an FP64 FMA chain per row on the FP32 vectors
 *                   widened exactly (error of FP64 recursive summation).
 * Both read 8 value bytes per entry (the double-float pairs are a resident copy of
 * A_l beside the FP64 and FP32 ones) and round the result once to single.  The same
 * switch selects the arithmetic of the FP32 V-cycle's coarsest solve z = A_L^{-1} b
 * (the explicit inverse as double-float pairs with pair sums, or in FP64 with the
 * input widened first); its result is rounded to single either way.  On GB300
 * the FP64 form is co-limited by the FP64 FMA rate (one FMA per entry), the
 * double-float form by HBM.  Captured PCG graphs of h are rebuilt on the next
 * solve.  AMGE_EINVAL for another value or a NULL h. */
enum { AMGE_WIDE_FP64 = 0, AMGE_WIDE_DF = 1 };
amge_status amge_set_wide_arith(amge_hier* h, int32_t arith);

/* Per-kernel launch counts and timing.  Every kernel launch of the solve path is
 * counted per kernel class; while timing is enabled each launch is also bracketed
 * by CUDA events on its stream.  amge_profile_read synchronises, and returns for
 * each kernel class c (0 <= c < AMGE_PROF_CLASSES) the number of kernel launches count[c]
 * and their summed device time ms[c] (0 for launches made while timing was off)
 * since the last read, then resets both.  Class ids: see AMGE_PROF_* below. */
enum {
  AMGE_PROF_A_FINE = 0,    /* level-0 A sweeps of the V-cycle (residuals, the final l1 sweep) */
  AMGE_PROF_A_COARSE = 1,  /* A sweeps on levels >= 1 */
  AMGE_PROF_GT = 2,
  AMGE_PROF_G = 3,
  AMGE_PROF_PT = 4,
  AMGE_PROF_P = 5,
  AMGE_PROF_COARSE = 6,    /* coarsest triangular solves */
  AMGE_PROF_PCG_SPMV = 7,  /* q = A p with p.q */
  AMGE_PROF_PCG_VEC = 8,   /* PCG vector updates, dots, casts */
  AMGE_PROF_VCYCLE_VEC = 9, /* V-cycle elementwise products (x = m^-1 b on entry to a level) */
  AMGE_PROF_AG = 10,        /* residual updates r -= (A G) y after an aux sweep (H(curl)) */
  AMGE_PROF_A_WIDE = 11,    /* FP32 V-cycle, level 0: products on the FP64 operator (AMGE_OP_A_WIDE) */
  AMGE_PROF_GS = 12,        /* Gauss-Seidel colour sweeps (amge_set_smoother) */
  AMGE_PROF_CLASSES = 13
};
amge_status amge_profile_enable(amge_hier* h, int32_t enable);
amge_status amge_profile_read(amge_hier* h, int64_t* count, double* ms);

/* FP64 FMA issue rate of the current device in TFMA/s (*tfma, host): a kernel of
 * independent FMA chains filling every SM, best of five timed launches on `stream`
 * (synchronised).  The second roofline of the FP64 sparse products, which issue one
 * FMA per stored 12-byte entry.  Errors: AMGE_EINVAL for NULL, AMGE_ECUDA. */
amge_status amge_fp64_fma_rate(double* tfma, void* stream);

/* FP64 tensor-core rate of the current device in TFLOP/s (*tflops, host): independent
 * mma.sync m8n8k4 FP64 tiles (512 FLOP each, operands in registers) in every warp of a
 * grid filling every SM, best of five timed launches on `stream` (synchronised).  The
 * ceiling of an FP64 GEMM on the tensor cores (the coarsest solve of a block of
 * right-hand sides); compare 2 x amge_fp64_fma_rate for the CUDA cores.
 * Errors: AMGE_EINVAL for NULL, AMGE_ECUDA. */
amge_status amge_fp64_mma_rate(double* tflops, void* stream);

/* Coarsest-level solve z = A_L^{-1} b without any device allocation.
 * The paper has no counterpart.  It serves callers that may not have the library
 * allocate device memory while they solve (a latency-critical loop that must not
 * take the device-wide synchronisation of cudaMalloc, or a host framework that
 * owns every device byte through its own pool): they upload the hierarchy once,
 * then pass only their own input and output vectors here.  It computes the same
 * products as amge_apply(h, AMGE_OP_COARSE, ...) in FP64, but keeps the
 * intermediate vector in a fixed file-scope device array of 4096 doubles (32 KiB,
 * held by every GPU that loads the library until the process exits).
 *   h             hierarchy uploaded on the current device
 *   b_dev, z_dev  device double [n_L] (n_L = coarsest dofs); must not overlap
 * Errors: AMGE_EINVAL for NULL arguments, a coarsest level larger than 4096 dofs,
 * or a hierarchy uploaded on another device than the current one; AMGE_ECUDA if the
 * device address of the array cannot be obtained.
 * The first call on each device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every call
 * shares the one array, so calls whose kernels overlap on the GPU (different
 * streams, no ordering between them) race on it; the array needs no clearing
 * (each call overwrites it before reading it).  Enqueued on `stream`. */
amge_status amge_coarse_solve_noalloc(const amge_hier* h, const double* b_dev, double* z_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Request server (continuous batching of solves on one GPU).
 *
 * A server owns one scheduler thread that does all of its GPU work on the device
 * that was current at creation.  amge_submit copies the right-hand sides and returns
 * a ticket at once; every right-hand side becomes a column solve that runs in a slot
 * -- a workspace of its own (vectors, Krylov state, reduction scratch, captured PCG
 * graph) over the submitted hierarchy's read-only operators, with its own stream.
 * Queued columns are admitted as soon as an idle slot of the same hierarchy exists or
 * a new slot fits the HBM budget (idle slots of other hierarchies are released
 * first, least recently used), and every running column is advanced without
 * blocking, so work of requests that arrive while others run overlaps on the device.
 * Each column gives exactly the result amge_pcg_solve gives for that right-hand side
 * on that hierarchy, whatever else is running.  Hierarchies must outlive the server.
 * ------------------------------------------------------------------------- */
typedef struct amge_server amge_server; /* opaque */

/* hbm_budget_bytes: device bytes the slots may hold (0 = 80% of the free memory at
 * creation); max_slots: concurrent column solves, 1 .. 4096. */
amge_status amge_server_create(size_t hbm_budget_bytes, int32_t max_slots, amge_server** out);

/* Queue a solve of nrhs (1 .. 32) right-hand sides b_host [n][nrhs] (copied before
 * return) on hierarchy h; the solution is written to x_host [n][nrhs], which must stay
 * valid until amge_poll / amge_wait has returned the final status.  Never blocks on
 * the GPU.  *ticket identifies the request. */
amge_status amge_submit(amge_server* s, amge_hier* h, const double* b_host, double* x_host, int32_t nrhs,
                        const amge_solve_opts* opts, uint64_t* ticket);

/* AMGE_EAGAIN while the request is pending.  Otherwise its final status (AMGE_OK,
 * AMGE_ENOTCONV, AMGE_ENONFINITE, AMGE_ECANCELED, AMGE_ENOMEM when its workspace can
 * never fit the budget, AMGE_ECUDA), with info[0 .. nrhs-1] filled (time_ms = time
 * from submission to completion); the ticket is then released. */
amge_status amge_poll(amge_server* s, uint64_t ticket, amge_info* info);

/* As amge_poll, waiting up to timeout_ms (< 0: no limit); AMGE_ETIMEOUT if the
 * request is still pending then (the ticket stays valid). */
amge_status amge_wait(amge_server* s, uint64_t ticket, int32_t timeout_ms, amge_info* info);

/* Cancel a pending request: columns not yet started are dropped, running ones finish;
 * the final status is AMGE_ECANCELED.  AMGE_EINVAL for an unknown or finished ticket. */
amge_status amge_cancel(amge_server* s, uint64_t ticket);

/* Queue depth (requests with columns not yet started), running column solves,
 * device bytes held by slots, number of slots. */
amge_status amge_server_stats(amge_server* s, int64_t* queued, int64_t* running_columns, size_t* bytes_in_use,
                              int32_t* slots);

/* Stop the scheduler (running columns are waited for, pending requests dropped) and
 * release every slot (NULL is ignored). */
void amge_server_destroy(amge_server* s);

/* Choose how single-right-hand-side PCG iterations are launched (default 1).
 * 1: the iteration is captured once per precision into a CUDA graph whose WHILE
 *    conditional node repeats it on the device until the recursive residual meets
 *    the tolerance or maxit is reached (one host round trip per graph launch);
 * 0: every kernel is launched from the host and the residual norm is read back
 *    after each iteration.
 * Both run the same kernels in the same order and give identical results.  While
 * per-launch timing is enabled (amge_profile_enable), the host-launched loop is used. */
amge_status amge_set_graphs(amge_hier* h, int32_t enable);

/* Process-wide: launch kernels with programmatic dependent launch (default 1), so a
 * kernel's blocks are scheduled while its predecessor in the stream finishes and
 * wait on the device for its results; 0 launches them plainly.  Results are
 * identical either way.  Applies to launches issued, and PCG graphs captured, after
 * the call (call amge_set_kernel or re-upload to recapture an existing graph). */
void amge_set_dependent_launch(int32_t enable);

/* Wait status of h's kernels with bounded waits (the bulk-staged product, kernel code
 * 3000): synchronizes `stream`, then *timed_out = 1 if such a kernel's wait for its
 * staged copy ran out (about one second) since the previous call, else 0, and clears
 * the flag.  A kernel that timed out stops early, so the results of the calls on h
 * since the previous check are then not valid; the CUDA context stays usable.
 * AMGE_EINVAL for NULL arguments, AMGE_ECUDA if the copy or the synchronization fails. */
amge_status amge_wait_status(amge_hier* h, void* stream, int32_t* timed_out);

/* The autotuner's kernel choice for every smoothing level's single-vector products:
 * lanes[(l * 2 + p) * 6 + op] for level l < levels-1, precision p (0 FP64, 1 FP32),
 * op 0..5 = A, P, P^T, G, G^T, AG; 0 = sliced ELL (one row per lane, one warp per
 * 32-row slice), 100 w (200, 400, 800) = sliced ELL with w warps sharing each slice,
 * 1000 / 1200 = sliced ELL with one / two warps per slice where each warp first issues
 * a bulk L2 prefetch of its slice's entries (candidates only for streamed operators,
 * those larger than half of L2; the others always prefetch), 3000 = sliced ELL with one
 * warp per slice whose entries are staged into shared memory by bulk asynchronous
 * copies two slices ahead (candidate only for streamed operators with stored values;
 * its waits are bounded, see amge_wait_status), 1600 = sliced ELL with one warp per
 * slice whose column indices are 16-bit offsets from the slice's smallest column
 * (candidate where every slice spans fewer than 65,536 columns and the values are
 * stored; 6 bytes per FP32 entry instead of 8; the FP32 V-cycle's double-float
 * residuals use the same columns where the FP32 A_l product does, and the fused aux
 * correction where the A G product does), 1700 = the same with each slice's entries
 * prefetched into L2 first (streamed operators), 1800 / 1900 = 1600 / 1700 with two warps
 * per slice, 2000 = one warp per slice on a grid of the resident capacity, each warp
 * walking many slices and loading the next one's entries while it gathers for the
 * current one (short-row operators),
 * 2..32 = vector CSR with that many lanes per row, -1 = operator not used (AG is stored only where
 * A G = A_l G_l is much sparser than A_l, i.e. for H(curl): there the residual after
 * an aux sweep is updated as r - (A G) y instead of recomputed as b - A x).  The
 * choice is made at upload by timing each candidate on the level's own operator
 * (see amge_autotune_times for how): the fastest sliced-ELL kernel, unless a vector
 * CSR kernel is at least 10% faster.
 * lanes must hold (levels-1)*12 entries. */
amge_status amge_autotune_report(const amge_hier* h, int32_t* lanes);

/* The autotuner's evidence: us[((l * 2 + p) * 6 + op) * 17 + c] = measured time per
 * launch in microseconds (STORE epilogue, ten launches replayed from a graph).  Where
 * a level's operators and the coarser ones take more than half of L2, so that a
 * V-cycle finds them evicted, each launch follows a read of twice L2's capacity and is
 * timed by its own pair of event records (best of five replays): the operator comes
 * from HBM as it does inside a V-cycle.  Otherwise, and for streamed operators larger
 * than L2, the ten launches run back to back and are timed as a whole (best of
 * three) -- also where the 2x L2 scratch cannot be allocated.  Candidate c in the order 0,
 * 200, 400, 800, 2, 4, 8, 16, 32, 1000, 1200, 3000, 1600, 1700, 1800, 1900, 2000; -1 where
 * a candidate was not measured (more warps than the operator's rows have entry pairs, a
 * prefetch or staging variant of an operator that is not streamed, 16-bit columns not
 * built) or the operator is not stored.  us must hold (levels-1)*204 floats. */
amge_status amge_autotune_times(const amge_hier* h, float* us);

/* Override one entry of that choice (level l < levels-1, precision 0/1, op 0..5 as
 * above; lanes = a kernel code as above: 0, 200, 400, 800, 1000, 1200, 1600, 1700, 1800,
 * 1900, 2000, 3000 or 2, 4, 8, 16, 32; the prefetch codes act as 0 / 200 / 1600 / 1800 on
 * operators that are not streamed, 3000 as 0 on sign-coded operators and on those whose
 * longest slice does not fit the stages, 1600 / 1700 / 1800 / 1900 as 0 / 1000 / 200 /
 * 1200 where the 16-bit columns are not built).  Captured PCG graphs
 * of h are rebuilt on the next solve.  Every kernel computes the same products (in a
 * different summation order), so a choice changes rounding, not results beyond it;
 * pinning the choices makes results reproducible across uploads.  Not to be called
 * while a call on h is in flight.  AMGE_EINVAL for an index out of range, an
 * operator that is not stored (-1 in the report) or another lane count. */
amge_status amge_set_kernel(amge_hier* h, int32_t level, int32_t precision, int32_t op, int32_t lanes);

/* Coarsest-level solver of single-vector V-cycles:
 *   AMGE_COARSE_DENSE  the default: a product with the explicit FP64 inverse of A_L
 *                      (double-float pairs in the FP32 V-cycle)
 *   AMGE_COARSE_AUX    the paper's (Sections 4.2, 5.1): `iters` PCG iterations (five in
 *                      the paper) from zero on A_L, preconditioned by the additive
 *                      auxiliary-space preconditioner of eq. 4.2,
 *                        B^{-1} = M^{-1} + Pihat S_v^+ Pihat^T + D B_D D^T,
 *                      M the l1-Jacobi diagonal, S_v = Pihat^T A_L Pihat; H(curl) (AMS):
 *                      D = D_0 at level L, B_D = S_g^+ with S_g = D^T A_L D; H(div) (ADS):
 *                      D = D_1 at level L and B_D the same construction for the curl-curl
 *                      matrix A_c = D^T A_L D with the edge interpolation pihat_inner (no
 *                      gradient term: A_c annihilates gradients).  S^+ is a symmetric
 *                      generalized inverse (pivoted Cholesky; the auxiliary matrices of
 *                      natural-boundary problems are singular), computed on the host
 *                      here, in FP64 (the paper solves these problems with BoomerAMG).
 *                      Runs in FP64 (the FP32 V-cycle widens its input and rounds the
 *                      result).  Blocks of right-hand sides keep the dense solve.
 * pihat: the interpolation of vector H1 into the problem space at the coarsest level
 * (n_L rows, 3 columns per vertex: column 3 v + c); D: the exterior derivative into the
 * problem space at the coarsest level; pihat_inner: (H(div) only) the interpolation into
 * the edge space.  Host CSR, read during the call.  Synchronises `stream`; captured PCG
 * graphs are rebuilt on the next solve.  AMGE_EINVAL for an unknown solver, iters
 * outside [1, 64], missing or mis-sized matrices, or a workspace view; AMGE_ENOMEM,
 * AMGE_ECUDA. */
enum { AMGE_COARSE_DENSE = 0, AMGE_COARSE_AUX = 1 };
amge_status amge_set_coarse_solver(amge_hier* h, int32_t solver, int32_t iters, const amge_csr* pihat,
                                   const amge_csr* D, const amge_csr* pihat_inner, void* stream);

/* The PCG product q = A_0 p (FP64, with the p.q partials): code 0 = 32-bit columns,
 * 1700 = 16-bit column offsets with each slice's entries prefetched into L2 (where
 * A_0 has 16-bit columns), 1000 = 32-bit columns with the prefetch.  Chosen at upload
 * by timing each (us[0..2] for 0, 1700, 1000: time per launch, -1 where not measured);
 * all form the same sums.  set = 0: report the choice in *code; set = 1: take *code as
 * the choice (1700 acts as 0 without 16-bit columns) and report what is used.  us (3
 * floats) may be NULL.  Captured PCG graphs are rebuilt on the next solve.
 * AMGE_EINVAL for NULL h or code, or another code. */
amge_status amge_pcg_kernel(amge_hier* h, int32_t set, int32_t* code, float* us);

/* Form of the FP32 V-cycle's double-float product on smoothing level `level`
 * (AMGE_WIDE_DF): 0 = 32-bit columns, 1 = 16-bit column offsets, 2 = 16-bit offsets
 * with each slice's entries prefetched into L2 (1 and 2 where the 16-bit columns are
 * built).  Chosen at upload by timing (us[0..2]: time per launch, -1 where not
 * measured).  set = 0: report it in *form; set = 1: take *form (1 and 2 act as 0
 * without 16-bit columns) and report what is used.  The forms sum each row's entries
 * in the same order (the 32-bit form with one warp per slice).  us may be NULL.
 * layout (may be NULL): the level's 16-bit columns of A_l, 0 = not built, 1 = one base
 * column per slice, 2 = one per row.
 * AMGE_EINVAL for NULL h or form, a level out of range or another form. */
amge_status amge_df_form(amge_hier* h, int32_t level, int32_t set, int32_t* form, float* us, int32_t* layout);

/* Kernel choice of the block (multi-right-hand-side) products for nrhs columns (2 ..
 * 32) and one precision, per smoothing level and operator (op order as above):
 * codes[l * 6 + op] = 0 CSR (a lane group per row), 1 / 2 sliced ELL with one / two
 * 16-byte vectors of columns per lane, -1 not stored or not tuned yet; and for the
 * coarsest product Z = A_L^{-1} B, codes[(levels-1) * 6] = 0 CUDA cores, 1 the FP64
 * tensor cores (mma.sync m8n8k4; nrhs a multiple of 8).  The library times the forms
 * per operator on the first block call with that nrhs and keeps the fastest; us
 * (optional) receives the measured time per launch (microseconds) of each form,
 * us[(l * 6 + op) * 3 + form], and the coarsest's two at us[(levels-1) * 18 + 0 / 1];
 * -1 where not measured.  codes holds (levels-1)*6 + 1 entries, us 3 times as many. */
amge_status amge_autotune_report_mm(amge_hier* h, int32_t nrhs, int32_t precision, int32_t* codes, float* us);

/* Pin one block kernel choice (code as above); op = 6 pins the coarsest product (level
 * ignored; code 1 needs nrhs a multiple of 8).  AMGE_EINVAL where the sliced-ELL form
 * does not apply to nrhs (nrhs must be a multiple of code * 16 / sizeof(value), at
 * most 8 lanes per row).  Pinned choices are not re-tuned. */
amge_status amge_set_kernel_mm(amge_hier* h, int32_t level, int32_t precision, int32_t op, int32_t nrhs,
                               int32_t code);

/* Release the hierarchy and all device memory it holds (NULL is ignored). */
void amge_hier_free(amge_hier* h);

/* Thread-local description of the last error on this thread ("" if none). */
const char* amge_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMGE_H */
