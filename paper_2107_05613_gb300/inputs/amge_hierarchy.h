/* Host FP64 generator of element-based AMG (AMGe) de Rham hierarchies.
 *
 * This is input generation, not the solve path: it builds, once and on the
 * host, every matrix the solve phase consumes (fine Whitney-form operators on a
 * Kuhn-split cube mesh, agglomerated coarse topologies, prolongators P_l from
 * PV traces and local extensions, integer coarse exterior derivatives, Galerkin
 * operators A_{l+1} = P_l^T A_l P_l).  Both the CUDA solve path and the CPU
 * oracle read its output as plain CSR arrays; neither links the other.
 *
 * Paper: Kalchev, Vassilevski, Villa, "Parallel Element-based Algebraic
 * Multigrid for H(curl) and H(div) Problems Using the ParELAG Library",
 * Sections 2-3 (eq. 2.2 forms, eq. 2.3 de Rham complex, Section 3.1 agglomerated
 * topology, eq. 3.5 PV traces, eqs. 3.6/3.8 extensions, Section 3.2.1 RAP).
 *
 * Conventions.
 *   Levels are numbered from 0 (finest) here; the paper numbers them from 1.
 *   Space index k = entity dimension: 0 = H1 (vertices), 1 = H(curl) (edges),
 *   2 = H(div) (faces), 3 = L2 (cells).  D_k maps space k to space k+1
 *   (D_0 = grad, D_1 = curl, D_2 = div) and is a signed integer incidence.
 *   Coefficient lettering: beta multiplies (Du, Dv), alpha multiplies (u, v)
 *   (the paper's eq. 2.2 letters them the other way round).
 */
#ifndef AMGE_HIERARCHY_H
#define AMGE_HIERARCHY_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { AMGH_FORM_HCURL = 1, AMGH_FORM_HDIV = 2 };
enum { AMGH_KIND_A = 0, AMGH_KIND_P = 1, AMGH_KIND_D = 2, AMGH_KIND_PI = 3, AMGH_KIND_PIHAT = 4 };
enum { AMGH_ALL_SPACES = 1, AMGH_TARGETS = 2, AMGH_TARGETS2 = 4 };

/* Build the hierarchy on an n^3 Kuhn-split unit cube.
 *   form        AMGH_FORM_HCURL (Nedelec edges) or AMGH_FORM_HDIV (Raviart-Thomas faces)
 *   num_levels  >= 1; 0 = coarsen 2x2x2 while the cell grid side m > 8 (and m even)
 *   beta, alpha per fine tetrahedron (6 n^3 values, tet t = 6*cube + permutation),
 *               NULL = all ones.  Must be > 0.
 *   flags       AMGH_ALL_SPACES: also build the prolongators of every lower space of
 *               the sequence (H1 for H(curl), H(curl) and H1 for H(div)) and the
 *               auxiliary-space data; otherwise only the spaces the problem needs.
 *               AMGH_TARGETS (not with AMGH_ALL_SPACES): polynomial approximation
 *               targets (Section 3.3.1) -- the interpolants of the vector monomials of
 *               degree <= 1 -- enrich the last coarsening: their traces on coarse
 *               edges (H(curl)) or faces (H(div)) orthogonal to the PV traces, and
 *               their mass projections onto the D-free bubbles of coarse faces and
 *               cells (Section 3.3.3), filtered of linear dependence and extended by
 *               eqs. 3.6 / 3.8, become extra coarse basis functions (columns of P
 *               after the coarse entities' ones); the coarsest matrix is the Galerkin
 *               product P^T A P with that P.
 *               AMGH_TARGETS2: the same with the monomials of degree <= 2, which also
 *               brings the cross-space bubbles of eqs. 3.7 / 3.9 (the targets'
 *               non-constant divergences and curls) into the coarsest space.
 *   nthreads    OpenMP threads (<= 0: library default).
 * Returns 0 and a handle in *out, or nonzero with amgh_error() describing it. */
int amgh_build(int form, int n, int num_levels, const double* beta, const double* alpha,
               int flags, int nthreads, void** out);
const char* amgh_error(void);
int amgh_num_levels(const void* h);
/* entity counts V, E, F, T at a level */
int amgh_level_counts(const void* h, int level, int64_t counts[4]);
/* kind A: problem matrix at `level` (k ignored); kind P: prolongator of space k from
 * level+1 to level; kind D: signed incidence D_k at `level`.  With all_spaces also
 * kind PI: co-chain projector of space k from `level` to level+1 (coarse rows; the
 * signed sum over each coarse entity's constituents, Pi P = I) and kind PIHAT: the
 * interpolation of vector H1 (column 3 v + c = component c at vertex v) into space
 * k = 1 (edges) or 2 (faces) at `level` (finest: exact for linear fields; coarser:
 * the recursion pihat^{l+1} = Pi^l pihat^l (P_0 (x) I_3) of Section 4.2).
 * info = {rows, cols, nnz}. */
int amgh_matrix_info(const void* h, int kind, int level, int k, int64_t info[3]);
int amgh_matrix_copy(const void* h, int kind, int level, int k, int32_t* row_ptr, int32_t* col,
                     double* val);
/* diagnostics: [0] max |lambda - coarse incidence| over (3.6) solves,
 *              [1] max relative residual of local solves,
 *              [2] max disagreement of coarse incidence over constituent choices,
 *              [3] setup seconds */
int amgh_diagnostics(const void* h, double out[4]);
/* approximation targets (AMGH_TARGETS): the coarse basis functions added and the
 * largest relative divergence of one of them on a constituent cell (0 without) */
int amgh_target_info(const void* h, int64_t* functions, double* constraint);
/* Fine-level assembly of the problem matrix A_0 written as a gather, for re-assembling
 * it from new coefficients: every stored entry q of A_0 (the CSR order of
 * amgh_matrix_copy) is the sum, in order, of
 *   beta[c] K[(c % 6) * s*s + idx] + alpha[c] M[(c % 6) * s*s + idx]
 * over its contributions t = coff[q] .. coff[q+1]-1 with c = ccell[t], idx = cidx[t]
 * (s = local_size: 6 edges (H(curl)) or 4 faces (H(div)) per cell; K = the derivative
 * term's element matrix, M = the mass term's, of the six Kuhn shapes).
 * info: *ncontrib = total contributions.  copy: K, M [6*s*s]; coff [nnz+1];
 * ccell, cidx [ncontrib]. */
int amgh_fine_assembly_info(const void* h, int64_t* ncontrib, int* local_size);
int amgh_fine_assembly_copy(const void* h, double* K, double* M, int32_t* coff, int32_t* ccell, uint8_t* cidx);
void amgh_free(void* h);

#ifdef __cplusplus
}
#endif
#endif
