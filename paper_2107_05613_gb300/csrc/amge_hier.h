// The device-resident hierarchy of the libamge C ABI (internal): per-level operators
// and workspaces in both precisions, the PCG workspace, captured graphs, profiling
// state.  Shared by the translation units that work on a hierarchy.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "amge_internal.h"

namespace amge {

constexpr int kNumTuneCodes = 17;  // candidates of the single-vector autotuner (kTuneCodes)

template <typename V>
struct LevelDev {
  int n = 0, naux = 0;
  DevSell<V> A, P, PT, G, GT;
  DevCsr<V> cA, cP, cPT, cG, cGT;  // CSR copies for the multi-RHS products
  // A G (n x naux), stored where it is cheaper to read than the residual it replaces:
  // the residual after an aux sweep is then updated as r - (A G) y instead of
  // recomputed as b - A x.  has_ag: stored (both precisions); use_ag: this precision's
  // V-cycle updates that way (FP64: A G much sparser than A; FP32: A G in FP32 cheaper
  // than the double-float residual of A)
  DevSell<V> AG;
  DevCsr<V> cAG;
  bool has_ag = false, use_ag = false;
  // G sign-coded with two entries per row in row order (the discrete gradient), for
  // the fused aux correction (launch_ag_fused); null where G has another shape
  int2* g2 = nullptr;
  // the same with up to four entries per row, padded (the discrete curl; H(div))
  int4* g4 = nullptr;
  // autotuned single-vector kernel per operator (A, P, PT, G, GT, AG): 0 = sliced
  // ELL, 100 w = sliced ELL with w warps per slice, 2..32 = vector CSR with that many
  // lanes per row, -1 = not stored
  int lanes[6] = {0, 0, 0, 0, 0, -1};
  // the autotuner's measured time per launch (us) of each candidate (kTuneCodes
  // order), -1 where not measured
  float tune_us[6][kNumTuneCodes] = {};
  // block (multi-right-hand-side) kernel per operator and column count: -1 = not
  // tuned yet, 0 = CSR, 1 / 2 = sliced ELL with 1 / 2 vectors of 16 bytes per lane
  int8_t mmk[6][kMaxRhs + 1];
  float mm_us[6][3] = {};  // the block tuner's time per launch (us) of each form, last tuned nrhs
  // Gauss-Seidel smoother (amge_set_smoother; FP64): A_l and A_aux = G^T A_l G with
  // rows grouped by colour (colour k: slices [cs[k], cs[k+1])), 1 / diagonal
  DevSell<V> gsA, gsX;
  std::vector<int> gsA_cs, gsX_cs;
  V *gsA_dinv = nullptr, *gsX_dinv = nullptr;
  V* t = nullptr;  // aux right-hand side G^T r of the Gauss-Seidel aux smoothing
  // FP32 V-cycle (lv32): A_l's values as double-float pairs {hi0, hi1, lo0, lo1} per
  // entry pair of the FP64 sliced-ELL copy (launch_sell_df)
  float4* Adf = nullptr;
  float2* cAdf = nullptr;  // the same for the CSR copy (block V-cycles)
  // form of the double-float product (timed at upload): 0 = 32-bit columns (warps per
  // slice of the FP64 A_l's code), 1 = 16-bit columns, 2 = 16-bit columns with the
  // per-slice L2 prefetch; us: time per launch of each, -1 where not measured
  int df_form = 0;
  float df_us[3] = {-1.f, -1.f, -1.f};
  V* minv = nullptr;
  V* mauxinv = nullptr;
  V *x = nullptr, *r = nullptr, *y = nullptr, *tmp = nullptr;
  V *b = nullptr, *z = nullptr;
  // block workspace ([n][nrhs] / [naux][nrhs]), allocated on the first multi-RHS call
  V *X = nullptr, *R = nullptr, *Y = nullptr, *T = nullptr, *B = nullptr, *Z = nullptr;
  LevelDev() { std::memset(mmk, -1, sizeof(mmk)); }
};

}  // namespace amge

using namespace amge;

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

// PCG loop captured once per precision: a WHILE conditional node whose body is one
// rotated iteration (z = B r, beta, p = z + beta p, q = A p, alpha, x and r updates,
// loop test), so a whole run of iterations needs no host round trip.
struct GraphPcg {
  bool built = false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle hw{};
  int64_t body[AMGE_PROF_CLASSES] = {};  // kernel launches of one body replay, per class
};

// The auxiliary-space coarsest solver (amge_set_coarse_solver, Section 4.2 eq. 4.2):
// operators of the coarsest level, the generalized inverses of its auxiliary
// matrices, work vectors and a reduction scratch of its own (the outer PCG's
// scalars stay live across the V-cycle).
struct CoarseAux {
  int iters = 5;
  int nv = 0, nd = 0, nv1 = 0;  // sizes: vector-H1 aux, D's columns, inner vector-H1 (ADS)
  bool ads = false;
  DevCsr<double> A, Pv, PvT, D, DT, Pi1, Pi1T;
  double *Gv = nullptr, *Gd = nullptr, *Gc = nullptr;  // generalized inverses (row-major)
  double *minv = nullptr, *mcinv = nullptr;
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *u = nullptr, *w = nullptr, *t = nullptr, *y = nullptr, *u2 = nullptr, *w2 = nullptr;
  double *bd = nullptr, *zd = nullptr;  // FP32 V-cycle: widened input, FP64 output
  double* tmp = nullptr;                // dense products' scratch
  RedScratch red;
  int rank_v = 0, rank_d = 0;           // ranks found for the generalized inverses
};

struct amge_hier {
  int form = 0, L = 0, nu_pre = 1, nu_post = 1;
  // smoother: AMGE_SMOOTHER_L1_JACOBI, or AMGE_SMOOTHER_SYM_GS on the gs_levels finest
  // smoothing levels (sweeps symmetric steps per smoothing; l1-Jacobi below them)
  int smoother = AMGE_SMOOTHER_L1_JACOBI, sweeps = 2, gs_levels = 0, gs_built = 0;
  // arithmetic of the FP32 V-cycle's residuals of corrected iterates (amge_set_wide_arith)
  int wide_arith = AMGE_WIDE_DF;
  int n0 = 0;
  int device = -1;  // CUDA device the operators live on (current at upload)
  std::vector<LevelDev<double>> lv64;
  std::vector<LevelDev<float>> lv32;
  DevSell<double> A0;  // finest operator for the outer PCG
  DevCsr<double> cA0;  // its CSR copy (multi-RHS products)
  int nC = 0;
  double *Linv = nullptr, *LinvT = nullptr, *ct = nullptr;
  double* Ainv = nullptr;  // explicit coarsest inverse (single-vector V-cycles)
  float2* Ainv_df = nullptr;  // the same as double-float pairs (FP32 V-cycles, AMGE_WIDE_DF)
  DevCsr<double> cAL;         // the coarsest matrix (CSR, FP64), for the auxiliary-space solver's setup
  CoarseAux* aux = nullptr;   // auxiliary-space coarsest solver, when selected (single vectors)
  CoarseAux* aux_store = nullptr;  // its data (owned; kept when the dense solver is selected again)
  double *pr = nullptr, *pz = nullptr, *pp = nullptr, *pq = nullptr;
  double *stage_b = nullptr, *stage_x = nullptr;
  float *s32_in = nullptr, *s32_out = nullptr;
  RedScratch red;
  RedScratchMM redmm;
  int mm_cap = 0;  // nrhs the block workspace was sized for
  bool mm_tuned[2][kMaxRhs + 1] = {};  // block kernels timed for (precision, nrhs)
  // block coarsest product Z = A_L^{-1} B per (precision, nrhs): 0 CUDA cores, 1 FP64
  // tensor cores (DMMA); the tuner's times (us) of both
  int8_t coarse_mm[2][kMaxRhs + 1] = {};
  float coarse_mm_us[2][kMaxRhs + 1][2] = {};
  GraphPcg gmm[2][kMaxRhs + 1];        // captured block PCG loops per (precision, nrhs)
  int* gstate_mm = nullptr;            // device: iterations done, maxit, non-finite flag
  int* pinned_state_mm = nullptr;
  double* GX = nullptr;                // block iterate of the graph-driven loop
  // coefficient updates (hierarchies made by amge_setup_upload): per-cell count and
  // the device data of the GPU re-setup
  int ncell = 0;
  amge::UpdatePlan* upd = nullptr;
  double *PR = nullptr, *PZ = nullptr, *PP = nullptr, *PQ = nullptr, *SB = nullptr, *SX = nullptr;
  float *S32in = nullptr, *S32out = nullptr;
  double* CT = nullptr;
  double* pinned_mm = nullptr;  // [SC_COUNT][kMaxRhs]
  double* pinned = nullptr;
  cudaEvent_t ev = nullptr;
  GraphPcg gpcg[2];
  cudaStream_t cap = nullptr;  // capture stream of the graphs
  int* gstate = nullptr;       // device: iterations done, maxit, non-finite flag
  int* kwait = nullptr;        // device: set by a bounded wait that ran out (amge_wait_status)
  // form of the PCG product q = A p (launch_pcg_spmv_dot; timed at upload)
  int pcg_form = 0;
  float pcg_spmv_us[3] = {-1.f, -1.f, -1.f};
  double* gx = nullptr;        // device: iterate of the graph-driven loop
  int* pinned_state = nullptr;
  bool use_graphs = true;
  std::vector<void*> allocs;
  size_t bytes = 0;     // device bytes this object allocated
  size_t op_bytes = 0;  // of which level operators (0 for a view)
  const amge_hier* base = nullptr;  // the hierarchy whose operators a view shares
  bool prof = false;
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_free;
  int64_t prof_count[AMGE_PROF_CLASSES] = {};
  int64_t launches[AMGE_PROF_CLASSES] = {};  // launches of each class, counted always
  double prof_ms[AMGE_PROF_CLASSES] = {};
};


