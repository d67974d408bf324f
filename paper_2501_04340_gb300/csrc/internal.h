// Internal declarations of the GB300 IETI-DP library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/ieti.h"
#include "model.h"

namespace ieti {

constexpr int NB = 64;            // panel width of the dense factorisations
constexpr int MAX_RHS = 64;

// Per-subdomain offsets (in elements) into the concatenated device buffers.
// Local r DOFs of subdomain k are ordered [r_V, pad, r_I, pad] with the r_I
// block starting at nVp (a multiple of NB) and n a multiple of NB; padding
// DOFs are decoupled identity rows. The dense blocks are column-major with
// leading dimension n.
struct SubDev {
  int64_t A;      // K_rr (n x n) in K64 and in the factor buffer
  int64_t Kp;     // K_rp (n x nP)
  int64_t Kpp;    // K_pp (nP x nP)
  int64_t S;      // S_rIrI and W = S_rIrI^-1 (ldI x nI, ldI = nI rounded up to 4)
  int64_t linv;   // inverses of the NB x NB diagonal blocks of the factor
  int64_t dof;    // local DOF table, n + nP entries
  int64_t rv;     // r-vectors (n rows)
  int64_t pv;     // p-vectors (nP rows)
  int64_t iv;     // interface vectors (nI rows)
  int n, nVp, nI, nP, nblk, ldI;
};

// kernel classes timed with CUDA events when profiling is enabled
enum ProfCat {
  PROF_ASM_K = 0, PROF_ASM_J, PROF_POTRF, PROF_TRSM, PROF_SYRK, PROF_FWD, PROF_BWD, PROF_LOCAL_W,
  PROF_LOCAL_S, PROF_GATHER, PROF_COARSE, PROF_PCG, PROF_RESID, PROF_OTHER, PROF_NCAT
};

struct Prof {
  bool on = false;
  unsigned mask = ~0u;     // classes timed (bit c: class c); launch groups of unnamed class only with all bits
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  double ms[PROF_NCAT] = {};
  int64_t calls[PROF_NCAT] = {};
};

// one subdomain's right-hand-side block of a batched triangular solve
struct SolveDesc {
  int64_t boff;   // offset of this subdomain's RHS block
  int b0;         // first panel of the solve range
  int ldb;        // leading dimension (rows of the range)
  int ncol;       // columns for this subdomain
  int pad_;
};

struct Ctx;
// which sweeps of a triangular solve to run
constexpr int SWEEP_FWD = 1;    // L Y = B (B is overwritten)
constexpr int SWEEP_BWD = 2;    // L^T X = Y (Y is overwritten)
constexpr int SWEEP_BOTH = 3;
// local DOF: direction d and global control-grid index (i, j, k) of its edge;
// d = -1 for padding
struct DofDev {
  int d, i, j, k;
};

// tile table of the streamed interface products (one per precision and operator)
struct StreamPlan {
  bool built = false;
  bool incomplete = false;   // a subdomain without interface rows has primal rows (not streamed)
  int ntiles = 0, grid = 0, stage_bytes = 0;
  int64_t bytes = 0;         // bytes streamed per column group
  void* d_tiles = nullptr;
  int* d_cta = nullptr;      // first tile of every CTA (grid + 1 entries)
  int2* d_ckr = nullptr;     // subdomains [x, y) that every CTA's tiles touch
  int rows_cap = 0;          // rows per tile at most (chosen by the autotuner)
  int row_target = 0;        // row-mode plan: tiles of whole rows of about this many bytes (0: rows_cap rows)
};

// one step of the blocked factorisation with its work lists (symbolic.cu)
struct FactorStep {
  int b = 0, kb = 1;             // panels b .. b+kb-1
  bool snap = false;             // S_rIrI snapshot before panel b
  int64_t trsm_off[2] = {0, 0};  // (subdomain, block row) items of the panel solves of b and b+1
  int trsm_cnt[2] = {0, 0};
  int64_t col_off = 0;           // kb == 2: pair rows of block column b+1 updated by panel b
  int col_cnt = 0;
  int64_t trail_off = 0;         // trailing-update items, those of the next panels first
  int trail_cnt = 0;
  int trail_cnt0 = 0;            // items that update the next step's panel columns
};

struct FactorPlan {
  bool built = false;
  std::vector<FactorStep> steps;
  int4* d_items = nullptr;       // (k, R, C) pair tiles (FP32) or (k, i, j) tiles (FP64)
  int2* d_trsm = nullptr;        // (k, block row)
};

// task lists of the multi-column dependency-driven solves (sweep_dep.cu)
struct McPlan {
  bool built = false;
  int4* d_tasks[2] = {nullptr, nullptr};   // forward, backward: (k, block, column tile, counter)
  int ntask[2] = {0, 0};
  unsigned long long* d_prog = nullptr;    // per (subdomain, column tile)
};

struct DeviceBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Ctx {
  Mesh mesh;
  Tables1D tab;
  Gram1D gram[3];
  Topology topo;
  std::vector<int> sub_of_patch;
  std::vector<double> nu, ctrl, src;
  int source_kind = 0, nrhs = 1;
  bool affine = false;
  std::string err;
  int64_t launches = 0;

  // sizes
  int nsub = 0;
  int64_t m_r = 0, n_gp = 0;
  int max_n = 0, max_nI = 0, max_nP = 0, max_nblk = 0, max_ldI = 0;
  Prof prof;
  int64_t tot_A = 0, tot_Kp = 0, tot_Kpp = 0, tot_S = 0, tot_linv = 0, tot_dof = 0;
  int64_t tot_rv = 0, tot_pv = 0, tot_iv = 0;
  std::vector<SubDev> sd_host;
  std::vector<double> gq_host;           // per patch: nu * L_c^2 / vol (affine path)
  std::vector<int> elem_host;            // per element: q, s0, s1, s2
  std::vector<double> gD_host;           // IETI_SOURCE_TRIG: boundary coefficients (nedge)
  std::vector<int32_t> belem_host;       // elements with a facet in a Dirichlet face
  int64_t nelem = 0;
  double* d_geo = nullptr;               // per element and Gauss point: X, weight |det DF| DF^-1 (assembly)
  // loads of box patches from separable 1D integrals (assemble.cu): coefficient
  // grid, 1D tables, slab geometry and Gauss points on the device
  bool sep_loads = true;                 // false (IETI_DEBUG_ELEMENT_LOADS): element quadrature for the loads
  double2* d_sep_C = nullptr;
  std::vector<double2> sep_C_host;
  int64_t sep_C_cap = 0;
  double2* d_sep_tab = nullptr;
  int64_t sep_tab_cap = 0;
  double* d_sep_geo = nullptr;           // per axis and slab: lower coordinate, length
  double* d_xq = nullptr;                // Gauss points on [0, 1]
  double* d_sep_ploc = nullptr;          // per patch-local edge and load case: its patch's load
  int64_t sep_ploc_cap = 0;
  // deterministic sums of the patch loads: per local DOF slot (r DOFs of all
  // subdomains, then p DOFs) the patch-local edges that carry it, in order
  int64_t* d_sep_gofs = nullptr;         // slots + 1 offsets into d_sep_glist
  int64_t* d_sep_glist = nullptr;
  int64_t* d_sep_gbase = nullptr;        // per slot: destination of load case 0 in jr (r slots) or jp
  int32_t* d_sep_gstride = nullptr;      // per slot: column stride of the destination
  int64_t sep_nslot = 0, sep_npl = 0;    // slots, patch-local edges
  bool geo_ready = false, geo_failed = false;
  int64_t* d_patch_eoff = nullptr;       // per patch: its first element (npatch + 1 entries)
  double* d_flux_part = nullptr;         // flux evaluation: per element and load case, 2 integrals
  int64_t flux_part_cap = 0;
  double* d_flux_out = nullptr;          // per patch and load case: 2 squared norms
  double* d_flux_amp = nullptr;          // reference amplitudes (MAX_RHS)

  // device memory
  std::vector<DeviceBuf> allocs;
  SubDev* d_sd = nullptr;
  DofDev* d_dof = nullptr;
  int64_t* d_r_edge = nullptr;           // global edge id of each local r / p DOF (-1 pad)
  int32_t* d_I_dual = nullptr;           // per interface DOF: multiplier index
  double* d_I_sign = nullptr;
  double* d_I_scale = nullptr;           // rho-scaling D^(k)
  int32_t* d_P_glob = nullptr;           // per primal DOF: coarse index
  int32_t* d_pair = nullptr;             // per multiplier: k1, i1, k2, i2
  int32_t* d_patch_code = nullptr;       // per patch-local edge: local DOF index, -1 dropped
  int64_t* d_patch_code_off = nullptr;
  int32_t* d_sub_of_patch = nullptr;
  int32_t* d_elem = nullptr;
  double* d_gD = nullptr;                // IETI_SOURCE_TRIG: boundary coefficients of A_ana (nedge), else null
  int32_t* d_belem = nullptr;            // elements with a facet in a Dirichlet face (lifting of the loads)
  int64_t nbelem = 0;
  double* d_tabN[3] = {nullptr, nullptr, nullptr};
  double* d_tabdN[3] = {nullptr, nullptr, nullptr};
  double* d_tabD[3] = {nullptr, nullptr, nullptr};
  double* d_wq = nullptr;
  double* d_ctrl = nullptr;
  double* d_nu = nullptr;
  double* d_src = nullptr;
  double* d_gq = nullptr;
  double* d_gram[3] = {nullptr, nullptr, nullptr};
  int32_t* d_slab_of[3] = {nullptr, nullptr, nullptr};
  int32_t* d_start[3] = {nullptr, nullptr, nullptr};
  int32_t* d_nspan[3] = {nullptr, nullptr, nullptr};

  double* K64 = nullptr;                 // assembled K_rr (kept for FP64 residuals)
  double* Kp64 = nullptr;
  double* Kpp64 = nullptr;
  double* jr = nullptr;                  // loads (n x nrhs per subdomain)
  double* jp = nullptr;
  void* L = nullptr;                     // factor (double or float)
  void* Linv = nullptr;
  void* S = nullptr;                     // S_rIrI (nI x nI, full)
  void* W = nullptr;                     // S_rIrI^-1
  double* Phi = nullptr;                 // K_rr^-1 K_rp (n x nP), FP64 storage
  void* Psi = nullptr;                   // L^-1 K_rp (n x nP), factor precision
  void* wyk = nullptr;                   // L^-1 j_r of the last interface right-hand side (factor precision)
  int64_t* d_uoff = nullptr;             // u-vector offsets of the subdomains (device copy)
  SolveDesc* d_desc_rv = nullptr;        // r-vector sweep ranges: [0, nsub) full, [nsub, 2 nsub) r_I rows
  int min_b0_I = 0;                      // first panel of the r_I range over all subdomains
  // tile-level symbolic analysis (symbolic.cu), built once from an assembled K_rr
  std::vector<int64_t> tile_off;         // per subdomain: first of its nblk^2 tile flags
  std::vector<int> blk_base;             // per subdomain: first of its block rows over all subdomains
  std::vector<unsigned char> kflags;     // nonzero tiles of K_rr
  std::vector<unsigned char> lflags;     // nonzero lower tiles of the factor
  FactorPlan fplan[2];                   // [0] FP64, [1] FP32 work lists
  bool symb_ready = false;
  double lfill = 1.0;                    // fraction of the lower tiles that are nonzero
  int64_t* d_lrow_ptr = nullptr;         // per block row: its nonzero tiles left of the diagonal (ascending)
  int32_t* d_lrow_col = nullptr;
  int64_t* d_lcol_ptr = nullptr;         // per block column: its nonzero tiles below the diagonal (descending)
  int32_t* d_lcol_row = nullptr;
  unsigned char* d_lflags = nullptr;
  int64_t* d_tile_off = nullptr;
  bool ktile_ready = false;
  int4* d_ktile_list = nullptr;          // nonzero lower tiles (k, I, J), I >= J, of K_rr
  int n_ktiles = 0;
  int4* d_ltile_list = nullptr;          // lower tiles (k, I, J) of the factor's pattern
  int n_ltiles = 0;
  int l_init_prec = -1;                  // precision whose full conversion zeroed the other tiles of L
  int64_t* d_ktile_row = nullptr;        // per block row (over all subdomains) + 1: start in d_ktile_col
  int32_t* d_ktile_col = nullptr;        // block columns J with a nonzero tile
  int* d_ktile_base = nullptr;           // per subdomain: its first block row
  // dependency-driven single-column sweeps (sweep_dep.cu)
  int2* d_dep_tasks[2][2] = {};          // [range][forward, backward]: (subdomain, block) in run order
  int dep_ntask[2][2] = {};
  int2* d_dep_tasks2[2][2] = {};         // the same for tasks of two blocks (first block of the pair)
  int dep_ntask2[2][2] = {};
  unsigned long long* d_dep_prog = nullptr;   // per subdomain: epoch << 20 | blocks published
  unsigned long long dep_epoch = 0;
  int* d_dep_err = nullptr;              // set when a sweep wait times out; the poll limit at byte 8
  int fault_pivot_sub = -1;              // testing aid: subdomain whose next factorisation gets a negative pivot
  int fp64_fallbacks = 0;                // FP32 factorisations redone in FP64 (non-positive FP32 pivot)
  bool force_fallback = false;           // testing aid: the next FP32 refinement treats its first correction as stalled
  McPlan mcplan[2];                      // [0] W solve, [1] Phi solve
  bool autotune = true;                  // false (IETI_DEBUG_NO_AUTOTUNE): keep the default tile shapes
  bool tuned[2] = {false, false};        // [fp32] tile shapes of the streamed products chosen
  cudaStream_t aux_stream = nullptr;     // low-priority stream of the factorisation's lookahead
  cudaEvent_t ev_fact[3] = {nullptr, nullptr, nullptr};
  double* SPi = nullptr;                 // coarse S_Pi (n_gp x n_gp)
  double* SPiInv = nullptr;              // its inverse
  int* d_err = nullptr;                  // device error word (subdomain id + 1 of a bad pivot)
  int* h_err = nullptr;                  // pinned mirror

  // work buffers
  void* wr[3] = {nullptr, nullptr, nullptr};   // r-vector work (T or double), max_rhs columns
  double* wr64[3] = {nullptr, nullptr, nullptr};
  double* wp64 = nullptr;                // p-vector work
  double* wi[2] = {nullptr, nullptr};    // interface work (nI x nrhs)
  double* wq_part = nullptr;             // per subdomain primal partials
  double* wc[2] = {nullptr, nullptr};    // coarse vectors
  double* wlam[8] = {};                  // PCG vectors (m_r x nrhs)
  float* wvf = nullptr;                  // FP32 PCG vectors of the streamed form (5 x m_r x nrhs)
  // graphs of the refinement step's launch sequence: [first step, correction]
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    int prec = -1, maxit = 0;
    double tol_in = 0;
    const double* a = nullptr;           // the caller's field buffer the graph writes
    int64_t nkern = 0;                   // kernel launches in the graph (counted at each replay)
  } sgraph[2];
  bool graph_ok = true;                  // capture works here (cleared at the first failure)
  cudaStream_t cap_stream = nullptr;     // the stream the graphs are captured on
  bool graph_pcg_persistent = false;     // the last directly launched step ran the persistent PCG
  double* wscal = nullptr;               // PCG scalars
  double* wred = nullptr;                // reduction partials
  int* wflag = nullptr;
  double* wglob = nullptr;               // global edge vectors (nedge x nrhs)
  double* whist = nullptr;               // PCG alpha/beta history of column 0
  double* wnorm = nullptr;               // column norms
  void* d_descbuf = nullptr;             // triangular-solve descriptors
  int2* d_pcsr = nullptr;                // contributors (k, c) of each coarse DOF
  int64_t* d_pcsr_off = nullptr;
  int64_t* d_primal_edges = nullptr;
  double* wres_r = nullptr;              // local residual r-vectors
  double* wres_p = nullptr;
  double* wxp = nullptr;                 // the field at the local p DOFs (residual)
  double* wlam_acc = nullptr;            // accumulated multipliers

  // streamed interface products (iface.cu)
  int sm_count = 0, smem_optin = 0;
  StreamPlan splan[2][2];                // [FP32 operators][with the Phi_I^T rows]
  StreamPlan rplan[2][2];                // the same for single-column row mode: tiles of equal bytes
  void* PhiT = nullptr;                  // rows of Phi_I^(k)T in the factor precision (nP x ldI)
  std::vector<int64_t> phio;             // their offsets
  int64_t* d_phio = nullptr;
  int4* d_gs = nullptr;                  // per multiplier: iv and i of both sides
  int2* d_gn = nullptr;                  // per multiplier: nI of both sides
  int2* d_gu = nullptr;                  // per multiplier: positions of both sides in the u vectors
  int4* d_jt = nullptr;                  // per local interface DOF: multiplier, other side's iv, i, nI
  std::vector<int64_t> uoff;             // per subdomain: offset of u_k (ldI_k entries)
  int64_t utot = 0;                      // column stride of the u vectors
  void* uall = nullptr;                  // prepared u vectors (factor precision, MAX_RHS columns)
  int32_t* d_gell_i = nullptr;           // coarse part of the F gather (ELL, m_r x gell_E)
  double* d_gell_v = nullptr;
  int gell_E = 0;
  int4* d_pcon = nullptr;                // contributors of each coarse DOF: (pv_k, c, nP_k)
  int64_t pcon_count = 0;
  int* d_stream_err = nullptr;           // set when a bulk-copy or tensor-core wait times out
  float* tc_img = nullptr;               // TF32 term images of the current panel (syrk_tc.cu)
  int* d_grp_off = nullptr;              // per subdomain: first 128-row group in tc_img
  bool syrk_tc = false;                  // IETI_DEBUG_SYRK_TC: FP32 trailing update with split TF32 tensor-core products
  int syrk_reserve = 24;                 // SMs left free by the overlapped FP32 trailing update

  bool assembled = false, factored = false, host_only = false;
  ieti_precision prec = IETI_FP64;
};

// error helpers
#define IETI_CUDA_TRY(ctx, call)                                                   \
  do {                                                                             \
    cudaError_t e__ = (call);                                                      \
    if (e__ != cudaSuccess) {                                                      \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e__);            \
      return IETI_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

#define IETI_LAUNCH_CHECK(ctx)                                                     \
  do {                                                                             \
    (ctx)->launches++;                                                             \
    cudaError_t e__ = cudaGetLastError();                                          \
    if (e__ != cudaSuccess) {                                                      \
      (ctx)->err = std::string("kernel launch: ") + cudaGetErrorString(e__) +      \
                   " at " + __FILE__ + ":" + std::to_string(__LINE__);             \
      return IETI_ERR_CUDA;                                                        \
    }                                                                              \
  } while (0)

// profiling marks (no-ops unless enabled); `cat` names the class at the start
// of the group where only some classes are timed
inline cudaEvent_t prof_begin(Ctx* c, cudaStream_t st, int cat = -1) {
  if (!c->prof.on) return nullptr;
  if (cat >= 0 ? !(c->prof.mask & (1u << cat)) : c->prof.mask != ~0u) return nullptr;
  if (c->prof.used + 2 > c->prof.pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->prof.pool.push_back(e);
    }
  }
  cudaEvent_t e = c->prof.pool[c->prof.used++];
  cudaEventRecord(e, st);
  return e;
}
inline void prof_end(Ctx* c, int cat, cudaEvent_t e0, cudaStream_t st) {
  if (!c->prof.on || !e0) return;
  cudaEvent_t e1 = c->prof.pool[c->prof.used++];
  cudaEventRecord(e1, st);
  c->prof.marks.push_back({cat, {e0, e1}});
}
// folds the recorded marks into per-class totals (synchronises)
void prof_collect(Ctx* c);

// assembly
ieti_status assemble_all(Ctx* c, cudaStream_t s);
// B = curl a at the Gauss points of every element and its squared L2 norms per
// patch (out: npatch x nrhs norms, then npatch x nrhs errors to the reference)
ieti_status flux_kernel_attrs(Ctx* c, int smem_max);
ieti_status eval_flux(Ctx* c, const double* a, int nrhs, int ref_kind, const double* amp_dev, double* part,
                      double* out, double* Bq, cudaStream_t st);
ieti_status assemble_kernel_attrs(Ctx* c, int smem_max);
ieti_status solve_kernel_attrs(Ctx* c, int smem_max);
// factorisation
ieti_status factor_all(Ctx* c, cudaStream_t s);
ieti_status factor_kernel_attrs(Ctx* c);
// FP32 trailing update on the tensor cores (syrk_tc.cu)
ieti_status syrk_tc_attrs(Ctx* c);
ieti_status syrk_tc_alloc(Ctx* c);
ieti_status syrk_tc(Ctx* c, const SubDev* d_sd, float* L, int b, int max_nblk, int nsub, cudaStream_t st);
// triangular sweeps with the local factors on nrhs-column r-vectors: over the
// whole r range (RV_FULL) or over the r_I rows only (RV_IRANGE; the forward
// sweep of a right-hand side that vanishes on the r_V rows, or the backward
// sweep that yields the r_I rows of the solution)
constexpr int RV_FULL = 0;
constexpr int RV_IRANGE = 1;
template <typename T>
ieti_status rv_solve(Ctx* c, int range, int which, T* B, T* Y, T* X, cudaStream_t s);
// tile patterns of K_rr and of the factor, factorisation work lists (symbolic.cu)
ieti_status build_ktiles(Ctx* c, cudaStream_t s);
ieti_status build_symbolic(Ctx* c, cudaStream_t s);
// the same sweeps for one column as dependency-driven block tasks (sweep_dep.cu);
// IETI_ERR_STATE if the device cannot run them
ieti_status dep_sweep_attrs(Ctx* c);
ieti_status dep_sweep_alloc(Ctx* c);
// poll limit of the dependency waits (a testing aid; default 2^22 polls)
ieti_status dep_set_poll_limit(Ctx* c, long long polls);
template <typename T>
ieti_status dep_sweep(Ctx* c, int range, int which, const T* B, T* Y, T* X, cudaStream_t s);
template <typename T>
ieti_status dep_mc_solve(Ctx* c, int slot, const std::vector<SolveDesc>& dh, const SolveDesc* dd, int which,
                         const T* B, T* Y, T* X, cudaStream_t s);
// streamed interface products (iface.cu)
ieti_status iface_alloc(Ctx* c);
ieti_status iface_prepare(Ctx* c, cudaStream_t s);
ieti_status iface_local(Ctx* c, bool fp32, bool with_phi, const double* x, const double* scale, double* t,
                        double* qpart, int nrhs, cudaStream_t s);
bool iface_coarse_fused(const Ctx* c);
ieti_status iface_gather_F(Ctx* c, const double* t, const double* qpart, const double* yc, int nrhs, double* y,
                           const double* dotv, double* part, int blocks, cudaStream_t s);
ieti_status iface_gather_P(Ctx* c, const double* t, int nrhs, double* z, const double* dotv, double* part,
                           int blocks, cudaStream_t s);
ieti_status iface_check(Ctx* c, cudaStream_t s);
// the PCG loop in one cooperative launch on the streamed products (pcg_stream.cu);
// IETI_ERR_STATE when that form does not apply
ieti_status pcg_stream(Ctx* c, double* lam, double* r, double* z, double* p, double* q, double tol2, int maxit,
                       bool fp32, cudaStream_t st);
// solver
// persistent PCG loop (state prepared by the caller); IETI_ERR_STATE if unavailable
ieti_status pcg_coop(Ctx* c, double* lam, double* r, double* z, double* p, double* q, double tol2, int maxit,
                     bool fp32, cudaStream_t st);
ieti_status apply_F(Ctx* c, const double* lam, double* y, int nrhs, bool fp32_ops, cudaStream_t s);
ieti_status apply_F_implicit(Ctx* c, const double* lam, double* y, cudaStream_t s);
ieti_status apply_precond(Ctx* c, const double* r, double* z, int nrhs, bool fp32_ops, cudaStream_t s);
ieti_status interface_rhs(Ctx* c, const double* jr, const double* jp, double* b, double* dprime,
                          int nrhs, cudaStream_t s);
ieti_status solve_all(Ctx* c, const double* lam0, double tol, int maxit, double tol_field,
                      double* a, double* lam_out, ieti_solve_info* info, cudaStream_t s);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// device copy of a host vector, owned by the context (freed with it)
template <typename T>
ieti_status dev_upload(Ctx* c, T** p, const std::vector<T>& h) {
  const size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed";
    return IETI_ERR_OOM;
  }
  c->allocs.push_back({q, bytes});
  *p = (T*)q;
  if (!h.empty()) IETI_CUDA_TRY(c, cudaMemcpy(q, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return IETI_OK;
}

// multi-column per-subdomain vectors: subdomain k's block of an nrhs-column
// vector starts at (offset_k * nrhs), column stride = local size
__host__ __device__ inline int64_t RV(const SubDev& s, int i, int col, int nrhs) {
  return s.rv * nrhs + i + (int64_t)s.n * col;
}
__host__ __device__ inline int64_t PV(const SubDev& s, int c, int col, int nrhs) {
  return s.pv * nrhs + c + (int64_t)s.nP * col;
}
__host__ __device__ inline int64_t IV(const SubDev& s, int i, int col, int nrhs) {
  return s.iv * nrhs + i + (int64_t)s.nI * col;
}

}  // namespace ieti
