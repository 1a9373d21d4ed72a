// Library context: mesh geometry, index maps, the leaf maps, the merge tree
// and solver workspaces.  Host-side only (compiled by nvcc as C++).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hps.h"
#include "common.cuh"

namespace hps {

// Merge-level GEMM roles (see merge.cu for the formulas).
enum MergeRole {
  MS = 0, MR, MX1A, MX1B, MX2A, MX2B, MOA, MOB, MOC, MOD,  // merged map T_pair
  PG1A, PG1B, PG2A, PG2B, PU1, PU2, PD1, PD2, PD3, PD4,     // sweep operators U, D
  N_MROLE
};
enum SweepRole { SUP = 0, SDN, N_SROLE };

struct Stage {
  int a = 0, b = 0;          // element block size of each subdomain
  int gx = 0, gy = 0;        // subdomain grid
  int nsub = 0, n = 0;       // subdomains, boundary length 2 (a + b) q
  std::vector<int> es;       // [nsub * n] storage position -> element-side index
  int* d_es = nullptr;       // device copy (stage 0 and coarse stage)
  void* T = nullptr;         // [nsub][n][n] ItI maps, tree precision
  void* vec = nullptr;       // [nsub * n][nrhs_cap] sweep vector, tree precision
  // gamma-cycle (stages k >= 1): the stage system M_{k+1} e = e_nb + T e on these rows
  int* d_nb = nullptr;       // [nsub * n] stage row across the face (-1 on the physical boundary)
  GemmDesc* d_tdesc = nullptr;  // [nsub] the n x n product T_s e_s of each subdomain
  void* gR = nullptr;        // [nsub * n][nrhs_cap] restricted residual of the coarse calls
  void* gE = nullptr;        // [nsub * n][nrhs_cap] accumulated coarse correction
};

struct Level {               // merge l: stage l-1 -> stage l
  int dir = 0;               // 0: x-merge, 1: y-merge
  int npairs = 0, m = 0, n = 0, p = 0;
  std::vector<int> i1, i2;   // children of pair P (stage l-1 subdomain indices)
  int* d_dst = nullptr;      // [npairs][2p] storage position in the merged subdomain of [E1; E2]
  int* d_up = nullptr;       // [npairs * 2p] merged row -> child row (down-sweep copy)
  void* W = nullptr;         // [npairs][m][2m]: [S | I] -> [. | S^{-1}]
  void* U = nullptr;         // [npairs][2p][2m] restriction: rho'_E = rho_E - U f
  void* Dm = nullptr;        // [npairs][2m][2n] prolongation: x = Dm [child1 ; child2]
  int* d_xmap = nullptr;     // [npairs * 2m] row of x -> child row (interface rows)
  GemmDesc* d_mdesc = nullptr;  // [N_MROLE][npairs]
  GemmDesc* d_sdesc = nullptr;  // [N_SROLE][npairs]
  // FP32 tree, interface >= 32 complex: U and Dm kept tiled (tile_operator, tc.cu) for the sweeps
  GemmDesc* d_tsdesc = nullptr;  // [N_SROLE][npairs]: the sweep descriptors with a_r = first block, a_c = blocks per row tile
  void* Ut = nullptr;           // tiled U  (replaces U)
  void* Dmt = nullptr;          // tiled Dm (replaces Dm)
};

struct Coarse {
  int n_int = 0;             // interior (unknown) positions over all coarse subdomains
  int max_int = 0;           // largest interior count of one coarse subdomain
  GemmDesc* d_cdesc = nullptr;  // [nsub] T_int,int g_int GEMM per coarse subdomain
  int* d_cnb = nullptr;      // [nsub*n] stage row across the face (-1 on the physical boundary)
  int* d_upos = nullptr;     // [n_int] stage row of unknown u
  int* d_ucnb = nullptr;     // [n_int] stage row across from unknown u
  void* Winv = nullptr;      // exact coarse: [n_int][2 n_int] -> right half = M_c^{-1}
  GemmDesc* d_desc = nullptr;  // exact coarse: the one GEMM descriptor
  // FP32 tree with bf16 sweeps: each subdomain's T_int,int tiled as three-term bf16 blocks (the
  // coarse GMRES products at FP32 accuracy on the sweep kernel), and its tiled descriptors
  void* Tt = nullptr;
  GemmDesc* d_tcdesc = nullptr;
  bool exact = false;
  std::vector<int> upos_h, ucnb_h;  // host copies of d_upos, d_ucnb (exact coarse assembly)
};

struct Alloc {
  void* p;
  size_t bytes;
};

}  // namespace hps

struct hps_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  hps_alloc_fn alloc = nullptr;
  hps_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::string err;
  int num_sms = 0;
  std::vector<hps::Alloc> allocs;
  size_t bytes_held = 0;

  // mesh
  bool have_mesh = false;
  int nx = 0, ny = 0, N = 0, q = 0, E = 0, nb = 0, L = 0;
  long long n_skel = 0, n_bdry = 0, n_es = 0;
  double h = 0;
  std::vector<double> xi, wref, Dref, Kref;    // reference GLL rule, D, K = D^T W D
  std::vector<int> es_nb, es_in, es_out, es_bdry;
  int *d_es_nb = nullptr, *d_es_in = nullptr, *d_es_out = nullptr, *d_es_bdry = nullptr;
  int* d_bdry_rows = nullptr;  // [n_bdry] identity helper for boundary transposes
  double *d_Dref = nullptr, *d_Kref = nullptr, *d_wref = nullptr;
  double* d_vtab = nullptr;    // interior solve and corner tables (volume.cu)
  double mu_min = 0;           // smallest eigenvalue of K_ii w.r.t. W_ii (reference element)

  // coefficient (computed on the device by hps_set_coeff, with each element's leaf route)
  bool have_coeff = false;
  double kappa = 0, eta = 0;
  double* d_c = nullptr;
  double* d_bstage = nullptr;  // device copy of host samples b
  int* d_route = nullptr;      // [E] 0: positive-definite route, 1: pivoted route
  int* d_lists = nullptr;      // [2E + 2]: elements of each route, then the two counts
  int* d_cerr = nullptr;       // set by the coefficient kernel on a non-finite sample
  int* pin_counts = nullptr;   // pinned host mirror of the two route counts

  // leaves
  bool have_leaves = false;
  int precision = HPS_FP64;
  double2* d_T = nullptr;      // [E][nb][nb] FP64, side order l, r, b, t
  int n_robust = 0;            // elements built by the pivoted route
  int* d_flag = nullptr;
  int* d_gemm_err = nullptr;   // set by a tensor-core GEMM whose bounded wait gave up

  // tree.  The plan (stage orders, merge maps, GEMM descriptors, coarse maps: everything that
  // depends on the mesh and L_exact only) survives new coefficients and leaves; the numeric
  // part (maps T, inverses, sweep operators, workspaces) is rebuilt by every hps_merge_levels.
  bool have_tree = false;
  int L_exact = 0;
  int plan_L = -1;                 // L_exact of the cached plan, -1: none
  size_t plan_x_elems = 0;
  int plan_max_pairs = 0;
  int* plan_map0 = nullptr;        // stage-0 positions within each element's map
  std::vector<hps::Stage> stages;
  std::vector<hps::Level> levels;  // levels[l] for l = 1..L_exact (levels[0] unused)
  hps::Coarse coarse;
  int nrhs_cap = 0;                // sweep buffers sized for this many columns
  int gamma = 1;                   // coarse calls per level of the preconditioner (1: V-cycle)
  int gamma_nrhs = 0;              // gamma-cycle buffers (Stage gR, gE, gW) sized for this many columns
  void* gW = nullptr;              // gamma-cycle product T e of the largest stage
  void* gemm_ws = nullptr;         // split-K partial products
  size_t gemm_ws_elems = 0;
  void* ws_X1 = nullptr;           // merge workspaces
  void* ws_X2 = nullptr;
  size_t ws_X_elems = 0;
  int* d_piv = nullptr;
  void* d_lu = nullptr;
  void* sw_x = nullptr;            // down-sweep interface solution [max npairs*2m][nrhs]
  void* ws_G = nullptr;            // merge workspace: G = A^{-1} in [f1 | f2] column order
  void* d_eye = nullptr;           // identity of the largest interface size
  int eye_ld = 0;
  // coarse GMRES
  int cg_k = 0, cg_nrhs = 0;
  void *cg_V = nullptr, *cg_w = nullptr, *cg_W = nullptr, *cg_H = nullptr, *cg_h1 = nullptr, *cg_h2 = nullptr;
  void *cg_nrm = nullptr, *cg_y = nullptr, *cg_g = nullptr, *cg_s = nullptr, *cg_part = nullptr;
  void *cg_beta = nullptr, *cg_floor = nullptr, *cg_c = nullptr, *cg_inv = nullptr, *cg_cnt = nullptr;
  long long cg_part_cap = 0;  // elements of cg_part
  int cg_cnt_cap = 0;         // counters in cg_cnt
  // exact coarse scratch
  void *ex_r = nullptr, *ex_e = nullptr;
  int ex_nrhs = 0;
  // the mixed path's V-cycle as a CUDA graph (captured once per nrhs, coarse steps and buffer
  // generation); the graph reads its input and output pointers from mg_ptr
  long long vc_gen = 0;            // bumped whenever a V-cycle buffer is (re)allocated or freed
  cudaGraphExec_t mg_exec = nullptr;
  int mg_nrhs = 0, mg_k = 0, mg_gamma = 1;
  long long mg_gen = -1, mg_count = 0;  // buffer generation and kernel count of the captured graph
  bool mg_nograph = false;         // capture failed once: launch directly
  cudaStream_t gs = nullptr;       // capture / replay stream of the graph
  cudaEvent_t gs_in = nullptr, gs_out = nullptr;
  void** mg_ptr = nullptr;         // device [2]: rho (float4*), z (float2*)

  // FP64 solver workspaces
  int fg_restart = 0, fg_nrhs = 0;
  double2 *fg_V = nullptr, *fg_Z = nullptr, *fg_x = nullptr, *fg_w = nullptr, *fg_rhs = nullptr, *fg_t = nullptr;
  double2 *fg_h = nullptr, *fg_part = nullptr, *fg_y = nullptr;
  double* fg_floor = nullptr;
  double2* pin_h = nullptr;  // pinned host mirror of fg_h
  double2* pin_y = nullptr;
  double* pin_floor = nullptr;
  // df64 outer FGMRES (HPS_OUTER_DF64): basis, residual and iterate as float pairs,
  // preconditioned directions in FP32, a df64 copy of the leaf maps
  int outer_arith = HPS_OUTER_DEFAULT;
  // the double-float Arnoldi matvec (hps_set_arnoldi_matvec) and the bf16 slices of the leaf
  // maps it multiplies on the tensor cores (cut from d_T at the start of every solve)
  int arnoldi_mv = HPS_MV_DEFAULT;
  uint16_t* ozk_A = nullptr;
  size_t ozk_A_elems = 0;
  // arithmetic of the sweep products of an FP32 tree (hps_set_sweep_arith), read when the tree
  // is built; sweep_bf16x3: the current tree's tiled sweep operators are bf16 hi/lo blocks
  int sweep_arith = HPS_SWEEP_DEFAULT;
  bool sweep_bf16x3 = false;
  bool fg_df = false;
  float4 *df_V = nullptr, *df_x = nullptr, *df_w = nullptr, *df_rhs = nullptr, *df_part = nullptr, *df_T = nullptr;
  float4* df_coef = nullptr;       // Gram-Schmidt update coefficients [2 restart + 3][nrhs]
  float4* pin_coef = nullptr;      // pinned host mirror of df_coef
  float2* df_Z = nullptr;
  double2 *pv_in = nullptr, *pv_out = nullptr;  // precond_apply/matvec ES staging
  // sources and volume solution (volume.cu): [E][nrhs][ni] interior and [E][nrhs][nb] edge arrays
  int vol_nrhs = 0;
  double2 *vol_B = nullptr, *vol_V = nullptr, *vol_U = nullptr, *vol_B2 = nullptr;
  double2 *vol_F = nullptr, *vol_G = nullptr;
  double2* vol_s = nullptr;    // staged sources
  size_t vol_s_elems = 0;
  double2* vol_H = nullptr;    // interior contributions H [n_es][nrhs]
  size_t vol_H_elems = 0;
  int pv_nrhs = 0;

  // profiling (hps_profile): CUDA events per phase on the context's stream
  bool prof = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[HPS_NPHASE] = {0};
  long long prof_launch[HPS_NPHASE] = {0};
  long long prof_calls[HPS_NPHASE] = {0};
  int cur_phase = -1;  // the innermost open PhaseScope's phase (-1: none)
  // kernel-class timing (hps_profile_kernels): events around each launch of a class
  struct KernEv {
    int kc;
    cudaEvent_t a, b;
  };
  bool kprof = false;
  std::vector<KernEv> kprof_ev;
  double kprof_ms[HPS_NKC] = {0}, kprof_bytes[HPS_NKC] = {0}, kprof_flops[HPS_NKC] = {0};
  long long kprof_launch[HPS_NKC] = {0};
  // tile autotuner mode (hps_set_autotune); the V-cycle key of the last uncaptured tuning pass
  int tune = HPS_TUNE_OFF;
  long long tune_pass_gen = -1;
  int tune_pass_nrhs = 0, tune_pass_k = -1, tune_pass_gamma = 0;
};

namespace hps {

int fail(hps_ctx* c, int code, const std::string& msg);
int cuda_fail(hps_ctx* c, cudaError_t e, const char* what);
void* dev_alloc(hps_ctx* c, size_t bytes);
void dev_free(hps_ctx* c, void* p);
template <typename T> T* dev_upload(hps_ctx* c, const std::vector<T>& v);
void free_tree(hps_ctx* c);     // numeric part and plan
void free_numeric(hps_ctx* c);  // numeric part only (the plan stays)
void free_solver(hps_ctx* c);
void free_fg(hps_ctx* c);  // FGMRES workspace (solve.cu)
void free_vol(hps_ctx* c); // source and volume-solution work arrays (volume.cu)
void free_vol_staging(hps_ctx* c);  // staged sources and the H buffer (volume.cu)
// H of every element for sources s (device [nrhs][E][(N+1)^2]) -> H_es [n_es][nrhs] (volume.cu)
int source_H(hps_ctx* c, const double2* s, int nrhs, double2* H_es);
int subtract_H(hps_ctx* c, double2* rho, const double2* H_es, int nrhs);
// Leaf maps of the listed positive-definite elements (device list of count) by the interior
// solver: the route for orders whose factor does not fit shared memory (volume.cu)
int fd_leaf_maps(hps_ctx* c, const int* elems, int count);
constexpr int LEAF_SMEM_MAX_N = 16;  // largest order of the shared-memory leaf kernel
const double2* stage_in(hps_ctx* c, const void* src, size_t elems, double2** buf, size_t* cap);
void free_graph(hps_ctx* c);
int ensure_sweep_buffers(hps_ctx* c, int nrhs);
int ensure_gamma_buffers(hps_ctx* c, int nrhs);  // gamma-cycle vectors (no-op for gamma = 1)

// tree operations (merge.cu)
int build_tree(hps_ctx* c, int L_exact, int exact_coarse);
template <typename R>
int mg_apply(hps_ctx* c, const double2* rho_es, double2* z_es, int nrhs, int inner_iters);
// the FP32 V-cycle on a df64 residual (its leading FP32 parts), FP32 result
int mg_apply_df(hps_ctx* c, const float4* rho_es, float2* z_es, int nrhs, int inner_iters);

}  // namespace hps

namespace hps {
// Attributes kernel launches to a phase and, when profiling is on, brackets the
// phase with CUDA events on the context's stream.
struct PhaseScope {
  hps_ctx* c;
  int ph;
  cudaEvent_t a = nullptr;
  long long* prev;
  int prev_phase;
  PhaseScope(hps_ctx* ctx, int phase);
  ~PhaseScope();
};
// With kernel-class timing on and the context's stream not capturing, brackets the launches
// made in its scope with CUDA events on the context's stream and credits their algorithmic
// bytes and flops to the class.
struct KernScope {
  hps_ctx* c;
  int kc;
  cudaEvent_t a = nullptr;
  KernScope(hps_ctx* ctx, int kclass, double bytes, double flops);
  ~KernScope();
};
}  // namespace hps

#define HPS_CK(ctx, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return hps::cuda_fail(ctx, e_, #call); \
  } while (0)
