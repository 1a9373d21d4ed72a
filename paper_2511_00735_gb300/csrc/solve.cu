// C ABI, second half: merge levels, skeleton RHS / matvec / preconditioner in
// the skeleton ("face") order, and the flexible GMRES (section 4.3), in FP64 or
// (mixed path) with its Arnoldi steps in double-float arithmetic.  On both paths
// every restart residual and the residual of the returned solution is formed
// with the FP64 matvec from the FP64 value of the iterate, so every convergence
// decision and every reported residual is an FP64 residual (FGMRES as iterative
// refinement, section 4.3).
//
// FGMRES runs on the element-side layout with residual-like vectors (the
// Arnoldi basis V) in outgoing coordinates rho = Pi r and solution-like
// vectors (Z, x) in incoming coordinates.  Pi is a permutation, so every inner
// product and norm equals the one of the skeleton-order vectors and the
// iterates are those of FGMRES on M g = RHS.  Classical Gram-Schmidt with one
// re-orthogonalisation pass; Givens rotations and the convergence test on the
// host (one small device-to-host copy per iteration).
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "ctx.h"
#include "df64.cuh"
#include "skel.cuh"

namespace hps {

void free_fg(hps_ctx* c) {
  void** bufs[] = {(void**)&c->fg_V, (void**)&c->fg_Z, (void**)&c->fg_x, (void**)&c->fg_w, (void**)&c->fg_rhs,
                   (void**)&c->fg_t, (void**)&c->fg_h, (void**)&c->fg_part, (void**)&c->fg_y, (void**)&c->fg_floor,
                   (void**)&c->df_V, (void**)&c->df_Z, (void**)&c->df_x, (void**)&c->df_w, (void**)&c->df_rhs, (void**)&c->df_part,
                   (void**)&c->df_T, (void**)&c->df_coef, (void**)&c->ozk_A};
  for (void** b : bufs) {
    dev_free(c, *b);
    *b = nullptr;
  }
  if (c->pin_h) cudaFreeHost(c->pin_h);
  if (c->pin_y) cudaFreeHost(c->pin_y);
  if (c->pin_floor) cudaFreeHost(c->pin_floor);
  if (c->pin_coef) cudaFreeHost(c->pin_coef);
  c->pin_h = c->pin_y = nullptr;
  c->pin_floor = nullptr;
  c->pin_coef = nullptr;
  c->fg_restart = c->fg_nrhs = 0;
  c->ozk_A_elems = 0;
}

// the tensor-core Arnoldi matvec for nrhs right-hand sides (else the SIMT double-float one)
bool use_ozk(const hps_ctx* c, int nrhs) { return c->arnoldi_mv != HPS_MV_SIMT && ozk_supported(c->nb, nrhs); }

// cut the current leaf maps into the tensor-core matvec's bf16 slices
int ozk_prepare(hps_ctx* c) {
  const size_t need = ozk_slices_elems(c->E, c->nb);
  if (need > c->ozk_A_elems) {
    dev_free(c, c->ozk_A);
    c->ozk_A = static_cast<uint16_t*>(dev_alloc(c, sizeof(uint16_t) * need));
    c->ozk_A_elems = c->ozk_A ? need : 0;
    if (!c->ozk_A) return fail(c, HPS_ENOMEM, "leaf-map slices");
  }
  HPS_CK(c, ozk_slice_T(c->d_T, c->ozk_A, c->E, c->nb, c->stream));
  return HPS_OK;
}

// w = Pi M z in double-float for the FP32 directions z (ES rows)
int arnoldi_matvec(hps_ctx* c, const float2* z, float4* w, int nrhs, int grid) {
  if (use_ozk(c, nrhs))
    HPS_CK(c, ozk_matvec(c->ozk_A, c->d_es_nb, z, w, c->E, c->nb, nrhs, c->num_sms, c->d_gemm_err, c->stream));
  else
    HPS_CK(c, df_matvec<float2>(c->df_T, c->d_es_nb, z, nullptr, w, c->E, c->nb, nrhs, grid, c->stream));
  return HPS_OK;
}


void subdomain_natural(const hps_ctx* c, int stage, int sub, std::vector<int>& out);

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ensure_pv(hps_ctx* c, int nrhs) {
  if (nrhs <= c->pv_nrhs) return HPS_OK;
  dev_free(c, c->pv_in);
  dev_free(c, c->pv_out);
  const size_t rows = std::max<long long>(c->n_es, c->n_bdry);
  c->pv_in = static_cast<double2*>(dev_alloc(c, sizeof(double2) * rows * nrhs));
  c->pv_out = static_cast<double2*>(dev_alloc(c, sizeof(double2) * rows * nrhs));
  if (!c->pv_in || !c->pv_out) return fail(c, HPS_ENOMEM, "staging vectors");
  c->pv_nrhs = nrhs;
  return HPS_OK;
}

bool use_df(const hps_ctx* c) {
  return c->outer_arith == HPS_OUTER_DF64 || (c->outer_arith == HPS_OUTER_DEFAULT && c->precision == HPS_MIXED);
}


// FGMRES workspace for `restart` and `nrhs`; df selects the df64 basis (float pairs) and FP32 directions
int ensure_fg(hps_ctx* c, int restart, int nrhs, bool df) {
  if (restart <= c->fg_restart && nrhs <= c->fg_nrhs && df == c->fg_df) return HPS_OK;
  if (df == c->fg_df) {
    restart = std::max(restart, c->fg_restart);
    nrhs = std::max(nrhs, c->fg_nrhs);
  }
  free_fg(c);
  const size_t vs = (size_t)c->n_es * nrhs;
  const size_t nblk = (size_t)bdot_blocks(c->n_es);
  c->fg_rhs = static_cast<double2*>(dev_alloc(c, sizeof(double2) * vs));
  c->fg_t = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)c->n_bdry * nrhs));
  const size_t hsz = (size_t)(2 * (restart + 1) + 1) * nrhs;
  c->fg_h = static_cast<double2*>(dev_alloc(c, sizeof(double2) * hsz));
  c->fg_part = static_cast<double2*>(dev_alloc(c, sizeof(double2) * nblk * (df ? 1 : restart + 1) * nrhs));
  c->fg_y = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)restart * nrhs));
  c->fg_floor = static_cast<double*>(dev_alloc(c, sizeof(double) * nrhs));
  bool ok = c->fg_rhs && c->fg_t && c->fg_h && c->fg_part && c->fg_y && c->fg_floor;
  if (df) {
    c->df_V = static_cast<float4*>(dev_alloc(c, sizeof(float4) * vs * (restart + 1)));
    c->df_Z = static_cast<float2*>(dev_alloc(c, sizeof(float2) * vs * restart));
    c->df_x = static_cast<float4*>(dev_alloc(c, sizeof(float4) * vs));
    c->df_w = static_cast<float4*>(dev_alloc(c, sizeof(float4) * vs));
    c->df_rhs = static_cast<float4*>(dev_alloc(c, sizeof(float4) * vs));
    c->df_part = static_cast<float4*>(dev_alloc(c, sizeof(float4) * nblk * (2 * (restart + 1) + 1) * nrhs));
    c->df_T = static_cast<float4*>(dev_alloc(c, sizeof(float4) * (size_t)c->E * c->nb * c->nb));
    c->df_coef = static_cast<float4*>(dev_alloc(c, sizeof(float4) * (size_t)(2 * restart + 3) * nrhs));
    ok = ok && c->df_V && c->df_Z && c->df_x && c->df_w && c->df_rhs && c->df_part && c->df_T && c->df_coef;
  } else {
    c->fg_V = static_cast<double2*>(dev_alloc(c, sizeof(double2) * vs * (restart + 1)));
    c->fg_Z = static_cast<double2*>(dev_alloc(c, sizeof(double2) * vs * restart));
    c->fg_x = static_cast<double2*>(dev_alloc(c, sizeof(double2) * vs));
    c->fg_w = static_cast<double2*>(dev_alloc(c, sizeof(double2) * vs));
    ok = ok && c->fg_V && c->fg_Z && c->fg_x && c->fg_w;
  }
  if (!ok) {
    free_fg(c);
    return fail(c, HPS_ENOMEM, "FGMRES workspace");
  }
  if (cudaMallocHost(&c->pin_h, sizeof(double2) * hsz) != cudaSuccess ||
      cudaMallocHost(&c->pin_y, sizeof(double2) * (size_t)restart * nrhs) != cudaSuccess ||
      cudaMallocHost(&c->pin_floor, sizeof(double) * nrhs) != cudaSuccess ||
      (df && cudaMallocHost(&c->pin_coef, sizeof(float4) * (size_t)(2 * restart + 3) * nrhs) != cudaSuccess)) {
    cudaGetLastError();
    free_fg(c);
    return fail(c, HPS_ENOMEM, "pinned host workspace");
  }
  c->fg_restart = restart;
  c->fg_nrhs = nrhs;
  c->fg_df = df;
  return HPS_OK;
}

int precond(hps_ctx* c, const double2* v, double2* z, int nrhs, int k) {
  PhaseScope ps(c, HPS_PH_PRECOND);
  if (k < 0) {
    HPS_CK(c, swap_add<double>(z, nullptr, v, c->d_es_nb, c->n_es, nrhs, c->stream));
    return HPS_OK;
  }
  return c->precision == HPS_FP64 ? mg_apply<double>(c, v, z, nrhs, k) : mg_apply<float>(c, v, z, nrhs, k);
}

using cd = std::complex<double>;

}  // namespace
}  // namespace hps

using namespace hps;

#define CHECK_CTX(c)                                                   \
  do {                                                                 \
    if (!(c)) return HPS_EINVAL;                                       \
    cudaError_t e0_ = cudaSetDevice((c)->device);                      \
    if (e0_ != cudaSuccess) return cuda_fail(c, e0_, "cudaSetDevice"); \
  } while (0)

extern "C" {

int hps_merge_levels(hps_ctx* c, int L_exact, int exact_coarse) {
  CHECK_CTX(c);
  if (!c->have_leaves) return fail(c, HPS_ENOTBUILT, "hps_build_leaves first");
  if (L_exact < 0 || L_exact > c->L) return fail(c, HPS_EINVAL, "0 <= L_exact <= L");
  int rc = build_tree(c, L_exact, exact_coarse);
  if (rc != HPS_OK) return rc;
  int gerr = 0;
  HPS_CK(c, cudaMemcpyAsync(&gerr, c->d_gemm_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HPS_CK(c, cudaStreamSynchronize(c->stream));
  if (gerr) {
    cudaMemsetAsync(c->d_gemm_err, 0, sizeof(int), c->stream);
    free_tree(c);
    return fail(c, HPS_ETIMEOUT, "a tensor-core GEMM of the merges timed out waiting for its MMAs");
  }
  return HPS_OK;
}

int hps_stage_T(hps_ctx* c, int stage, int sub, void* T_host) {
  CHECK_CTX(c);
  if (!c->have_tree) return fail(c, HPS_ENOTBUILT, "hps_merge_levels first");
  if (stage < 0 || stage > c->L_exact || !T_host) return fail(c, HPS_EINVAL, "stage");
  const Stage& S = c->stages[stage];
  if (sub < 0 || sub >= S.nsub) return fail(c, HPS_EINVAL, "subdomain");
  const int n = S.n;
  std::vector<double2> out((size_t)n * n);
  HPS_CK(c, cudaStreamSynchronize(c->stream));
  if (c->precision == HPS_FP64) {
    HPS_CK(c, cudaMemcpy(out.data(), static_cast<double2*>(S.T) + (size_t)sub * n * n, sizeof(double2) * n * n,
                         cudaMemcpyDeviceToHost));
  } else {
    std::vector<float2> tmp((size_t)n * n);
    HPS_CK(c, cudaMemcpy(tmp.data(), static_cast<float2*>(S.T) + (size_t)sub * n * n, sizeof(float2) * n * n,
                         cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < tmp.size(); ++i) out[i] = make_double2(tmp[i].x, tmp[i].y);
  }
  std::vector<int> nat;
  subdomain_natural(c, stage, sub, nat);
  std::vector<int> pos(n);
  for (int i = 0; i < n; ++i) {
    const int e = S.es[(size_t)sub * n + i];
    pos[i] = -1;
    for (int j = 0; j < n; ++j)
      if (nat[j] == e) pos[i] = j;
    if (pos[i] < 0) return fail(c, HPS_ECUDA, "internal: stage order");
  }
  double2* dst = static_cast<double2*>(T_host);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) dst[(size_t)pos[i] * n + pos[j]] = out[(size_t)i * n + j];
  return HPS_OK;
}

int hps_rhs(hps_ctx* c, const void* t, void* rhs, int nrhs) {
  CHECK_CTX(c);
  if (!c->have_leaves) return fail(c, HPS_ENOTBUILT, "hps_build_leaves first");
  if (!t || !rhs || nrhs < 1 || nrhs > 64) return fail(c, HPS_EINVAL, "pointers, 1 <= nrhs <= 64");
  int rc = ensure_pv(c, nrhs);
  if (rc) return rc;
  HPS_CK(c, user_to_rows(c->pv_in, static_cast<const double2*>(t), nullptr, c->n_bdry, nrhs, c->n_bdry, c->stream));
  HPS_CK(c, es_rhs(c->d_T, c->d_es_nb, c->d_es_bdry, c->pv_in, c->pv_out, c->E, c->nb, nrhs,
                   std::min(c->E, 8 * c->num_sms), c->stream));
  HPS_CK(c, rows_to_user(static_cast<double2*>(rhs), c->pv_out, c->d_es_out, c->n_es, nrhs, c->n_skel, c->stream));
  return HPS_OK;
}

int hps_skel_matvec(hps_ctx* c, const void* x, void* y, int nrhs) {
  CHECK_CTX(c);
  if (!c->have_leaves) return fail(c, HPS_ENOTBUILT, "hps_build_leaves first");
  if (!x || !y || nrhs < 1 || nrhs > 64) return fail(c, HPS_EINVAL, "pointers, 1 <= nrhs <= 64");
  int rc = ensure_pv(c, nrhs);
  if (rc) return rc;
  HPS_CK(c, user_to_rows(c->pv_in, static_cast<const double2*>(x), c->d_es_in, c->n_es, nrhs, c->n_skel, c->stream));
  HPS_CK(c, es_matvec(c->d_T, c->d_es_nb, c->pv_in, nullptr, c->pv_out, c->E, c->nb, nrhs,
                      std::min(c->E, 8 * c->num_sms), c->stream));
  HPS_CK(c, rows_to_user(static_cast<double2*>(y), c->pv_out, c->d_es_out, c->n_es, nrhs, c->n_skel, c->stream));
  return HPS_OK;
}

int hps_skel_matvec_mixed(hps_ctx* c, const void* x, void* y, int nrhs) {
  CHECK_CTX(c);
  if (!c->have_leaves) return fail(c, HPS_ENOTBUILT, "hps_build_leaves first");
  if (!x || !y || nrhs < 1 || nrhs > 64) return fail(c, HPS_EINVAL, "pointers, 1 <= nrhs <= 64");
  int rc = ensure_pv(c, nrhs);
  if (rc) return rc;
  const size_t vs = (size_t)c->n_es * nrhs;
  float2* z = static_cast<float2*>(dev_alloc(c, sizeof(float2) * vs));
  float4* w = static_cast<float4*>(dev_alloc(c, sizeof(float4) * vs));
  const bool ozk = use_ozk(c, nrhs);
  if (!ozk && !c->df_T)  // no double-float workspace yet: a later solve reallocates it, df_T included
    c->df_T = static_cast<float4*>(dev_alloc(c, sizeof(float4) * (size_t)c->E * c->nb * c->nb));
  if (!z || !w || (!ozk && !c->df_T)) {
    dev_free(c, z);
    dev_free(c, w);
    return fail(c, HPS_ENOMEM, "mixed matvec buffers");
  }
  cudaStream_t st = c->stream;
  auto ck = [&](cudaError_t e, const char* what) {
    if (rc == HPS_OK && e != cudaSuccess) rc = cuda_fail(c, e, what);
  };
  if (ozk) rc = ozk_prepare(c);
  else ck(df_from_d(c->df_T, c->d_T, (long long)c->E * c->nb * c->nb, st), "df_from_d");
  if (rc == HPS_OK) ck(user_to_rows(c->pv_in, static_cast<const double2*>(x), c->d_es_in, c->n_es, nrhs, c->n_skel, st),
                       "user_to_rows");
  if (rc == HPS_OK) ck(round_to_f2(z, c->pv_in, (long long)vs, st), "round_to_f2");
  if (rc == HPS_OK) rc = arnoldi_matvec(c, z, w, nrhs, std::min(c->E, 8 * c->num_sms));
  if (rc == HPS_OK) ck(df_to_d(c->pv_out, w, (long long)vs, st), "df_to_d");
  if (rc == HPS_OK)
    ck(rows_to_user(static_cast<double2*>(y), c->pv_out, c->d_es_out, c->n_es, nrhs, c->n_skel, st), "rows_to_user");
  int gerr = 0;
  if (rc == HPS_OK) {
    ck(cudaMemcpyAsync(&gerr, c->d_gemm_err, sizeof(int), cudaMemcpyDeviceToHost, st), "error flag");
    ck(cudaStreamSynchronize(st), "synchronize");
  }
  dev_free(c, z);
  dev_free(c, w);
  if (rc == HPS_OK && gerr) {
    cudaMemsetAsync(c->d_gemm_err, 0, sizeof(int), st);
    return fail(c, HPS_ETIMEOUT, "the tensor-core matvec timed out waiting for its copies or MMAs");
  }
  return rc;
}

int hps_set_arnoldi_matvec(hps_ctx* c, int method) {
  if (!c) return HPS_EINVAL;
  if (method != HPS_MV_DEFAULT && method != HPS_MV_SIMT && method != HPS_MV_TENSOR)
    return fail(c, HPS_EINVAL, "Arnoldi matvec: HPS_MV_DEFAULT, HPS_MV_SIMT or HPS_MV_TENSOR");
  c->arnoldi_mv = method;
  return HPS_OK;
}

int hps_precond_apply(hps_ctx* c, const void* r, void* z, int nrhs, int inner_iters) {
  CHECK_CTX(c);
  if (!c->have_tree) return fail(c, HPS_ENOTBUILT, "hps_merge_levels first");
  if (!r || !z || nrhs < 1 || nrhs > 64 || inner_iters < 0 || inner_iters > 60)
    return fail(c, HPS_EINVAL, "pointers, 1 <= nrhs <= 64, 0 <= inner_iters <= 60");
  int rc = ensure_pv(c, nrhs);
  if (rc) return rc;
  HPS_CK(c, user_to_rows(c->pv_in, static_cast<const double2*>(r), c->d_es_out, c->n_es, nrhs, c->n_skel, c->stream));
  rc = precond(c, c->pv_in, c->pv_out, nrhs, inner_iters);
  if (rc) return rc;
  HPS_CK(c, rows_to_user(static_cast<double2*>(z), c->pv_out, c->d_es_in, c->n_es, nrhs, c->n_skel, c->stream));
  return HPS_OK;
}

int hps_set_gamma(hps_ctx* c, int gamma) {
  if (!c) return HPS_EINVAL;
  if (gamma < 1 || gamma > 8) return fail(c, HPS_EINVAL, "1 <= gamma <= 8 coarse calls per level");
  c->gamma = gamma;
  return HPS_OK;
}

int hps_set_outer_arith(hps_ctx* c, int mode) {
  if (!c) return HPS_EINVAL;
  if (mode != HPS_OUTER_DEFAULT && mode != HPS_OUTER_FP64 && mode != HPS_OUTER_DF64)
    return fail(c, HPS_EINVAL, "outer arithmetic: HPS_OUTER_DEFAULT, HPS_OUTER_FP64 or HPS_OUTER_DF64");
  c->outer_arith = mode;
  return HPS_OK;
}

int hps_set_sweep_arith(hps_ctx* c, int mode) {
  if (!c) return HPS_EINVAL;
  if (mode != HPS_SWEEP_DEFAULT && mode != HPS_SWEEP_FP32 && mode != HPS_SWEEP_BF16X3)
    return fail(c, HPS_EINVAL, "sweep arithmetic: HPS_SWEEP_DEFAULT, HPS_SWEEP_FP32 or HPS_SWEEP_BF16X3");
  c->sweep_arith = mode;
  return HPS_OK;
}

int hps_gmres_solve(hps_ctx* c, const void* t, const void* s, int nrhs, double tol, int inner_iters, int restart,
                    int max_outer, void* g_out, hps_info* info) {
  CHECK_CTX(c);
  if (!c->have_leaves) return fail(c, HPS_ENOTBUILT, "hps_build_leaves first");
  if (inner_iters >= 0 && !c->have_tree) return fail(c, HPS_ENOTBUILT, "hps_merge_levels first (or inner_iters < 0)");
  if (!t || !g_out || nrhs < 1 || nrhs > 64 || !(tol > 0) || restart < 1 || restart > 200 || max_outer < 1 ||
      inner_iters > 60)
    return fail(c, HPS_EINVAL, "pointers, 1<=nrhs<=64, tol>0, 1<=restart<=200, max_outer>=1, inner_iters<=60");
  const bool df = use_df(c);
  if (df && c->precision != HPS_MIXED) return fail(c, HPS_EINVAL, "HPS_OUTER_DF64 needs HPS_MIXED leaves");
  const auto t0 = std::chrono::steady_clock::now();
  int rc = ensure_fg(c, restart, nrhs, df);
  if (rc) return rc;
  rc = ensure_pv(c, nrhs);
  if (rc) return rc;
  cudaStream_t st = c->stream;
  const long long n = c->n_es;
  const long long vs = n * nrhs;
  const int grid = std::min(c->E, 8 * c->num_sms);
  // boundary data -> [n_bdry][nrhs]
  const double2* t_dev = static_cast<const double2*>(t);
  if (!is_device_ptr(t)) {
    HPS_CK(c, cudaMemcpyAsync(c->pv_in, t, sizeof(double2) * (size_t)c->n_bdry * nrhs, cudaMemcpyHostToDevice, st));
    t_dev = c->pv_in;
  }
  {
    PhaseScope ps(c, HPS_PH_RHS);
    HPS_CK(c, user_to_rows(c->fg_t, t_dev, nullptr, c->n_bdry, nrhs, c->n_bdry, st));
    HPS_CK(c, es_rhs(c->d_T, c->d_es_nb, c->d_es_bdry, c->fg_t, c->fg_rhs, c->E, c->nb, nrhs, grid, st));
    if (s) {  // RHS -= H: the interior contributions of the sources (section 3.1, eq. ItIOperator)
      const size_t n_s = (size_t)nrhs * c->E * (c->N + 1) * (c->N + 1);
      const double2* sd = stage_in(c, s, n_s, &c->vol_s, &c->vol_s_elems);
      if (!sd) return fail(c, HPS_ENOMEM, "staging of the sources");
      const size_t nh = (size_t)c->n_es * nrhs;
      if (nh > c->vol_H_elems) {
        dev_free(c, c->vol_H);
        c->vol_H = static_cast<double2*>(dev_alloc(c, sizeof(double2) * nh));
        c->vol_H_elems = c->vol_H ? nh : 0;
        if (!c->vol_H) return fail(c, HPS_ENOMEM, "interior contributions");
      }
      HPS_CK(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), st));
      rc = source_H(c, sd, nrhs, c->vol_H);
      if (rc) return rc;
      rc = subtract_H(c, c->fg_rhs, c->vol_H, nrhs);
      if (rc) return rc;
    }
    if (df) {
      if (use_ozk(c, nrhs)) {
        rc = ozk_prepare(c);
        if (rc) return rc;
      } else {
        HPS_CK(c, df_from_d(c->df_T, c->d_T, (long long)c->E * c->nb * c->nb, st));
      }
    }
  }
  if (df) HPS_CK(c, df_from_d(c->df_rhs, c->fg_rhs, vs, st));
  double2* hbuf = c->fg_h;
  HPS_CK(c, bdot<double>(c->fg_rhs, 0, 1, c->fg_rhs, n, nrhs, c->fg_part, hbuf, 0, st));
  HPS_CK(c, cudaMemcpyAsync(c->pin_h, hbuf, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, st));
  HPS_CK(c, cudaStreamSynchronize(st));
  const auto t1 = std::chrono::steady_clock::now();
  std::vector<double> bnorm(nrhs);
  for (int r = 0; r < nrhs; ++r) bnorm[r] = std::sqrt(std::max(0.0, c->pin_h[r].x));
  if (df) HPS_CK(c, cudaMemsetAsync(c->df_x, 0, sizeof(float4) * (size_t)vs, st));
  else HPS_CK(c, zero<double>(c->fg_x, vs, st));

  // Explicit FP64 residual w = RHS - Pi M x of the current iterate and its squared norms in
  // hbuf[0..nrhs), on both paths.  The double-float path first rounds its iterate to FP64
  // (pv_in; that FP64 vector is also the one returned), forms the residual with the FP64
  // leaf maps in pv_out and restarts from it (rounded to double-float in df_w).
  auto residual = [&]() -> int {
    double2* w64 = df ? c->pv_out : c->fg_w;
    {
      PhaseScope ps(c, HPS_PH_MATVEC);
      if (df) HPS_CK(c, df_to_d(c->pv_in, c->df_x, vs, st));
      HPS_CK(c, es_matvec(c->d_T, c->d_es_nb, df ? c->pv_in : c->fg_x, c->fg_rhs, w64, c->E, c->nb, nrhs, grid, st));
    }
    HPS_CK(c, bdot<double>(w64, 0, 1, w64, n, nrhs, c->fg_part, hbuf, 0, st));
    if (df) HPS_CK(c, df_from_d(c->df_w, w64, vs, st));
    HPS_CK(c, cudaMemcpyAsync(c->pin_h, hbuf, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, st));
    HPS_CK(c, cudaStreamSynchronize(st));
    return HPS_OK;
  };

  std::vector<int> its(nrhs, 0);
  std::vector<char> done(nrhs, 0);
  std::vector<cd> H((size_t)(restart + 1) * restart * nrhs), g((size_t)(restart + 1) * nrhs);
  std::vector<double> cs((size_t)restart * nrhs);
  std::vector<cd> sn((size_t)restart * nrhs);
  std::vector<int> steps(nrhs);
  std::vector<double> res(nrhs, 0.0);
  bool fresh = false;  // pin_h holds the residual norms of the current iterate
  // Givens rotation of column col of right-hand side r (entries 0..col set, hn = H[col+1][col])
  auto rotate = [&](int r, int col, double hn) {
    cd* Hr = &H[(size_t)r * (restart + 1) * restart];
    double* csr = &cs[(size_t)r * restart];
    cd* snr = &sn[(size_t)r * restart];
    cd* gr = &g[(size_t)r * (restart + 1)];
    for (int i = 0; i < col; ++i) {
      const cd a = Hr[(size_t)i * restart + col], b = Hr[(size_t)(i + 1) * restart + col];
      Hr[(size_t)i * restart + col] = csr[i] * a + snr[i] * b;
      Hr[(size_t)(i + 1) * restart + col] = csr[i] * b - std::conj(snr[i]) * a;
    }
    const cd a = Hr[(size_t)col * restart + col];
    const double aa = std::abs(a);
    double cc;
    cd ss;
    if (hn == 0.0) { cc = 1.0; ss = 0.0; }
    else if (aa == 0.0) { cc = 0.0; ss = 1.0; }
    else {
      const double nu = std::hypot(aa, hn);
      cc = aa / nu;
      ss = (a / aa) * (hn / nu);
    }
    csr[col] = cc;
    snr[col] = ss;
    Hr[(size_t)col * restart + col] = cc * a + ss * hn;
    const cd gj = gr[col];
    gr[col] = cc * gj;
    gr[col + 1] = -std::conj(ss) * gj;
  };
  // host double -> double-float (re_hi, im_hi, re_lo, im_lo)
  auto to_df = [](cd v) {
    const float rh = (float)v.real(), ih = (float)v.imag();
    return make_float4(rh, ih, (float)(v.real() - (double)rh), (float)(v.imag() - (double)ih));
  };
  if (df) {
    // Two-pass Gram-Schmidt with the re-orthogonalisation lagged by one step.  Slot j of V
    // holds the tentative vector vt_j (once orthogonalised, normalised by an estimate) until
    // step j's reduction gives a = V_j^H vt_j, d = |vt_j|^2, b = V_j^H w_j, c = vt_j^H w_j,
    // e = |w_j|^2 in one pass; then v_j = (vt_j - V_j a) / rho with rho^2 = d - |a|^2 closes
    // column j-1 (H[:, j-1] += nu_{j-1} a, H[j][j-1] = nu_{j-1} rho), column j is
    // [b ; (c - a^H b) / rho], and one update pass writes v_j and
    // vt_{j+1} = (w_j - V_j b - h_jj v_j) / nu_j, nu_j^2 estimated as e - |b|^2 - |h_jj|^2.
    // z_j is the preconditioned tentative vector (flexible GMRES allows any direction); the
    // Arnoldi relation M Z = V H holds with the orthonormal final basis.
    std::vector<cd> htent((size_t)(restart + 1) * nrhs);
    std::vector<double> nu_prev(nrhs, 0.0), bet(nrhs, 0.0);
    for (int outer = 0; outer < max_outer; ++outer) {
      if (outer > 0) {
        rc = residual();
        if (rc) return rc;
      }
      fresh = true;
      bool all = true;
      std::vector<char> active(nrhs, 0);
      for (int r = 0; r < nrhs; ++r) {
        bet[r] = std::sqrt(std::max(0.0, c->pin_h[r].x));
        res[r] = bnorm[r] > 0 ? bet[r] / bnorm[r] : 0.0;
        done[r] = res[r] <= tol;
        active[r] = !done[r];
        all = all && done[r];
        for (int i = 0; i <= restart; ++i) g[(size_t)r * (restart + 1) + i] = 0.0;
        steps[r] = 0;
        c->pin_floor[r] = active[r] ? 0.0 : DBL_MAX;
      }
      if (all) break;
      fresh = false;
      HPS_CK(c, cudaMemcpyAsync(c->fg_floor, c->pin_floor, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
      if (outer == 0) HPS_CK(c, cudaMemcpyAsync(c->df_w, c->df_rhs, sizeof(float4) * vs, cudaMemcpyDeviceToDevice, st));
      HPS_CK(c, df_bscale(c->df_V, c->df_w, hbuf, c->fg_floor, n, nrhs, st));
      bool any = true;
      // When every active right-hand side is predicted to converge as column j-1 closes, step
      // j first closes it from the second-pass reduction alone, without preconditioning vt_j;
      // closed[r] marks a column already closed that way if the prediction fails.
      bool pred_close = false;
      std::vector<char> closed(nrhs, 0);
      for (int j = 0; j < restart && any; ++j) {
        float4* Vt = c->df_V + (size_t)j * vs;
        float2* Zj = c->df_Z + (size_t)j * vs;
        if (pred_close) {
          pred_close = false;
          {
            PhaseScope ps(c, HPS_PH_ORTHO);
            HPS_CK(c, df_dots2(c->df_V, vs, j + 1, Vt, Vt, n, nrhs, c->df_part, hbuf, st));
          }
          HPS_CK(c, cudaMemcpyAsync(c->pin_h, hbuf, sizeof(double2) * (size_t)(2 * (j + 1) + 1) * nrhs,
                                    cudaMemcpyDeviceToHost, st));
          HPS_CK(c, cudaStreamSynchronize(st));
          bool all_conv = true;
          for (int r = 0; r < nrhs; ++r) {
            if (!active[r]) continue;
            auto D = [&](int k) { const double2 v = c->pin_h[(size_t)k * nrhs + r]; return cd(v.x, v.y); };
            cd* Hr = &H[(size_t)r * (restart + 1) * restart];
            const cd* ht = &htent[(size_t)r * (restart + 1)];
            double sa = 0.0;
            for (int i = 0; i < j; ++i) sa += std::norm(D(2 * i));
            const double rho = std::sqrt(std::max(0.0, D(2 * j).real() - sa));
            for (int i = 0; i < j; ++i) Hr[(size_t)i * restart + (j - 1)] = ht[i] + nu_prev[r] * D(2 * i);
            const double hn = nu_prev[r] * rho;
            rotate(r, j - 1, hn);
            its[r] += 1;
            steps[r] = j;
            res[r] = bnorm[r] > 0 ? std::abs(g[(size_t)r * (restart + 1) + j]) / bnorm[r] : 0.0;
            closed[r] = 1;
            if (res[r] <= tol || hn <= 1e-300) active[r] = 0;
            else all_conv = false;
          }
          if (all_conv) {
            any = false;
            break;
          }
        }
        {
          PhaseScope ps(c, HPS_PH_PRECOND);
          if (inner_iters < 0) HPS_CK(c, df_swap_hi(Zj, Vt, c->d_es_nb, n, nrhs, st));
          else if ((rc = mg_apply_df(c, Vt, Zj, nrhs, inner_iters)) != HPS_OK) return rc;
        }
        {
          PhaseScope ps(c, HPS_PH_MATVEC);
          if ((rc = arnoldi_matvec(c, Zj, c->df_w, nrhs, grid)) != HPS_OK) return rc;
        }
        {
          PhaseScope ps(c, HPS_PH_ORTHO);
          HPS_CK(c, df_dots2(c->df_V, vs, j + 1, Vt, c->df_w, n, nrhs, c->df_part, hbuf, st));
        }
        HPS_CK(c, cudaMemcpyAsync(c->pin_h, hbuf, sizeof(double2) * (size_t)(2 * (j + 1) + 1) * nrhs,
                                  cudaMemcpyDeviceToHost, st));
        HPS_CK(c, cudaStreamSynchronize(st));
        any = false;
        bool pred_ok = true;
        const int rows_coef = 2 * j + 3;
        for (int r = 0; r < nrhs; ++r) {
          auto D = [&](int k) { const double2 v = c->pin_h[(size_t)k * nrhs + r]; return cd(v.x, v.y); };
          auto set_zero = [&]() {
            for (int k = 0; k < rows_coef; ++k) c->pin_coef[(size_t)k * nrhs + r] = make_float4(0.f, 0.f, 0.f, 0.f);
          };
          if (!active[r]) {
            set_zero();
            continue;
          }
          cd* Hr = &H[(size_t)r * (restart + 1) * restart];
          cd* ht = &htent[(size_t)r * (restart + 1)];
          double sa = 0.0;
          for (int i = 0; i < j; ++i) sa += std::norm(D(2 * i));
          const double rho = std::sqrt(std::max(0.0, D(2 * j).real() - sa));
          if (j > 0 && closed[r]) {
            closed[r] = 0;  // closed at the start of this step (a prediction that failed)
          } else if (j > 0) {  // close column j - 1
            for (int i = 0; i < j; ++i) Hr[(size_t)i * restart + (j - 1)] = ht[i] + nu_prev[r] * D(2 * i);
            const double hn = nu_prev[r] * rho;
            rotate(r, j - 1, hn);
            its[r] += 1;
            steps[r] = j;
            res[r] = bnorm[r] > 0 ? std::abs(g[(size_t)r * (restart + 1) + j]) / bnorm[r] : 0.0;
            if (res[r] <= tol || hn <= 1e-300) {
              active[r] = 0;
              set_zero();
              continue;
            }
          } else {
            g[(size_t)r * (restart + 1)] = bet[r] * rho;  // r0 = beta vt_0 = beta rho v_0
          }
          if (!(rho > 0.0)) {
            active[r] = 0;
            set_zero();
            continue;
          }
          cd ab = 0.0;
          double sb = 0.0;
          for (int i = 0; i < j; ++i) {
            ab += std::conj(D(2 * i)) * D(2 * i + 1);
            sb += std::norm(D(2 * i + 1));
            ht[i] = D(2 * i + 1);
          }
          const cd hjj = (D(2 * j + 1) - ab) / rho;
          ht[j] = hjj;
          const cd gam = hjj / rho;
          const double e = D(2 * (j + 1)).real();
          const double q = e - sb - std::norm(hjj);
          const double nu = std::sqrt(std::max(q, 1e-28 * e));
          if (!(nu > 0.0)) {
            active[r] = 0;
            set_zero();
            continue;
          }
          for (int i = 0; i < j; ++i) {
            c->pin_coef[(size_t)i * nrhs + r] = to_df(-D(2 * i) / rho);
            c->pin_coef[(size_t)(j + i) * nrhs + r] = to_df(-(D(2 * i + 1) - gam * D(2 * i)) / nu);
          }
          c->pin_coef[(size_t)(2 * j) * nrhs + r] = to_df(cd(1.0 / rho, 0.0));
          c->pin_coef[(size_t)(2 * j + 1) * nrhs + r] = to_df(cd(1.0 / nu, 0.0));
          c->pin_coef[(size_t)(2 * j + 2) * nrhs + r] = to_df(-gam / nu);
          nu_prev[r] = nu;
          any = true;
          // predicted residual once column j closes: the tentative column through the rotations
          // so far, subdiagonal nu (the second pass changes both by about the first pass's error)
          {
            const double* csr = &cs[(size_t)r * restart];
            const cd* snr = &sn[(size_t)r * restart];
            cd a = ht[0];
            for (int i = 0; i < j; ++i) a = csr[i] * ht[i + 1] - std::conj(snr[i]) * a;
            const double gmag = std::abs(g[(size_t)r * (restart + 1) + j]);
            const double pres = bnorm[r] > 0 ? gmag * nu / std::hypot(std::abs(a), nu) / bnorm[r] : 0.0;
            pred_ok = pred_ok && pres <= 0.999 * tol;
          }
        }
        if (!any) break;
        pred_close = pred_ok;
        HPS_CK(c, cudaMemcpyAsync(c->df_coef, c->pin_coef, sizeof(float4) * (size_t)rows_coef * nrhs,
                                  cudaMemcpyHostToDevice, st));
        PhaseScope ps(c, HPS_PH_ORTHO);
        HPS_CK(c, df_update2(c->df_V, vs, j, Vt, c->df_w, c->df_coef, Vt, c->df_V + (size_t)(j + 1) * vs, n, nrhs,
                             st));
      }
      // the last step's column is still open for the right-hand sides that kept going: close it
      bool open = false;
      for (int r = 0; r < nrhs; ++r) open = open || active[r];
      if (open) {
        const float4* Vl = c->df_V + (size_t)restart * vs;
        {
          PhaseScope ps(c, HPS_PH_ORTHO);
          HPS_CK(c, df_dots2(c->df_V, vs, restart + 1, Vl, Vl, n, nrhs, c->df_part, hbuf, st));
        }
        HPS_CK(c, cudaMemcpyAsync(c->pin_h, hbuf, sizeof(double2) * (size_t)(2 * (restart + 1) + 1) * nrhs,
                                  cudaMemcpyDeviceToHost, st));
        HPS_CK(c, cudaStreamSynchronize(st));
        for (int r = 0; r < nrhs; ++r) {
          if (!active[r]) continue;
          auto D = [&](int k) { const double2 v = c->pin_h[(size_t)k * nrhs + r]; return cd(v.x, v.y); };
          cd* Hr = &H[(size_t)r * (restart + 1) * restart];
          const cd* ht = &htent[(size_t)r * (restart + 1)];
          double sa = 0.0;
          for (int i = 0; i < restart; ++i) sa += std::norm(D(2 * i));
          const double rho = std::sqrt(std::max(0.0, D(2 * restart).real() - sa));
          for (int i = 0; i < restart; ++i) Hr[(size_t)i * restart + (restart - 1)] = ht[i] + nu_prev[r] * D(2 * i);
          rotate(r, restart - 1, nu_prev[r] * rho);
          its[r] += 1;
          steps[r] = restart;
          res[r] = bnorm[r] > 0 ? std::abs(g[(size_t)r * (restart + 1) + restart]) / bnorm[r] : 0.0;
        }
      }
      int jdone = 0;
      for (int r = 0; r < nrhs; ++r) jdone = std::max(jdone, steps[r]);
      if (jdone == 0) continue;
      for (int r = 0; r < nrhs; ++r) {
        const cd* Hr = &H[(size_t)r * (restart + 1) * restart];
        const cd* gr = &g[(size_t)r * (restart + 1)];
        std::vector<cd> y(jdone, 0.0);
        for (int i = steps[r] - 1; i >= 0; --i) {
          cd v = gr[i];
          for (int l = i + 1; l < steps[r]; ++l) v -= Hr[(size_t)i * restart + l] * y[l];
          const cd d = Hr[(size_t)i * restart + i];
          y[i] = std::abs(d) > 0 ? v / d : 0.0;
        }
        for (int i = 0; i < jdone; ++i) c->pin_y[(size_t)i * nrhs + r] = make_double2(y[i].real(), y[i].imag());
      }
      HPS_CK(c, cudaMemcpyAsync(c->fg_y, c->pin_y, sizeof(double2) * (size_t)jdone * nrhs, cudaMemcpyHostToDevice, st));
      HPS_CK(c, df_bupdate<float2>(c->df_x, c->df_Z, vs, jdone, c->fg_y, n, nrhs, 1.f, st));
    }
  } else
  for (int outer = 0; outer < max_outer; ++outer) {
    // explicit residual w = rhs - Pi M x (x = 0 at the start: w = rhs, norms already in hbuf)
    if (outer > 0) {
      rc = residual();
      if (rc) return rc;
    }
    fresh = true;
    bool all = true;
    std::vector<char> active(nrhs, 0);
    for (int r = 0; r < nrhs; ++r) {
      const double beta = std::sqrt(std::max(0.0, c->pin_h[r].x));
      res[r] = bnorm[r] > 0 ? beta / bnorm[r] : 0.0;
      done[r] = res[r] <= tol;
      active[r] = !done[r];
      all = all && done[r];
      for (int i = 0; i <= restart; ++i) g[(size_t)r * (restart + 1) + i] = 0.0;
      g[(size_t)r * (restart + 1)] = beta;
      steps[r] = 0;
      c->pin_floor[r] = active[r] ? 0.0 : DBL_MAX;
    }
    if (all) break;
    fresh = false;
    HPS_CK(c, cudaMemcpyAsync(c->fg_floor, c->pin_floor, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
    if (df) {
      if (outer == 0) HPS_CK(c, cudaMemcpyAsync(c->df_w, c->df_rhs, sizeof(float4) * vs, cudaMemcpyDeviceToDevice, st));
      HPS_CK(c, df_bscale(c->df_V, c->df_w, hbuf, c->fg_floor, n, nrhs, st));
    } else {
      HPS_CK(c, bscale<double>(c->fg_V, outer > 0 ? c->fg_w : c->fg_rhs, hbuf, c->fg_floor, n, nrhs, st));
    }
    int jdone = 0;
    for (int j = 0; j < restart; ++j) {
      double2* h1 = hbuf;
      double2* h2 = hbuf + (size_t)(restart + 1) * nrhs;
      double2* nr = hbuf + (size_t)2 * (restart + 1) * nrhs;
      if (df) {
        const float4* Vj = c->df_V + (size_t)j * vs;
        float2* Zj = c->df_Z + (size_t)j * vs;
        {
          PhaseScope ps(c, HPS_PH_PRECOND);
          if (inner_iters < 0) HPS_CK(c, df_swap_hi(Zj, Vj, c->d_es_nb, n, nrhs, st));
          else if ((rc = mg_apply_df(c, Vj, Zj, nrhs, inner_iters)) != HPS_OK) return rc;
        }
        {
          PhaseScope ps(c, HPS_PH_MATVEC);
          if ((rc = arnoldi_matvec(c, Zj, c->df_w, nrhs, grid)) != HPS_OK) return rc;
        }
        PhaseScope ps(c, HPS_PH_ORTHO);
        HPS_CK(c, df_bdot(c->df_V, vs, j + 1, c->df_w, n, nrhs, c->df_part, h1, st));
        HPS_CK(c, df_bupdate<float4>(c->df_w, c->df_V, vs, j + 1, h1, n, nrhs, -1.f, st));
        HPS_CK(c, df_bdot(c->df_V, vs, j + 1, c->df_w, n, nrhs, c->df_part, h2, st));
        HPS_CK(c, df_bupdate<float4>(c->df_w, c->df_V, vs, j + 1, h2, n, nrhs, -1.f, st));
        HPS_CK(c, df_bdot(c->df_w, 0, 1, c->df_w, n, nrhs, c->df_part, nr, st));
      } else {
        double2* Vj = c->fg_V + (size_t)j * vs;
        double2* Zj = c->fg_Z + (size_t)j * vs;
        rc = precond(c, Vj, Zj, nrhs, inner_iters);
        if (rc) return rc;
        {
          PhaseScope ps(c, HPS_PH_MATVEC);
          HPS_CK(c, es_matvec(c->d_T, c->d_es_nb, Zj, nullptr, c->fg_w, c->E, c->nb, nrhs, grid, st));
        }
        PhaseScope ps(c, HPS_PH_ORTHO);
        HPS_CK(c, bdot<double>(c->fg_V, vs, j + 1, c->fg_w, n, nrhs, c->fg_part, h1, 0, st));
        HPS_CK(c, (bupdate<double, double>(c->fg_w, c->fg_V, vs, j + 1, h1, n, nrhs, -1.0, st)));
        HPS_CK(c, bdot<double>(c->fg_V, vs, j + 1, c->fg_w, n, nrhs, c->fg_part, h2, 0, st));
        HPS_CK(c, (bupdate<double, double>(c->fg_w, c->fg_V, vs, j + 1, h2, n, nrhs, -1.0, st)));
        HPS_CK(c, bdot<double>(c->fg_w, 0, 1, c->fg_w, n, nrhs, c->fg_part, nr, 0, st));
      }
      HPS_CK(c, cudaMemcpyAsync(c->pin_h, hbuf, sizeof(double2) * (size_t)(2 * (restart + 1) + 1) * nrhs,
                                cudaMemcpyDeviceToHost, st));
      HPS_CK(c, cudaStreamSynchronize(st));
      jdone = j + 1;
      bool any = false;
      for (int r = 0; r < nrhs; ++r) {
        if (!active[r]) continue;
        cd* Hr = &H[(size_t)r * (restart + 1) * restart];
        for (int i = 0; i <= j; ++i) {
          const double2 a = c->pin_h[(size_t)i * nrhs + r];
          const double2 b = c->pin_h[(size_t)(restart + 1) * nrhs + (size_t)i * nrhs + r];
          Hr[(size_t)i * restart + j] = cd(a.x + b.x, a.y + b.y);
        }
        const double hn = std::sqrt(std::max(0.0, c->pin_h[(size_t)2 * (restart + 1) * nrhs + r].x));
        double* csr = &cs[(size_t)r * restart];
        cd* snr = &sn[(size_t)r * restart];
        cd* gr = &g[(size_t)r * (restart + 1)];
        for (int i = 0; i < j; ++i) {
          const cd a = Hr[(size_t)i * restart + j], b = Hr[(size_t)(i + 1) * restart + j];
          Hr[(size_t)i * restart + j] = csr[i] * a + snr[i] * b;
          Hr[(size_t)(i + 1) * restart + j] = csr[i] * b - std::conj(snr[i]) * a;
        }
        const cd a = Hr[(size_t)j * restart + j];
        const double aa = std::abs(a);
        double cc;
        cd ss;
        if (hn == 0.0) { cc = 1.0; ss = 0.0; }
        else if (aa == 0.0) { cc = 0.0; ss = 1.0; }
        else {
          const double nu = std::hypot(aa, hn);
          cc = aa / nu;
          ss = (a / aa) * (hn / nu);
        }
        csr[j] = cc;
        snr[j] = ss;
        Hr[(size_t)j * restart + j] = cc * a + ss * hn;
        const cd gj = gr[j];
        gr[j] = cc * gj;
        gr[j + 1] = -std::conj(ss) * gj;
        its[r] += 1;
        steps[r] = j + 1;
        res[r] = bnorm[r] > 0 ? std::abs(gr[j + 1]) / bnorm[r] : 0.0;
        if (res[r] <= tol || hn <= 1e-300) active[r] = 0;
        else any = true;
      }
      if (!any) break;
      if (j + 1 < restart) {
        for (int r = 0; r < nrhs; ++r) c->pin_floor[r] = active[r] ? 0.0 : DBL_MAX;
        HPS_CK(c, cudaMemcpyAsync(c->fg_floor, c->pin_floor, sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
        if (df) HPS_CK(c, df_bscale(c->df_V + (size_t)(j + 1) * vs, c->df_w, nr, c->fg_floor, n, nrhs, st));
        else HPS_CK(c, bscale<double>(c->fg_V + (size_t)(j + 1) * vs, c->fg_w, nr, c->fg_floor, n, nrhs, st));
      }
    }
    // y = R^{-1} g per right-hand side, then x += Z y
    for (int r = 0; r < nrhs; ++r) {
      const cd* Hr = &H[(size_t)r * (restart + 1) * restart];
      const cd* gr = &g[(size_t)r * (restart + 1)];
      std::vector<cd> y(jdone, 0.0);
      for (int i = steps[r] - 1; i >= 0; --i) {
        cd v = gr[i];
        for (int l = i + 1; l < steps[r]; ++l) v -= Hr[(size_t)i * restart + l] * y[l];
        const cd d = Hr[(size_t)i * restart + i];
        y[i] = std::abs(d) > 0 ? v / d : 0.0;
      }
      for (int i = 0; i < jdone; ++i) c->pin_y[(size_t)i * nrhs + r] = make_double2(y[i].real(), y[i].imag());
    }
    HPS_CK(c, cudaMemcpyAsync(c->fg_y, c->pin_y, sizeof(double2) * (size_t)jdone * nrhs, cudaMemcpyHostToDevice, st));
    if (df) HPS_CK(c, df_bupdate<float2>(c->df_x, c->df_Z, vs, jdone, c->fg_y, n, nrhs, 1.f, st));
    else HPS_CK(c, (bupdate<double, double>(c->fg_x, c->fg_Z, vs, jdone, c->fg_y, n, nrhs, 1.0, st)));
  }
  PhaseScope ps_other(c, HPS_PH_OTHER);
  // explicit residual of the returned iterate (already at hand when the last restart converged)
  if (!fresh) {
    rc = residual();
    if (rc) return rc;
  }
  std::vector<double> nrm2(nrhs);
  for (int r = 0; r < nrhs; ++r) nrm2[r] = c->pin_h[r].x;
  // solution in skeleton order (df: the FP64 iterate whose residual was just formed, in pv_in)
  const double2* x64 = df ? c->pv_in : c->fg_x;
  double2* gdev = static_cast<double2*>(g_out);
  const bool host_out = !is_device_ptr(g_out);
  if (host_out) gdev = c->pv_out;
  HPS_CK(c, rows_to_user(gdev, x64, c->d_es_in, n, nrhs, c->n_skel, st));
  if (host_out)
    HPS_CK(c, cudaMemcpyAsync(g_out, gdev, sizeof(double2) * (size_t)c->n_skel * nrhs, cudaMemcpyDeviceToHost, st));
  int gerr = 0;
  HPS_CK(c, cudaMemcpyAsync(&gerr, c->d_gemm_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HPS_CK(c, cudaStreamSynchronize(st));
  if (gerr) {
    cudaMemsetAsync(c->d_gemm_err, 0, sizeof(int), st);
    return fail(c, HPS_ETIMEOUT, "a tensor-core GEMM of the preconditioner timed out waiting for its MMAs");
  }
  int nconv = 0, maxit = 0;
  double maxres = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    res[r] = bnorm[r] > 0 ? std::sqrt(std::max(0.0, nrm2[r])) / bnorm[r] : 0.0;
    nconv += res[r] <= tol;
    maxit = std::max(maxit, its[r]);
    maxres = std::max(maxres, res[r]);
  }
  const auto t2 = std::chrono::steady_clock::now();
  if (info) {
    info->outer_iterations = maxit;
    info->converged = nconv;
    info->max_rel_residual = maxres;
    if (info->iterations)
      for (int r = 0; r < nrhs; ++r) info->iterations[r] = its[r];
    if (info->rel_residual)
      for (int r = 0; r < nrhs; ++r) info->rel_residual[r] = res[r];
    info->ms_rhs = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->ms_solve = std::chrono::duration<double, std::milli>(t2 - t1).count();
  }
  if (nconv < nrhs) return fail(c, HPS_ENOTCONV, "FGMRES stopped before the tolerance");
  return HPS_OK;
}

}  // extern "C"
