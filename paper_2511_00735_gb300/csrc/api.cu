// C ABI of libhps: context, mesh and index maps, coefficient, leaf build,
// RHS / matvec / preconditioner entry points and the FP64 flexible GMRES.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "ctx.h"
#include "skel.cuh"

namespace hps {

static std::atomic<long long> g_launches{0};
static thread_local long long* tl_phase_launch = nullptr;

void note_launch(int n) {
  g_launches += n;
  if (tl_phase_launch) *tl_phase_launch += n;
}

static cudaEvent_t get_event(hps_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

PhaseScope::PhaseScope(hps_ctx* ctx, int phase) : c(ctx), ph(phase), prev(tl_phase_launch), prev_phase(ctx->cur_phase) {
  tl_phase_launch = &c->prof_launch[ph];
  c->prof_calls[ph] += 1;
  c->cur_phase = ph;
  if (c->prof) {
    a = get_event(c);
    if (a) cudaEventRecord(a, c->stream);
  }
}

PhaseScope::~PhaseScope() {
  tl_phase_launch = prev;
  c->cur_phase = prev_phase;
  if (c->prof && a) {
    cudaEvent_t b = get_event(c);
    if (b) {
      cudaEventRecord(b, c->stream);
      c->prof_ev.push_back({ph, {a, b}});
    } else {
      c->ev_pool.push_back(a);
    }
  }
}

static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;  // unknown: treat as capturing (no event records)
  }
  return cs != cudaStreamCaptureStatusNone;
}

KernScope::KernScope(hps_ctx* ctx, int kclass, double bytes, double flops) : c(ctx), kc(kclass) {
  if (!c->kprof || kc < 0 || kc >= HPS_NKC || stream_capturing(c->stream)) return;
  a = get_event(c);
  if (!a) return;
  cudaEventRecord(a, c->stream);
  c->kprof_bytes[kc] += bytes;
  c->kprof_flops[kc] += flops;
  c->kprof_launch[kc] += 1;
}

KernScope::~KernScope() {
  if (!a) return;
  cudaEvent_t b = get_event(c);
  if (b) {
    cudaEventRecord(b, c->stream);
    c->kprof_ev.push_back({kc, a, b});
  } else {
    c->ev_pool.push_back(a);
  }
}

static void kprof_collect(hps_ctx* c) {
  if (c->kprof_ev.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& ke : c->kprof_ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ke.a, ke.b) == cudaSuccess) c->kprof_ms[ke.kc] += ms;
    else cudaGetLastError();
    c->ev_pool.push_back(ke.a);
    c->ev_pool.push_back(ke.b);
  }
  c->kprof_ev.clear();
}

static void prof_collect(hps_ctx* c) {
  if (c->prof_ev.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& pe : c->prof_ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) c->prof_ms[pe.first] += ms;
    else cudaGetLastError();
    c->ev_pool.push_back(pe.second.first);
    c->ev_pool.push_back(pe.second.second);
  }
  c->prof_ev.clear();
}

int fail(hps_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(hps_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, HPS_ENOMEM, m);
  return fail(c, HPS_ECUDA, m);
}

void* dev_alloc(hps_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, c->alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    c->allocs.push_back({p, bytes});
    c->bytes_held += bytes;
  }
  return p;
}

// Frees an allocation of this context; a pointer the context does not hold (already
// released, e.g. by hps_mesh's release of everything) is ignored, never freed twice.
void dev_free(hps_ctx* c, void* p) {
  if (!p) return;
  bool held = false;
  for (size_t i = 0; i < c->allocs.size(); ++i) {
    if (c->allocs[i].p == p) {
      c->bytes_held -= c->allocs[i].bytes;
      c->allocs.erase(c->allocs.begin() + i);
      held = true;
      break;
    }
  }
  if (!held) return;
  if (c->free_fn) c->free_fn(p, c->alloc_user);
  else cudaFree(p);
}

template <typename T>
T* dev_upload(hps_ctx* c, const std::vector<T>& v) {
  T* p = static_cast<T*>(dev_alloc(c, sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (!p) return nullptr;
  if (!v.empty() && cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
  return p;
}
template int* dev_upload<int>(hps_ctx*, const std::vector<int>&);
template double* dev_upload<double>(hps_ctx*, const std::vector<double>&);
template GemmDesc* dev_upload<GemmDesc>(hps_ctx*, const std::vector<GemmDesc>&);

#define FREE(ptr)            \
  do {                       \
    dev_free(c, (void*)ptr); \
    ptr = nullptr;           \
  } while (0)

void free_solver(hps_ctx* c) {
  free_fg(c);  // the FGMRES workspace (FP64 and double-float buffers, pinned mirrors)
  free_vol(c);
  free_vol_staging(c);
  FREE(c->pv_in); FREE(c->pv_out);
  c->pv_nrhs = 0;
}

// The captured V-cycle graph, its stream and events; the handles are reset, so a later
// solve captures again.
void free_graph(hps_ctx* c) {
  if (c->mg_exec) cudaGraphExecDestroy(c->mg_exec);
  if (c->gs) cudaStreamDestroy(c->gs);
  if (c->gs_in) cudaEventDestroy(c->gs_in);
  if (c->gs_out) cudaEventDestroy(c->gs_out);
  c->mg_exec = nullptr;
  c->gs = nullptr;
  c->gs_in = c->gs_out = nullptr;
  c->mg_gen = -1;
}

void free_numeric(hps_ctx* c) {
  for (auto& s : c->stages) {
    FREE(s.T); FREE(s.vec); FREE(s.gR); FREE(s.gE);
  }
  FREE(c->gW);
  c->gamma_nrhs = 0;
  for (auto& l : c->levels) {
    FREE(l.W); FREE(l.U); FREE(l.Dm); FREE(l.Ut); FREE(l.Dmt);
  }
  FREE(c->coarse.Winv); FREE(c->coarse.d_desc); FREE(c->coarse.Tt);
  FREE(c->gemm_ws); c->gemm_ws_elems = 0;
  FREE(c->ws_X1); FREE(c->ws_X2); FREE(c->d_piv); FREE(c->d_lu);
  FREE(c->sw_x); FREE(c->ws_G); FREE(c->d_eye);
  FREE(c->cg_V); FREE(c->cg_w); FREE(c->cg_W); FREE(c->cg_H); FREE(c->cg_h1); FREE(c->cg_h2);
  FREE(c->cg_nrm); FREE(c->cg_y); FREE(c->cg_g); FREE(c->cg_s); FREE(c->cg_part);
  FREE(c->cg_beta); FREE(c->cg_floor); FREE(c->cg_c); FREE(c->cg_inv); FREE(c->cg_cnt);
  FREE(c->ex_r); FREE(c->ex_e);
  c->ws_X_elems = 0;
  c->nrhs_cap = 0;
  c->cg_k = c->cg_nrhs = c->ex_nrhs = 0;
  c->have_tree = false;
  ++c->vc_gen;
}

void free_tree(hps_ctx* c) {
  free_numeric(c);
  for (auto& s : c->stages) {
    FREE(s.d_es); FREE(s.d_nb); FREE(s.d_tdesc);
  }
  for (auto& l : c->levels) {
    FREE(l.d_dst); FREE(l.d_up); FREE(l.d_xmap); FREE(l.d_mdesc); FREE(l.d_sdesc); FREE(l.d_tsdesc);
  }
  c->stages.clear();
  c->levels.clear();
  FREE(c->coarse.d_cdesc); FREE(c->coarse.d_cnb); FREE(c->coarse.d_upos); FREE(c->coarse.d_ucnb);
  FREE(c->coarse.d_tcdesc);
  c->coarse = Coarse();
  FREE(c->plan_map0);
  c->plan_L = -1;
}

// ---------------------------------------------------------------------------
// Reference GLL rule on [-1, 1] (nodes -1, +1 and the roots of P_N', weights
// 2 / (N (N+1) P_N(x)^2), differentiation matrix from the Lagrange basis),
// written here independently of any other implementation in the repository.
// ---------------------------------------------------------------------------
static void legendre_pair(int N, double x, double& pN, double& pNm1) {
  double a = 1.0, b = x;
  if (N == 0) { pN = 1.0; pNm1 = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    const double nxt = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b;
    b = nxt;
  }
  pN = b;
  pNm1 = a;
}

static void gll_build(int N, std::vector<double>& x, std::vector<double>& w, std::vector<double>& D) {
  x.assign(N + 1, 0.0);
  w.assign(N + 1, 0.0);
  D.assign((N + 1) * (N + 1), 0.0);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double p, pm;
      legendre_pair(N, t, p, pm);
      const double dp = N * (pm - t * p) / (1.0 - t * t);
      const double d2 = (2.0 * t * dp - N * (N + 1.0) * p) / (1.0 - t * t);
      const double dx = dp / d2;
      t -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[j] = t;
  }
  std::vector<double> P(N + 1);
  for (int j = 0; j <= N; ++j) {
    double pm;
    legendre_pair(N, x[j], P[j], pm);
    w[j] = 2.0 / (N * (N + 1.0) * P[j] * P[j]);
  }
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j)
      if (i != j) D[i * (N + 1) + j] = P[i] / (P[j] * (x[i] - x[j]));
  D[0] = -N * (N + 1.0) / 4.0;
  D[N * (N + 1) + N] = N * (N + 1.0) / 4.0;
}

// Smallest eigenvalue of the symmetric matrix A (n x n, row-major) by cyclic Jacobi rotations.
static double min_eig_sym(std::vector<double> A, int n) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = cs * akp - sn * akq;
          A[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = cs * apk - sn * aqk;
          A[q * n + k] = sn * apk + cs * aqk;
        }
      }
  }
  double m = A[0];
  for (int i = 1; i < n; ++i) m = std::min(m, A[i * n + i]);
  return m;
}

// Eigen-decomposition A = U diag(lam) U^T of a symmetric n x n matrix by cyclic Jacobi
// rotations; U's columns are the eigenvectors (row-major U[i * n + k] = component i of vector k).
static void eig_sym(std::vector<double> A, int n, std::vector<double>& lam, std::vector<double>& U) {
  U.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) U[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = cs * akp - sn * akq;
          A[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = cs * apk - sn * aqk;
          A[q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double ukp = U[(size_t)k * n + p], ukq = U[(size_t)k * n + q];
          U[(size_t)k * n + p] = cs * ukp - sn * ukq;
          U[(size_t)k * n + q] = sn * ukp + cs * ukq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

static inline int opp_side(int s) { return s ^ 1; }

}  // namespace hps

using namespace hps;

#define CHECK_CTX(c)                                  \
  do {                                                \
    if (!(c)) return HPS_EINVAL;                      \
    cudaError_t e0_ = cudaSetDevice((c)->device);     \
    if (e0_ != cudaSuccess) return cuda_fail(c, e0_, "cudaSetDevice"); \
  } while (0)

namespace hps {
void optin_all_once() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  optin_leaf();
  optin_blas();
  optin_df64();
  optin_skel();
  optin_tc();
  optin_ozk();
  optin_volume();
  done[dev] = true;
}
}  // namespace hps

extern "C" {

const char* hps_strerror(int s) {
  switch (s) {
    case HPS_OK: return "ok";
    case HPS_EINVAL: return "invalid argument";
    case HPS_ENOMEM: return "device allocation failed";
    case HPS_ENOTBUILT: return "prerequisite call missing";
    case HPS_ENOTCONV: return "FGMRES did not reach the tolerance";
    case HPS_ETIMEOUT: return "bounded device wait gave up";
    case HPS_ECUDA: return "CUDA runtime error";
    case HPS_ENODEV: return "no usable CUDA device";
    case HPS_EUNSUPPORTED: return "input not supported by this build";
    case HPS_ENUMERIC: return "factorisation broke down";
    default: return "unknown status";
  }
}

const char* hps_last_error(hps_ctx* c) { return c ? c->err.c_str() : "null context"; }

int hps_create(hps_ctx** out, int device, void* stream) {
  if (!out) return HPS_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return HPS_ENODEV;
  }
  if (device < 0 || device >= n) return HPS_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ENODEV;
  }
  optin_all_once();
  hps_ctx* c = new hps_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&c->d_flag, sizeof(int)) != cudaSuccess || cudaMalloc(&c->d_gemm_err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->d_cerr, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->pin_counts, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->d_flag);
    cudaFree(c->d_gemm_err);
    cudaFree(c->d_cerr);
    cudaFreeHost(c->pin_counts);
    delete c;
    return HPS_ENOMEM;
  }
  cudaMemset(c->d_flag, 0, sizeof(int));
  cudaMemset(c->d_gemm_err, 0, sizeof(int));
  cudaMemset(c->d_cerr, 0, sizeof(int));
  *out = c;
  return HPS_OK;
}

int hps_destroy(hps_ctx* c) {
  if (!c) return HPS_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_tree(c);
  free_solver(c);
  free_graph(c);
  while (!c->allocs.empty()) dev_free(c, c->allocs.back().p);
  c->mg_ptr = nullptr;  // freed with every other allocation
  cudaFree(c->d_flag);
  cudaFree(c->d_gemm_err);
  cudaFree(c->d_cerr);
  cudaFreeHost(c->pin_counts);
  for (auto& pe : c->prof_ev) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (auto& ke : c->kprof_ev) {
    cudaEventDestroy(ke.a);
    cudaEventDestroy(ke.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return HPS_OK;
}

int hps_set_allocator(hps_ctx* c, hps_alloc_fn a, hps_free_fn f, void* user) {
  if (!c) return HPS_EINVAL;
  if (c->have_mesh || !c->allocs.empty()) return fail(c, HPS_EINVAL, "allocator must be set before hps_mesh");
  if ((a == nullptr) != (f == nullptr)) return fail(c, HPS_EINVAL, "alloc and free must both be set or both NULL");
  c->alloc = a;
  c->free_fn = f;
  c->alloc_user = user;
  return HPS_OK;
}

int hps_mesh(hps_ctx* c, int nx, int ny, int N) {
  CHECK_CTX(c);
  if (nx != ny || nx < 2 || (nx & (nx - 1)) != 0)
    return fail(c, HPS_EINVAL, "nx == ny == 2^k with k >= 1 required");
  if (N < 2 || N > 24) return fail(c, HPS_EINVAL, "2 <= N <= 24 required");
  cudaStreamSynchronize(c->stream);
  free_tree(c);
  free_solver(c);
  free_graph(c);
  while (!c->allocs.empty()) dev_free(c, c->allocs.back().p);
  c->mg_ptr = nullptr;  // freed with every other allocation
  c->d_es_nb = c->d_es_in = c->d_es_out = c->d_es_bdry = c->d_bdry_rows = nullptr;
  c->d_Dref = c->d_Kref = c->d_wref = c->d_vtab = nullptr;
  c->d_c = c->d_bstage = nullptr;
  c->d_route = c->d_lists = nullptr;
  c->d_T = nullptr;
  c->have_mesh = c->have_coeff = c->have_leaves = c->have_tree = false;

  c->nx = nx; c->ny = ny; c->N = N; c->q = N - 1; c->E = nx * ny; c->nb = 4 * c->q;
  int k = 0;
  while ((1 << k) < nx) ++k;
  c->L = 2 * k;
  c->h = 1.0 / nx;
  const int q = c->q, E = c->E;
  const long long nfaces = (long long)(nx - 1) * ny + (long long)nx * (ny - 1);
  c->n_skel = 2 * nfaces * q;
  c->n_bdry = 2LL * (nx + ny) * q;
  c->n_es = (long long)E * c->nb;

  gll_build(N, c->xi, c->wref, c->Dref);
  const int n1 = N + 1;
  c->Kref.assign(n1 * n1, 0.0);
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) {
      double s = 0.0;
      for (int l = 0; l < n1; ++l) s += c->Dref[l * n1 + i] * c->wref[l] * c->Dref[l * n1 + j];
      c->Kref[i * n1 + j] = s;
    }
  // mu_min of K_ii w.r.t. W_ii: eigenvalues of W^{-1/2} K W^{-1/2} on the interior nodes
  std::vector<double> S(q * q);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j)
      S[i * q + j] = c->Kref[(i + 1) * n1 + (j + 1)] / std::sqrt(c->wref[i + 1] * c->wref[j + 1]);
  c->mu_min = min_eig_sym(S, q);

  // element-side maps
  c->es_nb.assign(c->n_es, -1);
  c->es_in.assign(c->n_es, -1);
  c->es_out.assign(c->n_es, -1);
  c->es_bdry.assign(c->n_es, -1);
  auto face_v = [&](int ix, int iy) { return (long long)ix + (long long)(nx - 1) * iy; };
  auto face_h = [&](int ix, int iy) { return (long long)(nx - 1) * ny + ix + (long long)nx * iy; };
  for (int e = 0; e < E; ++e) {
    const int ix = e % nx, iy = e / nx;
    for (int s = 0; s < 4; ++s) {
      int nbe = -1;
      long long f = -1;
      int slot = 0, bpos = -1;
      if (s == 0) {
        if (ix > 0) { nbe = e - 1; f = face_v(ix - 1, iy); slot = 1; } else bpos = iy;
      } else if (s == 1) {
        if (ix < nx - 1) { nbe = e + 1; f = face_v(ix, iy); slot = 0; } else bpos = ny + iy;
      } else if (s == 2) {
        if (iy > 0) { nbe = e - nx; f = face_h(ix, iy - 1); slot = 1; } else bpos = 2 * ny + ix;
      } else {
        if (iy < ny - 1) { nbe = e + nx; f = face_h(ix, iy); slot = 0; } else bpos = 2 * ny + nx + ix;
      }
      for (int kk = 0; kk < q; ++kk) {
        const long long p = ((long long)e * 4 + s) * q + kk;
        if (nbe >= 0) {
          c->es_nb[p] = (int)(((long long)nbe * 4 + opp_side(s)) * q + kk);
          c->es_in[p] = (int)((2 * f + slot) * q + kk);
        } else {
          c->es_bdry[p] = bpos * q + kk;
        }
      }
    }
  }
  for (long long p = 0; p < c->n_es; ++p)
    if (c->es_nb[p] >= 0) c->es_out[p] = c->es_in[c->es_nb[p]];

  std::vector<int> brow(c->n_bdry);
  for (long long i = 0; i < c->n_bdry; ++i) brow[i] = (int)i;
  c->d_es_nb = dev_upload(c, c->es_nb);
  c->d_es_in = dev_upload(c, c->es_in);
  c->d_es_out = dev_upload(c, c->es_out);
  c->d_es_bdry = dev_upload(c, c->es_bdry);
  c->d_bdry_rows = dev_upload(c, brow);
  c->d_Dref = dev_upload(c, c->Dref);
  c->d_Kref = dev_upload(c, c->Kref);
  c->d_wref = dev_upload(c, c->wref);
  {
    // interior solve and corner tables (volume.cu): S = V^{-1} K_ii V^{-1} = U diag(lam) U^T with
    // V = diag(w_i^1/2) on the interior nodes, V's diagonal, and the corner extrapolation weights
    // (Lagrange basis of the interior nodes at -1 and +1)
    std::vector<double> U, lam;
    eig_sym(S, q, lam, U);
    std::vector<double> tab(2 * q * q + 4 * q);
    std::copy(S.begin(), S.end(), tab.begin());
    std::copy(U.begin(), U.end(), tab.begin() + q * q);
    for (int i = 0; i < q; ++i) {
      tab[2 * q * q + i] = lam[i];
      tab[2 * q * q + q + i] = std::sqrt(c->wref[i + 1]);
      double wl = 1.0, wr = 1.0;
      for (int k = 0; k < q; ++k) {
        if (k == i) continue;
        wl *= (-1.0 - c->xi[k + 1]) / (c->xi[i + 1] - c->xi[k + 1]);
        wr *= (1.0 - c->xi[k + 1]) / (c->xi[i + 1] - c->xi[k + 1]);
      }
      tab[2 * q * q + 2 * q + i] = wl;
      tab[2 * q * q + 3 * q + i] = wr;
    }
    c->d_vtab = dev_upload(c, tab);
  }
  if (!c->d_vtab || !c->d_es_nb || !c->d_es_in || !c->d_es_out || !c->d_es_bdry || !c->d_bdry_rows || !c->d_Dref || !c->d_Kref ||
      !c->d_wref)
    return fail(c, HPS_ENOMEM, "index maps");
  c->have_mesh = true;
  return HPS_OK;
}

int hps_sizes(hps_ctx* c, long long* n_skel, long long* n_bdry, int* levels, long long* bytes_held) {
  if (!c) return HPS_EINVAL;
  if (!c->have_mesh) return fail(c, HPS_ENOTBUILT, "hps_mesh first");
  if (n_skel) *n_skel = c->n_skel;
  if (n_bdry) *n_bdry = c->n_bdry;
  if (levels) *levels = c->L;
  if (bytes_held) *bytes_held = (long long)c->bytes_held;
  return HPS_OK;
}

int hps_node_coords(hps_ctx* c, double* x, double* y) {
  if (!c || !x || !y) return HPS_EINVAL;
  if (!c->have_mesh) return fail(c, HPS_ENOTBUILT, "hps_mesh first");
  const int n1 = c->N + 1;
  for (int e = 0; e < c->E; ++e) {
    const int ix = e % c->nx, iy = e / c->nx;
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) {
        const long long o = (long long)e * n1 * n1 + i * n1 + j;
        x[o] = ix * c->h + (c->xi[i] + 1.0) * c->h / 2.0;
        y[o] = iy * c->h + (c->xi[j] + 1.0) * c->h / 2.0;
      }
  }
  return HPS_OK;
}

int hps_boundary_points(hps_ctx* c, double* x, double* y, double* nxo, double* nyo) {
  if (!c || !x || !y || !nxo || !nyo) return HPS_EINVAL;
  if (!c->have_mesh) return fail(c, HPS_ENOTBUILT, "hps_mesh first");
  const int q = c->q;
  for (int e = 0; e < c->E; ++e) {
    const int ix = e % c->nx, iy = e / c->nx;
    for (int s = 0; s < 4; ++s)
      for (int k = 0; k < q; ++k) {
        const long long p = ((long long)e * 4 + s) * q + k;
        const int b = c->es_bdry[p];
        if (b < 0) continue;
        const double t = (c->xi[k + 1] + 1.0) * c->h / 2.0;
        double X, Y, NX, NY;
        if (s == 0) { X = ix * c->h; Y = iy * c->h + t; NX = -1; NY = 0; }
        else if (s == 1) { X = (ix + 1) * c->h; Y = iy * c->h + t; NX = 1; NY = 0; }
        else if (s == 2) { X = ix * c->h + t; Y = iy * c->h; NX = 0; NY = -1; }
        else { X = ix * c->h + t; Y = (iy + 1) * c->h; NX = 0; NY = 1; }
        x[b] = X; y[b] = Y; nxo[b] = NX; nyo[b] = NY;
      }
  }
  return HPS_OK;
}

int hps_index_maps(hps_ctx* c, int* skel_in, int* skel_out, int* bdry) {
  if (!c) return HPS_EINVAL;
  if (!c->have_mesh) return fail(c, HPS_ENOTBUILT, "hps_mesh first");
  if (skel_in) std::memcpy(skel_in, c->es_in.data(), sizeof(int) * c->n_es);
  if (skel_out) std::memcpy(skel_out, c->es_out.data(), sizeof(int) * c->n_es);
  if (bdry) std::memcpy(bdry, c->es_bdry.data(), sizeof(int) * c->n_es);
  return HPS_OK;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int hps_set_coeff(hps_ctx* c, double kappa, double eta, const double* b) {
  CHECK_CTX(c);
  if (!c->have_mesh) return fail(c, HPS_ENOTBUILT, "hps_mesh first");
  if (!b || !std::isfinite(kappa) || !std::isfinite(eta) || eta == 0.0)
    return fail(c, HPS_EINVAL, "b non-null, finite kappa, finite non-zero eta required");
  const int nn = (c->N + 1) * (c->N + 1);
  const size_t bytes = sizeof(double) * (size_t)c->E * nn;
  // the coefficient and route buffers keep their size for the mesh: allocated once, then reused
  if (!c->d_c) c->d_c = static_cast<double*>(dev_alloc(c, bytes));
  if (!c->d_route) c->d_route = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)c->E));
  if (!c->d_lists) c->d_lists = static_cast<int*>(dev_alloc(c, sizeof(int) * (2 * (size_t)c->E + 2)));
  if (!c->d_c || !c->d_route || !c->d_lists) return fail(c, HPS_ENOMEM, "coefficient");
  const double* bd = b;
  if (!is_device_ptr(b)) {
    if (!c->d_bstage) c->d_bstage = static_cast<double*>(dev_alloc(c, bytes));
    if (!c->d_bstage) return fail(c, HPS_ENOMEM, "coefficient staging");
    HPS_CK(c, cudaMemcpyAsync(c->d_bstage, b, bytes, cudaMemcpyHostToDevice, c->stream));
    bd = c->d_bstage;
  }
  // Route per element (leaf.cu): the Cholesky route where the interior operator is provably
  // positive definite, max c (h/2)^2 < 0.98 * 2 mu_min, the pivoted robust route elsewhere.
  const double bound = 0.98 * 2.0 * c->mu_min / (0.25 * c->h * c->h);
  HPS_CK(c, cudaMemsetAsync(c->d_cerr, 0, sizeof(int), c->stream));
  HPS_CK(c, coeff_route(bd, kappa, c->E, nn, bound, c->d_c, c->d_route, c->d_cerr, 16 * c->num_sms, c->stream));
  c->have_leaves = false;
  c->have_tree = false;
  c->kappa = kappa;
  c->eta = eta;
  c->have_coeff = true;
  return HPS_OK;
}

int hps_build_leaves(hps_ctx* c, int precision) {
  CHECK_CTX(c);
  if (!c->have_coeff) return fail(c, HPS_ENOTBUILT, "hps_set_coeff first");
  if (precision != HPS_FP64 && precision != HPS_MIXED) return fail(c, HPS_EINVAL, "precision");
  cudaStream_t st = c->stream;
  cudaStreamSynchronize(st);
  free_numeric(c);
  if (!c->d_T) c->d_T = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)c->E * c->nb * c->nb));
  if (!c->d_T) return fail(c, HPS_ENOMEM, "leaf maps");
  int* d_good = c->d_lists;
  int* d_bad = c->d_lists + c->E;
  int* d_counts = c->d_lists + 2 * (size_t)c->E;
  LeafParams p;
  p.N = c->N; p.q = c->q; p.ni = c->q * c->q; p.nb = c->nb; p.E = c->E; p.cw = 8;
  p.h = c->h; p.eta = c->eta;
  p.c = c->d_c; p.Dh = c->d_Dref; p.Kh = c->d_Kref; p.wh = c->d_wref;
  p.T = c->d_T; p.flag = c->d_flag;
  HPS_CK(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), st));
  // the element lists of both routes (from hps_set_coeff's per-element route), their counts to
  // the host; the positive-definite route's kernel reads its count on the device and runs while
  // the host waits for the pivoted route's count
  HPS_CK(c, route_lists(c->d_route, c->E, d_good, d_bad, d_counts, st));
  HPS_CK(c, cudaMemcpyAsync(c->pin_counts, d_counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  cudaEvent_t ev_counts = nullptr;
  HPS_CK(c, cudaEventCreateWithFlags(&ev_counts, cudaEventDisableTiming));
  struct EvGuard {
    cudaEvent_t e;
    ~EvGuard() { cudaEventDestroy(e); }
  } evg{ev_counts};
  HPS_CK(c, cudaEventRecord(ev_counts, st));
  std::vector<void*> scratch;
  struct ScratchGuard {
    hps_ctx* c;
    std::vector<void*>& v;
    ~ScratchGuard() {
      if (!v.empty()) cudaStreamSynchronize(c->stream);
      for (void* s : v) dev_free(c, s);
    }
  } sg{c, scratch};
  if (c->N <= LEAF_SMEM_MAX_N) {
    const int grid = std::min(c->E, std::max(1, c->num_sms));
    double* Ascr = static_cast<double*>(dev_alloc(c, sizeof(double) * (size_t)grid * c->nb * c->nb));
    double* Zscr = static_cast<double*>(dev_alloc(c, sizeof(double) * (size_t)grid * 2 * p.ni * c->nb));
    if (Ascr) scratch.push_back(Ascr);
    if (Zscr) scratch.push_back(Zscr);
    if (!Ascr || !Zscr) return fail(c, HPS_ENOMEM, "leaf scratch");
    p.Zscr = Zscr;
    p.Ascr = Ascr;
    p.elems = d_good;
    p.count_dev = d_counts;
    PhaseScope ps(c, HPS_PH_LEAF);
    HPS_CK(c, launch_leaf(p, grid, st));
  }
  HPS_CK(c, cudaEventSynchronize(ev_counts));
  const int n_good = c->pin_counts[0];
  const int n_bad = c->pin_counts[1];
  if (c->N > LEAF_SMEM_MAX_N) {
    // the packed factor of L~_ii does not fit shared memory: the interior solver's route
    PhaseScope ps(c, HPS_PH_LEAF);
    const int rc = fd_leaf_maps(c, d_good, n_good);
    if (rc != HPS_OK) return rc;
  }
  if (n_bad > 0) {
    const size_t per = sizeof(double2) * (size_t)p.ni * (p.ni + p.nb);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n_bad, ((size_t)512 << 20) / per));
    double2* W = static_cast<double2*>(dev_alloc(c, per * chunk));
    int* piv = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)chunk * GJ_NB));
    double2* lu = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)chunk * GJ_NB * GJ_NB));
    for (void* q : {(void*)W, (void*)piv, (void*)lu})
      if (q) scratch.push_back(q);
    if (!W || !piv || !lu) return fail(c, HPS_ENOMEM, "robust leaf workspace");
    PhaseScope ps(c, HPS_PH_LEAF);
    for (int b0 = 0; b0 < n_bad; b0 += chunk) {
      const int nch = std::min(chunk, n_bad - b0);
      HPS_CK(c, robust_assemble(p, d_bad + b0, nch, W, st));
      HPS_CK(c, gj_solve<double>(W, p.ni, p.ni + p.nb, nch, piv, lu, c->d_flag, st));
      HPS_CK(c, robust_finish(p, d_bad + b0, nch, W, st));
    }
  }
  int* flags = c->pin_counts;  // the counts were read above; reuse the pinned words for the flags
  HPS_CK(c, cudaMemcpyAsync(&flags[0], c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  HPS_CK(c, cudaMemcpyAsync(&flags[1], c->d_cerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  HPS_CK(c, cudaStreamSynchronize(st));
  if (flags[1]) return fail(c, HPS_EINVAL, "non-finite coefficient sample");
  if (flags[0]) return fail(c, HPS_ENUMERIC, "singular element system (zero pivot or non-positive Cholesky pivot)");
  c->n_robust = n_bad;
  c->precision = precision;
  c->have_leaves = true;
  return HPS_OK;
}

int hps_leaf_T(hps_ctx* c, int e0, int count, void* T_host) {
  CHECK_CTX(c);
  if (!c->have_leaves) return fail(c, HPS_ENOTBUILT, "hps_build_leaves first");
  if (!T_host || e0 < 0 || count < 0 || e0 + count > c->E) return fail(c, HPS_EINVAL, "element range");
  HPS_CK(c, cudaStreamSynchronize(c->stream));
  HPS_CK(c, cudaMemcpy(T_host, c->d_T + (size_t)e0 * c->nb * c->nb, sizeof(double2) * (size_t)count * c->nb * c->nb,
                       cudaMemcpyDeviceToHost));
  return HPS_OK;
}

long long hps_kernel_launches(void) { return hps::g_launches.load(); }

int hps_profile(hps_ctx* c, int enable) {
  CHECK_CTX(c);
  prof_collect(c);
  if (enable) {
    for (int i = 0; i < HPS_NPHASE; ++i) {
      c->prof_ms[i] = 0.0;
      c->prof_launch[i] = 0;
      c->prof_calls[i] = 0;
    }
  }
  c->prof = enable != 0;
  return HPS_OK;
}

int hps_profile_read(hps_ctx* c, double* ms, long long* launches, long long* calls) {
  CHECK_CTX(c);
  prof_collect(c);
  for (int i = 0; i < HPS_NPHASE; ++i) {
    if (ms) ms[i] = c->prof_ms[i];
    if (launches) launches[i] = c->prof_launch[i];
    if (calls) calls[i] = c->prof_calls[i];
  }
  return HPS_OK;
}

int hps_profile_kernels(hps_ctx* c, int enable) {
  CHECK_CTX(c);
  kprof_collect(c);
  if (enable) {
    for (int i = 0; i < HPS_NKC; ++i) {
      c->kprof_ms[i] = c->kprof_bytes[i] = c->kprof_flops[i] = 0.0;
      c->kprof_launch[i] = 0;
    }
  }
  c->kprof = enable != 0;
  return HPS_OK;
}

int hps_profile_kernels_read(hps_ctx* c, double* ms, long long* launches, double* bytes, double* flops) {
  CHECK_CTX(c);
  kprof_collect(c);
  for (int i = 0; i < HPS_NKC; ++i) {
    if (ms) ms[i] = c->kprof_ms[i];
    if (launches) launches[i] = c->kprof_launch[i];
    if (bytes) bytes[i] = c->kprof_bytes[i];
    if (flops) flops[i] = c->kprof_flops[i];
  }
  return HPS_OK;
}

int hps_set_autotune(hps_ctx* c, int mode) {
  CHECK_CTX(c);
  if (mode != HPS_TUNE_OFF && mode != HPS_TUNE_ON && (mode < HPS_TUNE_FORCE || mode >= HPS_TUNE_FORCE + 64))
    return fail(c, HPS_EINVAL, "mode: HPS_TUNE_OFF, HPS_TUNE_ON or HPS_TUNE_FORCE + i (0 <= i < 64)");
  if (mode != c->tune) {
    c->tune = mode;
    ++c->vc_gen;  // the V-cycle graph holds the old launch configurations: capture it again
  }
  return HPS_OK;
}

int hps_autotune_table(char* buf, int len) { return autotune_table(buf, len); }

void hps_autotune_clear(void) { autotune_clear(); }

int hps_build_leaves_batch(hps_ctx** ctxs, int n, int precision) {
  if (!ctxs || n < 1) return HPS_EINVAL;
  hps_ctx* c0 = ctxs[0];
  CHECK_CTX(c0);
  if (precision != HPS_FP64 && precision != HPS_MIXED) return fail(c0, HPS_EINVAL, "precision");
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || ctxs[i]->device != c0->device) return fail(c0, HPS_EINVAL, "contexts on one device required");
    if (!ctxs[i]->have_coeff) return fail(c0, HPS_ENOTBUILT, "hps_set_coeff on every context first");
  }
  // classify every element of every context; group the Cholesky-route ones by GLL order
  std::vector<LeafElem> groups[LEAF_SMEM_MAX_N + 1];
  std::vector<std::vector<int>> big(n);  // positive-definite elements of orders above the leaf kernel's
  std::vector<std::vector<int>> bad(n);
  for (int i = 0; i < n; ++i) {
    hps_ctx* c = ctxs[i];
    cudaStreamSynchronize(c->stream);
    free_numeric(c);
    if (!c->d_T) c->d_T = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)c->E * c->nb * c->nb));
    if (!c->d_T) return fail(c0, HPS_ENOMEM, "leaf maps");
    const int n1 = c->N + 1;
    // the per-element routes and the finiteness flag from hps_set_coeff's kernel
    std::vector<int> route(c->E);
    int cerr = 0;
    HPS_CK(c0, cudaMemcpyAsync(route.data(), c->d_route, sizeof(int) * c->E, cudaMemcpyDeviceToHost, c->stream));
    HPS_CK(c0, cudaMemcpyAsync(&cerr, c->d_cerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    HPS_CK(c0, cudaStreamSynchronize(c->stream));
    if (cerr) return fail(c0, HPS_EINVAL, "non-finite coefficient sample in the batch");
    for (int e = 0; e < c->E; ++e) {
      if (route[e] == 0 && c->N > LEAF_SMEM_MAX_N) {
        big[i].push_back(e);
      } else if (route[e] == 0) {
        LeafElem d;
        d.c = c->d_c + (size_t)e * n1 * n1;
        d.T = c->d_T + (size_t)e * c->nb * c->nb;
        d.h = c->h;
        d.eta = c->eta;
        groups[c->N].push_back(d);
      } else {
        bad[i].push_back(e);
      }
    }
  }
  HPS_CK(c0, cudaMemsetAsync(c0->d_flag, 0, sizeof(int), c0->stream));
  std::vector<void*> scratch;
  int flag = 0;
  {
    PhaseScope ps(c0, HPS_PH_LEAF);
    for (int i = 0; i < n; ++i) {
      if (big[i].empty()) continue;
      hps_ctx* c = ctxs[i];
      int* d_big = static_cast<int*>(dev_alloc(c, sizeof(int) * big[i].size()));
      if (!d_big) return fail(c0, HPS_ENOMEM, "element list");
      HPS_CK(c0, cudaMemcpyAsync(d_big, big[i].data(), sizeof(int) * big[i].size(), cudaMemcpyHostToDevice,
                                 c->stream));
      const int rc = fd_leaf_maps(c, d_big, (int)big[i].size());
      dev_free(c, d_big);
      if (rc != HPS_OK) return fail(c0, rc, std::string("context ") + std::to_string(i) + ": " + c->err);
    }
    for (int N = 2; N <= LEAF_SMEM_MAX_N; ++N) {
      if (groups[N].empty()) continue;
      // reference tables of order N from any context with that order
      hps_ctx* cn = nullptr;
      for (int i = 0; i < n && !cn; ++i)
        if (ctxs[i]->N == N) cn = ctxs[i];
      const int nb = 4 * (N - 1);
      const int count = (int)groups[N].size();
      const int grid = std::min(count, std::max(1, c0->num_sms));
      LeafElem* d_ed = static_cast<LeafElem*>(dev_alloc(c0, sizeof(LeafElem) * groups[N].size()));
      double* Ascr = static_cast<double*>(dev_alloc(c0, sizeof(double) * (size_t)grid * nb * nb));
      double* Zscr = static_cast<double*>(dev_alloc(c0, sizeof(double) * (size_t)grid * 2 * (N - 1) * (N - 1) * nb));
      if (!d_ed || !Ascr || !Zscr) return fail(c0, HPS_ENOMEM, "batched leaf workspace");
      scratch.push_back(d_ed);
      scratch.push_back(Ascr);
      scratch.push_back(Zscr);
      HPS_CK(c0, cudaMemcpyAsync(d_ed, groups[N].data(), sizeof(LeafElem) * groups[N].size(), cudaMemcpyHostToDevice,
                                 c0->stream));
      LeafParams p;
      p.N = N; p.q = N - 1; p.ni = (N - 1) * (N - 1); p.nb = nb; p.E = count; p.cw = 8;
      p.h = 1.0; p.eta = 1.0; p.c = nullptr; p.T = nullptr;
      p.Dh = cn->d_Dref; p.Kh = cn->d_Kref; p.wh = cn->d_wref;
      p.Ascr = Ascr; p.Zscr = Zscr; p.flag = c0->d_flag;
      p.ed = d_ed; p.count = count;
      HPS_CK(c0, launch_leaf(p, grid, c0->stream));
    }
    for (int i = 0; i < n; ++i) {
      if (bad[i].empty()) continue;
      hps_ctx* c = ctxs[i];
      LeafParams p;
      p.N = c->N; p.q = c->q; p.ni = c->q * c->q; p.nb = c->nb; p.E = c->E; p.cw = 8;
      p.h = c->h; p.eta = c->eta;
      p.c = c->d_c; p.Dh = c->d_Dref; p.Kh = c->d_Kref; p.wh = c->d_wref;
      p.T = c->d_T; p.flag = c0->d_flag;
      const size_t per = sizeof(double2) * (size_t)p.ni * (p.ni + p.nb);
      const int chunk = (int)std::max<size_t>(1, std::min<size_t>(bad[i].size(), ((size_t)512 << 20) / per));
      double2* W = static_cast<double2*>(dev_alloc(c0, per * chunk));
      int* piv = static_cast<int*>(dev_alloc(c0, sizeof(int) * (size_t)chunk * GJ_NB));
      double2* lu = static_cast<double2*>(dev_alloc(c0, sizeof(double2) * (size_t)chunk * GJ_NB * GJ_NB));
      int* d_bad = static_cast<int*>(dev_alloc(c0, sizeof(int) * bad[i].size()));
      if (!W || !piv || !lu || !d_bad) return fail(c0, HPS_ENOMEM, "robust leaf workspace");
      scratch.insert(scratch.end(), {W, piv, lu, d_bad});
      HPS_CK(c0, cudaMemcpyAsync(d_bad, bad[i].data(), sizeof(int) * bad[i].size(), cudaMemcpyHostToDevice, c0->stream));
      for (size_t b0 = 0; b0 < bad[i].size(); b0 += chunk) {
        const int nch = (int)std::min<size_t>(chunk, bad[i].size() - b0);
        HPS_CK(c0, robust_assemble(p, d_bad + b0, nch, W, c0->stream));
        HPS_CK(c0, gj_solve<double>(W, p.ni, p.ni + p.nb, nch, piv, lu, c0->d_flag, c0->stream));
        HPS_CK(c0, robust_finish(p, d_bad + b0, nch, W, c0->stream));
      }
    }
  }
  HPS_CK(c0, cudaMemcpyAsync(&flag, c0->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c0->stream));
  HPS_CK(c0, cudaStreamSynchronize(c0->stream));
  for (void* s : scratch) dev_free(c0, s);
  if (flag) return fail(c0, HPS_ENUMERIC, "singular element system in the batch");
  for (int i = 0; i < n; ++i) {
    ctxs[i]->n_robust = (int)bad[i].size();
    ctxs[i]->precision = precision;
    ctxs[i]->have_leaves = true;
  }
  return HPS_OK;
}

int hps_release_workspace(hps_ctx* c) {
  CHECK_CTX(c);
  HPS_CK(c, cudaStreamSynchronize(c->stream));
  free_solver(c);
  for (auto& s : c->stages) {
    FREE(s.vec); FREE(s.gR); FREE(s.gE);
  }
  FREE(c->gW);
  c->gamma_nrhs = 0;
  FREE(c->sw_x);
  FREE(c->cg_V); FREE(c->cg_w); FREE(c->cg_W); FREE(c->cg_H); FREE(c->cg_h1); FREE(c->cg_h2);
  FREE(c->cg_nrm); FREE(c->cg_y); FREE(c->cg_g); FREE(c->cg_s); FREE(c->cg_part);
  FREE(c->cg_beta); FREE(c->cg_floor); FREE(c->cg_c); FREE(c->cg_inv); FREE(c->cg_cnt);
  FREE(c->ex_r); FREE(c->ex_e);
  c->nrhs_cap = 0;
  c->cg_k = c->cg_nrhs = c->ex_nrhs = 0;
  ++c->vc_gen;
  return HPS_OK;
}

}  // extern "C"
