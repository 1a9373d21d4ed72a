// hps_leaf_maps_noalloc: the leaf ItI build without any device allocation.
//
// Some callers cannot allocate device memory while they run: a process that
// has handed the whole device to its own memory pool (a stray cudaMalloc then
// fails or fragments the pool), or a latency-critical loop that must not call
// cudaMalloc/cudaFree because those calls can synchronise the device.  This
// entry point serves them: the caller passes the coefficient samples and the
// output buffer, and every other byte the kernel needs lives in one
// file-scope device array below, which each GPU that loads the library keeps
// until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/hps.h"
#include "common.cuh"
#include "skel.cuh"

namespace hps {
namespace {

constexpr int NA_MAX_N = 16;                       // largest GLL order accepted
constexpr int NA_MAX_NB = 4 * (NA_MAX_N - 1);      // 60 edge nodes per element
constexpr int NA_MAX_GRID = 160;                   // persistent CTAs (>= SMs of one GB300)
constexpr int NA_N1 = NA_MAX_N + 1;
constexpr int NA_TABLES = 3 * NA_N1 * NA_N1;       // reference D, K and weights (padded)
constexpr int NA_FLAG_SLOTS = 32;                  // one int flag, padded to 256 bytes
constexpr size_t NA_DOUBLES = (size_t)NA_TABLES + NA_FLAG_SLOTS + (size_t)NA_MAX_GRID * NA_MAX_NB * NA_MAX_NB;

// [tables | flag | per-CTA 4q x 4q workspace]: about 4.6 MB
static __device__ __align__(256) double g_leaf_scratch[NA_DOUBLES];

constexpr int NA_MAX_DEVICES = 64;
double* g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_mu;

// Reference GLL rule with fixed-size arrays (no allocation): nodes, weights, D.
void gll_fixed(int N, double* x, double* w, double* D) {
  x[0] = -1.0;
  x[N] = 1.0;
  auto leg = [N](double t, double& p, double& pm) {
    double a = 1.0, b = t;
    for (int k = 1; k < N; ++k) {
      const double nb = ((2.0 * k + 1.0) * t * b - k * a) / (k + 1.0);
      a = b;
      b = nb;
    }
    p = b;
    pm = a;
  };
  for (int j = 1; j < N; ++j) {
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double p, pm;
      leg(t, p, pm);
      const double dp = N * (pm - t * p) / (1.0 - t * t);
      const double d2 = (2.0 * t * dp - N * (N + 1.0) * p) / (1.0 - t * t);
      const double dx = dp / d2;
      t -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[j] = t;
  }
  double P[NA_N1];
  for (int j = 0; j <= N; ++j) {
    double pm;
    leg(x[j], P[j], pm);
    w[j] = 2.0 / (N * (N + 1.0) * P[j] * P[j]);
  }
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) D[i * (N + 1) + j] = i == j ? 0.0 : P[i] / (P[j] * (x[i] - x[j]));
  D[0] = -N * (N + 1.0) / 4.0;
  D[N * (N + 1) + N] = N * (N + 1.0) / 4.0;
}

// Device address of the scratch array on `device` (looked up once per device,
// with that device current).
int scratch_on(int device, double** out) {
  if (device < 0 || device >= NA_MAX_DEVICES) return HPS_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_leaf_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return HPS_ECUDA;
    }
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return HPS_OK;
}

int leaf_maps_noalloc_on(int device, cudaStream_t st, int N, double h, double eta, const double* c, int E,
                         void* T) {
  optin_all_once();
  double* base = nullptr;
  int rc = scratch_on(device, &base);
  if (rc != HPS_OK) return rc;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int grid = std::min(E, std::min(NA_MAX_GRID, std::max(1, sms)));

  // reference tables on the host stack, copied into the scratch array
  const int n1 = N + 1;
  double tab[NA_TABLES] = {0.0};
  double x[NA_N1], w[NA_N1], Dr[NA_N1 * NA_N1];
  gll_fixed(N, x, w, Dr);
  double* hD = tab;
  double* hK = tab + NA_N1 * NA_N1;
  double* hw = tab + 2 * NA_N1 * NA_N1;
  for (int i = 0; i < n1; ++i) {
    hw[i] = w[i];
    for (int j = 0; j < n1; ++j) {
      hD[i * n1 + j] = Dr[i * n1 + j];
      double s = 0.0;
      for (int l = 0; l < n1; ++l) s += Dr[l * n1 + i] * w[l] * Dr[l * n1 + j];
      hK[i * n1 + j] = s;
    }
  }
  int* flag = reinterpret_cast<int*>(base + NA_TABLES);
  if (cudaMemcpyAsync(base, tab, sizeof(tab), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ECUDA;
  }
  LeafParams p;
  p.N = N;
  p.q = N - 1;
  p.ni = (N - 1) * (N - 1);
  p.nb = 4 * (N - 1);
  p.E = E;
  p.cw = 8;
  p.h = h;
  p.eta = eta;
  p.c = c;
  p.Dh = base;
  p.Kh = base + NA_N1 * NA_N1;
  p.wh = base + 2 * NA_N1 * NA_N1;
  p.Ascr = base + NA_TABLES + NA_FLAG_SLOTS;
  p.T = static_cast<double2*>(T);
  p.flag = flag;
  if (launch_leaf(p, grid, st) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ECUDA;
  }
  int hflag = 0;
  if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ECUDA;
  }
  return hflag ? HPS_ENUMERIC : HPS_OK;
}

}  // namespace
}  // namespace hps

// The caller's current device is restored on every return path: this entry takes a bare
// device index, so it must not leave a multi-device caller on another device.
extern "C" int hps_leaf_maps_noalloc(int device, void* stream, int N, double h, double eta, const double* c, int E,
                                     void* T) {
  using namespace hps;
  if (N < 2 || N > NA_MAX_N) return HPS_EINVAL;        // larger orders exceed the static workspace
  if (E < 1 || !c || !T || !(h > 0.0) || !std::isfinite(eta) || eta == 0.0) return HPS_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return HPS_ENODEV;
  }
  if (device < 0 || device >= ndev) return HPS_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ECUDA;
  }
  const int rc = leaf_maps_noalloc_on(device, static_cast<cudaStream_t>(stream), N, h, eta, c, E, T);
  if (prev >= 0 && prev != device && cudaSetDevice(prev) != cudaSuccess) {
    cudaGetLastError();
    return rc != HPS_OK ? rc : HPS_ECUDA;
  }
  return rc;
}
