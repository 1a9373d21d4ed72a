// Sources s != 0 and the volume solution (section 3.1, eq. ItIOperator and the element solve
// L u = b that follows it; section 3.2, eq. localiti).
//
// Per element, with incoming impedance data f on the edge nodes iota_Gamma and interior
// right-hand side b~ = w_i w_j s (physical GLL weights), L u = [f ; b~] is solved by block
// elimination of the interior.  On the positive-definite route (the leaf build's route 0):
//     v   = L~_ii^{-1} b~,
//     u_G = P^{-1} (f - Dn_Gi v),   P^{-1} = (I - T) / (2 i eta)   (T the element's leaf map),
//     u_i = L~_ii^{-1} (b~ - L~_iG u_G),
// and the interior contribution of eq. ItIOperator (f = 0) is H = I_o u = -2 i eta u_G
//     = (I - T) Dn_Gi v.
// Elements on the pivoted route take the complex Schur complement S_i of the leaf build's
// robust route with the extra right-hand sides b~ (leaf.cu, robust_field).
//
// L~_ii solves (interior_solve_kernel).  In the scaled unknowns Y = V X V (V = diag(w^1/2) of
// the reference interior weights) the interior operator is
//     A Y = S Y + Y S - D o Y,   S = V^{-1} K^_ii V^{-1} = U diag(lam) U^T,  D = (h/2)^2 c,
// (K^ the reference stiffness; the Kronecker terms K^ (x) W^ + W^ (x) K^ are h-invariant).  The
// fast-diagonalisation operator P Y = S Y + Y S is inverted exactly by U ((U^T R U) / (lam_a +
// lam_b)) U^T and preconditions conjugate gradients (A is symmetric positive definite on this
// route: max D < lam_min(P) by the route's bound, so P^{-1} A has its spectrum in (0.02, 1 +
// |min D| / lam_min]).  CG runs in FP32 inside an FP64 iterative refinement whose residual is
// formed with the FP64 operator; the result meets a 1e-14 relative FP64 residual.
//
// Corners are removed from the discretization and filled afterwards (section 3.1): each corner
// value is the mean of the two one-sided extrapolations along its edges, the degree N-2
// polynomial through an edge's N-1 non-corner nodes evaluated at the edge's end.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.h"
#include "skel.cuh"

namespace hps {

namespace {

constexpr int VT = 256;          // threads of the element kernels
constexpr int VCH = 4;           // right-hand sides per chunk of the interior solve
constexpr int V_MAX_OUTER = 6;   // FP64 refinement steps
constexpr int V_MAX_INNER = 40;  // FP32 CG steps per refinement step

struct VolParams {
  int N, q, ni, nb, E, nrhs;
  double h, eta;
  const double* c;       // [E][(N+1)^2]
  const double* Dh;      // reference D [(N+1)^2]
  const double* Kh;      // reference K [(N+1)^2]
  const double* wh;      // reference weights [N+1]
  const double* tab;     // [S q^2 | U q^2 | lam q | sqrt(w_i) q | corner weights wl q, wr q]
  const double2* T;      // leaf maps [E][nb][nb]
  const int* elems;      // positive-definite route elements
  const int* count_dev;  // their count (device); null: count_host
  int count_host = 0;
  int b_shared = 0;      // interior solve: one right-hand-side set B [nrhs][ni] for every element
  int x_by_pos = 0;      // interior solve: X indexed by list position instead of element
};

// deterministic block sums of VCH per-thread partials; out[j] valid after the call
template <typename F>
__device__ __forceinline__ void block_sum(F (&v)[VCH], F* red, F* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < VCH; ++j)
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < VCH; ++j) red[w * VCH + j] = v[j];
  __syncthreads();
  if (threadIdx.x < VCH) {
    F s = F(0);
    for (int k = 0; k < nw; ++k) s += red[k * VCH + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

size_t interior_smem_bytes(int q) {
  const size_t ni = (size_t)q * q;
  return 8 * (q * q + ni)                  // S64, D64
         + 16 * 2 * VCH * ni               // X64, R64
         + 4 * (2 * q * q + 2 * ni)        // S32, U32, linv32, D32
         + 8 * 6 * VCH * ni                // x, r, z, p, Ap, t1 (float2)
         + 8 * 2 * VCH * (VT / 32) + 8 * 8 * VCH;  // reductions and scalars
}

// X = L~_ii^{-1} B for every positive-definite element and right-hand side (B, X: [E][nrhs][ni]).
__global__ void __launch_bounds__(VT) interior_solve_kernel(VolParams p, const double2* __restrict__ B,
                                                           double2* __restrict__ X) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int q = p.q, ni = p.ni, n1 = p.N + 1, nrhs = p.nrhs;
  double* S64 = reinterpret_cast<double*>(sm);
  double* D64 = S64 + q * q;
  double2* X64 = reinterpret_cast<double2*>(D64 + ni);
  double2* R64 = X64 + VCH * ni;
  float* S32 = reinterpret_cast<float*>(R64 + VCH * ni);
  float* U32 = S32 + q * q;
  float* L32 = U32 + q * q;   // 1 / (lam_a + lam_b)
  float* D32 = L32 + ni;
  float2* xv = reinterpret_cast<float2*>(D32 + ni);
  float2* rv = xv + VCH * ni;
  float2* zv = rv + VCH * ni;
  float2* pv = zv + VCH * ni;
  float2* av = pv + VCH * ni;
  float2* tv = av + VCH * ni;
  double* red64 = reinterpret_cast<double*>(tv + VCH * ni);
  float* red32 = reinterpret_cast<float*>(red64 + VCH * (VT / 32));
  double* sc64 = reinterpret_cast<double*>(red32 + 2 * VCH * (VT / 32));  // [8][VCH] scalars
  float* sc32 = reinterpret_cast<float*>(sc64 + 4 * VCH);
  const int tid = threadIdx.x, nth = blockDim.x;
  const double* tS = p.tab;
  const double* tU = tS + q * q;
  const double* tl = tU + q * q;
  const double* tv2 = tl + q;  // sqrt of the reference interior weights
  for (int l = tid; l < q * q; l += nth) {
    S64[l] = tS[l];
    S32[l] = (float)tS[l];
    U32[l] = (float)tU[l];
  }
  for (int l = tid; l < ni; l += nth) L32[l] = (float)(1.0 / (tl[l / q] + tl[l % q]));
  const double h2 = 0.25 * p.h * p.h;
  const int nel = p.count_dev ? *p.count_dev : p.count_host;
  for (int ei = blockIdx.x; ei < nel; ei += gridDim.x) {
    const int e = p.elems[ei];
    const long long eb = p.b_shared ? 0 : e;   // element index of B
    const long long ex = p.x_by_pos ? ei : e;  // element index of X
    __syncthreads();
    for (int l = tid; l < ni; l += nth) {
      const int a = l / q, b = l % q;
      const double d = h2 * p.c[(long long)e * n1 * n1 + (a + 1) * n1 + (b + 1)];
      D64[l] = d;
      D32[l] = (float)d;
    }
    for (int r0 = 0; r0 < nrhs; r0 += VCH) {
      const int cr = min(VCH, nrhs - r0);
      const int tot = cr * ni;
      // scaled right-hand side B' = V^{-1} B V^{-1} (the first residual), X = 0
      double bn[VCH] = {0.0};
      __syncthreads();
      for (int f = tid; f < VCH * ni; f += nth) {
        const int j = f / ni, l = f % ni;
        double2 b = make_double2(0.0, 0.0);
        if (j < cr) {
          const double s = 1.0 / (tv2[l / q] * tv2[l % q]);
          b = cscale(B[(eb * nrhs + r0 + j) * ni + l], s);
          bn[j] += b.x * b.x + b.y * b.y;
        }
        R64[f] = b;
        X64[f] = make_double2(0.0, 0.0);
      }
      double* bn2 = sc64;  // ||B'_j||^2
      block_sum(bn, red64, bn2);
      for (int outer = 0; outer < V_MAX_OUTER; ++outer) {
        // ---- FP32 preconditioned CG on A d = R64 ----
        for (int f = tid; f < VCH * ni; f += nth) {
          rv[f] = make_float2((float)R64[f].x, (float)R64[f].y);
          xv[f] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        // z = P^{-1} r (four products with U; r in rv, result in zv, tv temporary)
        auto precond = [&]() {
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni, l = f % ni, a = l / q, b = l % q;
            const float2* R = rv + j * ni;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < q; ++k) {
              const float u = U32[k * q + a];
              acc.x = fmaf(u, R[k * q + b].x, acc.x);
              acc.y = fmaf(u, R[k * q + b].y, acc.y);
            }
            tv[f] = acc;
          }
          __syncthreads();
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni, l = f % ni, a = l / q, b = l % q;
            const float2* T1 = tv + j * ni;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < q; ++k) {
              const float u = U32[k * q + b];
              acc.x = fmaf(T1[a * q + k].x, u, acc.x);
              acc.y = fmaf(T1[a * q + k].y, u, acc.y);
            }
            zv[f] = make_float2(acc.x * L32[l], acc.y * L32[l]);
          }
          __syncthreads();
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni, l = f % ni, a = l / q, b = l % q;
            const float2* Z = zv + j * ni;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < q; ++k) {
              const float u = U32[a * q + k];
              acc.x = fmaf(u, Z[k * q + b].x, acc.x);
              acc.y = fmaf(u, Z[k * q + b].y, acc.y);
            }
            tv[f] = acc;
          }
          __syncthreads();
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni, l = f % ni, a = l / q, b = l % q;
            const float2* T3 = tv + j * ni;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = 0; k < q; ++k) {
              const float u = U32[b * q + k];
              acc.x = fmaf(T3[a * q + k].x, u, acc.x);
              acc.y = fmaf(T3[a * q + k].y, u, acc.y);
            }
            zv[f] = acc;
          }
          __syncthreads();
        };
        precond();
        float rz[VCH] = {0.f}, rs0[VCH] = {0.f};
        for (int f = tid; f < tot; f += nth) {
          const int j = f / ni;
          pv[f] = zv[f];
          rz[j] += rv[f].x * zv[f].x + rv[f].y * zv[f].y;
          rs0[j] += rv[f].x * rv[f].x + rv[f].y * rv[f].y;
        }
        float* s_rz = sc32;
        float* s_r0 = sc32 + VCH;
        float* s_pap = sc32 + 2 * VCH;
        float* s_rn = sc32 + 3 * VCH;
        block_sum(rz, red32, s_rz);
        block_sum(rs0, red32, s_r0);
        for (int it = 0; it < V_MAX_INNER; ++it) {
          // Ap = S p + p S - D o p
          float pap[VCH] = {0.f};
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni, l = f % ni, a = l / q, b = l % q;
            const float2* P = pv + j * ni;
            float2 acc = make_float2(-D32[l] * P[l].x, -D32[l] * P[l].y);
            for (int k = 0; k < q; ++k) {
              const float s1 = S32[a * q + k], s2 = S32[k * q + b];
              acc.x = fmaf(s1, P[k * q + b].x, acc.x);
              acc.y = fmaf(s1, P[k * q + b].y, acc.y);
              acc.x = fmaf(P[a * q + k].x, s2, acc.x);
              acc.y = fmaf(P[a * q + k].y, s2, acc.y);
            }
            av[f] = acc;
            pap[j] += P[l].x * acc.x + P[l].y * acc.y;
          }
          block_sum(pap, red32, s_pap);
          float rn[VCH] = {0.f};
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni;
            const float al = s_pap[j] > 0.f ? s_rz[j] / s_pap[j] : 0.f;
            xv[f].x = fmaf(al, pv[f].x, xv[f].x);
            xv[f].y = fmaf(al, pv[f].y, xv[f].y);
            rv[f].x = fmaf(-al, av[f].x, rv[f].x);
            rv[f].y = fmaf(-al, av[f].y, rv[f].y);
            rn[j] += rv[f].x * rv[f].x + rv[f].y * rv[f].y;
          }
          block_sum(rn, red32, s_rn);
          bool done = true;
          for (int j = 0; j < cr; ++j) done = done && (s_rn[j] <= 1e-12f * s_r0[j]);
          if (done) break;
          precond();
          float rzn[VCH] = {0.f};
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni;
            rzn[j] += rv[f].x * zv[f].x + rv[f].y * zv[f].y;
          }
          float* s_rzn = sc32 + 4 * VCH;
          block_sum(rzn, red32, s_rzn);
          for (int f = tid; f < tot; f += nth) {
            const int j = f / ni;
            const float be = s_rz[j] > 0.f ? s_rzn[j] / s_rz[j] : 0.f;
            pv[f].x = fmaf(be, pv[f].x, zv[f].x);
            pv[f].y = fmaf(be, pv[f].y, zv[f].y);
          }
          __syncthreads();
          if (tid < VCH) s_rz[tid] = s_rzn[tid];
          __syncthreads();
        }
        // ---- FP64: X += d, R = B' - A X ----
        for (int f = tid; f < tot; f += nth) X64[f] = cadd(X64[f], make_double2(xv[f].x, xv[f].y));
        __syncthreads();
        double rn64[VCH] = {0.0};
        for (int f = tid; f < tot; f += nth) {
          const int j = f / ni, l = f % ni, a = l / q, b = l % q;
          const double2* Xj = X64 + j * ni;
          double2 ax = make_double2(-D64[l] * Xj[l].x, -D64[l] * Xj[l].y);
          for (int k = 0; k < q; ++k) {
            const double s1 = S64[a * q + k], s2 = S64[k * q + b];
            ax.x = fma(s1, Xj[k * q + b].x, ax.x);
            ax.y = fma(s1, Xj[k * q + b].y, ax.y);
            ax.x = fma(Xj[a * q + k].x, s2, ax.x);
            ax.y = fma(Xj[a * q + k].y, s2, ax.y);
          }
          const double s = 1.0 / (tv2[a] * tv2[b]);
          const double2 bb = cscale(B[(eb * nrhs + r0 + j) * ni + l], s);
          const double2 rr = csub(bb, ax);
          R64[f] = rr;
          rn64[j] += rr.x * rr.x + rr.y * rr.y;
        }
        double* s_rn64 = sc64 + VCH;
        block_sum(rn64, red64, s_rn64);
        bool conv = true;
        for (int j = 0; j < cr; ++j) conv = conv && (s_rn64[j] <= 1e-28 * bn2[j]);
        if (conv) break;
      }
      // X = V^{-1} Y V^{-1}
      for (int f = tid; f < tot; f += nth) {
        const int j = f / ni, l = f % ni;
        const double s = 1.0 / (tv2[l / q] * tv2[l % q]);
        X[(ex * nrhs + r0 + j) * ni + l] = cscale(X64[f], s);
      }
    }
  }
}

// b~ = (h/2)^2 w^_a w^_b s at the interior nodes: s user [nrhs][E][(N+1)^2] -> B [E][nrhs][ni]
__global__ void btilde_kernel(VolParams p, const double2* __restrict__ s, double2* __restrict__ B) {
  const int q = p.q, ni = p.ni, n1 = p.N + 1, nrhs = p.nrhs;
  const double h2 = 0.25 * p.h * p.h;
  const long long tot = (long long)p.E * nrhs * ni;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(l / ((long long)nrhs * ni));
    const int rem = (int)(l % ((long long)nrhs * ni));
    const int r = rem / ni, I = rem % ni, a = I / q + 1, b = I % q + 1;
    const double w = h2 * p.wh[a] * p.wh[b];
    B[l] = cscale(s[((long long)r * p.E + e) * n1 * n1 + a * n1 + b], w);
  }
}

// (Dn_Gi v)_g: outward normal derivative at edge node g from the interior values v (physical D)
__device__ __forceinline__ double2 dn_interior(const double* sD, int N, int q, const double2* v, int g) {
  const int n1 = N + 1, side = g / q, k = g % q + 1;
  double2 acc = make_double2(0.0, 0.0);
  if (side < 2) {  // left (0, k) / right (N, k): sum over x
    const double sg = side == 0 ? -1.0 : 1.0;
    const int row = side == 0 ? 0 : N;
    for (int m = 1; m <= q; ++m) acc = cadd(acc, cscale(v[(m - 1) * q + (k - 1)], sg * sD[row * n1 + m]));
  } else {  // bottom (k, 0) / top (k, N): sum over y
    const double sg = side == 2 ? -1.0 : 1.0;
    const int row = side == 2 ? 0 : N;
    for (int m = 1; m <= q; ++m) acc = cadd(acc, cscale(v[(k - 1) * q + (m - 1)], sg * sD[row * n1 + m]));
  }
  return acc;
}

// Positive-definite route, one CTA per element.  Source mode (F null, Bt null): H = (I - T) Dn_Gi v
// into H [E * nb][nrhs].  Volume mode: u_G = (I - T)(f - Dn_Gi v) / (2 i eta) into UG [E][nrhs][nb]
// and B2 = b~ - L~_iG u_G into B2 [E][nrhs][ni] (v, b~ null = 0).
__global__ void __launch_bounds__(VT) pd_edges_kernel(VolParams p, const double2* __restrict__ V,
                                                     const double2* __restrict__ F, const double2* __restrict__ Bt,
                                                     double2* __restrict__ H, double2* __restrict__ UG,
                                                     double2* __restrict__ B2) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1, nrhs = p.nrhs;
  double* sD = reinterpret_cast<double*>(sm);
  double* sK = sD + n1 * n1;
  double* sw = sK + n1 * n1;
  double2* z = reinterpret_cast<double2*>(sm + ((2 * n1 * n1 + n1) * 8 + 15) / 16 * 16);  // [nb][nrhs]
  double2* ug = z + nb * nrhs;                       // [nb][nrhs]
  const int tid = threadIdx.x, nth = blockDim.x;
  const double dsc = 2.0 / p.h;
  for (int l = tid; l < n1 * n1; l += nth) {
    sD[l] = dsc * p.Dh[l];
    sK[l] = p.Kh[l];
  }
  for (int l = tid; l < n1; l += nth) sw[l] = p.wh[l];
  const bool volume = UG != nullptr;
  const double inv2e = 0.5 / p.eta;
  const int nel = p.count_dev ? *p.count_dev : p.count_host;
  for (int ei = blockIdx.x; ei < nel; ei += gridDim.x) {
    const int e = p.elems[ei];
    __syncthreads();
    for (int f = tid; f < nb * nrhs; f += nth) {
      const int g = f / nrhs, r = f % nrhs;
      double2 d = V ? dn_interior(sD, N, q, V + ((long long)e * nrhs + r) * ni, g) : make_double2(0.0, 0.0);
      if (volume) {
        const double2 fi = F[((long long)e * nrhs + r) * nb + g];
        d = csub(fi, d);
      }
      z[f] = d;
    }
    __syncthreads();
    const double2* Te = p.T + (long long)e * nb * nb;
    for (int f = tid; f < nb * nrhs; f += nth) {
      const int g = f / nrhs, r = f % nrhs;
      double2 acc = z[f];
      for (int k = 0; k < nb; ++k) cfms(acc, Te[(long long)g * nb + k], z[k * nrhs + r]);
      if (!volume) {
        H[((long long)e * nb + g) * nrhs + r] = acc;
      } else {  // (I - T) z / (2 i eta) = -i (I - T) z / (2 eta)
        const double2 u = make_double2(acc.y * inv2e, -acc.x * inv2e);
        ug[f] = u;
        UG[((long long)e * nrhs + r) * nb + g] = u;
      }
    }
    if (!volume) continue;
    __syncthreads();
    // B2 = b~ - L~_iG u_G: interior node (a, b) couples to the edge nodes of its row and column
    for (int f = tid; f < ni * nrhs; f += nth) {
      const int r = f / ni, I = f % ni, a = I / q + 1, b = I % q + 1;
      double2 v = Bt ? Bt[((long long)e * nrhs + r) * ni + I] : make_double2(0.0, 0.0);
      const double2 ul = ug[(0 * q + b - 1) * nrhs + r], ur = ug[(1 * q + b - 1) * nrhs + r];
      const double2 ub = ug[(2 * q + a - 1) * nrhs + r], ut = ug[(3 * q + a - 1) * nrhs + r];
      v = csub(v, cscale(ul, sK[a * n1 + 0] * sw[b]));
      v = csub(v, cscale(ur, sK[a * n1 + N] * sw[b]));
      v = csub(v, cscale(ub, sw[a] * sK[b * n1 + 0]));
      v = csub(v, cscale(ut, sw[a] * sK[b * n1 + N]));
      B2[((long long)e * nrhs + r) * ni + I] = v;
    }
  }
}

// Incoming data of every element side: F [E][nrhs][nb] from the skeleton solution g (user order,
// [nrhs][n_skel]) and the boundary data t ([nrhs][n_bdry]).
__global__ void incoming_kernel(int E, int nb, int nrhs, const int* __restrict__ es_in,
                                const int* __restrict__ es_bdry, const double2* __restrict__ g, long long n_skel,
                                const double2* __restrict__ t, long long n_bdry, double2* __restrict__ F) {
  const long long tot = (long long)E * nrhs * nb;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(l / ((long long)nrhs * nb));
    const int rem = (int)(l % ((long long)nrhs * nb));
    const int r = rem / nb, gi = rem % nb;
    const long long pidx = (long long)e * nb + gi;
    const int u = es_in[pidx];
    double2 v = make_double2(0.0, 0.0);
    if (u >= 0) v = g[(long long)r * n_skel + u];
    else if (t) v = t[(long long)r * n_bdry + es_bdry[pidx]];
    F[l] = v;
  }
}

// u [nrhs][E][(N+1)^2]: interior from Ui, edges from UG, corners by extrapolation along the edges.
__global__ void assemble_kernel(VolParams p, const double2* __restrict__ Ui, const double2* __restrict__ UG,
                                double2* __restrict__ u) {
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1, nrhs = p.nrhs;
  const double* wl = p.tab + 2 * q * q + 2 * q;
  const double* wr = wl + q;
  const long long tot = (long long)p.E * nrhs * n1 * n1;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(l / ((long long)p.E * n1 * n1));
    const long long rem = l % ((long long)p.E * n1 * n1);
    const int e = (int)(rem / (n1 * n1)), nd = (int)(rem % (n1 * n1));
    const int i = nd / n1, j = nd % n1;
    const double2* ue = Ui + ((long long)e * nrhs + r) * ni;
    const double2* ge = UG + ((long long)e * nrhs + r) * nb;
    double2 v;
    const bool ei = i == 0 || i == N, ej = j == 0 || j == N;
    if (!ei && !ej) {
      v = ue[(i - 1) * q + (j - 1)];
    } else if (ei && !ej) {
      v = ge[(i == 0 ? 0 : q) + j - 1];
    } else if (!ei && ej) {
      v = ge[(j == 0 ? 2 * q : 3 * q) + i - 1];
    } else {  // corner: x-edge (left/right side at i) along y to end j, y-edge (bottom/top at j) along x to end i
      const double* wy = j == 0 ? wl : wr;
      const double* wx = i == 0 ? wl : wr;
      const double2* sx = ge + (i == 0 ? 0 : q);
      const double2* sy = ge + (j == 0 ? 2 * q : 3 * q);
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      for (int k = 0; k < q; ++k) {
        a = cadd(a, cscale(sx[k], wy[k]));
        b = cadd(b, cscale(sy[k], wx[k]));
      }
      v = cscale(cadd(a, b), 0.5);
    }
    u[l] = v;
  }
}

// rho -= H on the skeleton rows (element sides with a neighbour)
__global__ void sub_h_kernel(double2* __restrict__ rho, const double2* __restrict__ H, const int* __restrict__ nbr,
                             long long rows, int nrhs) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x)
    if (nbr[l / nrhs] >= 0) rho[l] = csub(rho[l], H[l]);
}

int grid_for(long long work) {
  long long b = (work + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(b, 16384));
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

VolParams vol_params(hps_ctx* c, int nrhs) {
  VolParams p;
  p.N = c->N; p.q = c->q; p.ni = c->q * c->q; p.nb = c->nb; p.E = c->E; p.nrhs = nrhs;
  p.h = c->h; p.eta = c->eta;
  p.c = c->d_c; p.Dh = c->d_Dref; p.Kh = c->d_Kref; p.wh = c->d_wref; p.tab = c->d_vtab;
  p.T = c->d_T;
  p.elems = c->d_lists;
  p.count_dev = c->d_lists + 2 * (size_t)c->E;
  return p;
}

LeafParams leaf_params(hps_ctx* c) {
  LeafParams p;
  p.N = c->N; p.q = c->q; p.ni = c->q * c->q; p.nb = c->nb; p.E = c->E; p.cw = 8;
  p.h = c->h; p.eta = c->eta;
  p.c = c->d_c; p.Dh = c->d_Dref; p.Kh = c->d_Kref; p.wh = c->d_wref;
  p.T = c->d_T; p.flag = c->d_flag;
  return p;
}

int ensure_vol(hps_ctx* c, int nrhs) {
  if (nrhs <= c->vol_nrhs) return HPS_OK;
  free_vol(c);
  const size_t ei = (size_t)c->E * nrhs * c->q * c->q, eb = (size_t)c->E * nrhs * c->nb;
  c->vol_B = static_cast<double2*>(dev_alloc(c, sizeof(double2) * ei));
  c->vol_V = static_cast<double2*>(dev_alloc(c, sizeof(double2) * ei));
  c->vol_U = static_cast<double2*>(dev_alloc(c, sizeof(double2) * ei));
  c->vol_B2 = static_cast<double2*>(dev_alloc(c, sizeof(double2) * ei));
  c->vol_F = static_cast<double2*>(dev_alloc(c, sizeof(double2) * eb));
  c->vol_G = static_cast<double2*>(dev_alloc(c, sizeof(double2) * eb));
  if (!c->vol_B || !c->vol_V || !c->vol_U || !c->vol_B2 || !c->vol_F || !c->vol_G) {
    free_vol(c);
    return fail(c, HPS_ENOMEM, "volume-solution workspace");
  }
  c->vol_nrhs = nrhs;
  return HPS_OK;
}

int interior_solve(hps_ctx* c, const double2* B, double2* X, int nrhs) {
  VolParams p = vol_params(c, nrhs);
  const int grid = std::max(1, std::min(c->E, 2 * c->num_sms));
  interior_solve_kernel<<<grid, VT, interior_smem_bytes(c->q), c->stream>>>(p, B, X);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  return HPS_OK;
}

size_t edges_smem_bytes(int N, int nrhs) {
  const int n1 = N + 1, nb = 4 * (N - 1);
  return ((sizeof(double) * (2 * n1 * n1 + n1) + 15) / 16 * 16) + sizeof(double2) * 2 * (size_t)nb * nrhs;
}

// Pivoted-route elements: Gauss-Jordan on [S_i | -R | b~] in chunks, then u_i, u_G (or H).
int robust_fields(hps_ctx* c, int nrhs, const double2* Bt, const double2* F, double2* Ui, double2* UG, double2* H) {
  const int nbad = c->n_robust;
  if (nbad == 0) return HPS_OK;
  LeafParams p = leaf_params(c);
  const int ld = p.ni + p.nb + nrhs;
  const size_t per = sizeof(double2) * (size_t)p.ni * ld;
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(nbad, ((size_t)512 << 20) / per));
  double2* W = static_cast<double2*>(dev_alloc(c, per * chunk));
  int* piv = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)chunk * GJ_NB));
  double2* lu = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)chunk * GJ_NB * GJ_NB));
  int rc = HPS_OK;
  if (!W || !piv || !lu) rc = fail(c, HPS_ENOMEM, "pivoted-route volume workspace");
  const int* bad = c->d_lists + c->E;
  for (int b0 = 0; rc == HPS_OK && b0 < nbad; b0 += chunk) {
    const int nch = std::min(chunk, nbad - b0);
    cudaError_t e = robust_assemble(p, bad + b0, nch, W, c->stream, nrhs, Bt);
    if (e == cudaSuccess) e = gj_solve<double>(W, p.ni, ld, nch, piv, lu, c->d_flag, c->stream);
    if (e == cudaSuccess) e = robust_field(p, bad + b0, nch, nrhs, W, F, Ui, UG, H, c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "pivoted-route element fields");
  }
  if (W || piv || lu) cudaStreamSynchronize(c->stream);
  dev_free(c, W);
  dev_free(c, piv);
  dev_free(c, lu);
  return rc;
}

// ---- leaf maps for orders whose packed factor does not fit shared memory (N > 16) ----
// Z = L~_ii^{-1} L~_iG by the interior solver, A = Dn_GG - Dn_Gi Z, P = A + i eta I,
// T = I - 2 i eta P^{-1} (the block elimination of section 3.1 that the leaf kernel runs in shared
// memory).  L~_iG couples an interior node only to the edge nodes of its own row and column of
// the tensor grid, with the h-invariant Kronecker weights K^[a][0 or N] w^_b (and transposed).
__global__ void fd_coupling_kernel(VolParams p, double2* __restrict__ B) {
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1;
  const long long tot = (long long)nb * ni;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(l / ni), I = (int)(l % ni);
    const int side = g / q, k = g % q + 1, a = I / q + 1, b = I % q + 1;
    double v = 0.0;
    if (side == 0 && b == k) v = p.Kh[a * n1 + 0] * p.wh[b];
    else if (side == 1 && b == k) v = p.Kh[a * n1 + N] * p.wh[b];
    else if (side == 2 && a == k) v = p.wh[a] * p.Kh[b * n1 + 0];
    else if (side == 3 && a == k) v = p.wh[a] * p.Kh[b * n1 + N];
    B[l] = make_double2(v, 0.0);
  }
}

// W[pos] = [P | I] (nb x 2 nb) from Z [pos][nb][ni] (the interior solves of the coupling columns)
__global__ void __launch_bounds__(VT) fd_leaf_p_kernel(VolParams p, const double2* __restrict__ Z,
                                                      double2* __restrict__ W) {
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1;
  __shared__ double sD[25 * 25];
  const double dsc = 2.0 / p.h;
  for (int l = threadIdx.x; l < n1 * n1; l += blockDim.x) sD[l] = dsc * p.Dh[l];
  __syncthreads();
  for (int pos = blockIdx.x; pos < p.count_host; pos += gridDim.x) {
    const double2* Zp = Z + (long long)pos * nb * ni;
    double2* Wp = W + (long long)pos * nb * 2 * nb;
    for (int f = threadIdx.x; f < nb * nb; f += blockDim.x) {
      const int g = f / nb, g2 = f % nb;
      const int sg = g / q, kg = g % q, s2 = g2 / q, k2 = g2 % q;
      // Dn_GG: each edge node couples to itself and to the opposite node of its line
      double dgg = 0.0;
      if (kg == k2) {
        const bool xline = sg < 2 && s2 < 2, yline = sg >= 2 && s2 >= 2;
        if (xline || yline) {
          const int lo = xline ? 0 : 2;
          const int row = (sg == lo) ? 0 : N, col = (s2 == lo) ? 0 : N;
          dgg = (sg == lo ? -1.0 : 1.0) * sD[row * n1 + col];
        }
      }
      const double2 dz = dn_interior(sD, N, q, Zp + (long long)g2 * ni, g);
      double2 v = make_double2(dgg - dz.x, -dz.y);
      if (g == g2) v.y += p.eta;
      Wp[(long long)g * 2 * nb + g2] = v;
      Wp[(long long)g * 2 * nb + nb + g2] = make_double2(g == g2 ? 1.0 : 0.0, 0.0);
    }
  }
}

// T = I - 2 i eta P^{-1} from the right half of W into the leaf maps of the listed elements
__global__ void fd_leaf_t_kernel(VolParams p, const double2* __restrict__ W, double2* __restrict__ T) {
  const int nb = p.nb;
  const long long tot = (long long)p.count_host * nb * nb;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int pos = (int)(l / ((long long)nb * nb));
    const int rem = (int)(l % ((long long)nb * nb));
    const int g = rem / nb, g2 = rem % nb;
    const double2 y = W[((long long)pos * nb + g) * 2 * nb + nb + g2];
    // -2 i eta (x + i y) = 2 eta y - 2 i eta x
    T[(long long)p.elems[pos] * nb * nb + rem] =
        make_double2((g == g2 ? 1.0 : 0.0) + 2.0 * p.eta * y.y, -2.0 * p.eta * y.x);
  }
}

}  // namespace

// Leaf maps of the listed positive-definite elements by the interior solver (any order N).
int fd_leaf_maps(hps_ctx* c, const int* elems, int count) {
  if (count <= 0) return HPS_OK;
  const int nb = c->nb, ni = c->q * c->q;
  const size_t per = sizeof(double2) * ((size_t)nb * ni + (size_t)nb * 2 * nb);
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(count, ((size_t)1 << 30) / per));
  double2* Bc = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)nb * ni));
  double2* Z = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)chunk * nb * ni));
  double2* W = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)chunk * nb * 2 * nb));
  int* piv = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)chunk * GJ_NB));
  double2* lu = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (size_t)chunk * GJ_NB * GJ_NB));
  struct Release {
    hps_ctx* c;
    std::vector<void*> v;
    ~Release() {
      cudaStreamSynchronize(c->stream);
      for (void* x : v) dev_free(c, x);
    }
  } rel{c, {Bc, Z, W, piv, lu}};
  if (!Bc || !Z || !W || !piv || !lu) return fail(c, HPS_ENOMEM, "leaf workspace (interior solver route)");
  cudaStream_t st = c->stream;
  VolParams p = vol_params(c, nb);
  fd_coupling_kernel<<<grid_for((long long)nb * ni), 256, 0, st>>>(p, Bc);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  for (int b0 = 0; b0 < count; b0 += chunk) {
    const int nch = std::min(chunk, count - b0);
    VolParams pc = p;
    pc.elems = elems + b0;
    pc.count_dev = nullptr;
    pc.count_host = nch;
    pc.b_shared = 1;
    pc.x_by_pos = 1;
    const int grid = std::max(1, std::min(nch, 2 * c->num_sms));
    interior_solve_kernel<<<grid, VT, interior_smem_bytes(c->q), st>>>(pc, Bc, Z);
    note_launch();
    HPS_CK(c, cudaGetLastError());
    fd_leaf_p_kernel<<<std::max(1, std::min(nch, 4 * c->num_sms)), VT, 0, st>>>(pc, Z, W);
    note_launch();
    HPS_CK(c, cudaGetLastError());
    HPS_CK(c, gj_invert<double>(W, nb, nch, piv, lu, c->d_flag, st));
    fd_leaf_t_kernel<<<grid_for((long long)nch * nb * nb), 256, 0, st>>>(pc, W, c->d_T);
    note_launch();
    HPS_CK(c, cudaGetLastError());
  }
  return HPS_OK;
}

// The per-element work arrays (sized by the number of right-hand sides).  The staged sources and
// the H buffer have their own sizes and are released by free_vol_staging only: a solve stages
// them before it sizes the work arrays.
void free_vol(hps_ctx* c) {
  void** bufs[] = {(void**)&c->vol_B, (void**)&c->vol_V, (void**)&c->vol_U, (void**)&c->vol_B2,
                   (void**)&c->vol_F, (void**)&c->vol_G};
  for (void** b : bufs) {
    dev_free(c, *b);
    *b = nullptr;
  }
  c->vol_nrhs = 0;
}

void free_vol_staging(hps_ctx* c) {
  dev_free(c, c->vol_s);
  dev_free(c, c->vol_H);
  c->vol_s = c->vol_H = nullptr;
  c->vol_s_elems = c->vol_H_elems = 0;
}

void optin_volume() { smem_optin(interior_solve_kernel); smem_optin(pd_edges_kernel); }

// H of every element for the sources s (device, user layout [nrhs][E][(N+1)^2]) into
// H_es [n_es][nrhs] (element-side rows, right-hand side fastest).
int source_H(hps_ctx* c, const double2* s, int nrhs, double2* H_es) {
  if (!s || !H_es) return fail(c, HPS_EINVAL, "internal: sources or H buffer missing");
  int rc = ensure_vol(c, nrhs);
  if (rc != HPS_OK) return rc;
  VolParams p = vol_params(c, nrhs);
  cudaStream_t st = c->stream;
  btilde_kernel<<<grid_for((long long)c->E * nrhs * p.ni), 256, 0, st>>>(p, s, c->vol_B);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  rc = interior_solve(c, c->vol_B, c->vol_V, nrhs);
  if (rc != HPS_OK) return rc;
  const int grid = std::max(1, std::min(c->E, 4 * c->num_sms));
  pd_edges_kernel<<<grid, VT, edges_smem_bytes(c->N, nrhs), st>>>(p, c->vol_V, nullptr, nullptr, H_es, nullptr,
                                                                  nullptr);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  return robust_fields(c, nrhs, c->vol_B, nullptr, c->vol_U, nullptr, H_es);
}

int subtract_H(hps_ctx* c, double2* rho, const double2* H_es, int nrhs) {
  if (!rho || !H_es) return fail(c, HPS_EINVAL, "internal: interior contributions missing");
  sub_h_kernel<<<grid_for(c->n_es * nrhs), 256, 0, c->stream>>>(rho, H_es, c->d_es_nb, c->n_es, nrhs);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  return HPS_OK;
}

// Staged device copy of a host-or-device complex array of `elems` values.
const double2* stage_in(hps_ctx* c, const void* src, size_t elems, double2** buf, size_t* cap) {
  if (on_device(src)) return static_cast<const double2*>(src);
  if (elems > *cap) {
    dev_free(c, *buf);
    *buf = static_cast<double2*>(dev_alloc(c, sizeof(double2) * elems));
    *cap = *buf ? elems : 0;
    if (!*buf) return nullptr;
  }
  if (cudaMemcpyAsync(*buf, src, sizeof(double2) * elems, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return *buf;
}

}  // namespace hps

using namespace hps;

extern "C" int hps_volume_solution(hps_ctx* c, const void* t, const void* s, const void* g, int nrhs, void* u) {
  if (!c) return HPS_EINVAL;
  cudaError_t e0 = cudaSetDevice(c->device);
  if (e0 != cudaSuccess) return cuda_fail(c, e0, "cudaSetDevice");
  if (!c->have_leaves) return fail(c, HPS_ENOTBUILT, "hps_build_leaves first");
  if (!g || !u || nrhs < 1 || nrhs > 64) return fail(c, HPS_EINVAL, "g and u non-null, 1 <= nrhs <= 64");
  int rc = ensure_vol(c, nrhs);
  if (rc != HPS_OK) return rc;
  cudaStream_t st = c->stream;
  const int n1 = c->N + 1;
  const size_t n_s = (size_t)nrhs * c->E * n1 * n1;
  // inputs on the device (host arrays are staged; g and t share one staging buffer)
  const size_t n_g = (size_t)nrhs * c->n_skel, n_t = (size_t)nrhs * c->n_bdry;
  const double2 *gd = nullptr, *td = nullptr, *sd = nullptr;
  double2* gt_buf = nullptr;
  if (!on_device(g) || (t && !on_device(t))) {
    gt_buf = static_cast<double2*>(dev_alloc(c, sizeof(double2) * (n_g + n_t)));
    if (!gt_buf) return fail(c, HPS_ENOMEM, "staging of g and t");
  }
  struct Free {
    hps_ctx* c;
    double2* p;
    ~Free() {
      if (p) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, p);
      }
    }
  } fr{c, gt_buf};
  if (on_device(g)) gd = static_cast<const double2*>(g);
  else {
    HPS_CK(c, cudaMemcpyAsync(gt_buf, g, sizeof(double2) * n_g, cudaMemcpyHostToDevice, st));
    gd = gt_buf;
  }
  if (t) {
    if (on_device(t)) td = static_cast<const double2*>(t);
    else {
      HPS_CK(c, cudaMemcpyAsync(gt_buf + n_g, t, sizeof(double2) * n_t, cudaMemcpyHostToDevice, st));
      td = gt_buf + n_g;
    }
  }
  if (s) {
    sd = stage_in(c, s, n_s, &c->vol_s, &c->vol_s_elems);
    if (!sd) return fail(c, HPS_ENOMEM, "staging of s");
  }
  VolParams p = vol_params(c, nrhs);
  HPS_CK(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), st));
  incoming_kernel<<<grid_for((long long)c->E * nrhs * c->nb), 256, 0, st>>>(c->E, c->nb, nrhs, c->d_es_in,
                                                                          c->d_es_bdry, gd, c->n_skel, td,
                                                                          c->n_bdry, c->vol_F);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  if (sd) {
    btilde_kernel<<<grid_for((long long)c->E * nrhs * p.ni), 256, 0, st>>>(p, sd, c->vol_B);
    note_launch();
    HPS_CK(c, cudaGetLastError());
    rc = interior_solve(c, c->vol_B, c->vol_V, nrhs);
    if (rc != HPS_OK) return rc;
  }
  const int grid = std::max(1, std::min(c->E, 4 * c->num_sms));
  pd_edges_kernel<<<grid, VT, edges_smem_bytes(c->N, nrhs), st>>>(p, sd ? c->vol_V : nullptr, c->vol_F,
                                                                  sd ? c->vol_B : nullptr, nullptr, c->vol_G,
                                                                  c->vol_B2);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  rc = interior_solve(c, c->vol_B2, c->vol_U, nrhs);
  if (rc != HPS_OK) return rc;
  rc = robust_fields(c, nrhs, sd ? c->vol_B : nullptr, c->vol_F, c->vol_U, c->vol_G, nullptr);
  if (rc != HPS_OK) return rc;
  const bool host_out = !on_device(u);
  double2* ud = static_cast<double2*>(u);
  double2* ubuf = nullptr;
  if (host_out) {
    ubuf = static_cast<double2*>(dev_alloc(c, sizeof(double2) * n_s));
    if (!ubuf) return fail(c, HPS_ENOMEM, "staging of u");
    ud = ubuf;
  }
  assemble_kernel<<<grid_for((long long)n_s), 256, 0, st>>>(p, c->vol_U, c->vol_G, ud);
  note_launch();
  HPS_CK(c, cudaGetLastError());
  if (host_out) HPS_CK(c, cudaMemcpyAsync(u, ud, sizeof(double2) * n_s, cudaMemcpyDeviceToHost, st));
  int flag = 0;
  HPS_CK(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  HPS_CK(c, cudaStreamSynchronize(st));
  if (ubuf) dev_free(c, ubuf);
  if (flag) return fail(c, HPS_ENUMERIC, "zero pivot in a pivoted-route element solve");
  return HPS_OK;
}
