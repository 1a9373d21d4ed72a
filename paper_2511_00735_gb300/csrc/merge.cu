// Nested-dissection merge tree and the multigrid V-cycle (sections 4.1-4.3).
//
// Stage k (k merges done) tiles the mesh with a x b element blocks,
// a = 2^ceil(k/2), b = 2^floor(k/2) (x-merges at odd levels, y-merges at even
// levels, Fig. 1).  Each subdomain's ItI map is stored "interface first": the
// side that the next merge eliminates comes first, then the other sides in the
// order l, r, b, t; the last stage (the coarse level) keeps l, r, b, t.
//
// Merge l pairs s1 (left/bottom) with s2 (right/top); interface alpha of s1 and
// beta of s2 (m unknowns each), outer parts E1, E2 (p = n - m each).  With the
// transmission condition in_2 = -out_1, in_1 = -out_2 the interface unknowns
// x = (in1_alpha, in2_beta) satisfy A x = f - B y with
//     A = [[I, T2_bb], [T1_aa, I]],   B y = (T2_bE2 y2, T1_aE1 y1),
// and A is reduced to its Schur complement S = I - T2_bb T1_aa:
//     x1 = S^{-1} (f1 - T2_bb f2),  x2 = f2 - T1_aa x1.
// The merged map (eq. globalfacesystem) T_pair = D - C A^{-1} B becomes
//     X1 = S^{-1} [ -T2_bb T1_aE1 | T2_bE2 ],   X2 = [ T1_aE1 | 0 ] - T1_aa X1,
//     T_pair = [[T1_E1E1, 0], [0, T2_E2E2]] - [[T1_E1a X1], [T2_E2b X2]].
//
// V-cycle (section 4.3, MG(M) = F + P MG(S) R (I - M F)): residuals live in
// "outgoing" coordinates (the residual of the equation owned by side p), so
// every step touches one pair only:
//   up:    z1 = S^{-1}(f1 - T2_bb f2), z2 = f2 - T1_aa z1,  f1 = rho2_beta, f2 = rho1_alpha,
//          rho'_E1 = rho1_E1 - T1_E1a z1,  rho'_E2 = rho2_E2 - T2_E2b z2;
//   down:  h1 = f1 - T2_bE2 e2_E2,  h2 = f2 - T1_aE1 e1_E1,
//          x1 = S^{-1}(h1 - T2_bb h2),  x2 = h2 - T1_aa x1   (= A^{-1}(r_x - B e)).
// The coarse system M_{L_exact+1} = I + Pi T_c is solved by a fixed number of
// GMRES steps from zero (or by a dense inverse).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ctx.h"
#include "df64.cuh"
#include "skel.cuh"

namespace hps {

namespace {

void natural_es(const hps_ctx* c, int sx, int sy, int a, int b, std::vector<int>& out) {
  out.clear();
  const int q = c->q, nx = c->nx;
  const int ix0 = sx * a, iy0 = sy * b;
  auto es = [&](int e, int s, int k) { return (e * 4 + s) * q + k; };
  for (int t = 0; t < b; ++t)
    for (int k = 0; k < q; ++k) out.push_back(es(ix0 + nx * (iy0 + t), 0, k));
  for (int t = 0; t < b; ++t)
    for (int k = 0; k < q; ++k) out.push_back(es(ix0 + a - 1 + nx * (iy0 + t), 1, k));
  for (int t = 0; t < a; ++t)
    for (int k = 0; k < q; ++k) out.push_back(es(ix0 + t + nx * iy0, 2, k));
  for (int t = 0; t < a; ++t)
    for (int k = 0; k < q; ++k) out.push_back(es(ix0 + t + nx * (iy0 + b - 1), 3, k));
}

// side ranges [lo, hi) in natural order
void side_range(int a, int b, int q, int side, int& lo, int& hi) {
  const int o[5] = {0, b * q, 2 * b * q, 2 * b * q + a * q, 2 * (a + b) * q};
  lo = o[side];
  hi = o[side + 1];
}

size_t csize(int prec) { return prec == HPS_FP64 ? sizeof(double2) : sizeof(float2); }

template <typename R>
cudaError_t gemm(hps_ctx* c, const GemmDesc* d, int nb, const void* A, long long lda, const void* B, long long ldb,
                 const void* C0, long long ldc0, void* C, long long ldc, double alpha, const int* maps, int mmax,
                 int nmax, int n_launch, int kmax = 0) {
  GemmArgs<R> a;
  a.A = static_cast<const c_t<R>*>(A);
  a.B = static_cast<const c_t<R>*>(B);
  a.C0 = static_cast<const c_t<R>*>(C0);
  a.C = static_cast<c_t<R>*>(C);
  a.lda = lda;
  a.ldb = ldb;
  a.ldc0 = ldc0;
  a.ldc = ldc;
  a.alpha = mk<R>(R(alpha), R(0));
  a.beta = mk<R>(R(1), R(0));
  a.desc = d;
  a.nbatch = nb;
  a.maps = maps;
  a.n_launch = n_launch;
  a.ws = static_cast<c_t<R>*>(c->gemm_ws);
  a.ws_elems = (long long)c->gemm_ws_elems;
  a.num_sms = c->num_sms > 0 ? c->num_sms : 148;
  a.err = c->d_gemm_err;  // FP32 GEMMs may take the tensor cores (their waits report through it)
  a.tune = c->tune;
  if (c->kprof && c->cur_phase == HPS_PH_MERGE) {
    const double e = (double)sizeof(c_t<R>) * nb;
    const double bytes = e * ((double)mmax * kmax + (double)kmax * nmax + (C0 ? 2.0 : 1.0) * mmax * nmax);
    KernScope ks(c, HPS_KC_MERGE_GEMM, bytes, 8.0 * mmax * nmax * kmax * nb);
    return launch_gemm<R>(a, mmax, nmax, c->stream, kmax);
  }
  return launch_gemm<R>(a, mmax, nmax, c->stream, kmax);
}

// The sweep products of a tiled level (FP32 tree): A = the tiled operator, tensor cores.
cudaError_t gemm_tiled(hps_ctx* c, const GemmDesc* d, int nb, const void* A, const void* B, long long ldb,
                       const void* C0, long long ldc0, void* C, long long ldc, double alpha, const int* maps, int mmax,
                       int nmax, int n_launch, int kmax, int terms) {
  GemmArgs<float> a;
  a.A = static_cast<const float2*>(A);
  a.B = static_cast<const float2*>(B);
  a.C0 = static_cast<const float2*>(C0);
  a.C = static_cast<float2*>(C);
  a.lda = mmax;  // the rows of the tiled layout (every pair of a launch is tiled alike)
  a.ldb = ldb;
  a.ldc0 = ldc0;
  a.ldc = ldc;
  a.alpha = mk<float>(float(alpha), 0.f);
  a.beta = mk<float>(1.f, 0.f);
  a.desc = d;
  a.nbatch = nb;
  a.maps = maps;
  a.n_launch = n_launch;
  a.ws = static_cast<float2*>(c->gemm_ws);
  a.ws_elems = (long long)c->gemm_ws_elems;
  a.num_sms = c->num_sms > 0 ? c->num_sms : 148;
  a.err = c->d_gemm_err;
  a.tune = c->tune;
  if (c->kprof && terms != 3) {  // the sweep products (the coarse products take terms = 3)
    // algorithmic bytes: the operator (8 B per complex entry in both formats), B, C0, C once each
    const double bytes = 8.0 * nb * ((double)mmax * kmax + (double)kmax * nmax + (C0 ? 2.0 : 1.0) * mmax * nmax);
    KernScope ks(c, HPS_KC_SWEEP, bytes, 8.0 * mmax * nmax * kmax * nb);
    return launch_tc_gemm_tiled(a, mmax, nmax, kmax, terms, a.err, c->stream);
  }
  return launch_tc_gemm_tiled(a, mmax, nmax, kmax, terms, a.err, c->stream);
}

// sweep operators kept tiled for the tensor cores (FP32 tree): every level with bf16x3 sweeps;
// with FP32 sweeps the levels with at least 32 interface rows per child (the small levels stay
// on the SIMT products)
bool level_tiled(const hps_ctx* c, const Level& Lv) { return c->sweep_bf16x3 || 2 * Lv.m >= 64; }

GemmDesc D(int a_r, int a_c, int b_r, int b_c, int c0_r, int c0_c, int c_r, int c_c, int m, int n, int k, int rmap = -1,
           int cmap = -1) {
  GemmDesc d;
  d.a_r = a_r; d.a_c = a_c; d.b_r = b_r; d.b_c = b_c; d.c0_r = c0_r; d.c0_c = c0_c; d.c_r = c_r; d.c_c = c_c;
  d.m = m; d.n = n; d.k = k; d.rmap = rmap; d.cmap = cmap;
  d.b_r2 = d.kb2 = d.c0_r2 = d.mc2 = 0;
  return d;
}

// with two-segment B (rows k >= kb2 from b_r2 + k - kb2) and C0 (rows i >= mc2 from c0_r2 + i - mc2)
GemmDesc D2(GemmDesc d, int b_r2, int kb2, int c0_r2, int mc2) {
  d.b_r2 = b_r2; d.kb2 = kb2; d.c0_r2 = c0_r2; d.mc2 = mc2;
  return d;
}

template <typename R>
int build_tree_t(hps_ctx* c, int L_exact, int exact) {
  using C = c_t<R>;
  const int q = c->q;
  const bool plan = c->plan_L != L_exact;  // build the mesh-dependent plan, or reuse the cached one
  c->L_exact = L_exact;
  std::vector<std::vector<int>> inv;
  std::vector<int> nat;
  if (plan) {
  c->stages.assign(L_exact + 1, Stage());
  c->levels.assign(L_exact + 1, Level());
  inv.assign(L_exact + 1, std::vector<int>());
  // ---- stage geometry and storage orders ----
  for (int k = 0; k <= L_exact; ++k) {
    Stage& S = c->stages[k];
    S.a = 1 << ((k + 1) / 2);
    S.b = 1 << (k / 2);
    S.gx = c->nx / S.a;
    S.gy = c->ny / S.b;
    S.nsub = S.gx * S.gy;
    S.n = 2 * (S.a + S.b) * q;
    S.es.assign((size_t)S.nsub * S.n, -1);
    inv[k].assign(c->n_es, -1);
    for (int sy = 0; sy < S.gy; ++sy)
      for (int sx = 0; sx < S.gx; ++sx) {
        const int s = sx + S.gx * sy;
        natural_es(c, sx, sy, S.a, S.b, nat);
        std::vector<int> order;
        if (k < L_exact) {
          const bool xm = ((k + 1) % 2) == 1;
          const int role = xm ? sx % 2 : sy % 2;
          const int iface = xm ? (role == 0 ? 1 : 0) : (role == 0 ? 3 : 2);
          int lo, hi;
          side_range(S.a, S.b, q, iface, lo, hi);
          for (int i = lo; i < hi; ++i) order.push_back(i);
          for (int sd = 0; sd < 4; ++sd) {
            if (sd == iface) continue;
            side_range(S.a, S.b, q, sd, lo, hi);
            for (int i = lo; i < hi; ++i) order.push_back(i);
          }
        } else {
          // coarse level: interior sides first (l, r, b, t order among them), then the physical ones
          const bool inner[4] = {sx > 0, sx < S.gx - 1, sy > 0, sy < S.gy - 1};
          for (int pass = 0; pass < 2; ++pass)
            for (int sd = 0; sd < 4; ++sd) {
              if (inner[sd] != (pass == 0)) continue;
              int lo, hi;
              side_range(S.a, S.b, q, sd, lo, hi);
              for (int i = lo; i < hi; ++i) order.push_back(i);
            }
        }
        for (int i = 0; i < S.n; ++i) {
          const int e = nat[order[i]];
          S.es[(size_t)s * S.n + i] = e;
          if (inv[k][e] != -1) return fail(c, HPS_ECUDA, "internal: element side on two subdomain boundaries");
          inv[k][e] = i;
        }
      }
  }
  // ---- levels: pairs, destination maps, checks ----
  size_t x_elems = 0;
  int max_pm = 0, max_p2m = 0, max_pairs = 0;
  for (int l = 1; l <= L_exact; ++l) {
    Level& Lv = c->levels[l];
    const Stage& P0 = c->stages[l - 1];
    const Stage& P1 = c->stages[l];
    Lv.dir = (l % 2 == 1) ? 0 : 1;
    Lv.n = P0.n;
    Lv.m = Lv.dir == 0 ? P0.b * q : P0.a * q;
    Lv.p = Lv.n - Lv.m;
    Lv.npairs = P1.nsub;
    if (2 * Lv.p != P1.n) return fail(c, HPS_ECUDA, "internal: merged boundary length");
    Lv.i1.resize(Lv.npairs);
    Lv.i2.resize(Lv.npairs);
    std::vector<int> dst((size_t)Lv.npairs * 2 * Lv.p), up((size_t)P1.nsub * P1.n, -1);
    for (int sy = 0; sy < P1.gy; ++sy)
      for (int sx = 0; sx < P1.gx; ++sx) {
        const int P = sx + P1.gx * sy;
        int s1, s2;
        if (Lv.dir == 0) {
          s1 = 2 * sx + P0.gx * sy;
          s2 = 2 * sx + 1 + P0.gx * sy;
        } else {
          s1 = sx + P0.gx * (2 * sy);
          s2 = sx + P0.gx * (2 * sy + 1);
        }
        Lv.i1[P] = s1;
        Lv.i2[P] = s2;
        for (int i = 0; i < Lv.m; ++i) {
          const int a1 = P0.es[(size_t)s1 * P0.n + i], a2 = P0.es[(size_t)s2 * P0.n + i];
          if (c->es_nb[a1] != a2) return fail(c, HPS_ECUDA, "internal: interface nodes do not match");
        }
        std::vector<char> seen(2 * Lv.p, 0);
        for (int i = 0; i < 2 * Lv.p; ++i) {
          const int child = i < Lv.p ? s1 : s2;
          const int ci = Lv.m + (i < Lv.p ? i : i - Lv.p);
          const int e = P0.es[(size_t)child * P0.n + ci];
          const int d = inv[l][e];
          if (d < 0 || P1.es[(size_t)P * P1.n + d] != e || seen[d])
            return fail(c, HPS_ECUDA, "internal: merge destination map");
          seen[d] = 1;
          dst[(size_t)P * 2 * Lv.p + i] = d;
          up[(size_t)P * P1.n + d] = child * P0.n + ci;
        }
      }
    Lv.d_dst = dev_upload(c, dst);
    Lv.d_up = dev_upload(c, up);
    if (!Lv.d_dst || !Lv.d_up) return fail(c, HPS_ENOMEM, "merge maps");
    x_elems = std::max(x_elems, (size_t)Lv.npairs * Lv.m * 2 * Lv.p);
    max_pm = std::max(max_pm, Lv.npairs * Lv.m);
    max_p2m = std::max(max_p2m, Lv.npairs * 2 * Lv.m);
    max_pairs = std::max(max_pairs, Lv.npairs);
  }
  c->plan_x_elems = x_elems;
  c->plan_max_pairs = max_pairs;
  // ---- descriptors ----
  for (int l = 1; l <= L_exact; ++l) {
    Level& Lv = c->levels[l];
    const int n = Lv.n, m = Lv.m, p = Lv.p, NP = Lv.npairs;
    std::vector<GemmDesc> md((size_t)N_MROLE * NP), sd((size_t)N_SROLE * NP);
    for (int P = 0; P < NP; ++P) {
      const int r1 = Lv.i1[P] * n, r2 = Lv.i2[P] * n;  // child row offsets in T / stage vectors
      const int w = P * m, x = P * m, t = P * 2 * p;
      const int dm1 = P * 2 * p, dm2 = P * 2 * p + p;  // dst map offsets for E1, E2
      md[MS * NP + P] = D(r2, 0, r1, 0, w, 0, w, 0, m, m, m);
      md[MR * NP + P] = D(r2, 0, r1, m, 0, 0, x, 0, m, p, m);
      md[MX1A * NP + P] = D(w, m, x, 0, 0, 0, x, 0, m, p, m);
      md[MX1B * NP + P] = D(w, m, r2, m, 0, 0, x, p, m, p, m);
      md[MX2A * NP + P] = D(r1, 0, x, 0, r1, m, x, 0, m, p, m);
      md[MX2B * NP + P] = D(r1, 0, x, p, 0, 0, x, p, m, p, m);
      md[MOA * NP + P] = D(r1 + m, 0, x, 0, r1 + m, m, t, 0, p, p, m, dm1, dm1);
      md[MOB * NP + P] = D(r1 + m, 0, x, p, 0, 0, t, 0, p, p, m, dm1, dm2);
      md[MOC * NP + P] = D(r2 + m, 0, x, 0, 0, 0, t, 0, p, p, m, dm2, dm1);
      md[MOD * NP + P] = D(r2 + m, 0, x, p, r2 + m, m, t, 0, p, p, m, dm2, dm2);
      // sweep operators: G = A^{-1} with columns [f1 | f2] (rows g..g+2m of the G workspace),
      // U = [T1_Ea G1 ; T2_Eb G2] (restriction), Dm = [G_f2 | -G_f2 T1_aE1 | G_f1 | -G_f1 T2_bE2]
      const int g = P * 2 * m, u = P * 2 * p, dd = P * 2 * m;
      md[PG1A * NP + P] = D(0, 0, 0, 0, w, m, g, 0, m, m, 0);          // G1[:, f1] = S^{-1}
      md[PG1B * NP + P] = D(w, m, r2, 0, 0, 0, g, m, m, m, m);         // G1[:, f2] = -S^{-1} T2_bb
      md[PG2A * NP + P] = D(r1, 0, g, 0, 0, 0, g + m, 0, m, m, m);     // G2[:, f1] = -T1_aa G1[:, f1]
      md[PG2B * NP + P] = D(r1, 0, g, m, 0, 0, g + m, m, m, m, m);     // G2[:, f2] = I - T1_aa G1[:, f2]
      md[PU1 * NP + P] = D(r1 + m, 0, g, 0, 0, 0, u, 0, p, 2 * m, m);  // U[E1] = T1_Ea G1
      md[PU2 * NP + P] = D(r2 + m, 0, g + m, 0, 0, 0, u + p, 0, p, 2 * m, m);  // U[E2] = T2_Eb G2
      md[PD1 * NP + P] = D(0, 0, 0, 0, g, m, dd, 0, 2 * m, m, 0);      // Dm[:, f2] = G[:, f2]
      md[PD2 * NP + P] = D(g, m, r1, m, 0, 0, dd, m, 2 * m, p, m);     // Dm[:, e1] = -G[:, f2] T1_aE1
      md[PD3 * NP + P] = D(0, 0, 0, 0, g, 0, dd, n, 2 * m, m, 0);      // Dm[:, f1] = G[:, f1]
      md[PD4 * NP + P] = D(g, 0, r2, m, 0, 0, dd, n + m, 2 * m, p, m); // Dm[:, e2] = -G[:, f1] T2_bE2
      // sweeps (vector rows; n = -1 -> number of right-hand sides)
      // up:   rho'_[E1;E2] = rho_[E1;E2] - U [f1; f2],  f1 = child2 rows 0..m, f2 = child1 rows 0..m
      sd[SUP * NP + P] = D2(D(u, 0, r2, 0, r1 + m, 0, u, 0, 2 * p, -1, 2 * m, dm1, -1), r1, m, r2 + m, p);
      // down: x = Dm [child1 rows 0..n ; child2 rows 0..n]  (into the x workspace)
      sd[SDN * NP + P] = D2(D(dd, 0, r1, 0, 0, 0, g, 0, 2 * m, -1, 2 * n), r2, n, 0, 0);
    }
    {
      std::vector<int> xmap((size_t)NP * 2 * m);
      for (int P = 0; P < NP; ++P)
        for (int i = 0; i < 2 * m; ++i)
          xmap[(size_t)P * 2 * m + i] = i < m ? Lv.i1[P] * n + i : Lv.i2[P] * n + (i - m);
      Lv.d_xmap = dev_upload(c, xmap);
      if (!Lv.d_xmap) return fail(c, HPS_ENOMEM, "interface map");
    }
    Lv.d_mdesc = dev_upload(c, md);
    Lv.d_sdesc = dev_upload(c, sd);
    if (!Lv.d_mdesc || !Lv.d_sdesc) return fail(c, HPS_ENOMEM, "descriptors");
    {
      // the same sweep products on the tiled operators (every level: whether a level is tiled
      // depends on the sweep arithmetic of each tree): a_r = the pair's first 512-byte unit,
      // a_c = its k chunks
      const long long pu = tiled_pair_units(2 * p, 2 * m), pd = tiled_pair_units(2 * m, 2 * n);
      if ((long long)NP * std::max(pu, pd) > 0x7fffffffLL) return fail(c, HPS_EUNSUPPORTED, "tiled operator size");
      std::vector<GemmDesc> td(sd);
      for (int P = 0; P < NP; ++P) {
        td[SUP * NP + P].a_r = (int)(P * pu);
        td[SUP * NP + P].a_c = (2 * m + TILE_K - 1) / TILE_K;
        td[SDN * NP + P].a_r = (int)(P * pd);
        td[SDN * NP + P].a_c = (2 * n + TILE_K - 1) / TILE_K;
      }
      Lv.d_tsdesc = dev_upload(c, td);
      if (!Lv.d_tsdesc) return fail(c, HPS_ENOMEM, "descriptors");
    }
  }
  }  // plan
  // ---- allocations ----
  for (int k = 0; k <= L_exact; ++k) {
    Stage& S = c->stages[k];
    S.T = dev_alloc(c, sizeof(C) * (size_t)S.nsub * S.n * S.n);
    if (!S.T) return fail(c, HPS_ENOMEM, "stage maps");
    if (plan && (k == 0 || k == L_exact)) {
      S.d_es = dev_upload(c, S.es);
      if (!S.d_es) return fail(c, HPS_ENOMEM, "stage index");
    }
  }
  for (int l = 1; l <= L_exact; ++l) {
    Level& Lv = c->levels[l];
    Lv.W = dev_alloc(c, sizeof(C) * (size_t)Lv.npairs * Lv.m * 2 * Lv.m);
    Lv.U = dev_alloc(c, sizeof(C) * (size_t)Lv.npairs * 2 * Lv.p * 2 * Lv.m);
    Lv.Dm = dev_alloc(c, sizeof(C) * (size_t)Lv.npairs * 2 * Lv.m * 2 * Lv.n);
    if (!Lv.W || !Lv.U || !Lv.Dm) return fail(c, HPS_ENOMEM, "interface inverses and sweep operators");
  }
  if (L_exact > 0) {
    const size_t x_elems = c->plan_x_elems;
    const int max_pairs = c->plan_max_pairs;
    c->ws_X1 = dev_alloc(c, sizeof(C) * x_elems);
    c->ws_X2 = dev_alloc(c, sizeof(C) * x_elems);
    c->d_piv = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)max_pairs * GJ_NB));
    c->d_lu = dev_alloc(c, sizeof(C) * (size_t)max_pairs * GJ_NB * GJ_NB);
    if (!c->ws_X1 || !c->ws_X2 || !c->d_piv || !c->d_lu) return fail(c, HPS_ENOMEM, "merge workspace");
    c->ws_X_elems = x_elems;
  }
  {
    size_t g_elems = 1;
    int mmax = 1;
    for (int l = 1; l <= L_exact; ++l) {
      g_elems = std::max(g_elems, (size_t)c->levels[l].npairs * 4 * c->levels[l].m * c->levels[l].m);
      mmax = std::max(mmax, c->levels[l].m);
    }
    c->ws_G = dev_alloc(c, sizeof(C) * g_elems);
    std::vector<C> eye((size_t)mmax * mmax, mk<R>(R(0), R(0)));
    for (int i = 0; i < mmax; ++i) eye[(size_t)i * mmax + i] = mk<R>(R(1), R(0));
    c->d_eye = dev_alloc(c, sizeof(C) * eye.size());
    if (!c->ws_G || !c->d_eye) return fail(c, HPS_ENOMEM, "sweep-operator workspace");
    HPS_CK(c, cudaMemcpy(c->d_eye, eye.data(), sizeof(C) * eye.size(), cudaMemcpyHostToDevice));
    c->eye_ld = mmax;
  }
  c->gemm_ws_elems = (size_t)1 << 22;  // split-K partials
  c->gemm_ws = dev_alloc(c, sizeof(C) * c->gemm_ws_elems);
  if (!c->gemm_ws) return fail(c, HPS_ENOMEM, "split-K workspace");
  // ---- stage 0 maps from the FP64 leaf maps ----
  {
    const Stage& S0 = c->stages[0];
    if (plan) {
      std::vector<int> map0((size_t)S0.nsub * S0.n);
      for (int e = 0; e < S0.nsub; ++e)
        for (int i = 0; i < S0.n; ++i) map0[(size_t)e * S0.n + i] = S0.es[(size_t)e * S0.n + i] - e * c->nb;
      c->plan_map0 = dev_upload(c, map0);
      if (!c->plan_map0) return fail(c, HPS_ENOMEM, "stage-0 map");
    }
    HPS_CK(c, (permute_blocks<double, R>(static_cast<C*>(S0.T), c->d_T, c->plan_map0, S0.nsub, S0.n, c->stream)));
  }
  // ---- merges ----
  HPS_CK(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  for (int l = 1; l <= L_exact; ++l) {
    Level& Lv = c->levels[l];
    const Stage& P0 = c->stages[l - 1];
    const Stage& P1 = c->stages[l];
    const int n = Lv.n, m = Lv.m, p = Lv.p, NP = Lv.npairs;
    const GemmDesc* md = Lv.d_mdesc;
    const void* T0 = P0.T;
    HPS_CK(c, eye2<R>(static_cast<C*>(Lv.W), m, NP, c->stream));
    HPS_CK(c, gemm<R>(c, md + MS * NP, NP, T0, n, T0, n, Lv.W, 2 * m, Lv.W, 2 * m, -1.0, nullptr, m, m, m, m));
    HPS_CK(c, gj_invert<R>(static_cast<C*>(Lv.W), m, NP, c->d_piv, static_cast<C*>(c->d_lu), c->d_flag, c->stream));
    HPS_CK(c, gemm<R>(c, md + MR * NP, NP, T0, n, T0, n, nullptr, 0, c->ws_X2, 2 * p, -1.0, nullptr, m, p, p, m));
    HPS_CK(c, gemm<R>(c, md + MX1A * NP, NP, Lv.W, 2 * m, c->ws_X2, 2 * p, nullptr, 0, c->ws_X1, 2 * p, 1.0, nullptr, m,
                      p, p, m));
    HPS_CK(c, gemm<R>(c, md + MX1B * NP, NP, Lv.W, 2 * m, T0, n, nullptr, 0, c->ws_X1, 2 * p, 1.0, nullptr, m, p, p, m));
    HPS_CK(c, gemm<R>(c, md + MX2A * NP, NP, T0, n, c->ws_X1, 2 * p, T0, n, c->ws_X2, 2 * p, -1.0, nullptr, m, p, p, m));
    HPS_CK(c, gemm<R>(c, md + MX2B * NP, NP, T0, n, c->ws_X1, 2 * p, nullptr, 0, c->ws_X2, 2 * p, -1.0, nullptr, m, p,
                      p, m));
    void* Tn = P1.T;
    HPS_CK(c, gemm<R>(c, md + MOA * NP, NP, T0, n, c->ws_X1, 2 * p, T0, n, Tn, 2 * p, -1.0, Lv.d_dst, p, p, p, m));
    HPS_CK(c, gemm<R>(c, md + MOB * NP, NP, T0, n, c->ws_X1, 2 * p, nullptr, 0, Tn, 2 * p, -1.0, Lv.d_dst, p, p, p, m));
    HPS_CK(c, gemm<R>(c, md + MOC * NP, NP, T0, n, c->ws_X2, 2 * p, nullptr, 0, Tn, 2 * p, -1.0, Lv.d_dst, p, p, p, m));
    HPS_CK(c, gemm<R>(c, md + MOD * NP, NP, T0, n, c->ws_X2, 2 * p, T0, n, Tn, 2 * p, -1.0, Lv.d_dst, p, p, p, m));
    // sweep operators
    void* G = c->ws_G;
    HPS_CK(c, gemm<R>(c, md + PG1A * NP, NP, nullptr, 0, nullptr, 0, Lv.W, 2 * m, G, 2 * m, 1.0, nullptr, m, m, m));
    HPS_CK(c, gemm<R>(c, md + PG1B * NP, NP, Lv.W, 2 * m, T0, n, nullptr, 0, G, 2 * m, -1.0, nullptr, m, m, m, m));
    HPS_CK(c, gemm<R>(c, md + PG2A * NP, NP, T0, n, G, 2 * m, nullptr, 0, G, 2 * m, -1.0, nullptr, m, m, m, m));
    HPS_CK(c, gemm<R>(c, md + PG2B * NP, NP, T0, n, G, 2 * m, c->d_eye, c->eye_ld, G, 2 * m, -1.0, nullptr, m, m, m,
                      m));
    HPS_CK(c, gemm<R>(c, md + PU1 * NP, 2 * NP, T0, n, G, 2 * m, nullptr, 0, Lv.U, 2 * m, 1.0, nullptr, p, 2 * m,
                      2 * m, m));
    HPS_CK(c, gemm<R>(c, md + PD1 * NP, NP, nullptr, 0, nullptr, 0, G, 2 * m, Lv.Dm, 2 * n, 1.0, nullptr, 2 * m, m, m));
    HPS_CK(c, gemm<R>(c, md + PD3 * NP, NP, nullptr, 0, nullptr, 0, G, 2 * m, Lv.Dm, 2 * n, 1.0, nullptr, 2 * m, m, m));
    HPS_CK(c, gemm<R>(c, md + PD2 * NP, NP, G, 2 * m, T0, n, nullptr, 0, Lv.Dm, 2 * n, -1.0, nullptr, 2 * m, p, p, m));
    HPS_CK(c, gemm<R>(c, md + PD4 * NP, NP, G, 2 * m, T0, n, nullptr, 0, Lv.Dm, 2 * n, -1.0, nullptr, 2 * m, p, p, m));
    if (sizeof(R) == 4 && level_tiled(c, Lv)) {
      // the sweeps stream U and Dm block by block: keep them tiled, drop the row-major copies
      const size_t bu = (size_t)NP * tiled_pair_units(2 * p, 2 * m) * TILE_UNIT;
      const size_t bd = (size_t)NP * tiled_pair_units(2 * m, 2 * n) * TILE_UNIT;
      Lv.Ut = dev_alloc(c, sizeof(float2) * bu);
      Lv.Dmt = dev_alloc(c, sizeof(float2) * bd);
      if (!Lv.Ut || !Lv.Dmt) return fail(c, HPS_ENOMEM, "tiled sweep operators");
      auto tile = c->sweep_bf16x3 ? tile_operator_bf16x3 : tile_operator;
      HPS_CK(c, tile(static_cast<float2*>(Lv.Ut), static_cast<const float2*>(Lv.U), NP, 2 * p, 2 * m, 2 * m,
                     (long long)2 * p * 2 * m, c->stream));
      HPS_CK(c, tile(static_cast<float2*>(Lv.Dmt), static_cast<const float2*>(Lv.Dm), NP, 2 * m, 2 * n, 2 * n,
                     (long long)2 * m * 2 * n, c->stream));
      dev_free(c, Lv.U);
      dev_free(c, Lv.Dm);
      Lv.U = Lv.Dm = nullptr;
    }
  }
  // ---- coarse level ----
  {
    const Stage& Sc = c->stages[L_exact];
    Coarse& cc = c->coarse;
    if (plan) {
    std::vector<int> cnb((size_t)Sc.nsub * Sc.n, -1), upos, ucnb;
    std::vector<GemmDesc> cdesc(Sc.nsub);
    int max_int = 0;
    for (int sy = 0; sy < Sc.gy; ++sy)
      for (int sx = 0; sx < Sc.gx; ++sx) {
        const int s = sx + Sc.gx * sy;
        const int ni = ((sx > 0) + (sx < Sc.gx - 1)) * Sc.b * q + ((sy > 0) + (sy < Sc.gy - 1)) * Sc.a * q;
        cdesc[s] = D(s * Sc.n, 0, s * Sc.n, 0, 0, 0, s * Sc.n, 0, ni, -1, ni);
        max_int = std::max(max_int, ni);
      }
    cc.max_int = max_int;
    std::vector<int> owner(c->n_es, -1);
    for (int s = 0; s < Sc.nsub; ++s)
      for (int i = 0; i < Sc.n; ++i) owner[Sc.es[(size_t)s * Sc.n + i]] = s;
    for (int s = 0; s < Sc.nsub; ++s)
      for (int i = 0; i < Sc.n; ++i) {
        const size_t r = (size_t)s * Sc.n + i;
        const int en = c->es_nb[Sc.es[r]];
        if (en < 0) continue;
        const int so = owner[en];
        const int d = inv[L_exact][en];
        if (so < 0 || so == s || d < 0) return fail(c, HPS_ECUDA, "internal: coarse neighbour map");
        cnb[r] = so * Sc.n + d;
        if (i >= cdesc[s].m) return fail(c, HPS_ECUDA, "internal: coarse interior order");
        upos.push_back((int)r);
      }
    cc.n_int = (int)upos.size();
    for (int u = 0; u < cc.n_int; ++u) ucnb.push_back(cnb[upos[u]]);
    {
      // the same products on the tiled operators: a_r = the subdomain's first unit, a_c = its k chunks
      const long long units = tiled_pair_units(max_int, max_int);
      if ((long long)Sc.nsub * units > 0x7fffffffLL) return fail(c, HPS_EUNSUPPORTED, "tiled coarse operator size");
      std::vector<GemmDesc> tcd(cdesc);
      for (int s2 = 0; s2 < Sc.nsub; ++s2) {
        tcd[s2].a_r = (int)(s2 * units);
        tcd[s2].a_c = (max_int + TILE_K - 1) / TILE_K;
      }
      cc.d_tcdesc = dev_upload(c, tcd);
      if (!cc.d_tcdesc) return fail(c, HPS_ENOMEM, "coarse descriptors");
    }
    cc.d_cdesc = dev_upload(c, cdesc);
    cc.d_cnb = dev_upload(c, cnb);
    cc.d_upos = dev_upload(c, upos);
    cc.d_ucnb = dev_upload(c, ucnb);
    if (!cc.d_cdesc || !cc.d_cnb || !cc.d_upos || !cc.d_ucnb) return fail(c, HPS_ENOMEM, "coarse maps");
    cc.upos_h = upos;
    cc.ucnb_h = ucnb;
    // gamma-cycle: the system of every stage k >= 1 (row across the face, one n x n product
    // per subdomain)
    for (int k = 1; k <= L_exact; ++k) {
      Stage& Sk = c->stages[k];
      std::vector<int> own(c->n_es, -1), nbk((size_t)Sk.nsub * Sk.n, -1);
      for (int s = 0; s < Sk.nsub; ++s)
        for (int i = 0; i < Sk.n; ++i) own[Sk.es[(size_t)s * Sk.n + i]] = s;
      std::vector<GemmDesc> td(Sk.nsub);
      for (int s = 0; s < Sk.nsub; ++s) {
        td[s] = D(s * Sk.n, 0, s * Sk.n, 0, 0, 0, s * Sk.n, 0, Sk.n, -1, Sk.n);
        for (int i = 0; i < Sk.n; ++i) {
          const int en = c->es_nb[Sk.es[(size_t)s * Sk.n + i]];
          if (en < 0) continue;
          const int so = own[en], d = inv[k][en];
          if (so < 0 || so == s || d < 0) return fail(c, HPS_ECUDA, "internal: stage neighbour map");
          nbk[(size_t)s * Sk.n + i] = so * Sk.n + d;
        }
      }
      Sk.d_nb = dev_upload(c, nbk);
      Sk.d_tdesc = dev_upload(c, td);
      if (!Sk.d_nb || !Sk.d_tdesc) return fail(c, HPS_ENOMEM, "stage maps for the gamma-cycle");
    }
    }  // plan
    cc.exact = exact != 0;
    const std::vector<int>& upos = cc.upos_h;
    const std::vector<int>& ucnb = cc.ucnb_h;
    if (cc.exact && cc.n_int > 0) {
      const int ni = cc.n_int;
      cc.Winv = dev_alloc(c, sizeof(C) * (size_t)ni * 2 * ni);
      if (!cc.Winv) return fail(c, HPS_ENOMEM, "coarse inverse");
      // dense M_c = I + Pi T_c on the interior positions, then [M_c | I] -> [. | M_c^{-1}]
      std::vector<int> compact((size_t)Sc.nsub * Sc.n, -1);
      for (int u = 0; u < ni; ++u) compact[upos[u]] = u;
      // host assembly from a host copy of T_c (small by construction of the exact mode)
      std::vector<C> Th((size_t)Sc.nsub * Sc.n * Sc.n);
      HPS_CK(c, cudaStreamSynchronize(c->stream));
      HPS_CK(c, cudaMemcpy(Th.data(), Sc.T, sizeof(C) * Th.size(), cudaMemcpyDeviceToHost));
      std::vector<C> Wh((size_t)ni * 2 * ni);
      for (auto& z : Wh) z = mk<R>(R(0), R(0));
      for (int u = 0; u < ni; ++u) {
        Wh[(size_t)u * 2 * ni + u] = mk<R>(R(1), R(0));
        Wh[(size_t)u * 2 * ni + ni + u] = mk<R>(R(1), R(0));
        const int across = ucnb[u];
        const int so = across / Sc.n, io = across % Sc.n;
        for (int j = 0; j < Sc.n; ++j) {
          const int v = compact[(size_t)so * Sc.n + j];
          if (v < 0) continue;
          const C t = Th[((size_t)so * Sc.n + io) * Sc.n + j];
          C& dst = Wh[(size_t)u * 2 * ni + v];
          dst.x += t.x;
          dst.y += t.y;
        }
      }
      HPS_CK(c, cudaMemcpy(cc.Winv, Wh.data(), sizeof(C) * Wh.size(), cudaMemcpyHostToDevice));
      std::vector<GemmDesc> dd(1, D(0, ni, 0, 0, 0, 0, 0, 0, ni, -1, ni));
      cc.d_desc = dev_upload(c, dd);
      if (!cc.d_desc) return fail(c, HPS_ENOMEM, "coarse descriptor");
      int* piv = static_cast<int*>(dev_alloc(c, sizeof(int) * GJ_NB));
      void* lu = dev_alloc(c, sizeof(C) * GJ_NB * GJ_NB);
      if (!piv || !lu) return fail(c, HPS_ENOMEM, "coarse workspace");
      HPS_CK(c, gj_invert<R>(static_cast<C*>(cc.Winv), ni, 1, piv, static_cast<C*>(lu), c->d_flag, c->stream));
      HPS_CK(c, cudaStreamSynchronize(c->stream));
      dev_free(c, piv);
      dev_free(c, lu);
    }
    if (sizeof(R) == 4 && !cc.exact && c->sweep_bf16x3 && cc.max_int > 0) {
      // the coarse GMRES streams T_int,int once per step: keep it tiled in three bf16 terms
      // (12 bytes per entry) for the sweep kernel's six-product path
      const size_t bytes = (size_t)Sc.nsub * tiled_pair_units(cc.max_int, cc.max_int) * TILE_UNIT * 12;
      cc.Tt = dev_alloc(c, bytes);
      if (!cc.Tt) return fail(c, HPS_ENOMEM, "tiled coarse operator");
      HPS_CK(c, tile_operator_bf16x6(cc.Tt, static_cast<const float2*>(Sc.T), Sc.nsub, cc.max_int, cc.max_int, Sc.n,
                                     (long long)Sc.n * Sc.n, c->stream));
      ++c->vc_gen;
    }
  }
  int flag = 0;
  HPS_CK(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HPS_CK(c, cudaStreamSynchronize(c->stream));
  if (flag) return fail(c, HPS_ENUMERIC, "zero pivot in an interface or coarse inversion");
  c->plan_L = L_exact;
  c->have_tree = true;
  return HPS_OK;
}

}  // namespace

int build_tree(hps_ctx* c, int L_exact, int exact_coarse) {
  if (c->plan_L == L_exact) free_numeric(c);  // same mesh and depth: keep the plan
  else free_tree(c);
  PhaseScope ps(c, HPS_PH_MERGE);
  // the format of this tree's tiled sweep operators (FP32 tree only)
  c->sweep_bf16x3 = c->precision != HPS_FP64 && c->sweep_arith != HPS_SWEEP_FP32;
  int rc = c->precision == HPS_FP64 ? build_tree_t<double>(c, L_exact, exact_coarse)
                                    : build_tree_t<float>(c, L_exact, exact_coarse);
  if (rc != HPS_OK) {
    cudaStreamSynchronize(c->stream);
    free_tree(c);
  }
  return rc;
}

int ensure_sweep_buffers(hps_ctx* c, int nrhs) {
  if (nrhs <= c->nrhs_cap) return HPS_OK;
  const size_t cs = csize(c->precision);
  for (auto& S : c->stages) {
    dev_free(c, S.vec);
    S.vec = dev_alloc(c, cs * (size_t)S.nsub * S.n * nrhs);
    if (!S.vec) return fail(c, HPS_ENOMEM, "sweep vectors");
  }
  size_t pm = 1, p2m = 1;
  for (int l = 1; l <= c->L_exact; ++l) {
    pm = std::max(pm, (size_t)c->levels[l].npairs * c->levels[l].m);
    p2m = std::max(p2m, (size_t)c->levels[l].npairs * 2 * c->levels[l].m);
  }
  (void)pm;
  dev_free(c, c->sw_x);
  c->sw_x = dev_alloc(c, cs * p2m * nrhs);
  if (!c->sw_x) return fail(c, HPS_ENOMEM, "sweep temporaries");
  c->nrhs_cap = nrhs;
  ++c->vc_gen;
  return HPS_OK;
}

int ensure_gamma_buffers(hps_ctx* c, int nrhs) {
  if (c->gamma <= 1 || nrhs <= c->gamma_nrhs) return HPS_OK;
  const size_t cs = csize(c->precision);
  size_t wmax = 1;
  for (int k = 1; k <= c->L_exact; ++k) {
    Stage& S = c->stages[k];
    const size_t el = (size_t)S.nsub * S.n * nrhs;
    dev_free(c, S.gR);
    dev_free(c, S.gE);
    S.gR = dev_alloc(c, cs * el);
    S.gE = dev_alloc(c, cs * el);
    if (!S.gR || !S.gE) return fail(c, HPS_ENOMEM, "gamma-cycle vectors");
    wmax = std::max(wmax, el);
  }
  dev_free(c, c->gW);
  c->gW = dev_alloc(c, cs * wmax);
  if (!c->gW) return fail(c, HPS_ENOMEM, "gamma-cycle product");
  c->gamma_nrhs = nrhs;
  ++c->vc_gen;
  return HPS_OK;
}

namespace {

template <typename R>
int ensure_cg(hps_ctx* c, int k, int nrhs) {
  if (k <= c->cg_k && nrhs <= c->cg_nrhs) return HPS_OK;
  k = std::max(k, c->cg_k);
  nrhs = std::max(nrhs, c->cg_nrhs);
  const Stage& Sc = c->stages[c->L_exact];
  const size_t rows = (size_t)Sc.nsub * Sc.n;
  const size_t cs = sizeof(c_t<R>);
  void** bufs[] = {&c->cg_V, &c->cg_w, &c->cg_W, &c->cg_H, &c->cg_h1, &c->cg_h2, &c->cg_nrm,
                   &c->cg_y, &c->cg_g, &c->cg_s, &c->cg_part, &c->cg_beta, &c->cg_floor, &c->cg_c,
                   &c->cg_inv, &c->cg_cnt};
  for (void** b : bufs) {
    dev_free(c, *b);
    *b = nullptr;
  }
  c->cg_V = dev_alloc(c, cs * (k + 1) * rows * nrhs);
  c->cg_w = dev_alloc(c, cs * rows * nrhs);
  c->cg_W = dev_alloc(c, cs * rows * nrhs);
  c->cg_H = dev_alloc(c, cs * (size_t)nrhs * (k + 1) * k);
  c->cg_h1 = dev_alloc(c, cs * (size_t)(k + 1) * nrhs);
  c->cg_h2 = dev_alloc(c, cs * (size_t)(k + 1) * nrhs);
  c->cg_nrm = dev_alloc(c, cs * nrhs);
  c->cg_y = dev_alloc(c, cs * (size_t)k * nrhs);
  c->cg_g = dev_alloc(c, cs * (size_t)(k + 1) * nrhs);
  c->cg_s = dev_alloc(c, cs * (size_t)k * nrhs);
  const int fb = cg_pass_blocks((long long)rows, nrhs);
  const size_t np = std::max((size_t)bdot_blocks((long long)rows), (size_t)fb + cg_groups(fb));
  c->cg_part = dev_alloc(c, cs * np * (k + 1) * nrhs);
  c->cg_part_cap = (long long)np * (k + 1) * nrhs;
  c->cg_beta = dev_alloc(c, sizeof(R) * nrhs);
  c->cg_floor = dev_alloc(c, sizeof(R) * nrhs);
  c->cg_c = dev_alloc(c, sizeof(R) * (size_t)k * nrhs);
  c->cg_inv = dev_alloc(c, sizeof(R) * nrhs);
  const size_t ncnt = 1 + (size_t)cg_groups(fb);
  c->cg_cnt = dev_alloc(c, sizeof(unsigned) * ncnt);
  c->cg_cnt_cap = (int)ncnt;
  for (void** b : bufs)
    if (!*b) return fail(c, HPS_ENOMEM, "coarse GMRES workspace");
  if (cudaMemsetAsync(c->cg_cnt, 0, sizeof(unsigned) * ncnt, c->stream) != cudaSuccess) return fail(c, HPS_ECUDA, "coarse GMRES counter");
  c->cg_k = k;
  ++c->vc_gen;
  c->cg_nrhs = nrhs;
  return HPS_OK;
}

template <typename R>
int ensure_ex(hps_ctx* c, int nrhs) {
  using C = c_t<R>;
  if (nrhs <= c->ex_nrhs) return HPS_OK;
  const Coarse& cc = c->coarse;
  dev_free(c, c->ex_r);
  dev_free(c, c->ex_e);
  c->ex_r = dev_alloc(c, sizeof(C) * (size_t)std::max(cc.n_int, 1) * nrhs);
  c->ex_e = dev_alloc(c, sizeof(C) * (size_t)std::max(cc.n_int, 1) * nrhs);
  ++c->vc_gen;
  if (!c->ex_r || !c->ex_e) return fail(c, HPS_ENOMEM, "exact coarse scratch");
  c->ex_nrhs = nrhs;
  return HPS_OK;
}

template <typename R>
int coarse_solve(hps_ctx* c, int nrhs, int k) {
  using C = c_t<R>;
  const Stage& Sc = c->stages[c->L_exact];
  const Coarse& cc = c->coarse;
  const long long rows = (long long)Sc.nsub * Sc.n;
  C* Vc = static_cast<C*>(Sc.vec);
  cudaStream_t st = c->stream;
  if (cc.n_int == 0 || (!cc.exact && k <= 0)) {
    HPS_CK(c, zero<R>(Vc, rows * nrhs, st));
    return HPS_OK;
  }
  if (cc.exact) {
    int rc0 = ensure_ex<R>(c, nrhs);
    if (rc0 != HPS_OK) return rc0;
    HPS_CK(c, (gather_rows<R, R>(static_cast<C*>(c->ex_r), Vc, cc.d_ucnb, cc.n_int, nrhs, st)));
    HPS_CK(c, gemm<R>(c, cc.d_desc, 1, cc.Winv, 2LL * cc.n_int, c->ex_r, nrhs, nullptr, 0, c->ex_e, nrhs, 1.0, nullptr,
                      cc.n_int, nrhs, nrhs));
    HPS_CK(c, zero<R>(Vc, rows * nrhs, st));
    HPS_CK(c, (scatter_rows<R, R>(Vc, static_cast<C*>(c->ex_e), cc.d_upos, cc.n_int, nrhs, st)));
    return HPS_OK;
  }
  int rc = ensure_cg<R>(c, k, nrhs);
  if (rc != HPS_OK) return rc;
  C* V = static_cast<C*>(c->cg_V);
  C* w = static_cast<C*>(c->cg_w);
  C* W = static_cast<C*>(c->cg_W);
  C* h1 = static_cast<C*>(c->cg_h1);
  C* h2 = static_cast<C*>(c->cg_h2);
  C* nrm = static_cast<C*>(c->cg_nrm);
  C* part = static_cast<C*>(c->cg_part);
  R* beta = static_cast<R*>(c->cg_beta);
  R* floor = static_cast<R*>(c->cg_floor);
  const long long vs = rows * nrhs;
  const R tol = sizeof(R) == 8 ? R(1e-14) : R(1e-6);
  if (cg_pass_fits<R>(k, nrhs)) {
    // fused passes: start, then per step the operator product of the unnormalised w and
    // three passes (apply + first projection, second projection, norm + Hessenberg column)
    CgPass<R> p;
    p.V = V;
    p.vs = vs;
    p.w = w;
    p.W = W;
    p.g = Vc;
    p.nb = cc.d_cnb;
    p.rows = rows;
    p.nrhs = nrhs;
    p.k = k;
    p.part = part;
    p.cnt = static_cast<unsigned*>(c->cg_cnt);
    p.part_cap = c->cg_part_cap;
    p.cnt_cap = c->cg_cnt_cap;
    p.h1 = h1;
    p.h2 = h2;
    p.H = static_cast<C*>(c->cg_H);
    p.beta = beta;
    p.floor = floor;
    p.inv = static_cast<R*>(c->cg_inv);
    p.tol = tol;
    HPS_CK(c, cg_pass<R>(CG_START, p, st));
    for (int j = 0; j < k; ++j) {
      p.j = j;
      if (cc.Tt)
        HPS_CK(c, gemm_tiled(c, cc.d_tcdesc, Sc.nsub, cc.Tt, w, nrhs, nullptr, 0, W, nrhs, 1.0, nullptr, cc.max_int,
                             nrhs, nrhs, cc.max_int, 3));
      else
        HPS_CK(c, gemm<R>(c, cc.d_cdesc, Sc.nsub, Sc.T, Sc.n, w, nrhs, nullptr, 0, W, nrhs, 1.0, nullptr, cc.max_int,
                          nrhs, nrhs, cc.max_int));
      HPS_CK(c, cg_pass<R>(CG_APPLY, p, st));
      HPS_CK(c, cg_pass<R>(CG_PROJECT, p, st));
      HPS_CK(c, cg_pass<R>(CG_CLOSE, p, st));
    }
    HPS_CK(c, lsq<R>(static_cast<C*>(c->cg_H), beta, floor, static_cast<C*>(c->cg_y), static_cast<C*>(c->cg_g),
                     static_cast<R*>(c->cg_c), static_cast<C*>(c->cg_s), k, nrhs, st));
    HPS_CK(c, bcombine<R>(Vc, V, vs, k, static_cast<C*>(c->cg_y), rows, nrhs, st));
    return HPS_OK;
  }
  // r_c = Pi rho_c (incoming coordinates of the coarse unknowns)
  HPS_CK(c, swap_add<R>(w, nullptr, Vc, cc.d_cnb, rows, nrhs, st));
  HPS_CK(c, bdot<R>(w, 0, 1, w, rows, nrhs, part, nrm, 0, st));
  HPS_CK(c, beta_floor<R>(beta, floor, nrm, tol, nrhs, st));
  HPS_CK(c, bscale<R>(V, w, nrm, nullptr, rows, nrhs, st));
  for (int j = 0; j < k; ++j) {
    C* Vj = V + j * vs;
    if (cc.Tt)
      HPS_CK(c, gemm_tiled(c, cc.d_tcdesc, Sc.nsub, cc.Tt, Vj, nrhs, nullptr, 0, W, nrhs, 1.0, nullptr, cc.max_int, nrhs,
                           nrhs, cc.max_int, 3));
    else
      HPS_CK(c, gemm<R>(c, cc.d_cdesc, Sc.nsub, Sc.T, Sc.n, Vj, nrhs, nullptr, 0, W, nrhs, 1.0, nullptr, cc.max_int,
                        nrhs, nrhs, cc.max_int));
    HPS_CK(c, swap_add<R>(w, Vj, W, cc.d_cnb, rows, nrhs, st));
    HPS_CK(c, bdot<R>(V, vs, j + 1, w, rows, nrhs, part, h1, 0, st));
    HPS_CK(c, (bupdate<R, R>(w, V, vs, j + 1, h1, rows, nrhs, R(-1), st)));
    HPS_CK(c, bdot<R>(V, vs, j + 1, w, rows, nrhs, part, h2, 0, st));
    HPS_CK(c, (bupdate<R, R>(w, V, vs, j + 1, h2, rows, nrhs, R(-1), st)));
    HPS_CK(c, bdot<R>(w, 0, 1, w, rows, nrhs, part, nrm, 0, st));
    HPS_CK(c, hstore<R>(static_cast<C*>(c->cg_H), h1, h2, nrm, j, k, nrhs, st));
    HPS_CK(c, bscale<R>(V + (j + 1) * vs, w, nrm, floor, rows, nrhs, st));
  }
  HPS_CK(c, lsq<R>(static_cast<C*>(c->cg_H), beta, floor, static_cast<C*>(c->cg_y), static_cast<C*>(c->cg_g),
                   static_cast<R*>(c->cg_c), static_cast<C*>(c->cg_s), k, nrhs, st));
  HPS_CK(c, zero<R>(Vc, rows * nrhs, st));
  HPS_CK(c, (bupdate<R, R>(Vc, V, vs, k, static_cast<C*>(c->cg_y), rows, nrhs, R(1), st)));
  return HPS_OK;
}


// MG of the stage-l system (section 4.3): the residual in P_l.vec on entry (outgoing
// coordinates), the correction in P_l.vec on return (incoming coordinates).  Below the coarse
// stage: the up-sweep of merge level l+1 (smoother A^{-1} and restriction), the stage-(l+1)
// system solved by gamma calls of this function, each on the current residual
// r_c - M_{l+2} e (gamma = 1: one call, the V-cycle), then the down-sweep (prolongation).
template <typename R>
int mg_level(hps_ctx* c, int l, int nrhs, int k) {
  using C = c_t<R>;
  if (l == c->L_exact) return coarse_solve<R>(c, nrhs, k);
  cudaStream_t st = c->stream;
  const Level& Lv = c->levels[l + 1];
  const Stage& P0 = c->stages[l];
  const Stage& P1 = c->stages[l + 1];
  const int n = Lv.n, m = Lv.m, p = Lv.p, NP = Lv.npairs;
  // up-sweep: rho'_E = rho_E - U f
  if (Lv.Ut)
    HPS_CK(c, gemm_tiled(c, Lv.d_tsdesc + SUP * NP, NP, Lv.Ut, P0.vec, nrhs, P0.vec, nrhs, P1.vec, nrhs, -1.0,
                         Lv.d_dst, 2 * p, nrhs, nrhs, 2 * m, c->sweep_bf16x3 ? 2 : 0));
  else
    HPS_CK(c, gemm<R>(c, Lv.d_sdesc + SUP * NP, NP, Lv.U, 2 * m, P0.vec, nrhs, P0.vec, nrhs, P1.vec, nrhs, -1.0,
                      Lv.d_dst, 2 * p, nrhs, nrhs, 2 * m));
  if (c->gamma <= 1) {
    int rc = mg_level<R>(c, l + 1, nrhs, k);
    if (rc != HPS_OK) return rc;
  } else {
    const long long rows = (long long)P1.nsub * P1.n;
    C* v1 = static_cast<C*>(P1.vec);
    C* gR = static_cast<C*>(P1.gR);
    C* gE = static_cast<C*>(P1.gE);
    HPS_CK(c, cudaMemcpyAsync(gR, v1, sizeof(C) * rows * nrhs, cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < c->gamma; ++it) {
      if (it > 0) {  // P1.vec = r_c - M_{l+2} e:  (M e)_r = e_{nb(r)} + (T e)_r
        HPS_CK(c, gemm<R>(c, P1.d_tdesc, P1.nsub, P1.T, P1.n, gE, nrhs, nullptr, 0, c->gW, nrhs, 1.0, nullptr, P1.n,
                          nrhs, nrhs, P1.n));
        HPS_CK(c, stage_residual<R>(v1, gR, gE, static_cast<const C*>(c->gW), P1.d_nb, rows, nrhs, st));
      }
      int rc = mg_level<R>(c, l + 1, nrhs, k);
      if (rc != HPS_OK) return rc;
      HPS_CK(c, accumulate<R>(gE, v1, rows * nrhs, it == 0, it == c->gamma - 1 ? v1 : nullptr, st));
    }
  }
  // down-sweep: children's outer rows from the merged solution, x = Dm [child1; child2], x into the interface rows
  C* v0 = static_cast<C*>(P0.vec);
  HPS_CK(c, (scatter_rows<R, R>(v0, static_cast<const C*>(P1.vec), Lv.d_up, (long long)P1.nsub * P1.n, nrhs, st)));
  if (Lv.Dmt)
    HPS_CK(c, gemm_tiled(c, Lv.d_tsdesc + SDN * NP, NP, Lv.Dmt, v0, nrhs, nullptr, 0, c->sw_x, nrhs, 1.0, nullptr,
                         2 * m, nrhs, nrhs, 2 * n, c->sweep_bf16x3 ? 2 : 0));
  else
    HPS_CK(c, gemm<R>(c, Lv.d_sdesc + SDN * NP, NP, Lv.Dm, 2 * n, v0, nrhs, nullptr, 0, c->sw_x, nrhs, 1.0, nullptr,
                      2 * m, nrhs, nrhs, 2 * n));
  HPS_CK(c, (scatter_rows<R, R>(v0, static_cast<const C*>(c->sw_x), Lv.d_xmap, (long long)NP * 2 * m, nrhs, st)));
  return HPS_OK;
}

// One MG application on the stage-0 sweep vector: rho in S0.vec on entry, z in S0.vec on return.
template <typename R>
int mg_core(hps_ctx* c, int nrhs, int k) {
  return mg_level<R>(c, 0, nrhs, k);
}

}  // namespace

template <typename R>
int mg_apply(hps_ctx* c, const double2* rho_es, double2* z_es, int nrhs, int k) {
  using C = c_t<R>;
  int rc = ensure_sweep_buffers(c, nrhs);
  if (rc == HPS_OK) rc = ensure_gamma_buffers(c, nrhs);
  if (rc != HPS_OK) return rc;
  cudaStream_t st = c->stream;
  const Stage& S0 = c->stages[0];
  const long long rows = (long long)S0.nsub * S0.n;
  HPS_CK(c, (gather_rows<double, R>(static_cast<C*>(S0.vec), rho_es, S0.d_es, rows, nrhs, st)));
  rc = mg_core<R>(c, nrhs, k);
  if (rc != HPS_OK) return rc;
  HPS_CK(c, (scatter_rows<R, double>(z_es, static_cast<const C*>(S0.vec), S0.d_es, rows, nrhs, st)));
  return HPS_OK;
}

int mg_apply_df(hps_ctx* c, const float4* rho_es, float2* z_es, int nrhs, int k) {
  int rc = ensure_sweep_buffers(c, nrhs);
  if (rc == HPS_OK) rc = ensure_gamma_buffers(c, nrhs);
  if (rc != HPS_OK) return rc;
  if (c->precision != HPS_MIXED) return fail(c, HPS_EINVAL, "internal: df64 outer needs the FP32 tree");
  // every buffer the V-cycle touches exists before a capture
  if (c->coarse.exact) rc = ensure_ex<float>(c, nrhs);
  else if (c->coarse.n_int > 0 && k > 0) rc = ensure_cg<float>(c, k, nrhs);
  if (rc != HPS_OK) return rc;
  cudaStream_t st = c->stream;
  if (!c->mg_ptr) {
    c->mg_ptr = static_cast<void**>(dev_alloc(c, 2 * sizeof(void*)));
    if (!c->mg_ptr) return fail(c, HPS_ENOMEM, "V-cycle pointer block");
  }
  // this call's vectors go to the device by kernel arguments, stream-ordered before the graph
  HPS_CK(c, set_pointers(c->mg_ptr, rho_es, z_es, st));
  const Stage& S0 = c->stages[0];
  const long long rows = (long long)S0.nsub * S0.n;
  auto body = [&]() -> int {  // launches on c->stream (the capture stream while capturing)
    HPS_CK(c, df_gather_hi_ind(static_cast<float2*>(S0.vec), reinterpret_cast<const float4* const*>(c->mg_ptr),
                               S0.d_es, rows, nrhs, c->stream));
    int r2 = mg_core<float>(c, nrhs, k);
    if (r2 != HPS_OK) return r2;
    HPS_CK(c, scatter_f2_ind(reinterpret_cast<float2* const*>(c->mg_ptr) + 1, static_cast<const float2*>(S0.vec),
                             S0.d_es, rows, nrhs, c->stream));
    return HPS_OK;
  };
  if (c->mg_nograph) return body();
  // the graph runs on the context's own capture stream, ordered after and before the caller's
  // stream by events (the caller's stream may be the legacy default stream, which cannot capture)
  if (!c->gs) {
    if (cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gs_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->gs_out, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      c->mg_nograph = true;
      return body();
    }
  }
  const bool recapture =
      !(c->mg_exec && c->mg_nrhs == nrhs && c->mg_k == k && c->mg_gamma == c->gamma && c->mg_gen == c->vc_gen);
  if (recapture && c->tune == HPS_TUNE_ON &&
      !(c->tune_pass_gen == c->vc_gen && c->tune_pass_nrhs == nrhs && c->tune_pass_k == k &&
        c->tune_pass_gamma == c->gamma)) {
    // one direct application first, so that the autotuner times this V-cycle's shapes (it
    // cannot while they are captured); the next application captures the tuned launches
    c->tune_pass_gen = c->vc_gen;
    c->tune_pass_nrhs = nrhs;
    c->tune_pass_k = k;
    c->tune_pass_gamma = c->gamma;
    return body();
  }
  HPS_CK(c, cudaEventRecord(c->gs_in, st));
  HPS_CK(c, cudaStreamWaitEvent(c->gs, c->gs_in, 0));
  if (recapture) {
    if (c->mg_exec) cudaGraphExecDestroy(c->mg_exec);
    c->mg_exec = nullptr;
    // one capture at a time in the process (contexts of several host threads)
    static std::mutex capture_mu;
    std::lock_guard<std::mutex> lk(capture_mu);
    const long long l0 = hps_kernel_launches();
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      c->mg_nograph = true;
      return body();
    }
    c->stream = c->gs;  // every launch of the V-cycle goes to the capture stream
    const int rb = body();
    c->stream = st;
    const cudaError_t ec = cudaStreamEndCapture(c->gs, &graph);
    const long long captured = hps_kernel_launches() - l0;
    note_launch(-(int)captured);  // recorded into the graph, not run: counted per replay
    cudaError_t ei = cudaErrorUnknown;
    if (rb == HPS_OK && ec == cudaSuccess && graph) ei = cudaGraphInstantiate(&c->mg_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      // no graph on this context from now on: the same launches run directly
      cudaGetLastError();
      c->mg_exec = nullptr;
      c->mg_nograph = true;
      return body();
    }
    c->mg_nrhs = nrhs;
    c->mg_k = k;
    c->mg_gamma = c->gamma;
    c->mg_gen = c->vc_gen;
    c->mg_count = captured;
  }
  HPS_CK(c, cudaGraphLaunch(c->mg_exec, c->gs));
  HPS_CK(c, cudaEventRecord(c->gs_out, c->gs));
  HPS_CK(c, cudaStreamWaitEvent(st, c->gs_out, 0));
  note_launch((int)c->mg_count);
  return HPS_OK;
}

template int mg_apply<double>(hps_ctx*, const double2*, double2*, int, int);
template int mg_apply<float>(hps_ctx*, const double2*, double2*, int, int);

}  // namespace hps

namespace hps {
void subdomain_natural(const hps_ctx* c, int stage, int sub, std::vector<int>& out) {
  const Stage& S = c->stages[stage];
  natural_es(c, sub % S.gx, sub / S.gx, S.a, S.b, out);
}
}  // namespace hps
