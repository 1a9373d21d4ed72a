// Batched leaf impedance-to-impedance maps (section 3.1, eq. ItIOperator), FP64.
//
// The paper defines T = I_o L^{-1} I(:, iota_Gamma) with L the element matrix
// whose boundary rows are the incoming impedance operator I_i = Dn + i eta and
// whose interior rows are those of L~ = K(x)M + M(x)K - diag(c) M(x)M.  Solving
// L y = e_gamma by block elimination of the interior unknowns gives the same T:
//
//   interior rows:  L~_iG y_G + L~_ii y_i = 0       =>  y_i = -Z y_G,  Z = L~_ii^{-1} L~_iG
//   boundary rows:  (Dn_GG - Dn_Gi Z + i eta) y_G = e_gamma
//   => Y_G = P^{-1},  P = A + i eta I,  A = Dn_GG - Dn_Gi Z   (real, 4q x 4q)
//   => T = I_o Y = Dn Y - i eta Y_G = I - 2 i eta P^{-1}.
//
// L~_ii is real and symmetric; it is positive definite when
// c < lambda_min(K(x)M + M(x)K, M(x)M) on the interior (the host checks this
// with a rigorous bound before launching), so Z comes from a real L D L^T
// (square-root-free Cholesky) factorisation in shared memory (packed unit lower
// triangle with d on the diagonal, 203 KB at N = 16): every update of the
// factorisation and of the two triangular solves is a single FP64 FMA.
// The 4q x 4q complex P is inverted by Gauss-Jordan with partial pivoting.
//
// One persistent CTA per SM (the factor needs almost all of the 227 KB of
// shared memory); CTAs stride over the elements.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "dense.cuh"
#include "dfops.cuh"
#include "skel.cuh"

namespace hps {

namespace {

__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

__global__ void __launch_bounds__(256, 1) leaf_kernel(LeafParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1, cw = p.cw;
  const int npk = ni * (ni + 1) / 2;
  double* Lp = reinterpret_cast<double*>(smem_raw);   // packed lower triangle of L~_ii
  double* Bc = Lp + npk;                              // [ni][cw] chunk of right-hand sides
  double* colk = Bc + ni * cw;                        // [ni] column k of the factor
  // tables live past both the factor region and the Gauss-Jordan region
  const int reg0 = max(npk + ni * cw + ni, 2 * nb * 2 * nb);
  double* sD = Lp + reg0;                             // [n1*n1] physical D
  double* sK = sD + n1 * n1;                          // [n1*n1] reference K (h-invariant)
  double* sw = sK + n1 * n1;                          // [n1] reference weights
  double* sc = sw + n1;                               // [n1*n1] c of this element
  const int tid = threadIdx.x, nth = blockDim.x;
  double* A = p.Ascr + (long long)blockIdx.x * nb * nb;

  for (int l = tid; l < n1 * n1; l += nth) sK[l] = p.Kh[l];
  for (int l = tid; l < n1; l += nth) sw[l] = p.wh[l];

  const int nel = p.count_dev ? *p.count_dev : (p.elems || p.ed) ? p.count : p.E;
  for (int ei = blockIdx.x; ei < nel; ei += gridDim.x) {
    const int e = p.elems ? p.elems[ei] : ei;
    const double h = p.ed ? p.ed[ei].h : p.h;
    const double eta = p.ed ? p.ed[ei].eta : p.eta;
    const double* ce = p.ed ? p.ed[ei].c : p.c + (long long)e * n1 * n1;
    double2* To = p.ed ? p.ed[ei].T : p.T + (long long)e * nb * nb;
    const double h2 = 0.25 * h * h;  // (h/2)^2
    const double dsc = 2.0 / h;
    __syncthreads();
    for (int l = tid; l < n1 * n1; l += nth) {
      sc[l] = ce[l];
      sD[l] = dsc * p.Dh[l];
    }
    __syncthreads();
    // ---- assemble L~_ii: interior node I = (i-1) q + (j-1), i, j in 1..q ----
    // L~[(i,j),(i',j')] = K^[i,i'] w^_j d_jj' + w^_i K^[j,j'] d_ii' - c_ij (h/2)^2 w^_i w^_j d_IJ
    for (int l = tid; l < npk; l += nth) {
      // invert pk: row r with r(r+1)/2 <= l
      int r = (int)((sqrt(8.0 * l + 1.0) - 1.0) * 0.5);
      while (r * (r + 1) / 2 > l) --r;
      while ((r + 1) * (r + 2) / 2 <= l) ++r;
      const int cc = l - r * (r + 1) / 2;
      const int i = r / q + 1, j = r % q + 1, i2 = cc / q + 1, j2 = cc % q + 1;
      double v = 0.0;
      if (j == j2) v += sK[i * n1 + i2] * sw[j];
      if (i == i2) v += sw[i] * sK[j * n1 + j2];
      if (r == cc) v -= sc[i * n1 + j] * h2 * sw[i] * sw[j];
      Lp[l] = v;
    }
    __syncthreads();
    // ---- right-looking L D L^T (unit lower U, diagonal d), column scaling deferred one step ----
    double prev_inv = 0.0;
    for (int k = 0; k < ni; ++k) {
      for (int i = k + tid; i < ni; i += nth) colk[i] = Lp[pk(i, k)];
      __syncthreads();
      double dk = colk[k];
      if (!(dk > 0.0)) {
        if (tid == 0) atomicCAS(p.flag, 0, ei + 1);
        dk = 1.0;
      }
      const double inv = 1.0 / dk;
      if (k > 0)
        for (int i = k + tid; i < ni; i += nth) Lp[pk(i, k - 1)] *= prev_inv;  // U(i, k-1), diagonal keeps d
      const int warp = tid / 32, lane = tid % 32, nw = nth / 32;
      for (int i = k + 1 + warp; i < ni; i += nw) {
        const double f = colk[i] * inv;
        double* row = Lp + pk(i, 0);
        for (int j = k + 1 + lane; j <= i; j += 32) row[j] -= f * colk[j];
      }
      prev_inv = inv;
      __syncthreads();
    }

    // ---- Z = L~_ii^{-1} L~_iG by chunks of cw columns, A = Dn_GG - Dn_Gi Z ----
    for (int g0 = 0; g0 < nb; g0 += cw) {
      const int w = nb - g0 < cw ? nb - g0 : cw;
      for (int l = tid; l < ni * cw; l += nth) Bc[l] = 0.0;
      __syncthreads();
      // L~_iG columns: l(j'): K^[i,0] w^_j' at (i,j'); r(j'): K^[i,N] w^_j';
      //                b(i'): w^_i' K^[j,0] at (i',j);  t(i'): w^_i' K^[j,N]
      for (int l = tid; l < w * q; l += nth) {
        const int cc = l / q, t = l % q + 1;  // t runs along the interior line
        const int g = g0 + cc, side = g / q, s = g % q + 1;
        int I;
        double v;
        if (side == 0) { I = (t - 1) * q + (s - 1); v = sK[t * n1 + 0] * sw[s]; }
        else if (side == 1) { I = (t - 1) * q + (s - 1); v = sK[t * n1 + N] * sw[s]; }
        else if (side == 2) { I = (s - 1) * q + (t - 1); v = sw[s] * sK[t * n1 + 0]; }
        else { I = (s - 1) * q + (t - 1); v = sw[s] * sK[t * n1 + N]; }
        Bc[I * cw + cc] = v;
      }
      __syncthreads();
      // forward: U y = b (unit lower), one FMA per update
      for (int k = 0; k < ni - 1; ++k) {
        const int cnt = (ni - k - 1) * w;
        for (int l = tid; l < cnt; l += nth) {
          const int i = k + 1 + l / w, cc = l % w;
          Bc[i * cw + cc] -= Lp[pk(i, k)] * Bc[k * cw + cc];
        }
        __syncthreads();
      }
      // diagonal: z = D^{-1} y
      for (int l = tid; l < ni * w; l += nth) {
        const int i = l / w, cc = l % w;
        Bc[i * cw + cc] /= Lp[pk(i, i)];
      }
      __syncthreads();
      // backward: U^T x = z
      for (int k = ni - 1; k > 0; --k) {
        const double* row = Lp + pk(k, 0);
        const int cnt = k * w;
        for (int l = tid; l < cnt; l += nth) {
          const int i = l / w, cc = l % w;
          Bc[i * cw + cc] -= row[i] * Bc[k * cw + cc];
        }
        __syncthreads();
      }
      // A(:, chunk): Dn rows l(j): -D[0,i'] on (i',j); r(j): D[N,i']; b(i): -D[0,j'] on (i,j'); t(i): D[N,j']
      for (int l = tid; l < nb * w; l += nth) {
        const int g = l / w, cc = l % w, gc = g0 + cc;
        const int side = g / q, s = g % q + 1;
        double acc = 0.0;
        for (int t = 1; t <= q; ++t) {
          int I;
          double dcoef;
          if (side == 0) { I = (t - 1) * q + (s - 1); dcoef = -sD[0 * n1 + t]; }
          else if (side == 1) { I = (t - 1) * q + (s - 1); dcoef = sD[N * n1 + t]; }
          else if (side == 2) { I = (s - 1) * q + (t - 1); dcoef = -sD[0 * n1 + t]; }
          else { I = (s - 1) * q + (t - 1); dcoef = sD[N * n1 + t]; }
          acc += dcoef * Bc[I * cw + cc];
        }
        // Dn_GG: same-position node and the opposite side's node on the same line
        const int sidec = gc / q, sc2 = gc % q + 1;
        double dgg = 0.0;
        if (sc2 == s) {
          const bool xside = side < 2, xsidec = sidec < 2;
          if (xside == xsidec) {
            const int rowN = (side == 0 || side == 2) ? 0 : N;     // which D row
            const int colN = (sidec == 0 || sidec == 2) ? 0 : N;   // which node column
            const double sg = (side == 0 || side == 2) ? -1.0 : 1.0;
            dgg = sg * sD[rowN * n1 + colN];
          }
        }
        A[g * nb + gc] = dgg - acc;
      }
      __syncthreads();
    }

    // ---- P = A + i eta I, Gauss-Jordan [P | I] -> P^{-1}, T = I - 2 i eta P^{-1} ----
    double2* W = reinterpret_cast<double2*>(smem_raw);  // reuses the factor's space
    const int ld = 2 * nb;
    for (int l = tid; l < nb * ld; l += nth) {
      const int g = l / ld, j = l % ld;
      double2 v = make_double2(0.0, 0.0);
      if (j < nb) {
        v.x = A[g * nb + j];
        if (j == g) v.y = eta;
      } else if (j - nb == g) {
        v.x = 1.0;
      }
      W[l] = v;
    }
    __syncthreads();
    gj_smem<double>(W, nb, ld, ld, nullptr);
    for (int l = tid; l < nb * nb; l += nth) {
      const int g = l / nb, j = l % nb;
      const double2 y = W[g * ld + nb + j];
      To[l] = make_double2((g == j ? 1.0 : 0.0) + 2.0 * eta * y.y, -2.0 * eta * y.x);
    }
  }
}

// ---------------------------------------------------------------------------
// The same maps with the interior solve in FP32 plus FP64 iterative refinement.
//
// On the Cholesky route L~_ii is symmetric positive definite and well
// conditioned (GLL weak form: condition number about 150-200 at N = 16 for the
// coefficients the host admits), so an FP32 L D L^T factor is a good
// approximate inverse: with Z_0 = 0 and
//     R_k = L~_iG - L~_ii Z_k   (FP64),   Z_{k+1} = Z_k + (L D L^T)^{-1} R_k   (FP32 solve)
// every step gains about -log10(cond * eps_32) = 5 digits, and Z converges to
// the FP64 solution (classical mixed-precision iterative refinement).  The
// residual costs only 2 q^3 + q^2 FP64 FMAs per column because L~_ii is a sum
// of Kronecker products plus a diagonal:
//     (L~ Z)_(i,j) = w_j sum_i' K[i,i'] Z_(i',j) + w_i sum_j' K[j,j'] Z_(i,j') - c_ij (h/2)^2 w_i w_j Z_(i,j),
// against ni^2 for a dense FP64 solve.  The FP32 factor lives packed in shared
// memory (half the FP64 size) and the 4q right-hand sides are solved together
// by row blocks: a block-wide GEMM update from the solved rows, then a short
// triangle per column in registers.  The FP64 iterate Z stays in a per-CTA
// global workspace.  The refinement stops once the predicted next correction is
// below 1e-14 of Z (ratio of the last two corrections); the element is flagged
// if that takes more than IR_MAX steps.  A, P = A + i eta I and the FP64
// Gauss-Jordan inverse are as in leaf_kernel.
// ---------------------------------------------------------------------------
constexpr int IR_MAX = 10;
constexpr int TB = 16;     // row block of the triangular solves
constexpr int TBL = TB + 1;  // row stride of a stored diagonal-block inverse (staggered banks)
constexpr int PB = 16;     // panel width of the FP32 L D L^T
constexpr int IR_NT = 512;  // threads per CTA

__host__ __device__ inline int ir_ldy(int nb) { return (nb + 3) / 4 * 4 + 4; }  // 16-byte rows, staggered banks
__host__ __device__ inline int ir_npk_pad(int ni) { return (ni * (ni + 1) / 2 + 3) / 4 * 4; }

// block-wide max of a non-negative value (all threads get the result)
__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = fmax(r, red[w]);
  return r;
}

// Block-wide pivot search over rows [lo, hi) of column col (largest |re| + |im|, ties to
// the lower row); scratch: 2 * (blockDim / 32) doubles.  Two barriers; every thread gets
// the row.  The caller separates consecutive calls by a barrier.
__device__ int ir_argmax_col(const double2* W, int ld, int col, int lo, int hi, double* scratch) {
  double best = -1.0;
  int bi = -1;
  for (int r = lo + (int)threadIdx.x; r < hi; r += (int)blockDim.x) {
    const double2 w = W[r * ld + col];
    const double v = fabs(w.x) + fabs(w.y);
    if (v > best) {
      best = v;
      bi = r;
    }
  }
  warp_argmax(best, bi);
  const int nw = (int)(blockDim.x / 32), w = threadIdx.x / 32, lane = threadIdx.x % 32;
  int* si = reinterpret_cast<int*>(scratch + nw);
  if (lane == 0) {
    scratch[w] = best;
    si[w] = bi;
  }
  __syncthreads();
  double b2 = lane < nw ? scratch[lane] : -1.0;
  int i2 = lane < nw ? si[lane] : -1;
  warp_argmax(b2, i2);  // every warp reduces the per-warp winners itself
  i2 = __shfl_sync(0xffffffffu, i2, 0);
  __syncthreads();
  return i2 >= 0 ? i2 : lo;
}

__global__ void __launch_bounds__(IR_NT, 1) leaf_ir_kernel(LeafParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1;
  const int ldy = ir_ldy(nb);
  float* Lp = reinterpret_cast<float*>(smem_raw);     // packed FP32 factor: unit lower U, d on the diagonal
  float* Y = Lp + ir_npk_pad(ni);                      // [ni][ldy] right-hand sides / corrections, FP32
  const size_t reg0 = max((size_t)ir_npk_pad(ni) * 4 + (size_t)ni * ldy * 4, (size_t)nb * 2 * nb * 16);
  double* sD = reinterpret_cast<double*>(smem_raw + (reg0 + 15) / 16 * 16);  // [n1*n1] physical D
  double* sK = sD + n1 * n1;                           // [n1*n1] reference K
  double* sw = sK + n1 * n1;                           // [n1] reference weights
  double* sc = sw + n1;                                // [n1*n1] c of this element
  double* red = sc + n1 * n1;                          // [2 * IR_NT / 32] reductions
  float2* sKd = reinterpret_cast<float2*>(red + 2 * (IR_NT / 32));  // [n1*n1] K in double-float
  float2* swd = sKd + n1 * n1;                         // [n1] weights in double-float
  float2* cwd = swd + n1;                              // [n1*n1] c h^2/4 w_i w_j of this element, double-float
  float2* sDe = cwd + n1 * n1;                         // [2][n1] rows 0 and N of D in double-float
  float* Binv = reinterpret_cast<float*>(sDe + 2 * n1);  // [ceil(ni/TB)][TB][TBL] inverses of U's diagonal blocks
  const int tid = threadIdx.x, nth = blockDim.x;
  double* A = p.Ascr + (long long)blockIdx.x * nb * nb;
  // the refinement's iterate Z in double-float (the FP64 scratch holds the pairs)
  float2* Zd = reinterpret_cast<float2*>(p.Zscr + (long long)blockIdx.x * 2 * ni * nb);
  float2* S1 = Zd + (long long)ni * nb;  // [ni][nb] first Kronecker sum of the residual, double-float
  auto to_df = [](double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  };

  for (int l = tid; l < n1 * n1; l += nth) {
    sK[l] = p.Kh[l];
    sKd[l] = to_df(p.Kh[l]);
  }
  for (int l = tid; l < n1; l += nth) {
    sw[l] = p.wh[l];
    swd[l] = to_df(p.wh[l]);
  }

  const int nel = p.count_dev ? *p.count_dev : (p.elems || p.ed) ? p.count : p.E;
  for (int ei = blockIdx.x; ei < nel; ei += gridDim.x) {
    const int e = p.elems ? p.elems[ei] : ei;
    const double h = p.ed ? p.ed[ei].h : p.h;
    const double eta = p.ed ? p.ed[ei].eta : p.eta;
    const double* ce = p.ed ? p.ed[ei].c : p.c + (long long)e * n1 * n1;
    double2* To = p.ed ? p.ed[ei].T : p.T + (long long)e * nb * nb;
    const double h2 = 0.25 * h * h;
    const double dsc = 2.0 / h;
    __syncthreads();
    for (int l = tid; l < n1 * n1; l += nth) {
      sc[l] = ce[l];
      sD[l] = dsc * p.Dh[l];
      const int i = l / n1, j = l % n1;
      cwd[l] = to_df(ce[l] * h2 * p.wh[i] * p.wh[j]);
      if (i == 0) sDe[j] = to_df(dsc * p.Dh[l]);
      if (i == N) sDe[n1 + j] = to_df(dsc * p.Dh[l]);
    }
    __syncthreads();
    // ---- assemble L~_ii (FP32, packed lower triangle), one warp per row ----
    {
      const int warp = tid / 32, lane = tid % 32, nw = nth / 32;
      for (int r = warp; r < ni; r += nw) {
        const int i = r / q + 1, j = r % q + 1;
        float* row = Lp + pk(r, 0);
        for (int cc = lane; cc <= r; cc += 32) {
          const int i2 = cc / q + 1, j2 = cc % q + 1;
          // FP32 (leading parts): the factor only preconditions the refinement, whose
          // residual uses the double-float operator
          float v = 0.f;
          if (j == j2) v += sKd[i * n1 + i2].x * swd[j].x;
          if (i == i2) v += swd[i].x * sKd[j * n1 + j2].x;
          if (r == cc) v -= cwd[i * n1 + j].x;
          row[cc] = v;
        }
      }
    }
    __syncthreads();
    // ---- FP32 blocked right-looking L D L^T: panels of PB columns are factored column by
    //      column, then the trailing matrix takes one rank-PB update, register-tiled 4 x 4
    //      from k-major copies of the panel (scaled L and L D) ----
    {
      const int mpad = (ni + 3) / 4 * 4;
      float* Ps = Y;                 // [PB][mpad] panel rows below it: L (unit lower, scaled)
      float* Pd = Ps + PB * mpad;    // [PB][mpad] the same times d
      float* colk = Pd + PB * mpad;  // [ni]
      for (int p0 = 0; p0 < ni; p0 += PB) {
        const int pe = min(p0 + PB, ni);
        for (int l = tid; l < 2 * PB * mpad; l += nth) Ps[l] = 0.f;  // padding rows and columns stay 0
        for (int k = p0; k < pe; ++k) {
          for (int i = k + tid; i < ni; i += nth) colk[i] = Lp[pk(i, k)];
          __syncthreads();
          float dk = colk[k];
          if (!(dk > 0.f)) {
            if (tid == 0) atomicCAS(p.flag, 0, ei + 1);
            dk = 1.f;
          }
          const float inv = 1.f / dk;
          for (int i = k + 1 + tid; i < ni; i += nth) {
            float* row = Lp + pk(i, 0);
            const float f = colk[i] * inv;
            const int je = min(i, pe - 1);
            for (int j = k + 1; j <= je; ++j) row[j] -= f * colk[j];
            row[k] = f;  // U(i, k)
            if (i >= pe) {
              Ps[(k - p0) * mpad + (i - pe)] = f;
              Pd[(k - p0) * mpad + (i - pe)] = colk[i];
            }
          }
          __syncthreads();
        }
        const int m = ni - pe;
        if (m <= 0) continue;
        const int nt = (m + 3) / 4, ntiles = nt * (nt + 1) / 2;
        for (int tt = tid; tt < ntiles; tt += nth) {
          int ti = (int)((sqrtf(8.f * tt + 1.f) - 1.f) * 0.5f);
          while (ti * (ti + 1) / 2 > tt) --ti;
          while ((ti + 1) * (ti + 2) / 2 <= tt) ++ti;
          const int tj = tt - ti * (ti + 1) / 2;
          float acc[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 4
          for (int kk = 0; kk < PB; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(Ps + kk * mpad + 4 * ti);
            const float4 b4 = *reinterpret_cast<const float4*>(Pd + kk * mpad + 4 * tj);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = pe + 4 * ti + u;
            if (i >= ni) continue;
            float* row = Lp + pk(i, 0);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int j = pe + 4 * tj + v;
              if (j <= i) row[j] -= acc[u][v];
            }
          }
        }
        __syncthreads();
      }
    }
    // ---- inverses of U's TB x TB diagonal blocks (unit lower): thread (block, column c)
    //      solves U_bb x = e_c by forward substitution; zero outside the block's rows ----
    for (int l = tid; l < (ni + TB - 1) / TB * TB; l += nth) {
      const int b = l / TB, c = l % TB, r0 = b * TB, nr = min(TB, ni - r0);
      float x[TB];
#pragma unroll
      for (int t = 0; t < TB; ++t) {
        float v = t == c ? 1.f : 0.f;
        if (t > c && t < nr) {
          const float* Ut = Lp + pk(r0 + t, r0);
#pragma unroll
          for (int u = 0; u < t; ++u)
            if (u >= c) v -= Ut[u] * x[u];
        }
        x[t] = v;
      }
      float* Bi = Binv + b * TB * TBL;
#pragma unroll
      for (int t = 0; t < TB; ++t) Bi[t * TBL + c] = (t < nr && c < nr) ? x[t] : 0.f;
    }
    __syncthreads();
    // ---- refinement: Z <- Z + (L D L^T)^{-1} (L~_iG - L~_ii Z) ----
    double rel_prev = 1.0;
    bool done = false;
    for (int it = 0; it < IR_MAX && !done; ++it) {
      // residual in double-float (error-free products, TwoSum accumulation: about 48 bits on the
      // FP32 pipes), rounded into Y:
      //   r(i,j,g) = K_b w_s - w_j sum_t K[i][t] Z(t,j,g) - w_i sum_t K[j][t] Z(i,t,g) + c_ij Z(i,j,g).
      // The first sum runs over one column (j, g) of Z, the second over one row (i, g): a thread
      // keeps that line of Z in registers and forms all q sums from it; the first sums go
      // through global scratch (S1) to the thread of the matching row.
      constexpr int QMAX = 15;  // q <= 15 (N <= 16)
      if (it > 0) {
        for (int l = tid; l < q * nb; l += nth) {
          const int j = l / nb + 1, g = l % nb;
          float2 zc[QMAX];
#pragma unroll
          for (int t = 0; t < QMAX; ++t)
            if (t < q) zc[t] = Zd[(long long)(t * q + (j - 1)) * nb + g];
          for (int i = 1; i <= q; ++i) {
            float ss = 0.f, sc2 = 0.f;
#pragma unroll
            for (int t = 0; t < QMAX; ++t)
              if (t < q) {
                const float2 ka = sKd[i * n1 + t + 1];
                dfops::dot2(ss, sc2, ka.x, ka.y, zc[t].x, zc[t].y);
              }
            float2 o;
            dfops::fast2(ss, sc2, o.x, o.y);
            S1[(long long)((i - 1) * q + (j - 1)) * nb + g] = o;
          }
        }
        __syncthreads();
      }
      for (int l = tid; l < q * nb; l += nth) {
        const int i = l / nb + 1, g = l % nb;
        const int side = g / q, s = g % q + 1;
        float2 zr[QMAX];
        if (it > 0) {
#pragma unroll
          for (int t = 0; t < QMAX; ++t)
            if (t < q) zr[t] = Zd[(long long)((i - 1) * q + t) * nb + g];
        }
        for (int j = 1; j <= q; ++j) {
          const int I = (i - 1) * q + (j - 1);
          float rs = 0.f, rc = 0.f;  // boundary coupling K_b w_s, then minus L~_ii Z
          {
            float2 kb = make_float2(0.f, 0.f);
            if (side == 0 && j == s) kb = sKd[i * n1 + 0];
            else if (side == 1 && j == s) kb = sKd[i * n1 + N];
            else if (side == 2 && i == s) kb = sKd[j * n1 + 0];
            else if (side == 3 && i == s) kb = sKd[j * n1 + N];
            const float2 ws = swd[s];
            dfops::dot2(rs, rc, kb.x, kb.y, ws.x, ws.y);
          }
          if (it > 0) {
            float s2s = 0.f, s2c = 0.f;
            float2 zij = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < QMAX; ++t)
              if (t < q) {
                const float2 kb = sKd[j * n1 + t + 1];
                dfops::dot2(s2s, s2c, kb.x, kb.y, zr[t].x, zr[t].y);
                if (t == j - 1) zij = zr[t];
              }
            float s2h, s2l;
            dfops::fast2(s2s, s2c, s2h, s2l);
            const float2 s1 = S1[(long long)I * nb + g];
            const float2 wj = swd[j], wi = swd[i], cw = cwd[i * n1 + j];
            dfops::dot2(rs, rc, -wj.x, -wj.y, s1.x, s1.y);
            dfops::dot2(rs, rc, -wi.x, -wi.y, s2h, s2l);
            dfops::dot2(rs, rc, cw.x, cw.y, zij.x, zij.y);
          }
          Y[I * ldy + g] = __fadd_rn(rs, rc);
        }
      }
      __syncthreads();
      // forward U y = r, diagonal, backward U^T x = z, by row blocks of TB: the rows above
      // (below) a block enter through one block-wide GEMM update (thread: one row x four
      // columns), then one lane per column finishes the TB x TB triangle in registers
      {
        const int gr = tid / 16, gq = tid % 16;  // GEMM-update row and column quad
        const bool gact = 4 * gq < nb;
        for (int r0 = 0; r0 < ni; r0 += TB) {
          const int nr = min(TB, ni - r0);
          if (r0 > 0 && gact && gr < nr) {
            const float* Ur = Lp + pk(r0 + gr, 0);
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int k = 0; k < r0; ++k) {
              const float u = Ur[k];
              const float4 y = *reinterpret_cast<const float4*>(Y + k * ldy + 4 * gq);
              acc.x += u * y.x; acc.y += u * y.y; acc.z += u * y.z; acc.w += u * y.w;
            }
            float4* yo = reinterpret_cast<float4*>(Y + (r0 + gr) * ldy + 4 * gq);
            float4 v = *yo;
            v.x -= acc.x; v.y -= acc.y; v.z -= acc.z; v.w -= acc.w;
            *yo = v;
          }
          __syncthreads();
          {
            // the block's triangle through its stored inverse: warp w takes columns 4w .. 4w + 3,
            // eight lanes per column, lane rows t0 and t0 + 8 (the column is read by its eight
            // lanes before any of them writes: the warp is synchronised in between)
            const int col = 4 * (tid / 32) + (tid % 32) / 8, t0 = tid % 8;
            const bool cv = col < nb;
            const float* Bi = Binv + (r0 / TB) * TB * TBL;
            float yv[TB];
#pragma unroll
            for (int u = 0; u < TB; ++u) yv[u] = (cv && u < nr) ? Y[(r0 + u) * ldy + col] : 0.f;
            float o0 = 0.f, o1 = 0.f;
#pragma unroll
            for (int u = 0; u < TB; ++u) {
              if (u <= t0) o0 = fmaf(Bi[t0 * TBL + u], yv[u], o0);
              if (u <= t0 + 8) o1 = fmaf(Bi[(t0 + 8) * TBL + u], yv[u], o1);
            }
            __syncwarp();
            if (cv && t0 < nr) Y[(r0 + t0) * ldy + col] = o0;
            if (cv && t0 + 8 < nr) Y[(r0 + t0 + 8) * ldy + col] = o1;
          }
          __syncthreads();
        }
        for (int l = tid; l < ni * nb; l += nth) {  // z = D^{-1} y
          const int I = l / nb;
          Y[I * ldy + l % nb] /= Lp[pk(I, I)];
        }
        __syncthreads();
        // the same row blocks as the forward pass (their inverses are stored), last first
        for (int bb = (ni + TB - 1) / TB - 1; bb >= 0; --bb) {
          const int r0 = bb * TB, nr = min(TB, ni - r0), r1 = r0 + nr;
          if (r1 < ni && gact && gr < nr) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int k = r1; k < ni; ++k) {
              const float u = Lp[pk(k, r0 + gr)];
              const float4 x = *reinterpret_cast<const float4*>(Y + k * ldy + 4 * gq);
              acc.x += u * x.x; acc.y += u * x.y; acc.z += u * x.z; acc.w += u * x.w;
            }
            float4* xo = reinterpret_cast<float4*>(Y + (r0 + gr) * ldy + 4 * gq);
            float4 v = *xo;
            v.x -= acc.x; v.y -= acc.y; v.z -= acc.z; v.w -= acc.w;
            *xo = v;
          }
          __syncthreads();
          {
            // U_bb^T x = y through the transposed inverse, laid out as in the forward pass
            const int col = 4 * (tid / 32) + (tid % 32) / 8, t0 = tid % 8;
            const bool cv = col < nb;
            const float* Bi = Binv + (r0 / TB) * TB * TBL;
            float xv[TB];
#pragma unroll
            for (int u = 0; u < TB; ++u) xv[u] = (cv && u < nr) ? Y[(r0 + u) * ldy + col] : 0.f;
            float o0 = 0.f, o1 = 0.f;
#pragma unroll
            for (int u = 0; u < TB; ++u) {
              if (u >= t0) o0 = fmaf(Bi[u * TBL + t0], xv[u], o0);
              if (u >= t0 + 8) o1 = fmaf(Bi[u * TBL + t0 + 8], xv[u], o1);
            }
            __syncwarp();
            if (cv && t0 < nr) Y[(r0 + t0) * ldy + col] = o0;
            if (cv && t0 + 8 < nr) Y[(r0 + t0 + 8) * ldy + col] = o1;
          }
          __syncthreads();
        }
      }
      __syncthreads();
      // Z += correction (double-float), sizes for the stopping test
      float mdf = 0.f, mzf = 0.f;
      for (int l = tid; l < ni * nb; l += nth) {
        const int I = l / nb, g = l % nb;
        const float d = Y[I * ldy + g];
        const float2 z = it == 0 ? make_float2(0.f, 0.f) : Zd[l];
        float t, e;
        dfops::two_sum(z.x, d, t, e);
        float2 zn;
        dfops::fast2(t, __fadd_rn(z.y, e), zn.x, zn.y);
        Zd[l] = zn;
        mdf = fmaxf(mdf, fabsf(d));
        mzf = fmaxf(mzf, fabsf(zn.x));
      }
      const double md = block_max((double)mdf, red);
      const double mz = block_max((double)mzf, red);
      const double rel = mz > 0.0 ? md / mz : 0.0;
      if (it > 0) {
        // converged when the predicted next correction is below 1e-14 of Z, or when the
        // corrections have stopped contracting at the double-float residual's floor
        // (about cond(L~_ii) 2^-48: elements near the positive-definite bound reach it first)
        const double rho = fmax(rel / rel_prev, 1e-6);
        done = rel * rho <= 1e-14 || (it >= 2 && rho >= 0.25 && rel <= 1e-10);
      }
      if (!(rel == rel)) done = false;
      rel_prev = rel > 0.0 ? rel : 1e-300;
      if (rel == 0.0) done = true;
      if (!done && it == IR_MAX - 1 && tid == 0) atomicCAS(p.flag, 0, ei + 1);
      __syncthreads();
    }

    // ---- A = Dn_GG - Dn_Gi Z (products accumulated in double-float, A in FP64) ----
    for (int l = tid; l < nb * nb; l += nth) {
      const int g = l / nb, gc = l % nb;
      const int side = g / q, s = g % q + 1;
      float as = 0.f, ac = 0.f;
      for (int t = 1; t <= q; ++t) {
        int I;
        float2 dcoef;
        if (side == 0) { I = (t - 1) * q + (s - 1); dcoef = sDe[t]; dcoef.x = -dcoef.x; dcoef.y = -dcoef.y; }
        else if (side == 1) { I = (t - 1) * q + (s - 1); dcoef = sDe[n1 + t]; }
        else if (side == 2) { I = (s - 1) * q + (t - 1); dcoef = sDe[t]; dcoef.x = -dcoef.x; dcoef.y = -dcoef.y; }
        else { I = (s - 1) * q + (t - 1); dcoef = sDe[n1 + t]; }
        const float2 z = Zd[(long long)I * nb + gc];
        dfops::dot2(as, ac, dcoef.x, dcoef.y, z.x, z.y);
      }
      const double acc = (double)as + (double)ac;
      const int sidec = gc / q, sc2 = gc % q + 1;
      double dgg = 0.0;
      if (sc2 == s) {
        const bool xside = side < 2, xsidec = sidec < 2;
        if (xside == xsidec) {
          const int rowN = (side == 0 || side == 2) ? 0 : N;
          const int colN = (sidec == 0 || sidec == 2) ? 0 : N;
          const double sg = (side == 0 || side == 2) ? -1.0 : 1.0;
          dgg = sg * sD[rowN * n1 + colN];
        }
      }
      A[g * nb + gc] = dgg - acc;
    }
    __syncthreads();
    // ---- P = A + i eta I, in-place Gauss-Jordan with partial pivoting -> P^{-1} in double-float
    //      (pairs of FP32, about 48 bits, on the FP32 pipes), T = I - 2 i eta P^{-1} ----
    {
      float4* W = reinterpret_cast<float4*>(smem_raw);  // [nb][nb] complex df64, reuses the factor's space
      float4* colk = W + nb * nb;                        // [nb] column k after the interchange
      float4* rowk = colk + nb;                          // [nb] scaled pivot row
      float4* rowo = rowk + nb;                          // [nb] row k before the interchange (becomes row pv)
      float4* coln = rowo + nb;                          // [nb] column k as left by step k - 1 (contiguous)
      float* cval = reinterpret_cast<float*>(coln + nb);  // [IR_NT / 64] pivot candidates of the next column
      int* crow = reinterpret_cast<int*>(cval + IR_NT / 64);
      int* perm = crow + IR_NT / 64;                     // [nb] pivot rows, then the column order
      const int jc = tid % 64, rg = tid / 64, nrg = nth / 64;  // column and row group of this thread
      for (int l = tid; l < nb * nb; l += nth) {
        const int g = l / nb, j = l % nb;
        W[l] = dfops::from_d2(make_double2(A[l], g == j ? eta : 0.0));
      }
      __syncthreads();
      // the pivot of column k is searched while column k is updated at step k - 1: the
      // thread of column k in each row group keeps its largest |re| + |im| (leading parts)
      if (jc == 0) {
        float best = -1.f;
        int bi = -1;
        for (int i = rg; i < nb; i += nrg) {
          const float4 w = W[i * nb];
          coln[i] = w;
          const float v = fabsf(w.x) + fabsf(w.y);
          if (v > best) { best = v; bi = i; }
        }
        cval[rg] = best;
        crow[rg] = bi;
      }
      __syncthreads();
      for (int k = 0; k < nb; ++k) {
        int pv = -1;
        float pb = -1.f;
        for (int c = 0; c < nrg; ++c) {  // largest candidate, ties to the lower row
          const float v = cval[c];
          const int r = crow[c];
          if (r >= 0 && (v > pb || (v == pb && r < pv))) { pb = v; pv = r; }
        }
        if (pv < 0) pv = k;
        // interchange rows k and pv logically: pivot row, column k and the old row k are staged
        if (tid < nb) {
          const int j = tid;
          const float4 piv = coln[pv];
          const float4 inv = dfops::cinv(piv);
          rowo[j] = W[k * nb + j];
          rowk[j] = j == k ? inv : dfops::cmul(W[pv * nb + j], inv);
          colk[j] = j == k ? piv : (j == pv ? coln[k] : coln[j]);
          if (j == 0) {
            if (piv.x == 0.f && piv.y == 0.f) atomicCAS(p.flag, 0, ei + 1);
            perm[k] = pv;
          }
        }
        __syncthreads();
        if (jc < nb) {
          const float4 rk = rowk[jc];
          const bool cand = jc == k + 1;
          float best = -1.f;
          int bi = -1;
#pragma unroll 2
          for (int i = rg; i < nb; i += nrg) {
            if (i == k) {
              W[i * nb + jc] = rk;
              if (cand) coln[i] = rk;
            } else {
              const float4 src = i == pv ? rowo[jc] : W[i * nb + jc];
              const float4 v = dfops::cfms(jc == k ? make_float4(0.f, 0.f, 0.f, 0.f) : src, colk[i], rk);
              W[i * nb + jc] = v;
              if (cand) {
                coln[i] = v;
                if (i > k) {
                  const float m = fabsf(v.x) + fabsf(v.y);
                  if (m > best) { best = m; bi = i; }
                }
              }
            }
          }
          if (cand) {
            cval[rg] = best;
            crow[rg] = bi;
          }
        }
        __syncthreads();
      }
      // the row interchanges, undone last first as column interchanges, compose to one column order
      if (tid == 0) {
        int* sig = perm + nb;  // [nb]
        for (int c = 0; c < nb; ++c) sig[c] = c;
        for (int k = nb - 1; k >= 0; --k) {
          const int pk2 = perm[k];
          const int t = sig[k];
          sig[k] = sig[pk2];
          sig[pk2] = t;
        }
      }
      __syncthreads();
      const int* sig = perm + nb;
      for (int l = tid; l < nb * nb; l += nth) {
        const int g = l / nb, j = l % nb;
        const double2 y = dfops::to_d2(W[g * nb + sig[j]]);
        To[l] = make_double2((g == j ? 1.0 : 0.0) + 2.0 * eta * y.y, -2.0 * eta * y.x);
      }
    }
  }
}

}  // namespace


// ---------------------------------------------------------------------------
// Robust route (any element the impedance problem is solvable on).  The edge
// rows I_i = Dn + i eta couple each node only to the opposite node of its line,
// so L_GG is block diagonal with one 2x2 block per line,
//     Mb = [[-D00 + i eta, -D0N], [DN0, DNN + i eta]]   (order: left/bottom, right/top),
// the same for every line and always invertible.  Eliminating the edge nodes
// first leaves the complex interior Schur complement
//     S_i = L~_ii - R Dn_Gi,   R = L~_iG L_GG^{-1},
// with Y_i = -S_i^{-1} R (pivoted Gauss-Jordan on [S_i | -R]) and
//     Y_G = L_GG^{-1} (I - Dn_Gi Y_i),  T = I - 2 i eta Y_G.
// ---------------------------------------------------------------------------
namespace {

struct Minv2 {
  double2 a, b, c, d;  // inverse of Mb, row-major
};

__device__ __forceinline__ Minv2 mb_inverse(const double* Dp, int N, double eta) {
  const int n1 = N + 1;
  const double2 m00 = make_double2(-Dp[0], eta), m01 = make_double2(-Dp[N], 0.0);
  const double2 m10 = make_double2(Dp[N * n1], 0.0), m11 = make_double2(Dp[N * n1 + N], eta);
  const double2 det = csub(cmul(m00, m11), cmul(m01, m10));
  const double2 id = cinv(det);
  Minv2 r;
  r.a = cmul(m11, id);
  r.b = cmul(make_double2(-m01.x, -m01.y), id);
  r.c = cmul(make_double2(-m10.x, -m10.y), id);
  r.d = cmul(m00, id);
  return r;
}

// Entry (I, col) of [S_i | -R] for an element with coefficient samples ce (col < ni: S_i, else -R).
__device__ __forceinline__ double2 robust_entry(const LeafParams& p, const double* sD, const Minv2& mi,
                                                const double* ce, int I, int col) {
  const int N = p.N, q = p.q, ni = p.ni, n1 = N + 1;
  const double h2 = 0.25 * p.h * p.h;
  const int ti = I / q + 1, tj = I % q + 1;
  // R entries of row I on its two lines (x-pair of line tj, y-pair of line ti)
  const double a0 = p.Kh[ti * n1 + 0] * p.wh[tj], aN = p.Kh[ti * n1 + N] * p.wh[tj];
  const double c0 = p.wh[ti] * p.Kh[tj * n1 + 0], cN = p.wh[ti] * p.Kh[tj * n1 + N];
  const double2 Rl = cadd(cscale(mi.a, a0), cscale(mi.c, aN)), Rr = cadd(cscale(mi.b, a0), cscale(mi.d, aN));
  const double2 Rb = cadd(cscale(mi.a, c0), cscale(mi.c, cN)), Rt = cadd(cscale(mi.b, c0), cscale(mi.d, cN));
  double2 v = make_double2(0.0, 0.0);
  if (col < ni) {
    const int ui = col / q + 1, uj = col % q + 1;
    double lt = 0.0;
    if (tj == uj) lt += p.Kh[ti * n1 + ui] * p.wh[tj];
    if (ti == ui) lt += p.wh[ti] * p.Kh[tj * n1 + uj];
    if (I == col) lt -= ce[ti * n1 + tj] * h2 * p.wh[ti] * p.wh[tj];
    v.x = lt;
    if (tj == uj) v = csub(v, cadd(cscale(Rl, -sD[0 * n1 + ui]), cscale(Rr, sD[N * n1 + ui])));
    if (ti == ui) v = csub(v, cadd(cscale(Rb, -sD[0 * n1 + uj]), cscale(Rt, sD[N * n1 + uj])));
  } else {
    const int g = col - ni, side = g / q, s = g % q + 1;
    // -R[I][g]
    if (side == 0 && s == tj) v = Rl;
    else if (side == 1 && s == tj) v = Rr;
    else if (side == 2 && s == ti) v = Rb;
    else if (side == 3 && s == ti) v = Rt;
    v = make_double2(-v.x, -v.y);
  }
  return v;
}

// W[b] = [S_i | -R | extra columns]: column ni + nb + r of row I is Bx[(e * nrhs + r) * ni + I]
// (the interior right-hand side of right-hand side r of element e), or 0 when Bx is null.
__global__ void robust_assemble_kernel(LeafParams p, const int* __restrict__ elems, int count, int extra,
                                       const double2* __restrict__ Bx, double2* __restrict__ W) {
  const int N = p.N, ni = p.ni, nb = p.nb, n1 = N + 1, ld = ni + nb + extra;
  const double dsc = 2.0 / p.h;
  __shared__ double sD[25 * 25];
  for (int l = threadIdx.x; l < n1 * n1; l += blockDim.x) sD[l] = dsc * p.Dh[l];
  __syncthreads();
  const Minv2 mi = mb_inverse(sD, N, p.eta);
  const long long tot = (long long)count * ni * ld;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(l / ((long long)ni * ld));
    const int rem = (int)(l % ((long long)ni * ld));
    const int I = rem / ld, col = rem % ld;
    const int e = elems[b];
    double2 v;
    if (col < ni + nb) {
      v = robust_entry(p, sD, mi, p.c + (long long)e * n1 * n1, I, col);
    } else {
      const int r = col - ni - nb;
      v = Bx ? Bx[((long long)e * extra + r) * ni + I] : make_double2(0.0, 0.0);
    }
    W[(long long)b * ni * ld + (long long)I * ld + col] = v;
  }
}

__global__ void robust_finish_kernel(LeafParams p, const int* __restrict__ elems, int count,
                                     const double2* __restrict__ W) {
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1, ld = ni + nb;
  const double dsc = 2.0 / p.h;
  __shared__ double sD[25 * 25];
  for (int l = threadIdx.x; l < n1 * n1; l += blockDim.x) sD[l] = dsc * p.Dh[l];
  __syncthreads();
  const Minv2 mi = mb_inverse(sD, N, p.eta);
  const long long tot = (long long)count * 2 * q * nb;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(l / (2LL * q * nb));
    const int rem = (int)(l % (2LL * q * nb));
    const int line = rem / nb, col = rem % nb;
    const double2* Y = W + (long long)b * ni * ld + ni;  // Y_i[J][col] at Y[J * ld + col]
    double2 z0, z1;  // Z on the line's first node (l or b) and second node (r or t)
    int g0, g1;
    if (line < q) {  // x-pair: l_j, r_j with j = line + 1; interior nodes (ui, j)
      const int j = line + 1;
      g0 = j - 1;
      g1 = q + j - 1;
      z0 = make_double2(g0 == col ? 1.0 : 0.0, 0.0);
      z1 = make_double2(g1 == col ? 1.0 : 0.0, 0.0);
      for (int ui = 1; ui <= q; ++ui) {
        const double2 y = Y[(long long)((ui - 1) * q + (j - 1)) * ld + col];
        z0 = cadd(z0, cscale(y, sD[0 * n1 + ui]));
        z1 = csub(z1, cscale(y, sD[N * n1 + ui]));
      }
    } else {  // y-pair: b_i, t_i with i = line - q + 1; interior nodes (i, uj)
      const int i = line - q + 1;
      g0 = 2 * q + i - 1;
      g1 = 3 * q + i - 1;
      z0 = make_double2(g0 == col ? 1.0 : 0.0, 0.0);
      z1 = make_double2(g1 == col ? 1.0 : 0.0, 0.0);
      for (int uj = 1; uj <= q; ++uj) {
        const double2 y = Y[(long long)((i - 1) * q + (uj - 1)) * ld + col];
        z0 = cadd(z0, cscale(y, sD[0 * n1 + uj]));
        z1 = csub(z1, cscale(y, sD[N * n1 + uj]));
      }
    }
    const double2 y0 = cadd(cmul(mi.a, z0), cmul(mi.b, z1));
    const double2 y1 = cadd(cmul(mi.c, z0), cmul(mi.d, z1));
    double2* To = p.T + (long long)elems[b] * nb * nb;
    // T = I - 2 i eta Y_G:  -2 i eta (x + i y) = 2 eta y - 2 i eta x
    To[(long long)g0 * nb + col] = make_double2((g0 == col ? 1.0 : 0.0) + 2.0 * p.eta * y0.y, -2.0 * p.eta * y0.x);
    To[(long long)g1 * nb + col] = make_double2((g1 == col ? 1.0 : 0.0) + 2.0 * p.eta * y1.y, -2.0 * p.eta * y1.x);
  }
}

// Element fields of the pivoted route after Gauss-Jordan on [S_i | -R | b~_0 .. b~_{nrhs-1}]
// (right part = [Y_i | S_i^{-1} b~_r]): u_i = Y_i f_r + S_i^{-1} b~_r for incoming data f_r
// (F[(e * nrhs + r) * nb + g], null = 0), then per edge line u_G = Mb^{-1} (f - Dn_Gi u_i).
__global__ void robust_field_interior_kernel(LeafParams p, const int* __restrict__ elems, int count, int nrhs,
                                             const double2* __restrict__ W, const double2* __restrict__ F,
                                             double2* __restrict__ Ui) {
  const int ni = p.ni, nb = p.nb, ld = ni + nb + nrhs;
  const long long tot = (long long)count * nrhs * ni;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(l / ((long long)nrhs * ni));
    const int rem = (int)(l % ((long long)nrhs * ni));
    const int r = rem / ni, I = rem % ni;
    const int e = elems[b];
    const double2* row = W + (long long)b * ni * ld + (long long)I * ld;
    double2 u = row[ni + nb + r];
    if (F) {
      const double2* f = F + ((long long)e * nrhs + r) * nb;
      for (int g = 0; g < nb; ++g) cfma(u, row[ni + g], f[g]);
    }
    Ui[((long long)e * nrhs + r) * ni + I] = u;
  }
}

// u_G on the edge nodes from u_i (Ui) and f (F, null = 0); written to UG[(e * nrhs + r) * nb + g], or,
// when H is given, the interior contribution H = I_o u = -2 i eta u_G (f = 0) to
// H[(e * nb + g) * nrhs + r].
__global__ void robust_field_edges_kernel(LeafParams p, const int* __restrict__ elems, int count, int nrhs,
                                          const double2* __restrict__ Ui, const double2* __restrict__ F,
                                          double2* __restrict__ UG, double2* __restrict__ H) {
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1;
  const double dsc = 2.0 / p.h;
  __shared__ double sD[25 * 25];
  for (int l = threadIdx.x; l < n1 * n1; l += blockDim.x) sD[l] = dsc * p.Dh[l];
  __syncthreads();
  const Minv2 mi = mb_inverse(sD, N, p.eta);
  const long long tot = (long long)count * nrhs * 2 * q;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(l / ((long long)nrhs * 2 * q));
    const int rem = (int)(l % ((long long)nrhs * 2 * q));
    const int r = rem / (2 * q), line = rem % (2 * q);
    const int e = elems[b];
    const double2* u = Ui + ((long long)e * nrhs + r) * ni;
    const double2* f = F ? F + ((long long)e * nrhs + r) * nb : nullptr;
    int g0, g1;
    double2 z0 = make_double2(0.0, 0.0), z1 = make_double2(0.0, 0.0);
    if (line < q) {  // x-pair l_j, r_j; interior nodes (ui, j)
      const int j = line + 1;
      g0 = j - 1;
      g1 = q + j - 1;
      for (int ui = 1; ui <= q; ++ui) {
        const double2 y = u[(ui - 1) * q + (j - 1)];
        z0 = cadd(z0, cscale(y, sD[0 * n1 + ui]));
        z1 = csub(z1, cscale(y, sD[N * n1 + ui]));
      }
    } else {  // y-pair b_i, t_i; interior nodes (i, uj)
      const int i = line - q + 1;
      g0 = 2 * q + i - 1;
      g1 = 3 * q + i - 1;
      for (int uj = 1; uj <= q; ++uj) {
        const double2 y = u[(i - 1) * q + (uj - 1)];
        z0 = cadd(z0, cscale(y, sD[0 * n1 + uj]));
        z1 = csub(z1, cscale(y, sD[N * n1 + uj]));
      }
    }
    if (f) {
      z0 = cadd(z0, f[g0]);
      z1 = cadd(z1, f[g1]);
    }
    const double2 y0 = cadd(cmul(mi.a, z0), cmul(mi.b, z1));
    const double2 y1 = cadd(cmul(mi.c, z0), cmul(mi.d, z1));
    if (H) {  // -2 i eta (x + i y) = 2 eta y - 2 i eta x
      H[((long long)e * nb + g0) * nrhs + r] = make_double2(2.0 * p.eta * y0.y, -2.0 * p.eta * y0.x);
      H[((long long)e * nb + g1) * nrhs + r] = make_double2(2.0 * p.eta * y1.y, -2.0 * p.eta * y1.x);
    } else {
      UG[((long long)e * nrhs + r) * nb + g0] = y0;
      UG[((long long)e * nrhs + r) * nb + g1] = y1;
    }
  }
}

}  // namespace

cudaError_t robust_field(const LeafParams& p, const int* elems, int count, int nrhs, const double2* W,
                         const double2* F, double2* Ui, double2* UG, double2* H, cudaStream_t s) {
  long long blocks = ((long long)count * nrhs * p.ni + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  if (blocks < 1) return cudaSuccess;
  robust_field_interior_kernel<<<(int)blocks, 256, 0, s>>>(p, elems, count, nrhs, W, F, Ui);
  note_launch();
  blocks = ((long long)count * nrhs * 2 * p.q + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  robust_field_edges_kernel<<<(int)blocks, 256, 0, s>>>(p, elems, count, nrhs, Ui, F, UG, H);
  note_launch();
  return cudaGetLastError();
}

cudaError_t robust_assemble(const LeafParams& p, const int* elems, int count, double2* W, cudaStream_t s,
                            int extra, const double2* Bx) {
  const long long tot = (long long)count * p.ni * (p.ni + p.nb + extra);
  long long blocks = (tot + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  robust_assemble_kernel<<<(int)blocks, 256, 0, s>>>(p, elems, count, extra, Bx, W);
  note_launch();
  return cudaGetLastError();
}

cudaError_t robust_finish(const LeafParams& p, const int* elems, int count, const double2* W, cudaStream_t s) {
  const long long tot = (long long)count * 2 * p.q * p.nb;
  long long blocks = (tot + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  robust_finish_kernel<<<(int)blocks, 256, 0, s>>>(p, elems, count, W);
  note_launch();
  return cudaGetLastError();
}

size_t leaf_smem_bytes(int N, int cw) {
  const int q = N - 1, ni = q * q, nb = 4 * q, n1 = N + 1;
  const size_t r1 = (size_t)ni * (ni + 1) / 2 + (size_t)ni * cw + ni;
  const size_t r2 = (size_t)2 * nb * 2 * nb;  // double2 [nb][2 nb] in doubles
  return sizeof(double) * ((r1 > r2 ? r1 : r2) + 3 * n1 * n1 + n1);
}

void optin_leaf() {
  smem_optin(leaf_ir_kernel);
  smem_optin(leaf_kernel);
}

size_t leaf_ir_smem_bytes(int N) {
  const int q = N - 1, ni = q * q, nb = 4 * q, n1 = N + 1;
  const size_t reg0 = std::max((size_t)ir_npk_pad(ni) * 4 + (size_t)ni * ir_ldy(nb) * 4, (size_t)nb * 2 * nb * 16);
  return (reg0 + 15) / 16 * 16 + sizeof(double) * (3 * n1 * n1 + n1 + 2 * (IR_NT / 32)) +
         sizeof(float2) * (2 * n1 * n1 + 3 * n1) + sizeof(float) * (size_t)((ni + TB - 1) / TB) * TB * TBL;
}

namespace {

// One warp per element: c at its nodes, the maximum of c and the finiteness of b by warp
// reductions.
__global__ void coeff_route_kernel(const double* __restrict__ b, double k2, int E, int nn, double bound,
                                   double* __restrict__ c, int* __restrict__ route, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < E; e += gridDim.x * wpb) {
    const double* be = b + (long long)e * nn;
    double* ceo = c + (long long)e * nn;
    double cm = -INFINITY;
    bool finite = true;
    for (int l = lane; l < nn; l += 32) {
      const double bv = be[l];
      finite = finite && isfinite(bv);
      const double cv = k2 * (1.0 - bv);
      ceo[l] = cv;
      cm = fmax(cm, cv);
    }
    for (int o = 16; o > 0; o >>= 1) cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    const bool all_finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      route[e] = cm < bound ? 0 : 1;
      if (!all_finite) atomicExch(err, 1);
    }
  }
}

// Single CTA of 1024 threads: chunk by chunk, ballots give each element's rank within its
// warp, a scan over the 32 warp totals its rank within the chunk.
__global__ void __launch_bounds__(1024) route_lists_kernel(const int* __restrict__ route, int E,
                                                           int* __restrict__ good, int* __restrict__ bad,
                                                           int* __restrict__ counts) {
  __shared__ int wg[32], wb[32], tot[2];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int base_g = 0, base_b = 0;
  for (int e0 = 0; e0 < E; e0 += 1024) {
    const int e = e0 + tid;
    const int r = e < E ? route[e] : -1;
    const unsigned bg = __ballot_sync(0xffffffffu, r == 0), bb = __ballot_sync(0xffffffffu, r == 1);
    if (lane == 0) {
      wg[w] = __popc(bg);
      wb[w] = __popc(bb);
    }
    __syncthreads();
    if (w == 0) {
      const int vg = wg[lane], vb = wb[lane];
      int ig = vg, ib = vb;
      for (int o = 1; o < 32; o <<= 1) {
        const int tg = __shfl_up_sync(0xffffffffu, ig, o), tb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
          ig += tg;
          ib += tb;
        }
      }
      wg[lane] = ig - vg;
      wb[lane] = ib - vb;
      if (lane == 31) {
        tot[0] = ig;
        tot[1] = ib;
      }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    if (r == 0) good[base_g + wg[w] + __popc(bg & below)] = e;
    if (r == 1) bad[base_b + wb[w] + __popc(bb & below)] = e;
    base_g += tot[0];
    base_b += tot[1];
    __syncthreads();
  }
  if (tid == 0) {
    counts[0] = base_g;
    counts[1] = base_b;
  }
}

}  // namespace

cudaError_t coeff_route(const double* b, double kappa, int E, int nn, double bound, double* c, int* route, int* err,
                        int grid, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  grid = std::max(1, std::min(grid, (E + 7) / 8));
  coeff_route_kernel<<<grid, 256, 0, s>>>(b, kappa * kappa, E, nn, bound, c, route, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t route_lists(const int* route, int E, int* good, int* bad, int* counts, cudaStream_t s) {
  route_lists_kernel<<<1, 1024, 0, s>>>(route, E, good, bad, counts);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_leaf(const LeafParams& p, int grid, cudaStream_t s) {
  if (p.Zscr) leaf_ir_kernel<<<grid, IR_NT, leaf_ir_smem_bytes(p.N), s>>>(p);
  else leaf_kernel<<<grid, 256, leaf_smem_bytes(p.N, p.cw), s>>>(p);
  note_launch();
  return cudaGetLastError();
}

}  // namespace hps
