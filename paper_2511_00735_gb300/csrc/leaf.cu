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

#include "common.cuh"
#include "dense.cuh"
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

  const int nel = (p.elems || p.ed) ? p.count : p.E;
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
// memory (half the FP64 size), the 4q right-hand sides are solved together,
// each column by four lanes of one warp (no block barriers inside the
// triangular solves), and the FP64 iterate Z stays in a per-CTA global
// workspace.  The refinement stops once the predicted next correction is
// below 1e-14 of Z (ratio of the last two corrections); the element is flagged
// if that takes more than IR_MAX steps.  A, P = A + i eta I and the FP64
// Gauss-Jordan inverse are as in leaf_kernel.
// ---------------------------------------------------------------------------
constexpr int IR_MAX = 10;

__host__ __device__ inline int ir_ldy(int nb) { return (nb + 23) / 32 * 32 + 8; }  // = 8 mod 32: no bank conflicts
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

__global__ void __launch_bounds__(256, 1) leaf_ir_kernel(LeafParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1;
  const int npk = ni * (ni + 1) / 2, ldy = ir_ldy(nb);
  float* Lp = reinterpret_cast<float*>(smem_raw);     // packed FP32 factor: unit lower U, d on the diagonal
  float* Y = Lp + ir_npk_pad(ni);                      // [ni][ldy] right-hand sides / corrections, FP32
  const size_t reg0 = max((size_t)ir_npk_pad(ni) * 4 + (size_t)ni * ldy * 4, (size_t)nb * 2 * nb * 16);
  double* sD = reinterpret_cast<double*>(smem_raw + (reg0 + 15) / 16 * 16);  // [n1*n1] physical D
  double* sK = sD + n1 * n1;                           // [n1*n1] reference K
  double* sw = sK + n1 * n1;                           // [n1] reference weights
  double* sc = sw + n1;                                // [n1*n1] c of this element
  double* red = sc + n1 * n1;                          // [8] reductions
  const int tid = threadIdx.x, nth = blockDim.x;
  double* A = p.Ascr + (long long)blockIdx.x * nb * nb;
  double* Z = p.Zscr + (long long)blockIdx.x * ni * nb;

  for (int l = tid; l < n1 * n1; l += nth) sK[l] = p.Kh[l];
  for (int l = tid; l < n1; l += nth) sw[l] = p.wh[l];

  const int nel = (p.elems || p.ed) ? p.count : p.E;
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
    }
    __syncthreads();
    // ---- assemble L~_ii (FP32, packed lower triangle) ----
    for (int l = tid; l < npk; l += nth) {
      int r = (int)((sqrt(8.0 * l + 1.0) - 1.0) * 0.5);
      while (r * (r + 1) / 2 > l) --r;
      while ((r + 1) * (r + 2) / 2 <= l) ++r;
      const int cc = l - r * (r + 1) / 2;
      const int i = r / q + 1, j = r % q + 1, i2 = cc / q + 1, j2 = cc % q + 1;
      double v = 0.0;
      if (j == j2) v += sK[i * n1 + i2] * sw[j];
      if (i == i2) v += sw[i] * sK[j * n1 + j2];
      if (r == cc) v -= sc[i * n1 + j] * h2 * sw[i] * sw[j];
      Lp[l] = (float)v;
    }
    __syncthreads();
    // ---- FP32 right-looking L D L^T (column k kept in Y's space while it is updated) ----
    {
      float* colk = Y;
      float prev_inv = 0.f;
      for (int k = 0; k < ni; ++k) {
        for (int i = k + tid; i < ni; i += nth) colk[i] = Lp[pk(i, k)];
        __syncthreads();
        float dk = colk[k];
        if (!(dk > 0.f)) {
          if (tid == 0) atomicCAS(p.flag, 0, ei + 1);
          dk = 1.f;
        }
        const float inv = 1.f / dk;
        if (k > 0)
          for (int i = k + tid; i < ni; i += nth) Lp[pk(i, k - 1)] *= prev_inv;
        const int warp = tid / 32, lane = tid % 32, nw = nth / 32;
        for (int i = k + 1 + warp; i < ni; i += nw) {
          const float f = colk[i] * inv;
          float* row = Lp + pk(i, 0);
          for (int j = k + 1 + lane; j <= i; j += 32) row[j] -= f * colk[j];
        }
        prev_inv = inv;
        __syncthreads();
      }
    }
    // ---- refinement: Z <- Z + (L D L^T)^{-1} (L~_iG - L~_ii Z) ----
    const int part = tid % 4;  // four lanes per right-hand side column
    const bool cact = tid / 4 < nb;
    const int col = cact ? tid / 4 : 0;  // idle lanes read column 0 and write nothing
    double rel_prev = 1.0;
    bool done = false;
    for (int it = 0; it < IR_MAX && !done; ++it) {
      // residual (FP64), rounded into Y
      for (int l = tid; l < ni * nb; l += nth) {
        const int I = l / nb, g = l % nb;
        const int i = I / q + 1, j = I % q + 1;
        const int side = g / q, s = g % q + 1;
        double bv = 0.0;
        if (side == 0 && j == s) bv = sK[i * n1 + 0] * sw[s];
        else if (side == 1 && j == s) bv = sK[i * n1 + N] * sw[s];
        else if (side == 2 && i == s) bv = sw[s] * sK[j * n1 + 0];
        else if (side == 3 && i == s) bv = sw[s] * sK[j * n1 + N];
        if (it > 0) {
          double s1 = 0.0, s2 = 0.0;
          for (int t = 1; t <= q; ++t) {
            s1 += sK[i * n1 + t] * Z[(long long)((t - 1) * q + (j - 1)) * nb + g];
            s2 += sK[j * n1 + t] * Z[(long long)((i - 1) * q + (t - 1)) * nb + g];
          }
          bv -= sw[j] * s1 + sw[i] * s2 - sc[i * n1 + j] * h2 * sw[i] * sw[j] * Z[(long long)I * nb + g];
        }
        Y[I * ldy + g] = (float)bv;
      }
      __syncthreads();
      // forward: U y = r (unit lower), four lanes per column, warp-synchronous
      for (int i = 1; i < ni; ++i) {
        float a0 = 0.f, a1 = 0.f;
        const float* Ui = Lp + pk(i, 0);
        int k = part;
        for (; k + 4 < i; k += 8) {
          a0 += Ui[k] * Y[k * ldy + col];
          a1 += Ui[k + 4] * Y[(k + 4) * ldy + col];
        }
        if (k < i) a0 += Ui[k] * Y[k * ldy + col];
        float sum = a0 + a1;
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if (cact && part == 0) Y[i * ldy + col] -= sum;
        __syncwarp();
      }
      // diagonal
      if (cact)
        for (int i = part; i < ni; i += 4) Y[i * ldy + col] /= Lp[pk(i, i)];
      __syncwarp();
      // backward: U^T x = z
      for (int i = ni - 2; i >= 0; --i) {
        float a0 = 0.f, a1 = 0.f;
        int k = i + 1 + part;
        for (; k + 4 < ni; k += 8) {
          a0 += Lp[pk(k, i)] * Y[k * ldy + col];
          a1 += Lp[pk(k + 4, i)] * Y[(k + 4) * ldy + col];
        }
        if (k < ni) a0 += Lp[pk(k, i)] * Y[k * ldy + col];
        float sum = a0 + a1;
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if (cact && part == 0) Y[i * ldy + col] -= sum;
        __syncwarp();
      }
      __syncthreads();
      // Z += correction (FP64), sizes for the stopping test
      double md = 0.0, mz = 0.0;
      for (int l = tid; l < ni * nb; l += nth) {
        const int I = l / nb, g = l % nb;
        const double d = (double)Y[I * ldy + g];
        const double z = (it == 0 ? 0.0 : Z[l]) + d;
        Z[l] = z;
        md = fmax(md, fabs(d));
        mz = fmax(mz, fabs(z));
      }
      md = block_max(md, red);
      mz = block_max(mz, red);
      const double rel = mz > 0.0 ? md / mz : 0.0;
      if (it > 0) {
        const double rho = fmax(rel / rel_prev, 1e-6);
        done = rel * rho <= 1e-14;
      }
      if (!(rel == rel)) done = false;
      rel_prev = rel > 0.0 ? rel : 1e-300;
      if (rel == 0.0) done = true;
      if (!done && it == IR_MAX - 1 && tid == 0) atomicCAS(p.flag, 0, ei + 1);
      __syncthreads();
    }

    // ---- A = Dn_GG - Dn_Gi Z (FP64) ----
    for (int l = tid; l < nb * nb; l += nth) {
      const int g = l / nb, gc = l % nb;
      const int side = g / q, s = g % q + 1;
      double acc = 0.0;
      for (int t = 1; t <= q; ++t) {
        int I;
        double dcoef;
        if (side == 0) { I = (t - 1) * q + (s - 1); dcoef = -sD[0 * n1 + t]; }
        else if (side == 1) { I = (t - 1) * q + (s - 1); dcoef = sD[N * n1 + t]; }
        else if (side == 2) { I = (s - 1) * q + (t - 1); dcoef = -sD[0 * n1 + t]; }
        else { I = (s - 1) * q + (t - 1); dcoef = sD[N * n1 + t]; }
        acc += dcoef * Z[(long long)I * nb + gc];
      }
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
    // ---- P = A + i eta I, Gauss-Jordan [P | I] -> P^{-1}, T = I - 2 i eta P^{-1} ----
    double2* W = reinterpret_cast<double2*>(smem_raw);
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

__global__ void robust_assemble_kernel(LeafParams p, const int* __restrict__ elems, int count,
                                       double2* __restrict__ W) {
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1, ld = ni + nb;
  const double dsc = 2.0 / p.h, h2 = 0.25 * p.h * p.h;
  __shared__ double sD[17 * 17];
  for (int l = threadIdx.x; l < n1 * n1; l += blockDim.x) sD[l] = dsc * p.Dh[l];
  __syncthreads();
  const Minv2 mi = mb_inverse(sD, N, p.eta);
  const long long tot = (long long)count * ni * ld;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(l / ((long long)ni * ld));
    const int rem = (int)(l % ((long long)ni * ld));
    const int I = rem / ld, col = rem % ld;
    const int e = elems[b];
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
      if (I == col) lt -= p.c[(long long)e * n1 * n1 + ti * n1 + tj] * h2 * p.wh[ti] * p.wh[tj];
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
    W[(long long)b * ni * ld + (long long)I * ld + col] = v;
  }
}

__global__ void robust_finish_kernel(LeafParams p, const int* __restrict__ elems, int count,
                                     const double2* __restrict__ W) {
  const int N = p.N, q = p.q, ni = p.ni, nb = p.nb, n1 = N + 1, ld = ni + nb;
  const double dsc = 2.0 / p.h;
  __shared__ double sD[17 * 17];
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

}  // namespace

cudaError_t robust_assemble(const LeafParams& p, const int* elems, int count, double2* W, cudaStream_t s) {
  const long long tot = (long long)count * p.ni * (p.ni + p.nb);
  long long blocks = (tot + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  robust_assemble_kernel<<<(int)blocks, 256, 0, s>>>(p, elems, count, W);
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

size_t leaf_ir_smem_bytes(int N) {
  const int q = N - 1, ni = q * q, nb = 4 * q, n1 = N + 1;
  const size_t reg0 = std::max((size_t)ir_npk_pad(ni) * 4 + (size_t)ni * ir_ldy(nb) * 4, (size_t)nb * 2 * nb * 16);
  return (reg0 + 15) / 16 * 16 + sizeof(double) * (3 * n1 * n1 + n1 + 8);
}

cudaError_t launch_leaf(const LeafParams& p, int grid, cudaStream_t s) {
  if (p.Zscr) {
    smem_optin(leaf_ir_kernel);
    leaf_ir_kernel<<<grid, 256, leaf_ir_smem_bytes(p.N), s>>>(p);
  } else {
    smem_optin(leaf_kernel);
    leaf_kernel<<<grid, 256, leaf_smem_bytes(p.N, p.cw), s>>>(p);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace hps
