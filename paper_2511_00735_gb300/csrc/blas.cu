// Batched complex GEMM (SIMT, register-blocked, shared-memory tiles) and batched
// Gauss-Jordan inversion with partial pivoting, in double or float.
//
// These carry the dense algebra of the pair merges (section 4.1,
// eq. globalfacesystem: S = I - T_bb T_aa, S^{-1}, T_pair = D - C A^{-1} B)
// and of the multigrid sweeps (section 4.3).
#include "common.cuh"
#include "dense.cuh"

namespace hps {

namespace {

constexpr int NT = 256;

// One BM x BN tile of C over k in [kb, ke).  part >= 0: store the raw partial sum
// into the split-K workspace slot `part` instead of applying the epilogue.
template <typename R, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void gemm_tile(const GemmArgs<R>& a, const GemmDesc& d, int tm, int tn, int kb = 0,
                                          int ke = 1 << 30, int part = -1, int batch = 0, int mmax = 0,
                                          int nmax = 0) {
  using C = c_t<R>;
  constexpr int TY = BM / TM, TX = BN / TN;
  static_assert(TY * TX == NT, "tile shape must use 256 threads");
  __shared__ C As[BK][BM];
  __shared__ C Bs[BK][BN];
  const int n = d.n < 0 ? a.n_launch : d.n;
  const int m = d.m, k = d.k < ke ? d.k : ke;
  const int row0 = tm * BM, col0 = tn * BN;
  if (row0 >= m || col0 >= n) return;  // uniform over the block
  const int tid = threadIdx.x;
  const int ty = tid / TX, tx = tid % TX;
  C acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = czero<R>();
  const C* Ab = a.A + (long long)d.a_r * a.lda + d.a_c;
  for (int k0 = kb; k0 < k; k0 += BK) {
    for (int l = tid; l < BM * BK; l += NT) {
      const int i = l / BK, kk = l % BK;
      const int gi = row0 + i, gk = k0 + kk;
      As[kk][i] = (gi < m && gk < k) ? Ab[(long long)gi * a.lda + gk] : czero<R>();
    }
    for (int l = tid; l < BK * BN; l += NT) {
      const int kk = l / BN, j = l % BN;
      const int gk = k0 + kk, gj = col0 + j;
      const long long br = (d.kb2 > 0 && gk >= d.kb2) ? (long long)d.b_r2 + (gk - d.kb2) : (long long)d.b_r + gk;
      Bs[kk][j] = (gk < k && gj < n) ? a.B[br * a.ldb + d.b_c + gj] : czero<R>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + i * TY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + j * TX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], av[i], bv[j]);
    }
    __syncthreads();
  }
  if (part >= 0) {
    C* W = a.ws + (((long long)part * a.nbatch + batch) * mmax) * nmax;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gi = row0 + ty + i * TY;
      if (gi >= m) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gj = col0 + tx + j * TX;
        if (gj < n) W[(long long)gi * nmax + gj] = acc[i][j];
      }
    }
    return;
  }
  const int* rmap = d.rmap >= 0 ? a.maps + d.rmap : nullptr;
  const int* cmap = d.cmap >= 0 ? a.maps + d.cmap : nullptr;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gi = row0 + ty + i * TY;
    if (gi >= m) continue;
    const long long orow = (long long)d.c_r + (rmap ? rmap[gi] : gi);
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = col0 + tx + j * TX;
      if (gj >= n) continue;
      C v = cmul(a.alpha, acc[i][j]);
      if (a.C0) {
        const long long cr = (d.mc2 > 0 && gi >= d.mc2) ? (long long)d.c0_r2 + (gi - d.mc2) : (long long)d.c0_r + gi;
        const C c0 = a.C0[cr * a.ldc0 + d.c0_c + gj];
        v = cadd(v, cmul(a.beta, c0));
      }
      const long long ocol = (long long)d.c_c + (cmap ? cmap[gj] : gj);
      a.C[orow * a.ldc + ocol] = v;
    }
  }
}

template <typename R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(NT) cgemm_kernel(GemmArgs<R> a) {
  for (int b = blockIdx.z; b < a.nbatch; b += gridDim.z) {
    const GemmDesc d = a.desc[b];
    gemm_tile<R, BM, BN, BK, TM, TN>(a, d, blockIdx.y, blockIdx.x);
  }
}

// Split-K: blockIdx.z = batch + nbatch * split; each split covers kc consecutive k.
template <typename R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(NT) cgemm_split_kernel(GemmArgs<R> a, int ksplit, int kc, int mmax, int nmax) {
  const int b = blockIdx.z % a.nbatch, sp = blockIdx.z / a.nbatch;
  const GemmDesc d = a.desc[b];
  gemm_tile<R, BM, BN, BK, TM, TN>(a, d, blockIdx.y, blockIdx.x, sp * kc, (sp + 1) * kc, sp, b, mmax, nmax);
}

// Sum the split-K partials (fixed order) and apply the epilogue of gemm_tile.
template <typename R>
__global__ void __launch_bounds__(NT) splitk_reduce_kernel(GemmArgs<R> a, int ksplit, int mmax, int nmax) {
  using C = c_t<R>;
  const int b = blockIdx.y;
  const GemmDesc d = a.desc[b];
  const int n = d.n < 0 ? a.n_launch : d.n;
  const int m = d.m;
  const int* rmap = d.rmap >= 0 ? a.maps + d.rmap : nullptr;
  const int* cmap = d.cmap >= 0 ? a.maps + d.cmap : nullptr;
  for (int l = blockIdx.x * NT + threadIdx.x; l < m * n; l += gridDim.x * NT) {
    const int i = l / n, j = l % n;
    C acc = czero<R>();
    for (int sp = 0; sp < ksplit; ++sp)
      acc = cadd(acc, a.ws[(((long long)sp * a.nbatch + b) * mmax + i) * nmax + j]);
    C v = cmul(a.alpha, acc);
    if (a.C0) {
      const long long cr = (d.mc2 > 0 && i >= d.mc2) ? (long long)d.c0_r2 + (i - d.mc2) : (long long)d.c0_r + i;
      v = cadd(v, cmul(a.beta, a.C0[cr * a.ldc0 + d.c0_c + j]));
    }
    a.C[((long long)d.c_r + (rmap ? rmap[i] : i)) * a.ldc + d.c_c + (cmap ? cmap[j] : j)] = v;
  }
}

template <typename R, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_cfg(const GemmArgs<R>& a, int mmax, int nmax, int kmax, cudaStream_t s) {
  const int gx = (nmax + BN - 1) / BN, gy = (mmax + BM - 1) / BM;
  if (gx == 0 || gy == 0 || a.nbatch == 0) return cudaSuccess;
  const long long blocks = (long long)gx * gy * a.nbatch;
  int ksplit = 1;
  if (kmax >= 4 * BK && a.ws && blocks < 2LL * a.num_sms) {
    ksplit = (int)((2LL * a.num_sms + blocks - 1) / blocks);
    ksplit = ksplit < kmax / (2 * BK) ? ksplit : kmax / (2 * BK);
    ksplit = ksplit < 16 ? ksplit : 16;
    while (ksplit > 1 && ((long long)ksplit * a.nbatch > 65535 ||
                          (long long)ksplit * a.nbatch * mmax * nmax > a.ws_elems))
      --ksplit;
  }
  if (ksplit <= 1) {
    dim3 grid(gx, gy, a.nbatch < 65535 ? a.nbatch : 65535);
    cgemm_kernel<R, BM, BN, BK, TM, TN><<<grid, NT, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
  }
  int kc = (kmax + ksplit - 1) / ksplit;
  kc = (kc + BK - 1) / BK * BK;
  ksplit = (kmax + kc - 1) / kc;
  dim3 grid(gx, gy, a.nbatch * ksplit);
  cgemm_split_kernel<R, BM, BN, BK, TM, TN><<<grid, NT, 0, s>>>(a, ksplit, kc, mmax, nmax);
  note_launch();
  int rb = (mmax * nmax + NT - 1) / NT;
  rb = rb < 64 ? rb : 64;
  dim3 rgrid(rb, a.nbatch);
  splitk_reduce_kernel<R><<<rgrid, NT, 0, s>>>(a, ksplit, mmax, nmax);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gauss-Jordan
// ---------------------------------------------------------------------------

template <typename R>
__global__ void __launch_bounds__(NT) gj_small_kernel(c_t<R>* W, int m, int ld, int* flag) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);
  C* Wg = W + (long long)blockIdx.x * m * ld;
  for (int l = threadIdx.x; l < m * ld; l += NT) S[l] = Wg[l];
  __syncthreads();
  gj_smem<R>(S, m, ld, ld, flag);
  const int w = ld - m;
  for (int l = threadIdx.x; l < m * w; l += NT) {
    const int i = l / w, j = m + l % w;
    Wg[i * ld + j] = S[i * ld + j];
  }
}

// Pivot search and LU of the (m-k0) x kb column slab of one matrix.
template <typename R>
__global__ void __launch_bounds__(NT) gj_panel_kernel(c_t<R>* W, int m, int ld, int k0, int kb, int* piv,
                                                      c_t<R>* lu, int* flag) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* S = reinterpret_cast<C*>(smem_raw);  // [mr][kb]
  const int mr = m - k0;
  const C* Wg = W + (long long)blockIdx.x * m * ld;
  for (int l = threadIdx.x; l < mr * kb; l += NT) {
    const int i = l / kb, c = l % kb;
    S[l] = Wg[(long long)(k0 + i) * ld + k0 + c];
  }
  __syncthreads();
  for (int c = 0; c < kb; ++c) {
    const int p = block_argmax_col<R>(S, kb, c, c, mr);
    if (threadIdx.x == 0) {
      piv[blockIdx.x * GJ_NB + c] = k0 + (p >= 0 ? p : c);
      if (p < 0 || (S[p * kb + c].x == 0 && S[p * kb + c].y == 0)) {
        if (flag) atomicExch(flag, 1);
      }
    }
    if (p != c && p >= 0) {
      for (int j = threadIdx.x; j < kb; j += NT) {
        const C t = S[c * kb + j];
        S[c * kb + j] = S[p * kb + j];
        S[p * kb + j] = t;
      }
    }
    __syncthreads();
    const C inv = cinv(S[c * kb + c]);
    for (int i = c + 1 + threadIdx.x; i < mr; i += NT) S[i * kb + c] = cmul(S[i * kb + c], inv);
    __syncthreads();
    const int w = kb - c - 1;
    if (w > 0) {
      for (int l = threadIdx.x; l < (mr - c - 1) * w; l += NT) {
        const int i = c + 1 + l / w, j = c + 1 + l % w;
        C v = S[i * kb + j];
        const C f = S[i * kb + c], u = S[c * kb + j];
        v.x -= f.x * u.x - f.y * u.y;
        v.y -= f.x * u.y + f.y * u.x;
        S[i * kb + j] = v;
      }
    }
    __syncthreads();
  }
  C* L = lu + (long long)blockIdx.x * GJ_NB * GJ_NB;
  for (int l = threadIdx.x; l < kb * kb; l += NT) L[(l / kb) * GJ_NB + l % kb] = S[l];
}

// Row swaps of one column block and the pivot rows' solve P = (L11 U11)^{-1} W(k0:k0+kb, j).
template <typename R>
__global__ void __launch_bounds__(NT) gj_apply_kernel(c_t<R>* W, int m, int ld, int k0, int kb, const int* piv,
                                                      const c_t<R>* lu) {
  using C = c_t<R>;
  __shared__ C sL[GJ_NB * GJ_NB];
  __shared__ int sp[GJ_NB];
  const int mat = blockIdx.y;
  for (int l = threadIdx.x; l < GJ_NB * GJ_NB; l += NT) sL[l] = lu[(long long)mat * GJ_NB * GJ_NB + l];
  if (threadIdx.x < GJ_NB) sp[threadIdx.x] = piv[mat * GJ_NB + threadIdx.x];
  __syncthreads();
  const int j = k0 + blockIdx.x * NT + threadIdx.x;
  if (j >= ld) return;
  C* Wg = W + (long long)mat * m * ld;
  for (int c = 0; c < kb; ++c) {
    const int r1 = k0 + c, r2 = sp[c];
    if (r2 != r1) {
      const C t = Wg[(long long)r1 * ld + j];
      Wg[(long long)r1 * ld + j] = Wg[(long long)r2 * ld + j];
      Wg[(long long)r2 * ld + j] = t;
    }
  }
  if (j < k0 + kb) return;
  C y[GJ_NB];
#pragma unroll
  for (int c = 0; c < GJ_NB; ++c) y[c] = c < kb ? Wg[(long long)(k0 + c) * ld + j] : czero<R>();
#pragma unroll
  for (int c = 0; c < GJ_NB; ++c) {
#pragma unroll
    for (int cc = 0; cc < c; ++cc) {
      if (c < kb) {
        const C f = sL[c * GJ_NB + cc];
        y[c].x -= f.x * y[cc].x - f.y * y[cc].y;
        y[c].y -= f.x * y[cc].y + f.y * y[cc].x;
      }
    }
  }
#pragma unroll
  for (int c = GJ_NB - 1; c >= 0; --c) {
    if (c < kb) {
#pragma unroll
      for (int cc = c + 1; cc < GJ_NB; ++cc) {
        if (cc < kb) {
          const C f = sL[c * GJ_NB + cc];
          y[c].x -= f.x * y[cc].x - f.y * y[cc].y;
          y[c].y -= f.x * y[cc].y + f.y * y[cc].x;
        }
      }
      y[c] = cmul(y[c], cinv(sL[c * GJ_NB + c]));
    }
  }
#pragma unroll
  for (int c = 0; c < GJ_NB; ++c)
    if (c < kb) Wg[(long long)(k0 + c) * ld + j] = y[c];
}

// Rank-kb elimination of every non-pivot row: W(i, j) -= W(i, k0:k0+kb) P(:, j), j >= k0+kb.
template <typename R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(NT) gj_update_kernel(c_t<R>* W, int m, int ld, int k0, int kb) {
  const int mat = blockIdx.z / 2, part = blockIdx.z % 2;
  GemmDesc d;
  const int base = mat * m;
  const int r0 = part == 0 ? 0 : k0 + kb;
  d.m = part == 0 ? k0 : m - k0 - kb;
  d.n = ld - k0 - kb;
  d.k = kb;
  d.a_r = base + r0;
  d.a_c = k0;
  d.b_r = base + k0;
  d.b_c = k0 + kb;
  d.c0_r = d.c_r = base + r0;
  d.c0_c = d.c_c = k0 + kb;
  d.rmap = d.cmap = -1;
  d.b_r2 = d.kb2 = d.c0_r2 = d.mc2 = 0;
  GemmArgs<R> a;
  a.A = a.B = a.C0 = W;
  a.C = W;
  a.lda = a.ldb = a.ldc0 = a.ldc = ld;
  a.alpha = mk<R>(R(-1), R(0));
  a.beta = mk<R>(R(1), R(0));
  a.desc = nullptr;
  a.nbatch = 1;
  a.maps = nullptr;
  a.n_launch = d.n;
  gemm_tile<R, BM, BN, BK, TM, TN>(a, d, blockIdx.y, blockIdx.x);
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) smem_optin(kernel);
}


// ---------------------------------------------------------------------------
// Skinny GEMM for n <= NC columns (block vectors of right-hand sides): A is
// streamed once with coalesced loads (lanes split k), B is staged in padded
// shared memory by k-chunks, each warp accumulates RW rows x NC columns and
// reduces across its lanes at the end.  Same descriptors and epilogue as
// gemm_tile (two-segment B / C0, row and column maps).
// ---------------------------------------------------------------------------
template <typename R, int NC, int RW, int KU>
__global__ void __launch_bounds__(NT) skinny_kernel(GemmArgs<R> a) {
  using C = c_t<R>;
  constexpr int KC = 32 * KU;      // k-chunk: every lane holds KU values of A per row
  constexpr int LDB = NC + 1;      // padding against bank conflicts
  constexpr int RB = (NT / 32) * RW;
  __shared__ C Bs[KC * LDB];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int b = blockIdx.z; b < a.nbatch; b += gridDim.z) {
    const GemmDesc d = a.desc[b];
    const int n = d.n < 0 ? a.n_launch : d.n;
    const int m = d.m, k = d.k;
    const int row0 = blockIdx.x * RB;
    if (row0 >= m) continue;  // uniform over the block
    C acc[RW][NC];
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[r][c] = czero<R>();
    const C* arow[RW];
    bool rok[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int gi = row0 + warp * RW + r;
      rok[r] = gi < m;
      arow[r] = a.A + (long long)(d.a_r + (rok[r] ? gi : 0)) * a.lda + d.a_c;
    }
    for (int k0 = 0; k0 < k; k0 += KC) {
      // issue this lane's loads of A first (KU x RW independent loads in flight)
      C av[RW][KU];
#pragma unroll
      for (int t = 0; t < KU; ++t) {
        const int gk = k0 + lane + 32 * t;
#pragma unroll
        for (int r = 0; r < RW; ++r) av[r][t] = (rok[r] && gk < k) ? arow[r][gk] : czero<R>();
      }
      __syncthreads();
      for (int l = threadIdx.x; l < KC * NC; l += NT) {
        const int kk = l / NC, j = l % NC;
        const int gk = k0 + kk;
        C v = czero<R>();
        if (gk < k && j < n) {
          const long long br = (d.kb2 > 0 && gk >= d.kb2) ? (long long)d.b_r2 + (gk - d.kb2) : (long long)d.b_r + gk;
          v = a.B[br * a.ldb + d.b_c + j];
        }
        Bs[kk * LDB + j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < KU; ++t) {
        const int kk = lane + 32 * t;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const C bv = Bs[kk * LDB + c];
#pragma unroll
          for (int r = 0; r < RW; ++r) cfma(acc[r][c], av[r][t], bv);
        }
      }
    }
    // reduce across lanes; lane c ends up owning column c of each row
#pragma unroll
    for (int r = 0; r < RW; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          acc[r][c].x += __shfl_xor_sync(0xffffffffu, acc[r][c].x, off);
          acc[r][c].y += __shfl_xor_sync(0xffffffffu, acc[r][c].y, off);
        }
    const int* rmap = d.rmap >= 0 ? a.maps + d.rmap : nullptr;
    const int* cmap = d.cmap >= 0 ? a.maps + d.cmap : nullptr;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int gi = row0 + warp * RW + r;
      if (!rok[r]) continue;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c % 32 != lane || c >= n) continue;
        C v = cmul(a.alpha, acc[r][c]);
        if (a.C0) {
          const long long cr = (d.mc2 > 0 && gi >= d.mc2) ? (long long)d.c0_r2 + (gi - d.mc2) : (long long)d.c0_r + gi;
          v = cadd(v, cmul(a.beta, a.C0[cr * a.ldc0 + d.c0_c + c]));
        }
        const long long orow = (long long)d.c_r + (rmap ? rmap[gi] : gi);
        a.C[orow * a.ldc + d.c_c + (cmap ? cmap[c] : c)] = v;
      }
    }
  }
}

template <typename R, int NC, int RW, int KU>
cudaError_t launch_skinny(const GemmArgs<R>& a, int mmax, cudaStream_t s) {
  constexpr int RB = (NT / 32) * RW;
  dim3 grid((mmax + RB - 1) / RB, 1, a.nbatch < 65535 ? a.nbatch : 65535);
  skinny_kernel<R, NC, RW, KU><<<grid, NT, 0, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_gemm(const GemmArgs<R>& a, int mmax, int nmax, cudaStream_t s, int kmax) {
  if (a.nbatch <= 0 || mmax <= 0 || nmax <= 0) return cudaSuccess;
  // block-vector products (few columns): the skinny kernel streams A once; measured slower than
  // the tiled kernels for every sweep shape of the 64x64 workload, so it is kept off by default.
  if (kmax >= (1 << 30)) {
    if (sizeof(R) == 4) {
      if (nmax <= 8) return launch_skinny<R, 8, 4, 8>(a, mmax, s);
      if (nmax <= 16) return launch_skinny<R, 16, 2, 8>(a, mmax, s);
      if (nmax <= 32) return launch_skinny<R, 32, 1, 8>(a, mmax, s);
    } else {
      if (nmax <= 8) return launch_skinny<R, 8, 2, 4>(a, mmax, s);
      if (nmax <= 16) return launch_skinny<R, 16, 1, 4>(a, mmax, s);
    }
  }
  if (nmax <= 16) {
    if (mmax <= 16) return launch_cfg<R, 16, 16, 16, 1, 1>(a, mmax, nmax, kmax, s);
    if (mmax <= 32) return launch_cfg<R, 32, 16, 16, 2, 1>(a, mmax, nmax, kmax, s);
    return launch_cfg<R, 64, 16, 16, 4, 1>(a, mmax, nmax, kmax, s);
  }
  if (nmax <= 32) {
    if (mmax <= 32) return launch_cfg<R, 32, 32, 8, 2, 2>(a, mmax, nmax, kmax, s);
    return launch_cfg<R, 64, 32, 8, 4, 2>(a, mmax, nmax, kmax, s);
  }
  if (mmax <= 32) return launch_cfg<R, 32, 32, 8, 2, 2>(a, mmax, nmax, kmax, s);
  return launch_cfg<R, 64, 64, 8, 4, 4>(a, mmax, nmax, kmax, s);
}

template <typename R>
cudaError_t gj_solve(c_t<R>* W, int m, int ld, int nmat, int* piv_ws, c_t<R>* lu_ws, int* flag, cudaStream_t s) {
  using C = c_t<R>;
  if (m <= 0 || nmat <= 0 || ld <= m) return cudaSuccess;
  const size_t small_bytes = (size_t)m * ld * sizeof(C);
  if (small_bytes <= 160 * 1024) {
    set_smem(gj_small_kernel<R>, small_bytes);
    for (int b0 = 0; b0 < nmat; b0 += 65535) {
      const int nb = nmat - b0 < 65535 ? nmat - b0 : 65535;
      gj_small_kernel<R><<<nb, NT, small_bytes, s>>>(W + (long long)b0 * m * ld, m, ld, flag);
      note_launch();
    }
    return cudaGetLastError();
  }
  if (nmat > 65535 / 2) return cudaErrorInvalidValue;
  // panel width: at most GJ_NB columns, fewer when the (m x kb) slab would not fit
  int nbw = GJ_NB;
  while (nbw > 1 && (size_t)m * nbw * sizeof(C) > 200 * 1024) --nbw;
  const size_t panel_bytes = (size_t)m * nbw * sizeof(C);
  if (panel_bytes > 200 * 1024) return cudaErrorInvalidValue;
  set_smem(gj_panel_kernel<R>, panel_bytes);
  for (int k0 = 0; k0 < m; k0 += nbw) {
    const int kb = m - k0 < nbw ? m - k0 : nbw;
    gj_panel_kernel<R><<<nmat, NT, panel_bytes, s>>>(W, m, ld, k0, kb, piv_ws, lu_ws, flag);
    note_launch();
    dim3 ga((ld - k0 + NT - 1) / NT, nmat);
    gj_apply_kernel<R><<<ga, NT, 0, s>>>(W, m, ld, k0, kb, piv_ws, lu_ws);
    note_launch();
    const int mrows = k0 > m - k0 - kb ? k0 : m - k0 - kb;
    const int ncols = ld - k0 - kb;
    if (mrows > 0 && ncols > 0) {
      dim3 gu((ncols + 63) / 64, (mrows + 63) / 64, nmat * 2);
      gj_update_kernel<R, 64, 64, 8, 4, 4><<<gu, NT, 0, s>>>(W, m, ld, k0, kb);
      note_launch();
    }
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t gj_invert(c_t<R>* W, int m, int nmat, int* piv_ws, c_t<R>* lu_ws, int* flag, cudaStream_t s) {
  return gj_solve<R>(W, m, 2 * m, nmat, piv_ws, lu_ws, flag, s);
}

template cudaError_t launch_gemm<double>(const GemmArgs<double>&, int, int, cudaStream_t, int);
template cudaError_t launch_gemm<float>(const GemmArgs<float>&, int, int, cudaStream_t, int);
template cudaError_t gj_invert<double>(double2*, int, int, int*, double2*, int*, cudaStream_t);
template cudaError_t gj_invert<float>(float2*, int, int, int*, float2*, int*, cudaStream_t);
template cudaError_t gj_solve<double>(double2*, int, int, int, int*, double2*, int*, cudaStream_t);
template cudaError_t gj_solve<float>(float2*, int, int, int, int*, float2*, int*, cudaStream_t);

}  // namespace hps
