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
        cfms(v, f, u);
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
        cfms(y[c], f, y[cc]);
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
          cfms(y[c], f, y[cc]);
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



// ---------------------------------------------------------------------------
// Block-vector GEMM (n <= 16 columns per block, the right-hand sides of the
// multigrid sweeps and of the coarse solve).  One thread owns RPT output rows
// and all 16 columns of each in registers: per k it reads one A value per row
// from a padded shared-memory tile (conflict-free) and the 16 B values of
// that k by broadcast, i.e. 16 x RPT complex FMAs per RPT + 8 (FP32) shared
// loads.  The A and B tiles of the next k-chunk stream in with cp.async while
// the current one is multiplied (two buffers), so the global loads need no
// registers and overlap the arithmetic.  Same descriptors and epilogue as
// gemm_tile (two-segment B / C0, row and column maps); blockIdx.y selects a
// 16-column slice, blockIdx.z = batch + nbatch * split for split-K (partials
// in the workspace, reduced in fixed order by splitk_reduce_kernel).
// ---------------------------------------------------------------------------
constexpr int RG_NT = 128, RG_NC = 16, RG_KC = 16;

template <typename R, int RPT>
constexpr size_t rowgemm_smem() {
  return 2 * sizeof(c_t<R>) * ((size_t)RG_NT * RPT * (RG_KC + 1) + (size_t)RG_KC * RG_NC);
}

// asynchronous global -> shared copy of one complex value; zero-filled when !pred
template <typename C>
__device__ __forceinline__ void cp_async_c(C* dst, const C* src, bool pred) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  const int nbytes = pred ? (int)sizeof(C) : 0;
  if (sizeof(C) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(src), "r"(nbytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// the 16 B values of one k (a 16-column row of the B tile, 16-byte aligned)
template <typename C>
__device__ __forceinline__ void load_brow(const C* src, C (&bv)[RG_NC]) {
  if constexpr (sizeof(C) == 8) {
#pragma unroll
    for (int q = 0; q < RG_NC / 2; ++q) {
      const float4 t = reinterpret_cast<const float4*>(src)[q];
      bv[2 * q] = make_float2(t.x, t.y);
      bv[2 * q + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < RG_NC; ++j) bv[j] = src[j];
  }
}

template <typename R, int RPT>
__global__ void __launch_bounds__(RG_NT) rowgemm_kernel(GemmArgs<R> a, int ksplit, int kc, int mmax, int nmax) {
  using C = c_t<R>;
  constexpr int BM = RG_NT * RPT, LDA = RG_KC + 1;
  constexpr int ASZ = BM * LDA, BSZ = RG_KC * RG_NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Bs = reinterpret_cast<C*>(smem_raw);  // [2][KC][16] (first: 16-byte aligned rows)
  C* As = Bs + 2 * BSZ;                    // [2][BM][LDA]
  const int b = blockIdx.z % a.nbatch, sp = blockIdx.z / a.nbatch;
  const GemmDesc d = a.desc[b];
  const int n = d.n < 0 ? a.n_launch : d.n;
  const int m = d.m;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * RG_NC;
  if (row0 >= m || col0 >= n) return;  // uniform over the block
  const int kb = ksplit > 1 ? sp * kc : 0;
  const int ke = ksplit > 1 ? min(d.k, kb + kc) : d.k;
  const int tid = threadIdx.x;
  const C* Ab = a.A + (long long)d.a_r * a.lda + d.a_c;
  // issue the copies of chunk [k0, k0 + KC) into buffer `buf`
  auto load = [&](int k0, int buf) {
    C* Ad = As + buf * ASZ;
    C* Bd = Bs + buf * BSZ;
#pragma unroll 4
    for (int l = tid; l < BM * RG_KC; l += RG_NT) {
      const int i = l / RG_KC, kk = l % RG_KC;
      const int gi = row0 + i, gk = k0 + kk;
      const bool ok = gi < m && gk < ke;
      cp_async_c(Ad + i * LDA + kk, ok ? Ab + (long long)gi * a.lda + gk : Ab, ok);
    }
    for (int l = tid; l < BSZ; l += RG_NT) {
      const int kk = l / RG_NC, j = l % RG_NC;
      const int gk = k0 + kk, gj = col0 + j;
      const bool ok = gk < ke && gj < n;
      const long long br = (d.kb2 > 0 && gk >= d.kb2) ? (long long)d.b_r2 + (gk - d.kb2) : (long long)d.b_r + gk;
      cp_async_c(Bd + l, ok ? a.B + br * a.ldb + d.b_c + gj : a.B, ok);
    }
    cp_async_commit();
  };
  C acc[RPT][RG_NC];
#pragma unroll
  for (int i = 0; i < RPT; ++i)
#pragma unroll
    for (int j = 0; j < RG_NC; ++j) acc[i][j] = czero<R>();
  if (kb < ke) load(kb, 0);
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += RG_KC, buf ^= 1) {
    if (k0 + RG_KC < ke) {
      load(k0 + RG_KC, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const C* Ac = As + buf * ASZ;
    const C* Bc = Bs + buf * BSZ;
#pragma unroll 4
    for (int kk = 0; kk < RG_KC; ++kk) {
      C bv[RG_NC];
      load_brow(Bc + kk * RG_NC, bv);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const C av = Ac[(tid + i * RG_NT) * LDA + kk];
#pragma unroll
        for (int j = 0; j < RG_NC; ++j) cfma(acc[i][j], av, bv[j]);
      }
    }
    __syncthreads();  // buffer `buf` is refilled two chunks later
  }
  if (ksplit > 1) {
    C* W = a.ws + (((long long)sp * a.nbatch + b) * mmax) * nmax;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int gi = row0 + tid + i * RG_NT;
      if (gi >= m) continue;
#pragma unroll
      for (int j = 0; j < RG_NC; ++j) {
        const int gj = col0 + j;
        if (gj < n) W[(long long)gi * nmax + gj] = acc[i][j];
      }
    }
    return;
  }
  const int* rmap = d.rmap >= 0 ? a.maps + d.rmap : nullptr;
  const int* cmap = d.cmap >= 0 ? a.maps + d.cmap : nullptr;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int gi = row0 + tid + i * RG_NT;
    if (gi >= m) continue;
    const long long orow = (long long)d.c_r + (rmap ? rmap[gi] : gi);
    const long long cr = (d.mc2 > 0 && gi >= d.mc2) ? (long long)d.c0_r2 + (gi - d.mc2) : (long long)d.c0_r + gi;
#pragma unroll
    for (int j = 0; j < RG_NC; ++j) {
      const int gj = col0 + j;
      if (gj >= n) continue;
      C v = cmul(a.alpha, acc[i][j]);
      if (a.C0) v = cadd(v, cmul(a.beta, a.C0[cr * a.ldc0 + d.c0_c + gj]));
      a.C[orow * a.ldc + d.c_c + (cmap ? cmap[gj] : gj)] = v;
    }
  }
}

template <typename R, int RPT>
cudaError_t launch_rowgemm(const GemmArgs<R>& a, int mmax, int nmax, int kmax, cudaStream_t s) {
  constexpr int BM = RG_NT * RPT;
  constexpr size_t smem = rowgemm_smem<R, RPT>();
  const int gx = (mmax + BM - 1) / BM, gy = (nmax + RG_NC - 1) / RG_NC;
  const long long blocks = (long long)gx * gy * a.nbatch;
  // resident blocks per SM from the shared-memory footprint; split K until the GPU is covered
  const long long per_sm = (long long)(227 * 1024 / (smem + 1024));
  const long long target = (per_sm > 0 ? per_sm : 1) * a.num_sms;
  int ksplit = 1;
  if (kmax >= 4 * RG_KC && a.ws && blocks < target) {
    ksplit = (int)((target + blocks - 1) / blocks);
    ksplit = ksplit < kmax / (2 * RG_KC) ? ksplit : kmax / (2 * RG_KC);
    ksplit = ksplit < 32 ? ksplit : 32;
    while (ksplit > 1 && ((long long)ksplit * a.nbatch > 65535 ||
                          (long long)ksplit * a.nbatch * mmax * nmax > a.ws_elems))
      --ksplit;
  }
  int kc = kmax;
  if (ksplit > 1) {
    kc = (kmax + ksplit - 1) / ksplit;
    kc = (kc + RG_KC - 1) / RG_KC * RG_KC;
    ksplit = (kmax + kc - 1) / kc;
  }
  if ((long long)a.nbatch * ksplit > 65535) return cudaErrorInvalidValue;
  dim3 grid(gx, gy, a.nbatch * ksplit);
  rowgemm_kernel<R, RPT><<<grid, RG_NT, smem, s>>>(a, ksplit, kc, mmax, nmax);
  note_launch();
  if (ksplit > 1) {
    int rb = (mmax * nmax + NT - 1) / NT;
    rb = rb < 64 ? rb : 64;
    dim3 rgrid(rb, a.nbatch);
    splitk_reduce_kernel<R><<<rgrid, NT, 0, s>>>(a, ksplit, mmax, nmax);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_gemm(const GemmArgs<R>& a, int mmax, int nmax, cudaStream_t s, int kmax) {
  if (a.nbatch <= 0 || mmax <= 0 || nmax <= 0) return cudaSuccess;
  // FP32 products on the tensor cores (3xTF32): the merges of the upper levels and the
  // block-vector products of the sweeps and the coarse solve with long rows
  if constexpr (sizeof(R) == 4) {
    if (a.err && mmax >= 64 && kmax >= 64 && (nmax >= 64 || nmax <= 32) && a.nbatch <= 65535)
      return launch_tc_gemm(a, mmax, nmax, kmax, a.err, s);
  }
  // block-vector products (the sweeps' and the coarse solve's right-hand sides)
  if (nmax <= 16 && kmax > 0 && mmax > 32) {
    if (sizeof(R) == 4 && mmax > RG_NT) return launch_rowgemm<R, 2>(a, mmax, nmax, kmax, s);
    return launch_rowgemm<R, 1>(a, mmax, nmax, kmax, s);
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

void optin_blas() {
  smem_optin(rowgemm_kernel<float, 1>);
  smem_optin(rowgemm_kernel<float, 2>);
  smem_optin(rowgemm_kernel<double, 1>);
  smem_optin(gj_small_kernel<float>);
  smem_optin(gj_small_kernel<double>);
  smem_optin(gj_panel_kernel<float>);
  smem_optin(gj_panel_kernel<double>);
}

cudaError_t splitk_reduce(const GemmArgs<float>& a, int ksplit, int mmax, int nmax, cudaStream_t s) {
  int rb = (mmax * nmax + NT - 1) / NT;
  rb = rb < 64 ? rb : 64;
  splitk_reduce_kernel<float><<<dim3(rb, a.nbatch), NT, 0, s>>>(a, ksplit, mmax, nmax);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_gemm<double>(const GemmArgs<double>&, int, int, cudaStream_t, int);
template cudaError_t launch_gemm<float>(const GemmArgs<float>&, int, int, cudaStream_t, int);
template cudaError_t gj_invert<double>(double2*, int, int, int*, double2*, int*, cudaStream_t);
template cudaError_t gj_invert<float>(float2*, int, int, int*, float2*, int*, cudaStream_t);
template cudaError_t gj_solve<double>(double2*, int, int, int, int*, double2*, int*, cudaStream_t);
template cudaError_t gj_solve<float>(float2*, int, int, int, int*, float2*, int*, cudaStream_t);

}  // namespace hps
