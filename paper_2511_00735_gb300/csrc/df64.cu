// Double-float ("df64") vector kernels for the outer FGMRES of the mixed path.
//
// GB300 executes FP32 fused multiply-adds about 58x faster than FP64 ones, so the
// FP64-class work of the outer iteration -- the skeleton matvec and the
// Gram-Schmidt dot products and updates -- runs on pairs of floats (hi, lo) with
// |lo| <= ulp(hi)/2, i.e. about 48 significand bits.  Building blocks are the
// error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and the
// FMA-based TwoProduct, accumulated as in the compensated dot product "Dot2"
// (Ogita, Rump, Oishi, SIAM J. Sci. Comput. 26 (2005)): the running sum keeps
// its rounding errors and the products' errors in a separate float that is
// added once at the end.  Relative error of a length-n sum ~ n eps32^2 cond,
// far below the 1e-10 residual the solver certifies; the final residual of a
// solve is recomputed in true FP64.
//
// Storage: one complex df64 number is a float4 (re_hi, im_hi, re_lo, im_lo).
#include "common.cuh"
#include "df64.cuh"
#include "dfops.cuh"
#include "skel.cuh"

namespace hps {

namespace {
constexpr int NT = 256;

inline int nblocks(long long work, int cap) {
  long long b = (work + NT - 1) / NT;
  if (b < 1) b = 1;
  return (int)(b > cap ? cap : b);
}

// Blocks of `kernel` (threads per block, dynamic shared memory) that the current device runs at
// once: one full wave.  Streaming kernels sized to whole waves leave no partly filled last wave.
template <typename K>
int full_wave(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1 || sms < 1) {
    cudaGetLastError();
    return 0;  // unknown: the caller keeps its own count
  }
  return per * sms;
}

using dfops::dot2;
using dfops::fast2;
using dfops::two_sum;

struct cacc {  // complex df64 accumulator
  float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
};

// acc += a * b   (complex, a and b df64)
__device__ __forceinline__ void cdot2(cacc& acc, float4 a, float4 b) {
  dot2(acc.rs, acc.rc, a.x, a.z, b.x, b.z);
  dot2(acc.rs, acc.rc, -a.y, -a.w, b.y, b.w);
  dot2(acc.is, acc.ic, a.x, a.z, b.y, b.w);
  dot2(acc.is, acc.ic, a.y, a.w, b.x, b.z);
}
// acc += a * b   (complex, a df64, b FP32)
__device__ __forceinline__ void cdot2f(cacc& acc, float4 a, float2 b) {
  dfops::dot2f(acc.rs, acc.rc, a.x, a.z, b.x);
  dfops::dot2f(acc.rs, acc.rc, -a.y, -a.w, b.y);
  dfops::dot2f(acc.is, acc.ic, a.x, a.z, b.y);
  dfops::dot2f(acc.is, acc.ic, a.y, a.w, b.x);
}
// acc += conj(a) * b
__device__ __forceinline__ void cdot2_conj(cacc& acc, float4 a, float4 b) {
  dot2(acc.rs, acc.rc, a.x, a.z, b.x, b.z);
  dot2(acc.rs, acc.rc, a.y, a.w, b.y, b.w);
  dot2(acc.is, acc.ic, a.x, a.z, b.y, b.w);
  dot2(acc.is, acc.ic, -a.y, -a.w, b.x, b.z);
}
// acc += a (df64 complex value)
__device__ __forceinline__ void cadd2(cacc& acc, float4 a) {
  dot2(acc.rs, acc.rc, a.x, a.z, 1.f, 0.f);
  dot2(acc.is, acc.ic, a.y, a.w, 1.f, 0.f);
}
__device__ __forceinline__ float4 cfin(const cacc& a) {
  float4 r;
  fast2(a.rs, a.rc, r.x, r.z);
  fast2(a.is, a.ic, r.y, r.w);
  return r;
}
__device__ __forceinline__ float4 from_f2(float2 v) { return make_float4(v.x, v.y, 0.f, 0.f); }
using dfops::from_d2;
using dfops::to_d2;
__device__ __forceinline__ float4 ld(const float4* p, long long i) { return p[i]; }
__device__ __forceinline__ float4 ld(const float2* p, long long i) { return from_f2(p[i]); }

}  // namespace

// ---------------------------------------------------------------------------
__global__ void df_from_d_kernel(float4* __restrict__ dst, const double2* __restrict__ src, long long n) {
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < n; l += (long long)gridDim.x * NT)
    dst[l] = from_d2(src[l]);
}
__global__ void df_to_d_kernel(double2* __restrict__ dst, const float4* __restrict__ src, long long n) {
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < n; l += (long long)gridDim.x * NT)
    dst[l] = to_d2(src[l]);
}
cudaError_t df_from_d(float4* dst, const double2* src, long long n, cudaStream_t s) {
  df_from_d_kernel<<<nblocks(n, 8192), NT, 0, s>>>(dst, src, n);
  note_launch();
  return cudaGetLastError();
}
cudaError_t df_to_d(double2* dst, const float4* src, long long n, cudaStream_t s) {
  df_to_d_kernel<<<nblocks(n, 8192), NT, 0, s>>>(dst, src, n);
  note_launch();
  return cudaGetLastError();
}

// Gathers and scatters take GU elements per thread per pass (indices, then loads, then stores,
// each GU independent), so a thread has GU dependent map -> data chains in flight.
constexpr int GU = 4;

// rows of leading parts (FP32) through a row map: dst[row][r] = hi(src[map[row]][r]) (map < 0 -> 0),
// with the source pointer read from device memory (graph-replayable with a new source)
__global__ void df_gather_hi_ind_kernel(float2* __restrict__ dst, const float4* const* __restrict__ srcp,
                                        const int* __restrict__ map, long long rows, int nrhs) {
  // the leading FP32 pair of each double-float complex (8-byte loads)
  const float2* src = reinterpret_cast<const float2*>(*srcp);
  const long long tot = rows * nrhs, stride = (long long)gridDim.x * NT;
  for (long long l0 = blockIdx.x * (long long)NT + threadIdx.x; l0 < tot; l0 += GU * stride) {
    int m[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      m[u] = l < tot ? map[l / nrhs] : -1;
    }
    float2 v[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      v[u] = m[u] >= 0 ? src[2 * ((long long)m[u] * nrhs + l % nrhs)] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      if (l < tot) dst[l] = v[u];
    }
  }
}
cudaError_t df_gather_hi_ind(float2* dst, const float4* const* srcp, const int* map, long long rows, int nrhs,
                             cudaStream_t s) {
  df_gather_hi_ind_kernel<<<nblocks((rows * nrhs + GU - 1) / GU, 8192), NT, 0, s>>>(dst, srcp, map, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

__global__ void set_pointers_kernel(void** dst, const void* a, void* b) {
  dst[0] = const_cast<void*>(a);
  dst[1] = b;
}
cudaError_t set_pointers(void** dst, const void* a, void* b, cudaStream_t s) {
  set_pointers_kernel<<<1, 1, 0, s>>>(dst, a, b);
  note_launch();
  return cudaGetLastError();
}

// dst[map[row]][r] = src[row][r] (map < 0: skipped) with dst read from device memory
__global__ void scatter_f2_ind_kernel(float2* const* __restrict__ dstp, const float2* __restrict__ src,
                                      const int* __restrict__ map, long long rows, int nrhs) {
  float2* dst = *dstp;
  const long long tot = rows * nrhs, stride = (long long)gridDim.x * NT;
  for (long long l0 = blockIdx.x * (long long)NT + threadIdx.x; l0 < tot; l0 += GU * stride) {
    int m[GU];
    float2 v[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      m[u] = l < tot ? map[l / nrhs] : -1;
      v[u] = l < tot ? src[l] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      if (m[u] >= 0) dst[(long long)m[u] * nrhs + l % nrhs] = v[u];
    }
  }
}
cudaError_t scatter_f2_ind(float2* const* dstp, const float2* src, const int* map, long long rows, int nrhs,
                           cudaStream_t s) {
  scatter_f2_ind_kernel<<<nblocks((rows * nrhs + GU - 1) / GU, 8192), NT, 0, s>>>(dstp, src, map, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Outer matvec  y_p = x_{nb(p)} + sum_b T_e[a][b] x_{e,b}  (nb(p) >= 0), else 0;
// residual form y = c0 - that when c0 != null.  T in df64, x FP32 or df64.
template <typename X>
__global__ void __launch_bounds__(NT) df_matvec_kernel(const float4* __restrict__ T, const int* __restrict__ nbr,
                                                       const X* __restrict__ x, const float4* __restrict__ c0,
                                                       float4* __restrict__ y, int E, int nb, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  X* xs = reinterpret_cast<X*>(smem_raw);  // [nb][nrhs] this element's x (FP32 or df64 as given)
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    const long long base = (long long)e * nb;
    for (int l = threadIdx.x; l < nb * nrhs; l += NT) xs[l] = x[base * nrhs + l];
    __syncthreads();
    const float4* Te = T + (long long)e * nb * nb;
    for (int l = threadIdx.x; l < nb * nrhs; l += NT) {
      const int a = l / nrhs, r = l % nrhs;
      const long long p = base + a;
      const int q = nbr[p];
      float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q >= 0) {
        // two accumulators (even and odd b) halve the dependency chain through TwoSum
        cacc acc, acc2;
        cadd2(acc, ld(x, (long long)q * nrhs + r));
        const float4* Tr = Te + (long long)a * nb;
        int b = 0;
        for (; b + 1 < nb; b += 2) {
          if constexpr (sizeof(X) == sizeof(float2)) {  // x FP32: no lo products
            cdot2f(acc, Tr[b], xs[b * nrhs + r]);
            cdot2f(acc2, Tr[b + 1], xs[(b + 1) * nrhs + r]);
          } else {
            cdot2(acc, Tr[b], xs[b * nrhs + r]);
            cdot2(acc2, Tr[b + 1], xs[(b + 1) * nrhs + r]);
          }
        }
        if (b < nb) {
          if constexpr (sizeof(X) == sizeof(float2)) cdot2f(acc, Tr[b], xs[b * nrhs + r]);
          else cdot2(acc, Tr[b], xs[b * nrhs + r]);
        }
        cadd2(acc, cfin(acc2));
        if (c0) {
          const float4 cv = c0[p * nrhs + r];
          acc.rs = -acc.rs; acc.rc = -acc.rc; acc.is = -acc.is; acc.ic = -acc.ic;
          cadd2(acc, cv);
        }
        out = cfin(acc);
      }
      y[p * nrhs + r] = out;
    }
  }
}

template <typename X>
cudaError_t df_matvec(const float4* T, const int* nbr, const X* x, const float4* c0, float4* y, int E, int nb, int nrhs,
                      int grid, cudaStream_t s) {
  const size_t smem = sizeof(X) * (size_t)nb * nrhs;
  df_matvec_kernel<X><<<grid, NT, smem, s>>>(T, nbr, x, c0, y, E, nb, nrhs);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t df_matvec<float2>(const float4*, const int*, const float2*, const float4*, float4*, int, int, int,
                                       int, cudaStream_t);
template cudaError_t df_matvec<float4>(const float4*, const int*, const float4*, const float4*, float4*, int, int, int,
                                       int, cudaStream_t);

// ---------------------------------------------------------------------------
// h[i][r] = sum_rows conj(V_i) w   (two-pass, fixed order; block partials in df64, final sum in FP64)
// Vectors in groups of DG per block (blockIdx.y = group): w is read once per group.
constexpr int DG = 8;
__global__ void __launch_bounds__(NT) df_bdot_partial_kernel(const float4* __restrict__ V, long long vstride, int nvec,
                                                             const float4* __restrict__ w, long long rows, int nrhs,
                                                             int rpad, float4* __restrict__ partial, long long chunk) {
  __shared__ float4 red[DG][NT];
  const int r = threadIdx.x % rpad, lrow = threadIdx.x / rpad, rper = NT / rpad;
  const int i0 = blockIdx.y * DG, ng = min(DG, nvec - i0);
  const long long lo = blockIdx.x * chunk, hi = lo + chunk < rows ? lo + chunk : rows;
  cacc acc[DG];
  if (r < nrhs) {
    for (long long row = lo + lrow; row < hi; row += rper) {
      const long long l = row * nrhs + r;
      const float4 wv = w[l];
#pragma unroll
      for (int g = 0; g < DG; ++g)
        if (g < ng) cdot2_conj(acc[g], V[(i0 + g) * vstride + l], wv);
    }
  }
#pragma unroll
  for (int g = 0; g < DG; ++g) red[g][threadIdx.x] = cfin(acc[g]);
  __syncthreads();
  for (int s2 = rper / 2; s2 > 0; s2 >>= 1) {
    if (lrow < s2) {
#pragma unroll
      for (int g = 0; g < DG; ++g) {
        if (g >= ng) break;
        cacc t;
        cadd2(t, red[g][threadIdx.x]);
        cadd2(t, red[g][threadIdx.x + s2 * rpad]);
        red[g][threadIdx.x] = cfin(t);
      }
    }
    __syncthreads();
  }
  if (lrow == 0 && r < nrhs)
    for (int g = 0; g < ng; ++g) partial[((long long)blockIdx.x * nvec + i0 + g) * nrhs + r] = red[g][r];
}

__global__ void df_bdot_final_kernel(const float4* __restrict__ partial, int nblk, int nvec, int nrhs,
                                     double2* __restrict__ out) {
  const int warp = (blockIdx.x * NT + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= nvec * nrhs) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = lane; b < nblk; b += 32) {
    const double2 v = to_d2(partial[(long long)b * nvec * nrhs + warp]);
    acc.x += v.x;
    acc.y += v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if (lane == 0) out[warp] = acc;
}

cudaError_t df_bdot(const float4* V, long long vstride, int nvec, const float4* w, long long rows, int nrhs,
                    float4* partial, double2* out, cudaStream_t s) {
  if (nrhs > NT || nvec <= 0) return cudaErrorInvalidValue;
  int rpad = 1;
  while (rpad < nrhs) rpad <<= 1;
  const int nblk = bdot_blocks(rows);
  const long long chunk = (rows + nblk - 1) / nblk;
  df_bdot_partial_kernel<<<dim3(nblk, (nvec + DG - 1) / DG), NT, 0, s>>>(V, vstride, nvec, w, rows, nrhs, rpad,
                                                                         partial, chunk);
  note_launch();
  df_bdot_final_kernel<<<(nvec * nrhs * 32 + NT - 1) / NT, NT, 0, s>>>(partial, nblk, nvec, nrhs, out);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Two-pass Gram-Schmidt step (one reduction, one update per Arnoldi step).
//
// df_dots2: D[2i] = sum conj(X_i) y0, D[2i+1] = sum conj(X_i) y1 (i < nvec, X_i = V + i*vstride)
// and D[2 nvec] = sum conj(y1) y1, over rows, per right-hand side, FP64 result [2 nvec + 1][nrhs].
// Groups of DG2 vectors per block (blockIdx.y); y0 and y1 are read once per group.
// The y0 products (the tentative vector: the second Gram-Schmidt pass and its norm) are
// accumulated in double-float; the y1 products (the new Krylov vector: first-pass
// coefficients and its norm, whose errors the next step's second pass removes) in FP32 on the
// leading parts.
constexpr int DG2 = 8, NT2 = 128;
__global__ void __launch_bounds__(NT2, 3) df_dots2_partial_kernel(const float4* __restrict__ V, long long vstride,
                                                               int nvec, const float4* __restrict__ y0,
                                                               const float4* __restrict__ y1, long long rows,
                                                               int nrhs, int rpad, float4* __restrict__ partial,
                                                               long long chunk) {
  __shared__ float4 red[2 * DG2 + 1][NT2];
  const int r = threadIdx.x % rpad, lrow = threadIdx.x / rpad, rper = NT2 / rpad;
  const int i0 = blockIdx.y * DG2, ng = min(DG2, nvec - i0);
  const bool extra = blockIdx.y == 0;
  const int nout = 2 * nvec + 1;
  const long long lo = blockIdx.x * chunk, hi = lo + chunk < rows ? lo + chunk : rows;
  cacc a0[DG2];
  float2 a1[DG2];
  float ee = 0.f;
#pragma unroll
  for (int g = 0; g < DG2; ++g) a1[g] = make_float2(0.f, 0.f);
  if (r < nrhs) {
    // the next row's values are loaded while the current row is accumulated
    float4 u0, u1, x[DG2], nu0, nu1, nx[DG2];
    auto load = [&](long long row, float4& v0, float4& v1, float4 (&xv)[DG2]) {
      const long long l = row * nrhs + r;
      v0 = y0[l];
      v1 = y1[l];
#pragma unroll
      for (int g = 0; g < DG2; ++g)
        if (g < ng) xv[g] = V[(i0 + g) * vstride + l];
    };
    long long row = lo + lrow;
    if (row < hi) load(row, u0, u1, x);
    for (; row < hi; row += rper) {
      const long long nrow = row + rper;
      if (nrow < hi) load(nrow, nu0, nu1, nx);
      if (extra) ee = fmaf(u1.x, u1.x, fmaf(u1.y, u1.y, ee));
#pragma unroll
      for (int g = 0; g < DG2; ++g) {
        if (g < ng) {
          cdot2_conj(a0[g], x[g], u0);
          a1[g].x = fmaf(x[g].x, u1.x, fmaf(x[g].y, u1.y, a1[g].x));  // conj(x) u1, leading parts
          a1[g].y = fmaf(x[g].x, u1.y, fmaf(-x[g].y, u1.x, a1[g].y));
        }
      }
      u0 = nu0;
      u1 = nu1;
#pragma unroll
      for (int g = 0; g < DG2; ++g) x[g] = nx[g];
    }
  }
#pragma unroll
  for (int g = 0; g < DG2; ++g) {
    red[2 * g][threadIdx.x] = cfin(a0[g]);
    red[2 * g + 1][threadIdx.x] = make_float4(a1[g].x, a1[g].y, 0.f, 0.f);
  }
  red[2 * DG2][threadIdx.x] = make_float4(ee, 0.f, 0.f, 0.f);
  __syncthreads();
  for (int s2 = rper / 2; s2 > 0; s2 >>= 1) {
    if (lrow < s2) {
      for (int k = 0; k < 2 * DG2 + 1; ++k) {
        if (k < 2 * DG2 && k / 2 >= ng) continue;
        if (k == 2 * DG2 && !extra) continue;
        cacc t;
        cadd2(t, red[k][threadIdx.x]);
        cadd2(t, red[k][threadIdx.x + s2 * rpad]);
        red[k][threadIdx.x] = cfin(t);
      }
    }
    __syncthreads();
  }
  if (lrow == 0 && r < nrhs) {
    float4* P = partial + (long long)blockIdx.x * nout * nrhs;
    for (int g = 0; g < ng; ++g) {
      P[(2 * (i0 + g)) * nrhs + r] = red[2 * g][r];
      P[(2 * (i0 + g) + 1) * nrhs + r] = red[2 * g + 1][r];
    }
    if (extra) P[(2 * nvec) * nrhs + r] = red[2 * DG2][r];
  }
}

// at most bdot_blocks(rows) (the partial buffers are sized by it) and at most one full wave, so
// that the vector groups (blockIdx.y) run in whole waves
int df_dots2_blocks(long long rows) {
  const int b = bdot_blocks(rows), w = full_wave(df_dots2_partial_kernel, NT2, 0);
  return w > 0 && w < b ? w : b;
}

cudaError_t df_dots2(const float4* V, long long vstride, int nvec, const float4* y0, const float4* y1, long long rows,
                     int nrhs, float4* partial, double2* out, cudaStream_t s) {
  if (nrhs > NT2 / 2 || nvec <= 0) return cudaErrorInvalidValue;
  int rpad = 1;
  while (rpad < nrhs) rpad <<= 1;
  const int nblk = df_dots2_blocks(rows);
  const long long chunk = (rows + nblk - 1) / nblk;
  df_dots2_partial_kernel<<<dim3(nblk, (nvec + DG2 - 1) / DG2), NT2, 0, s>>>(V, vstride, nvec, y0, y1, rows, nrhs,
                                                                             rpad, partial, chunk);
  note_launch();
  const int nout = 2 * nvec + 1;
  df_bdot_final_kernel<<<(nout * nrhs * 32 + NT - 1) / NT, NT, 0, s>>>(partial, nblk, nout, nrhs, out);
  note_launch();
  return cudaGetLastError();
}

// df_update2: out_v = sv vt + sum_{i<nvec} ca_i V_i  and  out_w = sw w + svw vt + sum_{i<nvec} cb_i V_i
// (the ca products in FP32: they are second-pass corrections of the first pass's error size),
// coefficients df64 in global memory [2 nvec + 3][nrhs]: ca (nvec rows), cb (nvec rows), sv, sw, svw.
// out_v may be vt itself (each element is read before it is written, by the same thread).
__global__ void df_update2_kernel(const float4* __restrict__ V, long long vstride, int nvec, const float4* vt,
                                  const float4* __restrict__ w, const float4* __restrict__ coef, float4* out_v,
                                  float4* __restrict__ out_w, long long rows, int nrhs) {
  const long long tot = rows * nrhs;
  const float4* ca = coef;
  const float4* cb = coef + (long long)nvec * nrhs;
  const float4* sc = coef + 2LL * nvec * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const int r = (int)(l % nrhs);
    const float4 x = vt[l], y = w[l];
    cacc av, aw;
    cdot2(av, __ldg(sc + r), x);
    cdot2(aw, __ldg(sc + nrhs + r), y);
    cdot2(aw, __ldg(sc + 2 * nrhs + r), x);
    // the second-pass coefficients ca are of the size of the first pass's error, so their
    // products need only FP32 (leading parts): the sum enters the double-float result once
    float2 pv = make_float2(0.f, 0.f);
    for (int i = 0; i < nvec; ++i) {
      const float4 v = V[i * vstride + l];
      const float4 a = __ldg(ca + (long long)i * nrhs + r);
      pv.x = fmaf(a.x, v.x, fmaf(-a.y, v.y, pv.x));
      pv.y = fmaf(a.x, v.y, fmaf(a.y, v.x, pv.y));
      cdot2(aw, __ldg(cb + (long long)i * nrhs + r), v);
    }
    cadd2(av, make_float4(pv.x, pv.y, 0.f, 0.f));
    out_v[l] = cfin(av);
    out_w[l] = cfin(aw);
  }
}

cudaError_t df_update2(const float4* V, long long vstride, int nvec, const float4* vt, const float4* w,
                       const float4* coef, float4* out_v, float4* out_w, long long rows, int nrhs, cudaStream_t s) {
  // grid-stride over the elements with one full wave of blocks
  const int wave = full_wave(df_update2_kernel, NT, 0);
  df_update2_kernel<<<nblocks(rows * nrhs, wave > 0 ? wave : 4096), NT, 0, s>>>(V, vstride, nvec, vt, w, coef, out_v,
                                                                                 out_w, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

// w += sign * sum_i V_i h_i   (V df64 or FP32, h FP64 converted to df64 once per block)
template <typename VT>
__global__ void df_bupdate_kernel(float4* __restrict__ w, const VT* __restrict__ V, long long vstride, int nvec,
                                  const double2* __restrict__ h, long long rows, int nrhs, float sign) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* hs = reinterpret_cast<float4*>(smem_raw);  // [nvec][nrhs]
  for (int l = threadIdx.x; l < nvec * nrhs; l += NT) {
    const double2 v = h[l];
    hs[l] = from_d2(make_double2(sign * v.x, sign * v.y));
  }
  __syncthreads();
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const int r = (int)(l % nrhs);
    cacc acc;
    cadd2(acc, w[l]);
    for (int i = 0; i < nvec; ++i) cdot2(acc, ld(V, i * vstride + l), hs[i * nrhs + r]);
    w[l] = cfin(acc);
  }
}
template <typename VT>
cudaError_t df_bupdate(float4* w, const VT* V, long long vstride, int nvec, const double2* h, long long rows, int nrhs,
                       float sign, cudaStream_t s) {
  if (nvec <= 0) return cudaSuccess;
  const size_t smem = sizeof(float4) * (size_t)nvec * nrhs;
  df_bupdate_kernel<VT><<<nblocks(rows * nrhs, 4096), NT, smem, s>>>(w, V, vstride, nvec, h, rows, nrhs, sign);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t df_bupdate<float4>(float4*, const float4*, long long, int, const double2*, long long, int, float,
                                        cudaStream_t);
template cudaError_t df_bupdate<float2>(float4*, const float2*, long long, int, const double2*, long long, int, float,
                                        cudaStream_t);

// out = w * (1 / sqrt(re dots[r])) when that norm exceeds floor[r], else 0 (norm and inverse in FP64)
__global__ void df_bscale_kernel(float4* __restrict__ out, const float4* __restrict__ w,
                                 const double2* __restrict__ dots, const double* __restrict__ floor, long long rows,
                                 int nrhs) {
  __shared__ float4 inv[NT];
  for (int r = threadIdx.x; r < nrhs; r += NT) {
    const double nrm = sqrt(dots[r].x > 0.0 ? dots[r].x : 0.0);
    const double iv = nrm > (floor ? floor[r] : 0.0) ? 1.0 / nrm : 0.0;
    inv[r] = from_d2(make_double2(iv, 0.0));
  }
  __syncthreads();
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const float4 a = w[l], s = inv[(int)(l % nrhs)];
    cacc acc;
    dot2(acc.rs, acc.rc, a.x, a.z, s.x, s.z);
    dot2(acc.is, acc.ic, a.y, a.w, s.x, s.z);
    out[l] = cfin(acc);
  }
}
cudaError_t df_bscale(float4* out, const float4* w, const double2* dots, const double* floor, long long rows, int nrhs,
                      cudaStream_t s) {
  df_bscale_kernel<<<nblocks(rows * nrhs, 8192), NT, 0, s>>>(out, w, dots, floor, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

// z[p] = v[nb(p)] (identity preconditioner in incoming coordinates), FP32 hi parts
__global__ void df_swap_hi_kernel(float2* __restrict__ z, const float4* __restrict__ v, const int* __restrict__ nbr,
                                  long long rows, int nrhs) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const long long row = l / nrhs;
    const int r = (int)(l % nrhs);
    const int m = nbr[row];
    const float4 a = m >= 0 ? v[(long long)m * nrhs + r] : make_float4(0.f, 0.f, 0.f, 0.f);
    z[l] = make_float2(a.x, a.y);
  }
}
cudaError_t df_swap_hi(float2* z, const float4* v, const int* nbr, long long rows, int nrhs, cudaStream_t s) {
  df_swap_hi_kernel<<<nblocks(rows * nrhs, 8192), NT, 0, s>>>(z, v, nbr, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

void optin_df64() {
  smem_optin(df_matvec_kernel<float2>);
  smem_optin(df_matvec_kernel<float4>);
  smem_optin(df_bupdate_kernel<float4>);
  smem_optin(df_bupdate_kernel<float2>);
}

}  // namespace hps
