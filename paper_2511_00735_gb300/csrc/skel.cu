// Skeleton-level kernels (section 3.2): the FP64 matvec with M = I + Pi T in
// element-side layout, RHS assembly from boundary data, layout gathers and
// scatters (with precision conversion), the coarse-level operator of the
// multigrid hierarchy (section 4.3), and block-vector Krylov primitives.
//
// Layouts.  A block vector holds `nrhs` columns, stored row-major
// [rows][nrhs] (right-hand side fastest).  Element-side ("ES") rows are
// p = (e*4 + side)*q + k.  Residual-like vectors are kept in "outgoing"
// coordinates rho_p = r_{pi(p)} (the equation owned by the outgoing relation
// on side p) and solution-like vectors in "incoming" coordinates, so that
// the outer matvec reads  (Pi M g)_p = g_{nb(p)} + (T_e g_e)_p  per element.
#include "common.cuh"
#include "skel.cuh"

namespace hps {

namespace {
constexpr int NT = 256;

inline int nblocks(long long work, int per = NT, int cap = 1 << 20) {
  long long b = (work + per - 1) / per;
  if (b < 1) b = 1;
  return (int)(b > cap ? cap : b);
}
}  // namespace

// ---------------------------------------------------------------------------
// Outer matvec:  y_p = [ x_{nb(p)} + sum_b T_e[a][b] x_{e,b} ]  (nb(p) >= 0), 0 otherwise;
// with c0 != null: y = c0 - that  (residual form).
// One block per element, x_e staged in shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) es_matvec_kernel(const double2* __restrict__ T, const int* __restrict__ nbr,
                                                       const double2* __restrict__ x, const double2* __restrict__ c0,
                                                       double2* __restrict__ y, int E, int nb, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* xs = reinterpret_cast<double2*>(smem_raw);  // [nb][nrhs]
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();
    const long long base = (long long)e * nb;
    for (int l = threadIdx.x; l < nb * nrhs; l += NT) xs[l] = x[base * nrhs + l];
    __syncthreads();
    const double2* Te = T + (long long)e * nb * nb;
    for (int l = threadIdx.x; l < nb * nrhs; l += NT) {
      const int a = l / nrhs, r = l % nrhs;
      const long long p = base + a;
      const int q = nbr[p];
      double2 out = make_double2(0.0, 0.0);
      if (q >= 0) {
        double2 acc = x[(long long)q * nrhs + r];
        const double2* Tr = Te + (long long)a * nb;
        for (int b = 0; b < nb; ++b) cfma(acc, Tr[b], xs[b * nrhs + r]);
        out = acc;
        if (c0) out = csub(c0[p * nrhs + r], acc);
      } else if (c0) {
        out = make_double2(0.0, 0.0);
      }
      y[p * nrhs + r] = out;
    }
  }
}

cudaError_t es_matvec(const double2* T, const int* nbr, const double2* x, const double2* c0, double2* y, int E,
                      int nb, int nrhs, int grid, cudaStream_t s) {
  const size_t smem = sizeof(double2) * (size_t)nb * nrhs;
  es_matvec_kernel<<<grid, NT, smem, s>>>(T, nbr, x, c0, y, E, nb, nrhs);
  note_launch();
  return cudaGetLastError();
}

void optin_skel() { smem_optin(es_matvec_kernel); }

// ---------------------------------------------------------------------------
// RHS in outgoing coordinates: rho_p = -sum_{b on the boundary} T_e[a][b] t_{bdry(e,b)}
// for interior p (nb(p) >= 0), 0 otherwise.  t is [n_bdry][nrhs].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) es_rhs_kernel(const double2* __restrict__ T, const int* __restrict__ nbr,
                                                    const int* __restrict__ bdry, const double2* __restrict__ t,
                                                    double2* __restrict__ rho, int E, int nb, int nrhs) {
  for (int e = blockIdx.x; e < E; e += gridDim.x) {
    const long long base = (long long)e * nb;
    const double2* Te = T + (long long)e * nb * nb;
    // elements without a side on the physical boundary contribute nothing (most of them)
    int mine = 0;
    for (int b = threadIdx.x; b < nb; b += NT) mine |= bdry[base + b] >= 0;
    const bool touches = __syncthreads_or(mine) != 0;
    for (int l = threadIdx.x; l < nb * nrhs; l += NT) {
      const int a = l / nrhs, r = l % nrhs;
      const long long p = base + a;
      double2 acc = make_double2(0.0, 0.0);
      if (touches && nbr[p] >= 0) {
        for (int b = 0; b < nb; ++b) {
          const int bi = bdry[base + b];
          if (bi >= 0) cfma(acc, Te[(long long)a * nb + b], t[(long long)bi * nrhs + r]);
        }
      }
      rho[p * nrhs + r] = make_double2(-acc.x, -acc.y);
    }
  }
}

cudaError_t es_rhs(const double2* T, const int* nbr, const int* bdry, const double2* t, double2* rho, int E, int nb,
                   int nrhs, int grid, cudaStream_t s) {
  es_rhs_kernel<<<grid, NT, 0, s>>>(T, nbr, bdry, t, rho, E, nb, nrhs);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layout changes.
// ---------------------------------------------------------------------------
// Gathers and scatters take GU elements per thread per pass (indices, then loads, then stores,
// each GU independent), so a thread has GU dependent map -> data chains in flight.
constexpr int GU = 4;

template <typename RS, typename RD>
__global__ void gather_rows_kernel(c_t<RD>* __restrict__ dst, const c_t<RS>* __restrict__ src, const int* __restrict__ map,
                                   long long rows, int nrhs) {
  const long long tot = rows * nrhs, stride = (long long)gridDim.x * NT;
  for (long long l0 = blockIdx.x * (long long)NT + threadIdx.x; l0 < tot; l0 += GU * stride) {
    int m[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      m[u] = l < tot ? map[l / nrhs] : -1;
    }
    c_t<RD> v[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      v[u] = m[u] >= 0 ? cvt<RD, RS>(src[(long long)m[u] * nrhs + l % nrhs]) : czero<RD>();
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      if (l < tot) dst[l] = v[u];
    }
  }
}

template <typename RS, typename RD>
__global__ void scatter_rows_kernel(c_t<RD>* __restrict__ dst, const c_t<RS>* __restrict__ src, const int* __restrict__ map,
                                    long long rows, int nrhs) {
  const long long tot = rows * nrhs, stride = (long long)gridDim.x * NT;
  for (long long l0 = blockIdx.x * (long long)NT + threadIdx.x; l0 < tot; l0 += GU * stride) {
    int m[GU];
    c_t<RS> v[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      m[u] = l < tot ? map[l / nrhs] : -1;
      v[u] = l < tot ? src[l] : czero<RS>();
    }
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const long long l = l0 + u * stride;
      if (m[u] >= 0) dst[(long long)m[u] * nrhs + l % nrhs] = cvt<RD, RS>(v[u]);
    }
  }
}

template <typename RS, typename RD>
cudaError_t gather_rows(c_t<RD>* dst, const c_t<RS>* src, const int* map, long long rows, int nrhs, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  gather_rows_kernel<RS, RD><<<nblocks(rows * nrhs, NT * GU, 8192), NT, 0, s>>>(dst, src, map, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}
template <typename RS, typename RD>
cudaError_t scatter_rows(c_t<RD>* dst, const c_t<RS>* src, const int* map, long long rows, int nrhs, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  scatter_rows_kernel<RS, RD><<<nblocks(rows * nrhs, NT * GU, 8192), NT, 0, s>>>(dst, src, map, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

// user [nrhs][n] <-> rows [rows][nrhs] through map (row -> index in n, -1 = none)
__global__ void user_to_rows_kernel(double2* __restrict__ dst, const double2* __restrict__ src, const int* __restrict__ map,
                                    long long rows, int nrhs, long long n) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const long long row = l / nrhs;
    const int r = (int)(l % nrhs);
    const int m = map ? map[row] : (int)row;
    dst[l] = m >= 0 ? src[(long long)r * n + m] : make_double2(0.0, 0.0);
  }
}
__global__ void rows_to_user_kernel(double2* __restrict__ dst, const double2* __restrict__ src, const int* __restrict__ map,
                                    long long rows, int nrhs, long long n) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const long long row = l / nrhs;
    const int r = (int)(l % nrhs);
    const int m = map ? map[row] : (int)row;
    if (m >= 0) dst[(long long)r * n + m] = src[l];
  }
}
cudaError_t user_to_rows(double2* dst, const double2* src, const int* map, long long rows, int nrhs, long long n,
                         cudaStream_t s) {
  user_to_rows_kernel<<<nblocks(rows * nrhs, NT, 8192), NT, 0, s>>>(dst, src, map, rows, nrhs, n);
  note_launch();
  return cudaGetLastError();
}
cudaError_t rows_to_user(double2* dst, const double2* src, const int* map, long long rows, int nrhs, long long n,
                         cudaStream_t s) {
  rows_to_user_kernel<<<nblocks(rows * nrhs, NT, 8192), NT, 0, s>>>(dst, src, map, rows, nrhs, n);
  note_launch();
  return cudaGetLastError();
}

// dst[s][i][j] = src[s][map[s*n+i]][map[s*n+j]] (n x n blocks), with conversion.
template <typename RS, typename RD>
__global__ void permute_blocks_kernel(c_t<RD>* __restrict__ dst, const c_t<RS>* __restrict__ src, const int* __restrict__ map,
                                      int nsub, int n) {
  const long long tot = (long long)nsub * n * n;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const long long s = l / ((long long)n * n);
    const int rem = (int)(l % ((long long)n * n));
    const int i = rem / n, j = rem % n;
    const int si = map[s * n + i], sj = map[s * n + j];
    dst[l] = cvt<RD, RS>(src[(s * n + si) * (long long)n + sj]);
  }
}
template <typename RS, typename RD>
cudaError_t permute_blocks(c_t<RD>* dst, const c_t<RS>* src, const int* map, int nsub, int n, cudaStream_t s) {
  permute_blocks_kernel<RS, RD><<<nblocks((long long)nsub * n * n, NT, 16384), NT, 0, s>>>(dst, src, map, nsub, n);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coarse level (the T_c g products run as batched GEMMs on interior-first storage).
// ---------------------------------------------------------------------------
// out_p = nb(p) >= 0 ? (a ? a_p : 0) + b_{nb(p)} : 0
template <typename R>
__global__ void swap_add_kernel(c_t<R>* __restrict__ out, const c_t<R>* __restrict__ a, const c_t<R>* __restrict__ b,
                                const int* __restrict__ nbr, long long rows, int nrhs) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const long long row = l / nrhs;
    const int r = (int)(l % nrhs);
    const int m = nbr[row];
    c_t<R> v = czero<R>();
    if (m >= 0) {
      v = b[(long long)m * nrhs + r];
      if (a) v = cadd(v, a[l]);
    }
    out[l] = v;
  }
}
template <typename R>
cudaError_t swap_add(c_t<R>* out, const c_t<R>* a, const c_t<R>* b, const int* nbr, long long rows, int nrhs,
                     cudaStream_t s) {
  swap_add_kernel<R><<<nblocks(rows * nrhs, NT, 8192), NT, 0, s>>>(out, a, b, nbr, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void stage_residual_kernel(c_t<R>* __restrict__ out, const c_t<R>* __restrict__ r,
                                      const c_t<R>* __restrict__ e, const c_t<R>* __restrict__ w,
                                      const int* __restrict__ nbr, long long rows, int nrhs) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const int m = nbr[l / nrhs];
    c_t<R> v = czero<R>();
    if (m >= 0) v = csub(r[l], cadd(e[(long long)m * nrhs + (l % nrhs)], w[l]));
    out[l] = v;
  }
}
template <typename R>
cudaError_t stage_residual(c_t<R>* out, const c_t<R>* r, const c_t<R>* e, const c_t<R>* w, const int* nbr,
                           long long rows, int nrhs, cudaStream_t s) {
  stage_residual_kernel<R><<<nblocks(rows * nrhs, NT, 8192), NT, 0, s>>>(out, r, e, w, nbr, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void accumulate_kernel(c_t<R>* __restrict__ acc, const c_t<R>* __restrict__ x, long long n, int first,
                                  c_t<R>* __restrict__ out) {
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < n; l += (long long)gridDim.x * NT) {
    const c_t<R> v = first ? x[l] : cadd(acc[l], x[l]);
    acc[l] = v;
    if (out) out[l] = v;
  }
}
template <typename R>
cudaError_t accumulate(c_t<R>* acc, const c_t<R>* x, long long n, bool first, c_t<R>* out, cudaStream_t s) {
  accumulate_kernel<R><<<nblocks(n, NT, 8192), NT, 0, s>>>(acc, x, n, first ? 1 : 0, out);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Block-vector Krylov primitives.  V holds nvec vectors of `rows` rows, vector
// i at V + i*vstride.  Reductions are two-pass and deterministic.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(NT) bdot_partial_kernel(const c_t<R>* __restrict__ V, long long vstride, int nvec,
                                                          const c_t<R>* __restrict__ w, long long rows, int nrhs,
                                                          int rpad, c_t<R>* __restrict__ partial, long long chunk) {
  __shared__ c_t<R> red[NT];
  const int r = threadIdx.x % rpad, lrow = threadIdx.x / rpad, rper = NT / rpad;
  const long long lo = blockIdx.x * chunk, hi = lo + chunk < rows ? lo + chunk : rows;
  for (int i = 0; i < nvec; ++i) {
    c_t<R> acc = czero<R>();
    if (r < nrhs) {
      const c_t<R>* Vi = V + i * vstride;
      for (long long row = lo + lrow; row < hi; row += rper)
        cfma_conj(acc, Vi[row * nrhs + r], w[row * nrhs + r]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s2 = rper / 2; s2 > 0; s2 >>= 1) {
      if (lrow < s2) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s2 * rpad]);
      __syncthreads();
    }
    if (lrow == 0 && r < nrhs) partial[((long long)blockIdx.x * nvec + i) * nrhs + r] = red[r];
    __syncthreads();
  }
}

template <typename R>
__global__ void bdot_final_kernel(const c_t<R>* __restrict__ partial, int nblk, int nvec, int nrhs,
                                  c_t<R>* __restrict__ out, int accumulate) {
  // one warp per output: lanes stride over the block partials, fixed-order butterfly sum
  const int warp = (blockIdx.x * NT + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= nvec * nrhs) return;
  c_t<R> acc = czero<R>();
  for (int b = lane; b < nblk; b += 32) acc = cadd(acc, partial[(long long)b * nvec * nrhs + warp]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if (lane == 0) out[warp] = accumulate ? cadd(out[warp], acc) : acc;
}

int bdot_blocks(long long rows) {
  long long b = (rows + 63) / 64;
  if (b < 1) b = 1;
  return (int)(b > 512 ? 512 : b);
}

template <typename R>
cudaError_t bdot(const c_t<R>* V, long long vstride, int nvec, const c_t<R>* w, long long rows, int nrhs,
                 c_t<R>* partial, c_t<R>* out, int accumulate, cudaStream_t s) {
  if (nrhs > NT || nvec <= 0) return cudaErrorInvalidValue;
  int rpad = 1;
  while (rpad < nrhs) rpad <<= 1;
  const int nblk = bdot_blocks(rows);
  const long long chunk = (rows + nblk - 1) / nblk;
  bdot_partial_kernel<R><<<nblk, NT, 0, s>>>(V, vstride, nvec, w, rows, nrhs, rpad, partial, chunk);
  note_launch();
  bdot_final_kernel<R><<<(nvec * nrhs * 32 + NT - 1) / NT, NT, 0, s>>>(partial, nblk, nvec, nrhs, out, accumulate);
  note_launch();
  return cudaGetLastError();
}

// w += sign * sum_i V_i h_i   (h: [nvec][nrhs])
template <typename R, typename RH>
__global__ void bupdate_kernel(c_t<R>* __restrict__ w, const c_t<R>* __restrict__ V, long long vstride, int nvec,
                               const c_t<RH>* __restrict__ h, long long rows, int nrhs, R sign) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const int r = (int)(l % nrhs);
    c_t<R> acc = czero<R>();
    for (int i = 0; i < nvec; ++i) cfma(acc, V[i * vstride + l], cvt<R, RH>(h[i * nrhs + r]));
    w[l] = cadd(w[l], cscale(acc, sign));
  }
}
template <typename R, typename RH>
cudaError_t bupdate(c_t<R>* w, const c_t<R>* V, long long vstride, int nvec, const c_t<RH>* h, long long rows, int nrhs,
                    R sign, cudaStream_t s) {
  if (nvec <= 0) return cudaSuccess;
  bupdate_kernel<R, RH><<<nblocks(rows * nrhs, NT, 8192), NT, 0, s>>>(w, V, vstride, nvec, h, rows, nrhs, sign);
  note_launch();
  return cudaGetLastError();
}

// out = w / nrm[r] where nrm[r] = sqrt(re dots[r]) > floor[r] (floor may be null), else 0;
// also stores nrm into nrm_out when non-null.
template <typename R>
__global__ void bscale_kernel(c_t<R>* __restrict__ out, const c_t<R>* __restrict__ w, const c_t<R>* __restrict__ dots,
                              const R* __restrict__ floor, long long rows, int nrhs) {
  __shared__ R inv[NT];
  for (int r = threadIdx.x; r < nrhs; r += NT) {
    const R nrm = sqrt(dots[r].x > R(0) ? dots[r].x : R(0));
    inv[r] = nrm > (floor ? floor[r] : R(0)) ? R(1) / nrm : R(0);
  }
  __syncthreads();
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT)
    out[l] = cscale(w[l], inv[(int)(l % nrhs)]);
}
template <typename R>
cudaError_t bscale(c_t<R>* out, const c_t<R>* w, const c_t<R>* dots, const R* floor, long long rows, int nrhs,
                   cudaStream_t s) {
  bscale_kernel<R><<<nblocks(rows * nrhs, NT, 8192), NT, 0, s>>>(out, w, dots, floor, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coarse GMRES bookkeeping on the device (one thread per right-hand side).
// ---------------------------------------------------------------------------
// H[r][i][j] (ldh = k+1 rows, column j): store column j = h1 + h2 (i <= j) and
// the subdiagonal sqrt(re nrm2); beta[r] from the first norm.
template <typename R>
__global__ void hstore_kernel(c_t<R>* __restrict__ H, const c_t<R>* __restrict__ h1, const c_t<R>* __restrict__ h2,
                              const c_t<R>* __restrict__ nrm2, int j, int k, int nrhs) {
  const int r = blockIdx.x * NT + threadIdx.x;
  if (r >= nrhs) return;
  c_t<R>* Hr = H + (long long)r * (k + 1) * k;
  for (int i = 0; i <= j; ++i) Hr[i * k + j] = cadd(h1[i * nrhs + r], h2[i * nrhs + r]);
  const R nn = nrm2[r].x > R(0) ? sqrt(nrm2[r].x) : R(0);
  Hr[(j + 1) * k + j] = mk<R>(nn, R(0));
}
template <typename R>
cudaError_t hstore(c_t<R>* H, const c_t<R>* h1, const c_t<R>* h2, const c_t<R>* nrm2, int j, int k, int nrhs,
                   cudaStream_t s) {
  hstore_kernel<R><<<(nrhs + NT - 1) / NT, NT, 0, s>>>(H, h1, h2, nrm2, j, k, nrhs);
  note_launch();
  return cudaGetLastError();
}

// beta[r] = sqrt(re nrm2[r]); floor[r] = tol * beta[r]
template <typename R>
__global__ void beta_kernel(R* __restrict__ beta, R* __restrict__ floor, const c_t<R>* __restrict__ nrm2, R tol, int nrhs) {
  const int r = blockIdx.x * NT + threadIdx.x;
  if (r >= nrhs) return;
  const R b = nrm2[r].x > R(0) ? sqrt(nrm2[r].x) : R(0);
  beta[r] = b;
  floor[r] = tol * b;
}
template <typename R>
cudaError_t beta_floor(R* beta, R* floor, const c_t<R>* nrm2, R tol, int nrhs, cudaStream_t s) {
  beta_kernel<R><<<(nrhs + NT - 1) / NT, NT, 0, s>>>(beta, floor, nrm2, tol, nrhs);
  note_launch();
  return cudaGetLastError();
}

// Least squares min || beta e1 - Hbar y || by complex Givens rotations
//   G = [[c, s], [-conj(s), c]],  c = |a| / nu,  s = (a / |a|) (b / nu),  nu = sqrt(|a|^2 + b^2),
// which maps (a, b) (b real >= 0, the Arnoldi subdiagonal) to (a nu / |a|, 0).
// Stops after the first column whose subdiagonal is <= floor[r] (happy breakdown).
// H: [nrhs][k+1][k]; y: [k][nrhs]; workspaces g [nrhs][k+1], cs [nrhs][k], sn [nrhs][k].
template <typename R>
__global__ void lsq_kernel(c_t<R>* __restrict__ H, const R* __restrict__ beta, const R* __restrict__ floor,
                           c_t<R>* __restrict__ y, c_t<R>* __restrict__ gws, R* __restrict__ cws,
                           c_t<R>* __restrict__ sws, int k, int nrhs) {
  const int r = blockIdx.x * NT + threadIdx.x;
  if (r >= nrhs) return;
  c_t<R>* Hr = H + (long long)r * (k + 1) * k;
  c_t<R>* g = gws + (long long)r * (k + 1);
  R* cr = cws + (long long)r * k;
  c_t<R>* sr = sws + (long long)r * k;
  for (int i = 0; i <= k; ++i) g[i] = czero<R>();
  g[0] = mk<R>(beta[r], R(0));
  int steps = k;
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < j; ++i) {
      const c_t<R> a = Hr[i * k + j], b = Hr[(i + 1) * k + j];
      Hr[i * k + j] = cadd(cscale(a, cr[i]), cmul(sr[i], b));
      Hr[(i + 1) * k + j] = csub(cscale(b, cr[i]), cmul(mk<R>(sr[i].x, -sr[i].y), a));
    }
    const c_t<R> a = Hr[j * k + j];
    const R b = Hr[(j + 1) * k + j].x;
    const R aa = sqrt(a.x * a.x + a.y * a.y);
    R c;
    c_t<R> sn;
    if (b == R(0)) {
      c = R(1);
      sn = czero<R>();
    } else if (aa == R(0)) {
      c = R(0);
      sn = mk<R>(R(1), R(0));
    } else {
      const R nu = sqrt(aa * aa + b * b);
      c = aa / nu;
      sn = mk<R>(a.x / aa * (b / nu), a.y / aa * (b / nu));
    }
    cr[j] = c;
    sr[j] = sn;
    Hr[j * k + j] = cadd(cscale(a, c), cscale(sn, b));
    Hr[(j + 1) * k + j] = czero<R>();
    const c_t<R> gj = g[j];
    g[j] = cscale(gj, c);
    g[j + 1] = cmul(mk<R>(-sn.x, sn.y), gj);  // -conj(s) g_j
    if (b <= floor[r]) {
      steps = j + 1;
      break;
    }
  }
  for (int j = steps - 1; j >= 0; --j) {
    c_t<R> v = g[j];
    for (int i = j + 1; i < steps; ++i) v = csub(v, cmul(Hr[j * k + i], y[i * nrhs + r]));
    y[j * nrhs + r] = cmul(v, cinv(Hr[j * k + j]));
  }
  for (int j = steps; j < k; ++j) y[j * nrhs + r] = czero<R>();
}
template <typename R>
cudaError_t lsq(c_t<R>* H, const R* beta, const R* floor, c_t<R>* y, c_t<R>* gws, R* cws, c_t<R>* sws, int k,
                int nrhs, cudaStream_t s) {
  lsq_kernel<R><<<(nrhs + NT - 1) / NT, NT, 0, s>>>(H, beta, floor, y, gws, cws, sws, k, nrhs);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused coarse-GMRES passes.  One thread per (row, right-hand side): thread (lrow, r) of a
// block takes row lo + lrow of the block's rper rows; every load of a pass is independent of
// the others (one memory round trip).  Block partials are reduced in two levels by the last
// block to arrive: the last block of each group of CG_GROUP blocks sums the group's partials
// in block order, the last group reducer sums the group sums in group order (deterministic).
// ---------------------------------------------------------------------------
constexpr int CG_GROUP = 16;

// one block per rper rows, at most two per SM: a block loops over rows gridDim.x * rper apart, so
// that the passes' two-level reductions handle a few hundred partials, not one per 8 rows
int cg_pass_blocks(long long rows, int nrhs) {
  int rpad = 1;
  while (rpad < nrhs) rpad <<= 1;
  const long long rper = NT / rpad;
  long long b = (rows + rper - 1) / rper;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    cudaGetLastError();  // unknown SM count: one block per rper rows
  else if (sms > 0 && b > 2LL * sms)
    b = 2LL * sms;
  return (int)(b < 1 ? 1 : b);
}

template <typename R, int MODE>
__global__ void __launch_bounds__(NT) cg_pass_kernel(CgPass<R> p, int rpad) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char cg_smem[];
  C* red = reinterpret_cast<C*>(cg_smem);  // [nvec][NT / 32][rpad]
  __shared__ int is_last;
  const int r = threadIdx.x % rpad, lrow = threadIdx.x / rpad, rper = NT / rpad;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nvec = (MODE == CG_START || MODE == CG_CLOSE) ? 1 : p.j + 1;  // dot products per column
  const int nupd = (MODE == CG_PROJECT || MODE == CG_CLOSE) ? p.j + 1 : 0;
  C acc[CG_KMAX];
#pragma unroll
  for (int i = 0; i < CG_KMAX; ++i) acc[i] = czero<R>();
  for (long long row = (long long)blockIdx.x * rper + lrow; r < p.nrhs && row < p.rows;
       row += (long long)gridDim.x * rper) {
    const long long l = row * p.nrhs + r;
    C x, vj = czero<R>();
    if (MODE == CG_START) {
      const int m = p.nb[row];
      x = (m >= 0 && m < p.rows) ? p.g[(long long)m * p.nrhs + r] : czero<R>();
    } else if (MODE == CG_APPLY) {
      const R sc = p.inv[r];
      const C wl = p.w[l];
      const int m = p.nb[row];
      vj = cscale(wl, sc);
      x = (m >= 0 && m < p.rows) ? cscale(cadd(wl, p.W[(long long)m * p.nrhs + r]), sc) : czero<R>();
      p.V[p.j * p.vs + l] = vj;
    } else {
      const C* hin = MODE == CG_PROJECT ? p.h1 : p.h2;
      C v[CG_KMAX], h[CG_KMAX];
#pragma unroll
      for (int i = 0; i < CG_KMAX; ++i)
        if (i < nupd) {
          v[i] = p.V[i * p.vs + l];
          h[i] = hin[i * p.nrhs + r];
        }
      x = p.w[l];
#pragma unroll
      for (int i = 0; i < CG_KMAX; ++i)
        if (i < nupd) cfms(x, v[i], h[i]);
      if (MODE == CG_PROJECT) {
#pragma unroll
        for (int i = 0; i < CG_KMAX; ++i)
          if (i < nvec) cfma_conj(acc[i], v[i], x);
      }
    }
    p.w[l] = x;
    if (MODE == CG_START || MODE == CG_CLOSE) {
      cfma_conj(acc[0], x, x);
    } else if (MODE == CG_APPLY) {
#pragma unroll
      for (int i = 0; i < CG_KMAX; ++i)
        if (i < nvec) cfma_conj(acc[i], i == p.j ? vj : p.V[i * p.vs + l], x);
    }
  }
  // block partials: lanes of one r within a warp by shuffles, then the warps in order
#pragma unroll
  for (int i = 0; i < CG_KMAX; ++i) {
    if (i >= nvec) break;
    C a = acc[i];
    for (int off = rpad; off < 32; off <<= 1) {
      a.x += __shfl_xor_sync(0xffffffffu, a.x, off);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, off);
    }
    if (lane < rpad) red[(i * (NT / 32) + warp) * rpad + lane] = a;
  }
  __syncthreads();
  const int nout = nvec * p.nrhs;
  const int nwr = (NT / 32) < (rper * rpad + 31) / 32 ? (NT / 32) : (rper * rpad + 31) / 32;  // warps holding rows
  for (int o = threadIdx.x; o < nout; o += NT) {
    const int i = o / p.nrhs, q = o % p.nrhs;
    C a = czero<R>();
    for (int w2 = 0; w2 < nwr; ++w2) a = cadd(a, red[(i * (NT / 32) + w2) * rpad + q]);
    p.part[(long long)blockIdx.x * nout + o] = a;
  }
  // level 1: the last block of this group sums the group's partials
  const int grp = blockIdx.x / CG_GROUP, ngrp = (gridDim.x + CG_GROUP - 1) / CG_GROUP;
  const int b0 = grp * CG_GROUP, b1 = min((int)gridDim.x, b0 + CG_GROUP);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(p.cnt + 1 + grp, 1u) == (unsigned)(b1 - b0 - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  C* gsum = p.part + (long long)gridDim.x * nout;
  for (int o = threadIdx.x; o < nout; o += NT) {
    C a = czero<R>();
    for (int b = b0; b < b1; ++b) a = cadd(a, __ldcg(&p.part[(long long)b * nout + o]));
    gsum[(long long)grp * nout + o] = a;
  }
  if (threadIdx.x == 0) p.cnt[1 + grp] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(p.cnt, 1u) == (unsigned)(ngrp - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // level 2: the last group reducer sums the groups and finishes the pass
  C* fin = red;  // nout <= CG_KMAX * rpad fits in the partial buffer
  for (int o = threadIdx.x; o < nout; o += NT) {
    C a = czero<R>();
    for (int g2 = 0; g2 < ngrp; ++g2) a = cadd(a, __ldcg(&gsum[(long long)g2 * nout + o]));
    if (MODE == CG_APPLY) p.h1[o] = a;
    else if (MODE == CG_PROJECT) p.h2[o] = a;
    fin[o] = a;
  }
  __syncthreads();
  if (MODE == CG_START) {
    for (int q = threadIdx.x; q < p.nrhs; q += NT) {
      const R b = fin[q].x > R(0) ? sqrt(fin[q].x) : R(0);
      p.beta[q] = b;
      p.floor[q] = p.tol * b;
      p.inv[q] = b > R(0) ? R(1) / b : R(0);
    }
  } else if (MODE == CG_CLOSE) {
    for (int q = threadIdx.x; q < p.nrhs; q += NT) {
      C* Hr = p.H + (long long)q * (p.k + 1) * p.k;
      for (int i = 0; i <= p.j; ++i) Hr[i * p.k + p.j] = cadd(p.h1[i * p.nrhs + q], p.h2[i * p.nrhs + q]);
      const R nn = fin[q].x > R(0) ? sqrt(fin[q].x) : R(0);
      Hr[(p.j + 1) * p.k + p.j] = mk<R>(nn, R(0));
      p.inv[q] = nn > p.floor[q] ? R(1) / nn : R(0);
    }
  }
  if (threadIdx.x == 0) p.cnt[0] = 0u;  // ready for the next pass
}

template <typename R>
bool cg_pass_fits(int k, int nrhs) {
  int rpad = 1;
  while (rpad < nrhs) rpad <<= 1;
  return nrhs > 0 && rpad <= 32 && k + 1 <= CG_KMAX &&
         (size_t)CG_KMAX * (NT / 32) * rpad * sizeof(c_t<R>) <= 48 * 1024;
}

template <typename R>
cudaError_t cg_pass(int mode, const CgPass<R>& p, cudaStream_t s) {
  if (!cg_pass_fits<R>(p.k, p.nrhs) || p.j > p.k || (mode == CG_CLOSE && p.j >= p.k)) return cudaErrorInvalidValue;
  int rpad = 1;
  while (rpad < p.nrhs) rpad <<= 1;
  const int nblk = cg_pass_blocks(p.rows, p.nrhs);
  const int nvec = (mode == CG_START || mode == CG_CLOSE) ? 1 : p.j + 1;
  if ((long long)(nblk + cg_groups(nblk)) * nvec * p.nrhs > p.part_cap || 1 + cg_groups(nblk) > p.cnt_cap)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)nvec * (NT / 32) * rpad * sizeof(c_t<R>);
  switch (mode) {
    case CG_START: cg_pass_kernel<R, CG_START><<<nblk, NT, smem, s>>>(p, rpad); break;
    case CG_APPLY: cg_pass_kernel<R, CG_APPLY><<<nblk, NT, smem, s>>>(p, rpad); break;
    case CG_PROJECT: cg_pass_kernel<R, CG_PROJECT><<<nblk, NT, smem, s>>>(p, rpad); break;
    case CG_CLOSE: cg_pass_kernel<R, CG_CLOSE><<<nblk, NT, smem, s>>>(p, rpad); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename R>
__global__ void bcombine_kernel(c_t<R>* __restrict__ x, const c_t<R>* __restrict__ V, long long vstride, int nvec,
                                const c_t<R>* __restrict__ y, long long rows, int nrhs) {
  const long long tot = rows * nrhs;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const int r = (int)(l % nrhs);
    c_t<R> acc = czero<R>();
    for (int i = 0; i < nvec; ++i) cfma(acc, V[i * vstride + l], y[i * nrhs + r]);
    x[l] = acc;
  }
}
template <typename R>
cudaError_t bcombine(c_t<R>* x, const c_t<R>* V, long long vstride, int nvec, const c_t<R>* y, long long rows, int nrhs,
                     cudaStream_t s) {
  bcombine_kernel<R><<<nblocks(rows * nrhs, NT, 8192), NT, 0, s>>>(x, V, vstride, nvec, y, rows, nrhs);
  note_launch();
  return cudaGetLastError();
}

// fill
template <typename R>
__global__ void zero_kernel(c_t<R>* __restrict__ x, long long n) {
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < n; l += (long long)gridDim.x * NT) x[l] = czero<R>();
}
template <typename R>
cudaError_t zero(c_t<R>* x, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zero_kernel<R><<<nblocks(n, NT, 8192), NT, 0, s>>>(x, n);
  note_launch();
  return cudaGetLastError();
}

// W = [I | I] for nmat matrices of m rows (leading dimension 2m)
template <typename R>
__global__ void eye2_kernel(c_t<R>* __restrict__ W, int m, int nmat) {
  const long long tot = (long long)nmat * m * 2 * m;
  for (long long l = blockIdx.x * (long long)NT + threadIdx.x; l < tot; l += (long long)gridDim.x * NT) {
    const int rem = (int)(l % (2LL * m * m));
    const int i = rem / (2 * m), j = rem % (2 * m);
    W[l] = mk<R>((j == i || j == i + m) ? R(1) : R(0), R(0));
  }
}
template <typename R>
cudaError_t eye2(c_t<R>* W, int m, int nmat, cudaStream_t s) {
  eye2_kernel<R><<<nblocks((long long)nmat * m * 2 * m, NT, 16384), NT, 0, s>>>(W, m, nmat);
  note_launch();
  return cudaGetLastError();
}

#define HPS_INST_R(R)                                                                                                   \
  template cudaError_t swap_add<R>(c_t<R>*, const c_t<R>*, const c_t<R>*, const int*, long long, int, cudaStream_t);   \
  template cudaError_t bdot<R>(const c_t<R>*, long long, int, const c_t<R>*, long long, int, c_t<R>*, c_t<R>*, int,     \
                               cudaStream_t);                                                                           \
  template cudaError_t bscale<R>(c_t<R>*, const c_t<R>*, const c_t<R>*, const R*, long long, int, cudaStream_t);       \
  template cudaError_t hstore<R>(c_t<R>*, const c_t<R>*, const c_t<R>*, const c_t<R>*, int, int, int, cudaStream_t);  \
  template cudaError_t beta_floor<R>(R*, R*, const c_t<R>*, R, int, cudaStream_t);                                      \
  template cudaError_t lsq<R>(c_t<R>*, const R*, const R*, c_t<R>*, c_t<R>*, R*, c_t<R>*, int, int,        \
                              cudaStream_t);                  \
  template cudaError_t zero<R>(c_t<R>*, long long, cudaStream_t);                                                       \
  template cudaError_t stage_residual<R>(c_t<R>*, const c_t<R>*, const c_t<R>*, const c_t<R>*, const int*, long long,  \
                                         int, cudaStream_t);                                                            \
  template cudaError_t accumulate<R>(c_t<R>*, const c_t<R>*, long long, bool, c_t<R>*, cudaStream_t);                                                       \
  template cudaError_t cg_pass<R>(int, const CgPass<R>&, cudaStream_t);                                                 \
  template bool cg_pass_fits<R>(int, int);                                                                               \
  template cudaError_t bcombine<R>(c_t<R>*, const c_t<R>*, long long, int, const c_t<R>*, long long, int, cudaStream_t); \
  template cudaError_t eye2<R>(c_t<R>*, int, int, cudaStream_t);

HPS_INST_R(double)
HPS_INST_R(float)

template cudaError_t bupdate<double, double>(double2*, const double2*, long long, int, const double2*, long long, int,
                                             double, cudaStream_t);
template cudaError_t bupdate<float, float>(float2*, const float2*, long long, int, const float2*, long long, int, float,
                                           cudaStream_t);
template cudaError_t gather_rows<double, double>(double2*, const double2*, const int*, long long, int, cudaStream_t);
template cudaError_t gather_rows<double, float>(float2*, const double2*, const int*, long long, int, cudaStream_t);
template cudaError_t gather_rows<float, float>(float2*, const float2*, const int*, long long, int, cudaStream_t);
template cudaError_t scatter_rows<double, double>(double2*, const double2*, const int*, long long, int, cudaStream_t);
template cudaError_t scatter_rows<float, double>(double2*, const float2*, const int*, long long, int, cudaStream_t);
template cudaError_t scatter_rows<float, float>(float2*, const float2*, const int*, long long, int, cudaStream_t);
template cudaError_t permute_blocks<double, double>(double2*, const double2*, const int*, int, int, cudaStream_t);
template cudaError_t permute_blocks<double, float>(float2*, const double2*, const int*, int, int, cudaStream_t);

}  // namespace hps
