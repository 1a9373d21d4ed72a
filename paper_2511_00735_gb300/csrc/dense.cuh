// Shared-memory dense helpers used by several kernels: block-wide pivot search
// and Gauss-Jordan inversion with partial pivoting (ties go to the lower row).
#pragma once

#include "common.cuh"

namespace hps {
namespace {

constexpr int DNT = 256;  // threads per block of every kernel that calls these

// Warp-wide argmax of (v, i): larger v wins, ties go to the lower index.
template <typename V>
__device__ __forceinline__ void warp_argmax(V& v, int& i) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    V ov = __shfl_down_sync(0xffffffffu, v, off);
    int oi = __shfl_down_sync(0xffffffffu, i, off);
    if (ov > v || (ov == v && oi >= 0 && (i < 0 || oi < i))) {
      v = ov;
      i = oi;
    }
  }
}

// Block-wide argmax over rows [lo, hi) of cabs1(S[row * ld + col]).  All threads
// must call it (any block size up to 1024); returns the winning row in every thread.
template <typename R>
__device__ int block_argmax_col(const c_t<R>* S, int ld, int col, int lo, int hi) {
  __shared__ R s_v[32];
  __shared__ int s_i[32];
  __shared__ int s_res;
  const int nw = (int)(blockDim.x / 32);
  R best = R(-1);
  int bi = -1;
  for (int r = lo + (int)threadIdx.x; r < hi; r += (int)blockDim.x) {
    const R v = cabs1(S[(long long)r * ld + col]);
    if (v > best) {
      best = v;
      bi = r;
    }
  }
  warp_argmax(best, bi);
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    s_v[w] = best;
    s_i[w] = bi;
  }
  __syncthreads();
  if (w == 0) {
    best = lane < nw ? s_v[lane] : R(-1);
    bi = lane < nw ? s_i[lane] : -1;
    warp_argmax(best, bi);
    if (lane == 0) s_res = bi;
  }
  __syncthreads();
  const int res = s_res;
  __syncthreads();
  return res;
}

// In-shared-memory Gauss-Jordan on W (n rows x ncols, leading dimension ld):
// partial pivoting on column k over rows k..n-1; after the loop the columns
// n..ncols-1 hold S^{-1} times the original right part.
template <typename R>
__device__ void gj_smem(c_t<R>* W, int n, int ld, int ncols, int* flag) {
  using C = c_t<R>;
  for (int k = 0; k < n; ++k) {
    const int p = block_argmax_col<R>(W, ld, k, k, n);
    if (p != k && p >= 0) {
      for (int j = k + threadIdx.x; j < ncols; j += DNT) {
        const C t = W[k * ld + j];
        W[k * ld + j] = W[p * ld + j];
        W[p * ld + j] = t;
      }
    }
    __syncthreads();
    const C piv = W[k * ld + k];
    if (threadIdx.x == 0 && piv.x == 0 && piv.y == 0 && flag) atomicExch(flag, 1);
    const C inv = cinv(piv);
    __syncthreads();
    for (int j = k + 1 + threadIdx.x; j < ncols; j += DNT) W[k * ld + j] = cmul(W[k * ld + j], inv);
    __syncthreads();
    const int w = ncols - k - 1;
    for (int l = threadIdx.x; l < n * w; l += DNT) {
      const int i = l / w, j = k + 1 + l % w;
      if (i == k) continue;
      const C f = W[i * ld + k];
      C v = W[i * ld + j];
      const C pk = W[k * ld + j];
      cfms(v, f, pk);
      W[i * ld + j] = v;
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace hps
