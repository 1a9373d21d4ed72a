// Shared device helpers: interleaved complex arithmetic in double / float,
// the batched-GEMM descriptor and launch declarations of every kernel family.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hps {

// Counts one kernel launch (total and per profiling phase of the calling context).
void note_launch(int n = 1);

// Raise a kernel's dynamic shared-memory limit once to the device's opt-in maximum
// (a per-launch value would race between host threads launching different sizes).
template <typename K>
inline void smem_optin(K kernel) {
  int dev = 0, mx = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) mx -= (int)fa.sharedSizeBytes;  // minus static smem
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaGetLastError();
}

// Raise the dynamic shared-memory limit of every kernel that needs more than 48 KB, once
// per device (called by hps_create and hps_leaf_maps_noalloc with the device current), so
// that no launch path calls cudaFuncSetAttribute while other host threads launch or capture.
void optin_all_once();
void optin_leaf();
void optin_blas();
void optin_df64();
void optin_skel();
void optin_volume();

template <typename R> struct cplx;
template <> struct cplx<double> { using T = double2; };
template <> struct cplx<float> { using T = float2; };
template <typename R> using c_t = typename cplx<R>::T;

template <typename R>
__host__ __device__ __forceinline__ c_t<R> mk(R a, R b) {
  c_t<R> z;
  z.x = a;
  z.y = b;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ c_t<R> czero() { return mk<R>(R(0), R(0)); }

template <typename T> __host__ __device__ __forceinline__ T cadd(T a, T b) {
  T z; z.x = a.x + b.x; z.y = a.y + b.y; return z;
}
template <typename T> __host__ __device__ __forceinline__ T csub(T a, T b) {
  T z; z.x = a.x - b.x; z.y = a.y - b.y; return z;
}
template <typename T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
  T z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cfma(T& acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b (four FMAs)
template <typename T> __host__ __device__ __forceinline__ void cfms(T& acc, T a, T b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename T> __host__ __device__ __forceinline__ void cfma_conj(T& acc, T a, T b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
template <typename T> __host__ __device__ __forceinline__ T cscale(T a, decltype(a.x) s) {
  T z; z.x = a.x * s; z.y = a.y * s; return z;
}
template <typename T> __host__ __device__ __forceinline__ decltype(T().x) cabs1(T a) {
  return fabs(a.x) + fabs(a.y);
}
// 1 / a, scaled to avoid overflow in |a|^2
template <typename T> __host__ __device__ __forceinline__ T cinv(T a) {
  auto s = fabs(a.x) > fabs(a.y) ? fabs(a.x) : fabs(a.y);
  T z;
  if (s == 0) { z.x = 0; z.y = 0; return z; }
  auto ar = a.x / s, ai = a.y / s;
  auto d = (ar * ar + ai * ai) * s;
  z.x = ar / d;
  z.y = -ai / d;
  return z;
}
template <typename D, typename S>
__host__ __device__ __forceinline__ c_t<D> cvt(c_t<S> a) {
  return mk<D>(D(a.x), D(a.y));
}

// One batched-GEMM problem: C(m x n) = beta * C0 + alpha * A(m x k) * B(k x n).
// Operand X starts at element (x_r * ldx + x_c) of its base pointer; all
// matrices are row-major complex.  rmap / cmap >= 0 give offsets into the
// launch's map array: row i of C is written to row c_r + map[rmap + i], column
// j to c_c + map[cmap + j].  n < 0 means "the launch's n" (number of RHS).
// Two-segment operands: when kb2 > 0, rows k >= kb2 of B come from row
// b_r2 + (k - kb2); when mc2 > 0, rows i >= mc2 of C0 come from row
// c0_r2 + (i - mc2) (used to read two merge children as one operand).
struct GemmDesc {
  int a_r, a_c, b_r, b_c, c0_r, c0_c, c_r, c_c;
  int m, n, k;
  int rmap, cmap;
  int b_r2, kb2, c0_r2, mc2;
};

template <typename R> struct GemmArgs {
  const c_t<R>* A;
  const c_t<R>* B;
  const c_t<R>* C0;  // may be null: no beta term
  c_t<R>* C;
  long long lda, ldb, ldc0, ldc;
  c_t<R> alpha, beta;
  const GemmDesc* desc;  // device array [nbatch]
  int nbatch;
  const int* maps;       // device
  int n_launch;          // value of n for descriptors with n < 0
  // split-K workspace (optional): partial products [split][batch][mmax][nmax]
  c_t<R>* ws = nullptr;
  long long ws_elems = 0;
  int num_sms = 148;
  int* err = nullptr;    // device flag for the tensor-core path's bounded waits; null: SIMT only
  int tune = 0;          // host only: the tile autotuner's mode for this launch (HPS_TUNE_*)
};

// FP32 complex GEMM on the tensor cores (tc.cu): batched like launch_gemm, for tiles of
// 128 rows x 64 complex columns; *err is set when a bounded wait gives up.
cudaError_t launch_tc_gemm(const GemmArgs<float>& a, int mmax, int nmax, int kmax, int* err, cudaStream_t s);
// The same product with A stored tiled by tile_operator (descriptor a_r = the pair's first unit
// of the tiled layout, a_c = its k chunks; lda = the rows the layout was tiled with, the same
// for every pair of the launch, while a descriptor's m may be smaller).  terms = 0: FP32 blocks
// (tile_operator), 3xTF32; terms = 2: A tiled by tile_operator_bf16x3 and multiplied as
// hi*hi + hi*lo + lo*hi of bf16 splits (about 3 * 2^-16 relative error); terms = 3: A tiled by
// tile_operator_bf16x6, the six products of three-term bf16 splits with term indices summing to
// at most 2 (about FP32 accuracy).
cudaError_t launch_tc_gemm_tiled(const GemmArgs<float>& a, int mmax, int nmax, int kmax, int terms, int* err,
                                 cudaStream_t s);
// The tile autotuner's process-wide table (tc.cu): as text into buf (NUL-terminated, at most
// len bytes), returning the number of shapes; and emptied.
int autotune_table(char* buf, int len);
void autotune_clear();
// TL[P][row tile][k chunk] = 128 x 8 complex blocks of the operators A_P (rows x K, leading
// dimension lda, pair P at A + P * pair_stride), each contiguous in the tensor-core tile order,
// zero-padded past rows and K.
cudaError_t tile_operator(float2* TL, const float2* A, int npairs, int rows, int K, int lda, long long pair_stride,
                          cudaStream_t s);
// The same blocks as bf16 hi and lo tiles (hi = bf16(x), lo = bf16(x - hi)) in the 16-bit
// core-matrix order; a block occupies the same 8 KB.
cudaError_t tile_operator_bf16x3(float2* TL, const float2* A, int npairs, int rows, int K, int lda,
                                 long long pair_stride, cudaStream_t s);
// The same blocks as three bf16 term tiles (hi, mid = bf16(x - hi), lo = bf16(x - hi - mid)):
// 12 bytes per entry, 1.5 times the FP32 layout's bytes (block offsets scale the same way).
cudaError_t tile_operator_bf16x6(void* TL, const float2* A, int npairs, int rows, int K, int lda,
                                 long long pair_stride, cudaStream_t s);
constexpr int TILE_M = 128, TILE_K = 8;  // rows and complex k of one operator block
// Tiled operator layout (tile_operator, tile_operator_bf16x3): per pair, row tile rt and k
// chunk kt make one block of 128 rows x 8 complex k in the tensor-core order, blocks ordered
// (rt, kt); the blocks of the last row tile keep only its rows rounded up to 8 (a compact block
// is the prefix of a full one).  Offsets count 512-byte units (8 rows x 8 complex k).
constexpr int TILE_UNIT = 64;  // float2 per unit
__host__ __device__ inline int tiled_row_tiles(int rows) { return (rows + TILE_M - 1) / TILE_M; }
__host__ __device__ inline int tiled_last_rows(int rows) {
  return (rows - TILE_M * (tiled_row_tiles(rows) - 1) + 7) / 8 * 8;
}
__host__ __device__ inline long long tiled_pair_units(int rows, int K) {
  const int nkt = (K + TILE_K - 1) / TILE_K;
  return (long long)nkt * ((tiled_row_tiles(rows) - 1) * (TILE_M / 8) + tiled_last_rows(rows) / 8);
}
// unit offset, inside its pair, of block (rt, kt) of an operator with `rows` rows and nkt k
// chunks; rows_blk = the rows the block stores
__host__ __device__ inline long long tiled_block_unit(int rows, int nkt, int rt, int kt, int& rows_blk) {
  rows_blk = rt < tiled_row_tiles(rows) - 1 ? TILE_M : tiled_last_rows(rows);
  return (long long)rt * nkt * (TILE_M / 8) + (long long)kt * (rows_blk / 8);
}
// Fixed-order sum of ksplit partial tiles from a.ws with the descriptor epilogue (blas.cu).
cudaError_t splitk_reduce(const GemmArgs<float>& a, int ksplit, int mmax, int nmax, cudaStream_t s);
void optin_tc();
// The double-float Arnoldi matvec y = Pi M z on the tensor cores by exact splitting (ozk.cu):
// T (FP64 leaf maps) cut once per solve into bf16 slices (OA, ozk_slices_elems entries), z FP32,
// y double-float; rows 4q <= 92, 1 <= nrhs <= 32.
bool ozk_supported(int nb, int nrhs);
size_t ozk_slices_elems(int E, int nb);
cudaError_t ozk_slice_T(const double2* T, uint16_t* OA, int E, int nb, cudaStream_t s);
cudaError_t ozk_matvec(const uint16_t* OA, const int* nbr, const float2* z, float4* y, int E, int nb, int nrhs,
                       int num_sms, int* err, cudaStream_t s);
cudaError_t round_to_f2(float2* dst, const double2* src, long long n, cudaStream_t s);
void optin_ozk();

// kmax > 0 enables splitting K across blocks when the grid would not fill the GPU.
template <typename R>
cudaError_t launch_gemm(const GemmArgs<R>& a, int mmax, int nmax, cudaStream_t s, int kmax = 0);

// Gauss-Jordan inversion of nmat augmented matrices W = [S | I] (m x 2m, row-major,
// matrix b at W + b*m*2m).  Partial pivoting; on exit W(:, m:2m) = S^{-1}.
// flag: device int, set to 1 if a zero pivot was met.
// piv_ws: device ints [nmat * GJ_NB]; lu_ws: device [nmat * GJ_NB * GJ_NB] elements.
constexpr int GJ_NB = 16;
template <typename R>
cudaError_t gj_invert(c_t<R>* W, int m, int nmat, int* piv_ws, c_t<R>* lu_ws, int* flag,
                      cudaStream_t s);
// General form: W = [S | B] (m x ld, ld > m) -> right part S^{-1} B (same pivoting).
template <typename R>
cudaError_t gj_solve(c_t<R>* W, int m, int ld, int nmat, int* piv_ws, c_t<R>* lu_ws, int* flag, cudaStream_t s);

}  // namespace hps
