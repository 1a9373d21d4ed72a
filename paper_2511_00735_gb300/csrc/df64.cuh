// Double-float (df64) kernels of the outer FGMRES: a complex df64 number is a
// float4 (re_hi, im_hi, re_lo, im_lo) with the value (re_hi + re_lo) + i (im_hi + im_lo).
#pragma once

#include "common.cuh"

namespace hps {

cudaError_t df_from_d(float4* dst, const double2* src, long long n, cudaStream_t s);
cudaError_t df_to_d(double2* dst, const float4* src, long long n, cudaStream_t s);
// dst[0] = a, dst[1] = b in stream order (one thread)
cudaError_t set_pointers(void** dst, const void* a, void* b, cudaStream_t s);
// a row gather of leading parts dst[row][r] = hi(src[map[row]][r]) (map < 0 -> 0) whose source
// pointer is read from device memory, and a row scatter dst[map[row]][r] = src[row][r] whose
// destination pointer is read from device memory (a captured graph replays them with new vectors)
cudaError_t df_gather_hi_ind(float2* dst, const float4* const* srcp, const int* map, long long rows, int nrhs,
                             cudaStream_t s);
cudaError_t scatter_f2_ind(float2* const* dstp, const float2* src, const int* map, long long rows, int nrhs,
                           cudaStream_t s);
// z[p] = hi(v[nb(p)]) (0 on the physical boundary): the identity preconditioner in incoming coordinates
cudaError_t df_swap_hi(float2* z, const float4* v, const int* nbr, long long rows, int nrhs, cudaStream_t s);

// y = Pi M x (c0 == null) or y = c0 - Pi M x on the element-side layout; T df64 [E][nb][nb]
template <typename X>
cudaError_t df_matvec(const float4* T, const int* nbr, const X* x, const float4* c0, float4* y, int E, int nb, int nrhs,
                      int grid, cudaStream_t s);

// out[i][r] = sum_rows conj(V_i[row][r]) w[row][r] (i < nvec), FP64 result; partial holds
// bdot_blocks(rows) * nvec * nrhs df64 numbers
cudaError_t df_bdot(const float4* V, long long vstride, int nvec, const float4* w, long long rows, int nrhs,
                    float4* partial, double2* out, cudaStream_t s);
// one pass over V_0..V_{nvec-1}: out[2i] = sum conj(V_i) y0, out[2i+1] = sum conj(V_i) y1,
// out[2 nvec] = sum conj(y1) y1; FP64 [2 nvec + 1][nrhs]; partial holds
// df_dots2_blocks(rows) * (2 nvec + 1) * nrhs df64 numbers
int df_dots2_blocks(long long rows);
cudaError_t df_dots2(const float4* V, long long vstride, int nvec, const float4* y0, const float4* y1, long long rows,
                     int nrhs, float4* partial, double2* out, cudaStream_t s);
// one pass over V_0..V_{nvec-1}: out_v = sv vt + sum ca_i V_i, out_w = sw w + svw vt + sum cb_i V_i
// (coef: df64 [2 nvec + 3][nrhs] = ca rows, cb rows, sv, sw, svw); out_v may equal vt
cudaError_t df_update2(const float4* V, long long vstride, int nvec, const float4* vt, const float4* w,
                       const float4* coef, float4* out_v, float4* out_w, long long rows, int nrhs, cudaStream_t s);
// w += sign * sum_i V_i h_i
template <typename VT>
cudaError_t df_bupdate(float4* w, const VT* V, long long vstride, int nvec, const double2* h, long long rows, int nrhs,
                       float sign, cudaStream_t s);
// out = w / sqrt(re dots[r]) when that norm exceeds floor[r], else 0
cudaError_t df_bscale(float4* out, const float4* w, const double2* dots, const double* floor, long long rows, int nrhs,
                      cudaStream_t s);

}  // namespace hps
