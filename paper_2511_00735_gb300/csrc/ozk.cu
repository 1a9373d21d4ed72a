// The mixed path's Arnoldi matvec on the tensor cores by exact splitting.
//
// y_p = z_{nb(p)} + sum_b T_e[a][b] z_{e,b} (section 4.3, the skeleton operator Pi M applied in
// outgoing coordinates; p = element e's edge row a; 0 on the physical boundary) with the leaf
// maps T in FP64, z in FP32 and y in double-float (about 48 significant bits), the quantity the
// SIMT df_matvec_kernel forms with error-free FP32 products.
//
// Exact splitting (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications", Numer.
// Algorithms 59, 2012): per element the complex product is the real product A B' with A the
// real-expanded rows of T_e (A[i][2k] = Re T_ik, A[i][2k+1] = Im T_ik) and B' the expanded z
// (B'[2k][2r] = Re z, B'[2k+1][2r] = -Im z, B'[2k][2r+1] = Im z, B'[2k+1][2r+1] = Re z).  Each
// row i of A is cut into OZ_S slices of OZ_BITS bits aligned to the row's exponent E_i
// (|a| < 2^E_i): a = sum_s alpha_s 2^(E_i - OZ_BITS s) + (below 2^(E_i - 49)), alpha_s integers
// with |alpha_s| < 2^OZ_BITS; each column j of B' likewise with the column exponent F_j (the two
// columns of one right-hand side share it).  A slice value alpha 2^e is exact in bf16 (8-bit
// significand), a product of two slices is exact, and a k-sum of them is an integer times
// 2^(E_i + F_j - OZ_BITS (s + t)) below 2^14 K; all products with the same d = s + t share that
// scale, so one FP32 accumulator per d holds their sum exactly while it stays below 2^24 (K <=
// 148 real k for every d <= 8: every GLL order up to 18; above, the two smallest groups may
// round by a unit of 2^(-7 d), far below the result's last bit).  The products with
// d <= OZ_D are formed (per k chunk of 16 and A slice s, the B slices t = 1 .. 8 - s side by side
// in one or two kind::f16 MMAs of N up to 256), the rest dropped; the dropped
// part and the slice truncation are below about 2^-45 of max|A_i.| max|B'_.j| K.  The seven
// accumulators are summed in double-float by TwoSum from the largest, then the neighbour term
// z_{nb(p)}.
//
// One persistent CTA per SM (the seven accumulators of an element take 7 x 2 NC tensor-memory
// columns), 512 threads:
//   warp 0   (one thread) bulk copies: the element's z rows into one of two buffers, the A slices
//            of each k chunk (sliced once per solve by ozk_slice_T) into a ring of stages;
//   warp 1   (one thread) the chunk's MMAs (10 for 32 right-hand sides), committed to the stage's
//            empty barrier and,
//            after the element's last chunk, to the accumulator barrier;
//   warps 2-7 the column exponents of the element's z, then per chunk the 7 bf16 slices of B'
//            (integer bit extraction);
//   warps 8-15 the epilogue, two warps per lane quarter w % 4 = rows 32 (w % 4) .. + 31, each
//            on half the columns: each thread copies its half of the neighbour row z_{nb(p)}
//            into shared memory while the MMAs run, then sums the accumulators in double-float,
//            adds the neighbour term and stores df64; then the accumulators are free.
// Every wait is bounded; a wait that gives up sets *err and the roles drain.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "dfops.cuh"
#include "tcgen05.cuh"

namespace hps {
namespace {
using namespace tcg;
using dfops::two_sum;

constexpr int OZ_BITS = 7;        // bits per slice
constexpr int OZ_S = 7;           // slices per operand
constexpr int OZ_D = 8;           // products with s + t <= OZ_D are formed
constexpr int OZ_G = OZ_D - 1;    // accumulators: d = 2 .. OZ_D
constexpr int OZ_KR = 16;         // real k per chunk = one kind::f16 MMA
// MMA rows MM: 64 when the element's 4q edge rows fit (GLL order <= 16), else 128 (the rest unused)
// rows of an M = 64 accumulator per tensor-memory lane quarter (lanes 32 w .. 32 w + RPQ - 1)
constexpr int OZ_M64_RPQ = 16;
constexpr int OZ_SLICERS = 6;                 // warps 2-7
constexpr int OZ_EPI = 8;                     // warps 8-15: two per tensor-memory lane quarter
constexpr int OZ_NT = 32 * (2 + OZ_SLICERS + OZ_EPI);
constexpr int OZ_NBMAX = 92;      // 4q at GLL order 24

template <int NC, int MM> struct OzTile {
  static constexpr int N = 2 * NC;                       // MMA N: real columns
  // A region: 7 slices of up to 96 rows x 16 bf16 back to back, plus room for the MMA's reads of
  // 128 rows from the last slice
  static constexpr int ROWS = MM == 64 ? 64 : 96;         // most rows a chunk's A slices keep
  static constexpr int S = MM == 64 ? 5 : 3;              // stages
  static constexpr int NBM = MM == 64 ? 64 : OZ_NBMAX;    // most edge rows of an element
  static constexpr int A_REGION = OZ_S * ROWS * OZ_KR * 2 + (MM - 8) * OZ_KR * 2;
  static constexpr int B_SLICE = N * OZ_KR * 2;          // one slice of B' for one chunk
  static constexpr int STAGE = ((A_REGION + OZ_S * B_SLICE) + 1023) / 1024 * 1024;
  static constexpr int ZBUF = NBM * NC * 8;              // one element's z rows (FP32 complex)
  static constexpr int NLD = NC / 2 + 1;                 // neighbour staging row (half the columns)
  static constexpr int NBUF = OZ_EPI * 32 * NLD * 8;     // the epilogue warps' neighbour rows
  static constexpr size_t SMEM = (size_t)S * STAGE + 2 * (size_t)ZBUF + NBUF + 1024;
  static constexpr int TCOLS = OZ_G * N <= 256 ? 256 : 512;
  // kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M
  static constexpr int TPM = 256 / N;                     // B slices per MMA (N <= 256)
  static __device__ __forceinline__ uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MM >> 4) << 24);
  }
};

// bf16 bits of sign * alpha 2^p (0 <= alpha < 128 an integer; exact, alpha has <= 7 bits),
// assembled from the integer: leading bit at 2^(p + msb), the bits below it as the mantissa;
// a value below the normal range (never for entries within 2^-77 of their row's or column's
// largest) becomes 0
__device__ __forceinline__ uint16_t slice_bits(uint32_t alpha, int p, uint32_t sign) {
  const int msb = 31 - __clz(alpha | 1u);          // alpha = 0 gives 0 below
  const int be = p + msb + 127;                     // biased exponent
  const uint32_t mant = (alpha << (7 - msb)) & 0x7Fu;
  const uint32_t bits = (sign << 15) | ((uint32_t)be << 7) | mant;
  return (alpha != 0 && be > 0 && be < 255) ? (uint16_t)bits : (uint16_t)0;
}
// The OZ_S slices of a value with integer magnitude m times 2^pe, below 2^e:
// q = floor(|x| 2^(49 - e)) < 2^49, alpha_s = bits 49 - 7s .. 55 - 7s of q (|x| truncated
// toward zero in 7-bit chunks), slice s = sign * alpha_s 2^(e - 7 s).  Integer operations only.
__device__ __forceinline__ void slices_of(uint64_t m, int pe, uint32_t sign, int e, uint16_t* out) {
  const int shift = pe + (OZ_BITS * OZ_S) - e;  // q = m 2^shift
  uint64_t q = 0;
  if (m != 0) q = shift >= 0 ? (shift < 64 ? m << shift : 0) : (-shift < 64 ? m >> -shift : 0);
#pragma unroll
  for (int s = 1; s <= OZ_S; ++s)
    out[s - 1] = slice_bits((uint32_t)(q >> (OZ_BITS * (OZ_S - s))) & ((1u << OZ_BITS) - 1), e - OZ_BITS * s, sign);
}
// the slices of x (|x| < 2^e); subnormal x counts as 0
__device__ __forceinline__ void slice7(double x, int e, uint16_t* out) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const uint64_t m = ex == 0 ? 0 : ((b & ((1ull << 52) - 1)) | (1ull << 52));
  slices_of(m, ex - 1075, (uint32_t)(b >> 63), e, out);
}
__device__ __forceinline__ void slice7f(float x, int e, uint16_t* out) {
  const uint32_t b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xFF);
  const uint64_t m = ex == 0 ? 0 : ((b & 0x7FFFFFu) | 0x800000u);
  slices_of(m, ex - 150, b >> 31, e, out);
}
// smallest e with |x| < 2^e for every |x| <= m (0 when m == 0): m = f 2^e, 0.5 <= f < 1
__device__ __forceinline__ int exp_above(double m) {
  if (!(m > 0.0)) return 0;
  return (int)((((unsigned long long)__double_as_longlong(m)) >> 52) & 0x7FF) - 1022;
}
__device__ __forceinline__ int exp_above_f(float m) {
  if (!(m > 0.f)) return 0;
  return (int)((__float_as_uint(m) >> 23) & 0xFF) - 126;
}

// A slices: OA[e][kc][s][rows_pad x 16 bf16 in core_off16 order], zero past 4q rows and 8q k.
// One warp per (element, padded row).
__global__ void ozk_slice_T_kernel(const double2* __restrict__ T, uint16_t* __restrict__ OA, int E, int nb,
                                   int rows_pad, int nkc) {
  const int lane = threadIdx.x % 32;
  const long long nwarp = (long long)gridDim.x * (blockDim.x / 32);
  const int K = 2 * nb, KP = nkc * OZ_KR;
  for (long long w = blockIdx.x * (long long)(blockDim.x / 32) + threadIdx.x / 32; w < (long long)E * rows_pad;
       w += nwarp) {
    const int e = (int)(w / rows_pad), i = (int)(w % rows_pad);
    const double2* Ti = T + ((long long)e * nb + i) * nb;
    double m = 0.0;
    if (i < nb)
      for (int k = lane; k < nb; k += 32) m = fmax(m, fmax(fabs(Ti[k].x), fabs(Ti[k].y)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    const int ex = exp_above(m);
    for (int k = lane; k < KP; k += 32) {
      uint16_t sl[OZ_S];
      if (i < nb && k < K) {
        const double2 t = Ti[k / 2];
        slice7((k & 1) ? t.y : t.x, ex, sl);
      } else {
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) sl[s] = 0;
      }
      const int kc = k / OZ_KR;
      uint16_t* blk = OA + ((long long)e * nkc + kc) * OZ_S * rows_pad * OZ_KR;
      const uint32_t off = core_off16(i, k % OZ_KR) / 2;
#pragma unroll
      for (int s = 0; s < OZ_S; ++s) blk[(long long)s * rows_pad * OZ_KR + off] = sl[s];
    }
  }
}

template <int NC, int MM>
__global__ void __launch_bounds__(OZ_NT, 1) ozk_matvec_kernel(const uint16_t* __restrict__ OA,
                                                              const int* __restrict__ nbr,
                                                              const float2* __restrict__ z, float4* __restrict__ y,
                                                              int E, int nb, int nrhs, int rows_pad, int nkc,
                                                              int* err) {
  using TB = OzTile<NC, MM>;
  constexpr int OZ_STAGES = TB::S;
  constexpr int N = TB::N, STAGE = TB::STAGE, B_SLICE = TB::B_SLICE, A_REGION = TB::A_REGION;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[OZ_STAGES], conv[OZ_STAGES], empty[OZ_STAGES], zfull[2], zfree[2], accf,
      acce, fin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail_store;
  volatile int& s_fail = s_fail_store;
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float2* zbuf = reinterpret_cast<float2*>(ring + (size_t)OZ_STAGES * STAGE);  // [2][nb][nrhs]
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const uint32_t a_slice = (uint32_t)rows_pad * OZ_KR * 2;  // bytes of one A slice of a chunk
  const uint32_t a_bytes = OZ_S * a_slice;
  const uint32_t z_bytes = (uint32_t)nb * nrhs * 8;
  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < OZ_STAGES; ++i) {
      mbar_init(&full[i], 1);  // the producer's expect_tx arrival
      mbar_init(&conv[i], OZ_SLICERS);  // the B-slicing warps
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&zfull[i], 1);
      mbar_init(&zfree[i], OZ_SLICERS);
    }
    mbar_init(&accf, 1);
    mbar_init(&acce, OZ_EPI);
    mbar_init(&fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "n"(TB::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  auto wait = [&](uint64_t* b, uint32_t parity) -> bool {  // warp-uniform result
    bool ok = !s_fail && mbar_wait(smem_u32(b), parity);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) s_fail = 1;
    return ok;
  };
  auto wait1 = [&](uint64_t* b, uint32_t parity) -> bool {  // single-thread roles
    if (!s_fail && mbar_wait(smem_u32(b), parity)) return true;
    s_fail = 1;
    return false;
  };

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      long long g = 0;
      int ie = 0;
      bool ok = true;
      for (int e = blockIdx.x; e < E && ok; e += gridDim.x, ++ie) {
        const int zb = ie & 1;
        if (ie >= 2 && !wait1(&zfree[zb], (uint32_t)(((ie >> 1) - 1) & 1))) break;
        expect_tx(&zfull[zb], z_bytes);
        bulk_copy(smem_u32(zbuf + (size_t)zb * TB::NBM * NC), z + (long long)e * nb * nrhs, z_bytes, &zfull[zb]);
        for (int c = 0; c < nkc; ++c, ++g) {
          const int st = (int)(g % OZ_STAGES);
          if (g >= OZ_STAGES && !wait1(&empty[st], (uint32_t)(((g / OZ_STAGES) - 1) & 1))) {
            ok = false;
            break;
          }
          expect_tx(&full[st], a_bytes);
          bulk_copy(smem_u32(ring + (size_t)st * STAGE), OA + ((long long)e * nkc + c) * OZ_S * rows_pad * OZ_KR,
                    a_bytes, &full[st]);
        }
      }
      // no bulk copy may still be landing when the CTA ends
      for (long long gg = g - OZ_STAGES > 0 ? g - OZ_STAGES : 0; gg < g; ++gg)
        mbar_wait(smem_u32(&full[gg % OZ_STAGES]), (uint32_t)((gg / OZ_STAGES) & 1));
      for (int j = ie - 2 > 0 ? ie - 2 : 0; j < ie; ++j) mbar_wait(smem_u32(&zfull[j & 1]), (uint32_t)((j >> 1) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      long long g = 0;
      int ie = 0;
      bool ok = true, issued = false;
      for (int e = blockIdx.x; e < E && ok; e += gridDim.x, ++ie) {
        if (ie >= 1 && !wait1(&acce, (uint32_t)((ie - 1) & 1))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < nkc; ++c, ++g) {
          const int st = (int)(g % OZ_STAGES);
          const uint32_t par = (uint32_t)((g / OZ_STAGES) & 1);
          if (!wait1(&full[st], par) || !wait1(&conv[st], par)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(ring + (size_t)st * STAGE), sb = sa + A_REGION;
          // A slice s times the B slices t = 1 .. OZ_D - s at once: the B slices lie side by side
          // along N and their accumulators d = s + t too, so one MMA of N = (number of t) x 2 NC
          // (at most 256) covers several products; the s = 1 MMAs of the first chunk start every
          // accumulator
#pragma unroll
          for (int s = 1; s <= OZ_S; ++s) {
            const int tmax = OZ_D - s < OZ_S ? OZ_D - s : OZ_S;
#pragma unroll
            for (int t0 = 1; t0 <= tmax; t0 += TB::TPM) {
              const int nt = tmax - t0 + 1 < TB::TPM ? tmax - t0 + 1 : TB::TPM;
              mma_bf16(tmem + (uint32_t)((s + t0 - 2) * N), smem_desc16(sa + (uint32_t)(s - 1) * a_slice),
                       smem_desc16(sb + (uint32_t)(t0 - 1) * B_SLICE), TB::idesc(nt * N),
                       (c > 0 || s > 1) ? 1u : 0u);
            }
          }
          tc_commit(&empty[st]);
          issued = true;
        }
        if (!ok) break;
        tc_commit(&accf);
      }
      if (issued) {
        tc_commit(&fin);
        mbar_wait(smem_u32(&fin), 0);
      }
    }
  } else if (warp <= 1 + OZ_SLICERS) {
    // ---------------- column exponents and B' slices ----------------
    const int tb = tid - 64;
    constexpr int SPT = ((OZ_KR / 2) * NC + 32 * OZ_SLICERS - 1) / (32 * OZ_SLICERS);  // entries per thread
    long long g = 0;
    int ie = 0;
    bool ok = true;
    for (int e = blockIdx.x; e < E && ok; e += gridDim.x, ++ie) {
      const int zb = ie & 1;
      if (!wait(&zfull[zb], (uint32_t)((ie >> 1) & 1))) break;
      const float2* zs = zbuf + (size_t)zb * TB::NBM * NC;
      // this thread only ever slices right-hand side rr (l = tb mod 32 OZ_SLICERS below): its column
      // exponent, shared by the columns 2 rr and 2 rr + 1 of B'
      const int rr = tb % NC;
      int F = 0;
      if (rr < nrhs) {
        float m = 0.f;
        for (int k = 0; k < nb; ++k) {
          const float2 v = zs[k * nrhs + rr];
          m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        F = exp_above_f(m);
      }
      for (int c = 0; c < nkc; ++c, ++g) {
        const int st = (int)(g % OZ_STAGES);
        // the stage's A has landed, so its previous MMAs are done: its B' may be rewritten
        if (!wait(&full[st], (uint32_t)((g / OZ_STAGES) & 1))) {
          ok = false;
          break;
        }
        unsigned char* sb = ring + (size_t)st * STAGE + A_REGION;
        // complex (kk, r) of the chunk -> B'^T rows 2r: (Re, -Im), 2r+1: (Im, Re) at real k 2kk, 2kk+1;
        // a thread loads all its entries (l = tb + 32 OZ_SLICERS u) before it slices any, so the
        // loads and the independent slicing chains overlap
        float2 v[SPT];
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
          const int l = tb + 32 * OZ_SLICERS * u, kk = l / NC, k = c * (OZ_KR / 2) + kk;
          v[u] = (l < (OZ_KR / 2) * NC && k < nb && rr < nrhs) ? zs[k * nrhs + rr] : make_float2(0.f, 0.f);
        }
        uint16_t re[SPT][OZ_S], im[SPT][OZ_S];
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
          slice7f(v[u].x, F, re[u]);
          slice7f(v[u].y, F, im[u]);
        }
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
          const int l = tb + 32 * OZ_SLICERS * u;
          if (l >= (OZ_KR / 2) * NC) break;
          const int kk = l / NC, r = rr;
          const uint32_t o0 = core_off16(2 * r, 2 * kk), o1 = core_off16(2 * r + 1, 2 * kk);
#pragma unroll
          for (int t = 0; t < OZ_S; ++t) {
            unsigned char* bt = sb + t * B_SLICE;
            *reinterpret_cast<uint32_t*>(bt + o0) = (uint32_t)re[u][t] | ((uint32_t)(im[u][t] ^ 0x8000u) << 16);
            *reinterpret_cast<uint32_t*>(bt + o1) = (uint32_t)im[u][t] | ((uint32_t)re[u][t] << 16);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[st]);
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(&zfree[zb]);  // this warp is done with the element's z rows
    }
  } else {
    // ---------------- epilogue ----------------
    constexpr int NLD = TB::NLD;
    // warp w: lane quarter w % 4 (rows), column half (w - 8) / 4
    const int quarter = warp & 3, half = (warp - 2 - OZ_SLICERS) / 4;
    // accumulator row of this lane (past every element row when the lane holds none)
    const int i = MM == 128 ? 32 * quarter + lane : (lane < OZ_M64_RPQ ? OZ_M64_RPQ * quarter + lane : 1 << 20);
    const int r0 = half * (NC / 2), r1 = min(nrhs, r0 + NC / 2);
    // this thread's half of its neighbour row z_{nb(p)}, copied in while the element's MMAs run
    float2* nrow = reinterpret_cast<float2*>(ring + (size_t)OZ_STAGES * STAGE + 2 * (size_t)TB::ZBUF) +
                   ((warp - 2 - OZ_SLICERS) * 32 + lane) * NLD;
    int ie = 0;
    for (int e = blockIdx.x; e < E; e += gridDim.x, ++ie) {
      const long long p = (long long)e * nb + i;
      const int q = i < nb ? nbr[p] : -1;
      if (q >= 0)
        for (int r = r0; r < r1; ++r) cp_async8z(smem_u32(nrow + (r - r0)), z + (long long)q * nrhs + r, 8u);
      cp_async_commit();
      if (!wait(&accf, (uint32_t)(ie & 1))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      cp_async_wait<0>();
      // 8-column blocks of this warp's half: the 7 accumulators' loads issued together, one wait
#pragma unroll 1
      for (int gb = half * (N / 16); gb < (half + 1) * (N / 16); ++gb) {
        uint32_t v[OZ_G][8];
#pragma unroll
        for (int d = 0; d < OZ_G; ++d) {
          const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(d * N + gb * 8);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]), "=r"(v[d][5]),
                         "=r"(v[d][6]), "=r"(v[d][7])
                       : "r"(ta));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float hs[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          hs[j] = __uint_as_float(v[0][j]);
          lo[j] = 0.f;
#pragma unroll
          for (int d = 1; d < OZ_G; ++d) {
            float t, er;
            two_sum(hs[j], __uint_as_float(v[d][j]), t, er);
            hs[j] = t;
            lo[j] = __fadd_rn(lo[j], er);
          }
        }
        if (i < nb) {
#pragma unroll
          for (int j2 = 0; j2 < 4; ++j2) {
            const int r = gb * 4 + j2;
            if (r >= nrhs) continue;
            float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q >= 0) {
              const float2 zn = nrow[r - r0];
              float t, er;
              two_sum(hs[2 * j2], zn.x, t, er);
              const float lre = __fadd_rn(lo[2 * j2], er);
              two_sum(t, lre, o.x, o.z);
              two_sum(hs[2 * j2 + 1], zn.y, t, er);
              const float lim = __fadd_rn(lo[2 * j2 + 1], er);
              two_sum(t, lim, o.y, o.w);
            }
            y[p * nrhs + r] = o;
          }
        }
      }
      // the accumulators are read: the next element's MMAs may overwrite them
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce);
    }
    cp_async_wait<0>();  // no copy lands after the CTA ends
  }
  __syncthreads();
  if (tid == 0 && s_fail) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TB::TCOLS) : "memory");
}

}  // namespace

bool ozk_supported(int nb, int nrhs) { return nb <= OZ_NBMAX && nb % 2 == 0 && nrhs >= 1 && nrhs <= 32; }

size_t ozk_slices_elems(int E, int nb) {
  const int rows_pad = (nb + 7) / 8 * 8, nkc = (2 * nb + OZ_KR - 1) / OZ_KR;
  return (size_t)E * nkc * OZ_S * rows_pad * OZ_KR;
}

cudaError_t ozk_slice_T(const double2* T, uint16_t* OA, int E, int nb, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  const int rows_pad = (nb + 7) / 8 * 8, nkc = (2 * nb + OZ_KR - 1) / OZ_KR;
  const long long warps = (long long)E * rows_pad;
  const long long blocks = std::min<long long>((warps + 7) / 8, 65536);
  ozk_slice_T_kernel<<<(int)blocks, 256, 0, s>>>(T, OA, E, nb, rows_pad, nkc);
  note_launch();
  return cudaGetLastError();
}

cudaError_t ozk_matvec(const uint16_t* OA, const int* nbr, const float2* z, float4* y, int E, int nb, int nrhs,
                       int num_sms, int* err, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  if (!ozk_supported(nb, nrhs)) return cudaErrorInvalidValue;
  const int rows_pad = (nb + 7) / 8 * 8, nkc = (2 * nb + OZ_KR - 1) / OZ_KR;
  const int grid = std::min(E, num_sms);
  if (rows_pad <= 64) {
    if (nrhs <= 16)
      ozk_matvec_kernel<16, 64><<<grid, OZ_NT, OzTile<16, 64>::SMEM, s>>>(OA, nbr, z, y, E, nb, nrhs, rows_pad, nkc, err);
    else
      ozk_matvec_kernel<32, 64><<<grid, OZ_NT, OzTile<32, 64>::SMEM, s>>>(OA, nbr, z, y, E, nb, nrhs, rows_pad, nkc, err);
  } else {
    if (nrhs <= 16)
      ozk_matvec_kernel<16, 128><<<grid, OZ_NT, OzTile<16, 128>::SMEM, s>>>(OA, nbr, z, y, E, nb, nrhs, rows_pad, nkc,
                                                                          err);
    else
      ozk_matvec_kernel<32, 128><<<grid, OZ_NT, OzTile<32, 128>::SMEM, s>>>(OA, nbr, z, y, E, nb, nrhs, rows_pad, nkc,
                                                                          err);
  }
  note_launch();
  return cudaGetLastError();
}

__global__ void round_to_f2_kernel(float2* __restrict__ dst, const double2* __restrict__ src, long long n) {
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < n; l += (long long)gridDim.x * blockDim.x)
    dst[l] = make_float2((float)src[l].x, (float)src[l].y);
}

cudaError_t round_to_f2(float2* dst, const double2* src, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 65536);
  round_to_f2_kernel<<<(int)blocks, 256, 0, s>>>(dst, src, n);
  note_launch();
  return cudaGetLastError();
}

void optin_ozk() {
  smem_optin(ozk_matvec_kernel<16, 64>);
  smem_optin(ozk_matvec_kernel<32, 64>);
  smem_optin(ozk_matvec_kernel<16, 128>);
  smem_optin(ozk_matvec_kernel<32, 128>);
}

}  // namespace hps
