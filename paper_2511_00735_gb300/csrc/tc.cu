// Batched complex FP32 GEMM on the fifth-generation tensor cores (tcgen05) for the
// merge levels (section 4.1: S = I - T_bb T_aa, X1, X2, T_pair = D - C A^{-1} B and the
// sweep operators are all batched complex GEMMs with scatter epilogues).
//
// Complex product as one real product.  With A stored interleaved (re, im) it already is
// the real matrix [m][2k]; B (k x n complex) is expanded while it is staged into
//     B'[2k][2n] = [[Re b, Im b], [-Im b, Re b]]   per complex entry,
// so that A_real B' = C interleaved: C[i][2j] = sum_k Re a Re b - Im a Im b and
// C[i][2j+1] = sum_k Re a Im b + Im a Re b.
//
// FP32 accuracy from TF32 inputs (3xTF32): every operand x is split x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi); the tile product accumulates hi*hi + hi*lo + lo*hi in
// FP32 in tensor memory (the dropped lo*lo term is below 2^-22 relative).
//
// One CTA (128 threads) computes a 128-row x 64-complex-column tile: all threads split one
// k-chunk (8 complex) of A and B into shared memory in the canonical no-swizzle K-major
// layout (8-row x 16-byte core matrices), one thread issues the 6 tcgen05.mma (M = 128,
// N = 128 real, K = 8) of the chunk and commits them to the chunk's mbarrier; two stages,
// and each thread fetches the next chunk's values into registers before the current one
// is multiplied.  Three CTAs fit on an SM (97 KB of shared memory, 384 TMEM columns).
// The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. output rows) and applies the same descriptor epilogue as the SIMT GEMM
// (alpha, beta * C0 with a two-segment C0, row and column maps).  Every mbarrier wait is
// bounded; a wait that gives up sets *err and the tile is left unwritten.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hps.h"
#include "common.cuh"
#include "tcgen05.cuh"

namespace hps {
namespace {
using namespace tcg;

constexpr int TC_NT = 128;
constexpr int TC_M = 128;              // output rows per CTA = TMEM lanes
constexpr int TC_KC = 8;               // complex k per chunk
constexpr int TC_KR = 2 * TC_KC;       // real k per chunk = 2 MMA k-steps of 8
constexpr int A_PER = TC_M * TC_KC / TC_NT;   // complex A values each thread stages per chunk
constexpr uint32_t LBO = 128;          // bytes between core matrices along k
constexpr uint32_t SBO = (TC_KR / 4) * 128;  // bytes between 8-row groups
constexpr int A_TILE = TC_M * TC_KR;   // floats in one A tile (8 KB)
// per column tile NC (complex columns per CTA): MMA N = 2 NC real columns
template <int NC> struct TcTile {
  static constexpr int NR = 2 * NC;
  static constexpr int B_PER = TC_KC * NC / TC_NT;  // complex B values each thread stages per chunk
  static constexpr int B_TILE = NR * TC_KR;         // floats in one B' tile
  static constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;  // hi and lo of A and B'
  static constexpr int TCOLS = NR < 32 ? 32 : NR;   // tensor-memory columns (power of two >= 32)
  // instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, N, M
  static constexpr uint32_t IDESC =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NR >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
};

// byte offset of element (r, k) in a tile: core matrix (r/8, k/4), row r%8, column k%4
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(r >> 3) * SBO + (uint32_t)(k >> 2) * LBO + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 3) * 4;
}

// shared-memory matrix descriptor: start >> 4, leading (k) and stride (row group) byte
// offsets >> 4, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// Staging order of the A tile: element e covers core matrix e / 16 (row group, k group) and
// position e % 16 in it (row (e % 16) / 2, complex k (e % 2)), so that the 8-byte stores of a
// warp fill two whole core matrices (conflict-free) while its loads still read whole 32-byte
// sectors (8 rows x 4 complex).
__device__ __forceinline__ void a_elem(int e, int& r, int& kc) {
  constexpr int KG = TC_KC / 2;  // k groups (2 complex each) per chunk
  const int cm = e >> 4, w = e & 15;
  r = (cm / KG) * 8 + (w >> 1);
  kc = (cm % KG) * 2 + (w & 1);
}

// Complex entry (kc, nc) of a TC_KC x NC chunk of B handled for index l.  Within the 32
// consecutive l of one warp instruction, lane bits 0-1 give nc % 4, bit 2 gives kc % 2 and bits
// 3-4 give nc / 4 % 4; with b_rows' row order the warp's 8-byte B' stores then cover all 16
// bank pairs twice (the minimum of 2 wavefronts; 32 consecutive nc gave 8), and its loads still
// read 16 consecutive columns of two rows.
__device__ __forceinline__ void b_elem(int l, int NC, int& kc, int& nc) {
  const int w = l >> 5, ln = l & 31, ncq = NC >> 4;
  nc = (ln & 3) | ((ln >> 3) << 2) | ((w % ncq) << 4);
  kc = ((ln >> 2) & 1) | ((w / ncq) << 1);
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
  const float r = x - __uint_as_float(hi);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}


// The B' tiles of complex (kc, nc) = v: real column 2nc gets (Re b, -Im b), column 2nc+1 gets
// (Im b, Re b) at real k = 2kc, 2kc+1; lanes with bit 3 set store the odd row first, so that
// each store instruction mixes even and odd rows (see b_elem).
__device__ __forceinline__ void b_rows(float* Bh, float* Bl, int kc, int nc, float2 v, int l) {
  uint2 h0, l0, h1, l1;
  split_tf32(v.x, h0.x, l0.x);
  split_tf32(-v.y, h0.y, l0.y);
  split_tf32(v.y, h1.x, l1.x);
  h1.y = h0.x;
  l1.y = l0.x;
  // row 2nc + 1 lies 16 bytes (4 floats) after row 2nc in the same core matrix
  const uint32_t sw = (l >> 3) & 1;
  const uint32_t oa = core_off(2 * nc, 2 * kc) / 4 + 4 * sw, ob = oa + 4 - 8 * sw;
  uint2 ha, la, hb, lb;
  ha.x = sw ? h1.x : h0.x;
  ha.y = sw ? h1.y : h0.y;
  hb.x = sw ? h0.x : h1.x;
  hb.y = sw ? h0.y : h1.y;
  la.x = sw ? l1.x : l0.x;
  la.y = sw ? l1.y : l0.y;
  lb.x = sw ? l0.x : l1.x;
  lb.y = sw ? l0.y : l1.y;
  *reinterpret_cast<uint2*>(Bh + oa) = ha;
  *reinterpret_cast<uint2*>(Bl + oa) = la;
  *reinterpret_cast<uint2*>(Bh + ob) = hb;
  *reinterpret_cast<uint2*>(Bl + ob) = lb;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate) {
  asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(
                   tmem),
               "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
               : "memory");
}

// blockIdx.z = batch + nbatch * split; with ksplit > 1 each split covers kc complex k and stores
// its raw tile in the split-K workspace (reduced in fixed order by splitk_reduce)
template <int NC>
__global__ void __launch_bounds__(TC_NT, 3) tc_gemm_kernel(GemmArgs<float> a, int* err, int ksplit, int kc, int mmax,
                                                           int nmax) {
  using TT = TcTile<NC>;
  constexpr int NR = TT::NR, B_PER = TT::B_PER, B_TILE = TT::B_TILE, STAGE = TT::STAGE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int bb = blockIdx.z % a.nbatch, sp = blockIdx.z / a.nbatch;
  const GemmDesc d = a.desc[bb];
  const int n = d.n < 0 ? a.n_launch : d.n, m = d.m;
  const int kb = ksplit > 1 ? sp * kc : 0;
  const int kk = ksplit > 1 ? min(d.k, kb + kc) : d.k;  // this split covers complex k in [kb, kk)
  const int row0 = blockIdx.y * TC_M, col0 = blockIdx.x * NC;
  if (row0 >= m || col0 >= n) return;  // uniform over the block, before any tensor-memory use
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "n"(TT::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  const float2* Ab = a.A + (long long)d.a_r * a.lda + d.a_c;
  const int nk = kk > kb ? (kk - kb + TC_KC - 1) / TC_KC : 0;
  // the next chunk's operands are fetched into registers one iteration ahead
  float2 ra[A_PER], rb[B_PER];
  auto fetch = [&](int kt) {
    const int k0 = kb + kt * TC_KC;
#pragma unroll
    for (int u = 0; u < A_PER; ++u) {
      int r, kc;
      a_elem(tid + u * TC_NT, r, kc);
      const int gi = row0 + r, gk = k0 + kc;
      ra[u] = (gi < m && gk < kk) ? Ab[(long long)gi * a.lda + gk] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < B_PER; ++u) {
      int kc, nc;
      b_elem(tid + u * TC_NT, NC, kc, nc);
      const int gk = k0 + kc, gj = col0 + nc;
      float2 v = make_float2(0.f, 0.f);
      if (gk < kk && gj < n) {
        const long long br = (d.kb2 > 0 && gk >= d.kb2) ? (long long)d.b_r2 + (gk - d.kb2) : (long long)d.b_r + gk;
        v = a.B[br * a.ldb + d.b_c + gj];
      }
      rb[u] = v;
    }
  };
  bool ok = true;
  if (nk > 0) fetch(0);
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int s = kt & 1;
    if (kt >= 2 && !mbar_wait(smem_u32(&mbar[s]), ((kt >> 1) - 1) & 1)) {
      s_fail = 1;  // every thread sees the same timeout: the loop ends uniformly below
    }
    __syncthreads();
    if (s_fail) {
      ok = false;
      break;
    }
    float* Ah = base + s * STAGE;
    float* Al = Ah + A_TILE;
    float* Bh = Al + A_TILE;
    float* Bl = Bh + B_TILE;
    // A: 128 rows x TC_KC complex, (re, im) -> real columns 2kc, 2kc+1 of the row
#pragma unroll
    for (int u = 0; u < A_PER; ++u) {
      int r, kc;
      a_elem(tid + u * TC_NT, r, kc);
      uint2 h, lo;
      split_tf32(ra[u].x, h.x, lo.x);
      split_tf32(ra[u].y, h.y, lo.y);
      const uint32_t off = core_off(r, 2 * kc) / 4;
      *reinterpret_cast<uint2*>(Ah + off) = h;
      *reinterpret_cast<uint2*>(Al + off) = lo;
    }
    // B': the fetched complex entries split into the hi/lo tiles
#pragma unroll
    for (int u = 0; u < B_PER; ++u) {
      int kc, nc;
      b_elem(tid + u * TC_NT, NC, kc, nc);
      b_rows(Bh, Bl, kc, nc, rb[u], tid + u * TC_NT);
    }
    if (kt + 1 < nk) fetch(kt + 1);  // in flight while this chunk is multiplied
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
#pragma unroll
      for (int ks = 0; ks < TC_KR / 8; ++ks) {
        const uint32_t step = ks * 2 * LBO;  // two core matrices = 8 real k
        mma_tf32(tmem, smem_desc(ah + step), smem_desc(bh + step), TT::IDESC, (kt > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(ah + step), smem_desc(bl + step), TT::IDESC, 1u);
        mma_tf32(tmem, smem_desc(al + step), smem_desc(bh + step), TT::IDESC, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[s]))
                   : "memory");
    }
  }
  if (ok && nk > 0 && !mbar_wait(smem_u32(&mbar[(nk - 1) & 1]), ((nk - 1) >> 1) & 1)) s_fail = 1;
  __syncthreads();
  ok = ok && !s_fail;  // uniform over the block (tcgen05.ld is warp-collective)
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // let the MMAs already issued finish before the tensor memory is released
    if (nk > 0) mbar_wait(smem_u32(&mbar[(nk - 1) & 1]), ((nk - 1) >> 1) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const int row = 32 * warp + lane, gi = row0 + row;
  const int* rmap = d.rmap >= 0 ? a.maps + d.rmap : nullptr;
  const int* cmap = d.cmap >= 0 ? a.maps + d.cmap : nullptr;
  const long long orow = gi < m ? (long long)d.c_r + (rmap ? rmap[gi] : gi) : 0;
  const long long cr = (d.mc2 > 0 && gi >= d.mc2) ? (long long)d.c0_r2 + (gi - d.mc2) : (long long)d.c0_r + gi;
  if (ok) {
    float2* W = ksplit > 1 ? a.ws + (((long long)sp * a.nbatch + bb) * mmax) * nmax : nullptr;
#pragma unroll 1
    for (int c0 = 0; c0 < NR; c0 += 16) {
      uint32_t v[16];
      if (nk > 0) {
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
      if (gi < m) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gj = col0 + c0 / 2 + j;
          if (gj >= n) continue;
          const float2 acc = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
          if (W) {
            W[(long long)gi * nmax + gj] = acc;
            continue;
          }
          float2 o = cmul(a.alpha, acc);
          if (a.C0) o = cadd(o, cmul(a.beta, a.C0[cr * a.ldc0 + d.c0_c + gj]));
          a.C[orow * a.ldc + d.c_c + (cmap ? cmap[gj] : gj)] = o;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TT::TCOLS) : "memory");
}

// Sweep products on operators stored tiled (tile_operator): each pair's operator is laid out as
// blocks of 128 rows x 8 complex k, each block one contiguous 8 KB in the MMA's core-matrix
// order and zero-padded past the operator's rows and k, so a CTA's k-chunk is one sequential
// 8 KB read (the row-major operator gave 64-byte pieces of 128 rows per chunk).  The blocks come
// in by asynchronous copies (cp.async, 16 bytes per thread and instruction) into a ring of TCP_S
// raw stages, TCP_S - 1 chunks ahead of the one being multiplied; each chunk is then split from
// its raw stage into the hi/lo tiles of the 3xTF32 product (same offsets) and multiplied as in
// tc_gemm_kernel.  GemmDesc.a_r is the pair's first block and a_c its blocks per row tile.
constexpr int TCP_ARAW = TC_M * TC_KC * 8;  // bytes of one operator block (8 KB)

template <int NC> struct TcpTile {
  static constexpr int S = NC <= 32 ? 4 : 3;               // raw stages
  static constexpr int BRAW = TC_KC * NC * 8;             // bytes of one raw B stage
  static constexpr int RAW = TCP_ARAW + BRAW;             // bytes of one raw stage (a multiple of 1024)
  static constexpr size_t SMEM = (size_t)S * RAW + (size_t)2 * TcTile<NC>::STAGE * sizeof(float) + 1024;
};


constexpr int TCS_NT = 256;  // 8 warps: the splitting work is spread over twice the threads

template <int NC>
__global__ void __launch_bounds__(TCS_NT, 2) tcs_gemm_kernel(GemmArgs<float> a, int* err, int ksplit, int kc, int mmax,
                                                             int nmax) {
  using TT = TcTile<NC>;
  using TP = TcpTile<NC>;
  constexpr int NR = TT::NR, B_TILE = TT::B_TILE, STAGE = TT::STAGE, TCP_S = TP::S;
  constexpr int G = NR / 16;          // 16-column groups of the accumulator
  constexpr int GH = G / 2;           // groups per warp quarter (two warps share each TMEM lane quarter)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* base = reinterpret_cast<float*>(ring + (size_t)TCP_S * TP::RAW);  // 1024-aligned: RAW is a multiple of 1024
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int bb = blockIdx.z % a.nbatch, sp = blockIdx.z / a.nbatch;
  const GemmDesc d = a.desc[bb];
  const int n = d.n < 0 ? a.n_launch : d.n, m = d.m;
  const int kb = ksplit > 1 ? sp * kc : 0;
  const int kk = ksplit > 1 ? min(d.k, kb + kc) : d.k;  // this split covers complex k in [kb, kk)
  const int row0 = blockIdx.y * TC_M, col0 = blockIdx.x * NC;
  if (row0 >= m || col0 >= n) return;  // uniform over the block, before any tensor-memory use
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "n"(TT::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // epilogue roles: warp w reads TMEM lane quarter w % 4 (output rows) and column groups
  // [h * GH, (h + 1) * GH), h = w / 4; its row data is loaded now so its latency hides behind
  // the k loop
  const int quarter = warp & 3, half = warp >> 2;
  const int row = 32 * quarter + lane, gi = row0 + row;
  const int* rmap = d.rmap >= 0 ? a.maps + d.rmap : nullptr;
  const int* cmap = d.cmap >= 0 ? a.maps + d.cmap : nullptr;
  const long long orow = gi < m ? (long long)d.c_r + (rmap ? rmap[gi] : gi) : 0;
  const long long cr = (d.mc2 > 0 && gi >= d.mc2) ? (long long)d.c0_r2 + (gi - d.mc2) : (long long)d.c0_r + gi;
  constexpr int NCH = NC / 2;  // complex columns of this warp's half
  float2 c0v[NCH];
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int gj = col0 + half * NCH + j;
    c0v[j] = (ksplit == 1 && a.C0 && gi < m && gj < n) ? cmul(a.beta, a.C0[cr * a.ldc0 + d.c0_c + gj])
                                                       : make_float2(0.f, 0.f);
  }

  // this CTA's blocks: row tile blockIdx.y of its pair, chunks from kb / TC_KC on, rows_blk rows each
  int rows_blk;
  const float2* Ab =
      a.A + ((long long)d.a_r + tiled_block_unit((int)a.lda, d.a_c, blockIdx.y, kb / TC_KC, rows_blk)) * TILE_UNIT;
  const int nk = kk > kb ? (kk - kb + TC_KC - 1) / TC_KC : 0;
  const uint32_t ring_s = smem_u32(ring);
  // chunk kt (if any) into raw stage kt % TCP_S; always one commit group per call
  auto issue = [&](int kt) {
    if (kt < nk) {
      const int k0 = kb + kt * TC_KC;
      const uint32_t ra = ring_s + (uint32_t)((kt % TCP_S) * TP::RAW);
      unsigned char* rap = ring + (size_t)(kt % TCP_S) * TP::RAW;
      const char* src = reinterpret_cast<const char*>(Ab + (long long)kt * rows_blk * TC_KC);
#pragma unroll
      for (int i = 0; i < TCP_ARAW / (16 * TCS_NT); ++i) {
        const int o = (tid + i * TCS_NT) * 16;
        if (o < rows_blk * TC_KC * 8) cp_async16(ra + o, src + o);  // rows past a compact block: unused
      }
      for (int l = tid; l < TC_KC * NC; l += TCS_NT) {
        const int kc2 = l / NC, nc = l % NC;
        const int gk = k0 + kc2, gj = col0 + nc;
        const uint32_t off = (uint32_t)(TCP_ARAW + l * 8);
        if (gk < kk && gj < n) {
          const long long br = (d.kb2 > 0 && gk >= d.kb2) ? (long long)d.b_r2 + (gk - d.kb2) : (long long)d.b_r + gk;
          cp_async8(ra + off, a.B + br * a.ldb + d.b_c + gj);
        } else {
          *reinterpret_cast<float2*>(rap + off) = make_float2(0.f, 0.f);
        }
      }
    }
    cp_async_commit();
  };
  bool ok = true;
#pragma unroll 1
  for (int kt = 0; kt < TCP_S - 1; ++kt) issue(kt);
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int s = kt & 1;
    // raw stage (kt - 1) % TCP_S was read by every thread before the last barrier: refill it
    issue(kt + TCP_S - 1);
    cp_async_wait<TCP_S - 1>();  // this thread's copies of chunk kt have landed
    if (kt >= 2 && !mbar_wait(smem_u32(&mbar[s]), ((kt >> 1) - 1) & 1)) {
      s_fail = 1;  // every thread sees the same timeout: the loop ends uniformly below
    }
    __syncthreads();
    if (s_fail) {
      ok = false;
      break;
    }
    const unsigned char* rap = ring + (size_t)(kt % TCP_S) * TP::RAW;
    float* Ah = base + s * STAGE;
    float* Al = Ah + A_TILE;
    float* Bh = Al + A_TILE;
    float* Bl = Bh + B_TILE;
    // A: the raw block is already in the tile's core-matrix order; split each (re, im) in place
#pragma unroll
    for (int u = 0; u < TCP_ARAW / (8 * TCS_NT); ++u) {
      const int o = tid + u * TCS_NT;  // float2 index
      const float2 v = reinterpret_cast<const float2*>(rap)[o];
      uint2 h, lo;
      split_tf32(v.x, h.x, lo.x);
      split_tf32(v.y, h.y, lo.y);
      reinterpret_cast<uint2*>(Ah)[o] = h;
      reinterpret_cast<uint2*>(Al)[o] = lo;
    }
    // B': the raw chunk (row-major TC_KC x NC complex) split into the hi/lo tiles
    for (int l = tid; l < TC_KC * NC; l += TCS_NT) {
      int kc2, nc;
      b_elem(l, NC, kc2, nc);
      b_rows(Bh, Bl, kc2, nc, *reinterpret_cast<const float2*>(rap + TCP_ARAW + (kc2 * NC + nc) * 8), l);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
#pragma unroll
      for (int ks = 0; ks < TC_KR / 8; ++ks) {
        const uint32_t step = ks * 2 * LBO;  // two core matrices = 8 real k
        mma_tf32(tmem, smem_desc(ah + step), smem_desc(bh + step), TT::IDESC, (kt > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, smem_desc(ah + step), smem_desc(bl + step), TT::IDESC, 1u);
        mma_tf32(tmem, smem_desc(al + step), smem_desc(bh + step), TT::IDESC, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[s]))
                   : "memory");
    }
  }
  cp_async_wait<0>();  // no copy of this CTA is left in flight (the last groups may be empty)
  if (ok && nk > 0 && !mbar_wait(smem_u32(&mbar[(nk - 1) & 1]), ((nk - 1) >> 1) & 1)) s_fail = 1;
  __syncthreads();
  ok = ok && !s_fail;  // uniform over the block (tcgen05.ld is warp-collective)
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // let the MMAs already issued finish before the tensor memory is released
    if (nk > 0) mbar_wait(smem_u32(&mbar[(nk - 1) & 1]), ((nk - 1) >> 1) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (ok) {
    float2* W = ksplit > 1 ? a.ws + (((long long)sp * a.nbatch + bb) * mmax) * nmax : nullptr;
#pragma unroll
    for (int gq = 0; gq < GH; ++gq) {
      const int c0 = (half * GH + gq) * 16;  // real column of this group
      uint32_t v[16];
      if (nk > 0) {
        const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
      if (gi < m) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gj = col0 + c0 / 2 + j;
          if (gj >= n) continue;
          const float2 acc = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
          if (W) {
            W[(long long)gi * nmax + gj] = acc;
            continue;
          }
          const float2 o = cadd(cmul(a.alpha, acc), c0v[gq * 8 + j]);
          a.C[orow * a.ldc + d.c_c + (cmap ? cmap[gj] : gj)] = o;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TT::TCOLS) : "memory");
}

// Sweep products with the operator stored pre-split in bf16 ("bf16x3").
//
// The sweep operators U and Dm are formed once per tree and then only multiplied, so they are
// stored, block by block (128 rows x 8 complex k), as the bf16 tile hi = bf16(x) followed by the
// bf16 tile lo = bf16(x - hi) in the 16-bit K-major no-swizzle layout (8-row x 16-byte core
// matrices): one bulk copy brings a k chunk of A into shared memory exactly as the MMA reads it,
// and no thread touches A.  The block vector B is split the same way in the kernel (and
// real-expanded as in the FP32 kernels); the product accumulates hi*hi + hi*lo + lo*hi with
// kind::f16 MMAs (bf16 inputs, FP32 accumulator in tensor memory).  hi + lo represents x to
// 2^-16 relative and the dropped lo*lo term is below 2^-16, so each product carries a relative
// error of about 3 * 2^-16 against the FP32 product.  The same kernel with three terms (hi, mid,
// lo; "bf16x6") forms the six products whose term indices sum to at most 2 and keeps FP32
// accuracy (the coarse GMRES operator products).
//
// Persistent and warp-specialised, 256 threads, two CTAs per SM:
//   warp 0      producer: per k chunk one cp.async.bulk of the A block (completing on the
//               stage's full barrier with its byte count) and cp.async of the raw B chunk
//               (cp.async.mbarrier.arrive on the same barrier; one more bulk copy when the
//               chunk is contiguous), up to S stages ahead;
//   warp 1      one thread issues the chunk's three (six) MMAs once its B tiles are split, commits
//               them to the stage's empty barrier (the producer then refills the stage) and a
//               tile's last chunk to its accumulator's full barrier; two accumulators in tensor
//               memory alternate by tile, so a tile's epilogue overlaps the next tile's MMAs;
//   warps 2-3   split the raw B chunk into the stage's bf16 term B' tiles;
//   warps 4-7   epilogue: warp w owns tensor-memory lanes 32 (w % 4) .. + 31 (its 32 output
//               rows).  It copies the tile's C0 rows into its shared-memory staging
//               asynchronously while the MMAs run, then combines them with the accumulator
//               rows in place (thread = row), releases the accumulator and writes the staging
//               out along rows, so that C0 loads and C stores are coalesced.
// Every wait is bounded; a wait that gives up (or that starts after another role gave up) ends
// the role's loops, *err is set, and the copies and MMAs in flight are waited for before the
// tensor memory is released.
constexpr int TCB_NT = 256;  // 8 warps

// TERMS = 2: x = hi + lo (bf16x3, 3 products); TERMS = 3: x = hi + mid + lo, the products with
// term indices i + j <= 2 (6 products, about FP32 accuracy: "bf16x6")
template <int NC, int TERMS = 2> struct TcbTile {
  static constexpr int S = TERMS == 3 ? (NC <= 16 ? 4 : 3) : (NC <= 16 ? 6 : 5);  // stages
  static constexpr int NR = 2 * NC;                      // real output columns
  static constexpr int A_TILE = TC_M * TC_KR * 2;         // one bf16 term tile of a block (4 KB)
  static constexpr int A_BYTES = TERMS * A_TILE;          // the block's term tiles
  static constexpr int BRAW = TC_KC * NC * 8;             // raw complex B chunk
  static constexpr int BT = NR * TC_KR * 2;               // one bf16 B' tile
  static constexpr int STAGE = A_BYTES + BRAW + TERMS * BT;  // a multiple of 1024
  static constexpr int TCOLS = 2 * NR < 32 ? 32 : 2 * NR; // two accumulators
  // instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NR >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
  static constexpr int EPI_LD = NC + 2;                   // epilogue staging row (padded, 16-byte aligned), complex
  static constexpr int EPI = 4 * 32 * EPI_LD * 8;         // staging of the four epilogue warps
  static constexpr size_t SMEM = (size_t)S * STAGE + EPI + 1024;
};
static_assert(TcbTile<16>::STAGE % 1024 == 0 && TcbTile<32>::STAGE % 1024 == 0, "stage alignment");
static_assert(TcbTile<16, 3>::STAGE % 1024 == 0 && TcbTile<32, 3>::STAGE % 1024 == 0, "stage alignment");
static_assert(2 * TcbTile<16, 3>::SMEM <= 228 * 1024 && 2 * TcbTile<32, 3>::SMEM <= 228 * 1024, "two CTAs per SM");
static_assert(TcbTile<16>::A_BYTES == TC_M * TC_KC * 8, "a bf16x3 block occupies one FP32 block");

__device__ __forceinline__ void split_bf16(float x, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));  // x - h is exact in FP32
}
// x = t[0] + t[1] + ... + t[TERMS - 1] + r in bf16 terms, each the rounding of what the previous
// ones leave (every difference is exact in FP32); |r| <= 2^-(8 TERMS) |x| about
template <int TERMS>
__device__ __forceinline__ void split_terms(float x, uint32_t (&t)[TERMS]) {
#pragma unroll
  for (int i = 0; i < TERMS; ++i) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    t[i] = __bfloat16_as_ushort(h);
    x -= __bfloat162float(h);
  }
}

// tile t of a persistent launch: row tile, column tile, batch entry and k split
struct TileInfo {
  int bb, sp, rt, ct, m, n, kb, kk, nk;
  bool live;
};
__device__ __forceinline__ TileInfo tile_info(const GemmArgs<float>& a, int NC, int t, int gx, int gy, int ksplit,
                                              int kc) {
  TileInfo ti;
  const int z = t / (gx * gy), rem = t % (gx * gy);
  ti.rt = rem / gx;
  ti.ct = rem % gx;
  ti.bb = z % a.nbatch;
  ti.sp = z / a.nbatch;
  const GemmDesc& d = a.desc[ti.bb];
  ti.n = d.n < 0 ? a.n_launch : d.n;
  ti.m = d.m;
  ti.kb = ksplit > 1 ? ti.sp * kc : 0;
  ti.kk = ksplit > 1 ? min(d.k, ti.kb + kc) : d.k;
  ti.nk = ti.kk > ti.kb ? (ti.kk - ti.kb + TC_KC - 1) / TC_KC : 0;
  ti.live = ti.rt * TC_M < ti.m && ti.ct * NC < ti.n;
  return ti;
}

template <int NC, int TERMS>
__global__ void __launch_bounds__(TCB_NT, 2) tcb_gemm_kernel(GemmArgs<float> a, int* err, int ksplit, int kc,
                                                             int mmax, int nmax, int gx, int gy, int ntiles) {
  using TB = TcbTile<NC, TERMS>;
  constexpr int NR = TB::NR, STAGE = TB::STAGE, A_BYTES = TB::A_BYTES, BRAW = TB::BRAW, BT = TB::BT;
  constexpr int A_TILE = TB::A_TILE;
  constexpr int TCB_S = TB::S;
  constexpr int G = NR / 16;  // 16-column groups of an accumulator
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[TCB_S], conv[TCB_S], empty[TCB_S], accf[2], acce[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail_store;
  volatile int& s_fail = s_fail_store;
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < TCB_S; ++i) {
      mbar_init(&full[i], 33);  // the 32 producer lanes' cp.async arrivals + the bulk copies' expect_tx arrival
      mbar_init(&conv[i], 2);   // the two B-splitting warps
      mbar_init(&empty[i], 1);  // tcgen05.commit of the chunk's MMAs
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);  // tcgen05.commit of a tile's last chunk
      mbar_init(&acce[i], 4);  // the four epilogue warps
    }
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
  // bounded wait with a warp-uniform result (the warps' tcgen05.ld are warp-collective)
  auto wait = [&](uint64_t* b, uint32_t parity) -> bool {
    bool ok = !s_fail && mbar_wait(smem_u32(b), parity);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) s_fail = 1;
    return ok;
  };
  auto wait1 = [&](uint64_t* b, uint32_t parity) -> bool {  // single-thread role
    if (!s_fail && mbar_wait(smem_u32(b), parity)) return true;
    s_fail = 1;
    return false;
  };

  if (warp == 0) {
    // ---------------- producer ----------------
    long long g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const TileInfo ti = tile_info(a, NC, t, gx, gy, ksplit, kc);
      if (!ti.live) continue;
      const GemmDesc d = a.desc[ti.bb];
      int rows_blk;  // rows stored in this row tile's blocks (a multiple of 8)
      // the tiled layout in bytes: an entry takes TERMS 4-byte words (a unit: 64 entries)
      const char* Ab = reinterpret_cast<const char*>(a.A) +
                       ((long long)d.a_r + tiled_block_unit((int)a.lda, d.a_c, ti.rt, ti.kb / TC_KC, rows_blk)) *
                           (TILE_UNIT * 4 * TERMS);
      const uint32_t half = (uint32_t)rows_blk * (TC_KR * 2);  // bytes of one term tile of the block
      const int col0 = ti.ct * NC;
      for (int kt = 0; kt < ti.nk; ++kt, ++g) {
        const int st = (int)(g % TCB_S);
        if (g >= TCB_S && !wait(&empty[st], (uint32_t)(((g / TCB_S) - 1) & 1))) {
          ok = false;
          break;
        }
        unsigned char* sp = ring + (size_t)st * STAGE;
        const uint32_t rb = smem_u32(sp + A_BYTES);
        const int k0 = ti.kb + kt * TC_KC;
        // the B chunk is one contiguous 16-byte aligned run when its 8 rows lie in one segment,
        // inside the split, and are whole rows of NC columns of a B with NC columns per row
        const long long br0 = (d.kb2 > 0 && k0 >= d.kb2) ? (long long)d.b_r2 + (k0 - d.kb2) : (long long)d.b_r + k0;
        const float2* bsrc = a.B + br0 * a.ldb + d.b_c + col0;
        const bool bulk_b = k0 + TC_KC <= ti.kk && !(d.kb2 > 0 && k0 < d.kb2 && k0 + TC_KC > d.kb2) &&
                            a.ldb == NC && col0 + NC <= ti.n && (reinterpret_cast<uintptr_t>(bsrc) & 15) == 0;
        if (lane == 0) {
          // term tile i to the stage's 4 KB slot i; rows past a compact block keep stale values
          // and only feed accumulator rows that are not stored
          const char* src = Ab + (long long)kt * rows_blk * TC_KC * 4 * TERMS;
          expect_tx(&full[st], TERMS * half + (bulk_b ? (uint32_t)BRAW : 0u));
#pragma unroll
          for (int i = 0; i < TERMS; ++i) bulk_copy(smem_u32(sp) + i * A_TILE, src + i * half, half, &full[st]);
          if (bulk_b) bulk_copy(rb, bsrc, BRAW, &full[st]);
        }
        if (!bulk_b) {
          for (int l = lane; l < TC_KC * NC; l += 32) {
            const int kc2 = l / NC, nc = l % NC;
            const int gk = k0 + kc2, gj = col0 + nc;
            if (gk < ti.kk && gj < ti.n) {
              const long long br =
                  (d.kb2 > 0 && gk >= d.kb2) ? (long long)d.b_r2 + (gk - d.kb2) : (long long)d.b_r + gk;
              cp_async8z(rb + l * 8, a.B + br * a.ldb + d.b_c + gj, 8u);
            } else {
              cp_async8z(rb + l * 8, a.B, 0u);  // zero fill, nothing read
            }
          }
        }
        cp_async_arrive(&full[st]);  // every lane arrives (at once when it issued no copy)
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // no bulk copy may still be landing when the CTA ends: the last chunk of each stage has
    // completed its full barrier (at once unless a role gave up before consuming it)
    if (lane == 0)
      for (long long gg = g - TCB_S > 0 ? g - TCB_S : 0; gg < g; ++gg)
        mbar_wait(smem_u32(&full[gg % TCB_S]), (uint32_t)((gg / TCB_S) & 1));
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      long long g = 0;
      int tc = 0;  // tiles with a k range so far (they alternate between the accumulators)
      bool ok = true, issued = false;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileInfo ti = tile_info(a, NC, t, gx, gy, ksplit, kc);
        if (!ti.live || ti.nk == 0) continue;
        const int buf = tc & 1;
        if (tc >= 2 && !wait1(&acce[buf], (uint32_t)(((tc >> 1) - 1) & 1))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(buf * NR);
        for (int kt = 0; kt < ti.nk; ++kt, ++g) {
          const int st = (int)(g % TCB_S);
          const uint32_t par = (uint32_t)((g / TCB_S) & 1);
          if (!wait1(&full[st], par) || !wait1(&conv[st], par)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(ring + (size_t)st * STAGE), sb = sa + A_BYTES + BRAW;
          // the products of A term i and B term j with i + j < TERMS
          bool first = kt == 0;
#pragma unroll
          for (int i = 0; i < TERMS; ++i)
#pragma unroll
            for (int j = 0; i + j < TERMS; ++j) {
              mma_bf16(acc, smem_desc16(sa + i * A_TILE), smem_desc16(sb + j * BT), TB::IDESC, first ? 0u : 1u);
              first = false;
            }
          tc_commit(&empty[st]);
          issued = true;
        }
        if (!ok) break;
        tc_commit(&accf[buf]);
        ++tc;
      }
      // every MMA issued by this thread has completed before the tensor memory is released
      if (issued) {
        tc_commit(&fin);
        mbar_wait(smem_u32(&fin), 0);
      }
    }
  } else if (warp <= 3) {
    // ---------------- B splitters ----------------
    // Thread ct takes the chunk's entries l = ct + 64 u (BPT of them): it loads all of them
    // before it stores any, so their shared-memory latencies overlap.  Entry l is complex
    // (kc, nc) with, for lane bits ln = l % 32 and w = l / 32, nc % 4 = ln % 4, kc % 4 = ln / 4 % 4,
    // nc / 4 % 2 = ln / 16 and the rest of nc and kc from w; a lane with ln / 16 = 1 stores its
    // odd B'^T row first.  Each store instruction of a warp then writes 32 distinct banks
    // (bank ((2nc + row parity) % 8) * 4 + kc % 4).
    constexpr int BPT = TC_KC * NC / 64, NCW = NC / 8;
    const int ct = tid - 64;
    long long g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const TileInfo ti = tile_info(a, NC, t, gx, gy, ksplit, kc);
      if (!ti.live) continue;
      for (int kt = 0; kt < ti.nk; ++kt, ++g) {
        const int st = (int)(g % TCB_S);
        if (!wait(&full[st], (uint32_t)((g / TCB_S) & 1))) {
          ok = false;
          break;
        }
        unsigned char* sp = ring + (size_t)st * STAGE;
        const float2* raw = reinterpret_cast<const float2*>(sp + A_BYTES);
        unsigned char* bh = sp + A_BYTES + BRAW;  // B' term tile j at bh + j BT
        const int sw = lane >> 4;
        float2 v[BPT];
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
          const int w = (ct + 64 * u) >> 5;
          const int nc = (lane & 3) | (sw << 2) | ((w % NCW) << 3), kc2 = ((lane >> 2) & 3) | ((w / NCW) << 2);
          v[u] = raw[kc2 * NC + nc];
        }
        // complex (kc, nc) -> B'^T row 2nc: (Re b, -Im b), row 2nc+1: (Im b, Re b) at real k 2kc, 2kc+1
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
          const int w = (ct + 64 * u) >> 5;
          const int nc = (lane & 3) | (sw << 2) | ((w % NCW) << 3), kc2 = ((lane >> 2) & 3) | ((w / NCW) << 2);
          uint32_t re[TERMS], im[TERMS];
          split_terms<TERMS>(v[u].x, re);
          split_terms<TERMS>(v[u].y, im);
          // row 2nc + 1 lies 16 bytes after row 2nc in the same core matrix
          const uint32_t oa = core_off16(2 * nc, 2 * kc2) + 16u * sw, ob = oa + 16u - 32u * sw;
#pragma unroll
          for (int j = 0; j < TERMS; ++j) {
            // term j of -Im b is the sign flip of term j of Im b
            const uint32_t e = re[j] | ((im[j] ^ 0x8000u) << 16), o = im[j] | (re[j] << 16);
            *reinterpret_cast<uint32_t*>(bh + j * BT + oa) = sw ? o : e;
            *reinterpret_cast<uint32_t*>(bh + j * BT + ob) = sw ? e : o;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[st]);
      }
    }
  } else {
    // ---------------- epilogue ----------------
    constexpr int LD = TB::EPI_LD;
    const int quarter = warp & 3;
    float2* stg = reinterpret_cast<float2*>(ring + (size_t)TCB_S * STAGE) + quarter * 32 * LD;
    int tc = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const TileInfo ti = tile_info(a, NC, t, gx, gy, ksplit, kc);
      if (!ti.live) continue;
      const GemmDesc d = a.desc[ti.bb];
      const int row0 = ti.rt * TC_M + 32 * quarter, col0 = ti.ct * NC;
      const int* rmap = d.rmap >= 0 ? a.maps + d.rmap : nullptr;
      const int* cmap = d.cmap >= 0 ? a.maps + d.cmap : nullptr;
      // output and C0 rows of row row0 + lane, shuffled to the lanes that move them
      const int gl = row0 + lane;
      const long long orow_l = gl < ti.m ? (long long)d.c_r + (rmap ? rmap[gl] : gl) : 0;
      const long long cr_l = (d.mc2 > 0 && gl >= d.mc2) ? (long long)d.c0_r2 + (gl - d.mc2) : (long long)d.c0_r + gl;
      float2* W = ksplit > 1 ? a.ws + (((long long)ti.sp * a.nbatch + ti.bb) * mmax) * nmax : nullptr;
      const bool has_c0 = !W && a.C0;
      // rows move along the lanes, two complex (16 bytes) per lane when every row of C0 and of the
      // output starts on a 16-byte boundary and no column map applies, else one (8 bytes)
      const bool vec = !cmap && (col0 % 2) == 0 &&
                       (W ? (nmax % 2 == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0)
                          : (a.ldc % 2 == 0 && d.c_c % 2 == 0 && (reinterpret_cast<uintptr_t>(a.C) & 15) == 0)) &&
                       (!has_c0 || (a.ldc0 % 2 == 0 && d.c0_c % 2 == 0 && (reinterpret_cast<uintptr_t>(a.C0) & 15) == 0));
      // C0 into the staging by asynchronous copies issued while the tile's MMAs run (zero where
      // there is no C0 term or no such row / column)
      if (vec) {
        constexpr int LPR = NC / 2, RPP = 32 / LPR;  // lanes per row, rows per pass
        const int lr = lane / LPR, jc = (lane % LPR) * 2, gj = col0 + jc;
#pragma unroll 4
        for (int i = 0; i < 32 / RPP; ++i) {
          const int r = i * RPP + lr;
          const long long cr = __shfl_sync(0xffffffffu, cr_l, r);
          const uint32_t nb = (has_c0 && row0 + r < ti.m) ? (gj + 1 < ti.n ? 16u : gj < ti.n ? 8u : 0u) : 0u;
          cp_async16z(smem_u32(stg + r * LD + jc), nb ? a.C0 + cr * a.ldc0 + d.c0_c + gj : a.B, nb);
        }
      } else {
        const int lr = lane / NC, jc = lane % NC, gj = col0 + jc;
#pragma unroll 4
        for (int i = 0; i < NC; ++i) {
          const int r = i * (32 / NC) + lr;
          const long long cr = __shfl_sync(0xffffffffu, cr_l, r);
          const bool in = has_c0 && row0 + r < ti.m && gj < ti.n;
          cp_async8z(smem_u32(stg + r * LD + jc), in ? a.C0 + cr * a.ldc0 + d.c0_c + gj : a.B, in ? 8u : 0u);
        }
      }
      cp_async_commit();
      const int buf = tc & 1;
      if (ti.nk > 0) {
        if (!wait(&accf[buf], (uint32_t)((tc >> 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      cp_async_wait<0>();
      __syncwarp();
      // staging[row] = alpha * accumulator row + beta * C0 row (thread = row, 16-byte accesses)
#pragma unroll
      for (int gq = 0; gq < G; ++gq) {
        uint32_t v[16];
        if (ti.nk > 0) {
          const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * NR + gq * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(ta));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float4* q = reinterpret_cast<float4*>(stg + lane * LD + gq * 8 + 2 * j);
          const float2 a0 = make_float2(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]));
          const float2 a1 = make_float2(__uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
          float2 o0 = a0, o1 = a1;
          if (!W) {
            const float4 c = *q;
            o0 = cadd(cmul(a.alpha, a0), cmul(a.beta, make_float2(c.x, c.y)));
            o1 = cadd(cmul(a.alpha, a1), cmul(a.beta, make_float2(c.z, c.w)));
          }
          *q = make_float4(o0.x, o0.y, o1.x, o1.y);
        }
      }
      if (ti.nk > 0) {
        // the accumulator is read: the MMAs of the tile after next may overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[buf]);
        ++tc;
      }
      __syncwarp();
      // staging -> C (or the split-K workspace) along rows
      if (vec) {
        constexpr int LPR = NC / 2, RPP = 32 / LPR;
        const int lr = lane / LPR, jc = (lane % LPR) * 2, gj = col0 + jc;
#pragma unroll 8
        for (int i = 0; i < 32 / RPP; ++i) {
          const int r = i * RPP + lr, gi = row0 + r;
          const long long orow = __shfl_sync(0xffffffffu, orow_l, r);
          if (gi < ti.m && gj < ti.n) {
            const float4 o = *reinterpret_cast<const float4*>(stg + r * LD + jc);
            float2* dst = W ? W + (long long)gi * nmax + gj : a.C + orow * a.ldc + d.c_c + gj;
            if (gj + 1 < ti.n) *reinterpret_cast<float4*>(dst) = o;
            else *dst = make_float2(o.x, o.y);
          }
        }
      } else {
        const int lr = lane / NC, jc = lane % NC, gj = col0 + jc;
#pragma unroll 8
        for (int i = 0; i < NC; ++i) {
          const int r = i * (32 / NC) + lr, gi = row0 + r;
          const long long orow = __shfl_sync(0xffffffffu, orow_l, r);
          if (gi < ti.m && gj < ti.n) {
            const float2 o = stg[r * LD + jc];
            if (W)
              W[(long long)gi * nmax + gj] = o;
            else
              a.C[orow * a.ldc + d.c_c + (cmap ? cmap[gj] : gj)] = o;
          }
        }
      }
      __syncwarp();  // the staging is rewritten by the next tile
    }
  }
  __syncthreads();
  if (tid == 0 && s_fail) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TB::TCOLS) : "memory");
}

// cpsm persistent CTAs per SM (1 or 2); split K while there are fewer tiles than split_mult x
// the CTAs (0: never)
template <int NC, int TERMS>
cudaError_t launch_tcb(const GemmArgs<float>& a, int mmax, int nmax, int kmax, int* err, cudaStream_t s, int cpsm,
                       int split_mult) {
  const int gx = (nmax + NC - 1) / NC, gy = (mmax + TC_M - 1) / TC_M;
  const long long tiles = (long long)gx * gy * a.nbatch;
  const long long slots = (long long)cpsm * a.num_sms, target = split_mult * slots;
  int ksplit = 1;
  if (kmax >= 8 * TC_KC && a.ws && tiles < target) {
    ksplit = (int)((target + tiles - 1) / tiles);
    ksplit = ksplit < kmax / (4 * TC_KC) ? ksplit : kmax / (4 * TC_KC);
    ksplit = ksplit < 16 ? ksplit : 16;
    while (ksplit > 1 && (long long)ksplit * a.nbatch * mmax * nmax > a.ws_elems) --ksplit;
  }
  int kc = kmax;
  if (ksplit > 1) {
    kc = (kmax + ksplit - 1) / ksplit;
    kc = (kc + TC_KC - 1) / TC_KC * TC_KC;
    ksplit = (kmax + kc - 1) / kc;
  }
  const long long ntiles = tiles * ksplit;
  if (ntiles == 0) return cudaSuccess;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)(ntiles < slots ? ntiles : slots);
  tcb_gemm_kernel<NC, TERMS><<<grid, TCB_NT, TcbTile<NC, TERMS>::SMEM, s>>>(a, err, ksplit, kc, mmax, nmax, gx, gy,
                                                                            (int)ntiles);
  note_launch();
  if (ksplit > 1) return splitk_reduce(a, ksplit, mmax, nmax, s);
  return cudaGetLastError();
}

template <int NC>
constexpr size_t tc_gemm_smem() { return (size_t)2 * TcTile<NC>::STAGE * sizeof(float) + 1024; }

// split K until about split_mult CTAs per SM are busy (a CTA streams its k range serially;
// 0: never split)
template <int NC, bool PIPE>
cudaError_t launch_tc(const GemmArgs<float>& a, int mmax, int nmax, int kmax, int* err, cudaStream_t s,
                      int split_mult) {
  const int gx = (nmax + NC - 1) / NC, gy = (mmax + TC_M - 1) / TC_M;
  const long long blocks = (long long)gx * gy * a.nbatch;
  const long long target = (long long)split_mult * a.num_sms;
  int ksplit = 1;
  if (kmax >= 8 * TC_KC && a.ws && blocks < target) {
    ksplit = (int)((target + blocks - 1) / blocks);
    ksplit = ksplit < kmax / (4 * TC_KC) ? ksplit : kmax / (4 * TC_KC);
    ksplit = ksplit < 16 ? ksplit : 16;
    while (ksplit > 1 && ((long long)ksplit * a.nbatch > 65535 ||
                          (long long)ksplit * a.nbatch * mmax * nmax > a.ws_elems))
      --ksplit;
  }
  int kc = kmax;
  if (ksplit > 1) {
    kc = (kmax + ksplit - 1) / ksplit;
    kc = (kc + TC_KC - 1) / TC_KC * TC_KC;
    ksplit = (kmax + kc - 1) / kc;
  }
  if ((long long)a.nbatch * ksplit > 65535) return cudaErrorInvalidValue;
  dim3 grid(gx, gy, a.nbatch * ksplit);
  if constexpr (PIPE) tcs_gemm_kernel<NC><<<grid, TCS_NT, TcpTile<NC>::SMEM, s>>>(a, err, ksplit, kc, mmax, nmax);
  else tc_gemm_kernel<NC><<<grid, TC_NT, tc_gemm_smem<NC>(), s>>>(a, err, ksplit, kc, mmax, nmax);
  note_launch();
  if (ksplit > 1) return splitk_reduce(a, ksplit, mmax, nmax, s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tile autotuner
// A launch configuration of one kernel family: column-tile width nc (complex columns), CTAs per
// SM of the persistent bf16 kernels (tcb: two terms, tcb6: three), and the split-K target
// (multiples of the CTAs or SMs).
// Candidate 0 of every list is the fixed heuristic (HPS_TUNE_OFF).
enum TuneFamily { TF_TC = 0, TF_TCS = 1, TF_TCB = 2, TF_TCB6 = 3 };
const char* const kFamilyName[4] = {"tc", "tcs", "tcb", "tcb6"};
struct TuneCand {
  int nc, cpsm, split;
};

// the narrowest column tile of the family that covers nmax in one tile
int natural_nc(int fam, int nmax) {
  if (fam == TF_TCB || fam == TF_TCB6) return nmax <= 16 ? 16 : 32;
  return nmax <= 16 ? 16 : nmax <= 32 ? 32 : 64;
}

std::vector<TuneCand> tune_candidates(int fam, int nmax) {
  const int nc0 = natural_nc(fam, nmax), nc1 = nc0 / 2;  // half-width tiles: twice the tiles
  std::vector<TuneCand> v;
  if (fam == TF_TCB || fam == TF_TCB6) {
    v = {{nc0, 2, 1}, {nc0, 2, 0}, {nc0, 1, 1}, {nc0, 2, 2}};
    if (nc1 >= 16) {
      v.push_back({nc1, 2, 1});
      v.push_back({nc1, 2, 0});
    }
  } else {
    const int def = fam == TF_TCS ? 2 : 3;
    v = {{nc0, 1, def}, {nc0, 1, 0}, {nc0, 1, 2 * def}};
    if (nc1 >= 16) {
      v.push_back({nc1, 1, def});
      v.push_back({nc1, 1, 0});
    }
  }
  return v;
}

cudaError_t run_candidate(int fam, const TuneCand& t, const GemmArgs<float>& a, int mmax, int nmax, int kmax, int* err,
                          cudaStream_t s) {
  if (fam == TF_TCB) {
    if (t.nc == 16) return launch_tcb<16, 2>(a, mmax, nmax, kmax, err, s, t.cpsm, t.split);
    return launch_tcb<32, 2>(a, mmax, nmax, kmax, err, s, t.cpsm, t.split);
  }
  if (fam == TF_TCB6) {
    if (t.nc == 16) return launch_tcb<16, 3>(a, mmax, nmax, kmax, err, s, t.cpsm, t.split);
    return launch_tcb<32, 3>(a, mmax, nmax, kmax, err, s, t.cpsm, t.split);
  }
  if (a.nbatch > 65535) return cudaErrorInvalidValue;
  if (fam == TF_TCS) {
    if (t.nc == 16) return launch_tc<16, true>(a, mmax, nmax, kmax, err, s, t.split);
    if (t.nc == 32) return launch_tc<32, true>(a, mmax, nmax, kmax, err, s, t.split);
    return launch_tc<64, true>(a, mmax, nmax, kmax, err, s, t.split);
  }
  if (t.nc == 16) return launch_tc<16, false>(a, mmax, nmax, kmax, err, s, t.split);
  if (t.nc == 32) return launch_tc<32, false>(a, mmax, nmax, kmax, err, s, t.split);
  return launch_tc<64, false>(a, mmax, nmax, kmax, err, s, t.split);
}

using TuneKey = std::tuple<int, int, int, int, int, int>;  // family, mmax, nmax, kmax, nbatch, SMs
struct TuneEntry {
  int idx;
  float ms0, ms_best;  // two launches of candidate 0 and of the winner
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;

// Times each candidate (one untimed launch, then two between events) and returns the winner;
// -1 when a launch or the timing failed (nothing cached).
int tune_shape(int fam, const std::vector<TuneCand>& cands, const GemmArgs<float>& a, int mmax, int nmax, int kmax,
               int* err, cudaStream_t s, float& ms0, float& ms_best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return -1;
  }
  int best = -1;
  ms0 = ms_best = 0.f;
  for (size_t i = 0; i < cands.size(); ++i) {
    if (run_candidate(fam, cands[i], a, mmax, nmax, kmax, err, s) != cudaSuccess) {
      cudaGetLastError();
      if (i == 0) break;  // the heuristic itself failed: leave the error to the caller's launch
      continue;
    }
    cudaEventRecord(e0, s);
    cudaError_t r = run_candidate(fam, cands[i], a, mmax, nmax, kmax, err, s);
    if (r == cudaSuccess) r = run_candidate(fam, cands[i], a, mmax, nmax, kmax, err, s);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (r != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (i == 0) ms0 = ms;
    if (best < 0 || ms < ms_best) {
      best = (int)i;
      ms_best = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

cudaError_t tuned_launch(int fam, const GemmArgs<float>& a, int mmax, int nmax, int kmax, int* err, cudaStream_t s) {
  const std::vector<TuneCand> cands = tune_candidates(fam, nmax);
  if (a.tune >= HPS_TUNE_FORCE)
    return run_candidate(fam, cands[(size_t)(a.tune - HPS_TUNE_FORCE) % cands.size()], a, mmax, nmax, kmax, err, s);
  if (a.tune != HPS_TUNE_ON) return run_candidate(fam, cands[0], a, mmax, nmax, kmax, err, s);
  const TuneKey key{fam, mmax, nmax, kmax, a.nbatch, a.num_sms};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return run_candidate(fam, cands[it->second.idx], a, mmax, nmax, kmax, err, s);
  }
  // tuning re-runs the product: only outside capture, and only when C aliases neither input
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;
  }
  const void* c = a.C;
  if (cs != cudaStreamCaptureStatusNone || c == (const void*)a.C0 || c == (const void*)a.B || c == (const void*)a.A)
    return run_candidate(fam, cands[0], a, mmax, nmax, kmax, err, s);
  float ms0 = 0.f, msb = 0.f;
  const int best = tune_shape(fam, cands, a, mmax, nmax, kmax, err, s, ms0, msb);
  if (best < 0) return run_candidate(fam, cands[0], a, mmax, nmax, kmax, err, s);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = TuneEntry{best, ms0, msb};
  }
  return run_candidate(fam, cands[best], a, mmax, nmax, kmax, err, s);  // the call's result is the winner's
}

}  // namespace

cudaError_t launch_tc_gemm(const GemmArgs<float>& a, int mmax, int nmax, int kmax, int* err, cudaStream_t s) {
  if (a.nbatch <= 0 || mmax <= 0 || nmax <= 0) return cudaSuccess;
  if (a.nbatch > 65535) return cudaErrorInvalidValue;
  return tuned_launch(TF_TC, a, mmax, nmax, kmax, err, s);
}

cudaError_t launch_tc_gemm_tiled(const GemmArgs<float>& a, int mmax, int nmax, int kmax, int terms, int* err,
                                 cudaStream_t s) {
  if (a.nbatch <= 0 || mmax <= 0 || nmax <= 0) return cudaSuccess;
  if (terms == 2) return tuned_launch(TF_TCB, a, mmax, nmax, kmax, err, s);  // wide B: tiles side by side
  if (terms == 3) return tuned_launch(TF_TCB6, a, mmax, nmax, kmax, err, s);
  if (a.nbatch > 65535) return cudaErrorInvalidValue;
  return tuned_launch(TF_TCS, a, mmax, nmax, kmax, err, s);
}

int autotune_table(char* buf, int len) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string out;
  for (const auto& kv : g_tune) {
    const auto& k = kv.first;
    const TuneCand t = tune_candidates(std::get<0>(k), std::get<2>(k))[kv.second.idx];
    char line[192];
    snprintf(line, sizeof line, "%s m=%d n=%d k=%d batch=%d sms=%d -> #%d nc=%d cta/sm=%d split=%d; %.4f -> %.4f ms\n",
             kFamilyName[std::get<0>(k)], std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k),
             std::get<5>(k), kv.second.idx, t.nc, t.cpsm, t.split, kv.second.ms0 / 2, kv.second.ms_best / 2);
    out += line;
  }
  if (buf && len > 0) {
    const size_t n = out.size() < (size_t)(len - 1) ? out.size() : (size_t)(len - 1);
    out.copy(buf, n);
    buf[n] = 0;
  }
  return (int)g_tune.size();
}

void autotune_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

// Block (P, rt, kt) of the tiled layout and the entry w of that block for entry l of the whole
// layout (entries in layout order: a unit of 64 entries = 512 bytes in both formats).
__device__ __forceinline__ void tiled_entry(long long l, int rows, int nrt, int nkt, long long pair_entries,
                                            long long& blk_entry, int& P, int& rt, int& kt, int& w) {
  P = (int)(l / pair_entries);
  const long long off = l % pair_entries;
  const long long full = (long long)(nrt - 1) * nkt * (TC_M * TC_KC);  // entries of the full row tiles
  int bs;
  if (off < full) {
    bs = TC_M * TC_KC;
    rt = (int)(off / ((long long)nkt * bs));
    const long long rem = off % ((long long)nkt * bs);
    kt = (int)(rem / bs);
    w = (int)(rem % bs);
  } else {
    bs = tiled_last_rows(rows) * TC_KC;
    rt = nrt - 1;
    kt = (int)((off - full) / bs);
    w = (int)((off - full) % bs);
  }
  blk_entry = l - w;  // first entry of the block
}

// FP32 blocks: entry w = float2 w of the block in core_off order
__global__ void tile_operator_kernel(float2* __restrict__ TL, const float2* __restrict__ A, int npairs, int rows,
                                     int K, int lda, long long pair_stride, int nrt, int nkt, long long pair_entries) {
  const long long tot = (long long)npairs * pair_entries;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    long long be;
    int P, rt, kt, w;
    tiled_entry(l, rows, nrt, nkt, pair_entries, be, P, rt, kt, w);
    // invert core_off(r, 2 kc) / 8: row group r/8 (SBO = 512 B), k group (2 kc)/4 (LBO = 128 B),
    // row r%8 (16 B), pair (2 kc)%4 / 2 (8 B)
    const int byte = w * 8;
    const int rg = byte / (int)SBO, rem = byte % (int)SBO;
    const int kg = rem / (int)LBO, rem2 = rem % (int)LBO;
    const int r = rg * 8 + rem2 / 16, kc = kg * 2 + (rem2 % 16) / 8;
    const int gi = rt * TC_M + r, gk = kt * TC_KC + kc;
    TL[l] = (gi < rows && gk < K) ? A[(long long)P * pair_stride + (long long)gi * lda + gk] : make_float2(0.f, 0.f);
  }
}

// bf16x3 blocks: [hi tile | lo tile], each rows_blk x 16 real k of bf16 in the 16-bit core-matrix
// order; one 32-bit word = the (Re, Im) pair of one complex entry, entry w = word w of both tiles
__global__ void tile_operator_bf16x3_kernel(uint32_t* __restrict__ TL, const float2* __restrict__ A, int npairs,
                                            int rows, int K, int lda, long long pair_stride, int nrt, int nkt,
                                            long long pair_entries) {
  const long long tot = (long long)npairs * pair_entries;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    long long be;
    int P, rt, kt, w;
    tiled_entry(l, rows, nrt, nkt, pair_entries, be, P, rt, kt, w);
    const int rows_blk = rt < nrt - 1 ? TC_M : tiled_last_rows(rows);
    // invert core_off16(r, 2 kc) / 4: row group r/8 (SBO16 = 64 words), k group (2 kc)/8
    // (LBO16 = 32 words), row r%8 (4 words), pair kc%4
    const int rg = w / 64, kg = (w % 64) / 32, wi = w % 32;
    const int r = rg * 8 + wi / 4, kc = kg * 4 + wi % 4;
    const int gi = rt * TC_M + r, gk = kt * TC_KC + kc;
    const float2 x = (gi < rows && gk < K) ? A[(long long)P * pair_stride + (long long)gi * lda + gk] : make_float2(0.f, 0.f);
    uint32_t rh, rl, ih, il;
    split_bf16(x.x, rh, rl);
    split_bf16(x.y, ih, il);
    uint32_t* blk = TL + 2 * be;  // a block of e entries takes 2e words
    blk[w] = rh | (ih << 16);
    blk[rows_blk * TC_KC + w] = rl | (il << 16);
  }
}

// bf16x6 blocks: [hi | mid | lo] tiles of the same layout, one word per entry in each
__global__ void tile_operator_bf16x6_kernel(uint32_t* __restrict__ TL, const float2* __restrict__ A, int npairs,
                                            int rows, int K, int lda, long long pair_stride, int nrt, int nkt,
                                            long long pair_entries) {
  const long long tot = (long long)npairs * pair_entries;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < tot; l += (long long)gridDim.x * blockDim.x) {
    long long be;
    int P, rt, kt, w;
    tiled_entry(l, rows, nrt, nkt, pair_entries, be, P, rt, kt, w);
    const int rows_blk = rt < nrt - 1 ? TC_M : tiled_last_rows(rows);
    const int rg = w / 64, kg = (w % 64) / 32, wi = w % 32;
    const int r = rg * 8 + wi / 4, kc = kg * 4 + wi % 4;
    const int gi = rt * TC_M + r, gk = kt * TC_KC + kc;
    const float2 x = (gi < rows && gk < K) ? A[(long long)P * pair_stride + (long long)gi * lda + gk] : make_float2(0.f, 0.f);
    uint32_t re[3], im[3];
    split_terms<3>(x.x, re);
    split_terms<3>(x.y, im);
    uint32_t* blk = TL + 3 * be;  // a block of e entries takes 3e words
#pragma unroll
    for (int i = 0; i < 3; ++i) blk[i * rows_blk * TC_KC + w] = re[i] | (im[i] << 16);
  }
}

template <typename Kern, typename T>
cudaError_t launch_tile(Kern kern, T* TL, const float2* A, int npairs, int rows, int K, int lda, long long pair_stride,
                        cudaStream_t s) {
  const int nrt = tiled_row_tiles(rows), nkt = (K + TC_KC - 1) / TC_KC;
  const long long pair_entries = tiled_pair_units(rows, K) * TILE_UNIT;
  const long long tot = (long long)npairs * pair_entries;
  long long blocks = (tot + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (blocks < 1) return cudaSuccess;
  kern<<<(int)blocks, 256, 0, s>>>(TL, A, npairs, rows, K, lda, pair_stride, nrt, nkt, pair_entries);
  note_launch();
  return cudaGetLastError();
}

cudaError_t tile_operator(float2* TL, const float2* A, int npairs, int rows, int K, int lda, long long pair_stride,
                          cudaStream_t s) {
  return launch_tile(tile_operator_kernel, TL, A, npairs, rows, K, lda, pair_stride, s);
}

cudaError_t tile_operator_bf16x3(float2* TL, const float2* A, int npairs, int rows, int K, int lda,
                                 long long pair_stride, cudaStream_t s) {
  return launch_tile(tile_operator_bf16x3_kernel, reinterpret_cast<uint32_t*>(TL), A, npairs, rows, K, lda,
                     pair_stride, s);
}

cudaError_t tile_operator_bf16x6(void* TL, const float2* A, int npairs, int rows, int K, int lda,
                                 long long pair_stride, cudaStream_t s) {
  return launch_tile(tile_operator_bf16x6_kernel, static_cast<uint32_t*>(TL), A, npairs, rows, K, lda, pair_stride,
                     s);
}

void optin_tc() {
  smem_optin(tc_gemm_kernel<16>);
  smem_optin(tc_gemm_kernel<32>);
  smem_optin(tc_gemm_kernel<64>);
  smem_optin(tcb_gemm_kernel<16, 2>);
  smem_optin(tcb_gemm_kernel<32, 2>);
  smem_optin(tcb_gemm_kernel<16, 3>);
  smem_optin(tcb_gemm_kernel<32, 3>);
  smem_optin(tcs_gemm_kernel<16>);
  smem_optin(tcs_gemm_kernel<32>);
  smem_optin(tcs_gemm_kernel<64>);
}

}  // namespace hps
