// k-space part of E on the tcgen05 tensor cores (sm_103a): E_k = A A^T over the light
// tail of the k-vector table, from 16-bit planes of each FP32 operand value.
//
// The heaviest k-vectors (the head) are summed in FP64 by a SIMT kernel beforehand; these
// kernels add the tail.  The k-vectors are sorted by decreasing weight W_K and every
// product of a column is bounded by its W_K, so the tail needs fewer bits as it goes; the
// host picks per 64-column K-block (a cos or sin half of 64 k-vectors):
//   six BF16 products a0 b0 + a0 b1 + a1 b0 + a0 b2 + a1 b1 + a2 b0 (a = a0 + a1 + a2,
//     ~2^-24 of each product), for the heavier part;
//   three FP16 products h0 g0 + h0 g1 + h1 g0 of the block's power-of-two scaled values
//     (x = h0 + h1, within 5 x 2^-22), or one, h0 g0 (within 2^-10 + 2^-23), or, for the
//     lightest blocks, one E4M3 product (within 0.13),
// such that each reduced group's summed weight times its bound stays below 1e-8 (E
// entries are O(1)).  BF16 x BF16, FP16 x FP16 and E4M3 x E4M3 products are exact in the
// FP32 accumulator.
//
// Tiles of 256 x 256 outputs of the lower triangle, one CTA each.  Warp roles: TMA producer, single-thread MMA issuer, eight epilogue warps.
// All 512 TMEM columns hold two M = 128, N = 256 FP32 accumulators.  After each
// accumulation chunk of the host's schedule the MMAs pause while the epilogue adds the
// accumulator (times the chunk's scale) into the tile's running hi / lo floats by an
// error-free two-sum; the last chunk adds hi + lo + the accumulator to the head (float
// pairs, float arithmetic only) and writes float E (or the head).
//
// Every wait is bounded: on timeout the kernel records an error code and leaves; the
// host reports a CPM_ECUDA-class failure instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "async_copy.cuh"
#include "cpm_internal.cuh"

namespace cpm {

namespace {

constexpr int kTile = 128;           // output tile edge
constexpr int kBlockK = 64;          // operand columns per K-block of the schedule

// Shared-memory matrix descriptor: K-major tile, 128-byte swizzle, rows of 128 B,
// 8-row groups 1024 B apart (SBO), version 1, layout type 2 (SWIZZLE_128B).
template <int BK>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // K-major tile, rows of BK * 2 bytes, 8-row groups SBO apart, version 1, swizzle
  // 128 B (layout type 2) for BK = 64 or 64 B (layout type 4) for BK = 32
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);     // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused when swizzled)
  d |= (uint64_t)((8 * BK * 2) >> 4) << 32;    // stride byte offset: 8 rows
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)(BK == 64 ? 2 : 4) << 61;     // swizzle mode
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A and B both K-major, M = 128, N = n;
// operand type BF16 (bf16 = true) or FP16.
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int n) {
  return (1u << 4) | (bf16 ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTile >> 4) << 24);
}

// Instruction descriptor, kind::f8f6f4: D = F32, A = B = E4M3 (format 0), both K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_f8(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

#define TMEM_LD32(taddr, r)                                                                  \
  asm volatile(                                                                              \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"   \
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];" \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),  \
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),           \
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),        \
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),        \
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),        \
        "=r"(r[31])                                                                          \
      : "r"(taddr))

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tri_tile(int t, int& I, int& J) {
  int r = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  I = r;
  J = t - r * (r + 1) / 2;
}

// ---- the tile kernel ------------------------------------------------------------------
//
// The whole of TMEM holds one 256 x 256 output tile: two M = 128, N = 256 accumulators
// (rows i0 .. i0 + 127 and i0 + 128 .. i0 + 255); against 128 x 128 tiles this halves the
// operand bytes per MMA, which is what limits these stages.
//   SIX = true (BF16, the six-product K-blocks): stages of 32 columns of planes 0-2 for the
//     tile's 256 rows and 256 columns (96 KB, 24 MMAs of 128 x 256 x 16); two stages.
//   SIX = false (FP16 / FP8): three-product stages (32 columns of planes 0 and 1, 64 KB,
//     12 MMAs), then one-product FP16 stages (64 columns of plane 0, 64 KB, 8 MMAs), then
//     FP8 stages (the 128 columns of one [cos | sin] pair, 64 KB, 8 MMAs); three stages.
// The tensor cores' FP32 adds lose ~0.1 ulp each on average, not centred, so the
// accumulator is drained after each accumulation chunk: the MMAs pause while the
// epilogue adds it, by an error-free two-sum, into the tile's running hi / lo floats in
// the SM's 512 KB scratch slot (each thread's entries laid out for whole-warp 512-byte
// accesses; small enough for all SMs' slots to stay in L2).  The head (float pairs) is
// touched once per tile.  Off the diagonal the k-space terms oscillate in sign; the
// diagonal, where every term is positive, takes the exact weight sum (range_weight, FP64
// on the host, as a float pair).  Eight
// epilogue warps: TMEM lane quarter warp % 4, column half (warp - 2) / 4.
constexpr int kStripTile = 256;
constexpr int kStripThreads = 320;  // 10 warps: TMA, MMA, 8 epilogue

template <bool SIX>
struct StripCfg {
  static constexpr int kStages = SIX ? 2 : 3;
  static constexpr int kStageBytes = (SIX ? 96 : 64) * 1024;
  static constexpr int kPlanes = SIX ? 3 : 2;   // planes of a narrow (32-column) stage
  static constexpr int kProds = SIX ? 6 : 3;    // products of a narrow stage
};

struct StripArgs {
  int n, npad;
  int tiles;      // lower-triangle 256 x 256 tiles
  int kb_begin;   // first K-block
  int kb_end;     // one past the last K-block
  int kb3_end;    // SIX = false: K-blocks before this take three products, the rest one,
  int kb8_begin;  //   from this one (even) on in FP8
  int kb_col0;    // the operand planes start at this K-block
  const uint32_t* chunk_end;  // bit per K-block: an accumulation chunk ends after it
  const int* kexp;            // per K-block: FP16 blocks hold 2^kexp a (0 for BF16 blocks)
  float* scratch; // per SM 2 x 65,536 floats (the tile's running hi / lo sums)
  int scratch_slots;  // SM slots in scratch (%nsmid)
  float2* head;   // [n][ldh] head + everything before kb_begin as float pairs (hi, lo),
                  //   lower triangle
  int64_t ldh;
  float* E;       // float E, or null: the sum goes back into head (FP64)
  int64_t ldE;
  int* err;
  int diag_exact;  // the diagonal takes w_diag in place of its accumulated sum
  float wd_hi, wd_lo;  // sum of W_K over the launch's k-vectors, as a float pair
  const uint32_t* tile_map;  // tile t -> (I << 16) | J, or null: row-major triangle order
};

// One epilogue thread's 32 final tail values (row `row`, columns jb .. jb + 31), each a
// float pair (th, tl), plus the head: the head segment (float pairs, ~2^-48 of each
// entry) is loaded whole before any store (16-byte vectors where the segment lies below
// the diagonal and inside n); the pairs meet in an error-free two-sum of the high parts
// and a rounded add of the low ones, then one renormalising step.  The sum goes to float
// E (the high part: the float nearest the pair), or back to the head without E.  The
// diagonal entry takes the exact weight sum.  Float arithmetic only: this GPU runs FP64
// at 1/64 of the float rate, and this runs once for every entry of every tile.
__device__ __forceinline__ void strip_final(const StripArgs& a, const float (&th)[32],
                                            const float (&tl)[32], int row, int jb) {
  const int jmax = min(a.n - 1, row);
  if (jb > jmax) return;
  float2* hp = a.head + (int64_t)row * a.ldh + jb;
  const bool full = jb + 31 <= jmax;
  float hh[32], hl[32];
  if (full) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const float4 x = reinterpret_cast<const float4*>(hp)[u];
      hh[2 * u] = x.x;
      hl[2 * u] = x.y;
      hh[2 * u + 1] = x.z;
      hl[2 * u + 1] = x.w;
    }
  } else {
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const float2 x = jb + t <= jmax ? hp[t] : make_float2(0.f, 0.f);
      hh[t] = x.x;
      hl[t] = x.y;
    }
  }
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const bool dg = a.diag_exact && jb + t == row;
    const float bh = dg ? a.wd_hi : th[t], bl = dg ? a.wd_lo : tl[t];
    const float s = __fadd_rn(hh[t], bh);
    const float bb = __fsub_rn(s, hh[t]);
    const float e = __fadd_rn(__fsub_rn(hh[t], __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    const float lo = __fadd_rn(__fadd_rn(hl[t], bl), e);
    hh[t] = __fadd_rn(s, lo);
    hl[t] = __fsub_rn(lo, __fsub_rn(hh[t], s));
  }
  if (a.E) {
    float* ep = a.E + (int64_t)row * a.ldE + jb;
    if (full) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        reinterpret_cast<float4*>(ep)[u] =
            make_float4(hh[4 * u], hh[4 * u + 1], hh[4 * u + 2], hh[4 * u + 3]);
    } else {
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (jb + t <= jmax) ep[t] = hh[t];
    }
  } else if (full) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
      reinterpret_cast<float4*>(hp)[u] =
          make_float4(hh[2 * u], hl[2 * u], hh[2 * u + 1], hl[2 * u + 1]);
  } else {
#pragma unroll
    for (int t = 0; t < 32; ++t)
      if (jb + t <= jmax) hp[t] = make_float2(hh[t], hl[t]);
  }
}

// The running sums of the tiles in the SMs' scratch slots (78 MB for 152 SMs) are read
// and written with an evict-last L2 policy, so that the operand streams, which pass
// through L2 once per tile, do not push them out to DRAM between drains.
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_keep(const float4* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_keep(float4* p, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}

// The final chunk's tail of one group of 32 accumulators: the running (hi, lo) sums of
// the earlier chunks (ci > 0) plus the accumulator times its scale, by a two-sum.
__device__ __forceinline__ void final_tail(bool earlier, const float4* hi4, const float4* lo4,
                                           int grp, const uint32_t (&acc)[32], float scale,
                                           uint64_t keep, float (&th)[32], float (&tl)[32]) {
  if (earlier) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 a4 = ld_keep(hi4 + grp + u * 32, keep), b4 = ld_keep(lo4 + grp + u * 32, keep);
      th[4 * u] = a4.x, th[4 * u + 1] = a4.y, th[4 * u + 2] = a4.z, th[4 * u + 3] = a4.w;
      tl[4 * u] = b4.x, tl[4 * u + 1] = b4.y, tl[4 * u + 2] = b4.z, tl[4 * u + 3] = b4.w;
    }
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const float v = __uint_as_float(acc[t]) * scale;
      const float s = __fadd_rn(th[t], v);
      const float bb = __fsub_rn(s, th[t]);
      const float e = __fadd_rn(__fsub_rn(th[t], __fsub_rn(s, bb)), __fsub_rn(v, bb));
      th[t] = s;
      tl[t] = __fadd_rn(tl[t], e);
    }
  } else {
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      th[t] = __uint_as_float(acc[t]) * scale;
      tl[t] = 0.f;
    }
  }
}

// Tile geometry: lower-triangle tile `tile` (row-major over the triangle).
struct StripTile {
  int i0, j0, rb, cb;
  bool diag;
  __device__ StripTile(int tile, int npad, const uint32_t* map) {
    int I, J;
    if (map) {
      const uint32_t v = map[tile];
      I = (int)(v >> 16);
      J = (int)(v & 0xffffu);
    } else {
      tri_tile(tile, I, J);
    }
    i0 = I * kStripTile;
    j0 = J * kStripTile;
    diag = I == J;
    // row and column halves inside the padded operand (npad is a multiple of 128)
    rb = i0 + kTile < npad ? 2 : 1;
    cb = j0 + kTile < npad ? 2 : 1;
  }
};

// The loads of a wide (one-plane, 128-byte-row) stage: A half r at r x 16 KB, B halves
// at 32 KB and 48 KB.
__device__ __forceinline__ void wide_loads(uint8_t* st, const CUtensorMap* map, uint64_t* bar,
                                           int x, const StripTile& tg) {
  constexpr int kWide = kTile * 64 * 2;
  mbar_expect_tx(bar, (tg.rb + tg.cb) * kWide);
  for (int r = 0; r < tg.rb; ++r) tma_load_2d(st + r * kWide, map, bar, x, tg.i0 + r * kTile);
  for (int c = 0; c < tg.cb; ++c)
    tma_load_2d(st + 2 * kWide + c * kWide, map, bar, x, tg.j0 + c * kTile);
}

// Each CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... (one, when the grid covers
// the tiles); the ring's stage count and the accumulator's chunk count run on across
// tiles.  The scratch slot is the SM's: its shared memory and TMEM admit one CTA of this
// kernel per SM at a time.
template <bool SIX>
__global__ void __launch_bounds__(kStripThreads, 1)
k_ek_strip(const __grid_constant__ CUtensorMap map0w, const __grid_constant__ CUtensorMap map0n,
           const __grid_constant__ CUtensorMap map1n, const __grid_constant__ CUtensorMap map2n,
           const __grid_constant__ CUtensorMap map8, StripArgs args) {
  // map0w: plane 0 in 128 x 64 boxes (128-byte swizzle); map0n / map1n / map2n: planes
  // 0-2 in 128 x 32 boxes (64-byte swizzle); map8: the FP8 plane in 128 x 128 boxes
  // (128-byte swizzle)
  using Cfg = StripCfg<SIX>;
  constexpr int kStages = Cfg::kStages, kStageBytes = Cfg::kStageBytes;
  constexpr int P = Cfg::kPlanes;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* ring = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages];
  __shared__ __align__(8) uint64_t acc_full, acc_empty;
  __shared__ uint32_t tmem_base_s;
  constexpr int kNarrow = kTile * 32 * 2, kWide = kTile * 64 * 2;  // 8 KB and 16 KB tiles

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // narrow stages (two per K-block), then wide FP16 ones (one per one-product K-block),
  // then FP8 ones (one per [cos | sin] pair of one-product K-blocks); the same for every
  // tile
  const int nnarrow =
      2 * (SIX ? args.kb_end - args.kb_begin
               : max(0, min(args.kb_end, args.kb3_end) - args.kb_begin));
  const int kb1 = max(args.kb_begin, args.kb3_end);
  const int kb8 = SIX ? args.kb_end : max(args.kb_begin, args.kb8_begin);
  const int nwide = SIX ? 0 : max(0, min(args.kb_end, kb8) - kb1);
  const int t8 = nnarrow + nwide;  // first FP8 stage
  const int nst = t8 + (SIX ? 0 : max(0, args.kb_end - kb8) / 2);
  // K-block of stage t (an FP8 stage: the second of its pair), and whether stage t is its
  // last
  auto stage_block = [&](int t, bool& last_of_block) {
    if (t < nnarrow) {
      last_of_block = (t & 1) != 0;
      return args.kb_begin + t / 2;
    }
    last_of_block = true;
    if (t < t8) return kb1 + (t - nnarrow);
    return kb8 + 2 * (t - t8) + 1;
  };
  // an accumulation chunk ends with stage t: the tile's last stage, or the last stage of
  // a K-block whose chunk bit is set
  auto chunk_ends = [&](int t) {
    if (t + 1 == nst) return true;
    bool last;
    const int g = stage_block(t, last);
    return last && ((args.chunk_end[g >> 5] >> (g & 31)) & 1u) != 0u;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_addr(&tmem_base_s))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const int tile0 = (int)blockIdx.x;
  const int tstep = (int)gridDim.x;

  if (warp == 0) {
    // ---- TMA producer ------------------------------------------------------------
    if (lane == 0) {
      uint32_t g = 0;  // stages issued by this CTA
      bool ok = true;
      for (int tile = tile0; tile < args.tiles && ok; tile += tstep) {
        const StripTile tg(tile, args.npad, args.tile_map);
        for (int t = 0; t < nst; ++t, ++g) {
          const int s = g % kStages;
          ok = mbar_wait(&empty_bar[s], ((g / kStages) & 1) ^ 1, args.err, 11);
          if (!ok) break;
          uint8_t* st = ring + s * kStageBytes;
          if (t < nnarrow) {
            // 32 columns of planes 0 .. P-1: A plane p half r at slot 2p + r, B plane p
            // half c at slot 2P + 2p + c (the two B halves adjacent: one N = 256 operand)
            const int x = (args.kb_begin - args.kb_col0) * kBlockK + t * 32;
            mbar_expect_tx(&full_bar[s], P * (tg.rb + tg.cb) * kNarrow);
#pragma unroll
            for (int p = 0; p < P; ++p) {
              const CUtensorMap* mp = p == 0 ? &map0n : p == 1 ? &map1n : &map2n;
              for (int r = 0; r < tg.rb; ++r)
                tma_load_2d(st + (2 * p + r) * kNarrow, mp, &full_bar[s], x, tg.i0 + r * kTile);
              for (int c = 0; c < tg.cb; ++c)
                tma_load_2d(st + (2 * P + 2 * p + c) * kNarrow, mp, &full_bar[s], x,
                            tg.j0 + c * kTile);
            }
          } else if (t >= t8) {
            // 128 FP8 columns (a [cos | sin] pair): A half r at r x 16 KB, B halves at
            // 32 KB and 48 KB
            const int x = (kb8 - args.kb_col0 + 2 * (t - t8)) * kBlockK;
            wide_loads(st, &map8, &full_bar[s], x, tg);
          } else {
            // 64 columns of plane 0: A half r at r x 16 KB, B halves at 32 KB and 48 KB
            const int x = (kb1 - args.kb_col0 + (t - nnarrow)) * kBlockK;
            wide_loads(st, &map0w, &full_bar[s], x, tg);
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----------------------------------------------------------------
    if (lane == 0) {
      // products (p, q) with p + q <= 2 in the order (0,0) (0,1) (1,0) (0,2) (1,1) (2,0):
      // A plane p, B plane q; the three-product form is the first three
      constexpr uint32_t kPa = 0x210100u, kPb = 0x012010u;
      uint32_t g = 0, chunk = 0;  // stages consumed, chunks committed by this CTA
      bool ok = true;
      for (int tile = tile0; tile < args.tiles && ok; tile += tstep) {
        const StripTile tg(tile, args.npad, args.tile_map);
        // on a diagonal tile the first row half needs only the first 128 columns
        constexpr uint32_t kId256 = idesc_f16(SIX, 256), kId128 = idesc_f16(SIX, 128);
        const uint32_t id0 = tg.diag ? kId128 : kId256;
        bool first = true;  // first stage of an accumulation chunk
        for (int t = 0; t < nst; ++t, ++g) {
          const int s = g % kStages;
          ok = mbar_wait(&full_bar[s], (g / kStages) & 1, args.err, 13);
          if (!ok) break;
          if (first && chunk > 0) {  // the epilogue has read the previous chunk
            ok = mbar_wait(&acc_empty, (chunk - 1) & 1, args.err, 12);
            if (!ok) break;
          }
          tc_fence_after();
          const uint32_t st = smem_addr(ring + s * kStageBytes);
          if (t < nnarrow) {
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
              for (int r = 0; r < tg.rb; ++r)
#pragma unroll
                for (int p = 0; p < Cfg::kProds; ++p) {
                  const int pa = (kPa >> (4 * p)) & 15, pb = (kPb >> (4 * p)) & 15;
                  const uint64_t da = smem_desc<32>(st + (2 * pa + r) * kNarrow + ks * 32);
                  const uint64_t db = smem_desc<32>(st + (2 * P + 2 * pb) * kNarrow + ks * 32);
                  mma_f16(tmem + (uint32_t)(r * 256), da, db, r == 0 ? id0 : kId256,
                              (first && ks == 0 && p == 0) ? 0u : 1u);
                }
          } else if (t >= t8) {
            // 128-byte rows of 128 FP8 values: K = 32 (32 bytes) per MMA
            constexpr uint32_t kF8_256 = idesc_f8(256), kF8_128 = idesc_f8(128);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              for (int r = 0; r < tg.rb; ++r) {
                const uint64_t da = smem_desc<64>(st + r * kWide + ks * 32);
                const uint64_t db = smem_desc<64>(st + 2 * kWide + ks * 32);
                mma_f8(tmem + (uint32_t)(r * 256), da, db,
                       (r == 0 && tg.diag) ? kF8_128 : kF8_256, (first && ks == 0) ? 0u : 1u);
              }
          } else {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              for (int r = 0; r < tg.rb; ++r) {
                const uint64_t da = smem_desc<64>(st + r * kWide + ks * 32);
                const uint64_t db = smem_desc<64>(st + 2 * kWide + ks * 32);
                mma_f16(tmem + (uint32_t)(r * 256), da, db, r == 0 ? id0 : kId256,
                            (first && ks == 0) ? 0u : 1u);
              }
          }
          first = false;
          // frees the stage once these MMAs have read it
          mma_commit(&empty_bar[s]);
          if (chunk_ends(t)) {
            mma_commit(&acc_full);
            ++chunk;
            first = true;
          }
        }
      }
    }
  } else {
    // ---- epilogue: warps 2-9, TMEM lane quarter q = warp % 4, column half h ---------
    // A chunk before a tile's last goes, times 2^-2kexp (exact), by an error-free two-sum
    // into the tile's running hi / lo floats in the SM's scratch slot (each thread its
    // own 8 x 32 entries, laid out so that a warp's accesses are contiguous); the last
    // chunk adds hi + lo + acc to head.
    const int q = warp & 3, h = (warp - 2) >> 2, ew = warp - 2;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint64_t keep = l2_evict_last();  // the scratch slot's L2 policy
    float4* hi4 = nullptr;
    float4* lo4 = nullptr;
    bool ok = true;
    {
      uint32_t smid;
      asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
      if ((int)smid < args.scratch_slots) {
        hi4 = reinterpret_cast<float4*>(args.scratch + (size_t)smid * 2 * 65536) +
              (size_t)ew * 8 * 8 * 32 + lane;
        lo4 = hi4 + 65536 / 4;
      } else {
        atomicCAS(args.err, 0, 15);  // no slot: give up (the other roles' waits see it)
        ok = false;
      }
    }
    uint32_t chunk = 0;
    for (int tile = tile0; tile < args.tiles && ok; tile += tstep) {
      const StripTile tg(tile, args.npad, args.tile_map);
      int ci = 0;  // chunk index within the tile
      for (int t0 = 0; t0 < nst; ++ci) {
        int t1 = t0;
        while (!chunk_ends(t1)) ++t1;
        const bool final_chunk = t1 + 1 == nst;
        bool unused;
        const float scale = __int_as_float((127 - 2 * args.kexp[stage_block(t0, unused)]) << 23);
        ok = mbar_wait(&acc_full, chunk & 1, args.err, 14);
        if (!ok) break;
        tc_fence_after();
        for (int r = 0; r < tg.rb; ++r) {
          const int row = tg.i0 + r * kTile + 32 * q + lane;
#pragma unroll 1
          for (int cl = 0; cl < 4; ++cl) {
            const int cg = 4 * h + cl;
            if (tg.diag && r == 0 && cg >= kTile / 32) break;  // above the diagonal
            if (tg.j0 + cg * 32 >= args.n) break;
            uint32_t acc[32];
            TMEM_LD32(tmem + lane_base + (uint32_t)(r * 256 + cg * 32), acc);
            tmem_wait_ld();
            const int grp = (r * 4 + cl) * 8 * 32;  // float4 offset of this group
            if (final_chunk) {
              float th[32], tl[32];
              final_tail(ci > 0, hi4, lo4, grp, acc, scale, keep, th, tl);
              if (row < args.n) strip_final(args, th, tl, row, tg.j0 + cg * 32);
            } else {
              float hv[32], lv[32];
              if (ci > 0) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                  const float4 a4 = ld_keep(hi4 + grp + u * 32, keep);
                  const float4 b4 = ld_keep(lo4 + grp + u * 32, keep);
                  hv[4 * u] = a4.x, hv[4 * u + 1] = a4.y, hv[4 * u + 2] = a4.z, hv[4 * u + 3] = a4.w;
                  lv[4 * u] = b4.x, lv[4 * u + 1] = b4.y, lv[4 * u + 2] = b4.z, lv[4 * u + 3] = b4.w;
                }
              } else {
#pragma unroll
                for (int t = 0; t < 32; ++t) hv[t] = lv[t] = 0.f;
              }
#pragma unroll
              for (int t = 0; t < 32; ++t) {
                // two-sum: hv + a = s + e exactly
                const float a = __uint_as_float(acc[t]) * scale;
                const float s = __fadd_rn(hv[t], a);
                const float bb = __fsub_rn(s, hv[t]);
                const float e = __fadd_rn(__fsub_rn(hv[t], __fsub_rn(s, bb)), __fsub_rn(a, bb));
                hv[t] = s;
                lv[t] = __fadd_rn(lv[t], e);
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                st_keep(hi4 + grp + u * 32,
                        make_float4(hv[4 * u], hv[4 * u + 1], hv[4 * u + 2], hv[4 * u + 3]), keep);
                st_keep(lo4 + grp + u * 32,
                        make_float4(lv[4 * u], lv[4 * u + 1], lv[4 * u + 2], lv[4 * u + 3]), keep);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty);
        ++chunk;
        t0 = t1 + 1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem)
                 : "memory");
  }
}

// E = head (lower triangle) when the tail contributes nothing to the last window: the
// float nearest each (hi, lo) pair.
__global__ void k_head_to_float(const float2* __restrict__ head, int64_t ldh,
                                float* __restrict__ E, int64_t ldE, int n) {
  const int j = blockIdx.x * 32 + threadIdx.x;
  for (int i = blockIdx.y * 32 + threadIdx.y; i < min(n, (int)(blockIdx.y + 1) * 32); i += 8)
    if (j < n && j <= i) {
      const float2 x = head[(int64_t)i * ldh + j];
      E[(int64_t)i * ldE + j] = x.x + x.y;
    }
}

// 2-D map of a [rows][cols] plane of 16-bit values (bytes = false) in 128-row boxes of bk
// columns (bk = 64: 128-byte swizzle, bk = 32: 64-byte), or of bytes (bytes = true) in
// 128 x 128 boxes (128-byte swizzle).
bool make_map(CUtensorMap* m, const void* base, int rows, int64_t cols, int bk,
              bool bytes = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * (bytes ? 1 : 2)};
  cuuint32_t box[2] = {(cuuint32_t)(bytes ? 128 : bk), (cuuint32_t)kTile};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, bytes ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            bytes || bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Diagonal of the K-blocks [kb0, kb1): every k-vector adds W_K (cos^2 + sin^2) to E_ii,
// so where the range holds whole [cos | sin] pairs (both ends even: K-block b is the cos
// or sin half of k-vectors 64 (b / 2) ..) the diagonal is their summed weight, exact in
// FP64, instead of an FP32 tensor-core sum of same-sign terms, whose rounding errors add
// up (measured ~1e-7 too low at 12,800 atoms).  Returns 0 where an end is odd.
int range_weight(const double* kw, int kb0, int kb1, double* w) {
  *w = 0.0;
  if (!kw || (kb0 & 1) || (kb1 & 1)) return 0;
  double s = 0.0, comp = 0.0;  // Neumaier-compensated sum
  for (int k = 32 * kb0; k < 32 * kb1; ++k) {
    const double t = s + kw[k];
    comp += std::fabs(s) >= std::fabs(kw[k]) ? (s - t) + kw[k] : (kw[k] - t) + s;
    s = t;
  }
  *w = s + comp;
  return 1;
}

}  // namespace

__global__ void k_nsmid(int* out) {
  uint32_t v;
  asm volatile("mov.u32 %0, %%nsmid;" : "=r"(v));
  *out = (int)v;
}

// The order in which the CTAs of the tile kernels take the nt (nt + 1) / 2 lower-triangle
// tiles: blocks of 12 x 12 tiles (about one wave of the 152 SMs), the blocks in row-major
// triangle order and the tiles of a block row by row.  The tiles in flight then share 12
// operand row blocks and 12 column blocks, which they stream at about the same K
// position, so the L2 serves most of their operand loads; in plain row-major order they
// share one row block and stream ~150 different column blocks.
std::vector<uint32_t> ek_tile_order(int nt) {
  constexpr int G = 12;
  std::vector<uint32_t> map;
  map.reserve((size_t)nt * (nt + 1) / 2);
  const int nb = (nt + G - 1) / G;
  for (int bi = 0; bi < nb; ++bi)
    for (int bj = 0; bj <= bi; ++bj)
      for (int a = 0; a < G; ++a) {
        const int I = bi * G + a;
        if (I >= nt) break;
        for (int b = 0; b < G; ++b) {
          const int J = bj * G + b;
          if (J > I) break;
          map.push_back(((uint32_t)I << 16) | (uint32_t)J);
        }
      }
  return map;
}

// Floats of k_ek_strip scratch per SM slot.
int64_t ek_strip_scratch_floats() { return 2 * 65536; }

// SM identifiers of the current device (%nsmid: the largest %smid + 1, which may exceed the
// SM count), written to the device int *d_out.
void launch_nsmid(int* d_out, cudaStream_t s) {
  k_nsmid<<<1, 1, 0, s>>>(d_out);
  note_launch();
}

// K-blocks [kb_begin, kb_end) of the lower triangle from the 16-bit planes holding the
// K-blocks kb_col0 .. kb_col0 + plane_cols / 64; the result plus head goes to float E, or
// back into head (FP64) when E is null.  Two launches, the first adding its K-range to
// head and the second writing E: the six-product (BF16) K-blocks, then the three- and
// one-product (FP16) ones.  `mid`, when given, is recorded before the second.
int launch_ek_tc(const void* p0, const void* p1, const void* p2, const void* p8, int npad,
                 int64_t plane_cols, int kb_col0, int n, int kb_begin, int kb_end, int kb6_end,
                 int kb3_end, int kb8_begin,
                 const uint32_t* chunk_end, const int* kexp, float2* head, int64_t ldh,
                 float* E, int64_t ldE, int* err, const double* kw, float* scratch,
                 int scratch_slots, const uint32_t* tile_map, cudaEvent_t mid,
                 cudaStream_t s) {
  if (!scratch || scratch_slots < 1 || (kb6_end & 1) || (kb_begin & 1) || (kb8_begin & 1))
    return CPM_EINVAL;
  CUtensorMap m0, m0n, m1n, m2n, m8;
  if (!make_map(&m0, p0, npad, plane_cols, 64) || !make_map(&m0n, p0, npad, plane_cols, 32) ||
      !make_map(&m1n, p1, npad, plane_cols, 32) || !make_map(&m2n, p2, npad, plane_cols, 32) ||
      !make_map(&m8, p8, npad, plane_cols, 128, true))
    return CPM_ECUDA;
  const int smem6 = StripCfg<true>::kStages * StripCfg<true>::kStageBytes + 1024;
  const int smem31 = StripCfg<false>::kStages * StripCfg<false>::kStageBytes + 1024;
  if (cudaFuncSetAttribute(k_ek_strip<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem6) != cudaSuccess ||
      cudaFuncSetAttribute(k_ek_strip<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem31) != cudaSuccess)
    return CPM_ECUDA;
  // the six-product part [kb_begin, x6_end) and the rest [l_begin, kb_end); kb6_end is
  // even, so each part holds whole [cos | sin] block pairs
  const int x6_end = std::min(kb_end, kb6_end);
  const int l_begin = std::max(kb_begin, x6_end);
  const int nt = (n + kStripTile - 1) / kStripTile;
  StripArgs a;
  a.n = n;
  a.npad = npad;
  a.tiles = nt * (nt + 1) / 2;
  a.kb3_end = kb3_end;
  a.kb8_begin = kb8_begin;
  a.kb_col0 = kb_col0;
  a.chunk_end = chunk_end;
  a.kexp = kexp;
  a.scratch = scratch;
  a.scratch_slots = scratch_slots;
  a.head = head;
  a.ldh = ldh;
  a.ldE = ldE;
  a.err = err;
  a.tile_map = tile_map;
  // one CTA per tile; the hardware hands each SM its next tile as it frees up, in the
  // order of the tile map
  auto launch = [&](bool six) {
    const int smem = six ? smem6 : smem31;
    if (six)
      k_ek_strip<true><<<a.tiles, kStripThreads, smem, s>>>(m0, m0n, m1n, m2n, m8, a);
    else
      k_ek_strip<false><<<a.tiles, kStripThreads, smem, s>>>(m0, m0n, m1n, m2n, m8, a);
    note_launch();
    return cudaGetLastError();
  };
  if (kb_begin < x6_end) {
    a.kb_begin = kb_begin;
    a.kb_end = x6_end;
    a.E = l_begin < kb_end ? nullptr : E;
    {
      double w = 0.0;
      a.diag_exact = range_weight(kw, a.kb_begin, a.kb_end, &w);
      a.wd_hi = (float)w;
      a.wd_lo = (float)(w - (double)a.wd_hi);
    }
    if (launch(true) != cudaSuccess) return CPM_ECUDA;
  }
  if (mid) cudaEventRecord(mid, s);
  if (l_begin < kb_end) {
    a.kb_begin = l_begin;
    a.kb_end = kb_end;
    a.E = E;
    {
      double w = 0.0;
      a.diag_exact = range_weight(kw, a.kb_begin, a.kb_end, &w);
      a.wd_hi = (float)w;
      a.wd_lo = (float)(w - (double)a.wd_hi);
    }
    if (launch(false) != cudaSuccess) return CPM_ECUDA;
  }
  if (kb_begin >= kb_end && E)  // nothing of the tail in this window
    (k_head_to_float<<<dim3((n + 31) / 32, (n + 31) / 32), dim3(32, 8), 0, s>>>(head, ldh, E,
                                                                              ldE, n),
     note_launch());
  return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_ECUDA;
}

}  // namespace cpm
