// Preconditioned conjugate gradient on E_n q = b (Sec. III B 2) and the neutralisation
// step of Eq. 35.
//
// Every scalar lives on the device: per-block partial sums are reduced by one warp per
// right-hand side, so the host only polls a small status array every few iterations.
// Vectors are FP64; the matvec streams E in its storage type (FP32: float products with
// FP64 row sums).  The PCG-DC preconditioner is not symmetric, so beta is the flexible
// Polak-Ribiere form r_{k+1}^T (z_{k+1} - z_k) / (r_k^T z_k).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "async_copy.cuh"
#include "cpm_internal.cuh"

namespace cpm {

namespace {

struct ColState {
  double rz;      // r^T z of the current iterate
  double bb;      // b^T b
  double alpha;
  double beta;
  double relres;  // ||r|| / ||b||
  int iter;
  int done;       // 0 running, 1 converged, 2 breakdown
  int restart;    // residual replacement reopened a converged column: p = z next
  int pad_;
};

constexpr int kThreads = 256;
constexpr int kMvWarps = 8;

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide sum of NV values per thread; result valid in thread 0.
template <int NV>
__device__ void block_sum(double (&v)[NV], double* sm /* [32*NV] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = warp_sum(v[t]);
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < NV; ++t) sm[warp * NV + t] = v[t];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      double x = lane < nw ? sm[lane * NV + t] : 0.0;
      v[t] = warp_sum(x);
    }
  }
  __syncthreads();
}

// FP64 E (the plain baseline build): q[r] = E p[r] for NR columns from c0, one warp per
// row with FP64 products and sums, plus the per-block partial of p^T q.
template <int NR>
__global__ void __launch_bounds__(kThreads)
k_matvec_f64(const double* __restrict__ E, int64_t ldE, int n, const double* __restrict__ pv,
             int64_t ldv, int c0, int nrhs, double* __restrict__ q,
             double* __restrict__ pq_part, const ColState* __restrict__ st) {
  __shared__ double sm[32 * NR];
  c0 += blockIdx.y * NR;  // one column group per grid row
  if (st) {  // converged columns are not multiplied again (uniform per block)
    bool live = false;
#pragma unroll
    for (int r = 0; r < NR; ++r) live |= st[c0 + r].done == 0;
    if (!live) {
      if (threadIdx.x < NR) pq_part[(int64_t)blockIdx.x * nrhs + c0 + threadIdx.x] = 0.0;
      return;
    }
  }
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * kMvWarps + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * kMvWarps;
  double pq[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) pq[r] = 0.0;
  for (int row = wid; row < n; row += nwarps) {
    const double* e = E + (int64_t)row * ldE;
    double acc[NR][2];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = 0.0;
    for (int64_t c = lane * 2; c < ldE; c += 64) {
      const double2 ev = __ldg(reinterpret_cast<const double2*>(e + c));
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const double2 hv = *reinterpret_cast<const double2*>(pv + (int64_t)(c0 + r) * ldv + c);
        acc[r][0] = fma(ev.x, hv.x, acc[r][0]);
        acc[r][1] = fma(ev.y, hv.y, acc[r][1]);
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const double s = warp_sum(acc[r][0] + acc[r][1]);
      if (lane == 0) {
        const int64_t o = (int64_t)(c0 + r) * ldv + row;
        q[o] = s;
        pq[r] += s * pv[o];
      }
    }
  }
  block_sum<NR>(pq, sm);
  if (threadIdx.x == 0)
#pragma unroll
    for (int r = 0; r < NR; ++r) pq_part[(int64_t)blockIdx.x * nrhs + c0 + r] = pq[r];
}

// Float pair (hi, lo) += (bh, bl): the high parts meet in an error-free two-sum, the low
// parts (already ~2^-24 of the high ones) in one rounded add.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (bh - bb);
  lo = lo + bl + e;
  hi = s;
}

// FP32 E, the path every float build takes: q[r] = E p[r] for NR columns from c0 and the
// per-block partial of p^T q.  A block owns kMvRows rows; its eight warps split the
// padded row into 128-column groups (one float4 per lane), so each float4 of the
// direction pair (hi, lo) is loaded once per group and used for all kMvRows rows, and
// the grid has n / kMvRows blocks of equal work for the scheduler to balance.  Products
// and the running sum are error-free (two-product, two-sum, one chain per row and column
// per lane), so the stored float E is applied to ~1e-14 rather than to float rounding of
// every product and sum -- otherwise PCG converges to the solution of a slightly
// different matrix (1e-6 of q at the 512-atom cell); lanes and warps combine float
// pairs, and only the final per-row value goes to FP64 -- FP64 runs at 1/64 of the FP32
// rate here.  E is read with the streaming hint so the direction stays resident in L2.
constexpr int kMvRows = 4;

// WS warps share a group of kMvRows rows (8: the column split above, for long rows;
// 1: every warp owns its rows, for short rows where eight warps would idle).
template <int NR, int WS>
__global__ void __launch_bounds__(kThreads)
k_matvec_f32(const float* __restrict__ E, int64_t ldE, int n, const float* __restrict__ pv,
             const float* __restrict__ plo, const double* __restrict__ p64, int64_t ldv,
             int c0, int nrhs, double* __restrict__ q, double* __restrict__ pq_part,
             const ColState* __restrict__ st) {
  constexpr int RB = kMvRows;
  constexpr int RBB = RB * (kMvWarps / WS);  // rows per block
  c0 += blockIdx.y * NR;  // one column group per grid row
  if (st) {  // converged columns are not multiplied again (uniform per block)
    bool live = false;
#pragma unroll
    for (int r = 0; r < NR; ++r) live |= st[c0 + r].done == 0;
    if (!live) {
      if (threadIdx.x < NR) pq_part[(int64_t)blockIdx.x * nrhs + c0 + threadIdx.x] = 0.0;
      return;
    }
  }
  __shared__ float2 sm[kMvWarps][RB * NR];
  __shared__ double spq[RBB * NR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gi = warp / WS, sub = warp % WS;  // row group of this warp, its column share
  const int row0 = blockIdx.x * RBB + gi * RB;
  const int ngroups = (int)(ldE >> 7);
  const float* erow[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) erow[i] = E + (int64_t)min(row0 + i, n - 1) * ldE;
  float part[RB][NR], perr[RB][NR];
#pragma unroll
  for (int i = 0; i < RB; ++i)
#pragma unroll
    for (int r = 0; r < NR; ++r) part[i][r] = perr[i][r] = 0.f;
  for (int g = sub; g < ngroups; g += WS) {
    const int64_t cc = (int64_t)g * 128 + lane * 4;
    float ev[RB][4];
#pragma unroll
    for (int i = 0; i < RB; ++i)
      *reinterpret_cast<float4*>(ev[i]) = __ldcs(reinterpret_cast<const float4*>(erow[i] + cc));
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int64_t o = (int64_t)(c0 + r) * ldv + cc;
      float hv[4], lv[4];
      *reinterpret_cast<float4*>(hv) = __ldg(reinterpret_cast<const float4*>(pv + o));
      *reinterpret_cast<float4*>(lv) = __ldg(reinterpret_cast<const float4*>(plo + o));
#pragma unroll
      for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float e = ev[i][w];
          const float pr = e * hv[w];
          const float s = part[i][r] + pr;
          const float bb = s - part[i][r];
          const float e2 = (part[i][r] - (s - bb)) + (pr - bb);
          perr[i][r] = fmaf(e, lv[w], perr[i][r] + (fmaf(e, hv[w], -pr) + e2));
          part[i][r] = s;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < RB; ++i)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float h = part[i][r], l = perr[i][r];
#pragma unroll
      for (int o = 16; o; o >>= 1)
        pair_add(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
      if (lane == 0) sm[warp][i * NR + r] = make_float2(h, l);
    }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < RBB * NR) {  // t = (row group, row, column)
    const int tg = t / (RB * NR), ti = t % (RB * NR);
    float h = sm[tg * WS][ti].x, l = sm[tg * WS][ti].y;
#pragma unroll
    for (int w = 1; w < WS; ++w) pair_add(h, l, sm[tg * WS + w][ti].x, sm[tg * WS + w][ti].y);
    const int i = ti / NR, r = ti % NR, row = blockIdx.x * RBB + tg * RB + i;
    double pq = 0.0;
    if (row < n) {
      const int64_t o = (int64_t)(c0 + r) * ldv + row;
      const double v = (double)h + (double)l;
      q[o] = v;
      pq = v * p64[o];
    }
    spq[t] = pq;
  }
  __syncthreads();
  if (t < NR) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RBB; ++i) s += spq[i * NR + t];
    pq_part[(int64_t)blockIdx.x * nrhs + c0 + t] = s;
  }
}

constexpr int kFastCols = 16;  // columns of one group of a many-column solve

// The inner matvec of a many-column solve, streamed by TMA: q[c] = E p_c for the 16
// columns of one column group, E read from HBM once for all of them.  A unit is 256 rows
// of E times one of `splits` equal shares of its columns; the host picks the share count
// so that the units fill whole waves of the GPU.  One thread issues the copies (a 256 x 64
// tile of E as two 128-byte-swizzled 256 x 32 TMA boxes, evict-first in L2, and the
// group's 64 x 16 directions by one bulk copy) into a three-stage ring with full / empty
// mbarriers, two stages ahead of its own warp (eight warps of 255 registers: two to each
// scheduler); each warp w takes 8 of a stage's 64 columns, lane l rows l + 32 i (i < 8):
// each E value is read from shared memory once (a float4 of four columns, the swizzle
// keeps the eight lanes of each quarter-warp on distinct banks) and each direction value
// is a broadcast.  Products and the per-lane partial sums are plain float, as
// before (a lane sums 8 columns a stage over the unit's share: ~1e-6 of the row's partial
// sums, not the ~1e-14 of k_matvec_f32, so the solver uses it only between residual
// replacements, which recompute b - E x with k_matvec_f32); warps combine through shared
// memory (pairwise, in float), and the last unit of a row block to finish (a counter per
// row block, reset by that unit) adds the shares' FP64 partials in share order, writes q
// and the p^T q partial of the block.  Every wait is bounded: on timeout the kernel
// records an error code in *err and leaves once its copies have landed.
constexpr int kStRows = 256;
constexpr int kStK = 64;
constexpr int kStStages = 3;
constexpr int kStWarps = 8;
constexpr int kStThreads = kStWarps * 32;
constexpr int kStBox = kStRows * 32 * 4;                   // 32 KB: a 256 x 32 box of E
constexpr int kStXBytes = kStK * kFastCols * 4;            // 4 KB of directions
constexpr int kStStageBytes = 2 * kStBox + kStXBytes;      // 68 KB
constexpr int kStSmem = kStStages * kStStageBytes + 1024;  // and 1 KB for the alignment
constexpr int kStOut = kStRows * kFastCols;                // 4,096 outputs a unit

struct StreamArgs {
  int n, nst, splits, nrb;  // rows; 64-column stages a row; shares; row blocks
  const float* xt;          // directions, [group][ldv][16]
  const double* p64;
  int64_t ldv;
  int g0, nrhs;
  double* part;     // [group][nrb * splits][4096] FP64 partials of the units
  unsigned* count;  // [group][nrb] finished units, zero between launches
  double* q;
  double* pq_part;  // [nrb][nrhs]
  const ColState* st;
  int* err;
};

__global__ void __launch_bounds__(kStThreads, 1)
k_matvec_stream(const __grid_constant__ CUtensorMap emap, StreamArgs a) {
  extern __shared__ __align__(1024) uint8_t sraw[];
  uint8_t* ring = (uint8_t*)(((uintptr_t)sraw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStStages], empty[kStStages];
  __shared__ int s_issued, s_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = a.g0 + blockIdx.y, c0 = grp * kFastCols;
  const int ncol = min(kFastCols, a.nrhs - c0);
  const int rb = blockIdx.x / a.splits, sp = blockIdx.x % a.splits;
  if (a.st) {  // a group with every column converged is not multiplied (uniform per grid row)
    bool live = false;
    for (int r = 0; r < ncol; ++r) live |= a.st[c0 + r].done == 0;
    if (!live) {
      if (sp == 0 && tid < ncol) a.pq_part[(int64_t)rb * a.nrhs + c0 + tid] = 0.0;
      return;
    }
  }
  const int kt0 = (int)((int64_t)sp * a.nst / a.splits);
  const int cnt = (int)((int64_t)(sp + 1) * a.nst / a.splits) - kt0;
  const int row0 = rb * kStRows;
  if (tid == 0) {
    for (int s = 0; s < kStStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kStWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_issued = 0;
  }
  __syncthreads();
  // acc[r][j]: columns 2 j and 2 j + 1 of row l + 32 r, updated by paired FMAs (two
  // IEEE fmas in one instruction: half the issue slots of scalar ones)
  float2 acc[8][kFastCols / 2];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < kFastCols / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  // stage i into its slot once every warp has released the slot's previous stage
  const uint64_t pol = tid == 0 ? l2_evict_first() : 0;
  const float* xg = a.xt + (int64_t)grp * a.ldv * kFastCols;
  auto issue = [&](int i) -> bool {
    const int slot = i % kStStages;
    if (i >= kStStages && !mbar_wait(&empty[slot], ((i / kStStages) - 1) & 1, a.err, 21))
      return false;
    uint8_t* sb = ring + slot * kStStageBytes;
    const int k0 = (kt0 + i) * kStK;
    mbar_expect_tx(&full[slot], kStStageBytes);
    tma_load_2d_hint(sb, &emap, &full[slot], k0, row0, pol);
    tma_load_2d_hint(sb + kStBox, &emap, &full[slot], k0 + 32, row0, pol);
    bulk_load(sb + 2 * kStBox, xg + (int64_t)k0 * kFastCols, kStXBytes, &full[slot]);
    s_issued = i + 1;
    return true;
  };
  bool ok = true;
  if (tid == 0)
    for (int i = 0; i < min(cnt, kStStages - 1) && ok; ++i) ok = issue(i);
  // products: warp w takes columns 8 w .. 8 w + 7 of each stage
  const int box = warp >> 2;
  for (int i = 0; i < cnt; ++i) {
    if (tid == 0 && ok && i + kStStages - 1 < cnt) ok = issue(i + kStStages - 1);
    const int slot = i % kStStages;
    if (!mbar_wait(&full[slot], (i / kStStages) & 1, a.err, 22)) break;
    const uint8_t* sb = ring + slot * kStStageBytes;
    const uint8_t* eb = sb + box * kStBox + lane * 128;
    const float4* xs = reinterpret_cast<const float4*>(sb + 2 * kStBox) + warp * 8 * 4;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      // 16-byte chunk (warp & 3) * 2 + c of the row, at its swizzled place
      const int ch = (((warp & 3) * 2 + c) ^ (lane & 7)) * 16;
      float4 e[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        e[r] = *reinterpret_cast<const float4*>(eb + r * 32 * 128 + ch);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        float xv[kFastCols];
#pragma unroll
        for (int v = 0; v < 4; ++v)
          *reinterpret_cast<float4*>(xv + 4 * v) = xs[(4 * c + kk) * 4 + v];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float ev = kk == 0 ? e[r].x : kk == 1 ? e[r].y : kk == 2 ? e[r].z : e[r].w;
          const float2 e2 = make_float2(ev, ev);
#pragma unroll
          for (int j = 0; j < kFastCols / 2; ++j)
            acc[r][j] = __ffma2_rn(e2, make_float2(xv[2 * j], xv[2 * j + 1]), acc[r][j]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[slot]);
  }
  __syncthreads();
  if (tid == 0) {  // copies still in flight (after an error): let them land before leaving
    const int issued = s_issued;
    for (int i = max(0, issued - kStStages); i < issued; ++i)
      mbar_wait_drain(&full[i % kStStages], (i / kStStages) & 1);
    s_flag = *(volatile int*)a.err;
  }
  __syncthreads();
  if (s_flag) return;
  // warps' partials to shared memory: output o = (16 r + cc) 32 + lane of warp w at
  // red[w][o] (whole-warp 128-byte rows)
  float* red = reinterpret_cast<float*>(ring);
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int cc = 0; cc < kFastCols; ++cc)
      red[warp * kStOut + (r * kFastCols + cc) * 32 + lane] =
          (cc & 1) ? acc[r][cc >> 1].y : acc[r][cc >> 1].x;
  __syncthreads();
  double v[kStOut / (kStWarps * 32)];  // outputs o = tid + 256 m
#pragma unroll
  for (int m = 0; m < kStOut / (kStWarps * 32); ++m) {
    const int o = tid + kStWarps * 32 * m;
    // the eight warps' partials pairwise in float (three roundings of each, against the
    // thousands in every partial), then FP64
    float pw[kStWarps];
#pragma unroll
    for (int w = 0; w < kStWarps; ++w) pw[w] = red[w * kStOut + o];
    v[m] = (double)(((pw[0] + pw[1]) + (pw[2] + pw[3])) + ((pw[4] + pw[5]) + (pw[6] + pw[7])));
  }
  constexpr int kM = kStOut / (kStWarps * 32);
  if (a.splits > 1) {
    const int64_t unit = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    double* mine = a.part + unit * kStOut;
#pragma unroll
    for (int m = 0; m < kM; ++m) mine[tid + kStWarps * 32 * m] = v[m];
    __threadfence();
    __syncthreads();
    unsigned* counter = a.count + (int64_t)blockIdx.y * a.nrb + rb;
    if (tid == 0) s_flag = atomicAdd(counter, 1u) == (unsigned)(a.splits - 1);
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    const double* shares = a.part + ((int64_t)blockIdx.y * gridDim.x + (int64_t)rb * a.splits) * kStOut;
#pragma unroll
    for (int m = 0; m < kM; ++m) {
      const int o = tid + kStWarps * 32 * m;
      double sum = 0.0;
      for (int s = 0; s < a.splits; ++s) sum += __ldcg(shares + (int64_t)s * kStOut + o);
      v[m] = sum;
    }
    if (tid == 0) *counter = 0u;
  }
  // o = (16 r + cc) 32 + lane: thread t holds column w = t / 32 for even m, w + 8 for odd
  double pq_even = 0.0, pq_odd = 0.0;
#pragma unroll
  for (int m = 0; m < kM; ++m) {
    const int o = tid + kStWarps * 32 * m;
    const int cc = (o >> 5) & 15, row = row0 + (o >> 9) * 32 + (o & 31);
    if (row < a.n && cc < ncol) {
      const int64_t at = (int64_t)(c0 + cc) * a.ldv + row;
      a.q[at] = v[m];
      const double t = v[m] * a.p64[at];
      if (m & 1) pq_odd += t;
      else pq_even += t;
    }
  }
  pq_even = warp_sum(pq_even);
  pq_odd = warp_sum(pq_odd);
  if (lane == 0) {
    if (warp < ncol) a.pq_part[(int64_t)rb * a.nrhs + c0 + warp] = pq_even;
    if (warp + 8 < ncol) a.pq_part[(int64_t)rb * a.nrhs + c0 + warp + 8] = pq_odd;
  }
}

// Units of the streamed matvec: `splits` shares of each row's columns such that row
// blocks x shares x groups fills whole waves of `sms` CTAs best (a smaller share count
// unless a larger one fills 2% more of the last wave).
int stream_splits(int nrb, int groups, int nst, int sms) {
  int best = 1;
  double best_eff = -1.0;
  for (int sp = 1; sp <= std::min(8, nst); ++sp) {
    const int64_t units = (int64_t)nrb * sp * groups;
    const int64_t waves = (units + sms - 1) / sms;
    const double eff = (double)units / (double)(waves * sms);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
  }
  return best;
}

// TMA map of the float E [n][ldE] in 256-row x 32-column boxes, 128-byte swizzle; rows past
// n read as zero.
bool make_stream_map(CUtensorMap* m, const float* E, int n, int64_t ldE) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ldE, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ldE * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)kStRows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(E), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Ragged batch: column c is system c with its own float E (ld, n); one column per grid
// row, the same arithmetic as k_matvec_f32<1>.  Row blocks past the system's n write a
// zero partial.
__global__ void __launch_bounds__(kThreads)
k_matvec_ragged(const SysCol* __restrict__ sys, const float* __restrict__ pv,
                const float* __restrict__ plo, const double* __restrict__ p64, int64_t ldv,
                int nrhs, double* __restrict__ q, double* __restrict__ pq_part,
                const ColState* __restrict__ st) {
  constexpr int RB = kMvRows;
  __shared__ float2 sm[kMvWarps][RB];
  __shared__ double spq[RB];
  const int c = blockIdx.y;
  const int n = (st && st[c].done) ? 0 : sys[c].n;  // converged: only the zero partial
  const int64_t ldE = sys[c].ldE;
  const float* E = sys[c].E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row0 = blockIdx.x * RB;
  if (row0 >= n) {  // uniform per block
    if (threadIdx.x == 0) pq_part[(int64_t)blockIdx.x * nrhs + c] = 0.0;
    return;
  }
  const int ngroups = (int)(ldE >> 7);
  const float* erow[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) erow[i] = E + (int64_t)min(row0 + i, n - 1) * ldE;
  float part[RB], perr[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) part[i] = perr[i] = 0.f;
  const float* ph = pv + (int64_t)c * ldv;
  const float* pl = plo + (int64_t)c * ldv;
  for (int g = warp; g < ngroups; g += kMvWarps) {
    const int64_t cc = (int64_t)g * 128 + lane * 4;
    float ev[RB][4];
#pragma unroll
    for (int i = 0; i < RB; ++i)
      *reinterpret_cast<float4*>(ev[i]) = __ldcs(reinterpret_cast<const float4*>(erow[i] + cc));
    float hv[4], lv[4];
    *reinterpret_cast<float4*>(hv) = __ldg(reinterpret_cast<const float4*>(ph + cc));
    *reinterpret_cast<float4*>(lv) = __ldg(reinterpret_cast<const float4*>(pl + cc));
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const float e = ev[i][w];
        const float pr = e * hv[w];
        const float s = part[i] + pr;
        const float bb = s - part[i];
        const float e2 = (part[i] - (s - bb)) + (pr - bb);
        perr[i] = fmaf(e, lv[w], perr[i] + (fmaf(e, hv[w], -pr) + e2));
        part[i] = s;
      }
  }
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    float h = part[i], l = perr[i];
#pragma unroll
    for (int o = 16; o; o >>= 1)
      pair_add(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
    if (lane == 0) sm[warp][i] = make_float2(h, l);
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < RB) {
    float h = sm[0][t].x, l = sm[0][t].y;
#pragma unroll
    for (int w = 1; w < kMvWarps; ++w) pair_add(h, l, sm[w][t].x, sm[w][t].y);
    const int row = row0 + t;
    double pq = 0.0;
    if (row < n) {
      const int64_t o = (int64_t)c * ldv + row;
      const double v = (double)h + (double)l;
      q[o] = v;
      pq = v * p64[o];
    }
    spq[t] = pq;
  }
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RB; ++i) s += spq[i];
    pq_part[(int64_t)blockIdx.x * nrhs + c] = s;
  }
}

// alpha = r^T z / p^T q for every running column.
__global__ void k_alpha(const double* __restrict__ pq_part, int nparts, int nrhs,
                        ColState* __restrict__ st) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= nrhs) return;
  double s = 0.0;
  for (int b = lane; b < nparts; b += 32) s += pq_part[(int64_t)b * nrhs + col];
  s = warp_sum(s);
  if (lane == 0) {
    ColState& c = st[col];
    if (c.done) {
      c.alpha = 0.0;
    } else if (!(s > 0.0) || !isfinite(s)) {
      c.alpha = 0.0;
      c.done = 2;
    } else {
      c.alpha = c.rz / s;
    }
  }
}

// x += alpha p, r -= alpha q; Jacobi/none also form z; partial dots
// [r^T z_new, r^T z_old, r^T r, sum r].
template <int PRE>
__global__ void __launch_bounds__(kThreads)
k_update(int n, int64_t ldv, int nrhs, const ColState* __restrict__ st,
         double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
         const double* __restrict__ p, const double* __restrict__ q,
         const double* __restrict__ inv_diag, double* __restrict__ dots,
         const SysCol* __restrict__ sys) {
  __shared__ double sm[32 * 4];
  {
    const int col = blockIdx.y;  // one right-hand side per grid row
    if (sys) {  // ragged batch: this column's system
      n = sys[col].n;
      inv_diag = sys[col].inv_diag;
    }
    const double a = st[col].alpha;
    const bool active = st[col].done == 0;
    if (!active) return;  // converged column: its dots are not read (uniform per block)
    double v[4] = {0, 0, 0, 0};
    const int64_t o = (int64_t)col * ldv;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      double ri = r[o + i];
      if (active) {
        x[o + i] += a * p[o + i];
        ri -= a * q[o + i];
        r[o + i] = ri;
      }
      if (PRE != CPM_PRECOND_DC) {
        const double zo = z[o + i];
        const double zn = PRE == CPM_PRECOND_JACOBI ? ri * inv_diag[i] : ri;
        if (active) z[o + i] = zn;
        v[0] += ri * zn;
        v[1] += ri * zo;
      }
      v[2] += ri * ri;
      v[3] += ri;
    }
    block_sum<4>(v, sm);
    if (threadIdx.x == 0)
      for (int t = 0; t < 4; ++t) dots[((int64_t)blockIdx.x * nrhs + col) * 4 + t] = v[t];
  }
}

// z = P r (+ p_gap * sum r on the complement of the pattern) for PCG-DC, one thread per
// row; partial dots [r^T z_new, r^T z_old] into slots 0, 1.  rsum_part may be the dots
// buffer itself: the kernel only reads its slot 3 and only writes slots 0 and 1.
__global__ void __launch_bounds__(kThreads)
k_dc_apply(int n, int64_t ldv, int nrhs, const ColState* __restrict__ st,
           const int64_t* __restrict__ off, const int* __restrict__ idx,
           const double* __restrict__ prow, double pgap, const double* __restrict__ r,
           double* __restrict__ z, const double* __restrict__ rsum_part, int nparts,
           double* __restrict__ dots, int first, const SysCol* __restrict__ sys) {
  __shared__ double sm[32 * 2];
  __shared__ double s_rsum;
  {
    const int col = blockIdx.y;
    if (sys) {  // ragged batch: this column's system
      n = sys[col].n;
      off = sys[col].nbr_off;
      idx = sys[col].nbr_idx;
      prow = sys[col].prow;
      pgap = sys[col].pgap;
    }
    const bool active = first || st[col].done == 0;
    if (!active) return;  // converged column (uniform per block)
    if (threadIdx.x < 32) {
      double s = 0.0;
      if (pgap != 0.0)
        for (int b = threadIdx.x; b < nparts; b += 32) s += rsum_part[((int64_t)b * nrhs + col) * 4 + 3];
      s = warp_sum(s);
      if (threadIdx.x == 0) s_rsum = s;
    }
    __syncthreads();
    const double gsum = pgap * s_rsum;
    const int64_t o = (int64_t)col * ldv;
    double v[2] = {0, 0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      double acc = gsum;
      for (int64_t e = off[j]; e < off[j + 1]; ++e) acc += prow[e] * r[o + idx[e]];
      const double rj = r[o + j];
      const double zo = z[o + j];
      if (active) z[o + j] = acc;
      v[0] += rj * acc;
      v[1] += rj * zo;
    }
    block_sum<2>(v, sm);
    if (threadIdx.x == 0) {
      dots[((int64_t)blockIdx.x * nrhs + col) * 4 + 0] = v[0];
      dots[((int64_t)blockIdx.x * nrhs + col) * 4 + 1] = v[1];
    }
  }
}

// Reduce the dots, test convergence, form beta, and advance the column state.
__global__ void k_beta(const double* __restrict__ dots, int nparts, int nrhs, double tol,
                       int flexible, const ColState* __restrict__ cur,
                       ColState* __restrict__ next) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= nrhs) return;
  double s[3] = {0, 0, 0};
  for (int b = lane; b < nparts; b += 32)
    for (int t = 0; t < 3; ++t) s[t] += dots[((int64_t)b * nrhs + col) * 4 + t];
  for (int t = 0; t < 3; ++t) s[t] = warp_sum(s[t]);
  if (lane == 0) {
    ColState c = cur[col];
    if (c.done == 0) {
      c.iter += 1;
      c.relres = sqrt(s[2] / c.bb);
      if (!isfinite(c.relres)) {
        c.done = 2;
      } else if (c.relres <= tol) {
        c.done = 1;
      } else {
        c.beta = flexible ? (s[0] - s[1]) / c.rz : s[0] / c.rz;
        c.rz = s[0];
        if (!isfinite(c.beta) || !(c.rz != 0.0)) c.done = 2;
      }
    }
    next[col] = c;
  }
}

// p = z + beta p, and the matvec's copy: the value itself in FP64 storage, a float
// pair hi + lo (plo != nullptr) in float storage.
// first = 2: only the columns whose residual replacement reopened them (restart flag),
// which start again from p = z.  xt (float storage, many-column solves): the directions
// again, transposed per group of 16 columns, [group][row][16], for k_matvec_stream.
template <typename T>
__global__ void k_p_update(int n, int64_t ldv, int nrhs, const ColState* __restrict__ st,
                           const double* __restrict__ z, double* __restrict__ p,
                           T* __restrict__ pv, T* __restrict__ plo, int first,
                           float* __restrict__ xt = nullptr) {
  {
    const int col = blockIdx.y;
    if (first == 2 && !st[col].restart) return;
    if (first == 0 && st[col].done) return;
    const double bta = first ? 0.0 : st[col].beta;
    const int64_t o = (int64_t)col * ldv;
    float* xc = xt ? xt + ((int64_t)(col / kFastCols) * ldv * kFastCols + col % kFastCols)
                   : nullptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double v = z[o + i] + bta * p[o + i];
      p[o + i] = v;
      const T hi = (T)v;
      pv[o + i] = hi;
      if (plo) plo[o + i] = (T)(v - (double)hi);
      if (xc) xc[(int64_t)i * kFastCols] = (float)v;
    }
  }
}

// v = hi + lo as float pairs (the exact matvec's input), elementwise.
__global__ void k_split(const double* __restrict__ v, int64_t len, float* __restrict__ hi,
                        float* __restrict__ lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float h = (float)v[i];
    hi[i] = h;
    lo[i] = (float)(v[i] - (double)h);
  }
}

// The difference x - x_a of every column, in the transposed group layout of
// k_matvec_stream ([group][row][16]); rows past n stay zero (the workspace is zeroed).
__global__ void k_diff_t(int n, int64_t ldv, const double* __restrict__ x,
                         const double* __restrict__ xa, float* __restrict__ xdt) {
  const int col = blockIdx.y;
  const int64_t o = (int64_t)col * ldv;
  float* xc = xdt + ((int64_t)(col / kFastCols) * ldv * kFastCols + col % kFastCols);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    xc[(int64_t)i * kFastCols] = (float)(xa ? x[o + i] - xa[o + i] : x[o + i]);
}

// PCG-DC apply of the many-column solves of a float E: z = P r (+ p_gap sum r) for the
// 16 columns of a group in one pass over P (the per-column kernel above reads P once for
// every column).  rt holds r as floats in the streamed matvec's layout ([group][row][16]).
// A warp takes kDcRowsPerWarp consecutive rows, one at a time: it loads up to 128 of the
// row's entries at once (four coalesced loads of column indices and values a lane), then
// issues 16 independent 16-byte gathers a lane (lane l: entries 8 k + l / 4, columns
// 4 (l % 4) .. + 3, the index and value passed by shuffles) and sums the eight slots by
// shuffles at the row's end; the row's r and z are loaded before the gathers.  A row thus
// waits on three memory round trips, not one for every 32 entries, and the grid (64 rows
// a block, thousands of blocks) keeps every SM full.  The sums are float: P r is the
// preconditioner's output only (the flexible Polak-Ribiere step tolerates its rounding,
// ~1e-7 of z) and convergence is decided on replaced residuals.  Each block writes its
// partial dots [r^T z_new, r^T z_old] to dpart; k_dc_dots adds them in block order into
// the solver's dots (part 0; the other parts zero).  rsum_part may be the dots buffer
// itself (only slot 3 is read).
constexpr int kDcWarps = 8;
constexpr int kDcRowsPerWarp = 8;
constexpr int kDcRowsPerBlock = kDcWarps * kDcRowsPerWarp;
constexpr int kDcChunk = 128;  // entries loaded at once

__global__ void __launch_bounds__(kDcWarps * 32, 3)
k_dc_apply_t(int n, int64_t ldv, int nrhs, const ColState* __restrict__ st,
             const int64_t* __restrict__ off, const int* __restrict__ idx,
             const double* __restrict__ prow, double pgap, const float* __restrict__ rt,
             const double* __restrict__ r, double* __restrict__ z,
             const double* __restrict__ rsum_part, int nparts, double* __restrict__ dpart,
             int first) {
  __shared__ double s_gsum[kFastCols];
  __shared__ int s_active[kFastCols];
  __shared__ double s_red[kDcWarps][kFastCols][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = blockIdx.y, c0 = grp * kFastCols;
  for (int cc = warp; cc < kFastCols; cc += kDcWarps) {  // p_gap sums and active flags
    const int col = c0 + cc;
    double sr = 0.0;
    if (col < nrhs && pgap != 0.0)
      for (int b = lane; b < nparts; b += 32) sr += rsum_part[((int64_t)b * nrhs + col) * 4 + 3];
    sr = warp_sum(sr);
    if (lane == 0) {
      s_gsum[cc] = pgap * sr;
      s_active[cc] = col < nrhs && (first || st[col].done == 0);
    }
  }
  __syncthreads();
  const int slot = lane >> 2, cq = 4 * (lane & 3);
  // after the shuffles every lane holds its four columns' sums; lane l < 16 finishes
  // column c = 4 (l % 4) + l / 4, component l / 4 of its float4
  const int cf = cq + slot, comp = slot;
  const bool fin = lane < 16 && c0 + cf < nrhs;
  const bool act = fin && s_active[cf];
  const double gsum = fin ? s_gsum[cf] : 0.0;
  const int64_t oz = (int64_t)(c0 + cf) * ldv;
  const float* rg = rt + (int64_t)grp * ldv * kFastCols + cq;
  const int jw = blockIdx.x * kDcRowsPerBlock + warp * kDcRowsPerWarp;
  double v0 = 0.0, v1 = 0.0;
  for (int j = jw; j < min(n, jw + kDcRowsPerWarp); ++j) {
    double rj = 0.0, zo = 0.0;
    if (fin) {  // issued ahead of the gathers
      rj = r[oz + j];
      zo = z[oz + j];
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t e1 = off[j + 1];
    for (int64_t eb = off[j]; eb < e1; eb += kDcChunk) {
      const int left = (int)min((int64_t)kDcChunk, e1 - eb);  // entries in this chunk
      int id[kDcChunk / 32];
      float pe[kDcChunk / 32];
#pragma unroll
      for (int m = 0; m < kDcChunk / 32; ++m) {
        const int t = 32 * m + lane;
        id[m] = t < left ? __ldg(idx + eb + t) : 0;
        pe[m] = t < left ? (float)__ldg(prow + eb + t) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < kDcChunk / 8; ++k) {
        const int src = 8 * k + slot;  // entry of this chunk: load m = k / 4, lane 8 (k % 4) + slot
        const int ik = __shfl_sync(0xffffffffu, id[k >> 2], 8 * (k & 3) + slot);
        const float pk = __shfl_sync(0xffffffffu, pe[k >> 2], 8 * (k & 3) + slot);
        if (src < left) {
          const float4 rv = __ldg(reinterpret_cast<const float4*>(rg + (int64_t)ik * kFastCols));
          acc.x = fmaf(pk, rv.x, acc.x);
          acc.y = fmaf(pk, rv.y, acc.y);
          acc.z = fmaf(pk, rv.z, acc.z);
          acc.w = fmaf(pk, rv.w, acc.w);
        }
      }
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
    }
    if (fin) {
      const float a = comp == 0 ? acc.x : comp == 1 ? acc.y : comp == 2 ? acc.z : acc.w;
      const double zn = gsum + (double)a;
      if (act) z[oz + j] = zn;
      v0 += rj * zn;
      v1 += rj * zo;
    }
  }
  if (lane < 16) {
    s_red[warp][cf][0] = v0;
    s_red[warp][cf][1] = v1;
  }
  __syncthreads();
  if (threadIdx.x < 2 * kFastCols) {
    const int cc = threadIdx.x >> 1, t = threadIdx.x & 1;
    double sv = 0.0;
#pragma unroll
    for (int w = 0; w < kDcWarps; ++w) sv += s_red[w][cc][t];
    if (c0 + cc < nrhs) dpart[((int64_t)blockIdx.x * nrhs + c0 + cc) * 2 + t] = sv;
  }
}

// The blocks' partial dots of k_dc_apply_t, added in block order: part 0 of slots 0 and 1
// of every column takes the sums, parts 1 .. nparts - 1 zero (the readers add all parts).
__global__ void k_dc_dots(const double* __restrict__ dpart, int nblk, int nrhs,
                          double* __restrict__ dots, int nparts) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= nrhs) return;
  double s0 = 0.0, s1 = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    s0 += dpart[((int64_t)b * nrhs + col) * 2];
    s1 += dpart[((int64_t)b * nrhs + col) * 2 + 1];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  for (int b = lane; b < nparts; b += 32) {
    dots[((int64_t)b * nrhs + col) * 4] = b == 0 ? s0 : 0.0;
    dots[((int64_t)b * nrhs + col) * 4 + 1] = b == 0 ? s1 : 0.0;
  }
}

// Columns that broke down in the fast iteration count as converged for the next
// replacement, which recomputes their residual exactly and reopens them (restart).
__global__ void k_reopen_broken(ColState* __restrict__ st, int nrhs) {
  for (int col = threadIdx.x; col < nrhs; col += blockDim.x)
    if (st[col].done == 2) st[col].done = 1;
}

// Residual replacement from the anchor: r = r_a - q with q = E (x - x_a) from the fast
// matvec; otherwise as k_replace_r.
__global__ void __launch_bounds__(kThreads)
k_anchor_r(int n, int64_t ldv, int nrhs, const ColState* __restrict__ st,
           const double* __restrict__ ra, const double* __restrict__ q, double* __restrict__ r,
           double* __restrict__ z, const double* __restrict__ inv_diag, int pre,
           double* __restrict__ dots) {
  __shared__ double sm[32 * 4];
  const int col = blockIdx.y;
  if (st[col].done == 2) return;
  double v[4] = {0, 0, 0, 0};
  const int64_t o = (int64_t)col * ldv;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ri = ra[o + i] - q[o + i];
    r[o + i] = ri;
    if (pre != CPM_PRECOND_DC) {
      const double zi = pre == CPM_PRECOND_JACOBI ? ri * inv_diag[i] : ri;
      z[o + i] = zi;
      v[0] += ri * zi;
    }
    v[2] += ri * ri;
    v[3] += ri;
  }
  block_sum<4>(v, sm);
  if (threadIdx.x == 0)
    for (int t = 0; t < 4; ++t) dots[((int64_t)blockIdx.x * nrhs + col) * 4 + t] = v[t];
}

// Residual replacement, first part: r = b bscale - q with q = E x from the exact matvec;
// Jacobi / none also form z; partial dots [r^T z, -, r^T r, sum r] as k_update writes
// them (PCG-DC forms z in k_dc_apply next).  Columns that broke down are left alone.
__global__ void __launch_bounds__(kThreads)
k_replace_r(int n, int64_t ldv, int nrhs, const ColState* __restrict__ st,
            const double* __restrict__ b, double bscale, const double* __restrict__ q,
            double* __restrict__ r, double* __restrict__ z, const double* __restrict__ inv_diag,
            int pre, double* __restrict__ dots) {
  __shared__ double sm[32 * 4];
  const int col = blockIdx.y;
  if (st[col].done == 2) return;  // uniform per block; its dots are not read
  double v[4] = {0, 0, 0, 0};
  const int64_t o = (int64_t)col * ldv;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ri = b[(int64_t)col * n + i] * bscale - q[o + i];
    r[o + i] = ri;
    if (pre != CPM_PRECOND_DC) {
      const double zi = pre == CPM_PRECOND_JACOBI ? ri * inv_diag[i] : ri;
      z[o + i] = zi;
      v[0] += ri * zi;
    }
    v[2] += ri * ri;
    v[3] += ri;
  }
  block_sum<4>(v, sm);
  if (threadIdx.x == 0)
    for (int t = 0; t < 4; ++t) dots[((int64_t)blockIdx.x * nrhs + col) * 4 + t] = v[t];
}

// Residual replacement, second part: the true relative residual decides convergence; a
// column that had converged on its recursive residual but not on the true one runs again
// from p = z (restart flag); every running column continues with the replaced r, z and
// r^T z and its direction unchanged.
__global__ void k_replace_state(const double* __restrict__ dots, int nparts, int nrhs,
                                double tol, ColState* __restrict__ st) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= nrhs) return;
  double s0 = 0.0, s2 = 0.0;
  for (int b = lane; b < nparts; b += 32) {
    s0 += dots[((int64_t)b * nrhs + col) * 4 + 0];
    s2 += dots[((int64_t)b * nrhs + col) * 4 + 2];
  }
  s0 = warp_sum(s0);
  s2 = warp_sum(s2);
  if (lane == 0) {
    ColState c = st[col];
    if (c.done != 2) {
      c.relres = c.bb > 0.0 ? sqrt(s2 / c.bb) : 0.0;
      c.rz = s0;
      if (!isfinite(c.relres)) {
        c.done = 2;
      } else if (c.relres <= tol) {
        c.done = 1;
      } else {
        c.restart = c.done == 1 ? 1 : 0;
        c.done = 0;
        if (!(c.rz != 0.0)) c.done = 2;
      }
      if (c.done) c.restart = 0;
    }
    st[col] = c;
  }
}

// r = b - E x0 (q [+ q2] holds E x0 when use_guess) or r = b; x = x0 or 0.
__global__ void k_init_r(int n, int64_t ldv, int nrhs, const double* __restrict__ b,
                         double bscale, const double* __restrict__ q,
                         const double* __restrict__ q2, int use_guess, double* __restrict__ r,
                         double* __restrict__ x, double* __restrict__ z,
                         const double* __restrict__ inv_diag, int pre,
                         double* __restrict__ dots, const SysCol* __restrict__ sys) {
  __shared__ double sm[32 * 4];
  {
    const int col = blockIdx.y;
    const int64_t o = (int64_t)col * ldv;
    int nc = n;  // rows of this column's system (b rows are n apart)
    if (sys) {
      nc = sys[col].n;
      inv_diag = sys[col].inv_diag;
    }
    double v[4] = {0, 0, 0, 0};  // r^T z, b^T b, r^T r, sum r
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
      const double bi = b[(int64_t)col * n + i] * bscale;
      const double ri = use_guess ? bi - q[o + i] - (q2 ? q2[o + i] : 0.0) : bi;
      r[o + i] = ri;
      if (!use_guess) x[o + i] = 0.0;
      double zi = 0.0;
      if (pre != CPM_PRECOND_DC) {
        zi = pre == CPM_PRECOND_JACOBI ? ri * inv_diag[i] : ri;
        z[o + i] = zi;
      } else {
        z[o + i] = 0.0;
      }
      v[0] += ri * zi;
      v[1] += bi * bi;
      v[2] += ri * ri;
      v[3] += ri;
    }
    block_sum<4>(v, sm);
    if (threadIdx.x == 0)
      for (int t = 0; t < 4; ++t) dots[((int64_t)blockIdx.x * nrhs + col) * 4 + t] = v[t];
  }
}

__global__ void k_init_state(const double* __restrict__ dots, int nparts, int nrhs,
                             double tol, int pre, ColState* __restrict__ st) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= nrhs) return;
  double s[3] = {0, 0, 0};
  for (int b = lane; b < nparts; b += 32)
    for (int t = 0; t < 3; ++t) s[t] += dots[((int64_t)b * nrhs + col) * 4 + t];
  for (int t = 0; t < 3; ++t) s[t] = warp_sum(s[t]);
  (void)pre;
  if (lane == 0) {
    ColState c;
    c.rz = s[0];
    c.bb = s[1];
    c.alpha = 0.0;
    c.beta = 0.0;
    c.iter = 0;
    c.done = 0;
    c.restart = 0;
    c.pad_ = 0;
    if (c.bb == 0.0) {
      c.relres = 0.0;
      c.done = 1;
    } else {
      c.relres = sqrt(s[2] / c.bb);
      if (c.relres <= tol) c.done = 1;
    }
    st[col] = c;
  }
}

// The DC apply in the init phase writes r^T z into slot 0 of its own dots array.
__global__ void k_init_rz_dc(const double* __restrict__ dots_dc, int nparts, int nrhs,
                             ColState* __restrict__ st) {
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= nrhs) return;
  double s = 0.0;
  for (int b = lane; b < nparts; b += 32) s += dots_dc[((int64_t)b * nrhs + col) * 4];
  s = warp_sum(s);
  if (lane == 0) st[col].rz = s;
}

__global__ void k_neutralize(double* __restrict__ q, int n, const double* __restrict__ d,
                             const double* __restrict__ qsol) {
  __shared__ double sm[32];
  __shared__ double s_tot;
  const int col = blockIdx.x;
  double* qc = q + (int64_t)col * n;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[0] += qc[i];
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) s_tot = v[0] + (qsol ? qsol[col] : 0.0);
  __syncthreads();
  const double t = s_tot;
  for (int i = threadIdx.x; i < n; i += blockDim.x) qc[i] -= t * d[i];
}

__global__ void k_neutralize_ragged(double* __restrict__ q, int64_t ld,
                                    const SysCol* __restrict__ sys,
                                    const double* __restrict__ qsol) {
  __shared__ double sm[32];
  __shared__ double s_tot;
  const int col = blockIdx.x;
  const int n = sys[col].n;
  const double* d = sys[col].d;
  double* qc = q + (int64_t)col * ld;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[0] += qc[i];
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) s_tot = v[0] + (qsol ? qsol[col] : 0.0);
  __syncthreads();
  const double t = s_tot;
  for (int i = threadIdx.x; i < n; i += blockDim.x) qc[i] -= t * d[i];
}

// nrhs columns of n doubles between layouts with leading dimensions ldd and lds (device
// to device): one strided copy instead of one call per column.
cudaError_t copy_cols(double* dst, int64_t ldd, const double* src, int64_t lds, int n,
                      int nrhs, cudaStream_t s) {
  if (ldd == n && lds == n)
    return cudaMemcpyAsync(dst, src, (size_t)nrhs * n * sizeof(double), cudaMemcpyDeviceToDevice,
                           s);
  return cudaMemcpy2DAsync(dst, ldd * sizeof(double), src, lds * sizeof(double),
                           n * sizeof(double), nrhs, cudaMemcpyDeviceToDevice, s);
}

int sm_count(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v > 0 ? v : 1;
}

// Number of per-block p^T q partials a matvec writes (the block count of its launches).
// Float matvec shape: eight warps split long rows (at least 16 groups of 128 columns),
// otherwise every warp owns its rows.
bool mv_split_rows(const Ctx* c) { return (c->ldE >> 7) >= 16; }

int matvec_parts(const Ctx* c) {
  if (c->fp64()) return std::max(1, std::min((c->n + kMvWarps - 1) / kMvWarps, 4 * sm_count(c->device)));
  const int rbb = mv_split_rows(c) ? kMvRows : kMvRows * kMvWarps;
  return (c->n + rbb - 1) / rbb;
}

template <typename T>
void launch_matvec(const Ctx* c, const void* pv, const void* plo, const double* p64,
                   int64_t ldv, int nrhs, double* q, double* pq_part, int gm,
                   const ColState* st);

// Launches KERNEL<NR> over all nrhs columns: full groups of four columns as grid rows of
// one launch, then a pair and a single column for the remainder.
template <typename Launch>
void for_column_groups(int nrhs, Launch&& launch) {
  const int groups = nrhs / 4;
  for (int g0 = 0; g0 < groups; g0 += 65535)
    launch(std::integral_constant<int, 4>(), 4 * g0, std::min(groups - g0, 65535));
  int c0 = 4 * groups;
  if (nrhs - c0 >= 2) {
    launch(std::integral_constant<int, 2>(), c0, 1);
    c0 += 2;
  }
  if (nrhs - c0 == 1) launch(std::integral_constant<int, 1>(), c0, 1);
}

// FP64 storage (the plain baseline build): one warp per row, FP64 products and sums.
template <>
void launch_matvec<double>(const Ctx* c, const void* pv, const void*, const double*,
                           int64_t ldv, int nrhs, double* q, double* pq_part, int gm,
                           const ColState* st) {
  const double* E = (const double*)c->E.ptr;
  const double* hi = (const double*)pv;
  for_column_groups(nrhs, [&](auto nr, int c0, int ny) {
    (k_matvec_f64<decltype(nr)::value><<<dim3(gm, ny), kThreads, 0, c->stream>>>(
         E, c->ldE, c->n, hi, ldv, c0, nrhs, q, pq_part, st), note_launch());
  });
}

// FP32 storage: k_matvec_f32, four columns per pass over E.
template <>
void launch_matvec<float>(const Ctx* c, const void* pv, const void* plo, const double* p64,
                          int64_t ldv, int nrhs, double* q, double* pq_part, int gm,
                          const ColState* st) {
  const float* E = (const float*)c->E.ptr;
  const float* hi = (const float*)pv;
  const float* lo = (const float*)plo;
  const bool split = mv_split_rows(c);
  for_column_groups(nrhs, [&](auto nr, int c0, int ny) {
    constexpr int NR = decltype(nr)::value;
    if (split)
      (k_matvec_f32<NR, kMvWarps><<<dim3(gm, ny), kThreads, 0, c->stream>>>(
           E, c->ldE, c->n, hi, lo, p64, ldv, c0, nrhs, q, pq_part, st), note_launch());
    else
      (k_matvec_f32<NR, 1><<<dim3(gm, ny), kThreads, 0, c->stream>>>(
           E, c->ldE, c->n, hi, lo, p64, ldv, c0, nrhs, q, pq_part, st), note_launch());
  });
}

}  // namespace

namespace {
int pcg_solve_kernels(Ctx* c, const SolveArgs& a);
}  // namespace

// The solve: the cluster-resident kernel (small electrodes) or the host-driven kernels.
// With solver_path 0 the choice is the context's online autotuner's: for each bucket of
// right-hand-side counts, the first eligible solve runs on the cluster path and the next
// on the host-driven one, each timed per iteration on the device; later solves of that
// bucket take the faster.  Both give the same iteration on the same matrix.
int pcg_solve(Ctx* c, const SolveArgs& a) {
  const bool eligible = !c->fp64() && !a.sys && !a.ws && c->n <= cluster_solve_max_atoms() &&
                        c->p.solver_path != 1;
  int bucket = 0;
  while (bucket < 7 && (2 << bucket) <= a.nrhs) ++bucket;
  int path = 1;
  if (eligible) {
    if (c->p.solver_path == 2) path = 2;
    else if (c->tune_path[bucket]) path = c->tune_path[bucket];
    else path = c->tune_cost[bucket][1] > 0.f ? 1 : 2;  // try the cluster path first
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool tuning = eligible && c->p.solver_path == 0 && !c->tune_path[bucket];
  if (tuning) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
  }
  int st = path == 2 ? pcg_solve_cluster(c, a) : pcg_solve_kernels(c, a);
  c->last_solve_path = path;
  if (tuning) {
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int iters = 1;
    for (int col = 0; a.iters && col < a.nrhs; ++col) iters = std::max(iters, a.iters[col]);
    if (st == CPM_OK || st == CPM_ENOCONV) {
      c->tune_cost[bucket][path - 1] = ms / iters;
      if (c->tune_cost[bucket][0] > 0.f && c->tune_cost[bucket][1] > 0.f)
        c->tune_path[bucket] = c->tune_cost[bucket][1] < c->tune_cost[bucket][0] ? 2 : 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return st;
}

namespace {

int pcg_solve_kernels(Ctx* c, const SolveArgs& a) {
  const int n = c->n, nrhs = a.nrhs;
  const int64_t ldv = c->ldE;
  const int sms = sm_count(c->device);
  // elementwise kernels: ge blocks per right-hand side, one grid row per right-hand side
  const int ge = std::max(1, std::min((n + kThreads - 1) / kThreads, 2 * sms));
  const dim3 g2(ge, nrhs);
  // p^T q partials per column: one per matvec block (the ragged kernel takes kMvRows rows
  // per block)
  const int gm_exact = a.sys ? (n + kMvRows - 1) / kMvRows : matvec_parts(c);
  // PCG-Normal and PCG-Full apply their P in the row form PCG-DC's takes
  const int pre = c->p.precond >= CPM_PRECOND_DC ? CPM_PRECOND_DC : c->p.precond;
  const bool f64 = c->fp64();
  // many columns of one float E: the inner iterations stream E once for every group of
  // 16 columns (k_matvec_stream, float sums), and a replaced residual takes the place of the
  // recursive one whenever a column's residual has fallen 100-fold since the last
  // replacement or it reports convergence; convergence is declared on replaced residuals
  // only.  A replacement is b - E x through the exact matvec (an anchor), or, once every
  // running column's anchor is within 1e-2 of its b, r_a - E (x - x_a) through the fast
  // matvec: the error of the fast sums then scales with the anchor's residual, not with
  // E x.  A breakdown in the fast iteration (its float sums can turn p^T E p negative near
  // a tight tolerance) switches the solve to the exact matvec for good, and the broken
  // columns start again from an exact residual.
  const bool fast0 = !f64 && !a.sys && nrhs >= 2 && c->p.matvec_mode == 0;
  bool fast = fast0;
  const int gm_fast = (n + kStRows - 1) / kStRows;  // row blocks of the streamed matvec
  int gm = fast ? gm_fast : gm_exact;
  const int groups = (nrhs + kFastCols - 1) / kFastCols;
  const size_t vbytes = (size_t)nrhs * ldv * sizeof(double);
  // the streamed matvec's units: row blocks x shares per group of a launch
  const int nst = (int)(c->ldE / kStK);
  const int glaunch = std::min(groups, 65535);
  const int splits = fast ? stream_splits(gm_fast, glaunch, nst, sms) : 1;
  const size_t cnt_bytes = (size_t)glaunch * gm_fast * sizeof(unsigned);
  const int nblk_dc = (n + kDcRowsPerBlock - 1) / kDcRowsPerBlock;  // blocks of the DC apply
  // layout: x r z p q (double) | pv (storage type) | [fast: xt | x hi | x lo | x - x_a |
  //         x_a | r_a | unit partials | counters, error flag] | pq_part | dots | dots_dc |
  //         states
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t ox = take(vbytes), orr = take(vbytes), oz = take(vbytes), op = take(vbytes),
               oq = take(vbytes), opv = take((f64 ? 1 : 2) * (size_t)nrhs * ldv * c->esz()),
               oxt = fast ? take((size_t)groups * kFastCols * ldv * sizeof(float)) : 0,
               oxs = fast ? take(2 * (size_t)nrhs * ldv * sizeof(float)) : 0,
               oxd = fast ? take((size_t)groups * kFastCols * ldv * sizeof(float)) : 0,
               oxa = fast ? take(vbytes) : 0, ora = fast ? take(vbytes) : 0,
               opart = fast && splits > 1
                           ? take((size_t)glaunch * gm_fast * splits * kStOut * sizeof(double))
                           : 0,
               ocnt = fast ? take(cnt_bytes + sizeof(int)) : 0,
               odp = fast ? take((size_t)nblk_dc * nrhs * 2 * sizeof(double)) : 0,
               opq = take((size_t)std::max(gm_fast, gm_exact) * nrhs * sizeof(double)),
               odt = take((size_t)ge * nrhs * 4 * sizeof(double)),
               odc = take((size_t)ge * nrhs * 4 * sizeof(double)),
               ost = take(2 * (size_t)nrhs * sizeof(ColState));
  int rc;
  char* base;
  if (a.ws) {  // caller-provided workspace (never grown)
    if (off > a.ws_bytes)
      return set_err(c, CPM_EINVAL, "solve workspace needs " + std::to_string(off) +
                                        " bytes; the fixed workspace holds " +
                                        std::to_string(a.ws_bytes));
    base = (char*)a.ws;
  } else {
    if ((rc = buf_reserve(c, &c->ws_solve, off))) return rc;
    base = (char*)c->ws_solve.ptr;
  }
  double* x = (double*)(base + ox);
  double* r = (double*)(base + orr);
  double* z = (double*)(base + oz);
  double* p = (double*)(base + op);
  double* q = (double*)(base + oq);
  void* pv = base + opv;
  // float storage: the low halves of the direction follow the high halves
  float* plo = f64 ? nullptr : (float*)pv + (size_t)nrhs * ldv;
  double* pq_part = (double*)(base + opq);
  double* dots = (double*)(base + odt);
  double* dots_dc = (double*)(base + odc);
  ColState* st = (ColState*)(base + ost);
  float* xt = fast ? (float*)(base + oxt) : nullptr;
  float* xhi = fast ? (float*)(base + oxs) : nullptr;
  float* xlo = fast ? xhi + (size_t)nrhs * ldv : nullptr;
  float* xdt = fast ? (float*)(base + oxd) : nullptr;  // x - x_a, transposed per group
  double* xa = fast ? (double*)(base + oxa) : nullptr;  // the anchor's x and r
  double* ra = fast ? (double*)(base + ora) : nullptr;
  double* dpart = fast ? (double*)(base + odp) : nullptr;  // the DC apply's block dots
  cudaStream_t s = c->stream;
  // the streamed matvec: its TMA map of E, units' partials and counters (zeroed above)
  CUtensorMap emap;
  double* part = fast && splits > 1 ? (double*)(base + opart) : nullptr;
  unsigned* counts = fast ? (unsigned*)(base + ocnt) : nullptr;
  int* mv_err = fast ? (int*)(base + ocnt + cnt_bytes) : nullptr;
  if (fast) {
    if (!make_stream_map(&emap, (const float*)c->E.ptr, n, c->ldE))
      return set_err(c, CPM_ECUDA, "TMA map of E for the streamed matvec");
    if (cuda_check(c, cudaFuncSetAttribute(k_matvec_stream,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kStSmem),
                   "streamed matvec smem"))
      return CPM_ECUDA;
  }
  auto stream_mv = [&](const float* xin, const ColState* cur) {
    StreamArgs sa{n, nst, splits, gm_fast, xin, p, ldv, 0, nrhs, part, counts, q, pq_part, cur,
                  mv_err};
    for (int g0 = 0; g0 < groups; g0 += 65535) {
      sa.g0 = g0;
      (k_matvec_stream<<<dim3(gm_fast * splits, std::min(groups - g0, 65535)), kStThreads,
                         kStSmem, s>>>(emap, sa),
       note_launch());
    }
  };
  // device timing of the solve's parts: event pairs from the context's pool
  size_t nev = 0;
  auto ev = [&]() -> cudaEvent_t {
    if (!a.timed) return nullptr;
    if (nev == c->ev_pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->ev_pool.push_back(e);
    }
    cudaEvent_t e = c->ev_pool[nev++];
    cudaEventRecord(e, c->stream);
    return e;
  };
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> t_mv, t_rep, t_dc;
  const cudaEvent_t t_begin = ev();
  // cur: the column states (converged columns are skipped), nullptr before they exist
  // z = P r for PCG-DC: the many-column float path in one pass over P for each group of
  // 16 columns (r first transposed to floats into the x - x_a buffer, free at this point),
  // every other solve per column
  auto dc_apply = [&](const ColState* cur, double* dots_out, int first) {
    const cudaEvent_t d0 = ev();
    if (fast) {
      (k_diff_t<<<g2, kThreads, 0, s>>>(n, ldv, r, nullptr, xdt), note_launch());
      (k_dc_apply_t<<<dim3(nblk_dc, groups), kDcWarps * 32, 0, s>>>(
           n, ldv, nrhs, cur, (const int64_t*)c->nbr_off.ptr, (const int*)c->nbr_idx.ptr,
           (const double*)c->prow.ptr, c->pgap, xdt, r, z, dots, ge, dpart, first),
       note_launch());
      (k_dc_dots<<<(nrhs + 7) / 8, 256, 0, s>>>(dpart, nblk_dc, nrhs, dots_out, ge),
       note_launch());
    } else {
      (k_dc_apply<<<g2, kThreads, 0, s>>>(n, ldv, nrhs, cur, (const int64_t*)c->nbr_off.ptr,
                                         (const int*)c->nbr_idx.ptr, (const double*)c->prow.ptr,
                                         c->pgap, r, z, dots, ge, dots_out, first, a.sys),
       note_launch());
    }
    t_dc.emplace_back(d0, ev());
  };
  auto matvec = [&](const ColState* cur) {
    if (fast) {  // the inner matvec of a many-column solve
      stream_mv(xt, cur);
    } else if (f64) {
      launch_matvec<double>(c, pv, nullptr, p, ldv, nrhs, q, pq_part, gm, cur);
    } else if (a.sys) {  // ragged batch: one system per column
      (k_matvec_ragged<<<dim3(gm, nrhs), kThreads, 0, s>>>(a.sys, (const float*)pv, plo, p, ldv,
                                                           nrhs, q, pq_part, cur), note_launch());
    } else {
      launch_matvec<float>(c, pv, plo, p, ldv, nrhs, q, pq_part, gm, cur);
    }
  };
  // zero the padded vectors so the matvec can read whole padded rows
  if (cuda_check(c, cudaMemsetAsync(base, 0, ost, s), "memset")) return CPM_ECUDA;

  const double* inv_diag = c->diag.ptr ? (const double*)c->diag.ptr + n : nullptr;
  // initial guess: q = E x0 through the solve's matvec (a many-column solve: the streamed
  // float one; its r0 is no anchor, and the first replacement recomputes b - E x exactly)
  const double* q2 = nullptr;
  if (a.use_guess) {
    if (cuda_check(c, copy_cols(x, ldv, a.x, n, n, nrhs, s), "copy guess")) return CPM_ECUDA;
    if (f64) (k_p_update<double><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, st, x, p, (double*)pv, nullptr, 1), note_launch());
    else (k_p_update<float><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, st, x, p, (float*)pv, plo, 1, xt), note_launch());
    if (fast) stream_mv(xt, nullptr);
    else matvec(nullptr);
  }
  const bool exact_r0 = !(fast && a.use_guess);
  (k_init_r<<<g2, kThreads, 0, s>>>(n, ldv, nrhs, a.b, a.bscale, q, q2, a.use_guess ? 1 : 0, r, x, z,
                                   inv_diag, pre, dots, a.sys), note_launch());
  const int wb = 8;  // warps per block for the per-column reductions
  const int gcol = (nrhs + wb - 1) / wb;
  (k_init_state<<<gcol, wb * 32, 0, s>>>(dots, ge, nrhs, a.tol, pre, st), note_launch());
  if (pre == CPM_PRECOND_DC) {
    dc_apply(st, dots_dc, 1);
    (k_init_rz_dc<<<gcol, wb * 32, 0, s>>>(dots_dc, ge, nrhs, st), note_launch());
  }
  if (f64) (k_p_update<double><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, st, z, p, (double*)pv, nullptr, 1), note_launch());
  else (k_p_update<float><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, st, z, p, (float*)pv, plo, 1, xt), note_launch());
  if (cuda_check(c, cudaGetLastError(), "pcg init")) return CPM_ECUDA;

  std::vector<ColState> host(nrhs);
  const int flexible = pre == CPM_PRECOND_DC ? 1 : 0;
  int it = 0;
  bool all_done = false;
  const int check_every = 4;
  // many-column solves: a column counts as converged once a replaced (true) residual says
  // so (verified); level is its relative residual at its last replacement
  std::vector<char> verified(nrhs, 0);
  std::vector<double> level(nrhs, 1.0);
  // state at the start of iteration `it` lives in st[(it & 1) * nrhs]
  auto poll = [&](int k) -> int {
    ColState* cur = st + (size_t)(k & 1) * nrhs;
    if (cuda_check(c, cudaMemcpyAsync(host.data(), cur, nrhs * sizeof(ColState),
                                      cudaMemcpyDeviceToHost, s),
                   "poll"))
      return CPM_ECUDA;
    int wait_err = 0;  // a bounded wait of the streamed matvec ran out
    if (mv_err && cuda_check(c, cudaMemcpyAsync(&wait_err, mv_err, sizeof(int),
                                                cudaMemcpyDeviceToHost, s),
                             "poll"))
      return CPM_ECUDA;
    if (cuda_check(c, cudaStreamSynchronize(s), "poll sync")) return CPM_ECUDA;
    if (wait_err)
      return set_err(c, CPM_ECUDA, "streamed matvec: a copy did not land in time (code " +
                                       std::to_string(wait_err) + ")");
    all_done = true;
    for (int col = 0; col < nrhs; ++col)
      all_done &= host[col].done == 2 || (host[col].done == 1 && (!fast || verified[col]));
    return CPM_OK;
  };
  // residual replacement (many-column solves): r = b - E x through the exact matvec for
  // every column, then z, r^T z and the convergence test on the true residual
  const int64_t vlen = (int64_t)nrhs * ldv;
  std::vector<double> anchor_level(nrhs, 1.0);  // relres at each column's anchor
  auto replace = [&](int k) -> int {
    ColState* cur = st + (size_t)(k & 1) * nrhs;
    const cudaEvent_t e0 = ev();
    // the fast sums' error (~1e-5 of |E (x - x_a)|, i.e. of the anchor's residual) must
    // stay a tenth of the tolerance: anchors within min(1e-2, 1e4 tol) of b
    bool from_anchor = fast;
    const double near = std::min(1e-2, 1e4 * a.tol);
    for (int col = 0; col < nrhs; ++col)
      if (host[col].done != 2 && anchor_level[col] > near) from_anchor = false;
    const int gvec = (int)std::min<int64_t>((vlen + kThreads - 1) / kThreads, 4 * sms);
    if (from_anchor) {  // r = r_a - E_fast (x - x_a)
      (k_diff_t<<<g2, kThreads, 0, s>>>(n, ldv, x, xa, xdt), note_launch());
      stream_mv(xdt, nullptr);
      (k_anchor_r<<<g2, kThreads, 0, s>>>(n, ldv, nrhs, cur, ra, q, r, z, inv_diag, pre, dots),
       note_launch());
    } else {  // r = b - E x, exactly; the new anchor
      (k_split<<<gvec, kThreads, 0, s>>>(x, vlen, xhi, xlo), note_launch());
      launch_matvec<float>(c, xhi, xlo, x, ldv, nrhs, q, pq_part, gm_exact, nullptr);
      (k_replace_r<<<g2, kThreads, 0, s>>>(n, ldv, nrhs, cur, a.b, a.bscale, q, r, z, inv_diag,
                                           pre, dots), note_launch());
      if (cuda_check(c, cudaMemcpyAsync(xa, x, vbytes, cudaMemcpyDeviceToDevice, s), "anchor x") ||
          cuda_check(c, cudaMemcpyAsync(ra, r, vbytes, cudaMemcpyDeviceToDevice, s), "anchor r"))
        return CPM_ECUDA;
    }
    if (pre == CPM_PRECOND_DC) dc_apply(cur, dots, 1);
    (k_replace_state<<<gcol, wb * 32, 0, s>>>(dots, ge, nrhs, a.tol, cur), note_launch());
    (k_p_update<float><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, cur, z, p, (float*)pv, plo, 2, xt),
     note_launch());
    t_rep.emplace_back(e0, ev());
    if (cuda_check(c, cudaGetLastError(), "residual replacement")) return CPM_ECUDA;
    if (int e = poll(k)) return e;
    for (int col = 0; col < nrhs; ++col) {
      level[col] = host[col].relres;
      verified[col] = host[col].done == 1;
      if (!from_anchor) anchor_level[col] = host[col].relres;
    }
    return poll(k);  // all_done with the verified flags
  };
  if ((rc = poll(0))) return rc;
  for (int col = 0; col < nrhs; ++col) {  // an exact r0 is the first anchor
    verified[col] = exact_r0 && host[col].done == 1;
    anchor_level[col] = exact_r0 ? host[col].relres : 1.0;
  }
  if (fast && (cuda_check(c, cudaMemcpyAsync(xa, x, vbytes, cudaMemcpyDeviceToDevice, s),
                          "anchor x") ||
               cuda_check(c, cudaMemcpyAsync(ra, r, vbytes, cudaMemcpyDeviceToDevice, s),
                          "anchor r")))
    return CPM_ECUDA;
  if ((rc = poll(0))) return rc;
  while (!all_done && it < a.maxit) {
    ColState* cur = st + (size_t)(it & 1) * nrhs;
    ColState* nxt = st + (size_t)((it + 1) & 1) * nrhs;
    const cudaEvent_t m0 = ev();
    matvec(cur);
    t_mv.emplace_back(m0, ev());
    (k_alpha<<<gcol, wb * 32, 0, s>>>(pq_part, gm, nrhs, cur), note_launch());
    if (pre == CPM_PRECOND_DC) {
      (k_update<CPM_PRECOND_DC><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, cur, x, r, z, p, q,
                                                       inv_diag, dots, a.sys), note_launch());
      dc_apply(cur, dots, 0);
    } else if (pre == CPM_PRECOND_JACOBI) {
      (k_update<CPM_PRECOND_JACOBI><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, cur, x, r, z, p, q,
                                                           inv_diag, dots, a.sys), note_launch());
    } else {
      (k_update<CPM_PRECOND_NONE><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, cur, x, r, z, p, q,
                                                         inv_diag, dots, a.sys), note_launch());
    }
    (k_beta<<<gcol, wb * 32, 0, s>>>(dots, ge, nrhs, a.tol, flexible, cur, nxt), note_launch());
    if (f64) (k_p_update<double><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, nxt, z, p, (double*)pv, nullptr, 0), note_launch());
    else (k_p_update<float><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, nxt, z, p, (float*)pv, plo, 0, fast ? xt : nullptr), note_launch());
    ++it;
    if (it % check_every == 0 || it == a.maxit) {
      if (cuda_check(c, cudaGetLastError(), "pcg iteration")) return CPM_ECUDA;
      if ((rc = poll(it))) return rc;
      bool broke = false;  // a column broke down in the fast iteration
      for (int col = 0; fast && col < nrhs; ++col) broke |= host[col].done == 2;
      if (fast0 && (!all_done || broke)) {
        bool need = it == a.maxit;
        for (int col = 0; col < nrhs; ++col) {
          const ColState& h = host[col];
          need |= (h.done == 1 && !verified[col]) || (h.done == 0 && h.relres <= 1e-2 * level[col]);
        }
        if (broke) {  // the exact matvec from here on; broken columns start again
          fast = false;
          gm = gm_exact;
          (k_reopen_broken<<<1, 256, 0, s>>>(st + (size_t)(it & 1) * nrhs, nrhs), note_launch());
          for (int col = 0; col < nrhs; ++col) anchor_level[col] = 1.0;
          need = true;
        }
        if (need && (rc = replace(it))) return rc;
      }
    }
  }
  if (!all_done && (rc = poll(it))) return rc;
  if (cuda_check(c, copy_cols(a.x, n, x, ldv, n, nrhs, s), "copy x")) return CPM_ECUDA;
  const cudaEvent_t t_end = ev();
  if (cuda_check(c, cudaStreamSynchronize(s), "pcg end")) return CPM_ECUDA;
  if (a.timed) {
    float ms = 0;
    cudaEventElapsedTime(&c->t_solve_ms, t_begin, t_end);
    c->t_solve_mv_ms = c->t_solve_rep_ms = c->t_solve_dc_ms = 0;
    for (auto& e : t_mv) c->t_solve_mv_ms += (cudaEventElapsedTime(&ms, e.first, e.second), ms);
    for (auto& e : t_rep) c->t_solve_rep_ms += (cudaEventElapsedTime(&ms, e.first, e.second), ms);
    for (auto& e : t_dc) c->t_solve_dc_ms += (cudaEventElapsedTime(&ms, e.first, e.second), ms);
    c->solve_replacements = (int)t_rep.size();
  }
  int status = CPM_OK;
  for (int col = 0; col < nrhs; ++col) {
    if (a.iters) a.iters[col] = host[col].iter;
    if (a.relres) a.relres[col] = host[col].relres;
    if (host[col].done == 2) status = CPM_EBREAKDOWN;
    else if (host[col].done == 0 && status == CPM_OK) status = CPM_ENOCONV;
  }
  if (status == CPM_EBREAKDOWN) return set_err(c, status, "PCG breakdown (p^T E p <= 0 or non-finite)");
  if (status == CPM_ENOCONV) return set_err(c, status, "PCG reached maxit before tol");
  return CPM_OK;
}

}  // namespace

// q = E_n p for nrhs columns (device arrays [nrhs][n]) through the solver's matvec; the
// matvec launches alone are timed with events on the context's stream (t_matvec_ms).
int apply_E(Ctx* c, int nrhs, const double* p_in, double* q_out) {
  const int n = c->n;
  const int64_t ldv = c->ldE;
  const bool f64 = c->fp64();
  const int sms = sm_count(c->device);
  const int ge = std::max(1, std::min((n + kThreads - 1) / kThreads, 2 * sms));
  const int gm = matvec_parts(c);  // p^T q partials per column
  const size_t vbytes = ((size_t)nrhs * ldv * sizeof(double) + 255) & ~size_t(255);
  const size_t hbytes = ((f64 ? 1 : 2) * (size_t)nrhs * ldv * c->esz() + 255) & ~size_t(255);
  const size_t pqbytes = (size_t)gm * nrhs * sizeof(double);
  const size_t need = 3 * vbytes + hbytes + pqbytes + 2 * nrhs * sizeof(ColState);
  int rc = buf_reserve(c, &c->ws_solve, need);
  if (rc) return rc;
  char* base = (char*)c->ws_solve.ptr;
  double* p = (double*)base;
  double* q = (double*)(base + vbytes);
  double* zin = (double*)(base + 2 * vbytes);
  void* pv = base + 3 * vbytes;
  float* plo = f64 ? nullptr : (float*)pv + (size_t)nrhs * ldv;
  double* pq_part = (double*)(base + 3 * vbytes + hbytes);
  ColState* st = (ColState*)(base + 3 * vbytes + hbytes + pqbytes);
  cudaStream_t s = c->stream;
  if (cuda_check(c, cudaMemsetAsync(base, 0, 3 * vbytes + hbytes, s), "memset")) return CPM_ECUDA;
  if (cuda_check(c, copy_cols(zin, ldv, p_in, n, n, nrhs, s), "p in")) return CPM_ECUDA;
  const dim3 g2(ge, nrhs);
  // first = 1: p = zin, and its float pair
  if (f64) (k_p_update<double><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, st, zin, p, (double*)pv, nullptr, 1), note_launch());
  else (k_p_update<float><<<g2, kThreads, 0, s>>>(n, ldv, nrhs, st, zin, p, (float*)pv, plo, 1), note_launch());
  cudaEventRecord(c->ev_tc[0], s);
  if (f64) launch_matvec<double>(c, pv, nullptr, p, ldv, nrhs, q, pq_part, gm, nullptr);
  else launch_matvec<float>(c, pv, plo, p, ldv, nrhs, q, pq_part, gm, nullptr);
  cudaEventRecord(c->ev_tc[1], s);
  if (cuda_check(c, cudaGetLastError(), "apply_E")) return CPM_ECUDA;
  if (cuda_check(c, copy_cols(q_out, n, q, ldv, n, nrhs, s), "q out")) return CPM_ECUDA;
  if (cuda_check(c, cudaStreamSynchronize(s), "apply_E sync")) return CPM_ECUDA;
  cudaEventElapsedTime(&c->t_matvec_ms, c->ev_tc[0], c->ev_tc[1]);
  return CPM_OK;
}

void launch_neutralize_ragged(double* q, int count, int64_t ld, const SysCol* sys,
                              const double* qsol, cudaStream_t s) {
  (k_neutralize_ragged<<<count, 1024, 0, s>>>(q, ld, sys, qsol), note_launch());
}

void launch_neutralize(double* q, int nrhs, int n, const double* d, const double* qsol,
                       cudaStream_t s) {
  (k_neutralize<<<nrhs, 1024, 0, s>>>(q, n, d, qsol), note_launch());
}

}  // namespace cpm
