// Electrode interaction matrix: structure-factor operand and the SIMT k-space GEMM with
// the real-space, self and slab-dipole terms fused into its epilogue.
//
//   E_n[i][j] = sum_K W_K cos(K.(r_i - r_j))                         (Eq. 23)
//             + sum_{images, r < rc} [erfc(g r) - erfc(alpha_ij r)] / r (Eq. 22)
//             + (i == j) (-2 g / sqrt(pi) + sqrt(2/pi) alpha_i)       (Eq. 22, Eq. 6)
//             + (4 pi / V) z_i z_j                                     (Eq. 39, dipole part)
//
// The reciprocal sum is split by cos(a - b) = cos a cos b + sin a sin b into A A^T with
// A[i] = [sqrt(W) cos(K.r_i) | sqrt(W) sin(K.r_i)]: a dense contraction over 2M terms.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "cpm_internal.cuh"

namespace cpm {

namespace {

constexpr double kTwo32 = 4294967296.0;

__global__ void k_fixed_point_coords(const double* __restrict__ xyz, int n, int npad,
                                     double lx, double ly, double lz,
                                     uint32_t* __restrict__ sfix) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  double L[3] = {lx, ly, lz};
  for (int d = 0; d < 3; ++d) {
    uint32_t v = 0;
    if (i < n) {
      double s = xyz[3 * i + d] / L[d];
      s -= floor(s);  // [0, 1)
      // s * 2^32 rounded; 2^32 itself wraps to 0, which is the same phase
      unsigned long long q = (unsigned long long)llrint(s * kTwo32);
      v = (uint32_t)(q & 0xffffffffull);
    }
    sfix[3 * i + d] = v;
  }
}

// A[i][c(k)] = sqrt(W_k) cos(theta), A[i][c(k) + 64] = sqrt(W_k) sin(theta),
// theta = 2 pi (h s_x + k s_y + l s_z), with the columns in blocks of 64 k-vectors:
// c(k) = 128 (k / 64) + k % 64.  The table is sorted by decreasing W_k, so the columns
// run from the heaviest reciprocal terms to the lightest.
// FP32 operand: the phase fraction is formed exactly in 32-bit fixed point (integer
// h, k, l times 2^-32-quantised fractional coordinates, wrapping mod 1), then one
// rounding to float and sincospif.  FP64 operand: fractional coordinates in double,
// reduced to [-1/2, 1/2] by rint, then sincospi.
// 16-bit planes of the tensor-core build, written with A (the weight-bounded product
// schedule of K-block b, 64 columns):
//   kb0 <= b < kb6: BF16, a = a0 + a1 + a2, each plane the rounding of the remainder of
//     the previous (six products);
//   kb6 <= b < kb8: FP16 of the block's power-of-two scaled value x = 2^kexp[b] a
//     (|x| < 1), x = h0 + h1 below kb3 (three products), h0 alone from kb3 on (one);
//   kb8 <= b: FP8 E4M3 of x = 2^kexp[b] a (|x| < 256), one product, in its own byte plane.
// FP16 keeps 11 bits a plane against BF16's 8, so two planes and three products hold
// ~2^-21 of each product where BF16 needs six; the narrow exponent ranges of FP16 and
// FP8 are what the per-block scale is for.
struct PlaneOut {
  uint16_t* p[3];
  uint8_t* p8;
  const int* kexp;  // per K-block
  int kb0, kb6, kb3, kb8;
};

__device__ __forceinline__ void write_planes(const PlaneOut& po, size_t e, int b, float a) {
  if (b < po.kb0) return;
  if (b >= po.kb6) {
    const float x = a * __int_as_float((127 + po.kexp[b]) << 23);  // exact: a power of two
    if (b >= po.kb8) {
      po.p8[e] = (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
      return;
    }
    const __half h0 = __float2half_rn(x);
    po.p[0][e] = __half_as_ushort(h0);
    if (b < po.kb3) po.p[1][e] = __half_as_ushort(__float2half_rn(x - __half2float(h0)));
    return;
  }
  const __nv_bfloat16 b0 = __float2bfloat16_rn(a);
  po.p[0][e] = __bfloat16_as_ushort(b0);
  const float r1 = a - __bfloat162float(b0);
  const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
  po.p[1][e] = __bfloat16_as_ushort(b1);
  po.p[2][e] = __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(b1)));
}

// A (lda = 2 mpad) and, with PLANES, the BF16 planes for the k-vectors [kbeg, kend)
// (multiples of 64), the planes laid out over that window only: row stride
// 2 (kend - kbeg), column kcol - 2 kbeg.  A may be null (a streamed build keeps no A).
template <bool PLANES>
__global__ void k_structure_operand_f32(const uint32_t* __restrict__ sfix, int npad, int n,
                                        const int* __restrict__ hkl,
                                        const double* __restrict__ sqw, int mpad, int kbeg,
                                        int kend, const float4* __restrict__ turn,
                                        float* __restrict__ A, PlaneOut po) {
  int k = kbeg + blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kend) return;
  const uint32_t h = (uint32_t)hkl[3 * k], kk = (uint32_t)hkl[3 * k + 1],
                 l = (uint32_t)hkl[3 * k + 2];
  const float w = (float)sqw[k];
  const size_t lda = 2 * (size_t)mpad;
  const size_t ldp = 2 * (size_t)(kend - kbeg);
  const size_t kcol = 128 * (size_t)(k >> 6) + (k & 63);
  const size_t pcol = kcol - 2 * (size_t)kbeg;
  const int bc = (int)(kcol >> 6);  // K-block of the cos column; the sin column is bc + 1
  for (int i = blockIdx.y; i < npad; i += gridDim.y) {
    float c = 0.f, s = 0.f;
    if (i < n) {
      const uint32_t ph = h * sfix[3 * i] + kk * sfix[3 * i + 1] + l * sfix[3 * i + 2];
      sincos_table(ph, turn, &s, &c);
      c *= w;
      s *= w;
    }
    if (A) {
      A[i * lda + kcol] = c;
      A[i * lda + kcol + 64] = s;
    }
    if (PLANES) {
      write_planes(po, i * ldp + pcol, bc, c);
      write_planes(po, i * ldp + pcol + 64, bc + 1, s);
    }
  }
}

__global__ void k_structure_operand_f64(const double* __restrict__ xyz, int npad, int n,
                                        const int* __restrict__ hkl,
                                        const double* __restrict__ sqw, int mpad, double lx,
                                        double ly, double lz, double* __restrict__ A) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= mpad) return;
  const double h = hkl[3 * k], kk = hkl[3 * k + 1], l = hkl[3 * k + 2];
  const double w = sqw[k];
  const size_t lda = 2 * (size_t)mpad;
  const size_t kcol = 128 * (size_t)(k >> 6) + (k & 63);
  for (int i = blockIdx.y; i < npad; i += gridDim.y) {
    double c = 0.0, s = 0.0;
    if (i < n) {
      double fx = xyz[3 * i] / lx, fy = xyz[3 * i + 1] / ly, fz = xyz[3 * i + 2] / lz;
      fx -= floor(fx);
      fy -= floor(fy);
      fz -= floor(fz);
      double f = h * fx + kk * fy + l * fz;
      f -= rint(f);
      sincospi(2.0 * f, &s, &c);
      c *= w;
      s *= w;
    }
    A[i * lda + kcol] = c;
    A[i * lda + kcol + 64] = s;
  }
}

struct Epi {
  const double* xyz;
  const double* alpha;
  int n;
  double L[3];
  double rc2, rc, g;
  double self_g;    // -2 g / sqrt(pi)
  double dip;       // 4 pi / V if slab else 0
  // where r_c is below half of every box edge, so that only the nearest image of a pair
  // can lie within r_c: fractional coordinates x 2^32, the edges x 2^-32 and r_c^2 with
  // a 1e-4 margin, for a float screen of the nearest image (else sfix is null)
  const uint32_t* sfix;
  float Lq[3];
  float rc2_screen;
};

Epi make_epi(const double* xyz, const double* alpha, int n, const Geometry& geo) {
  Epi ep;
  ep.xyz = xyz;
  ep.alpha = alpha;
  ep.n = n;
  for (int d = 0; d < 3; ++d) ep.L[d] = geo.L[d];
  ep.rc = geo.rc;
  ep.rc2 = geo.rc * geo.rc;
  ep.g = geo.g;
  ep.self_g = -2.0 * geo.g / sqrt(kPi);
  ep.dip = geo.slab ? 4.0 * kPi / geo.vol : 0.0;
  bool one_image = geo.sfix != nullptr;
  for (int d = 0; d < 3; ++d) {
    one_image = one_image && 2.0 * geo.rc < geo.L[d];
    ep.Lq[d] = (float)(geo.L[d] * 0x1p-32);
  }
  ep.sfix = one_image ? geo.sfix : nullptr;
  ep.rc2_screen = (float)(ep.rc2 * (1.0 + 1e-4));
  return ep;
}

// Real-space, self and dipole terms of one (i, j) entry, in FP64.  A pair whose nearest
// image lies clearly beyond r_c (float distance from the exact fixed-point difference)
// has the dipole term alone; the FP64 image sum below would add nothing to it.
__device__ double epilogue_terms(const Epi& ep, int i, int j) {
  if (ep.sfix) {
    const uint32_t* si = ep.sfix + 3 * i;
    const uint32_t* sj = ep.sfix + 3 * j;
    float r2 = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float x = (float)(int32_t)(si[d] - sj[d]) * ep.Lq[d];
      r2 = fmaf(x, x, r2);
    }
    if (r2 > ep.rc2_screen) return 0.0 + ep.dip * ep.xyz[3 * i + 2] * ep.xyz[3 * j + 2];
  }
  const double* ri = ep.xyz + 3 * i;
  const double* rj = ep.xyz + 3 * j;
  double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
  double ai = ep.alpha[i], aj = ep.alpha[j];
  // alpha_ij^-2 = alpha_i^-2 + alpha_j^-2; inf (point charge) contributes 0
  double inv2 = (isinf(ai) ? 0.0 : 1.0 / (ai * ai)) + (isinf(aj) ? 0.0 : 1.0 / (aj * aj));
  double aij = inv2 > 0.0 ? rsqrt(inv2) : INFINITY;
  int lo[3], hi[3];
  for (int t = 0; t < 3; ++t) {
    lo[t] = (int)ceil((-ep.rc - d[t]) / ep.L[t]);
    hi[t] = (int)floor((ep.rc - d[t]) / ep.L[t]);
  }
  double acc = 0.0;
  for (int a = lo[0]; a <= hi[0]; ++a) {
    double x = d[0] + a * ep.L[0];
    for (int b = lo[1]; b <= hi[1]; ++b) {
      double y = d[1] + b * ep.L[1];
      double xy = x * x + y * y;
      if (xy >= ep.rc2) continue;
      for (int c = lo[2]; c <= hi[2]; ++c) {
        double z = d[2] + c * ep.L[2];
        double r2 = xy + z * z;
        if (r2 >= ep.rc2 || r2 == 0.0) continue;  // r == 0 only for the i == j, n = 0 term
        double r = sqrt(r2);
        double t = erfc(ep.g * r);
        if (!isinf(aij)) t -= erfc(aij * r);
        acc += t / r;
      }
    }
  }
  if (i == j) acc += ep.self_g + (isinf(ai) ? 0.0 : 0.7978845608028654 * ai);
  acc += ep.dip * ri[2] * rj[2];
  return acc;
}

// Lower-triangle tile index t -> (I, J), I >= J.
__device__ __forceinline__ void tri_tile(int t, int& I, int& J) {
  int r = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  I = r;
  J = t - r * (r + 1) / 2;
}

// SIMT structure-factor GEMM, 256 threads, tile BM x BM, BK = 16, TM x TM per thread.
//
// FP64 operand: plain double accumulation.
// FP32 operand (FLUSH): the columns run from the heaviest reciprocal weights to the
// lightest, and the accumulation follows that order:
//   * the first heavy_steps k-steps (16 columns each, the steps whose weights sum above
//     2e-3): the float products are exact in double and are accumulated in FP64
//     registers;
//   * afterwards float partial sums are added into FP64 accumulators in shared memory
//     at the steps flagged in flush_mask (chosen on the host so that each chunk's
//     weights sum to about 1e-3, and at most 32 steps), so float rounding acts only on
//     chunk sums of light terms.
template <typename T, int BM>
struct TilePipe {
  static constexpr int BK = 16;
  static constexpr int EPT = BM * BK / 256;   // elements of A loaded per thread per tile
  static constexpr int TPR = BK / EPT;        // threads per tile row
  static constexpr int VEC = 16 / sizeof(T);  // elements per 16-byte load
  static constexpr int PAD = 16 / sizeof(T);
  static_assert(EPT % VEC == 0, "tile load must be whole 16-byte vectors");
};

template <typename T, int BM, int TM, bool FLUSH>
__global__ void __launch_bounds__(256)
k_ek_simt(const T* __restrict__ A, int64_t lda, int ktot, T* __restrict__ E, int64_t ldE,
          Epi ep, int heavy_steps, const uint32_t* __restrict__ flush_mask) {
  using P = TilePipe<T, BM>;
  constexpr int BK = P::BK, EPT = P::EPT, TPR = P::TPR, VEC = P::VEC, PAD = P::PAD;
  __shared__ __align__(16) T As[2][BK][BM + PAD];
  __shared__ __align__(16) T Bs[2][BK][BM + PAD];
  extern __shared__ double accd_s[];  // [TM*TM][256] when FLUSH

  int I, J;
  tri_tile(blockIdx.x, I, J);
  const int i0 = I * BM, j0 = J * BM;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lrow = tid / TPR, lk = (tid % TPR) * EPT;
  const T* pa = A + (int64_t)(i0 + lrow) * lda + lk;
  const T* pb = A + (int64_t)(j0 + lrow) * lda + lk;
  T ra[EPT], rb[EPT];

  auto load_regs = [&](int kt) {
    const int64_t off = (int64_t)kt * BK;
#pragma unroll
    for (int v = 0; v < EPT; v += VEC) {
      *reinterpret_cast<float4*>(&ra[v]) = *reinterpret_cast<const float4*>(pa + off + v);
      *reinterpret_cast<float4*>(&rb[v]) = *reinterpret_cast<const float4*>(pb + off + v);
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int v = 0; v < EPT; ++v) {
      As[buf][lk + v][lrow] = ra[v];
      Bs[buf][lk + v][lrow] = rb[v];
    }
  };
  auto frag = [&](int buf, int kk, T (&av)[TM], T (&bv)[TM]) {
#pragma unroll
    for (int g = 0; g < TM / 4; ++g)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        av[g * 4 + u] = As[buf][kk][g * (BM / 2) + ty * 4 + u];
        bv[g * 4 + u] = Bs[buf][kk][g * (BM / 2) + tx * 4 + u];
      }
  };

  const int nk = ktot / BK;
  load_regs(0);
  store_smem(0);
  __syncthreads();
  int kt = 0;

  if (FLUSH) {
    // heavy head: exact products, FP64 register accumulation
    double accd[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) accd[a][b] = 0.0;
    const int nh = nk < heavy_steps ? nk : heavy_steps;
    for (; kt < nh; ++kt) {
      const int cur = kt & 1;
      if (kt + 1 < nk) load_regs(kt + 1);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T av[TM], bv[TM];
        frag(cur, kk, av, bv);
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b)
            accd[a][b] = fma((double)av[a], (double)bv[b], accd[a][b]);
      }
      if (kt + 1 < nk) store_smem(cur ^ 1);
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) accd_s[(a * TM + b) * 256 + tid] = accd[a][b];
  }

  T acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
  for (; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) load_regs(kt + 1);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TM];
      frag(cur, kk, av, bv);
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    if (kt + 1 < nk) store_smem(cur ^ 1);
    if (FLUSH) {
      if (((flush_mask[kt >> 5] >> (kt & 31)) & 1u) || kt + 1 == nk) {
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b) {
            accd_s[(a * TM + b) * 256 + tid] += (double)acc[a][b];
            acc[a][b] = T(0);
          }
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int i = i0 + (a / 4) * (BM / 2) + ty * 4 + (a % 4);
#pragma unroll
    for (int b = 0; b < TM; ++b) {
      const int j = j0 + (b / 4) * (BM / 2) + tx * 4 + (b % 4);
      if (i >= ep.n || j >= ep.n || j > i) continue;
      double v = FLUSH ? accd_s[(a * TM + b) * 256 + tid] : (double)acc[a][b];
      v += epilogue_terms(ep, i, j);
      E[(int64_t)i * ldE + j] = (T)v;
    }
  }
}

// Head of the k-space sum in float-float arithmetic (lower-triangle 64 x 64 tiles, 4 x 4
// outputs per thread): each FP64 operand value is split into a float pair a = ah + al,
// and each term
//   a_i a_j = ah*bh (exact: rounded product plus its fma remainder) + ah*bl + al*bh
// (al*bl is below 2^-48 of the product) is added to a float pair (hi, lo) per output
// with an error-free two-sum.  About 11 float operations per term instead of one FP64
// FMA, which runs at 1/64 of the float rate on this GPU.  The epilogue adds the
// real-space, self and dipole terms in FP64 and writes the head matrix as float pairs
// (hi, lo): ~2^-48 of each entry, and the tensor-core tail adds to it in float.
__global__ void __launch_bounds__(256)
k_ek_head_ff(const float* __restrict__ Ah_g, const float* __restrict__ Al_g, int64_t lda,
             int ktot, float2* __restrict__ Eh, int64_t ldE, Epi ep) {
  constexpr int BM = 64, BK = 16, TM = 4, LD = BM + 4;
  __shared__ __align__(16) float Ah[BK][LD], Al[BK][LD], Bh[BK][LD], Bl[BK][LD];
  int I, J;
  tri_tile(blockIdx.x, I, J);
  const int i0 = I * BM, j0 = J * BM;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lrow = tid >> 2, lk = (tid & 3) * 4;
  float sh[TM][TM], sl[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) sh[a][b] = sl[a][b] = 0.f;
  const int64_t oa = (int64_t)(i0 + lrow) * lda + lk, ob = (int64_t)(j0 + lrow) * lda + lk;
  for (int k0 = 0; k0 < ktot; k0 += BK) {
    const float4 xh = __ldg(reinterpret_cast<const float4*>(Ah_g + oa + k0));
    const float4 xl = __ldg(reinterpret_cast<const float4*>(Al_g + oa + k0));
    const float4 yh = __ldg(reinterpret_cast<const float4*>(Ah_g + ob + k0));
    const float4 yl = __ldg(reinterpret_cast<const float4*>(Al_g + ob + k0));
    Ah[lk][lrow] = xh.x; Ah[lk + 1][lrow] = xh.y; Ah[lk + 2][lrow] = xh.z; Ah[lk + 3][lrow] = xh.w;
    Al[lk][lrow] = xl.x; Al[lk + 1][lrow] = xl.y; Al[lk + 2][lrow] = xl.z; Al[lk + 3][lrow] = xl.w;
    Bh[lk][lrow] = yh.x; Bh[lk + 1][lrow] = yh.y; Bh[lk + 2][lrow] = yh.z; Bh[lk + 3][lrow] = yh.w;
    Bl[lk][lrow] = yl.x; Bl[lk + 1][lrow] = yl.y; Bl[lk + 2][lrow] = yl.z; Bl[lk + 3][lrow] = yl.w;
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      float ah[TM], al[TM], bh[TM], bl[TM];
      *reinterpret_cast<float4*>(ah) = *reinterpret_cast<const float4*>(&Ah[kk][ty * 4]);
      *reinterpret_cast<float4*>(al) = *reinterpret_cast<const float4*>(&Al[kk][ty * 4]);
      *reinterpret_cast<float4*>(bh) = *reinterpret_cast<const float4*>(&Bh[kk][tx * 4]);
      *reinterpret_cast<float4*>(bl) = *reinterpret_cast<const float4*>(&Bl[kk][tx * 4]);
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) {
          const float p = ah[a] * bh[b];
          const float pe = fmaf(ah[a], bh[b], -p);
          const float s = sh[a][b] + p;
          const float bb = s - sh[a][b];
          const float e2 = (sh[a][b] - (s - bb)) + (p - bb);
          sl[a][b] = fmaf(al[a], bh[b], fmaf(ah[a], bl[b], sl[a][b] + (e2 + pe)));
          sh[a][b] = s;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int i = i0 + ty * 4 + a;
#pragma unroll
    for (int b = 0; b < TM; ++b) {
      const int j = j0 + tx * 4 + b;
      if (i >= ep.n || j >= ep.n || j > i) continue;
      const double v = (double)sh[a][b] + (double)sl[a][b] + epilogue_terms(ep, i, j);
      const float vh = (float)v;
      Eh[(int64_t)i * ldE + j] = make_float2(vh, (float)(v - (double)vh));
    }
  }
}

// The head operand columns [0, ktot) of every row as float pairs x = hi + lo (exact to
// ~2^-48), split once so the head GEMM loads floats only.
__global__ void k_split_head(const double* __restrict__ A, int64_t lda, int rows, int ktot,
                             float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t total = (int64_t)rows * ktot;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ktot, c = e % ktot;
    const double x = A[r * lda + c];
    const float h = (float)x;
    hi[e] = h;
    lo[e] = (float)(x - (double)h);
  }
}

template <typename T>
__global__ void k_mirror_lower(T* __restrict__ E, int n, int64_t ldE) {
  __shared__ T tile[32][33];
  const int R = blockIdx.y, C = blockIdx.x;
  if (R < C) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int y = ty; y < 32; y += 8) {
    int i = R * 32 + y, j = C * 32 + tx;
    tile[y][tx] = (i < n && j < n) ? E[(int64_t)i * ldE + j] : T(0);
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    // destination (C*32 + y, R*32 + tx) takes source (R*32 + tx, C*32 + y)
    int di = C * 32 + y, dj = R * 32 + tx;
    if (di < n && dj < n && dj > di) E[(int64_t)di * ldE + dj] = tile[tx][y];
  }
}

template <typename T>
__global__ void k_extract_diag(const T* __restrict__ E, int n, int64_t ldE,
                               double* __restrict__ diag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) diag[i] = (double)E[(int64_t)i * ldE + i];
}

template <typename T>
__global__ void k_get_E(const T* __restrict__ E, int n, int64_t ldE,
                        const double* __restrict__ xyz, double c0, double cz, double lz2_6,
                        int slab, const int* __restrict__ rows, int nrows,
                        double* __restrict__ out, int64_t ld) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int r = blockIdx.y; r < nrows; r += gridDim.y) {
    const int i = rows ? rows[r] : r;
    double v = (double)E[(int64_t)i * ldE + j];
    v += c0;
    if (slab) {
      double zi = xyz[3 * i + 2], zj = xyz[3 * j + 2];
      v += cz * (zi * zi + zj * zj + lz2_6);
    }
    out[(int64_t)r * ld + j] = v;
  }
}

}  // namespace

void launch_fixed_point_coords(const double* xyz, int n, int npad, const double L[3],
                               uint32_t* sfix, cudaStream_t s) {
  (k_fixed_point_coords<<<(npad + 127) / 128, 128, 0, s>>>(xyz, n, npad, L[0], L[1], L[2],
                                                          sfix), note_launch());
}

void launch_structure_operand_head(const double* xyz, int npad, int n, const int* hkl,
                                   const double* sqw, int kh, const double L[3], double* Ahead,
                                   cudaStream_t s) {
  dim3 grid((kh + 127) / 128, npad < 1024 ? npad : 1024);
  (k_structure_operand_f64<<<grid, 128, 0, s>>>(xyz, npad, n, hkl, sqw, kh, L[0], L[1], L[2],
                                               Ahead), note_launch());
}

void launch_structure_operand(bool fp64, const double* xyz, const uint32_t* sfix, int npad,
                              int n, const int* hkl, const double* sqw, int mpad,
                              const double L[3], void* A, void* const* planes, int kb0,
                              int kb6, int kb3, int kb8, const int* kexp, const void* turn,
                              int kbeg, int kend, cudaStream_t s) {
  dim3 grid((kend - kbeg + 127) / 128, npad < 1024 ? npad : 1024);
  PlaneOut po{};
  if (fp64) {
    dim3 g64((mpad + 127) / 128, npad < 1024 ? npad : 1024);
    (k_structure_operand_f64<<<g64, 128, 0, s>>>(xyz, npad, n, hkl, sqw, mpad, L[0], L[1],
                                                L[2], (double*)A), note_launch());
  } else if (planes) {
    for (int t = 0; t < 3; ++t) po.p[t] = (uint16_t*)planes[t];
    po.p8 = (uint8_t*)planes[3];
    po.kb8 = kb8;
    po.kexp = kexp;
    po.kb0 = kb0;
    po.kb6 = kb6;
    po.kb3 = kb3;
    (k_structure_operand_f32<true><<<grid, 128, 0, s>>>(sfix, npad, n, hkl, sqw, mpad, kbeg,
                                                        kend, (const float4*)turn, (float*)A,
                                                        po), note_launch());
  } else {
    (k_structure_operand_f32<false><<<grid, 128, 0, s>>>(sfix, npad, n, hkl, sqw, mpad, kbeg,
                                                         kend, (const float4*)turn, (float*)A,
                                                         po), note_launch());
  }
}

int launch_ek_simt(bool fp64, const void* A, int npad, int mpad, const double* xyz,
                   const double* alpha, int n, const Geometry& geo, void* E, int64_t ldE,
                   int heavy_steps, const uint32_t* flush_mask, cudaStream_t s) {
  const Epi ep = make_epi(xyz, alpha, n, geo);
  const int64_t lda = 2 * (int64_t)mpad;
  const int ktot = 2 * mpad;
  if (fp64) {
    constexpr int BM = 64;
    int nt = (n + BM - 1) / BM;
    int tiles = nt * (nt + 1) / 2;
    (k_ek_simt<double, BM, 4, false><<<tiles, 256, 0, s>>>((const double*)A, lda, ktot,
                                                          (double*)E, ldE, ep, 0, flush_mask), note_launch());
  } else {
    constexpr int BM = 128;
    int nt = (n + BM - 1) / BM;
    int tiles = nt * (nt + 1) / 2;
    size_t smem = 64 * 256 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_ek_simt<float, BM, 8, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return CPM_ECUDA;
    (k_ek_simt<float, BM, 8, true><<<tiles, 256, smem, s>>>((const float*)A, lda, ktot,
                                                           (float*)E, ldE, ep, heavy_steps,
                                                           flush_mask), note_launch());
  }
  return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_ECUDA;
}

// FP64-accurate head of the k-space sum (the first ktot columns of the FP64 head operand,
// row stride 2 kh, split into float pairs in hi/lo [npad][ktot]) plus the real-space,
// self and dipole terms, lower triangle, into Ehead as float pairs (hi, lo).
int launch_ek_head_f64(const double* Ahead, int kh, int ktot, int npad, float* hi, float* lo,
                       const double* xyz, const double* alpha, int n, const Geometry& geo,
                       float2* Ehead, int64_t ldE, cudaStream_t s) {
  const Epi ep = make_epi(xyz, alpha, n, geo);
  constexpr int BM = 64;
  const int nt = (n + BM - 1) / BM;
  const int tiles = nt * (nt + 1) / 2;
  (k_split_head<<<2048, 256, 0, s>>>(Ahead, 2 * (int64_t)kh, npad, ktot, hi, lo), note_launch());
  (k_ek_head_ff<<<tiles, 256, 0, s>>>(hi, lo, ktot, ktot, Ehead, ldE, ep), note_launch());
  return cudaGetLastError() == cudaSuccess ? CPM_OK : CPM_ECUDA;
}

void launch_mirror_lower(bool fp64, void* E, int n, int64_t ldE, cudaStream_t s) {
  int nb = (n + 31) / 32;
  dim3 grid(nb, nb), block(32, 8);
  if (fp64)
    (k_mirror_lower<double><<<grid, block, 0, s>>>((double*)E, n, ldE), note_launch());
  else
    (k_mirror_lower<float><<<grid, block, 0, s>>>((float*)E, n, ldE), note_launch());
}

void launch_extract_diag(bool fp64, const void* E, int n, int64_t ldE, double* diag,
                         cudaStream_t s) {
  if (fp64)
    (k_extract_diag<double><<<(n + 255) / 256, 256, 0, s>>>((const double*)E, n, ldE, diag), note_launch());
  else
    (k_extract_diag<float><<<(n + 255) / 256, 256, 0, s>>>((const float*)E, n, ldE, diag), note_launch());
}

// Rows of E (all n when rows is null, else rows[0..nrows)) into out[nrows][ld].
void launch_get_E(bool fp64, const void* E, int n, int64_t ldE, const double* xyz,
                  const Geometry& geo, int paper_form, const int* rows, int nrows, double* out,
                  int64_t ld, cudaStream_t s) {
  // Paper form (Eq. 22 + Eq. 39) = stored form - pi/(V g^2) - (2 pi/V)(z_i^2 + z_j^2 + Lz^2/6)
  double c0 = paper_form ? -kPi / (geo.vol * geo.g * geo.g) : 0.0;
  double cz = -2.0 * kPi / geo.vol;
  int slab = paper_form && geo.slab;
  dim3 grid((n + 255) / 256, nrows < 65535 ? nrows : 65535);
  if (fp64)
    (k_get_E<double><<<grid, 256, 0, s>>>((const double*)E, n, ldE, xyz, c0, cz,
                                         geo.L[2] * geo.L[2] / 6.0, slab, rows, nrows, out,
                                         ld), note_launch());
  else
    (k_get_E<float><<<grid, 256, 0, s>>>((const float*)E, n, ldE, xyz, c0, cz,
                                        geo.L[2] * geo.L[2] / 6.0, slab, rows, nrows, out,
                                        ld), note_launch());
}

}  // namespace cpm
