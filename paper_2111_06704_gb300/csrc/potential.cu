// Electrolyte potential on the electrode atoms (Eq. 25):
//   b^sol_i = sum_I q_I e_iI(alpha_i),   b_i = chi_i - k_e b^sol_i,
// with e_iI the point-Gaussian Ewald coefficient (alpha_iI = alpha_i) in the
// neutral-equivalent form (slab: dipole term (4 pi/V) z_i z_I only).
//
// Reciprocal part: ion structure factors v = [sqrt(W) Re S | sqrt(W) Im S],
// S_K = sum_I q_I exp(i K.r_I), then b^sol_k = A v with the electrode operand A of the
// E build (cos(K.(r_i - r_I)) split by angle addition).  Real part: direct pair sums
// over the images within the cutoff.
#include <math.h>

#include <algorithm>

#include "cpm_internal.cuh"

namespace cpm {

namespace {

constexpr int kSfThreads = 128;
constexpr int kIonChunk = 256;

// Fractional ion coordinates in 2^-32 fixed point, once per ion and frame: the phases of
// every k-vector and the real-space screening use them.
__global__ void k_ion_fixed(const double* __restrict__ ion_xyz, int64_t count, double lx,
                            double ly, double lz, uint32_t* __restrict__ sion) {
  const double L[3] = {lx, ly, lz};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = ion_xyz[e] / L[e % 3];
    s -= floor(s);
    sion[e] = (uint32_t)((unsigned long long)llrint(s * 4294967296.0) & 0xffffffffull);
  }
}

// exp(2 pi i j / 4096), j < 4096, as float pairs (cos hi, cos lo, sin hi, sin lo).
__global__ void k_turn_table(float4* __restrict__ T) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 4096) return;
  double s, c;
  sincospi(j / 2048.0, &s, &c);
  const float ch = (float)c, sh = (float)s;
  T[j] = make_float4(ch, (float)(c - ch), sh, (float)(s - sh));
}

// a * b for float pairs, to ~2^-44 relative (the lo * lo term dropped).
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& ph,
                                       float& pl) {
  ph = ah * bh;
  pl = fmaf(ah, bh, -ph) + fmaf(ah, bl, al * bh);
}

// a + b for float pairs (two-sum of the high parts).
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& sh,
                                       float& sl) {
  const float s = ah + bh;
  const float bb = s - ah;
  sl = ((ah - (s - bb)) + (bh - bb)) + (al + bl);
  sh = s;
}

// exp(2 pi i ph 2^-32) as float pairs, to ~1e-13: the top 12 bits of the phase index the
// exact table, the low 20 bits give an angle t < 2 pi 2^-12 whose sine and cosine follow
// from their Taylor series (t - t^3/6, 1 - t^2/2 + t^4/24; the next terms are below
// 1e-16), and the two rotations are multiplied in float pairs.
__device__ __forceinline__ void phasor_ff(uint32_t ph, const float4* __restrict__ T, float& ch,
                                          float& cl, float& sh, float& sl) {
  const float4 t4 = __ldg(T + (ph >> 20));
  const float low = (float)(ph & 0xFFFFFu);
  constexpr float kCh = 1.462918119976564e-09f;   // 2 pi 2^-32, high part
  constexpr float kCl = -4.070940267922164e-17f;  // and the rest
  const float th = low * kCh;
  const float tl = fmaf(low, kCh, -th) + low * kCl;
  const float p = th * th;
  const float pe = fmaf(th, th, -p) + 2.0f * th * tl;
  // cos t = 1 - t^2/2 + t^4/24
  const float half = 0.5f * p;
  const float c0 = 1.0f - half;
  const float c0l = ((1.0f - c0) - half) - 0.5f * pe + p * p * (1.0f / 24.0f);
  // sin t = t - t^3/6
  const float t3 = th * p * (1.0f / 6.0f);
  const float s0 = th - t3;
  const float s0l = ((th - s0) - t3) + tl;
  // (Tc + i Ts)(c0 + i s0)
  float ah, al, bh, bl;
  ff_mul(t4.x, t4.y, c0, c0l, ah, al);
  ff_mul(t4.z, t4.w, s0, s0l, bh, bl);
  ff_add(ah, al, -bh, -bl, ch, cl);
  ff_mul(t4.z, t4.w, c0, c0l, ah, al);
  ff_mul(t4.x, t4.y, s0, s0l, bh, bl);
  ff_add(ah, al, bh, bl, sh, sl);
}

// (h, l) += x by an error-free two-sum of the high part.
__device__ __forceinline__ void pair_add1(float& h, float& l, float x) {
  const float s = h + x;
  const float bb = s - h;
  l += (h - (s - bb)) + (x - bb);
  h = s;
}

constexpr int kSfBlock = 8;  // ions a float block sum of the tail k-vectors holds

// sin and cos of 2 pi ph 2^-32 from a 64-entry table of exp(2 pi i j / 64) (float cos and
// sin, in shared memory: 512 bytes, few bank conflicts for random entries) and the
// remaining angle t = 2 pi (ph mod 2^26) 2^-32 < 0.099 rad by angle addition, with
// cos t = 1 - t^2/2 + t^4/24 and sin t = t - t^3/6 + t^5/120 (the next terms, t^6/720 and
// t^7/5040, lie below float rounding).  At most 1.5 float ulp of 1 (0.5 on average).
__device__ __forceinline__ void sincos_t64(uint32_t ph, const float2* T, float* s, float* c) {
  const float2 e = T[ph >> 26];
  const float t = (float)(ph & 0x3FFFFFFu) * 1.462918119976564e-09f;  // 2 pi 2^-32
  const float t2 = t * t;
  const float ct = fmaf(t2, fmaf(t2, 1.0f / 24.0f, -0.5f), 1.0f);
  const float st = t * fmaf(t2, fmaf(t2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
  *c = fmaf(e.x, ct, -(e.y * st));
  *s = fmaf(e.y, ct, e.x * st);
}

// v[f][c(k)] = sqrt(W_k) sum_I q_I cos(theta_Ik), v[f][c(k) + 64] = sqrt(W_k) sum_I q_I sin,
// in the column layout of the electrode operand, c(k) = 128 (k / 64) + k % 64, from the
// exact fixed-point phases.  Sums over the ions run in error-free float pairs (S_K is a
// sum of O(n_ion) unit phasors whose float partial sums would lose bits; FP64 runs at
// 1/64 of the float rate here); the tail's terms go in float blocks of kSfBlock ions, each
// block's sum into the pair (a few ulp of a block, not of the whole sum).  The tail
// k-vectors take float sin/cos from the phasor table (sincos_table, about one ulp); the
// head (k < kh, the heaviest weights) takes float-pair phasors and goes out in FP64 to
// vhead for the FP64 head contraction.
__global__ void __launch_bounds__(kSfThreads, 8)
k_ion_sf_f32(const uint32_t* __restrict__ sion, const double* __restrict__ ion_q, int n_ion,
             const int* __restrict__ hkl, const double* __restrict__ sqw, int mpad, int kh,
             const float4* __restrict__ turn, float* __restrict__ vout,
             double* __restrict__ vhead) {
  __shared__ uint32_t sf[kIonChunk][3];
  __shared__ float sqh[kIonChunk], sql[kIonChunk];
  __shared__ float2 t64[64];  // exp(2 pi i j / 64): entries 64 j of the 4,096-entry table
  const int f = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t* fx = sion + (size_t)f * n_ion * 3;
  const double* q = ion_q + (size_t)f * n_ion;
  for (int j = threadIdx.x; j < 64; j += blockDim.x) {
    const float4 e = __ldg(turn + 64 * j);
    t64[j] = make_float2(e.x, e.z);
  }
  uint32_t h = 0, kk = 0, l = 0;
  if (k < mpad) {
    h = (uint32_t)hkl[3 * k];
    kk = (uint32_t)hkl[3 * k + 1];
    l = (uint32_t)hkl[3 * k + 2];
  }
  const bool head = k < kh;  // whole blocks take one branch unless they straddle kh
  float reh = 0.f, rel = 0.f, imh = 0.f, iml = 0.f;
  float rlo = 0.f, ilo = 0.f;  // tail: the charges' low parts times the phasors
  for (int base = 0; base < n_ion; base += kIonChunk) {
    const int cnt = min(kIonChunk, n_ion - base);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      sf[t][0] = fx[3 * (base + t)];
      sf[t][1] = fx[3 * (base + t) + 1];
      sf[t][2] = fx[3 * (base + t) + 2];
      const double qv = q[base + t];
      sqh[t] = (float)qv;
      sql[t] = (float)(qv - (double)sqh[t]);
    }
    __syncthreads();
    if (k >= mpad) continue;
    if (head) {
      for (int t = 0; t < cnt; ++t) {
        const uint32_t ph = h * sf[t][0] + kk * sf[t][1] + l * sf[t][2];
        float ch, cl, sh, sl, ph_, pl_;
        phasor_ff(ph, turn, ch, cl, sh, sl);
        ff_mul(sqh[t], sql[t], ch, cl, ph_, pl_);
        ff_add(reh, rel, ph_, pl_, reh, rel);
        ff_mul(sqh[t], sql[t], sh, sl, ph_, pl_);
        ff_add(imh, iml, ph_, pl_, imh, iml);
      }
    } else {
      // blocks of kSfBlock ions summed in float, then added to the pairs by a two-sum;
      // the charges' low parts (zero for charges that are floats) summed in float apart
      int t = 0;
      for (; t + kSfBlock <= cnt; t += kSfBlock) {
        float br = 0.f, bi = 0.f;
#pragma unroll
        for (int u = 0; u < kSfBlock; ++u) {
          const uint32_t ph = h * sf[t + u][0] + kk * sf[t + u][1] + l * sf[t + u][2];
          float sn, cs;
          sincos_t64(ph, t64, &sn, &cs);
          br = fmaf(sqh[t + u], cs, br);
          bi = fmaf(sqh[t + u], sn, bi);
          rlo = fmaf(sql[t + u], cs, rlo);
          ilo = fmaf(sql[t + u], sn, ilo);
        }
        pair_add1(reh, rel, br);
        pair_add1(imh, iml, bi);
      }
      for (; t < cnt; ++t) {
        const uint32_t ph = h * sf[t][0] + kk * sf[t][1] + l * sf[t][2];
        float sn, cs;
        sincos_t64(ph, t64, &sn, &cs);
        pair_fma(reh, rel, sqh[t], sql[t], cs);
        pair_fma(imh, iml, sqh[t], sql[t], sn);
      }
    }
  }
  if (k >= mpad) return;
  const double re = (double)reh + (double)rel + (double)rlo,
               im = (double)imh + (double)iml + (double)ilo;
  const double w = sqw[k];
  const size_t kcol = 128 * (size_t)(k >> 6) + (k & 63);  // operand column layout
  float* v = vout + (size_t)f * 2 * mpad;
  if (head) {  // FP64 values for the FP64 head contraction; zero float columns
    double* vh = vhead + (size_t)f * 2 * kh;
    vh[kcol] = w * re;
    vh[kcol + 64] = w * im;
    v[kcol] = 0.f;
    v[kcol + 64] = 0.f;
  } else {
    v[kcol] = (float)(w * re);
    v[kcol + 64] = (float)(w * im);
  }
}

// FP64 storage (the plain baseline build): the same sums with FP64 phases, sincospi and
// FP64 accumulation.
__global__ void __launch_bounds__(kSfThreads)
k_ion_sf_f64(const double* __restrict__ ion_xyz, const double* __restrict__ ion_q, int n_ion,
             const int* __restrict__ hkl, const double* __restrict__ sqw, int mpad, double lx,
             double ly, double lz, double* __restrict__ vout) {
  __shared__ double sd[kIonChunk][3];
  __shared__ double sq[kIonChunk];
  const int f = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const double* xyz = ion_xyz + (size_t)f * n_ion * 3;
  const double* q = ion_q + (size_t)f * n_ion;
  int h = 0, kk = 0, l = 0;
  if (k < mpad) {
    h = hkl[3 * k];
    kk = hkl[3 * k + 1];
    l = hkl[3 * k + 2];
  }
  double re = 0.0, im = 0.0;
  for (int base = 0; base < n_ion; base += kIonChunk) {
    const int cnt = min(kIonChunk, n_ion - base);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const double L[3] = {lx, ly, lz};
      for (int d = 0; d < 3; ++d) {
        double s = xyz[3 * (base + t) + d] / L[d];
        sd[t][d] = s - floor(s);
      }
      sq[t] = q[base + t];
    }
    __syncthreads();
    if (k >= mpad) continue;
    for (int t = 0; t < cnt; ++t) {
      double fr = h * sd[t][0] + kk * sd[t][1] + l * sd[t][2];
      fr -= rint(fr);
      double s, c;
      sincospi(2.0 * fr, &s, &c);
      re += sq[t] * c;
      im += sq[t] * s;
    }
  }
  if (k >= mpad) return;
  const double w = sqw[k];
  const size_t kcol = 128 * (size_t)(k >> 6) + (k & 63);
  double* v = vout + (size_t)f * 2 * mpad;
  v[kcol] = w * re;
  v[kcol + 64] = w * im;
}

// b^sol_k[f][i] = sum_c A[i][c] v[f][c]: one warp per electrode row and NF frames per
// grid row (the A row is read once per NF frames).  Float storage: 4-term float partials
// summed in error-free float pairs; FP64 storage: FP64 throughout.
template <typename T, int NF>
__global__ void __launch_bounds__(256)
k_bsol_kspace(const T* __restrict__ A, int n, int64_t lda, const T* __restrict__ v,
              int frames, double* __restrict__ bsol, int accumulate) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int f0 = blockIdx.y * NF;
  if (warp >= n) return;
  const T* a = A + (int64_t)warp * lda;
  constexpr int VEC = 16 / sizeof(T);
  T hi[NF], lo[NF];
#pragma unroll
  for (int r = 0; r < NF; ++r) hi[r] = lo[r] = T(0);
  for (int64_t c = lane * VEC; c < lda; c += 32 * VEC) {
    T av[VEC];
    *reinterpret_cast<float4*>(av) = __ldg(reinterpret_cast<const float4*>(a + c));
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      if (f0 + r >= frames) break;
      T vv[VEC];
      *reinterpret_cast<float4*>(vv) =
          __ldg(reinterpret_cast<const float4*>(v + (int64_t)(f0 + r) * lda + c));
      T s = T(0);
#pragma unroll
      for (int u = 0; u < VEC; ++u) s = fma(av[u], vv[u], s);
      if constexpr (sizeof(T) == 4) {
        const float t = hi[r] + s;
        const float bb = t - hi[r];
        lo[r] += (hi[r] - (t - bb)) + (s - bb);
        hi[r] = t;
      } else {
        hi[r] += s;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NF; ++r) {
    double x = (double)hi[r] + (double)lo[r];
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0 && f0 + r < frames) {
      double* dst = bsol + (int64_t)(f0 + r) * n + warp;
      *dst = accumulate ? *dst + x : x;
    }
  }
}

// Streamed builds keep no A: b^sol_k[f][i] = sum_{k >= kh} sqrt(W_k) [cos(K.r_i) v_c +
// sin(K.r_i) v_s] with the electrode phases formed on the fly (fixed point, sincos_table);
// the terms of kDirectBlock consecutive k-vectors are summed in float, and each block's
// sum goes into an error-free float pair (a two-sum), so the rounding of the plain sums
// grows with the block, not with the ~10^5 k-vectors.  One thread per electrode atom and up to
// kDirectFrames frames per block: each phasor is formed once and used for every frame of
// the block; the k-vectors of a chunk and their structure factors are staged in shared
// memory.  Frames go in pairs through paired float instructions (two IEEE results an
// instruction, a - b as fma(b, -1, a)): the values are those of one frame at a time.
constexpr int kDirectChunk = 128;
constexpr int kDirectFrames = 16;
constexpr int kDirectBlock = 8;  // divides every chunk: head and table ends are multiples of 16

__global__ void __launch_bounds__(128, 4)
k_bsol_kspace_direct(const uint32_t* __restrict__ sfix, int n, const int* __restrict__ hkl,
                     const double* __restrict__ sqw, int mpad, int kh,
                     const float4* __restrict__ turn, const float* __restrict__ v, int frames,
                     double* __restrict__ bsol, int nsplit, int64_t split_stride) {
  __shared__ uint32_t sh[kDirectChunk][3];
  // sqrt(W) (v_cos, v_sin) of frames 2 p and 2 p + 1: (c_2p, c_2p+1, s_2p, s_2p+1)
  __shared__ float4 sv[kDirectChunk][kDirectFrames / 2];
  const int f0 = blockIdx.y * kDirectFrames;
  const int nf = min(kDirectFrames, frames - f0);
  // block = atom block + nblk x share: share sp takes chunks [c0, c1) of the k range
  const int nblk = gridDim.x / nsplit, sp = blockIdx.x / nblk;
  const int i = (blockIdx.x - sp * nblk) * blockDim.x + threadIdx.x;
  const int nch = (mpad - kh + kDirectChunk - 1) / kDirectChunk;
  const int kbeg = kh + (int)((int64_t)sp * nch / nsplit) * kDirectChunk;
  const int kend = min(mpad, kh + (int)((int64_t)(sp + 1) * nch / nsplit) * kDirectChunk);
  double* out = bsol + sp * split_stride;
  uint32_t u0 = 0, u1 = 0, u2 = 0;
  if (i < n) {
    u0 = sfix[3 * i];
    u1 = sfix[3 * i + 1];
    u2 = sfix[3 * i + 2];
  }
  float2 hi[kDirectFrames / 2], lo[kDirectFrames / 2];
#pragma unroll
  for (int f = 0; f < kDirectFrames / 2; ++f) hi[f] = lo[f] = make_float2(0.f, 0.f);
  const float2 m1 = make_float2(-1.f, -1.f);
  for (int k0 = kbeg; k0 < kend; k0 += kDirectChunk) {
    const int cnt = min(kDirectChunk, kend - k0);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int k = k0 + t;
      sh[t][0] = (uint32_t)hkl[3 * k];
      sh[t][1] = (uint32_t)hkl[3 * k + 1];
      sh[t][2] = (uint32_t)hkl[3 * k + 2];
    }
    for (int e = threadIdx.x; e < cnt * (kDirectFrames / 2); e += blockDim.x) {
      const int t = e / (kDirectFrames / 2), fp = e % (kDirectFrames / 2);
      const int k = k0 + t;
      const size_t kcol = 128 * (size_t)(k >> 6) + (k & 63);
      const float w = (float)sqw[k];
      float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
      if (2 * fp < nf) {
        const float* vf = v + (size_t)(f0 + 2 * fp) * 2 * mpad;
        val.x = w * vf[kcol];
        val.z = w * vf[kcol + 64];
      }
      if (2 * fp + 1 < nf) {
        const float* vf = v + (size_t)(f0 + 2 * fp + 1) * 2 * mpad;
        val.y = w * vf[kcol];
        val.w = w * vf[kcol + 64];
      }
      sv[t][fp] = val;
    }
    __syncthreads();
    if (i >= n) continue;
    for (int tb = 0; tb < cnt; tb += kDirectBlock) {
      float2 blk[kDirectFrames / 2];
#pragma unroll
      for (int f = 0; f < kDirectFrames / 2; ++f) blk[f] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int tt = 0; tt < kDirectBlock; ++tt) {
        const int t = tb + tt;
        float sn, cs;
        sincos_table(sh[t][0] * u0 + sh[t][1] * u1 + sh[t][2] * u2, turn, &sn, &cs);
        const float2 sn2 = make_float2(sn, sn), cs2 = make_float2(cs, cs);
#pragma unroll
        for (int f = 0; f < kDirectFrames / 2; ++f) {
          const float4 vv = sv[t][f];
          blk[f] = __ffma2_rn(sn2, make_float2(vv.z, vv.w),
                              __ffma2_rn(cs2, make_float2(vv.x, vv.y), blk[f]));
        }
      }
#pragma unroll
      for (int f = 0; f < kDirectFrames / 2; ++f) {
        const float2 term = blk[f];
        const float2 s2 = __fadd2_rn(hi[f], term);
        const float2 bb = __ffma2_rn(hi[f], m1, s2);                          // s2 - hi
        const float2 a = __ffma2_rn(__ffma2_rn(bb, m1, s2), m1, hi[f]);       // hi - (s2 - bb)
        lo[f] = __fadd2_rn(lo[f], __fadd2_rn(a, __ffma2_rn(bb, m1, term)));   // + (term - bb)
        hi[f] = s2;
      }
    }
  }
  if (i < n)
#pragma unroll
    for (int f = 0; f < kDirectFrames; ++f) {
      const float h = (f & 1) ? hi[f >> 1].y : hi[f >> 1].x;
      const float l = (f & 1) ? lo[f >> 1].y : lo[f >> 1].x;
      if (f < nf) out[(size_t)(f0 + f) * n + i] = (double)h + (double)l;
    }
}

// FP64 real-space sum of one electrode-ion pair over every image within r_c:
// sum q_I [erfc(g r) - erfc(alpha_i r)] / r.
// When every box edge exceeds 2 r_c only the nearest image can be in range.
__device__ __forceinline__ double pair_images(const double* ri, double ai, const double* ion,
                                              const double* L, const double* invL,
                                              const bool* single, double rc, double rc2,
                                              double g) {
  double d[3] = {ri[0] - ion[0], ri[1] - ion[1], ri[2] - ion[2]};
  if (single[0] && single[1] && single[2]) {
    for (int u = 0; u < 3; ++u) d[u] -= L[u] * rint(d[u] * invL[u]);
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 >= rc2 || r2 == 0.0) return 0.0;
    const double r = sqrt(r2);
    double e = erfc(g * r);
    if (ai * r < 6.0) e -= erfc(ai * r);
    return ion[3] * e / r;
  }
  int lo[3], hi[3];
  for (int u = 0; u < 3; ++u) {
    if (single[u]) {  // box edge above 2 rc: only the minimum image can be in range
      d[u] -= L[u] * rint(d[u] * invL[u]);
      lo[u] = hi[u] = 0;
    } else {
      lo[u] = (int)ceil((-rc - d[u]) * invL[u]);
      hi[u] = (int)floor((rc - d[u]) * invL[u]);
    }
  }
  double acc = 0.0;
  for (int a = lo[0]; a <= hi[0]; ++a) {
    const double x = d[0] + a * L[0];
    for (int b = lo[1]; b <= hi[1]; ++b) {
      const double y = d[1] + b * L[1];
      const double xy = x * x + y * y;
      if (xy >= rc2) continue;
      for (int c = lo[2]; c <= hi[2]; ++c) {
        const double z = d[2] + c * L[2];
        const double r2 = xy + z * z;
        if (r2 >= rc2 || r2 == 0.0) continue;
        const double r = sqrt(r2);
        double e = erfc(g * r);
        // erfc(6) < 3e-17: beyond alpha r = 6 the Gaussian term is below double rounding
        // of the erfc(g r) term
        if (ai * r < 6.0) e -= erfc(ai * r);
        acc += ion[3] * e / r;
      }
    }
  }
  return acc;
}

// Real-space electrode-ion sums, slab dipole term, and b = chi - k_e b^sol.
// Four warps, 32 electrode atoms each (one a lane); ions staged through shared memory in
// chunks.  Each lane screens its atom against every ion and every image of it that can
// lie within r_c: the nearest image from the exact fixed-point coordinate difference,
// plus the host's list of whole-box shifts (just the zero shift when every box edge
// exceeds 2 r_c), in float (off by < 1e-3 A^2 in r^2, against a band of 0.01 A^2).  The
// images that pass go to one of two per-warp queues that outlive the chunks and are
// evaluated 32 at a time, all lanes busy, each atom then adding its queued values in
// queue order:
//   near images: FP64, from the FP64 coordinates kept in the queue, the image fixed by
//     the fixed-point nearest one and the shift (so the screen and the sum agree on it);
//   far images (r^2 >= r_split^2 where erfc(g r) / r <= 1e-4 1/A, r^2 below r_c^2 by more
//     than the float error, alpha r >= 6 so that the Gaussian term has vanished): float,
//     from the screen's r^2 (~1e-7 relative; the term to ~1e-6 of itself, <= 1e-10 1/A),
//     summed in float apart and added at the end.
// No warp runs both arithmetic paths in one pass.  A box so small that more than
// kMaxShifts shifts would be needed takes every image of a screened pair in FP64 instead.
// The float constants of the screen come from the host: FP64 runs at 1/64 of the float
// rate here, and a constant formed from the FP64 parameters would otherwise be re-formed
// inside the loop.
constexpr int kRealWarps = 4;

constexpr int kMaxShifts = 64;

struct RealScreen {
  float fs[3];    // L / 2^32: fixed-point units of each coordinate, A
  float screen2;  // r_c^2 + 0.01
  float cut2;     // r_c^2 (1 - 1e-5): far pairs lie below
  float far2;     // r_split^2 (r_c^2 when no pair is far)
  float g;        // Ewald splitting parameter, 1/A
  int all_single; // every box edge above 2 r_c
  int nshift;     // whole-box shifts screened (0: every image of a pair in FP64)
  float shift[kMaxShifts][3];       // k L, A
  signed char kshift[kMaxShifts][3];  // k
};

RealScreen real_screen(const Geometry& geo, double rsplit2) {
  RealScreen rs;
  for (int u = 0; u < 3; ++u) rs.fs[u] = (float)(geo.L[u] * 0x1p-32);
  const double rc2 = geo.rc * geo.rc;
  rs.screen2 = (float)rc2 + 0.01f;
  rs.cut2 = (float)(rc2 * (1.0 - 1e-5));
  rs.far2 = (float)rsplit2;
  rs.g = (float)geo.g;
  rs.all_single = 2.0 * geo.rc < geo.L[0] && 2.0 * geo.rc < geo.L[1] && 2.0 * geo.rc < geo.L[2];
  // shifts k with |k| <= floor((r_c + L / 2) / L) per direction (only k = 0 where
  // L > 2 r_c): every image within r_c of an atom, given the nearest one
  int m[3], total = 1;
  for (int u = 0; u < 3; ++u) {
    m[u] = 2.0 * geo.rc < geo.L[u] ? 0 : (int)floor((geo.rc + 0.5 * geo.L[u]) / geo.L[u]);
    total *= 2 * m[u] + 1;
  }
  rs.nshift = total <= kMaxShifts ? total : 0;
  int k = 0;
  for (int a = -m[0]; rs.nshift && a <= m[0]; ++a)
    for (int b = -m[1]; b <= m[1]; ++b)
      for (int c = -m[2]; c <= m[2]; ++c, ++k) {
        const int ks[3] = {a, b, c};
        for (int u = 0; u < 3; ++u) {
          rs.shift[k][u] = (float)(ks[u] * geo.L[u]);
          rs.kshift[k][u] = (signed char)ks[u];
        }
      }
  return rs;
}

// Screen modes: every box edge above 2 r_c (the nearest image only, near and far queues),
// a list of whole-box shifts (each shifted image screened, near and far queues), or every
// image of a screened pair in FP64 (boxes needing more than kMaxShifts shifts).
enum RealMode { kSingleImage = 0, kShiftList = 1, kAllImages = 2 };

template <int kMode>
__global__ void __launch_bounds__(kRealWarps * 32, 6)
k_bsol_real(const double* __restrict__ xyz, const double* __restrict__ alpha,
            const uint32_t* __restrict__ sfix, int n, const double* __restrict__ ion_xyz,
            const double* __restrict__ ion_q, const uint32_t* __restrict__ sion, int n_ion,
            double lx, double ly, double lz, double g, double rc, const RealScreen rs,
            double dip, const double* __restrict__ chi, const double* __restrict__ bsol_k,
            double* __restrict__ b_out, double* __restrict__ qsol) {
  __shared__ double sx[kIonChunk][4];
  __shared__ uint4 su[kIonChunk];  // fixed-point x, y, z (and a pad: one 16-byte load)
  __shared__ double sa[kRealWarps * 32][4];   // the block's atoms: x, y, z, alpha
  __shared__ double nq[kRealWarps][64][4];    // near queue: ion x, y, z, q,
  constexpr int kShiftWarps = kMode == kShiftList ? kRealWarps : 1;
  __shared__ int32_t ndl[kShiftWarps][64][3];  //   the fixed-point difference, the shift
  __shared__ uint8_t nsh[kShiftWarps][64];
  __shared__ float2 fq[kRealWarps][64];       // far queue: r^2, q
  __shared__ uint8_t nlane[kRealWarps][64], flane[kRealWarps][64];
  __shared__ double qval[kRealWarps][32];
  __shared__ float fval[kRealWarps][32];
  const int f = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double* ix = ion_xyz + (size_t)f * n_ion * 3;
  const double* iq = ion_q + (size_t)f * n_ion;
  const uint32_t* iu = sion + (size_t)f * n_ion * 3;
  uint32_t ui[3] = {0, 0, 0};
  float af2 = 0.f;  // alpha^2 of the lane's atom
  if (i < n) {
    ui[0] = sfix[3 * i];
    ui[1] = sfix[3 * i + 1];
    ui[2] = sfix[3 * i + 2];
    sa[threadIdx.x][0] = xyz[3 * i];
    sa[threadIdx.x][1] = xyz[3 * i + 1];
    sa[threadIdx.x][2] = xyz[3 * i + 2];
    sa[threadIdx.x][3] = alpha[i];
    af2 = (float)(alpha[i] * alpha[i]);
  }
  const double L[3] = {lx, ly, lz};
  const double rc2 = rc * rc;
  const double invL[3] = {1.0 / lx, 1.0 / ly, 1.0 / lz};
  const bool single[3] = {2.0 * rc < lx, 2.0 * rc < ly, 2.0 * rc < lz};
  // evaluates the first `cnt` queued images (one a lane); each atom adds its values in
  // queue order
  auto drain = [&](int cnt, double& acc) {
    __syncwarp();
    if (lane < cnt) {
      const int a = nlane[warp][lane];
      const double* at = sa[warp * 32 + a];
      const double* ion = nq[warp][lane];
      if constexpr (kMode == kShiftList) {
        // the image: the fixed-point nearest one (whole boxes k from the FP64 difference)
        // plus the queued shift (with every edge above 2 r_c the shift is zero, and the
        // nearest image by rint below is the same but where it lies beyond r_c)
        const int si = nsh[warp][lane];
        double r2 = 0.0;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const double dd = at[u] - ion[u];
          const double dfx = (double)ndl[warp][lane][u] * (L[u] * 0x1p-32);
          const double k = rint((dd - dfx) * invL[u]) - (double)rs.kshift[si][u];
          const double du = dd - k * L[u];
          r2 += du * du;
        }
        double v = 0.0;
        if (r2 < rc2 && r2 > 0.0) {
          const double r = sqrt(r2);
          double e = erfc(g * r);
          if (at[3] * r < 6.0) e -= erfc(at[3] * r);
          v = ion[3] * e / r;
        }
        qval[warp][lane] = v;
      } else {
        qval[warp][lane] = pair_images(at, at[3], ion, L, invL, single, rc, rc2, g);
      }
    }
    __syncwarp();
    for (int k = 0; k < cnt; ++k)
      if (nlane[warp][k] == lane) acc += qval[warp][k];
    __syncwarp();
  };
  auto drain_far = [&](int cnt, float& acc) {
    __syncwarp();
    if (lane < cnt) {
      const float2 e = fq[warp][lane];
      const float ir = rsqrtf(e.x);  // 1 / r to ~2 ulp
      fval[warp][lane] = e.y * (erfcf(rs.g * (e.x * ir)) * ir);
    }
    __syncwarp();
    for (int k = 0; k < cnt; ++k)
      if (flane[warp][k] == lane) acc += fval[warp][k];
    __syncwarp();
  };
  // sum q_I z_I and sum q_I over the frame: each thread takes the ions it stages
  double acc = 0.0, qz = 0.0, qs = 0.0;
  float accf = 0.f;
  int qn = 0, fn = 0;  // queued near and far pairs of this warp (warp-uniform)
  const unsigned below = (1u << lane) - 1u;
  for (int base = 0; base < n_ion; base += kIonChunk) {
    const int cnt = min(kIonChunk, n_ion - base);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      sx[t][0] = ix[3 * (base + t)];
      sx[t][1] = ix[3 * (base + t) + 1];
      sx[t][2] = ix[3 * (base + t) + 2];
      sx[t][3] = iq[base + t];
      su[t] = make_uint4(iu[3 * (base + t)], iu[3 * (base + t) + 1], iu[3 * (base + t) + 2], 0u);
      qz += sx[t][3] * sx[t][2];
      qs += sx[t][3];
    }
    __syncthreads();
    // one image of ion t (whole-box shift si) at r^2 = m2: classified, queued, and the
    // queues drained when full (no lane's image within the screen: nothing, one vote)
    auto place = [&](int t, int si, float m2, const int32_t (&dl)[3]) {
      const bool inr = i < n && m2 < rs.screen2;
      if (!__any_sync(0xffffffffu, inr)) return;
      bool far = false;
      if constexpr (kMode != kAllImages)
        far = inr && m2 >= rs.far2 && m2 < rs.cut2 && af2 * m2 >= 36.0f;
      const bool near = inr && !far;
      const unsigned mn = __ballot_sync(0xffffffffu, near);
      const unsigned mf = __ballot_sync(0xffffffffu, far);
      if (near) {
        const int at = qn + __popc(mn & below);
        nq[warp][at][0] = sx[t][0];
        nq[warp][at][1] = sx[t][1];
        nq[warp][at][2] = sx[t][2];
        nq[warp][at][3] = sx[t][3];
        if constexpr (kMode == kShiftList) {
          ndl[warp][at][0] = dl[0];
          ndl[warp][at][1] = dl[1];
          ndl[warp][at][2] = dl[2];
          nsh[warp][at] = (uint8_t)si;
        }
        nlane[warp][at] = (uint8_t)lane;
      }
      if (far) {
        const int at = fn + __popc(mf & below);
        fq[warp][at] = make_float2(m2, (float)sx[t][3]);
        flane[warp][at] = (uint8_t)lane;
      }
      qn += __popc(mn);
      fn += __popc(mf);
      if (qn >= 32) {
        drain(32, acc);
        if (lane < qn - 32) {
#pragma unroll
          for (int c = 0; c < 4; ++c) nq[warp][lane][c] = nq[warp][32 + lane][c];
          if constexpr (kMode == kShiftList) {
#pragma unroll
            for (int c = 0; c < 3; ++c) ndl[warp][lane][c] = ndl[warp][32 + lane][c];
            nsh[warp][lane] = nsh[warp][32 + lane];
          }
          nlane[warp][lane] = nlane[warp][32 + lane];
        }
        qn -= 32;
        __syncwarp();
      }
      if (fn >= 32) {
        drain_far(32, accf);
        if (lane < fn - 32) {
          fq[warp][lane] = fq[warp][32 + lane];
          flane[warp][lane] = flane[warp][32 + lane];
        }
        fn -= 32;
        __syncwarp();
      }
    };
    // the nearest image's fixed-point difference (dl) and float components (dn)
    auto nearest = [&](int t, int32_t (&dl)[3], float (&dn)[3]) {
      const uint4 ut = su[t];
      dl[0] = (int32_t)(ui[0] - ut.x);
      dl[1] = (int32_t)(ui[1] - ut.y);
      dl[2] = (int32_t)(ui[2] - ut.z);
#pragma unroll
      for (int u = 0; u < 3; ++u) dn[u] = (float)dl[u] * rs.fs[u];
    };
    if constexpr (kMode == kShiftList) {
      for (int t = 0; t < cnt; ++t) {
        int32_t dl[3] = {0, 0, 0};
        float dn[3] = {0.f, 0.f, 0.f};
        if (i < n) nearest(t, dl, dn);
        for (int si = 0; si < rs.nshift; ++si) {
          float m2 = 0.f;
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const float du = dn[u] + rs.shift[si][u];
            m2 = fmaf(du, du, m2);
          }
          place(t, si, m2, dl);
        }
      }
    } else {
      // two ions a step: their r^2 in paired instructions (each the scalar fma chain's
      // value), one vote over both, then each placed in ion order
      const int32_t dz[3] = {0, 0, 0};
      int t = 0;
      for (; t + 1 < cnt; t += 2) {
        float2 m2 = make_float2(0.f, 0.f);
        if (i < n) {
          int32_t da[3], db[3];
          float fa[3], fb[3];
          nearest(t, da, fa);
          nearest(t + 1, db, fb);
          const float2 d0 = make_float2(fa[0], fb[0]), d1 = make_float2(fa[1], fb[1]),
                       d2 = make_float2(fa[2], fb[2]);
          m2 = __ffma2_rn(d0, d0, __ffma2_rn(d1, d1, __fmul2_rn(d2, d2)));
        }
        const bool any = i < n && fminf(m2.x, m2.y) < rs.screen2;
        if (!__any_sync(0xffffffffu, any)) continue;
        place(t, 0, m2.x, dz);
        place(t + 1, 0, m2.y, dz);
      }
      if (t < cnt) {
        float m2 = 0.f;
        if (i < n) {
          int32_t dl[3];
          float dn[3];
          nearest(t, dl, dn);
          m2 = fmaf(dn[0], dn[0], fmaf(dn[1], dn[1], dn[2] * dn[2]));
        }
        place(t, 0, m2, dz);
      }
    }
  }
  if (qn > 0) drain(qn, acc);
  if (fn > 0) drain_far(fn, accf);
  acc += (double)accf;
  __shared__ double red[2][kRealWarps];
  for (int o = 16; o; o >>= 1) {
    qz += __shfl_xor_sync(0xffffffffu, qz, o);
    qs += __shfl_xor_sync(0xffffffffu, qs, o);
  }
  if (lane == 0) {
    red[0][warp] = qz;
    red[1][warp] = qs;
  }
  __syncthreads();
  qz = red[0][0] + red[0][1] + red[0][2] + red[0][3];
  qs = red[1][0] + red[1][1] + red[1][2] + red[1][3];
  if (i < n) {
    double bs = bsol_k[(size_t)f * n + i] + acc + dip * sa[threadIdx.x][2] * qz;
    b_out[(size_t)f * n + i] = chi[i] - kKe * bs;
  }
  if (i == 0 && qsol) qsol[f] = qs;
}


// ---- forces on the ions: F_I = -q_I d/dr_I sum_i q_i e_iI (Eq. S25 inside the Ewald
// sums of Eq. 22 / 25, the paper's form with Eq. 39) ------------------------------------
//
// Reciprocal part: d/dr_I cos(K.(r_i - r_I)) = sin(K.(r_i - r_I)) K, so with the
// electrode's charge-weighted structure factors (C_K, S_K) = sum_i q_i (cos, sin)(K.r_i),
// grad_I = sum_K W_K [S_K cos(K.r_I) - C_K sin(K.r_I)] K.  v holds sqrt(W) (C, S) in the
// operand's column layout (the ions' structure-factor kernel run over the electrode), so
// the term is sqrt(W_K) (v_s cos - v_c sin).  The head k-vectors (heaviest) in FP64 from
// FP64 phasors; the tail in float from the table phasors (about one ulp) summed in
// error-free float pairs; the integer h, k, l multiply last: K = 2 pi (h/Lx, k/Ly, l/Lz).
constexpr int kForceChunk = 256;

__global__ void __launch_bounds__(128)
k_force_kspace(const uint32_t* __restrict__ sion, int n_ion, const int* __restrict__ hkl,
               const double* __restrict__ sqw, int mpad, int kh,
               const float4* __restrict__ turn, const float* __restrict__ v,
               const double* __restrict__ vhead, double lx, double ly, double lz,
               double* __restrict__ grad) {
  __shared__ int sk[kForceChunk][3];
  __shared__ double sw[kForceChunk][3];  // head: sqrt(W), v_c, v_s in FP64
  __shared__ float swf[kForceChunk][3];  // tail: the same as floats (converted once here)
  const int f = blockIdx.y;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t* u = sion + ((size_t)f * n_ion + (I < n_ion ? I : 0)) * 3;
  const uint32_t u0 = u[0], u1 = u[1], u2 = u[2];
  const float* vf = v + (size_t)f * 2 * mpad;
  const double* vh = vhead + (size_t)f * 2 * (size_t)(kh > 0 ? kh : 1);
  double g64[3] = {0.0, 0.0, 0.0};
  float gh[3] = {0.f, 0.f, 0.f}, gl[3] = {0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < mpad; k0 += kForceChunk) {
    const int cnt = min(kForceChunk, mpad - k0);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int k = k0 + t;
      sk[t][0] = hkl[3 * k];
      sk[t][1] = hkl[3 * k + 1];
      sk[t][2] = hkl[3 * k + 2];
      const size_t kcol = 128 * (size_t)(k >> 6) + (k & 63);
      sw[t][0] = sqw[k];
      if (k < kh) {
        sw[t][1] = vh[kcol];
        sw[t][2] = vh[kcol + 64];
      } else {
        swf[t][0] = (float)sqw[k];
        swf[t][1] = vf[kcol];
        swf[t][2] = vf[kcol + 64];
      }
    }
    __syncthreads();
    if (I >= n_ion) continue;
    for (int t = 0; t < cnt; ++t) {
      const uint32_t ph = (uint32_t)sk[t][0] * u0 + (uint32_t)sk[t][1] * u1 +
                          (uint32_t)sk[t][2] * u2;
      if (k0 + t < kh) {
        double sn, cs;
        sincospi((double)(int32_t)ph * 0x1p-31, &sn, &cs);
        const double term = sw[t][0] * (sw[t][2] * cs - sw[t][1] * sn);
        g64[0] += term * sk[t][0];
        g64[1] += term * sk[t][1];
        g64[2] += term * sk[t][2];
      } else {
        float sn, cs;
        sincos_table(ph, turn, &sn, &cs);
        const float term = swf[t][0] * fmaf(swf[t][2], cs, -swf[t][1] * sn);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float x = term * (float)sk[t][d];  // h, k, l: small integers, exact
          const float s2 = gh[d] + x;
          const float bb = s2 - gh[d];
          gl[d] += (gh[d] - (s2 - bb)) + (x - bb);
          gh[d] = s2;
        }
      }
    }
  }
  if (I >= n_ion) return;
  const double twopi = 2.0 * kPi, L[3] = {lx, ly, lz};
  double* g = grad + ((size_t)f * n_ion + I) * 3;
  for (int d = 0; d < 3; ++d) g[d] = (g64[d] + (double)gh[d] + (double)gl[d]) * twopi / L[d];
}

// d/dr [erfc(g r) / r - erfc(a r) / r] (a = INFINITY: a point charge, no Gaussian term).
__device__ __forceinline__ double radial_derivative(double g, double a, double r) {
  const double two_sqrtpi = 1.1283791670955126;  // 2 / sqrt(pi)
  double num = -two_sqrtpi * g * exp(-(g * r) * (g * r));
  double e = erfc(g * r);
  if (isfinite(a)) {
    num += two_sqrtpi * a * exp(-(a * r) * (a * r));
    e -= erfc(a * r);
  }
  return num / r - e / (r * r);
}

// Real part and slab term, then F_I = -q_I grad_I.  One thread per ion (grid row: frame);
// electrode atoms staged by chunks.  A pair is screened in float from the exact
// fixed-point difference of its nearest image (0.01 A^2 band, as k_bsol_real); the pairs
// that pass sum every image within r_c in FP64: grad -= q_i f'(r) / r (r_i - r_I + R).
// The slab term of Eq. 39: grad_z += (4 pi / V) (sum_i q_i z_i - sum_i q_i z_I).
__global__ void __launch_bounds__(128)
k_force_real(const double* __restrict__ xyz, const double* __restrict__ alpha,
             const uint32_t* __restrict__ sfix, int n, const double* __restrict__ ion_xyz,
             const double* __restrict__ ion_q, const uint32_t* __restrict__ sion, int n_ion,
             const double* __restrict__ q, double lx, double ly, double lz, double g,
             double rc, const RealScreen rs, int slab, const double* __restrict__ grad_k,
             double* __restrict__ out) {
  __shared__ uint32_t su[kForceChunk][3];
  __shared__ double sx[kForceChunk][5];  // x, y, z, alpha, q
  __shared__ double red[2][128];
  const int f = blockIdx.y;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = I < n_ion;
  const size_t e = (size_t)f * n_ion + (live ? I : 0);
  const double ri[3] = {ion_xyz[3 * e], ion_xyz[3 * e + 1], ion_xyz[3 * e + 2]};
  const uint32_t ui[3] = {sion[3 * e], sion[3 * e + 1], sion[3 * e + 2]};
  const double* qf = q + (size_t)f * n;
  const double L[3] = {lx, ly, lz};
  const double invL[3] = {1.0 / lx, 1.0 / ly, 1.0 / lz};
  const double rc2 = rc * rc;
  double gr[3] = {0.0, 0.0, 0.0};
  double qz = 0.0, qs = 0.0;  // this thread's share of sum q_i z_i and sum q_i
  for (int base = 0; base < n; base += kForceChunk) {
    const int cnt = min(kForceChunk, n - base);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int i = base + t;
      su[t][0] = sfix[3 * i];
      su[t][1] = sfix[3 * i + 1];
      su[t][2] = sfix[3 * i + 2];
      sx[t][0] = xyz[3 * i];
      sx[t][1] = xyz[3 * i + 1];
      sx[t][2] = xyz[3 * i + 2];
      sx[t][3] = alpha[i];
      sx[t][4] = qf[i];
      qz += qf[i] * xyz[3 * i + 2];
      qs += qf[i];
    }
    __syncthreads();
    if (!live) continue;
    for (int t = 0; t < cnt; ++t) {
      float m2 = 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float du = (float)(int32_t)(su[t][d] - ui[d]) * rs.fs[d];
        m2 = fmaf(du, du, m2);
      }
      if (m2 >= rs.screen2) continue;
      // every image of the pair within r_c
      double d0[3];
      int lo[3], hi[3];
      for (int d = 0; d < 3; ++d) {
        d0[d] = sx[t][d] - ri[d];
        d0[d] -= L[d] * rint(d0[d] * invL[d]);
        lo[d] = (int)ceil((-rc - d0[d]) * invL[d]);
        hi[d] = (int)floor((rc - d0[d]) * invL[d]);
      }
      for (int a = lo[0]; a <= hi[0]; ++a)
        for (int b = lo[1]; b <= hi[1]; ++b)
          for (int c = lo[2]; c <= hi[2]; ++c) {
            const double dx = d0[0] + a * L[0], dy = d0[1] + b * L[1], dz = d0[2] + c * L[2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= rc2 || r2 == 0.0) continue;
            const double r = sqrt(r2);
            const double w = sx[t][4] * radial_derivative(g, sx[t][3], r) / r;
            gr[0] -= w * dx;
            gr[1] -= w * dy;
            gr[2] -= w * dz;
          }
    }
  }
  // the frame's sum q_i z_i and sum q_i over the block's threads
  red[0][threadIdx.x] = qz;
  red[1][threadIdx.x] = qs;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (!live) return;
  const double* gk = grad_k + e * 3;
  double gz = gr[2] + gk[2];
  if (slab) gz += (4.0 * kPi / (lx * ly * lz)) * (red[0][0] - red[1][0] * ri[2]);
  const double qI = ion_q[e];
  out[3 * e] = -qI * (gr[0] + gk[0]);
  out[3 * e + 1] = -qI * (gr[1] + gk[1]);
  out[3 * e + 2] = -qI * gz;
}

}  // namespace

void launch_ion_fixed(const double* ion_xyz, int frames, int n_ion, const double L[3],
                      uint32_t* sion, cudaStream_t s) {
  const int64_t count = (int64_t)frames * n_ion;
  const int blocks = (int)std::min<int64_t>((3 * count + 255) / 256, 4096);
  (k_ion_fixed<<<blocks, 256, 0, s>>>(ion_xyz, count, L[0], L[1], L[2], sion), note_launch());
}

void launch_turn_table(void* T, cudaStream_t s) {
  (k_turn_table<<<16, 256, 0, s>>>((float4*)T), note_launch());
}

void launch_ion_structure_factor(bool fp64, const double* ion_xyz, const uint32_t* sion,
                                 const double* ion_q, int frames, int n_ion, const int* hkl,
                                 const double* sqw, int mpad, int kh, const double L[3],
                                 const void* turn, void* v, double* vhead, cudaStream_t s) {
  if (fp64) {
    dim3 grid((mpad + kSfThreads - 1) / kSfThreads, frames);
    (k_ion_sf_f64<<<grid, kSfThreads, 0, s>>>(ion_xyz, ion_q, n_ion, hkl, sqw, mpad, L[0], L[1],
                                              L[2], (double*)v), note_launch());
  } else {
    dim3 grid((mpad + kSfThreads - 1) / kSfThreads, frames);
    (k_ion_sf_f32<<<grid, kSfThreads, 0, s>>>(sion, ion_q, n_ion, hkl, sqw, mpad, kh,
                                              (const float4*)turn, (float*)v, vhead),
     note_launch());
  }
}

namespace {

// The k-range shares of the direct sum, summed in share order into b^sol_k.
__global__ void k_sum_splits(const double* __restrict__ part, int nsplit, int64_t stride,
                             int64_t count, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double v = part[e];
    for (int sp = 1; sp < nsplit; ++sp) v += part[sp * stride + e];
    out[e] = v;
  }
}

}  // namespace

// Shares of the k range for the direct sum: the atom blocks of kDirectFrames-frame groups
// (four resident an SM) times the shares fill whole waves of `sms` SMs best (a larger
// count only where it fills 2% more of the last wave).
int bsol_direct_splits(int n, int frames, int mpad, int kh, int sms) {
  const int64_t blocks = (int64_t)((n + 127) / 128) * ((frames + kDirectFrames - 1) / kDirectFrames);
  const int nch = (mpad - kh + kDirectChunk - 1) / kDirectChunk;
  const int64_t cap = 4 * (int64_t)sms;
  int best = 1;
  double best_eff = -1.0;
  for (int sp = 1; sp <= std::min(4, std::max(1, nch)); ++sp) {
    const int64_t units = blocks * sp, waves = (units + cap - 1) / cap;
    const double eff = (double)units / (double)(waves * cap);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
  }
  return best;
}

// b^sol_k = A v: in float storage the head k-vectors (the heaviest weights) are
// contracted in FP64 against an FP64 copy of their operand columns.  Without A (a streamed
// build) the float part is the direct sum over the tail k-vectors.
void launch_bsol_kspace(bool fp64, const void* A, const double* Ahead, int n, int mpad, int kh,
                        const void* v, const double* vhead, int frames, double* bsol,
                        const uint32_t* sfix, const int* hkl, const double* sqw,
                        const void* turn, int nsplit, double* split_part, cudaStream_t s) {
  const int64_t lda = 2 * (int64_t)mpad;
  if (!A && !fp64) {
    const int fgroups = (frames + kDirectFrames - 1) / kDirectFrames;
    const int sp = split_part ? nsplit : 1;
    const int64_t stride = (int64_t)frames * n;  // between shares
    double* dst = sp > 1 ? split_part : bsol;
    for (int g0 = 0; g0 < fgroups; g0 += 65535) {
      const int f0 = g0 * kDirectFrames;
      (k_bsol_kspace_direct<<<dim3(sp * ((n + 127) / 128), std::min(fgroups - g0, 65535)), 128,
                              0, s>>>(sfix, n, hkl, sqw, mpad, kh, (const float4*)turn,
                                      (const float*)v + f0 * lda, frames - f0,
                                      dst + (int64_t)f0 * n, sp, stride),
       note_launch());
    }
    if (sp > 1)
      (k_sum_splits<<<(int)std::min<int64_t>((stride + 255) / 256, 8192), 256, 0, s>>>(
           split_part, sp, stride, stride, bsol),
       note_launch());
    for (int g0 = 0; kh > 0 && g0 < (frames + 3) / 4; g0 += 65535) {
      const int f0 = 4 * g0;
      const dim3 grid((n * 32 + 255) / 256, std::min((frames - f0 + 3) / 4, 65535));
      (k_bsol_kspace<double, 4><<<grid, 256, 0, s>>>(Ahead, n, 2 * (int64_t)kh,
                                                     vhead + f0 * 2 * (int64_t)kh, frames - f0,
                                                     bsol + (int64_t)f0 * n, 1), note_launch());
    }
    return;
  }
  for (int g0 = 0; g0 < (frames + 3) / 4; g0 += 65535) {
    const int f0 = 4 * g0;
    const dim3 grid((n * 32 + 255) / 256, std::min((frames - f0 + 3) / 4, 65535));
    if (fp64) {
      (k_bsol_kspace<double, 4><<<grid, 256, 0, s>>>((const double*)A, n, lda,
                                                     (const double*)v + f0 * lda, frames - f0,
                                                     bsol + (int64_t)f0 * n, 0), note_launch());
    } else {
      (k_bsol_kspace<float, 4><<<grid, 256, 0, s>>>((const float*)A, n, lda,
                                                    (const float*)v + f0 * lda, frames - f0,
                                                    bsol + (int64_t)f0 * n, 0), note_launch());
      if (kh > 0)
        (k_bsol_kspace<double, 4><<<grid, 256, 0, s>>>(Ahead, n, 2 * (int64_t)kh,
                                                       vhead + f0 * 2 * (int64_t)kh, frames - f0,
                                                       bsol + (int64_t)f0 * n, 1), note_launch());
    }
  }
}

void launch_bsol_real_and_finish(const double* xyz, const double* alpha, const uint32_t* sfix,
                                 int n, const double* ion_xyz, const double* ion_q,
                                 const uint32_t* sion, int frames, int n_ion,
                                 const Geometry& geo, const double* chi, const double* bsol_k,
                                 double* b_out, double* qsol, bool far_float, cudaStream_t s) {
  dim3 grid((n + kRealWarps * 32 - 1) / (kRealWarps * 32), frames);
  double dip = geo.slab ? 4.0 * kPi / geo.vol : 0.0;
  // r_split: erfc(g r) / r = 1e-4 / A (bisection); r_c (no far pairs) when the term never
  // gets that small or the FP64 build asks for FP64 throughout
  double lo = 1e-3, hi = geo.rc;
  if (!far_float || erfc(geo.g * hi) / hi > 1e-4) {
    lo = hi;
  } else {
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (erfc(geo.g * mid) / mid > 1e-4) lo = mid;
      else hi = mid;
    }
    lo = hi;
  }
  const RealScreen rs = real_screen(geo, lo * lo);
  auto kernel = rs.all_single ? k_bsol_real<kSingleImage>
                : rs.nshift   ? k_bsol_real<kShiftList>
                              : k_bsol_real<kAllImages>;
  (kernel<<<grid, kRealWarps * 32, 0, s>>>(xyz, alpha, sfix, n, ion_xyz, ion_q, sion, n_ion,
                                          geo.L[0], geo.L[1], geo.L[2], geo.g, geo.rc, rs, dip,
                                          chi, bsol_k, b_out, qsol),
   note_launch());
}

}  // namespace cpm

namespace cpm {

void launch_ion_forces(const double* xyz, const double* alpha, const uint32_t* sfix, int n,
                       const double* ion_xyz, const double* ion_q, const uint32_t* sion,
                       int frames, int n_ion, const double* q, const int* hkl,
                       const double* sqw, int mpad, int kh, const Geometry& geo,
                       const void* turn, const float* v, const double* vhead, double* grad,
                       double* out, cudaStream_t s) {
  const dim3 grid((n_ion + 127) / 128, frames);
  (k_force_kspace<<<grid, 128, 0, s>>>(sion, n_ion, hkl, sqw, mpad, kh, (const float4*)turn, v,
                                       vhead, geo.L[0], geo.L[1], geo.L[2], grad),
   note_launch());
  (k_force_real<<<grid, 128, 0, s>>>(xyz, alpha, sfix, n, ion_xyz, ion_q, sion, n_ion, q,
                                     geo.L[0], geo.L[1], geo.L[2], geo.g, geo.rc,
                                     real_screen(geo, geo.rc * geo.rc), geo.slab, grad, out),
   note_launch());
}

}  // namespace cpm
