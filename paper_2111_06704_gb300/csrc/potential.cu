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

#include "cpm_internal.cuh"

namespace cpm {

namespace {

constexpr int kSfThreads = 128;
constexpr int kIonChunk = 256;

// v[f][c(k)] = sqrt(W_k) sum_I q_I cos(theta_Ik), v[f][c(k) + 64] = sqrt(W_k) sum_I q_I sin,
// in the column layout of the electrode operand, c(k) = 128 (k / 64) + k % 64.
// FP32 path: exact fixed-point phases, sincospif, charge-weighted sums in FP64.
template <bool FP64>
__global__ void __launch_bounds__(kSfThreads)
k_ion_sf(const double* __restrict__ ion_xyz, const double* __restrict__ ion_q, int n_ion,
         const int* __restrict__ hkl, const double* __restrict__ sqw, int mpad, int kh,
         double lx, double ly, double lz, void* __restrict__ vout,
         double* __restrict__ vhead) {
  __shared__ uint32_t sf[kIonChunk][3];
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
        s -= floor(s);
        sd[t][d] = s;
        unsigned long long u = (unsigned long long)llrint(s * 4294967296.0);
        sf[t][d] = (uint32_t)(u & 0xffffffffull);
      }
      sq[t] = q[base + t];
    }
    __syncthreads();
    if (k < mpad) {
      if (FP64 || k < kh) {
        for (int t = 0; t < cnt; ++t) {
          double fr = h * sd[t][0] + kk * sd[t][1] + l * sd[t][2];
          fr -= rint(fr);
          double s, c;
          sincospi(2.0 * fr, &s, &c);
          re += sq[t] * c;
          im += sq[t] * s;
        }
      } else {
        for (int t = 0; t < cnt; ++t) {
          uint32_t ph = (uint32_t)h * sf[t][0] + (uint32_t)kk * sf[t][1] +
                        (uint32_t)l * sf[t][2];
          float fr = (float)(int32_t)ph * 2.3283064365386963e-10f;
          float s, c;
          sincospif(2.0f * fr, &s, &c);
          // float cos/sin, summed over the ions in double: S_K is a sum of O(n_ion)
          // unit phasors whose partial sums would otherwise lose float bits
          re = fma(sq[t], (double)c, re);
          im = fma(sq[t], (double)s, im);
        }
      }
    }
  }
  if (k < mpad) {
    const double w = sqw[k];
    const size_t kcol = 128 * (size_t)(k >> 6) + (k & 63);  // operand column layout
    if (!FP64 && k < kh) {
      // head k-vectors: FP64 values for the FP64 head contraction; zero float columns
      double* vh = vhead + (size_t)f * 2 * kh;
      vh[kcol] = w * re;
      vh[kcol + 64] = w * im;
      float* v = (float*)vout + (size_t)f * 2 * mpad;
      v[kcol] = 0.f;
      v[kcol + 64] = 0.f;
    } else if (FP64) {
      double* v = (double*)vout + (size_t)f * 2 * mpad;
      v[kcol] = w * re;
      v[kcol + 64] = w * im;
    } else {
      float* v = (float*)vout + (size_t)f * 2 * mpad;
      v[kcol] = (float)(w * re);
      v[kcol + 64] = (float)(w * im);
    }
  }
}

// b^sol_k[f][i] = sum_c A[i][c] v[f][c]: one warp per electrode row, up to 4 frames per
// pass (A row read once per pass).  FP32: float products, 8-term float partials
// summed in FP64.
template <typename T, int NF>
__global__ void __launch_bounds__(256)
k_bsol_kspace(const T* __restrict__ A, int n, int64_t lda, const T* __restrict__ v,
              int frames, int f0, double* __restrict__ bsol, int accumulate) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const T* a = A + (int64_t)warp * lda;
  constexpr int VEC = 16 / sizeof(T);
  double acc[NF];
#pragma unroll
  for (int r = 0; r < NF; ++r) acc[r] = 0.0;
  for (int64_t c = lane * VEC; c < lda; c += 32 * VEC) {
    T av[VEC];
    *reinterpret_cast<float4*>(av) = *reinterpret_cast<const float4*>(a + c);
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      if (f0 + r >= frames) break;
      T vv[VEC];
      *reinterpret_cast<float4*>(vv) =
          *reinterpret_cast<const float4*>(v + (int64_t)(f0 + r) * lda + c);
      T s = T(0);
#pragma unroll
      for (int u = 0; u < VEC; ++u) s = fma(av[u], vv[u], s);
      acc[r] += (double)s;
    }
  }
#pragma unroll
  for (int r = 0; r < NF; ++r) {
    double x = acc[r];
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0 && f0 + r < frames) {
      double* dst = bsol + (int64_t)(f0 + r) * n + warp;
      *dst = accumulate ? *dst + x : x;
    }
  }
}

// Real-space electrode-ion sums, slab dipole term, and b = chi - k_e b^sol.
// One thread per electrode atom; ions staged through shared memory.
__global__ void __launch_bounds__(128)
k_bsol_real(const double* __restrict__ xyz, const double* __restrict__ alpha, int n,
            const double* __restrict__ ion_xyz, const double* __restrict__ ion_q, int n_ion,
            double lx, double ly, double lz, double g, double rc, double dip,
            const double* __restrict__ chi, const double* __restrict__ bsol_k,
            double* __restrict__ b_out, double* __restrict__ qsol) {
  __shared__ double sx[kIonChunk][4];
  const int f = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double* ix = ion_xyz + (size_t)f * n_ion * 3;
  const double* iq = ion_q + (size_t)f * n_ion;
  double ri[3] = {0, 0, 0}, ai = INFINITY;
  if (i < n) {
    ri[0] = xyz[3 * i];
    ri[1] = xyz[3 * i + 1];
    ri[2] = xyz[3 * i + 2];
    ai = alpha[i];
  }
  const double L[3] = {lx, ly, lz};
  const double rc2 = rc * rc;
  const double invL[3] = {1.0 / lx, 1.0 / ly, 1.0 / lz};
  const bool single[3] = {2.0 * rc < lx, 2.0 * rc < ly, 2.0 * rc < lz};
  double acc = 0.0, qz = 0.0, qs = 0.0;
  for (int base = 0; base < n_ion; base += kIonChunk) {
    const int cnt = min(kIonChunk, n_ion - base);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      sx[t][0] = ix[3 * (base + t)];
      sx[t][1] = ix[3 * (base + t) + 1];
      sx[t][2] = ix[3 * (base + t) + 2];
      sx[t][3] = iq[base + t];
    }
    __syncthreads();
    for (int t = 0; t < cnt; ++t) {
      const double qI = sx[t][3];
      qz += qI * sx[t][2];
      qs += qI;
      if (i >= n) continue;
      double d[3] = {ri[0] - sx[t][0], ri[1] - sx[t][1], ri[2] - sx[t][2]};
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
      for (int a = lo[0]; a <= hi[0]; ++a) {
        double x = d[0] + a * L[0];
        for (int b = lo[1]; b <= hi[1]; ++b) {
          double y = d[1] + b * L[1];
          double xy = x * x + y * y;
          if (xy >= rc2) continue;
          for (int c = lo[2]; c <= hi[2]; ++c) {
            double z = d[2] + c * L[2];
            double r2 = xy + z * z;
            if (r2 >= rc2 || r2 == 0.0) continue;
            double r = sqrt(r2);
            double e = erfc(g * r);
            // erfc(6) < 3e-17: beyond alpha r = 6 the Gaussian term is below double
            // rounding of the erfc(g r) term
            if (ai * r < 6.0) e -= erfc(ai * r);
            acc += qI * e / r;
          }
        }
      }
    }
  }
  if (i < n) {
    double bs = bsol_k[(size_t)f * n + i] + acc + dip * ri[2] * qz;
    b_out[(size_t)f * n + i] = chi[i] - kKe * bs;
  }
  if (i == 0 && qsol) qsol[f] = qs;
}

}  // namespace

void launch_ion_structure_factor(bool fp64, const double* ion_xyz, const double* ion_q,
                                 int frames, int n_ion, const int* hkl, const double* sqw,
                                 int mpad, int kh, const double L[3], void* v, double* vhead,
                                 cudaStream_t s) {
  dim3 grid((mpad + kSfThreads - 1) / kSfThreads, frames);
  if (fp64)
    (k_ion_sf<true><<<grid, kSfThreads, 0, s>>>(ion_xyz, ion_q, n_ion, hkl, sqw, mpad, 0, L[0],
                                                L[1], L[2], v, vhead), note_launch());
  else
    (k_ion_sf<false><<<grid, kSfThreads, 0, s>>>(ion_xyz, ion_q, n_ion, hkl, sqw, mpad, kh,
                                                 L[0], L[1], L[2], v, vhead), note_launch());
}

// b^sol_k = A v: in float storage the head k-vectors (the heaviest weights) are
// contracted in FP64 against an FP64 copy of their operand columns.
void launch_bsol_kspace(bool fp64, const void* A, const double* Ahead, int n, int mpad, int kh,
                        const void* v, const double* vhead, int frames, double* bsol,
                        cudaStream_t s) {
  const int blocks = (n * 32 + 255) / 256;
  const int64_t lda = 2 * (int64_t)mpad;
  for (int f0 = 0; f0 < frames; f0 += 4) {
    if (fp64) {
      (k_bsol_kspace<double, 4><<<blocks, 256, 0, s>>>((const double*)A, n, lda,
                                                       (const double*)v, frames, f0, bsol, 0), note_launch());
    } else {
      (k_bsol_kspace<float, 4><<<blocks, 256, 0, s>>>((const float*)A, n, lda,
                                                      (const float*)v, frames, f0, bsol, 0), note_launch());
      if (kh > 0)
        (k_bsol_kspace<double, 4><<<blocks, 256, 0, s>>>(Ahead, n, 2 * (int64_t)kh, vhead,
                                                         frames, f0, bsol, 1), note_launch());
    }
  }
}

void launch_bsol_real_and_finish(bool fp64, const double* xyz, const double* alpha, int n,
                                 const double* ion_xyz, const double* ion_q, int frames,
                                 int n_ion, const Geometry& geo, const double* chi,
                                 const double* bsol_k, double* b_out, double* qsol,
                                 cudaStream_t s) {
  (void)fp64;
  dim3 grid((n + 127) / 128, frames);
  double dip = geo.slab ? 4.0 * kPi / geo.vol : 0.0;
  (k_bsol_real<<<grid, 128, 0, s>>>(xyz, alpha, n, ion_xyz, ion_q, n_ion, geo.L[0], geo.L[1],
                                   geo.L[2], geo.g, geo.rc, dip, chi, bsol_k, b_out, qsol), note_launch());
}

}  // namespace cpm
