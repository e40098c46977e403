// Fixed total charge per electrode (galvanostatic charge-discharge, GCD; Supplementary
// Note, Eq. S14-S24): the kernels around the context's PCG.  The PCG gives q^b = E^-1 b
// for the frames and a^h = E^-1 b^h for the indicator vectors b^h of the M electrodes
// (Eq. S22-S23); these kernels form the indicators, the per-electrode sums that make the
// capacitance coefficients C_ab (Eq. S24) and the charge defects Delta Q_a, invert C,
// and add q^Delta mu = A C^-1 Delta Q (Eq. S16-S20).  Every sum runs in a fixed order in
// FP64, so results repeat bit for bit.
#include "cpm_internal.cuh"

namespace cpm {
namespace {

constexpr int kGcdThreads = 256;

__device__ double block_sum_d(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// b^h_i = 1 on the atoms of electrode h, else 0 (Eq. S22); layout [h][i].
__global__ void k_gcd_indicators(const int* __restrict__ labels, int n, int m,
                                 double* __restrict__ bh) {
  const int64_t len = (int64_t)m * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int h = (int)(t / n), i = (int)(t - (int64_t)h * n);
    bh[t] = labels[i] == h ? 1.0 : 0.0;
  }
}

// out[v * m + a] = sum of x[v * n + i] over the atoms i of electrode a (the coarse
// graining of Eq. S18 and Eq. S24): block (v, a), a fixed summation order.
__global__ void __launch_bounds__(kGcdThreads)
k_gcd_sums(const double* __restrict__ x, int n, const int* __restrict__ labels, int m,
           double* __restrict__ out) {
  __shared__ double sm[kGcdThreads / 32];
  const int v = blockIdx.x, a = blockIdx.y;
  const double* xv = x + (int64_t)v * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (labels[i] == a) s += xv[i];
  s = block_sum_d(s, sm);
  if (threadIdx.x == 0) out[(int64_t)v * m + a] = s;
}

// C^-1 by Gauss-Jordan elimination with partial pivoting in one thread (m is at most
// CPM_GCD_MAX_ELECTRODES).  ct[b * m + a] = C_ab, the sums of column a^b over electrode
// a; C is symmetric up to the solves' tolerance and is used as formed.  status: 0, or 1
// when a pivot is below 1e-14 of the largest entry (C singular to working precision).
__global__ void k_gcd_invert(const double* __restrict__ ct, int m, double* __restrict__ cinv,
                             int* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int kM = CPM_GCD_MAX_ELECTRODES;
  double a[kM * kM], r[kM * kM];
  double big = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      a[i * kM + j] = ct[j * m + i];
      r[i * kM + j] = i == j ? 1.0 : 0.0;
      big = fmax(big, fabs(a[i * kM + j]));
    }
  *status = 0;
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs(a[i * kM + k]) > fabs(a[p * kM + k])) p = i;
    if (!(fabs(a[p * kM + k]) > 1e-14 * big)) {
      *status = 1;
      return;
    }
    if (p != k)
      for (int j = 0; j < m; ++j) {
        double t = a[k * kM + j];
        a[k * kM + j] = a[p * kM + j];
        a[p * kM + j] = t;
        t = r[k * kM + j];
        r[k * kM + j] = r[p * kM + j];
        r[p * kM + j] = t;
      }
    const double inv = 1.0 / a[k * kM + k];
    for (int j = 0; j < m; ++j) {
      a[k * kM + j] *= inv;
      r[k * kM + j] *= inv;
    }
    for (int i = 0; i < m; ++i) {
      if (i == k) continue;
      const double f = a[i * kM + k];
      if (f == 0.0) continue;
      for (int j = 0; j < m; ++j) {
        a[i * kM + j] -= f * a[k * kM + j];
        r[i * kM + j] -= f * r[k * kM + j];
      }
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) cinv[i * m + j] = r[i * kM + j];
}

// Delta mu_E = C^-1 (Q^0 - B^T q^b) per frame (Eq. S20): dmu[f * m + a] in e/A and, when
// asked, in volts.
__global__ void k_gcd_shifts(const double* __restrict__ cinv, const double* __restrict__ q0,
                             const double* __restrict__ sums, int nrhs, int m,
                             double* __restrict__ dmu, double* __restrict__ dmu_volts) {
  const int64_t len = (int64_t)nrhs * m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / m;
    const int a = (int)(t - f * m);
    double v = 0.0;
    for (int b = 0; b < m; ++b) v += cinv[a * m + b] * (q0[f * m + b] - sums[f * m + b]);
    dmu[t] = v;
    if (dmu_volts) dmu_volts[t] = v * kKe;
  }
}

// q += A Delta mu per frame (Eq. S16-S17 with the columns a^h of Eq. S23).
__global__ void k_gcd_apply(double* __restrict__ q, const double* __restrict__ amat,
                            const double* __restrict__ dmu, int n, int nrhs, int m) {
  const int64_t len = (int64_t)nrhs * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / n;
    const int i = (int)(t - f * n);
    double v = 0.0;
    for (int h = 0; h < m; ++h) v += amat[(int64_t)h * n + i] * dmu[f * m + h];
    q[t] += v;
  }
}

int grid_for(int64_t len) {
  return (int)std::min<int64_t>((len + kGcdThreads - 1) / kGcdThreads, 4096);
}

}  // namespace

void launch_gcd_indicators(const int* labels, int n, int m, double* bh, cudaStream_t s) {
  (k_gcd_indicators<<<grid_for((int64_t)m * n), kGcdThreads, 0, s>>>(labels, n, m, bh),
   note_launch());
}

void launch_gcd_sums(const double* x, int n, int nvec, const int* labels, int m, double* out,
                     cudaStream_t s) {
  (k_gcd_sums<<<dim3(nvec, m), kGcdThreads, 0, s>>>(x, n, labels, m, out), note_launch());
}

void launch_gcd_invert(const double* ct, int m, double* cinv, int* status, cudaStream_t s) {
  (k_gcd_invert<<<1, 32, 0, s>>>(ct, m, cinv, status), note_launch());
}

void launch_gcd_shifts(const double* cinv, const double* q0, const double* sums, int nrhs,
                       int m, double* dmu, double* dmu_volts, cudaStream_t s) {
  (k_gcd_shifts<<<grid_for((int64_t)nrhs * m), kGcdThreads, 0, s>>>(cinv, q0, sums, nrhs, m,
                                                                    dmu, dmu_volts),
   note_launch());
}

void launch_gcd_apply(double* q, const double* amat, const double* dmu, int n, int nrhs, int m,
                      cudaStream_t s) {
  (k_gcd_apply<<<grid_for((int64_t)nrhs * n), kGcdThreads, 0, s>>>(q, amat, dmu, n, nrhs, m),
   note_launch());
}

}  // namespace cpm
