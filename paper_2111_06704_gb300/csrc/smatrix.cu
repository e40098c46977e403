// The matrix path for a fixed electrode: S = E^-1 (I - 1 d^T) (Eq. 33), formed once, then
// the neutral charges of every frame by one dense product, q = S b - Q^sol d (Eq. 33 with
// the second step of Eq. 35: S b = q^b - Q^b d).  The context's PCG gives the columns
// E^-1 e_j; these kernels make the identity right-hand sides, subtract the rank-one
// neutralising part, and apply S to many frames at once.  FP64 throughout.
#include "cpm_internal.cuh"

namespace cpm {
namespace {

constexpr int kSmThreads = 256;
constexpr int kSmFrames = 4;  // frames per thread in the product

// x[j * n + i] = 1 if i == j else 0: the right-hand sides e_j, one per column j.
__global__ void k_identity(double* __restrict__ x, int n) {
  const int64_t len = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / n;
    x[t] = (t - j * n) == j ? 1.0 : 0.0;
  }
}

// In place on X[j * n + i] = (E^-1)_ij: S_ij = (E^-1)_ij - (E^-1 1)_i d_j, where
// E^-1 1 = C^ele d (Eq. S8-S9), so S_ij = X_ij - C^ele d_i d_j.
__global__ void k_smatrix_form(double* __restrict__ x, const double* __restrict__ d,
                               double c_ele, int n) {
  const int64_t len = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < len;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / n;
    const int i = (int)(t - j * n);
    x[t] -= c_ele * d[i] * d[j];
  }
}

// q[f * n + i] = bscale * sum_j S_ij b[f * n + j] - Q^sol_f d_i for kSmFrames frames per
// thread; S[j * n + i] = S_ij, read along i by neighbouring threads.
__global__ void __launch_bounds__(kSmThreads)
k_smatrix_apply(const double* __restrict__ S, const double* __restrict__ b,
                const double* __restrict__ qsol, const double* __restrict__ d, int n,
                int frames, double bscale, double* __restrict__ q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int f0 = blockIdx.y * kSmFrames;
  if (i >= n) return;
  const int nf = min(kSmFrames, frames - f0);
  double acc[kSmFrames] = {0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < n; ++j) {
    const double s = S[(int64_t)j * n + i];
#pragma unroll
    for (int t = 0; t < kSmFrames; ++t)
      if (t < nf) acc[t] += s * b[(int64_t)(f0 + t) * n + j];
  }
#pragma unroll
  for (int t = 0; t < kSmFrames; ++t)
    if (t < nf)
      q[(int64_t)(f0 + t) * n + i] = acc[t] * bscale - (qsol ? qsol[f0 + t] : 0.0) * d[i];
}

int grid_for(int64_t len) {
  return (int)std::min<int64_t>((len + kSmThreads - 1) / kSmThreads, 8192);
}

}  // namespace

int smatrix_max_frames() { return 65535 * kSmFrames; }

void launch_identity(double* x, int n, cudaStream_t s) {
  (k_identity<<<grid_for((int64_t)n * n), kSmThreads, 0, s>>>(x, n), note_launch());
}

void launch_smatrix_form(double* x, const double* d, double c_ele, int n, cudaStream_t s) {
  (k_smatrix_form<<<grid_for((int64_t)n * n), kSmThreads, 0, s>>>(x, d, c_ele, n),
   note_launch());
}

void launch_smatrix_apply(const double* S, const double* b, const double* qsol, const double* d,
                          int n, int frames, double bscale, double* q, cudaStream_t s) {
  const dim3 grid((n + kSmThreads - 1) / kSmThreads, (frames + kSmFrames - 1) / kSmFrames);
  (k_smatrix_apply<<<grid, kSmThreads, 0, s>>>(S, b, qsol, d, n, frames, bscale, q),
   note_launch());
}

}  // namespace cpm
