// PCG-DC preconditioner (Sec. III B 2, steps 1-3; Eq. 36).
//
// For every electrode atom tau: its neighbours j with |r_tau - r_j| <= r_cut (minimum
// image, tau included, sorted by index); the local matrix M_tau of Eq. 36 over them;
// column tau of M_tau^-1, i.e. the solution of M_tau x = e_tau, by Gaussian elimination
// with partial pivoting in FP64 shared memory (one block per atom).  The column is
// stored as P[j, tau] for the neighbours j; a transpose pass re-files it by row so the
// apply z_j = sum_tau P[j, tau] r_tau is a gather.
#include <math.h>

#include <algorithm>
#include <vector>

#include "cpm_internal.cuh"

namespace cpm {

namespace {

constexpr int kMaxLocal = 160;  // largest neighbourhood held in shared memory

__device__ __forceinline__ double min_image(double d, double L) { return d - L * rint(d / L); }

__device__ __forceinline__ double dist2(const double* a, const double* b, double lx, double ly,
                                        double lz) {
  double dx = min_image(a[0] - b[0], lx), dy = min_image(a[1] - b[1], ly),
         dz = min_image(a[2] - b[2], lz);
  return dx * dx + dy * dy + dz * dz;
}

// One warp per atom: count (fill == 0) or list (fill == 1) its neighbours in index order
// (r <= r_cut, or r < r_cut with strict).
// The candidates of a block are staged as float positions; the float minimum-image
// distance decides every pair outside a band of +-0.01 A^2 around r_cut^2 (float
// positions of a box below 1e4 A are off by < 1e-3 A, so the band is ample), and the
// pairs inside it are decided by the FP64 distance, as the definition asks.  The float
// constants come from the host (a constant formed from the FP64 parameters could be
// re-formed inside the loop, at 1/64 of the float rate).
constexpr int kNbrWarps = 8;
constexpr int kNbrStage = 1024;

struct NbrFloat {
  float L[3], inv[3];  // box edges and their reciprocals
  float lo2, hi2;      // r_cut^2 -+ 0.01: the band decided in FP64
};

__global__ void __launch_bounds__(kNbrWarps * 32)
k_neighbours(const double* __restrict__ xyz, int n, double lx, double ly, double lz,
             double rc2, const NbrFloat nf, int* __restrict__ cnt,
             const int64_t* __restrict__ off, int* __restrict__ idx, int fill, int strict) {
  __shared__ float4 sp[kNbrStage];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * kNbrWarps + warp;
  const bool live = t < n;
  const float Lx = nf.L[0], Ly = nf.L[1], Lz = nf.L[2];
  const float ix = nf.inv[0], iy = nf.inv[1], iz = nf.inv[2];
  const float lo2 = nf.lo2, hi2 = nf.hi2;
  float tx = 0.f, ty = 0.f, tz = 0.f;
  if (live) {
    tx = (float)xyz[3 * t];
    ty = (float)xyz[3 * t + 1];
    tz = (float)xyz[3 * t + 2];
  }
  int c = 0;
  for (int base = 0; base < n; base += kNbrStage) {
    const int cj = min(kNbrStage, n - base);
    __syncthreads();
    for (int e = threadIdx.x; e < cj; e += blockDim.x)
      sp[e] = make_float4((float)xyz[3 * (base + e)], (float)xyz[3 * (base + e) + 1],
                          (float)xyz[3 * (base + e) + 2], 0.f);
    __syncthreads();
    if (!live) continue;
    for (int jj = 0; jj < cj; jj += 32) {
      const int j = base + jj + lane;
      bool in = false;
      if (jj + lane < cj) {
        const float4 pj = sp[jj + lane];
        float dx = pj.x - tx, dy = pj.y - ty, dz = pj.z - tz;
        dx -= Lx * rintf(dx * ix);
        dy -= Ly * rintf(dy * iy);
        dz -= Lz * rintf(dz * iz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < lo2) in = true;
        else if (r2 <= hi2) {
          const double d2 = dist2(xyz + 3 * t, xyz + 3 * j, lx, ly, lz);
          in = strict ? d2 < rc2 : d2 <= rc2;
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (fill && in) idx[off[t] + c + __popc(m & ((1u << lane) - 1u))] = j;
      c += __popc(m);
    }
  }
  if (!fill && live && lane == 0) cnt[t] = c;
}

void launch_neighbours(const double* xyz, int n, const double* L, double rc2, int* cnt,
                       const int64_t* off, int* idx, int fill, int strict, cudaStream_t s) {
  NbrFloat nf;
  for (int u = 0; u < 3; ++u) {
    nf.L[u] = (float)L[u];
    nf.inv[u] = (float)(1.0 / L[u]);
  }
  nf.lo2 = (float)rc2 - 0.01f;
  nf.hi2 = (float)rc2 + 0.01f;
  const int blocks = (n + kNbrWarps - 1) / kNbrWarps;
  (k_neighbours<<<blocks, kNbrWarps * 32, 0, s>>>(xyz, n, L[0], L[1], L[2], rc2, nf, cnt, off,
                                                   idx, fill, strict),
   note_launch());
}

// The off-diagonal value of Eq. 36 for every pattern entry (j, j'): (erfc(g r) -
// erfc(g r_cut)) / r, zero for the atom itself and at r = r_cut.  Every local matrix
// M_tau only holds pairs within r_cut of each other, i.e. pattern entries, so the FP64
// erfc runs once per entry instead of once per entry of every local matrix.
__global__ void k_dc_pairs(const double* __restrict__ xyz, int n, double lx, double ly,
                           double lz, double g, double rcut, const int64_t* __restrict__ off,
                           const int* __restrict__ idx, double* __restrict__ val) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double erfc_rc = erfc(g * rcut);
  const double rc2 = rcut * rcut;
  for (int64_t e = off[j]; e < off[j + 1]; ++e) {
    const int k = idx[e];
    double v = 0.0;
    if (k != j) {
      const double r2 = dist2(xyz + 3 * j, xyz + 3 * k, lx, ly, lz);
      if (r2 < rc2) {
        const double r = sqrt(r2);
        v = (erfc(g * r) - erfc_rc) / r;
      }
    }
    val[e] = v;
  }
}

// Column tau of M_tau^-1 (Eq. 36), written to pcol[off[tau] .. off[tau+1]).  One block
// per atom.  The symmetric local matrix is filled in FP64 from the pattern's pair values
// (a pair of tau's neighbours closer than r_cut is an entry of the first one's pattern
// row: each warp walks a neighbour's row, coalesced, and finds each entry's position in
// tau's list, held in shared memory, by binary search) and kept as its packed upper
// triangle.  A float copy is factored P M = L U with partial pivoting (FP64 runs at 1/64
// of the float rate here, and the factorisation is m^3 / 3 multiply-adds), and the
// solution is refined against the FP64 matrix: x += (LU)^-1 P (e_tau - M x), residuals in
// FP64.  Each step shrinks the error by about kappa(M) 2^-24 (~1e-5 here), so the error
// left after adding a correction d is about that times |d|: refinement stops once
// |d| <= 1e-9 |x| (error ~1e-13 even at kappa(M) 2^-24 = 1e-4; typically after the
// second correction).
constexpr int kDcThreads = 128;
constexpr int kDcMaxRefine = 6;

__device__ __forceinline__ int sym_index(int a, int b, int m) {  // packed upper, a <= b
  return a * m - (a * (a - 1)) / 2 + (b - a);
}

// shared memory of k_dc_local for a neighbourhood of m atoms
size_t dc_local_smem(int m) {
  return (size_t)m * (m + 1) / 2 * sizeof(double) + 2 * (size_t)m * sizeof(double) +
         (size_t)m * (m + 1) * sizeof(float) + (size_t)m * sizeof(float) +
         2 * (size_t)m * sizeof(int) + 16;
}

__global__ void __launch_bounds__(kDcThreads)
k_dc_local(const double* __restrict__ alpha, const int64_t* __restrict__ off,
           const int* __restrict__ idx,
           const double* __restrict__ pval, double* __restrict__ pcol,
           int* __restrict__ status) {
  extern __shared__ double sm[];
  constexpr int kWarps = kDcThreads / 32;
  const int tau = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t o = off[tau];
  const int m = (int)(off[tau + 1] - o);
  const int ld = m + 1;                        // float row stride
  double* S = sm;                              // packed upper triangle of M (FP64)
  double* x = S + (size_t)m * (m + 1) / 2;     // solution (FP64)
  double* r = x + m;                           // residual (FP64)
  float* F = reinterpret_cast<float*>(r + m);  // [m][ld]: L (unit, below) and U
  float* y = F + (size_t)m * ld;               // correction (float)
  int* piv = reinterpret_cast<int*>(y + m);    // row exchanged with row k at step k
  int* list = piv + m;                         // tau's neighbours (ascending)
  __shared__ int s_piv, s_pos, s_done;
  __shared__ float s_val;
  for (int e = threadIdx.x; e < m * (m + 1) / 2; e += blockDim.x) S[e] = 0.0;
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    const int j = idx[o + a];
    list[a] = j;
    if (j == tau) s_pos = a;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    const double al = alpha[list[a]];
    S[sym_index(a, a, m)] = isinf(al) ? 0.0 : 0.7978845608028654 * al;  // sqrt(2/pi) alpha_i
  }
  for (int a = warp; a < m; a += kWarps) {
    const int ja = list[a];
    for (int64_t e = off[ja] + lane; e < off[ja + 1]; e += 32) {
      const int jb = idx[e];
      int lo = 0, hi = m;  // position of jb in tau's list, if there
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (list[mid] < jb) lo = mid + 1;
        else hi = mid;
      }
      if (lo < m && list[lo] == jb && lo > a) S[sym_index(a, lo, m)] = pval[e];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int a = e / m, b = e - a * m;
    F[a * ld + b] = (float)S[a <= b ? sym_index(a, b, m) : sym_index(b, a, m)];
  }
  __syncthreads();
  // ---- P M = L U in float, partial pivoting, whole rows exchanged ---------------------
  for (int k = 0; k < m; ++k) {
    if (warp == 0) {
      float best = -1.f;
      int bi = k;
      for (int a = k + lane; a < m; a += 32) {
        const float v = fabsf(F[a * ld + k]);
        if (v > best) {
          best = v;
          bi = a;
        }
      }
      for (int sh = 16; sh; sh >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, sh);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, sh);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_piv = bi;
        s_val = best;
        piv[k] = bi;
      }
    }
    __syncthreads();
    if (!(s_val > 0.f)) {
      if (threadIdx.x == 0) atomicExch(status, 1);
      return;  // singular local matrix (whole block leaves together)
    }
    const int pv = s_piv;
    if (pv != k)
      for (int b = threadIdx.x; b < m; b += blockDim.x) {
        const float t = F[k * ld + b];
        F[k * ld + b] = F[pv * ld + b];
        F[pv * ld + b] = t;
      }
    __syncthreads();
    const float inv = 1.f / F[k * ld + k];
    for (int a = k + 1 + warp; a < m; a += kWarps) {
      const float f = F[a * ld + k] * inv;
      for (int b = k + 1 + lane; b < m; b += 32) F[a * ld + b] -= f * F[k * ld + b];
      __syncwarp();
      if (lane == 0) F[a * ld + k] = f;
    }
    __syncthreads();
  }
  // ---- x = 0, r = e_tau; x += (LU)^-1 P r; r = e_tau - M x (FP64) ------------------------
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    x[a] = 0.0;
    r[a] = a == s_pos ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) s_done = 0;
  __syncthreads();
  for (int it = 0; it < kDcMaxRefine && !s_done; ++it) {
    if (warp == 0) {
      for (int a = lane; a < m; a += 32) y[a] = (float)r[a];
      __syncwarp();
      if (lane == 0)
        for (int k = 0; k < m; ++k)
          if (piv[k] != k) {
            const float t = y[k];
            y[k] = y[piv[k]];
            y[piv[k]] = t;
          }
      __syncwarp();
      for (int k = 0; k < m; ++k) {  // forward: unit lower L
        const float yk = y[k];
        for (int a = k + 1 + lane; a < m; a += 32) y[a] -= F[a * ld + k] * yk;
        __syncwarp();
      }
      for (int k = m - 1; k >= 0; --k) {  // back: U
        const float yk = y[k] / F[k * ld + k];
        __syncwarp();
        if (lane == 0) y[k] = yk;
        for (int a = lane; a < k; a += 32) y[a] -= F[a * ld + k] * yk;
        __syncwarp();
      }
      double dmax = 0.0, xmax = 0.0;
      for (int a = lane; a < m; a += 32) {
        x[a] += (double)y[a];
        dmax = fmax(dmax, fabs((double)y[a]));
        xmax = fmax(xmax, fabs(x[a]));
      }
      for (int sh = 16; sh; sh >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, sh));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, sh));
      }
      if (lane == 0 && dmax <= 1e-9 * xmax) s_done = 1;
    }
    __syncthreads();
    if (s_done) break;
    for (int a = warp; a < m; a += kWarps) {  // r = e_tau - M x, one warp per row
      double s = 0.0;
      for (int b = lane; b < m; b += 32)
        s += S[a <= b ? sym_index(a, b, m) : sym_index(b, a, m)] * x[b];
      for (int sh = 16; sh; sh >>= 1) s += __shfl_xor_sync(0xffffffffu, s, sh);
      if (lane == 0) r[a] = (a == s_pos ? 1.0 : 0.0) - s;
    }
    __syncthreads();
  }
  for (int a = threadIdx.x; a < m; a += blockDim.x) pcol[o + a] = x[a];
}

// prow[off[j] + position of tau in j's list] = pcol[off[tau] + a] - shift, j = idx[off[tau] + a]
__global__ void k_dc_transpose(int n, const int64_t* __restrict__ off, const int* __restrict__ idx,
                               const double* __restrict__ pcol, double shift,
                               double* __restrict__ prow) {
  const int tau = blockIdx.x;
  for (int64_t e = off[tau] + threadIdx.x; e < off[tau + 1]; e += blockDim.x) {
    const int j = idx[e];
    int64_t lo = off[j], hi = off[j + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (idx[mid] < tau) lo = mid + 1;
      else hi = mid;
    }
    if (lo < off[j + 1] && idx[lo] == tau) prow[lo] = pcol[e] - shift;
  }
}

__global__ void k_sum_blocks(const double* __restrict__ v, int64_t len, double* __restrict__ part) {
  __shared__ double sm[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    s += v[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

}  // namespace

// Sum of a device vector, deterministic (fixed block partials, host sum in order).
int device_sum(Ctx* c, const double* v, int64_t len, double* out) {
  const int blocks = 256;
  Buf tmp;
  if (int rc = buf_alloc(c, &tmp, blocks * sizeof(double))) return rc;
  (k_sum_blocks<<<blocks, 256, 0, c->stream>>>(v, len, (double*)tmp.ptr), note_launch());
  std::vector<double> h(blocks);
  int rc = cuda_check(c, cudaMemcpyAsync(h.data(), tmp.ptr, blocks * sizeof(double),
                                         cudaMemcpyDeviceToHost, c->stream), "sum copy");
  if (!rc) rc = cuda_check(c, cudaStreamSynchronize(c->stream), "sum sync");
  buf_free(c, &tmp);
  if (rc) return rc;
  double s = 0.0;
  for (double x : h) s += x;
  *out = s;
  return CPM_OK;
}

// Builds the neighbour pattern and the row form of P (without p_gap).
int build_dc_preconditioner(Ctx* c) {
  const int n = c->n;
  const double* L = c->p.box;
  const double rc = c->p.rcut_dc;
  if (!(rc > 0.0) || 2.0 * rc >= std::min(L[0], std::min(L[1], L[2])))
    return set_err(c, CPM_EINVAL, "rcut_dc must be positive and below half of every box edge");
  cudaStream_t s = c->stream;
  // workspace kept by the context (buf_reserve): the counts, the local solutions, a flag
  Buf &cnt = c->dc_cnt, &pcol = c->dc_pcol, &status = c->dc_status;
  if (int rc2 = buf_reserve(c, &cnt, (size_t)n * sizeof(int))) return rc2;
  launch_neighbours((const double*)c->xyz.ptr, n, L, rc * rc, (int*)cnt.ptr, nullptr, nullptr,
                    0, 0, s);
  std::vector<int> hc(n);
  int st = cuda_check(c, cudaMemcpyAsync(hc.data(), cnt.ptr, n * sizeof(int),
                                         cudaMemcpyDeviceToHost, s), "dc counts");
  if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "dc counts sync");
  if (st) return st;
  std::vector<int64_t> off(n + 1, 0);
  int mx = 0;
  for (int i = 0; i < n; ++i) {
    off[i + 1] = off[i] + hc[i];
    mx = std::max(mx, hc[i]);
  }
  if (mx > kMaxLocal)
    return set_err(c, CPM_EINVAL, "PCG-DC neighbourhood larger than 160 atoms; lower rcut_dc");
  c->nnz = off[n];
  if ((st = buf_reserve(c, &c->nbr_off, (n + 1) * sizeof(int64_t)))) return st;
  if ((st = buf_reserve(c, &c->nbr_idx, c->nnz * sizeof(int)))) return st;
  if ((st = buf_reserve(c, &c->prow, c->nnz * sizeof(double)))) return st;
  if ((st = buf_reserve(c, &pcol, c->nnz * sizeof(double)))) return st;
  if ((st = buf_reserve(c, &status, sizeof(int)))) return st;
  st = cuda_check(c, cudaMemcpyAsync(c->nbr_off.ptr, off.data(), (n + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, s), "dc offsets");
  if (!st) st = cuda_check(c, cudaMemsetAsync(status.ptr, 0, sizeof(int), s), "dc status");
  if (!st) {
    launch_neighbours((const double*)c->xyz.ptr, n, L, rc * rc, nullptr,
                      (const int64_t*)c->nbr_off.ptr, (int*)c->nbr_idx.ptr, 1, 0, s);
    const size_t smem = dc_local_smem(mx);
    st = cuda_check(c, cudaFuncSetAttribute(k_dc_local, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem), "dc smem");
    if (!st) {
      // pair values of the pattern, held in prow until the transpose overwrites it
      (k_dc_pairs<<<(n + 127) / 128, 128, 0, s>>>((const double*)c->xyz.ptr, n, L[0], L[1],
                                                  L[2], c->p.g_dc, rc,
                                                  (const int64_t*)c->nbr_off.ptr,
                                                  (const int*)c->nbr_idx.ptr,
                                                  (double*)c->prow.ptr), note_launch());
      (k_dc_local<<<n, kDcThreads, smem, s>>>((const double*)c->alpha.ptr,
                                              (const int64_t*)c->nbr_off.ptr,
                                              (const int*)c->nbr_idx.ptr,
                                              (const double*)c->prow.ptr, (double*)pcol.ptr,
                                              (int*)status.ptr), note_launch());
      (k_dc_transpose<<<n, 128, 0, s>>>(n, (const int64_t*)c->nbr_off.ptr,
                                       (const int*)c->nbr_idx.ptr, (const double*)pcol.ptr, 0.0,
                                       (double*)c->prow.ptr), note_launch());
      st = cuda_check(c, cudaGetLastError(), "dc kernels");
    }
  }
  int hs = 0;
  if (!st) st = cuda_check(c, cudaMemcpyAsync(&hs, status.ptr, sizeof(int),
                                              cudaMemcpyDeviceToHost, s), "dc status copy");
  if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "dc sync");
  if (st) return st;
  if (hs) return set_err(c, CPM_EINVAL, "a PCG-DC local matrix is singular");
  return CPM_OK;
}

// P[j][tau] = (E^-1)_{j tau} on the pattern, from the columns E^-1 e_tau (column-major,
// X[tau * n + j]); one block per row j.
__global__ void k_gather_inverse(int n, const int64_t* __restrict__ off,
                                 const int* __restrict__ idx, const double* __restrict__ X,
                                 double* __restrict__ prow) {
  const int j = blockIdx.x;
  for (int64_t e = off[j] + threadIdx.x; e < off[j + 1]; e += blockDim.x)
    prow[e] = X[(int64_t)idx[e] * n + j];
}

// PCG-Normal / PCG-Full (Sec. III B 2, Fig. 6a): the pattern of the pairs within the
// cutoff (minimum image; r < rcut_dc for Normal, r <= rcut_real for Full) and the entries
// of E^-1 on it, from the n columns E^-1 e_j solved by the context's PCG with the Jacobi
// preconditioner to 1e-10.  No p_gap fill.  n <= CPM_SMATRIX_MAX_ATOMS (two n x n FP64
// work arrays).
int build_sparse_inverse(Ctx* c) {
  const int n = c->n;
  const double* L = c->p.box;
  const bool full = c->p.precond == CPM_PRECOND_FULL;
  const double rc = full ? c->p.rcut_real : c->p.rcut_dc;
  if (n > CPM_SMATRIX_MAX_ATOMS)
    return set_err(c, CPM_EINVAL, "PCG-Normal / PCG-Full: n above CPM_SMATRIX_MAX_ATOMS");
  if (!(rc > 0.0)) return set_err(c, CPM_EINVAL, "PCG-Normal / PCG-Full: cutoff must be positive");
  cudaStream_t s = c->stream;
  Buf& cnt = c->dc_cnt;
  int st;
  if ((st = buf_reserve(c, &cnt, (size_t)n * sizeof(int)))) return st;
  launch_neighbours((const double*)c->xyz.ptr, n, L, rc * rc, (int*)cnt.ptr, nullptr, nullptr,
                    0, full ? 0 : 1, s);
  std::vector<int> hc(n);
  st = cuda_check(c, cudaMemcpyAsync(hc.data(), cnt.ptr, n * sizeof(int),
                                     cudaMemcpyDeviceToHost, s), "pattern counts");
  if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "pattern counts sync");
  if (st) return st;
  std::vector<int64_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + hc[i];
  c->nnz = off[n];
  c->pgap = 0.0;
  if ((st = buf_reserve(c, &c->nbr_off, (n + 1) * sizeof(int64_t))) ||
      (st = buf_reserve(c, &c->nbr_idx, c->nnz * sizeof(int))) ||
      (st = buf_reserve(c, &c->prow, c->nnz * sizeof(double))))
    return st;
  st = cuda_check(c, cudaMemcpyAsync(c->nbr_off.ptr, off.data(), (n + 1) * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, s), "pattern offsets");
  if (st) return st;
  launch_neighbours((const double*)c->xyz.ptr, n, L, rc * rc, nullptr,
                    (const int64_t*)c->nbr_off.ptr, (int*)c->nbr_idx.ptr, 1, full ? 0 : 1, s);
  // the columns of E^-1: one PCG over the n identity columns, Jacobi-preconditioned
  Buf ident, cols;
  const size_t bytes = (size_t)n * n * sizeof(double);
  if ((st = buf_alloc(c, &ident, bytes))) return st;
  if ((st = buf_alloc(c, &cols, bytes))) {
    buf_free(c, &ident);
    return st;
  }
  launch_identity((double*)ident.ptr, n, s);
  std::vector<int> it(n);
  std::vector<double> rr(n);
  SolveArgs a{n, (const double*)ident.ptr, 1.0, (double*)cols.ptr, false, 1e-10, 20000,
              it.data(), rr.data()};
  const int saved = c->p.precond;
  c->p.precond = CPM_PRECOND_JACOBI;
  st = pcg_solve(c, a);
  c->p.precond = saved;
  if (!st) {
    (k_gather_inverse<<<n, 128, 0, s>>>(n, (const int64_t*)c->nbr_off.ptr,
                                        (const int*)c->nbr_idx.ptr, (const double*)cols.ptr,
                                        (double*)c->prow.ptr), note_launch());
    st = cuda_check(c, cudaGetLastError(), "gather inverse");
  }
  if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "sparse inverse sync");
  buf_free(c, &ident);
  buf_free(c, &cols);
  return st;
}

__global__ void k_shift(double* __restrict__ v, int64_t len, double s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] -= s;
}

// The row form of P on its pattern, as Eq. 36 defines it (the p_gap shift taken back out).
int copy_precond(Ctx* c, int64_t* off, int* idx, double* val) {
  cudaStream_t s = c->stream;
  Buf tmp;
  int st = buf_alloc(c, &tmp, std::max<int64_t>(c->nnz, 1) * sizeof(double));
  if (st) return st;
  st = cuda_check(c, cudaMemcpyAsync(tmp.ptr, c->prow.ptr, c->nnz * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s), "P copy");
  if (!st && c->pgap != 0.0)
    (k_shift<<<256, 256, 0, s>>>((double*)tmp.ptr, c->nnz, -c->pgap), note_launch());
  if (!st) st = cuda_check(c, cudaMemcpyAsync(off, c->nbr_off.ptr, (c->n + 1) * sizeof(int64_t),
                                              cudaMemcpyDefault, s), "P offsets");
  if (!st) st = cuda_check(c, cudaMemcpyAsync(idx, c->nbr_idx.ptr, c->nnz * sizeof(int),
                                              cudaMemcpyDefault, s), "P columns");
  if (!st) st = cuda_check(c, cudaMemcpyAsync(val, tmp.ptr, c->nnz * sizeof(double),
                                              cudaMemcpyDefault, s), "P values");
  if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "P sync");
  buf_free(c, &tmp);
  return st;
}

// p_gap of Eq. 37 from C^ele = 1^T E^-1 1; stored as prow -= p_gap on the pattern.
int apply_p_gap(Ctx* c) {
  double sum_p = 0.0;
  if (int st = device_sum(c, (const double*)c->prow.ptr, c->nnz, &sum_p)) return st;
  const double n2 = (double)c->n * (double)c->n;
  const double nzero = n2 - (double)c->nnz;
  c->pgap = nzero > 0 ? (c->c_ele - sum_p) / nzero : 0.0;
  if (c->pgap != 0.0) (k_shift<<<256, 256, 0, c->stream>>>((double*)c->prow.ptr, c->nnz, c->pgap), note_launch());
  return cuda_check(c, cudaGetLastError(), "p_gap");
}

}  // namespace cpm
