// Cluster-resident PCG for small electrodes: one thread-block cluster of kCs CTAs per
// right-hand side runs the whole solve in one launch (Sec. III B 2's iteration, the same
// arithmetic as pcg.cu: error-free float-pair products of the stored float E, FP64
// vectors and reductions, flexible Polak-Ribiere beta with PCG-DC).
//
// Each CTA owns a slice of the rows; every CTA keeps the whole direction p (float pair)
// and the whole residual r (FP64) in shared memory, and writes the slices it updates into
// its peers' copies through distributed shared memory.  Dot products are exchanged the
// same way: each CTA stores its partial into a slot of every CTA, and after the cluster
// barrier every CTA sums the slots in rank order, so all of them take the same decisions
// (convergence, breakdown) on the same numbers.  Four cluster barriers an iteration;
// nothing goes back to the host until the solve ends, so a solve of a 512-atom electrode
// is one launch instead of about six launches an iteration and a poll every four.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "cpm_internal.cuh"

namespace cg = cooperative_groups;

namespace cpm {
namespace {

constexpr int kCs = 8;              // CTAs per cluster (portable cluster size)
constexpr int kCThreads = 256;
constexpr int kCWarps = kCThreads / 32;

struct ColOut {  // per right-hand side: iterations, status (1 converged, 2 breakdown, 0
  int iters;     // maxit reached), relative residual
  int status;
  double relres;
};

__device__ __forceinline__ double warp_sum_d(double x) {
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block sum of NV doubles per thread, stored by thread 0 into slot `slot` of every CTA of
// the cluster (slots[rank][NV] in each CTA).
template <int NV>
__device__ void exchange(cg::cluster_group& cl, double (&v)[NV], double* red, double* slots,
                         unsigned rank) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = warp_sum_d(v[t]);
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < NV; ++t) red[warp * NV + t] = v[t];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < kCWarps; ++w) s += red[w * NV + threadIdx.x];
    for (unsigned r = 0; r < kCs; ++r) {
      double* dst = cl.map_shared_rank(slots, r);
      dst[rank * NV + threadIdx.x] = s;
    }
  }
}

// Sum of slot t over the ranks, in rank order (after the cluster barrier).
__device__ __forceinline__ double slot_total(const double* slots, int nv, int t) {
  double s = 0.0;
  for (int r = 0; r < kCs; ++r) s += slots[r * nv + t];
  return s;
}

// Writes rows [r0, r1) of a per-row array into every CTA's copy (the CTA's own included).
template <typename T>
__device__ void broadcast_rows(cg::cluster_group& cl, T* arr, int r0, int r1) {
  for (unsigned r = 0; r < kCs; ++r) {
    T* dst = cl.map_shared_rank(arr, r);
    for (int i = r0 + (int)threadIdx.x; i < r1; i += kCThreads) dst[i] = arr[i];
  }
}

struct ClusterArgs {
  const float* E;
  int64_t ldE;
  int n, nrhs;
  const double* b;  // [nrhs][n], times bscale
  double bscale;
  double* x;        // [nrhs][n]: guess in (use_guess), solution out
  int use_guess;
  double tol;
  int maxit;
  int pre;          // CPM_PRECOND_*
  const double* inv_diag;
  const int64_t* off;
  const int* idx;
  const double* prow;
  double pgap;
  int flexible;
  ColOut* out;
};

// q_i = (E p)_i for the rows [r0, r1) from the shared float-pair copy of p (ph + pl):
// one warp per row, four columns a lane per step, error-free products and sums.
__device__ void rows_matvec(const ClusterArgs& a, const float* ph, const float* pl, int r0,
                            int r1, double* q) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ngroups = (int)(a.ldE >> 7);
  for (int row = r0 + warp; row < r1; row += kCWarps) {
    const float* e = a.E + (int64_t)row * a.ldE;
    float h = 0.f, l = 0.f;
    for (int g = 0; g < ngroups; ++g) {
      const int c = g * 128 + lane * 4;
      const float4 ev = __ldg(reinterpret_cast<const float4*>(e + c));
      const float4 hv = *reinterpret_cast<const float4*>(ph + c);
      const float4 lv = *reinterpret_cast<const float4*>(pl + c);
      pair_fma(h, l, hv.x, lv.x, ev.x);
      pair_fma(h, l, hv.y, lv.y, ev.y);
      pair_fma(h, l, hv.z, lv.z, ev.z);
      pair_fma(h, l, hv.w, lv.w, ev.w);
    }
    // combine the lanes' pairs in FP64 (exact enough: each is ~1e-14 of its sum)
    double v = warp_sum_d((double)h + (double)l);
    if (lane == 0) q[row - r0] = v;
  }
}

__global__ void __launch_bounds__(kCThreads)
k_pcg_cluster(ClusterArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const int col = blockIdx.x / kCs;
  const int n = a.n;
  const int per = (n + kCs - 1) / kCs;
  const int r0 = min(n, (int)rank * per), r1 = min(n, r0 + per);
  const int rows = r1 - r0;
  const int npad = (int)a.ldE;
  extern __shared__ __align__(16) uint8_t csm[];
  // full p (float pair) and r, then the own rows' x, z, q, p (FP64), then exchange slots
  float* ph = reinterpret_cast<float*>(csm);
  float* pl = ph + npad;
  double* rf = reinterpret_cast<double*>(pl + npad);
  double* xs = rf + npad;
  double* zs = xs + per;
  double* qs = zs + per;
  double* ps = qs + per;
  double* slotA = ps + per;        // [kCs][1]: p^T q
  double* slotB = slotA + kCs;     // [kCs][3]: r^T r, sum r, b^T b
  double* slotC = slotB + 3 * kCs; // [kCs][2]: r^T z_new, r^T z_old
  double* red = slotC + 2 * kCs;   // [warps][3]
  const double* bc = a.b + (int64_t)col * n;
  double* xc = a.x + (int64_t)col * n;
  const int tid = threadIdx.x;

  for (int i = tid; i < npad; i += kCThreads) {  // padding columns stay zero
    ph[i] = 0.f;
    pl[i] = 0.f;
    rf[i] = 0.0;
  }
  __syncthreads();
  // initial residual: r = b - E x0 (guess) or b
  for (int i = tid; i < rows; i += kCThreads) xs[i] = a.use_guess ? xc[r0 + i] : 0.0;
  if (a.use_guess) {
    for (int i = tid; i < rows; i += kCThreads) {
      const double v = xs[i];
      ph[r0 + i] = (float)v;
      pl[r0 + i] = (float)(v - (double)(float)v);
    }
    __syncthreads();
    broadcast_rows(cl, ph, r0, r1);
    broadcast_rows(cl, pl, r0, r1);
    cl.sync();
    rows_matvec(a, ph, pl, r0, r1, qs);
    __syncthreads();
  }
  {
    double v[3] = {0.0, 0.0, 0.0};
    for (int i = tid; i < rows; i += kCThreads) {
      const double bi = bc[r0 + i] * a.bscale;
      const double ri = a.use_guess ? bi - qs[i] : bi;
      rf[r0 + i] = ri;
      v[0] += ri * ri;
      v[1] += ri;
      v[2] += bi * bi;
    }
    __syncthreads();
    broadcast_rows(cl, rf, r0, r1);
    exchange<3>(cl, v, red, slotB, rank);
  }
  cl.sync();
  const double bb = slot_total(slotB, 3, 2);
  double rr = slot_total(slotB, 3, 0), rsum = slot_total(slotB, 3, 1);
  double relres = 0.0;
  int status;
  if (!isfinite(bb) || !isfinite(rr)) {
    status = 2;  // a non-finite right-hand side or guess
    relres = rr / bb;
  } else if (bb == 0.0) {
    status = 1;  // q = 0
  } else {
    relres = sqrt(rr / bb);
    status = relres <= a.tol ? 1 : 0;
  }
  // z = P r on the own rows (PCG-DC: the pattern of Eq. 36 plus the p_gap fill of Eq. 37)
  auto precondition = [&](double (&v)[2]) {
    const double gsum = a.pgap * rsum;
    for (int i = tid; i < rows; i += kCThreads) {
      const int j = r0 + i;
      double zn;
      if (a.pre == CPM_PRECOND_DC) {
        zn = gsum;
        for (int64_t e = a.off[j]; e < a.off[j + 1]; ++e) zn += a.prow[e] * rf[a.idx[e]];
      } else if (a.pre == CPM_PRECOND_JACOBI) {
        zn = rf[j] * a.inv_diag[j];
      } else {
        zn = rf[j];
      }
      v[0] += rf[j] * zn;
      v[1] += rf[j] * zs[i];
      zs[i] = zn;
    }
  };
  double rz = 0.0;
  if (status == 0) {
    double v[2] = {0.0, 0.0};
    for (int i = tid; i < rows; i += kCThreads) zs[i] = 0.0;
    precondition(v);
    exchange<2>(cl, v, red, slotC, rank);
    cl.sync();
    rz = slot_total(slotC, 2, 0);
    for (int i = tid; i < rows; i += kCThreads) {  // p = z
      const double v2 = zs[i];
      ps[i] = v2;
      ph[r0 + i] = (float)v2;
      pl[r0 + i] = (float)(v2 - (double)(float)v2);
    }
    __syncthreads();
    broadcast_rows(cl, ph, r0, r1);
    broadcast_rows(cl, pl, r0, r1);
    cl.sync();
  }
  int it = 0;
  while (status == 0 && it < a.maxit) {
    // q = E p, alpha = r^T z / p^T q
    rows_matvec(a, ph, pl, r0, r1, qs);
    __syncthreads();
    {
      double v[1] = {0.0};
      for (int i = tid; i < rows; i += kCThreads) v[0] += ps[i] * qs[i];
      exchange<1>(cl, v, red, slotA, rank);
    }
    cl.sync();
    const double pq = slot_total(slotA, 1, 0);
    if (!(pq > 0.0) || !isfinite(pq)) {
      status = 2;
      break;
    }
    const double alpha = rz / pq;
    // x += alpha p, r -= alpha q; ||r||, sum r
    {
      double v[3] = {0.0, 0.0, 0.0};
      for (int i = tid; i < rows; i += kCThreads) {
        xs[i] += alpha * ps[i];
        const double ri = rf[r0 + i] - alpha * qs[i];
        rf[r0 + i] = ri;
        v[0] += ri * ri;
        v[1] += ri;
      }
      __syncthreads();
      broadcast_rows(cl, rf, r0, r1);
      exchange<3>(cl, v, red, slotB, rank);
    }
    cl.sync();
    ++it;
    rr = slot_total(slotB, 3, 0);
    rsum = slot_total(slotB, 3, 1);
    relres = sqrt(rr / bb);
    if (!isfinite(relres)) {
      status = 2;
      break;
    }
    if (relres <= a.tol) {
      status = 1;
      break;
    }
    // z = P r, beta, p = z + beta p
    {
      double v[2] = {0.0, 0.0};
      precondition(v);
      exchange<2>(cl, v, red, slotC, rank);
    }
    cl.sync();
    const double rz_new = slot_total(slotC, 2, 0), rz_old = slot_total(slotC, 2, 1);
    const double beta = a.flexible ? (rz_new - rz_old) / rz : rz_new / rz;
    rz = rz_new;
    if (!isfinite(beta) || !(rz != 0.0)) {
      status = 2;
      break;
    }
    for (int i = tid; i < rows; i += kCThreads) {
      const double v2 = zs[i] + beta * ps[i];
      ps[i] = v2;
      ph[r0 + i] = (float)v2;
      pl[r0 + i] = (float)(v2 - (double)(float)v2);
    }
    __syncthreads();
    broadcast_rows(cl, ph, r0, r1);
    broadcast_rows(cl, pl, r0, r1);
    cl.sync();
  }
  for (int i = tid; i < rows; i += kCThreads) xc[r0 + i] = xs[i];
  if (rank == 0 && tid == 0) {
    a.out[col].iters = it;
    a.out[col].status = status;
    a.out[col].relres = relres;
  }
  cl.sync();  // no CTA leaves while a peer may still write into it
}

size_t cluster_smem(int npad, int n) {
  const int per = (n + kCs - 1) / kCs;
  return (size_t)npad * (4 + 4 + 8) + (size_t)per * 4 * 8 + (size_t)(kCs * 6 + kCWarps * 3) * 8;
}

}  // namespace

int cluster_solve_max_atoms() { return 4096; }

// The whole solve for every right-hand side in one launch; CPM_EINVAL when the electrode
// does not fit the kernel (float storage, n <= cluster_solve_max_atoms()).
int pcg_solve_cluster(Ctx* c, const SolveArgs& a) {
  if (c->fp64() || a.sys || a.ws || c->n > cluster_solve_max_atoms()) return CPM_EINVAL;
  const int n = c->n;
  ClusterArgs ca;
  ca.E = (const float*)c->E.ptr;
  ca.ldE = c->ldE;
  ca.n = n;
  ca.nrhs = a.nrhs;
  ca.b = a.b;
  ca.bscale = a.bscale;
  ca.x = a.x;
  ca.use_guess = a.use_guess ? 1 : 0;
  ca.tol = a.tol;
  ca.maxit = a.maxit;
  ca.pre = c->p.precond >= CPM_PRECOND_DC ? CPM_PRECOND_DC : c->p.precond;  // row-form P
  ca.inv_diag = c->diag.ptr ? (const double*)c->diag.ptr + n : nullptr;
  ca.off = (const int64_t*)c->nbr_off.ptr;
  ca.idx = (const int*)c->nbr_idx.ptr;
  ca.prow = (const double*)c->prow.ptr;
  ca.pgap = c->pgap;
  ca.flexible = ca.pre == CPM_PRECOND_DC ? 1 : 0;
  int st;
  if ((st = buf_reserve(c, &c->ws_cluster, (size_t)a.nrhs * sizeof(ColOut)))) return st;
  ca.out = (ColOut*)c->ws_cluster.ptr;
  const size_t smem = cluster_smem((int)c->ldE, n);
  if ((st = cuda_check(c, cudaFuncSetAttribute(k_pcg_cluster,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem), "cluster smem")))
    return st;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCs * a.nrhs);
  cfg.blockDim = dim3(kCThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kCs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if ((st = cuda_check(c, cudaLaunchKernelEx(&cfg, k_pcg_cluster, ca), "cluster pcg")))
    return st;
  note_launch();
  std::vector<ColOut> h(a.nrhs);
  if ((st = cuda_check(c, cudaMemcpyAsync(h.data(), ca.out, a.nrhs * sizeof(ColOut),
                                          cudaMemcpyDeviceToHost, c->stream), "cluster out")) ||
      (st = cuda_check(c, cudaStreamSynchronize(c->stream), "cluster sync")))
    return st;
  int status = CPM_OK;
  for (int col = 0; col < a.nrhs; ++col) {
    if (a.iters) a.iters[col] = h[col].iters;
    if (a.relres) a.relres[col] = h[col].relres;
    if (h[col].status == 2) status = CPM_EBREAKDOWN;
    else if (h[col].status == 0 && status == CPM_OK) status = CPM_ENOCONV;
  }
  if (status == CPM_EBREAKDOWN) return set_err(c, status, "PCG breakdown (p^T E p <= 0 or non-finite)");
  if (status == CPM_ENOCONV) return set_err(c, status, "PCG reached maxit before tol");
  return CPM_OK;
}

}  // namespace cpm
