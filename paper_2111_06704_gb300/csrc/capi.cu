// C ABI entry points (include/cpm.h): argument checks, staging of host arrays, the
// k-vector table, and the order of the build / potential / solve / neutralise steps.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "cpm_internal.cuh"

namespace cpm {

namespace {
std::atomic<long long> g_launches{0};
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int set_err(Ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_check(Ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CPM_OK;
  return set_err(c, CPM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int buf_alloc(Ctx* c, Buf* b, size_t bytes) {
  buf_free(c, b);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c->p.alloc) {
    p = c->p.alloc(bytes, c->p.alloc_user);
    if (!p) return set_err(c, CPM_ENOMEM, "allocator callback returned NULL");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, CPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  b->ptr = p;
  b->bytes = bytes;
  return CPM_OK;
}

void buf_free(Ctx* c, Buf* b) {
  if (!b->ptr) return;
  if (c->p.free) c->p.free(b->ptr, c->p.alloc_user);
  else cudaFree(b->ptr);
  b->ptr = nullptr;
  b->bytes = 0;
}

int buf_reserve(Ctx* c, Buf* b, size_t bytes) {
  if (b->ptr && b->bytes >= bytes) return CPM_OK;
  // the buffer may still be in use by queued work
  if (b->ptr) {
    int st = cuda_check(c, cudaStreamSynchronize(c->stream), "reserve sync");
    if (st) return st;
  }
  return buf_alloc(c, b, bytes);
}

int pointer_where(const Ctx* c, const void* p) {
  if (!p) return 0;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeManaged) return 1;
  if (at.type == cudaMemoryTypeDevice) return at.device == c->device ? 1 : -1;
  return 0;
}

int on_device(Ctx* c, const void* p, bool* dev) {
  const int w = pointer_where(c, p);
  if (w < 0)
    return set_err(c, CPM_EINVAL, "an array lives in the memory of another CUDA device than "
                                  "the context's");
  *dev = w > 0;
  return CPM_OK;
}

namespace {

// Returns a device pointer holding `bytes` of `src` (src itself if it is on the device).
int stage_in(Ctx* c, Buf* tmp, const void* src, size_t bytes, const void** out) {
  bool dev = false;
  if (int st = on_device(c, src, &dev)) return st;
  if (dev) {
    *out = src;
    return CPM_OK;
  }
  if (int st = buf_reserve(c, tmp, bytes)) return st;
  if (int st = cuda_check(c, cudaMemcpyAsync(tmp->ptr, src, bytes, cudaMemcpyHostToDevice,
                                             c->stream), "copy in"))
    return st;
  *out = tmp->ptr;
  return CPM_OK;
}

// Device destination for `dst` (dst itself when on the device); copy_out finishes it.
int stage_out(Ctx* c, Buf* tmp, void* dst, size_t bytes, void** out) {
  bool dev = false;
  if (int st = on_device(c, dst, &dev)) return st;
  if (dev) {
    *out = dst;
    return CPM_OK;
  }
  if (int st = buf_reserve(c, tmp, bytes)) return st;
  *out = tmp->ptr;
  return CPM_OK;
}

// Copies `count` elements of `src` (host or device) to the host vector `dst`.
template <typename T>
int to_host(Ctx* c, std::vector<T>& dst, const T* src, size_t count) {
  dst.resize(count);
  bool dev = false;
  if (int st = on_device(c, src, &dev)) return st;
  if (!dev) {
    std::copy(src, src + count, dst.begin());
    return CPM_OK;
  }
  return cuda_check(c, cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost),
                    "copy to host");
}

int copy_out(Ctx* c, void* dst, const void* dev, size_t bytes) {
  if (dst == dev) return CPM_OK;
  return cuda_check(c, cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, c->stream),
                    "copy out");
}

Geometry geometry(const Ctx* c) {
  Geometry g;
  for (int d = 0; d < 3; ++d) g.L[d] = c->p.box[d];
  g.vol = c->p.box[0] * c->p.box[1] * c->p.box[2];
  g.g = c->p.g_ewald;
  g.rc = c->p.rcut_real;
  g.slab = c->p.slab;
  g.sfix = (const uint32_t*)c->sfix.ptr;
  return g;
}

// Half-space reciprocal vectors with |K| <= Kc (Eq. 13, Eq. 20): h > 0, or h = 0 and
// k > 0, or h = k = 0 and l > 0; weights W = 2 (4 pi / V) exp(-K^2 / 4 g^2) / K^2,
// sorted by decreasing weight.
void kvector_table(const cpm_params& p, std::vector<int>& hkl, std::vector<double>& w) {
  const double lx = p.box[0], ly = p.box[1], lz = p.box[2];
  const double vol = lx * ly * lz;
  const double kc = 2.0 * p.g_ewald * sqrt(log(1.0 / p.kspace_eps));
  const int hmax = (int)floor(kc * lx / (2.0 * kPi));
  const int kmax = (int)floor(kc * ly / (2.0 * kPi));
  const int lmax = (int)floor(kc * lz / (2.0 * kPi));
  const double kc2 = kc * kc;
  hkl.clear();
  w.clear();
  for (int h = 0; h <= hmax; ++h)
    for (int k = -kmax; k <= kmax; ++k)
      for (int l = -lmax; l <= lmax; ++l) {
        if (!(h > 0 || (h == 0 && k > 0) || (h == 0 && k == 0 && l > 0))) continue;
        const double kx = 2.0 * kPi * h / lx, ky = 2.0 * kPi * k / ly, kz = 2.0 * kPi * l / lz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 > kc2) continue;
        hkl.push_back(h);
        hkl.push_back(k);
        hkl.push_back(l);
        w.push_back(2.0 * (4.0 * kPi / vol) * exp(-k2 / (4.0 * p.g_ewald * p.g_ewald)) / k2);
      }
  // heaviest weights first: the k-space accumulation handles the large terms first and
  // in higher precision (see the GEMM kernels)
  std::vector<size_t> order(w.size());
  for (size_t t = 0; t < order.size(); ++t) order[t] = t;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return w[a] > w[b]; });
  std::vector<int> hkl2(hkl.size());
  std::vector<double> w2(w.size());
  for (size_t t = 0; t < order.size(); ++t) {
    w2[t] = w[order[t]];
    for (int d = 0; d < 3; ++d) hkl2[3 * t + d] = hkl[3 * order[t] + d];
  }
  hkl.swap(hkl2);
  w.swap(w2);
}

// Host plan of the k-space sum, from the sorted k-vector weights w (mpad = their count
// rounded up to 64) and the precision alone: the head of leading k-steps summed in float-float or
// FP64, the flush mask of the SIMT builds, and the tensor-core tail's product regions,
// per-block scales and accumulation chunks.
struct KPlan {
  int heavy_steps = 0;  // leading 16-column k-steps of the head
  int kh = 0;           // k-vectors of the b^sol contraction kept in FP64
  int kb0 = 0, kb6 = 0, kb3 = 0, kb8 = 0, nkb = 0;  // tensor-core K-block regions
  std::vector<uint32_t> fmask;  // SIMT builds: k-steps after which float partials flush
  std::vector<uint32_t> cmask;  // tensor cores: K-blocks that end an accumulation chunk
  std::vector<int> kexp;        // tensor cores: per-K-block power-of-two scale
};

void plan_kspace(const std::vector<double>& w, int mpad, int precision, KPlan& pl) {
  const int m = (int)w.size();
  const bool f64 = precision == CPM_PREC_FP64;
  // Accumulation schedule of the float k-space GEMM.  k-step s covers 16 operand
  // columns: block s / 8 holds 64 k-vectors as [cos | sin], so its steps 0-3 and 4-7
  // carry the same weights.  Leading blocks whose steps carry more than 2e-3 of weight
  // are summed exactly in FP64; later float partials are flushed into FP64 once a chunk
  // has gathered about 1e-3 of weight or 32 steps.
  const int nk = 2 * mpad / 16;
  std::vector<uint32_t>& fmask = pl.fmask;
  fmask.assign((nk + 31) / 32, 0u);
  {
    std::vector<double> ws(nk, 0.0);
    for (int st = 0; st < nk; ++st) {
      const int k0 = 64 * (st / 8) + 16 * (st % 4);
      for (int t = 0; t < 16; ++t)
        if (k0 + t < m) ws[st] += w[k0 + t];
    }
    int heavy = 0;
    while (heavy < nk && ws[heavy] > 2e-3) ++heavy;
    heavy = std::min(std::min(nk, 128), (heavy + 7) / 8 * 8);  // at most 1024 k-vectors
    pl.heavy_steps = heavy;
    if (precision == CPM_PREC_BF16X6) {
      // the tensor-core build sums its six-product blocks in chunks of up to 5e-3 of
      // weight; only the steps heavier than that stay in the float-float head (16 of 56
      // steps at 12,800 atoms: the head kernel 30.7 -> 11.0 ms, E's off-diagonal RMS
      // error against FP64 4.9e-9 -> 6.2e-9 at 3,200 atoms)
      int h5 = 0;
      while (h5 < nk && ws[h5] > 5e-3) ++h5;
      pl.heavy_steps = std::min(heavy, (h5 + 7) / 8 * 8);
    }
    // head of the b^sol contraction kept in FP64: the heavy blocks, at least 256 and at
    // most 1024 k-vectors
    pl.kh = f64 ? 0 : std::min(mpad, std::max(256, std::min(1024, heavy / 8 * 64)));
    double cw = 0.0;
    int len = 0;
    for (int st = heavy; st < nk; ++st) {
      cw += ws[st];
      ++len;
      if (cw >= 1e-3 || len >= 32 || st == nk - 1) {
        fmask[st >> 5] |= 1u << (st & 31);
        cw = 0.0;
        len = 0;
      }
    }
  }

  // Tensor-core build: product schedule, per-block FP16 scales and accumulation chunks of
  // the 64-column K-blocks after the head (K-block b holds the cos or sin columns of
  // k-vectors 64 (b / 2) ..; a pair shares its weights).
  const int nkb = 2 * mpad / 64;
  std::vector<uint32_t>& cmask = pl.cmask;
  std::vector<int>& kexp = pl.kexp;
  cmask.assign((nkb + 31) / 32, 0u);
  kexp.assign(nkb, 0);
  pl.nkb = nkb;
  {
    // bwm[b]: 64 x the block's largest weight, which bounds the block's |a_i a_j| sums
    std::vector<double> bw(nkb, 0.0), bwm(nkb, 0.0);
    for (int b = 0; b < nkb; ++b)
      for (int t = 0; t < 64; ++t)
        if (64 * (b / 2) + t < m) {
          bw[b] += w[64 * (b / 2) + t];
          bwm[b] = std::max(bwm[b], 64.0 * w[64 * (b / 2) + t]);
        }
    // Product count (weights decrease along the table): trailing blocks whose summed
    // bound times the one-FP8 (E4M3) product error (2 x 2^-4 + 2^-8 + 3e-5, the last for
    // subnormals; bound 0.13) stays within 1e-8 take one FP8 product; the blocks before
    // them up to another 1e-8 at the one-FP16-product error (2^-10 + 2^-23) one FP16
    // product; the blocks before them up to another 1e-8 at the three-FP16-product error
    // (5 x 2^-22) three; the rest the six BF16 products (~2^-24).  All ends even: whole
    // [cos | sin] pairs per region, one more block with more products at most.
    const int kb0 = pl.heavy_steps / 4;
    const double budget = 1e-8;
    int kb8 = nkb;
    double tw = 0.0;
    while (kb8 > kb0 && (tw + bwm[kb8 - 1]) * 0.13 <= budget) tw += bwm[--kb8];
    kb8 = std::min(nkb, (kb8 + 1) & ~1);
    int kb3 = kb8;
    tw = 0.0;
    while (kb3 > kb0 && (tw + bwm[kb3 - 1]) * (0x1p-10 + 0x1p-23) <= budget) tw += bwm[--kb3];
    kb3 = std::min(kb8, (kb3 + 1) & ~1);
    int kb6 = kb3;
    tw = 0.0;
    while (kb6 > kb0 && (tw + bwm[kb6 - 1]) * 5 * 0x1p-22 <= budget) tw += bwm[--kb6];
    kb6 = std::min(kb3, (kb6 + 1) & ~1);
    pl.kb0 = kb0;
    pl.kb6 = kb6;
    pl.kb3 = kb3;
    pl.kb8 = kb8;
    // FP16 blocks: x = 2^e a with 2^e sqrt(max W) in [1/2, 1), so |x| < 1; FP8 blocks
    // 2^8 times that, [128, 256), inside E4M3's normal range (max 448)
    for (int b = kb6; b < nkb; ++b)
      if (bwm[b] > 0.0) kexp[b] = -ilogb(sqrt(bwm[b] / 64.0)) - 1 + (b >= kb8 ? 8 : 0);
    // Accumulation chunks.  Six-product blocks: up to 5e-3 of weight or 32 blocks (the
    // FP32 accumulation error of a chunk stays near 6e-8 x 5e-3 x sqrt(768 terms) ~ 1e-8;
    // measured: E unchanged at the 512-atom cell against 5e-4 / 8; at 3,200 atoms 2e-2 / 32
    // doubles the off-diagonal RMS error, 3.9e-9 -> 9.7e-9).  FP16 and FP8 blocks: one
    // scale per chunk (a chunk ends where the next block's scale differs, always after a
    // whole [cos | sin] pair), at most 512 blocks; their summed weight is below 1e-2.
    double cw = 0.0;
    int len = 0;
    for (int b = kb0; b < nkb; ++b) {
      cw += bw[b];
      ++len;
      const bool end = b == nkb - 1 || b + 1 == kb6 ||
                       (b < kb6 ? (cw >= 5e-3 || len >= 32)
                                : (kexp[b + 1] != kexp[b] || len >= 512));
      if (end) {
        cmask[b >> 5] |= 1u << (b & 31);
        cw = 0.0;
        len = 0;
      }
    }
  }
}

void release_workspace(Ctx* c) {
  Buf* ws[] = {&c->tc_planes[0], &c->tc_planes[1], &c->tc_planes[2], &c->tc_planes[3],
               &c->tc_head, &c->tc_err,
               &c->tc_hsplit, &c->tc_scratch, &c->dc_cnt, &c->dc_pcol, &c->dc_status, &c->ws_solve, &c->ws_in0, &c->ws_in1, &c->ws_in2,
               &c->ws_out0, &c->ws_out1, &c->ws_pot, &c->ws_guess, &c->ws_feat, &c->ws_cluster,
               &c->tc_tiles};
  for (Buf* b : ws) buf_free(c, b);
  c->tc_tiles_nt = 0;
}

void free_build(Ctx* c) {
  Buf* all[] = {&c->xyz, &c->alpha, &c->sfix, &c->hkl, &c->sqw, &c->flush, &c->chunk_end,
                &c->kexp,
                &c->Ahead, &c->A,
                &c->E, &c->diag,
                &c->nbr_off, &c->nbr_idx, &c->prow, &c->d, &c->shell_off, &c->shell_members, &c->p_f32,
                &c->turn, &c->gcd_labels, &c->gcd_a, &c->gcd_c, &c->gcd_cinv, &c->gcd_status,
                &c->gcd_scratch, &c->smat};
  for (Buf* b : all) buf_free(c, b);
  release_workspace(c);
  c->built = false;
  c->solve_only = false;
  c->shells_ready = false;
  c->gcd_m = 0;
  c->smat_ready = false;
  for (int b = 0; b < 8; ++b) {  // the solver's autotuner starts again with the next build
    c->tune_path[b] = 0;
    c->tune_cost[b][0] = c->tune_cost[b][1] = 0.f;
  }
}

__global__ void k_inverse_tail(double* diag, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) diag[n + i] = 1.0 / diag[i];
}

__global__ void k_fill(double* v, int64_t len, double x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = x;
}

// *bad = 1 when a coordinate is not finite or a width is neither positive and finite nor
// +INFINITY (a point charge); *bad starts at 0.
__global__ void k_check_geometry(const double* __restrict__ xyz, const double* __restrict__ alpha,
                                 int n, int* __restrict__ bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = alpha[i];
    if (!isfinite(xyz[3 * i]) || !isfinite(xyz[3 * i + 1]) || !isfinite(xyz[3 * i + 2]) ||
        !(a > 0.0) || isnan(a))
      *bad = 1;
  }
}

// dst [n][ld] (double) = src [n][ld] (float): exact widening of the stored matrix.
__global__ void k_widen(const float* __restrict__ src, double* __restrict__ dst, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

__global__ void k_scale(double* v, int64_t len, double s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= s;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace
}  // namespace cpm

using namespace cpm;

struct cpm_ctx : public cpm::Ctx {};

extern "C" {

void cpm_default_params(cpm_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->g_ewald = 0.3;
  p->rcut_real = 12.0;
  p->kspace_eps = 1e-8;
  p->slab = 1;
  p->precision = CPM_PREC_BF16X6;
  p->precond = CPM_PRECOND_DC;
  p->g_dc = 0.083;
  p->rcut_dc = 8.0;
  p->p_gap = 1;
}

static bool params_valid(const cpm_params* p) {
  if (!(p->box[0] > 0 && p->box[1] > 0 && p->box[2] > 0) || !(p->g_ewald > 0) ||
      !(p->rcut_real > 0) || !(p->kspace_eps > 0 && p->kspace_eps < 1))
    return false;
  if (p->precision != CPM_PREC_FP64 && p->precision != CPM_PREC_FP32 &&
      p->precision != CPM_PREC_BF16X6)
    return false;
  if (p->precond < CPM_PRECOND_NONE || p->precond > CPM_PRECOND_FULL) return false;
  if (p->stream_operand < 0 || p->stream_operand > 1 || p->k_window < 0) return false;
  if (p->matvec_mode < 0 || p->matvec_mode > 1) return false;
  if (p->solver_path < 0 || p->solver_path > 2) return false;
  if ((p->alloc == nullptr) != (p->free == nullptr)) return false;
  return true;
}

int cpm_create(cpm_ctx** out, const cpm_params* p) {
  if (!out || !p) return CPM_EINVAL;
  *out = nullptr;
  if (!params_valid(p)) return CPM_EINVAL;
  cpm_ctx* c = new (std::nothrow) cpm_ctx();
  if (!c) return CPM_ENOMEM;
  c->p = *p;
  c->stream = (cudaStream_t)p->stream;
  cudaEventCreate(&c->ev_tc[0]);
  cudaEventCreate(&c->ev_tc[1]);
  cudaEventCreate(&c->ev_tc[2]);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return CPM_ECUDA;
  }
  *out = c;
  return CPM_OK;
}

int cpm_destroy(cpm_ctx* c) {
  if (!c) return CPM_EINVAL;
  cudaStreamSynchronize(c->stream);
  free_build(c);
  cudaEventDestroy(c->ev_tc[0]);
  cudaEventDestroy(c->ev_tc[1]);
  cudaEventDestroy(c->ev_tc[2]);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_pot) cudaEventDestroy(e);
  delete c;
  return CPM_OK;
}

const char* cpm_last_error(const cpm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int cpm_plan_kspace(const cpm_params* p, cpm_kspace_plan* out, int* hkl, double* w,
                    int* kexp, uint8_t* chunk_end) {
  if (!p || !out || !params_valid(p)) return CPM_EINVAL;
  std::vector<int> h;
  std::vector<double> wt;
  cpm::kvector_table(*p, h, wt);
  const int m = (int)wt.size();
  const int mpad = (int)cpm::round_up(std::max(m, 1), 64);
  cpm::KPlan pl;
  cpm::plan_kspace(wt, mpad, p->precision, pl);
  out->m = m;
  out->m_pad = mpad;
  out->head_cols = 16 * pl.heavy_steps;
  out->kb_begin = pl.kb0;
  out->kb6_end = pl.kb6;
  out->kb3_end = pl.kb3;
  out->kb8_begin = pl.kb8;
  out->kb_end = pl.nkb;
  out->chunks = 0;
  for (int b = 0; b < pl.nkb; ++b) out->chunks += (pl.cmask[b >> 5] >> (b & 31)) & 1u;
  if (hkl) std::copy(h.begin(), h.end(), hkl);
  if (w) std::copy(wt.begin(), wt.end(), w);
  if (kexp) std::copy(pl.kexp.begin(), pl.kexp.end(), kexp);
  if (chunk_end)
    for (int b = 0; b < pl.nkb; ++b) chunk_end[b] = (uint8_t)((pl.cmask[b >> 5] >> (b & 31)) & 1u);
  return CPM_OK;
}

int cpm_release_workspace(cpm_ctx* c) {
  if (!c) return CPM_EINVAL;
  if (int st = cuda_check(c, cudaStreamSynchronize(c->stream), "release sync")) return st;
  release_workspace(c);
  return CPM_OK;
}

int cpm_build_E_copy(cpm_ctx* dst, cpm_ctx* src) {
  if (!dst || !src) return CPM_EINVAL;
  if (dst == src) return set_err(dst, CPM_EINVAL, "cpm_build_E_copy: dst and src are the same");
  if (!src->built) return set_err(dst, CPM_ENOTBUILT, "cpm_build_E_copy: src is not built");
  const cpm_params &pd = dst->p, &ps = src->p;
  if (dst->device != src->device || pd.box[0] != ps.box[0] || pd.box[1] != ps.box[1] ||
      pd.box[2] != ps.box[2] || pd.g_ewald != ps.g_ewald || pd.rcut_real != ps.rcut_real ||
      pd.kspace_eps != ps.kspace_eps || pd.slab != ps.slab)
    return set_err(dst, CPM_EINVAL, "cpm_build_E_copy: device, box or Ewald parameters differ");
  const bool copy_dc = pd.precond >= CPM_PRECOND_DC;  // PCG-DC, -Normal or -Full
  if (copy_dc && (ps.precond != pd.precond || pd.g_dc != ps.g_dc ||
                  pd.rcut_dc != ps.rcut_dc || pd.p_gap != ps.p_gap))
    return set_err(dst, CPM_EINVAL, "cpm_build_E_copy: a sparse preconditioner is copied "
                                    "from a src with the same one (g_dc, rcut_dc, p_gap)");
  if (!dst->fp64() && src->fp64())
    return set_err(dst, CPM_EINVAL, "cpm_build_E_copy: FP64 E cannot be narrowed");
  int st;
  if ((st = cuda_check(src, cudaStreamSynchronize(src->stream), "copy src sync"))) return st;
  free_build(dst);
  const int n = src->n;
  cudaStream_t s = dst->stream;
  dst->n = n;
  dst->npad = src->npad;
  dst->ldE = src->ldE;
  dst->vol = src->vol;
  dst->m = src->m;
  dst->mpad = src->mpad;
  dst->c_ele = src->c_ele;
  dst->d_iters = src->d_iters;
  const int64_t len = (int64_t)n * src->ldE;
  const size_t nb = (size_t)n * sizeof(double);
  if ((st = buf_alloc(dst, &dst->xyz, 3 * nb)) || (st = buf_alloc(dst, &dst->alpha, nb)) ||
      (st = buf_alloc(dst, &dst->E, (size_t)len * dst->esz())) ||
      (st = buf_alloc(dst, &dst->diag, 2 * nb)) || (st = buf_alloc(dst, &dst->d, nb))) {
    free_build(dst);
    return st;
  }
  const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
  st = cuda_check(dst, cudaMemcpyAsync(dst->xyz.ptr, src->xyz.ptr, 3 * nb, d2d, s), "xyz");
  if (!st) st = cuda_check(dst, cudaMemcpyAsync(dst->alpha.ptr, src->alpha.ptr, nb, d2d, s), "alpha");
  if (!st) st = cuda_check(dst, cudaMemcpyAsync(dst->diag.ptr, src->diag.ptr, 2 * nb, d2d, s), "diag");
  if (!st) st = cuda_check(dst, cudaMemcpyAsync(dst->d.ptr, src->d.ptr, nb, d2d, s), "d");
  if (!st) {
    if (dst->esz() == src->esz())
      st = cuda_check(dst, cudaMemcpyAsync(dst->E.ptr, src->E.ptr, (size_t)len * dst->esz(), d2d,
                                           s), "E");
    else
      (k_widen<<<4 * 152, 256, 0, s>>>((const float*)src->E.ptr, (double*)dst->E.ptr, len),
       note_launch());
  }
  if (!st && copy_dc) {
    dst->nnz = src->nnz;
    dst->pgap = src->pgap;
    const size_t ob = (size_t)(n + 1) * sizeof(int64_t);
    if ((st = buf_alloc(dst, &dst->nbr_off, ob)) ||
        (st = buf_alloc(dst, &dst->nbr_idx, (size_t)src->nnz * sizeof(int))) ||
        (st = buf_alloc(dst, &dst->prow, (size_t)src->nnz * sizeof(double)))) {
      free_build(dst);
      return st;
    }
    st = cuda_check(dst, cudaMemcpyAsync(dst->nbr_off.ptr, src->nbr_off.ptr, ob, d2d, s), "P");
    if (!st) st = cuda_check(dst, cudaMemcpyAsync(dst->nbr_idx.ptr, src->nbr_idx.ptr,
                                                  (size_t)src->nnz * sizeof(int), d2d, s), "P");
    if (!st) st = cuda_check(dst, cudaMemcpyAsync(dst->prow.ptr, src->prow.ptr,
                                                  (size_t)src->nnz * sizeof(double), d2d, s), "P");
  }
  if (!st) st = cuda_check(dst, cudaGetLastError(), "copy build");
  if (!st) st = cuda_check(dst, cudaStreamSynchronize(s), "copy build sync");
  if (st) {
    free_build(dst);
    return st;
  }
  dst->solve_only = true;
  dst->built = true;
  return CPM_OK;
}

int cpm_build_E(cpm_ctx* c, int n, const double* xyz, const double* alpha) {
  if (!c) return CPM_EINVAL;
  c->solve_only = false;
  for (int b = 0; b < 8; ++b) {  // the solver's autotuner starts again for this electrode
    c->tune_path[b] = 0;
    c->tune_cost[b][0] = c->tune_cost[b][1] = 0.f;
  }
  if (n < 1 || !xyz || !alpha) return set_err(c, CPM_EINVAL, "cpm_build_E: n >= 1 and arrays required");
  // buffers of the previous build are reused where large enough (reserve), not freed
  c->built = false;
  c->shells_ready = false;
  c->gcd_m = 0;  // the electrodes' solves and S belong to the previous E
  c->smat_ready = false;
  cudaStream_t s = c->stream;
  const bool f64 = c->fp64();
  int st;
  c->n = n;
  // rows of the operand: whole 256-row blocks for the tensor-core tail's CTA pairs
  c->npad = (int)round_up(n, c->p.precision == CPM_PREC_BF16X6 ? 256 : 128);
  c->ldE = round_up(n, 128);
  c->vol = c->p.box[0] * c->p.box[1] * c->p.box[2];
  // the k-vector table depends on the box, g and eps only: made once per context
  if (c->kv_w.empty()) kvector_table(c->p, c->kv_hkl, c->kv_w);
  std::vector<int> hkl = c->kv_hkl;
  const std::vector<double>& w = c->kv_w;
  c->m = (int)w.size();
  c->mpad = (int)round_up(std::max(c->m, 1), 64);
  hkl.resize(3 * (size_t)c->mpad, 0);
  std::vector<double> sqw(c->mpad, 0.0);
  for (int k = 0; k < c->m; ++k) sqw[k] = sqrt(w[k]);
  c->kw.assign(c->mpad, 0.0);
  std::copy(w.begin(), w.end(), c->kw.begin());
  KPlan pl;
  plan_kspace(w, c->mpad, c->p.precision, pl);
  c->heavy_steps = pl.heavy_steps;
  c->kh = pl.kh;
  c->kb6_end = pl.kb6;
  c->kb3_end = pl.kb3;
  c->kb8_begin = pl.kb8;
  const bool tc = c->p.precision == CPM_PREC_BF16X6;
  const std::vector<uint32_t>& fmask = pl.fmask;
  const std::vector<uint32_t>& cmask = pl.cmask;
  const std::vector<int>& kexp = pl.kexp;

  const size_t a_bytes = (size_t)c->npad * 2 * c->mpad * c->esz();
  // A larger than this is not kept: the tensor-core build streams it in k-windows and the
  // potential sums its k-space part directly (a streamed build)
  constexpr size_t kResidentOperandBytes = 32ull << 30;
  c->streamed = tc && (c->p.stream_operand == 1 || a_bytes > kResidentOperandBytes);
  const size_t e_bytes = (size_t)n * c->ldE * c->esz();
  if (c->streamed) buf_free(c, &c->A);
  if ((st = buf_reserve(c, &c->xyz, (size_t)n * 3 * sizeof(double))) ||
      (st = buf_reserve(c, &c->alpha, (size_t)n * sizeof(double))) ||
      (st = buf_reserve(c, &c->sfix, (size_t)c->npad * 3 * sizeof(uint32_t))) ||
      (st = buf_reserve(c, &c->hkl, hkl.size() * sizeof(int))) ||
      (st = buf_reserve(c, &c->sqw, sqw.size() * sizeof(double))) ||
      (st = buf_reserve(c, &c->flush, fmask.size() * sizeof(uint32_t))) ||
      (st = buf_reserve(c, &c->chunk_end, cmask.size() * sizeof(uint32_t))) ||
      (st = buf_reserve(c, &c->kexp, kexp.size() * sizeof(int))) ||
      (st = buf_reserve(c, &c->Ahead, (size_t)c->npad * 2 * std::max(c->kh, 1) * sizeof(double))) ||
      (!c->streamed && (st = buf_reserve(c, &c->A, a_bytes))) ||
      (st = buf_reserve(c, &c->E, e_bytes)) ||
      (st = buf_reserve(c, &c->diag, 2 * (size_t)n * sizeof(double))) ||
      (st = buf_reserve(c, &c->d, (size_t)n * sizeof(double)))) {
    free_build(c);
    return st;
  }
  auto fail = [&](int code) {
    free_build(c);
    return code;
  };
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
  const cudaMemcpyKind any = cudaMemcpyDefault;
  if ((st = cuda_check(c, cudaMemcpyAsync(c->xyz.ptr, xyz, (size_t)n * 3 * sizeof(double), any, s), "xyz")) ||
      (st = cuda_check(c, cudaMemcpyAsync(c->alpha.ptr, alpha, (size_t)n * sizeof(double), any, s), "alpha")) ||
      (st = cuda_check(c, cudaMemcpyAsync(c->hkl.ptr, hkl.data(), hkl.size() * sizeof(int), h2d, s), "hkl")) ||
      (st = cuda_check(c, cudaMemcpyAsync(c->sqw.ptr, sqw.data(), sqw.size() * sizeof(double), h2d, s), "sqw")) ||
      (st = cuda_check(c, cudaMemcpyAsync(c->flush.ptr, fmask.data(), fmask.size() * sizeof(uint32_t), h2d, s), "flush")) ||
      (st = cuda_check(c, cudaMemcpyAsync(c->chunk_end.ptr, cmask.data(), cmask.size() * sizeof(uint32_t), h2d, s), "chunks")) ||
      (st = cuda_check(c, cudaMemcpyAsync(c->kexp.ptr, kexp.data(), kexp.size() * sizeof(int), h2d, s), "scales")) ||
      (st = cuda_check(c, cudaMemsetAsync(c->E.ptr, 0, e_bytes, s), "E memset")) ||
      (st = cuda_check(c, cudaStreamSynchronize(s), "build upload")))
    return fail(st);
  {  // the geometry is checked before any kernel uses it (the diagonal buffer is free yet)
    int bad = 0;
    int* dbad = (int*)c->diag.ptr;
    if ((st = cuda_check(c, cudaMemsetAsync(dbad, 0, sizeof(int), s), "check flag"))) return fail(st);
    (k_check_geometry<<<std::min((n + 255) / 256, 1024), 256, 0, s>>>(
         (const double*)c->xyz.ptr, (const double*)c->alpha.ptr, n, dbad), note_launch());
    if ((st = cuda_check(c, cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s),
                         "check flag")) ||
        (st = cuda_check(c, cudaStreamSynchronize(s), "check sync")))
      return fail(st);
    if (bad)
      return fail(set_err(c, CPM_EINVAL, "cpm_build_E: a coordinate is not finite or a width "
                                         "is not positive (INFINITY marks a point charge)"));
  }

  cudaEvent_t ev[6];
  for (auto& e : ev) cudaEventCreate(&e);
  const Geometry geo = geometry(c);
  cudaEventRecord(ev[0], s);
  launch_fixed_point_coords((const double*)c->xyz.ptr, n, c->npad, c->p.box,
                            (uint32_t*)c->sfix.ptr, s);
  // the tensor-core workspace stays with the context for the next build (released by
  // cpm_release_workspace or cpm_destroy, and on a failed build)
  Buf* planes = c->tc_planes;
  Buf &ehead = c->tc_head, &errbuf = c->tc_err, &hsplit = c->tc_hsplit,
      &tcscratch = c->tc_scratch;
  auto fail_tc = [&]() { release_workspace(c); };
  const int head_cols = 16 * c->heavy_steps;
  // k-vectors whose BF16 planes are held at once: all of them, or in a streamed build a
  // window of ~12 GB of planes (12 bytes per row and k-vector)
  // window of planes sized to the device: half of the memory left free once the head
  // matrix is in place, between 12 and 64 GiB (14 bytes a row and k-vector: three BF16
  // planes and the FP8 one, cos and sin).  Each window costs one pass of every tile's
  // epilogue and of the head matrix, so fewer, larger windows are cheaper.  The first
  // streamed build of a geometry fixes the window, so that rebuilds repeat it exactly.
  int kwin = c->mpad;
  if (c->streamed) {
    if (c->p.k_window > 0) {
      kwin = std::max(64, std::min(c->mpad, c->p.k_window / 64 * 64));
    } else if (c->kwin_n == n && c->kwin_mpad == c->mpad && c->kwin > 0) {
      kwin = c->kwin;
    } else {
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      const int64_t head_b = c->tc_head.bytes >= (size_t)n * c->ldE * sizeof(double)
                                 ? 0 : (int64_t)n * c->ldE * (int64_t)sizeof(double);
      const int64_t held = (int64_t)c->tc_planes[0].bytes * 3 + (int64_t)c->tc_planes[3].bytes;
      int64_t budget = ((int64_t)fr - head_b + held) / 2;
      budget = std::max<int64_t>(12ll << 30, std::min<int64_t>(64ll << 30, budget));
      kwin = std::max(64, (int)std::min<int64_t>(c->mpad, budget / (14ll * c->npad) / 64 * 64));
      const int windows = (c->mpad + kwin - 1) / kwin;  // equal windows, none a sliver
      kwin = std::min(kwin, ((c->mpad + windows - 1) / windows + 63) / 64 * 64);
      c->kwin = kwin;
      c->kwin_n = n;
      c->kwin_mpad = c->mpad;
    }
  }
  if (tc) {
    const size_t pbytes = (size_t)c->npad * 2 * kwin * 2;
    if ((st = buf_reserve(c, &planes[0], pbytes)) || (st = buf_reserve(c, &planes[1], pbytes)) ||
        (st = buf_reserve(c, &planes[2], pbytes)) || (st = buf_reserve(c, &planes[3], pbytes / 2)) ||
        (st = buf_reserve(c, &ehead, (size_t)n * c->ldE * sizeof(double))) ||
        (st = buf_reserve(c, &errbuf, sizeof(int))) ||
        (c->nsmid == 0 &&
         (launch_nsmid((int*)errbuf.ptr, s),
          (st = cuda_check(c, cudaMemcpyAsync(&c->nsmid, errbuf.ptr, sizeof(int),
                                              cudaMemcpyDeviceToHost, s), "nsmid")) ||
              (st = cuda_check(c, cudaStreamSynchronize(s), "nsmid sync")) ||
              (c->nsmid = std::max(1, std::min(c->nsmid, 4096)), false))) ||
        (st = buf_reserve(c, &tcscratch, (size_t)c->nsmid * ek_strip_scratch_floats() * sizeof(float))) ||
        (st = buf_reserve(c, &hsplit, 2 * (size_t)c->npad * std::max(head_cols, 16) * sizeof(float))) ||
        (st = cuda_check(c, cudaMemsetAsync(errbuf.ptr, 0, sizeof(int), s), "err flag"))) {
      fail_tc();
      for (auto& e : ev) cudaEventDestroy(e);
      return fail(st);
    }
  }
  // A (and, for the tensor-core build, its BF16 planes where the schedule reads them);
  // a streamed build makes the planes window by window below.  The float operand's
  // phases come from the 4,096-entry phasor table (made once per context)
  if (!f64 && !c->turn.ptr) {
    if ((st = buf_alloc(c, &c->turn, 4096 * 4 * sizeof(float)))) {
      fail_tc();
      for (auto& e : ev) cudaEventDestroy(e);
      return fail(st);
    }
    launch_turn_table(c->turn.ptr, s);
  }
  void* plane_ptrs[4] = {planes[0].ptr, planes[1].ptr, planes[2].ptr, planes[3].ptr};
  if (!c->streamed)
    launch_structure_operand(f64, (const double*)c->xyz.ptr, (const uint32_t*)c->sfix.ptr,
                             c->npad, n, (const int*)c->hkl.ptr, (const double*)c->sqw.ptr,
                             c->mpad, c->p.box, c->A.ptr, tc ? plane_ptrs : nullptr,
                             c->heavy_steps / 4, c->kb6_end, c->kb3_end, c->kb8_begin,
                             (const int*)c->kexp.ptr, c->turn.ptr, 0, c->mpad, s);
  if (c->kh > 0)
    launch_structure_operand_head((const double*)c->xyz.ptr, c->npad, n, (const int*)c->hkl.ptr,
                                  (const double*)c->sqw.ptr, c->kh, c->p.box,
                                  (double*)c->Ahead.ptr, s);
  cudaEventRecord(ev[1], s);
  if (tc) {
    // head (heaviest k-vectors, float-float) with the real-space, self and dipole terms in
    // FP64, kept as float pairs; then the tensor-core tail, which adds the head in its
    // epilogue
    cudaEvent_t ev_head;
    cudaEventCreate(&ev_head);
    cudaEventRecord(ev_head, s);
    float* hhi = (float*)hsplit.ptr;
    st = launch_ek_head_f64((const double*)c->Ahead.ptr, c->kh, head_cols, c->npad, hhi,
                            hhi + (size_t)c->npad * std::max(head_cols, 16),
                            (const double*)c->xyz.ptr, (const double*)c->alpha.ptr, n, geo,
                            (float2*)ehead.ptr, c->ldE, s);
    // the tile order of the tensor-core launches (kept with the context per row-block count)
    const int nt = (n + 255) / 256;
    if (!st && c->tc_tiles_nt != nt) {
      const std::vector<uint32_t> order = ek_tile_order(nt);
      if (!(st = buf_reserve(c, &c->tc_tiles, order.size() * sizeof(uint32_t))))
        st = cuda_check(c, cudaMemcpyAsync(c->tc_tiles.ptr, order.data(),
                                           order.size() * sizeof(uint32_t),
                                           cudaMemcpyHostToDevice, s), "tile order");
      if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "tile order sync");
      c->tc_tiles_nt = st ? 0 : nt;
    }
    cudaEventRecord(c->ev_tc[0], s);
    // the tail, one k-window at a time: every window but the last carries the sum in the
    // head matrix (float pairs), the last writes float E.  A streamed build times the
    // tensor-core launches of every window apart from the operand planes made between them.
    std::vector<cudaEvent_t> wev;
    for (int kbeg = 0; kbeg < c->mpad && !st; kbeg += kwin) {
      const int kend = std::min(c->mpad, kbeg + kwin);
      const bool last = kend == c->mpad;
      if (c->streamed) {
        launch_structure_operand(false, (const double*)c->xyz.ptr, (const uint32_t*)c->sfix.ptr,
                                 c->npad, n, (const int*)c->hkl.ptr, (const double*)c->sqw.ptr,
                                 c->mpad, c->p.box, nullptr, plane_ptrs, c->heavy_steps / 4,
                                 c->kb6_end, c->kb3_end, c->kb8_begin, (const int*)c->kexp.ptr,
                                 c->turn.ptr, kbeg, kend, s);
        wev.resize(wev.size() + 2);
        cudaEventCreate(&wev[wev.size() - 2]);
        cudaEventCreate(&wev[wev.size() - 1]);
        cudaEventRecord(wev[wev.size() - 2], s);
      }
      st = launch_ek_tc(planes[0].ptr, planes[1].ptr, planes[2].ptr, planes[3].ptr, c->npad,
                        2 * (int64_t)(kend - kbeg), kbeg / 32, n,
                        std::max(c->heavy_steps / 4, kbeg / 32), kend / 32, c->kb6_end,
                        c->kb3_end, c->kb8_begin, (const uint32_t*)c->chunk_end.ptr,
                        (const int*)c->kexp.ptr,
                        (float2*)ehead.ptr,
                        c->ldE, last ? (float*)c->E.ptr : nullptr, c->ldE, (int*)errbuf.ptr,
                        c->kw.data(), (float*)tcscratch.ptr, c->nsmid,
                        (const uint32_t*)c->tc_tiles.ptr,
                        c->streamed ? nullptr : c->ev_tc[2], s);
      if (c->streamed) cudaEventRecord(wev.back(), s);
    }
    cudaEventRecord(c->ev_tc[1], s);
    int herr = 0;
    if (!st) st = cuda_check(c, cudaMemcpyAsync(&herr, errbuf.ptr, sizeof(int),
                                                cudaMemcpyDeviceToHost, s), "tc err");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "tc sync");
    if (!st && herr) st = set_err(c, CPM_ECUDA, "tensor-core k-space kernel: a pipeline wait timed out");
    if (!st) cudaEventElapsedTime(&c->t_tc_ms, c->ev_tc[0], c->ev_tc[1]);
    c->t_tc_loop_ms = c->t_tc_ms;
    if (!st && c->streamed) {  // the tensor-core launches alone
      c->t_tc_ms = 0;
      for (size_t w = 0; w + 1 < wev.size(); w += 2) {
        float ms = 0;
        cudaEventElapsedTime(&ms, wev[w], wev[w + 1]);
        c->t_tc_ms += ms;
      }
    }
    for (auto& e : wev) cudaEventDestroy(e);
    if (!st) cudaEventElapsedTime(&c->t_head_ms, ev_head, c->ev_tc[0]);
    c->t_light_ms = 0;
    if (!st && !c->streamed) cudaEventElapsedTime(&c->t_light_ms, c->ev_tc[2], c->ev_tc[1]);
    cudaEventDestroy(ev_head);
    if (st) fail_tc();
  } else {
    st = launch_ek_simt(f64, c->A.ptr, c->npad, c->mpad, (const double*)c->xyz.ptr,
                        (const double*)c->alpha.ptr, n, geo, c->E.ptr, c->ldE, c->heavy_steps,
                        (const uint32_t*)c->flush.ptr, s);
  }
  if (st) {
    for (auto& e : ev) cudaEventDestroy(e);
    return fail(st == CPM_ECUDA && c->err.empty() ? cuda_check(c, cudaGetLastError(), "k-space GEMM") : st);
  }
  cudaEventRecord(ev[2], s);
  launch_mirror_lower(f64, c->E.ptr, n, c->ldE, s);
  launch_extract_diag(f64, c->E.ptr, n, c->ldE, (double*)c->diag.ptr, s);
  (k_inverse_tail<<<(n + 255) / 256, 256, 0, s>>>((double*)c->diag.ptr, n), note_launch());
  if ((st = cuda_check(c, cudaGetLastError(), "E build")) ||
      (st = cuda_check(c, cudaStreamSynchronize(s), "E build sync"))) {
    for (auto& e : ev) cudaEventDestroy(e);
    return fail(st);
  }
  c->built = true;  // E is usable from here on (the solves below need it)

  cudaEventRecord(ev[3], s);
  if (c->p.precond == CPM_PRECOND_NORMAL || c->p.precond == CPM_PRECOND_FULL) {
    if ((st = build_sparse_inverse(c))) {
      for (auto& e : ev) cudaEventDestroy(e);
      return fail(st);
    }
  } else if (c->p.precond == CPM_PRECOND_DC) {
    if ((st = build_dc_preconditioner(c))) {
      for (auto& e : ev) cudaEventDestroy(e);
      return fail(st);
    }
  }
  cudaEventRecord(ev[4], s);
  // d' from E_n d' = 1 (Eq. S9), then d = d' / (1^T d') (Eq. S8)
  {
    double* ones = (double*)c->d.ptr;
    (k_fill<<<64, 256, 0, s>>>(ones, n, 1.0), note_launch());
    Buf dp;
    if ((st = buf_alloc(c, &dp, (size_t)n * sizeof(double)))) {
      for (auto& e : ev) cudaEventDestroy(e);
      return fail(st);
    }
    int it = 0;
    double rr = 0;
    SolveArgs a{1, ones, 1.0, (double*)dp.ptr, false, 1e-10, 20000, &it, &rr};
    const double saved_gap = c->pgap;
    c->pgap = 0.0;
    st = pcg_solve(c, a);
    c->pgap = saved_gap;
    c->d_iters = it;
    double csum = 0.0;
    if (!st) st = device_sum(c, (const double*)dp.ptr, n, &csum);
    if (!st) {
      c->c_ele = csum;
      st = cuda_check(c, cudaMemcpyAsync(c->d.ptr, dp.ptr, (size_t)n * sizeof(double),
                                         cudaMemcpyDeviceToDevice, s), "d copy");
      (k_scale<<<64, 256, 0, s>>>((double*)c->d.ptr, n, 1.0 / csum), note_launch());
    }
    if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "d sync");
    buf_free(c, &dp);
    if (st) {
      for (auto& e : ev) cudaEventDestroy(e);
      return fail(st);
    }
  }
  cudaEventRecord(ev[5], s);
  if (c->p.precond == CPM_PRECOND_DC && c->p.p_gap) {
    if ((st = apply_p_gap(c))) {
      for (auto& e : ev) cudaEventDestroy(e);
      return fail(st);
    }
  }
  cudaEventSynchronize(ev[5]);
  cudaEventElapsedTime(&c->t_phase_ms, ev[0], ev[1]);
  cudaEventElapsedTime(&c->t_kspace_ms, ev[1], ev[2]);
  cudaEventElapsedTime(&c->t_precond_ms, ev[3], ev[4]);
  cudaEventElapsedTime(&c->t_dsolve_ms, ev[4], ev[5]);
  for (auto& e : ev) cudaEventDestroy(e);
  return cuda_check(c, cudaStreamSynchronize(s), "build end");
}

int cpm_potential(cpm_ctx* c, int frames, int n_ion, const double* ion_xyz,
                  const double* ion_q, const double* chi, double* b_out, double* qsol_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_potential before cpm_build_E");
  if (c->solve_only)
    return set_err(c, CPM_EINVAL, "cpm_potential: a context built by cpm_build_E_copy has no "
                                  "k-space tables; compute b on the source context");
  if (frames < 1 || n_ion < 0 || !chi || !b_out || (n_ion > 0 && (!ion_xyz || !ion_q)))
    return set_err(c, CPM_EINVAL, "cpm_potential: bad arguments");
  const int n = c->n;
  cudaStream_t s = c->stream;
  const bool f64 = c->fp64();
  const double *dx = nullptr, *dq = nullptr, *dchi = nullptr;
  static const double zero = 0.0;
  int st;
  if (n_ion > 0) {
    if ((st = stage_in(c, &c->ws_in0, ion_xyz, (size_t)frames * n_ion * 3 * sizeof(double),
                       (const void**)&dx)) ||
        (st = stage_in(c, &c->ws_in1, ion_q, (size_t)frames * n_ion * sizeof(double),
                       (const void**)&dq)))
      return st;
  } else {
    dx = dq = &zero;  // never read
  }
  if ((st = stage_in(c, &c->ws_in2, chi, (size_t)n * sizeof(double), (const void**)&dchi)))
    return st;
  double *db = nullptr, *dqs = nullptr;
  if ((st = stage_out(c, &c->ws_out0, b_out, (size_t)frames * n * sizeof(double), (void**)&db)))
    return st;
  if (qsol_out && (st = stage_out(c, &c->ws_out1, qsol_out, (size_t)frames * sizeof(double),
                                  (void**)&dqs)))
    return st;
  // scratch: v [frames][2 mpad] (storage type) | v_head [frames][2 kh] | b^sol_k [frames][n]
  //          | fixed-point ion coordinates [frames][n_ion][3] | the direct sum's k-range
  //          shares [nsplit][frames][n] (a streamed build split into more than one)
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t vbytes = up((size_t)frames * 2 * c->mpad * c->esz());
  const size_t hbytes = up((size_t)frames * 2 * std::max(c->kh, 1) * sizeof(double));
  const size_t kbytes = up((size_t)frames * n * sizeof(double));
  const size_t ubytes = up((size_t)frames * std::max(n_ion, 1) * 3 * sizeof(uint32_t));
  int dev_sms = 1;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
  const int nsplit = !c->A.ptr && !f64
                         ? bsol_direct_splits(n, frames, c->mpad, c->kh, std::max(dev_sms, 1))
                         : 1;
  const size_t sbytes = nsplit > 1 ? (size_t)nsplit * kbytes : 0;
  if ((st = buf_reserve(c, &c->ws_pot, vbytes + hbytes + kbytes + ubytes + sbytes))) return st;
  if (!f64 && !c->turn.ptr) {
    if ((st = buf_alloc(c, &c->turn, 4096 * 4 * sizeof(float)))) return st;
    launch_turn_table(c->turn.ptr, s);
  }
  void* v = c->ws_pot.ptr;
  double* vh = (double*)((char*)c->ws_pot.ptr + vbytes);
  double* bk = (double*)((char*)c->ws_pot.ptr + vbytes + hbytes);
  uint32_t* sion = (uint32_t*)((char*)c->ws_pot.ptr + vbytes + hbytes + kbytes);
  double* spart =
      nsplit > 1 ? (double*)((char*)c->ws_pot.ptr + vbytes + hbytes + kbytes + ubytes) : nullptr;
  cudaEvent_t pev[4];
  for (int e = 0; e < 4; ++e) {
    while (c->ev_pot.size() < 4) {
      cudaEvent_t x;
      cudaEventCreate(&x);
      c->ev_pot.push_back(x);
    }
    pev[e] = c->ev_pot[e];
  }
  cudaEventRecord(pev[0], s);
  if (n_ion > 0) {
    launch_ion_fixed(dx, frames, n_ion, c->p.box, sion, s);
    launch_ion_structure_factor(f64, dx, sion, dq, frames, n_ion, (const int*)c->hkl.ptr,
                                (const double*)c->sqw.ptr, c->mpad, c->kh, c->p.box,
                                c->turn.ptr, v, vh, s);
  } else if ((st = cuda_check(c, cudaMemsetAsync(v, 0, vbytes + hbytes, s), "v zero"))) {
    return st;
  }
  cudaEventRecord(pev[1], s);
  launch_bsol_kspace(f64, c->A.ptr, (const double*)c->Ahead.ptr, n, c->mpad, c->kh, v, vh,
                     frames, bk, (const uint32_t*)c->sfix.ptr, (const int*)c->hkl.ptr,
                     (const double*)c->sqw.ptr, c->turn.ptr, nsplit, spart, s);
  cudaEventRecord(pev[2], s);
  launch_bsol_real_and_finish((const double*)c->xyz.ptr, (const double*)c->alpha.ptr,
                              (const uint32_t*)c->sfix.ptr, n, dx, dq, sion, frames, n_ion,
                              geometry(c), dchi, bk, db, dqs,
                              c->p.precision != CPM_PREC_FP64, s);
  cudaEventRecord(pev[3], s);
  if ((st = cuda_check(c, cudaGetLastError(), "potential kernels"))) return st;
  if (qsol_out && n_ion == 0 &&
      (st = cuda_check(c, cudaMemsetAsync(dqs, 0, frames * sizeof(double), s), "qsol zero")))
    return st;
  if ((st = copy_out(c, b_out, db, (size_t)frames * n * sizeof(double)))) return st;
  if (qsol_out && (st = copy_out(c, qsol_out, dqs, (size_t)frames * sizeof(double)))) return st;
  if ((st = cuda_check(c, cudaStreamSynchronize(s), "potential sync"))) return st;
  cudaEventElapsedTime(&c->t_pot_sf_ms, pev[0], pev[1]);
  cudaEventElapsedTime(&c->t_pot_kspace_ms, pev[1], pev[2]);
  cudaEventElapsedTime(&c->t_pot_real_ms, pev[2], pev[3]);
  return CPM_OK;
}

int cpm_ion_forces(cpm_ctx* c, int frames, int n_ion, const double* ion_xyz,
                   const double* ion_q, const double* q, double* f_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_ion_forces before cpm_build_E");
  if (c->solve_only)
    return set_err(c, CPM_EINVAL, "cpm_ion_forces: a context built by cpm_build_E_copy");
  if (frames < 1 || n_ion < 1 || !ion_xyz || !ion_q || !q || !f_out)
    return set_err(c, CPM_EINVAL, "cpm_ion_forces: bad arguments");
  const int n = c->n;
  cudaStream_t s = c->stream;
  const bool f64 = c->fp64();
  const double *dx = nullptr, *dq = nullptr, *dqe = nullptr;
  double* dout = nullptr;
  int st;
  if ((st = stage_in(c, &c->ws_in0, ion_xyz, (size_t)frames * n_ion * 3 * sizeof(double),
                     (const void**)&dx)) ||
      (st = stage_in(c, &c->ws_in1, ion_q, (size_t)frames * n_ion * sizeof(double),
                     (const void**)&dq)) ||
      (st = stage_in(c, &c->ws_in2, q, (size_t)frames * n * sizeof(double), (const void**)&dqe)) ||
      (st = stage_out(c, &c->ws_out0, f_out, (size_t)frames * n_ion * 3 * sizeof(double),
                      (void**)&dout)))
    return st;
  // scratch: structure factors v [frames][2 mpad] (storage type) | v_head [frames][2 kh] |
  //          fixed-point ion coordinates [frames][n_ion][3] | k-space gradients [frames][n_ion][3]
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const int kh = f64 ? c->mpad : c->kh;  // FP64 storage: every k-vector in FP64
  const size_t vbytes = up((size_t)frames * 2 * c->mpad * c->esz());
  const size_t hbytes = up((size_t)frames * 2 * std::max(c->kh, 1) * sizeof(double));
  const size_t ubytes = up((size_t)frames * n_ion * 3 * sizeof(uint32_t));
  const size_t gbytes = up((size_t)frames * n_ion * 3 * sizeof(double));
  if ((st = buf_reserve(c, &c->ws_pot, vbytes + hbytes + ubytes + gbytes))) return st;
  if (!f64 && !c->turn.ptr) {
    if ((st = buf_alloc(c, &c->turn, 4096 * 4 * sizeof(float)))) return st;
    launch_turn_table(c->turn.ptr, s);
  }
  char* base = (char*)c->ws_pot.ptr;
  void* v = base;
  double* vh = (double*)(base + vbytes);
  uint32_t* sion = (uint32_t*)(base + vbytes + hbytes);
  double* grad = (double*)(base + vbytes + hbytes + ubytes);
  launch_ion_fixed(dx, frames, n_ion, c->p.box, sion, s);
  // the electrode's charge-weighted structure factors, frame by frame: the ions' kernel
  // run over the electrode atoms (same coordinates every frame)
  for (int f = 0; f < frames; ++f)
    launch_ion_structure_factor(f64, (const double*)c->xyz.ptr, (const uint32_t*)c->sfix.ptr,
                                dqe + (size_t)f * n, 1, n, (const int*)c->hkl.ptr,
                                (const double*)c->sqw.ptr, c->mpad, c->kh, c->p.box,
                                c->turn.ptr, (char*)v + (size_t)f * 2 * c->mpad * c->esz(),
                                vh + (size_t)f * 2 * std::max(c->kh, 1), s);
  launch_ion_forces((const double*)c->xyz.ptr, (const double*)c->alpha.ptr,
                    (const uint32_t*)c->sfix.ptr, n, dx, dq, sion, frames, n_ion, dqe,
                    (const int*)c->hkl.ptr, (const double*)c->sqw.ptr, c->mpad, kh, geometry(c),
                    c->turn.ptr, (const float*)v, f64 ? (const double*)v : vh, grad, dout, s);
  if ((st = cuda_check(c, cudaGetLastError(), "ion forces"))) return st;
  if ((st = copy_out(c, f_out, dout, (size_t)frames * n_ion * 3 * sizeof(double)))) return st;
  return cuda_check(c, cudaStreamSynchronize(s), "ion forces sync");
}

int cpm_solve(cpm_ctx* c, int nrhs, const double* b, double* q_inout, int use_guess,
              double tol, int maxit, int* iters_out, double* relres_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_solve before cpm_build_E");
  if (nrhs < 1 || !b || !q_inout || !(tol > 0) || maxit < 1)
    return set_err(c, CPM_EINVAL, "cpm_solve: bad arguments");
  const int n = c->n;
  const size_t bytes = (size_t)nrhs * n * sizeof(double);
  const double* db = nullptr;
  double* dq = nullptr;
  int st;
  if ((st = stage_in(c, &c->ws_in0, b, bytes, (const void**)&db))) return st;
  bool q_dev = false;
  if ((st = on_device(c, q_inout, &q_dev))) return st;
  if (q_dev) {
    dq = q_inout;
  } else {
    if ((st = buf_reserve(c, &c->ws_out0, bytes))) return st;
    dq = (double*)c->ws_out0.ptr;
    if (use_guess && (st = cuda_check(c, cudaMemcpyAsync(dq, q_inout, bytes,
                                                         cudaMemcpyHostToDevice, c->stream),
                                      "guess in")))
      return st;
  }
  std::vector<int> it(nrhs);
  std::vector<double> rr(nrhs);
  SolveArgs a{nrhs, db, 1.0 / kKe, dq, use_guess != 0, tol, maxit, it.data(), rr.data()};
  const int solve_st = pcg_solve(c, a);
  if (solve_st != CPM_OK && solve_st != CPM_ENOCONV) return solve_st;
  if (!q_dev && (st = copy_out(c, q_inout, dq, bytes))) return st;
  if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "solve sync"))) return st;
  if (iters_out) memcpy(iters_out, it.data(), nrhs * sizeof(int));
  if (relres_out) memcpy(relres_out, rr.data(), nrhs * sizeof(double));
  return solve_st;
}

int cpm_neutralize(cpm_ctx* c, int nrhs, double* q_inout, const double* qsol) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_neutralize before cpm_build_E");
  if (nrhs < 1 || !q_inout) return set_err(c, CPM_EINVAL, "cpm_neutralize: bad arguments");
  const int n = c->n;
  const size_t bytes = (size_t)nrhs * n * sizeof(double);
  int st;
  double* dq = nullptr;
  const double* dqs = nullptr;
  bool q_dev = false;
  if ((st = on_device(c, q_inout, &q_dev))) return st;
  if (q_dev) {
    dq = q_inout;
  } else {
    if ((st = buf_reserve(c, &c->ws_out0, bytes))) return st;
    dq = (double*)c->ws_out0.ptr;
    if ((st = cuda_check(c, cudaMemcpyAsync(dq, q_inout, bytes, cudaMemcpyHostToDevice,
                                            c->stream), "q in")))
      return st;
  }
  if (qsol && (st = stage_in(c, &c->ws_in1, qsol, nrhs * sizeof(double), (const void**)&dqs)))
    return st;
  launch_neutralize(dq, nrhs, n, (const double*)c->d.ptr, dqs, c->stream);
  if ((st = cuda_check(c, cudaGetLastError(), "neutralize"))) return st;
  if (!q_dev && (st = copy_out(c, q_inout, dq, bytes))) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "neutralize sync");
}

int cpm_gcd_setup(cpm_ctx* c, int m, const int* labels, double tol, int maxit, double* c_out,
                  int* iters_out, double* relres_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_gcd_setup before cpm_build_E");
  if (m < 1 || m > CPM_GCD_MAX_ELECTRODES || !labels || !(tol > 0) || maxit < 1)
    return set_err(c, CPM_EINVAL, "cpm_gcd_setup: bad arguments");
  c->gcd_m = 0;
  const int n = c->n;
  cudaStream_t s = c->stream;
  int st;
  if ((st = cuda_check(c, cudaStreamSynchronize(s), "gcd sync"))) return st;
  // labels: every one in range and no electrode empty (checked on the host)
  std::vector<int> lab;
  if ((st = to_host(c, lab, labels, (size_t)n))) return st;
  std::vector<int> count(m, 0);
  for (int i = 0; i < n; ++i) {
    if (lab[i] < 0 || lab[i] >= m) return set_err(c, CPM_EINVAL, "cpm_gcd_setup: label out of range");
    ++count[lab[i]];
  }
  for (int a = 0; a < m; ++a)
    if (count[a] == 0) return set_err(c, CPM_EINVAL, "cpm_gcd_setup: an electrode has no atoms");
  const size_t vec_bytes = (size_t)m * n * sizeof(double);
  if ((st = buf_reserve(c, &c->gcd_labels, (size_t)n * sizeof(int))) ||
      (st = buf_reserve(c, &c->gcd_a, vec_bytes)) ||
      (st = buf_reserve(c, &c->ws_in2, vec_bytes)) ||
      (st = buf_reserve(c, &c->gcd_c, (size_t)m * m * sizeof(double))) ||
      (st = buf_reserve(c, &c->gcd_cinv, (size_t)m * m * sizeof(double))) ||
      (st = buf_reserve(c, &c->gcd_status, sizeof(int))))
    return st;
  int* dlab = (int*)c->gcd_labels.ptr;
  double* rhs = (double*)c->ws_in2.ptr;
  if ((st = cuda_check(c, cudaMemcpyAsync(dlab, lab.data(), (size_t)n * sizeof(int),
                                          cudaMemcpyHostToDevice, s), "gcd labels")))
    return st;
  // Eq. S22-S23: a^h = E^-1 b^h for every electrode, one PCG over m right-hand sides
  launch_gcd_indicators(dlab, n, m, rhs, s);
  if ((st = cuda_check(c, cudaGetLastError(), "gcd indicators"))) return st;
  std::vector<int> it(m);
  std::vector<double> rr(m);
  SolveArgs a{m, rhs, 1.0, (double*)c->gcd_a.ptr, false, tol, maxit, it.data(), rr.data()};
  const int solve_st = pcg_solve(c, a);
  if (iters_out) memcpy(iters_out, it.data(), m * sizeof(int));
  if (relres_out) memcpy(relres_out, rr.data(), m * sizeof(double));
  if (solve_st == CPM_ENOCONV)
    return set_err(c, CPM_ENOCONV, "cpm_gcd_setup: an electrode's solve missed tol");
  if (solve_st != CPM_OK) return solve_st;
  // Eq. S24: C_ab = sum over electrode a of a^b, then C^-1
  launch_gcd_sums((const double*)c->gcd_a.ptr, n, m, dlab, m, (double*)c->gcd_c.ptr, s);
  launch_gcd_invert((const double*)c->gcd_c.ptr, m, (double*)c->gcd_cinv.ptr,
                    (int*)c->gcd_status.ptr, s);
  if ((st = cuda_check(c, cudaGetLastError(), "gcd capacitance"))) return st;
  int singular = 0;
  std::vector<double> ct((size_t)m * m);
  if ((st = cuda_check(c, cudaMemcpyAsync(&singular, c->gcd_status.ptr, sizeof(int),
                                          cudaMemcpyDeviceToHost, s), "gcd status")) ||
      (st = cuda_check(c, cudaMemcpyAsync(ct.data(), c->gcd_c.ptr, ct.size() * sizeof(double),
                                          cudaMemcpyDeviceToHost, s), "gcd C")) ||
      (st = cuda_check(c, cudaStreamSynchronize(s), "gcd sync")))
    return st;
  if (singular) return set_err(c, CPM_EBREAKDOWN, "cpm_gcd_setup: C is singular");
  if (c_out) {
    std::vector<double> cv((size_t)m * m);
    for (int r = 0; r < m; ++r)
      for (int q = 0; q < m; ++q) cv[(size_t)r * m + q] = ct[(size_t)q * m + r] / kKe;  // e/V
    if ((st = cuda_check(c, cudaMemcpy(c_out, cv.data(), cv.size() * sizeof(double),
                                       cudaMemcpyDefault), "gcd C out")))
      return st;
  }
  c->gcd_m = m;
  return CPM_OK;
}

int cpm_gcd_charges(cpm_ctx* c, int nrhs, double* q_inout, const double* q0,
                    const double* qsol, double* dmu_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_gcd_charges before cpm_build_E");
  if (c->gcd_m < 1) return set_err(c, CPM_EINVAL, "cpm_gcd_charges before cpm_gcd_setup");
  if (nrhs < 1 || !q_inout || !q0) return set_err(c, CPM_EINVAL, "cpm_gcd_charges: bad arguments");
  const int n = c->n, m = c->gcd_m;
  cudaStream_t s = c->stream;
  int st;
  if ((st = cuda_check(c, cudaStreamSynchronize(s), "gcd sync"))) return st;
  // the totals must balance the electrolyte: E_n stands in for E only then
  std::vector<double> hq0, hqs(nrhs, 0.0);
  if ((st = to_host(c, hq0, q0, (size_t)nrhs * m))) return st;
  if (qsol && (st = to_host(c, hqs, qsol, (size_t)nrhs))) return st;
  for (int f = 0; f < nrhs; ++f) {
    double tot = hqs[f], mag = fabs(hqs[f]);
    for (int a = 0; a < m; ++a) {
      tot += hq0[(size_t)f * m + a];
      mag += fabs(hq0[(size_t)f * m + a]);
    }
    if (!(fabs(tot) <= 1e-9 * std::max(1.0, mag)))
      return set_err(c, CPM_EINVAL, "cpm_gcd_charges: electrode totals do not balance Q^sol");
  }
  const size_t bytes = (size_t)nrhs * n * sizeof(double);
  const size_t mbytes = (size_t)nrhs * m * sizeof(double);
  double* dq = nullptr;
  const double* dq0 = nullptr;
  double* ddmu = nullptr;
  bool q_dev = false;
  if ((st = on_device(c, q_inout, &q_dev))) return st;
  if (q_dev) {
    dq = q_inout;
  } else {
    if ((st = buf_reserve(c, &c->ws_out0, bytes))) return st;
    dq = (double*)c->ws_out0.ptr;
    if ((st = cuda_check(c, cudaMemcpyAsync(dq, q_inout, bytes, cudaMemcpyHostToDevice, s),
                         "q in")))
      return st;
  }
  if ((st = stage_in(c, &c->ws_in1, q0, mbytes, (const void**)&dq0))) return st;
  if (dmu_out && (st = stage_out(c, &c->ws_out1, dmu_out, mbytes, (void**)&ddmu))) return st;
  if ((st = buf_reserve(c, &c->gcd_scratch, 2 * mbytes))) return st;
  double* sums = (double*)c->gcd_scratch.ptr;
  double* dmu = sums + (size_t)nrhs * m;
  const int* dlab = (const int*)c->gcd_labels.ptr;
  launch_gcd_sums(dq, n, nrhs, dlab, m, sums, s);  // B^T q^b
  launch_gcd_shifts((const double*)c->gcd_cinv.ptr, dq0, sums, nrhs, m, dmu, ddmu, s);
  launch_gcd_apply(dq, (const double*)c->gcd_a.ptr, dmu, n, nrhs, m, s);
  if ((st = cuda_check(c, cudaGetLastError(), "gcd charges"))) return st;
  if (!q_dev && (st = copy_out(c, q_inout, dq, bytes))) return st;
  if (dmu_out && (st = copy_out(c, dmu_out, ddmu, mbytes))) return st;
  return cuda_check(c, cudaStreamSynchronize(s), "gcd charges sync");
}

int cpm_smatrix_build(cpm_ctx* c, double tol, int maxit, int* max_iters_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_smatrix_build before cpm_build_E");
  if (!(tol > 0) || maxit < 1) return set_err(c, CPM_EINVAL, "cpm_smatrix_build: bad arguments");
  const int n = c->n;
  if (n > CPM_SMATRIX_MAX_ATOMS)
    return set_err(c, CPM_EINVAL, "cpm_smatrix_build: n above CPM_SMATRIX_MAX_ATOMS");
  c->smat_ready = false;
  cudaStream_t s = c->stream;
  int st;
  const size_t bytes = (size_t)n * n * sizeof(double);
  if ((st = buf_reserve(c, &c->smat, bytes)) || (st = buf_reserve(c, &c->ws_in2, bytes)))
    return st;
  double* ident = (double*)c->ws_in2.ptr;
  double* x = (double*)c->smat.ptr;
  launch_identity(ident, n, s);
  if ((st = cuda_check(c, cudaGetLastError(), "identity"))) return st;
  // the columns E^-1 e_j: n right-hand sides of one PCG (b already in e/A: scale 1)
  std::vector<int> it(n);
  std::vector<double> rr(n);
  SolveArgs a{n, ident, 1.0, x, false, tol, maxit, it.data(), rr.data()};
  const int solve_st = pcg_solve(c, a);
  if (max_iters_out) *max_iters_out = *std::max_element(it.begin(), it.end());
  if (solve_st == CPM_ENOCONV)
    return set_err(c, CPM_ENOCONV, "cpm_smatrix_build: a column missed tol");
  if (solve_st != CPM_OK) return solve_st;
  launch_smatrix_form(x, (const double*)c->d.ptr, c->c_ele, n, s);
  if ((st = cuda_check(c, cudaGetLastError(), "smatrix form")) ||
      (st = cuda_check(c, cudaStreamSynchronize(s), "smatrix sync")))
    return st;
  c->smat_ready = true;
  return CPM_OK;
}

int cpm_smatrix_charges(cpm_ctx* c, int frames, const double* b, const double* qsol,
                        double* q_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_smatrix_charges before cpm_build_E");
  if (!c->smat_ready)
    return set_err(c, CPM_EINVAL, "cpm_smatrix_charges before cpm_smatrix_build");
  if (frames < 1 || frames > smatrix_max_frames() || !b || !q_out)
    return set_err(c, CPM_EINVAL, "cpm_smatrix_charges: bad arguments");
  const int n = c->n;
  cudaStream_t s = c->stream;
  const size_t bytes = (size_t)frames * n * sizeof(double);
  int st;
  const double* db = nullptr;
  const double* dqs = nullptr;
  double* dq = nullptr;
  if ((st = stage_in(c, &c->ws_in0, b, bytes, (const void**)&db))) return st;
  if (qsol && (st = stage_in(c, &c->ws_in1, qsol, frames * sizeof(double), (const void**)&dqs)))
    return st;
  if ((st = stage_out(c, &c->ws_out0, q_out, bytes, (void**)&dq))) return st;
  launch_smatrix_apply((const double*)c->smat.ptr, db, dqs, (const double*)c->d.ptr, n, frames,
                       1.0 / kKe, dq, s);
  if ((st = cuda_check(c, cudaGetLastError(), "smatrix apply"))) return st;
  if ((st = copy_out(c, q_out, dq, bytes))) return st;
  return cuda_check(c, cudaStreamSynchronize(s), "smatrix sync");
}

int cpm_get_E(cpm_ctx* c, int form, double* out, int64_t ld) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_get_E before cpm_build_E");
  if (!out || ld < c->n || (form != CPM_E_STORED && form != CPM_E_PAPER))
    return set_err(c, CPM_EINVAL, "cpm_get_E: bad arguments");
  const size_t bytes = (size_t)c->n * ld * sizeof(double);
  double* d = nullptr;
  int st;
  if ((st = stage_out(c, &c->ws_out0, out, bytes, (void**)&d))) return st;
  launch_get_E(c->fp64(), c->E.ptr, c->n, c->ldE, (const double*)c->xyz.ptr, geometry(c),
               form == CPM_E_PAPER, nullptr, c->n, d, ld, c->stream);
  if ((st = cuda_check(c, cudaGetLastError(), "get_E"))) return st;
  if ((st = copy_out(c, out, d, bytes))) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "get_E sync");
}

int cpm_get_E_rows(cpm_ctx* c, int form, int nrows, const int* rows, double* out, int64_t ld) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_get_E_rows before cpm_build_E");
  if (nrows < 1 || !rows || !out || ld < c->n || (form != CPM_E_STORED && form != CPM_E_PAPER))
    return set_err(c, CPM_EINVAL, "cpm_get_E_rows: bad arguments");
  std::vector<int> hr(nrows);
  int st = cuda_check(c, cudaMemcpyAsync(hr.data(), rows, nrows * sizeof(int), cudaMemcpyDefault,
                                         c->stream), "rows");
  if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "rows sync");
  if (st) return st;
  for (int r : hr)
    if (r < 0 || r >= c->n) return set_err(c, CPM_EINVAL, "cpm_get_E_rows: row out of range");
  const size_t bytes = (size_t)nrows * ld * sizeof(double);
  double* d = nullptr;
  const int* dr = nullptr;
  if ((st = stage_in(c, &c->ws_in0, hr.data(), nrows * sizeof(int), (const void**)&dr)) ||
      (st = stage_out(c, &c->ws_out0, out, bytes, (void**)&d)))
    return st;
  launch_get_E(c->fp64(), c->E.ptr, c->n, c->ldE, (const double*)c->xyz.ptr, geometry(c),
               form == CPM_E_PAPER, dr, nrows, d, ld, c->stream);
  if ((st = cuda_check(c, cudaGetLastError(), "get_E_rows"))) return st;
  if ((st = copy_out(c, out, d, bytes))) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "get_E_rows sync");
}

int cpm_apply_E(cpm_ctx* c, int nrhs, const double* p, double* q) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_apply_E before cpm_build_E");
  if (nrhs < 1 || !p || !q) return set_err(c, CPM_EINVAL, "cpm_apply_E: bad arguments");
  const size_t bytes = (size_t)nrhs * c->n * sizeof(double);
  const double* dp = nullptr;
  double* dq = nullptr;
  int st;
  if ((st = stage_in(c, &c->ws_in0, p, bytes, (const void**)&dp))) return st;
  if ((st = stage_out(c, &c->ws_out0, q, bytes, (void**)&dq))) return st;
  if ((st = apply_E(c, nrhs, dp, dq))) return st;
  if ((st = copy_out(c, q, dq, bytes))) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "apply_E sync");
}

int cpm_get_d(cpm_ctx* c, double* d_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_get_d before cpm_build_E");
  if (!d_out) return set_err(c, CPM_EINVAL, "cpm_get_d: null output");
  int st = cuda_check(c, cudaMemcpyAsync(d_out, c->d.ptr, (size_t)c->n * sizeof(double),
                                         cudaMemcpyDefault, c->stream), "get_d");
  if (st) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "get_d sync");
}

int cpm_get_precond(cpm_ctx* c, int64_t* off, int* idx, double* val) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_get_precond before cpm_build_E");
  if (c->p.precond < CPM_PRECOND_DC || !c->nbr_off.ptr)
    return set_err(c, CPM_EINVAL, "cpm_get_precond: the context was built without a sparse "
                                  "preconditioner (PCG-DC, -Normal or -Full)");
  if (!off || !idx || !val) return set_err(c, CPM_EINVAL, "cpm_get_precond: null output");
  return copy_precond(c, off, idx, val);
}

int cpm_get_info(cpm_ctx* c, cpm_info_t* out) {
  if (!c || !out) return CPM_EINVAL;
  memset(out, 0, sizeof(*out));
  out->n = c->n;
  out->m = c->m;
  out->nnz_p = c->nnz;
  out->p_gap = c->pgap;
  out->c_ele = c->c_ele;
  out->t_kspace_ms = c->t_kspace_ms;
  out->t_phase_ms = c->t_phase_ms;
  out->t_precond_ms = c->t_precond_ms;
  out->t_dsolve_ms = c->t_dsolve_ms;
  out->t_tc_ms = c->t_tc_ms;
  out->head_cols = 16 * c->heavy_steps;
  out->t_matvec_ms = c->t_matvec_ms;
  const int kb0 = c->heavy_steps / 4, kbn = 2 * c->mpad / 64;
  const bool tc = c->built && c->p.precision == CPM_PREC_BF16X6;
  out->tc_blocks[0] = tc ? c->kb6_end - kb0 : 0;
  out->tc_blocks[1] = tc ? c->kb3_end - c->kb6_end : 0;
  out->tc_blocks[2] = tc ? kbn - c->kb3_end : 0;
  out->tc_blocks_fp8 = tc ? kbn - c->kb8_begin : 0;
  out->t_head_ms = c->t_head_ms;
  out->t_tc_light_ms = c->t_light_ms;
  out->t_tc_loop_ms = c->t_tc_loop_ms;
  out->t_solve_ms = c->t_solve_ms;
  out->t_solve_matvec_ms = c->t_solve_mv_ms;
  out->t_solve_replace_ms = c->t_solve_rep_ms;
  out->solve_replacements = c->solve_replacements;
  out->t_solve_dc_ms = c->t_solve_dc_ms;
  out->t_pot_sf_ms = c->t_pot_sf_ms;
  out->t_pot_kspace_ms = c->t_pot_kspace_ms;
  out->t_pot_real_ms = c->t_pot_real_ms;
  out->solve_path = c->last_solve_path;
  out->d_iters = c->d_iters;
  out->launches = launch_count();
  return CPM_OK;
}

}  // extern "C"
