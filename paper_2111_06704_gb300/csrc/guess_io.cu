// The learned guess's set-up and storage: the network's initial parameters, the feature
// normalisation and the target scale from training samples, and a file format for a
// trained network.  The paper has no learned component: these are the project's own
// definitions (a counter-based SplitMix64 stream for the initial weights; FP64 sums in a
// fixed order for the statistics).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "cpm_internal.cuh"

namespace cpm {
namespace {

constexpr int kF = CPM_MLP_FEATURES;  // 32
constexpr int kP = CPM_MLP_PARAMS;    // 10,497
constexpr int kNormThreads = 256;
constexpr int kNormBlocks = 256;

// SplitMix64 (Steele, Lea and Flood, 2014): output number `k` (from 0) of the stream
// seeded with `seed`, as a double uniform in [0, 1) from its top 53 bits.
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// Layer-by-layer uniform initialisation: weights of a layer with `fan_in` inputs drawn
// from [-sqrt(6 / fan_in), sqrt(6 / fan_in)) (computed in FP64, stored as float), the
// output layer's weights scaled by 0.1 so that the first guesses stay near the previous
// step's charges, biases zero.  Parameter k takes stream number k.
__global__ void k_guess_init(uint64_t seed, float* __restrict__ params) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kP) return;
  // layers: (64 x 32), (64 x 64), (64 x 64), (1 x 64), each weights then biases
  const int out[4] = {64, 64, 64, 1}, in[4] = {32, 64, 64, 64};
  int base = 0;
  for (int l = 0; l < 4; ++l) {
    const int nw = out[l] * in[l];
    if (k < base + nw) {
      const double lim = sqrt(6.0 / in[l]) * (l == 3 ? 0.1 : 1.0);
      params[k] = (float)(lim * (2.0 * splitmix_uniform(seed, (uint64_t)k) - 1.0));
      return;
    }
    if (k < base + nw + out[l]) {
      params[k] = 0.0f;
      return;
    }
    base += nw + out[l];
  }
}

// Per-block partial sums of column c (c < 32: feature c, c = 32: the target) of
// (x - shift[c])^p for p = 1 (shift = 0) or 2 (shift = the mean); fixed order.
__global__ void __launch_bounds__(kNormThreads)
k_norm_partial(const float* __restrict__ feat, const float* __restrict__ target,
               int64_t samples, const double* __restrict__ shift, int square,
               double* __restrict__ part) {
  __shared__ double sm[kNormThreads];
  const int c = blockIdx.y;
  const double sh = square ? shift[c] : 0.0;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kNormThreads + threadIdx.x; i < samples;
       i += (int64_t)gridDim.x * kNormThreads) {
    const double x = (double)(c < kF ? feat[i * kF + c] : target[i]) - sh;
    acc += square ? x * x : x;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kNormThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[c * gridDim.x + blockIdx.x] = sm[0];
}

// out[c] = (sum of the blocks' partials of column c) / samples, in block order.
__global__ void k_norm_finish(const double* __restrict__ part, int blocks, int64_t samples,
                              double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c > kF) return;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += part[c * blocks + b];
  out[c] = s / (double)samples;
}

// The guess file: magic, version, sizes, target scale, parameters, normalisation, and an
// FNV-1a checksum of everything before it.
struct GuessFileHead {
  char magic[8];  // "CPMGUESS"
  uint32_t version, n_params, n_features, reserved;
  float target_scale;
  uint32_t pad;
};
static_assert(sizeof(GuessFileHead) == 32, "file header layout");

uint64_t fnv1a(const uint8_t* p, size_t len, uint64_t h = 0xcbf29ce484222325ull) {
  for (size_t i = 0; i < len; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

// Copies `bytes` between host or device arrays (device arrays of any device: a plain
// copy, no kernel reads them).
int copy_any(void* dst, const void* src, size_t bytes) {
  if (cudaMemcpy(dst, src, bytes, cudaMemcpyDefault) == cudaSuccess) return CPM_OK;
  cudaGetLastError();
  // without a usable CUDA runtime (no driver): plain host memory
  memcpy(dst, src, bytes);
  return CPM_OK;
}

}  // namespace
}  // namespace cpm

using namespace cpm;

struct cpm_ctx : public cpm::Ctx {};

extern "C" {

int cpm_guess_init(cpm_ctx* c, uint64_t seed, float* params) {
  if (!c) return CPM_EINVAL;
  if (!params || pointer_where(c, params) != 1)
    return set_err(c, CPM_EINVAL, "cpm_guess_init: params must be a device array");
  (k_guess_init<<<(kP + 255) / 256, 256, 0, c->stream>>>(seed, params), note_launch());
  if (int st = cuda_check(c, cudaGetLastError(), "guess init")) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "guess init sync");
}

int cpm_guess_norm(cpm_ctx* c, int64_t samples, const float* feat, const float* target,
                   float* norm, float* target_scale) {
  if (!c) return CPM_EINVAL;
  if (samples < 1 || !feat || !target || !norm || !target_scale ||
      pointer_where(c, feat) != 1 || pointer_where(c, target) != 1)
    return set_err(c, CPM_EINVAL, "cpm_guess_norm: samples >= 1, device feat and target");
  const int cols = kF + 1;
  Buf ws;  // partials [33][blocks], then the means and variances [2][33]
  int st;
  if ((st = buf_alloc(c, &ws, ((size_t)cols * kNormBlocks + 2 * cols) * sizeof(double))))
    return st;
  double* part = (double*)ws.ptr;
  double* mean = part + (size_t)cols * kNormBlocks;
  double* var = mean + cols;
  cudaStream_t s = c->stream;
  const dim3 grid(kNormBlocks, cols);
  (k_norm_partial<<<grid, kNormThreads, 0, s>>>(feat, target, samples, mean, 0, part), note_launch());
  (k_norm_finish<<<1, 64, 0, s>>>(part, kNormBlocks, samples, mean), note_launch());
  (k_norm_partial<<<grid, kNormThreads, 0, s>>>(feat, target, samples, mean, 1, part), note_launch());
  (k_norm_finish<<<1, 64, 0, s>>>(part, kNormBlocks, samples, var), note_launch());
  std::vector<double> h(2 * cols);
  st = cuda_check(c, cudaGetLastError(), "guess norm");
  if (!st) st = cuda_check(c, cudaMemcpyAsync(h.data(), mean, 2 * cols * sizeof(double),
                                              cudaMemcpyDeviceToHost, s), "guess norm out");
  if (!st) st = cuda_check(c, cudaStreamSynchronize(s), "guess norm sync");
  buf_free(c, &ws);
  if (st) return st;
  // mean, then the inverse standard deviation (0 for a constant feature)
  float hn[2 * kF];
  for (int j = 0; j < kF; ++j) {
    const double sd = sqrt(h[cols + j]);
    hn[j] = (float)h[j];
    hn[kF + j] = sd > 1e-12 ? (float)(1.0 / sd) : 0.0f;
  }
  const double ts = sqrt(h[cols + kF]);
  *target_scale = ts > 0.0 ? (float)ts : 1.0f;
  return cuda_check(c, cudaMemcpy(norm, hn, sizeof(hn), cudaMemcpyDefault), "norm out");
}

int cpm_guess_save(const char* path, const float* params, const float* norm,
                   float target_scale) {
  if (!path || !params || !norm) return CPM_EINVAL;
  std::vector<uint8_t> buf(sizeof(GuessFileHead) + (kP + 2 * kF) * sizeof(float));
  GuessFileHead hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "CPMGUESS", 8);
  hd.version = 1;
  hd.n_params = kP;
  hd.n_features = kF;
  hd.target_scale = target_scale;
  memcpy(buf.data(), &hd, sizeof(hd));
  copy_any(buf.data() + sizeof(hd), params, kP * sizeof(float));
  copy_any(buf.data() + sizeof(hd) + kP * sizeof(float), norm, 2 * kF * sizeof(float));
  const uint64_t sum = fnv1a(buf.data(), buf.size());
  FILE* f = fopen(path, "wb");
  if (!f) return CPM_EIO;
  const bool ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size() &&
                  fwrite(&sum, sizeof(sum), 1, f) == 1;
  return fclose(f) == 0 && ok ? CPM_OK : CPM_EIO;
}

int cpm_guess_load(const char* path, float* params, float* norm, float* target_scale) {
  if (!path || !params || !norm || !target_scale) return CPM_EINVAL;
  std::vector<uint8_t> buf(sizeof(GuessFileHead) + (kP + 2 * kF) * sizeof(float));
  uint64_t sum = 0;
  FILE* f = fopen(path, "rb");
  if (!f) return CPM_EIO;
  const bool ok = fread(buf.data(), 1, buf.size(), f) == buf.size() &&
                  fread(&sum, sizeof(sum), 1, f) == 1 && fgetc(f) == EOF;
  fclose(f);
  if (!ok) return CPM_EIO;
  GuessFileHead hd;
  memcpy(&hd, buf.data(), sizeof(hd));
  if (memcmp(hd.magic, "CPMGUESS", 8) != 0 || hd.version != 1 || hd.n_params != (uint32_t)kP ||
      hd.n_features != (uint32_t)kF || fnv1a(buf.data(), buf.size()) != sum)
    return CPM_EIO;
  *target_scale = hd.target_scale;
  copy_any(params, buf.data() + sizeof(hd), kP * sizeof(float));
  copy_any(norm, buf.data() + sizeof(hd) + kP * sizeof(float), 2 * kF * sizeof(float));
  return CPM_OK;
}

}  // extern "C"
