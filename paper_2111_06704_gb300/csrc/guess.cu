// Learned initial guess: per-atom features, a 32 -> 64 -> 64 -> 64 -> 1 SiLU network
// (forward, gradient, Adam), and the guess q0 = q_prev + scale * net(features).
//
// The paper has no learned component; the network and its features are the project's
// definition (see the FP64 oracle for the same definition written out).  Parameters are
// FP32 master values; with `bf16` set the forward and gradient use them rounded to BF16
// (FP32 accumulation throughout).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "cpm_internal.cuh"

namespace cpm {

namespace {

constexpr int kF = CPM_MLP_FEATURES;  // 32
constexpr int kH = 64;
constexpr int kP = CPM_MLP_PARAMS;    // 10,497
// parameter offsets: W1 [64][32], b1, W2 [64][64], b2, W3 [64][64], b3, W4 [64], b4
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + kH;
static_assert(ob4 + 1 == kP, "parameter layout");

// SiLU and its derivative through the fast exponential and reciprocal (relative error
// ~1e-6, far inside what a guess needs and what the oracle comparison allows): the
// forward pass spends as many instructions on 192 activations per sample as on its
// 10,497 multiply-adds otherwise.
__device__ __forceinline__ float sigmoid(float z) { return __frcp_rn(1.0f + __expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid(z); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = sigmoid(z);
  return s * (1.0f + z * (1.0f - s));
}

// Shell of every PCG-DC pattern entry (k - 1/2 <= r < k + 1/2, k = 1..8; 0 outside or
// for the atom itself).  The electrode is fixed, so this geometry is found once; the host
// then files the entries of each atom by shell.
__global__ void k_shell_codes(int n, const double* __restrict__ xyz, double lx, double ly,
                              double lz, const int64_t* __restrict__ off,
                              const int* __restrict__ idx, uint8_t* __restrict__ shell) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
  for (int64_t e = off[i]; e < off[i + 1]; ++e) {
    const int j = idx[e];
    int k = 0;
    if (j != i) {
      double dx = xyz[3 * j] - xi, dy = xyz[3 * j + 1] - yi, dz = xyz[3 * j + 2] - zi;
      dx -= lx * rint(dx / lx);
      dy -= ly * rint(dy / ly);
      dz -= lz * rint(dz / lz);
      k = (int)floor(sqrt(dx * dx + dy * dy + dz * dz) + 0.5);
      if (k < 1 || k > 8) k = 0;
    }
    shell[e] = (uint8_t)k;
  }
}

__global__ void k_to_float(const double* __restrict__ v, int64_t len, double add,
                           float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)(v[e] + add);
}

// The potentials of a frame as floats: (b - b_prev, b) per atom.
__global__ void k_guess_prep(int64_t len, const double* __restrict__ b,
                             const double* __restrict__ b_prev, float2* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)(b[e] - b_prev[e]), (float)b[e]);
}

// Features of atom i in frame f (unscaled): 0 the potential change Delta b = b - b_prev,
// 1-8 its means over the neighbour shells k = 1..8, 9 b, 10-17 the shell means of b,
// 18 chi, 19 the side of the electrode (+1 above the mean height), 20 (P Delta b) / k_e
// with the PCG-DC preconditioner's pattern entries, 21-31 zero.
constexpr int kFeatFrames = 4;     // frames per thread: index loads shared by them
constexpr int kFeatThreads = 128;  // atoms per block

__global__ void __launch_bounds__(kFeatThreads)
k_guess_features(int n, int frames, const float2* __restrict__ pot,
                 const double* __restrict__ chi, const double* __restrict__ xyz, double zmean,
                 const int64_t* __restrict__ sh_off, const int* __restrict__ sh_idx,
                 const int64_t* __restrict__ off, const int* __restrict__ idx,
                 const float* __restrict__ pf32, float* __restrict__ feat) {
  constexpr int FB = kFeatFrames;
  __shared__ float stage[kFeatThreads * (kF + 1)];
  const int i0 = blockIdx.x * kFeatThreads;
  const int i = i0 + threadIdx.x;
  const int f0 = blockIdx.y * FB;
  const bool live = i < n;
  float sd[FB][8], sb[FB][8], pz[FB];
#pragma unroll
  for (int u = 0; u < FB; ++u) {
    pz[u] = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) sd[u][k] = sb[u][k] = 0.f;
  }
  // a frame past the last reads frame 0 and is not written
  const float2* pf[FB];
#pragma unroll
  for (int u = 0; u < FB; ++u) pf[u] = pot + (int64_t)(f0 + u < frames ? f0 + u : 0) * n;
  int cnt[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) cnt[k] = 0;
  if (live) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t e0 = sh_off[(int64_t)i * 8 + k], e1 = sh_off[(int64_t)i * 8 + k + 1];
      cnt[k] = (int)(e1 - e0);
      for (int64_t e = e0; e < e1; ++e) {
        const int j = sh_idx[e];
#pragma unroll
        for (int u = 0; u < FB; ++u) {
          const float2 v = pf[u][j];
          sd[u][k] += v.x;
          sb[u][k] += v.y;
        }
      }
    }
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
      const int j = idx[e];
      const float w = pf32[e];
#pragma unroll
      for (int u = 0; u < FB; ++u) pz[u] = fmaf(w, pf[u][j].x, pz[u]);
    }
  }
  const float chi_i = live ? (float)chi[i] : 0.f;
  const float side = live && xyz[3 * i + 2] > zmean ? 1.f : -1.f;
  const int na = min(kFeatThreads, n - i0);
#pragma unroll
  for (int u = 0; u < FB; ++u) {
    if (f0 + u >= frames) break;  // uniform per block
    float* row = stage + threadIdx.x * (kF + 1);
    if (live) {
      const float2 self = pf[u][i];
      row[0] = self.x;
      row[9] = self.y;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float inv = cnt[k] ? 1.0f / (float)cnt[k] : 0.f;
        row[1 + k] = sd[u][k] * inv;
        row[10 + k] = sb[u][k] * inv;
      }
      row[18] = chi_i;
      row[19] = side;
      row[20] = pz[u] * (float)(1.0 / kKe);
#pragma unroll
      for (int c = 21; c < kF; ++c) row[c] = 0.f;
    }
    __syncthreads();
    // the block's atoms are consecutive: one contiguous, coalesced write per frame
    float* dst = feat + ((int64_t)(f0 + u) * n + i0) * kF;
    for (int e = threadIdx.x; e < na * kF; e += kFeatThreads)
      dst[e] = stage[(e / kF) * (kF + 1) + e % kF];
    __syncthreads();
  }
}

__device__ void load_params(const float* __restrict__ params, float* w, int bf16) {
  for (int k = threadIdx.x; k < kP; k += blockDim.x) {
    const float v = params[k];
    w[k] = bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
  }
}

// y[s] = net((feat[s] - mean) * inv_std), 128 samples per tile.  Weights (transposed,
// unit index fastest) and the activations of a tile (feature-major) sit in shared memory;
// each thread owns 8 samples x 4 units of a layer, so every float4 of weights and of
// activations it loads feeds 32 (or 16) FMAs.  The float4 slot of an activation row is
// XOR-swizzled with the row's unit group, which keeps the transposed stores of a layer's
// output free of bank conflicts.
constexpr int kTs = 128;          // samples per tile
constexpr int kFwdThreads = 256;  // 16 unit groups x 16 sample groups
constexpr int kWT = kP + 3;       // transposed weights, padded to a float4 boundary
constexpr size_t kFwdSmem = sizeof(float) * (kWT + 2 * kH * kTs);

__device__ __forceinline__ int act_at(int row, int s) {
  return row * kTs + 4 * ((s >> 2) ^ ((row >> 2) & 7)) + (s & 3);
}

// out[a][s] = silu(bias[a] + sum_c WT[c][a] in[c][s]) for this thread's 8 x 4 block.
template <int NIN>
__device__ __forceinline__ void fwd_layer(const float* __restrict__ WT,
                                          const float* __restrict__ bias,
                                          const float* __restrict__ in, float (&acc)[8][4],
                                          int ug, int sg) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[k][j] = bias[4 * ug + j];
#pragma unroll 8
  for (int c = 0; c < NIN; ++c) {
    const float4 w = *reinterpret_cast<const float4*>(WT + c * kH + 4 * ug);
    const float4 x0 = *reinterpret_cast<const float4*>(in + act_at(c, 8 * sg));
    const float4 x1 = *reinterpret_cast<const float4*>(in + act_at(c, 8 * sg + 4));
    const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[k][j] = fmaf(xv[k], wv[j], acc[k][j]);
  }
}

__device__ __forceinline__ void fwd_store(float* __restrict__ out, const float (&acc)[8][4],
                                          int ug, int sg) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int row = 4 * ug + j;
    *reinterpret_cast<float4*>(out + act_at(row, 8 * sg)) =
        make_float4(silu(acc[0][j]), silu(acc[1][j]), silu(acc[2][j]), silu(acc[3][j]));
    *reinterpret_cast<float4*>(out + act_at(row, 8 * sg + 4)) =
        make_float4(silu(acc[4][j]), silu(acc[5][j]), silu(acc[6][j]), silu(acc[7][j]));
  }
}

__global__ void __launch_bounds__(kFwdThreads, 2)
k_mlp_forward(const float* __restrict__ params, const float* __restrict__ norm, int bf16,
              int64_t samples, const float* __restrict__ feat, float* __restrict__ out,
              float scale, const double* __restrict__ q_prev, double* __restrict__ q0) {
  extern __shared__ __align__(16) float fsm[];
  float* WT1 = fsm;               // [kF][kH]
  float* WT2 = WT1 + kF * kH;     // [kH][kH]
  float* WT3 = WT2 + kH * kH;     // [kH][kH]
  float* bv = WT3 + kH * kH;      // b1, b2, b3, W4 [kH each], b4
  float* act0 = fsm + kWT;        // [kH][kTs]
  float* act1 = act0 + kH * kTs;  // [kH][kTs]
  const int t = threadIdx.x;
  for (int e = t; e < kP; e += kFwdThreads) {
    float v = params[e];
    if (bf16) v = __bfloat162float(__float2bfloat16_rn(v));
    int d;
    if (e < ob1) d = (e % kF) * kH + e / kF;                                  // W1[a][c]
    else if (e < oW2) d = kF * kH + 2 * kH * kH + (e - ob1);                 // b1
    else if (e < ob2) d = kF * kH + ((e - oW2) % kH) * kH + (e - oW2) / kH;  // W2
    else if (e < oW3) d = kF * kH + 2 * kH * kH + kH + (e - ob2);            // b2
    else if (e < ob3) d = kF * kH + kH * kH + ((e - oW3) % kH) * kH + (e - oW3) / kH;
    else if (e < oW4) d = kF * kH + 2 * kH * kH + 2 * kH + (e - ob3);        // b3
    else d = kF * kH + 2 * kH * kH + 3 * kH + (e - oW4);                     // W4, b4
    fsm[d] = v;
  }
  const int ug = t & 15, sg = t >> 4;
  const int64_t tiles = (samples + kTs - 1) / kTs;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t s0 = tile * kTs;
    __syncthreads();  // weights written / the previous tile's reads of act0 done
    for (int e = t; e < kTs * kF; e += kFwdThreads) {
      const int s = e / kF, c = e % kF;
      const int64_t gs = s0 + s;
      act0[act_at(c, s)] = gs < samples ? (feat[gs * kF + c] - norm[c]) * norm[kF + c] : 0.f;
    }
    __syncthreads();
    float acc[8][4];
    fwd_layer<kF>(WT1, bv, act0, acc, ug, sg);
    fwd_store(act1, acc, ug, sg);
    __syncthreads();
    fwd_layer<kH>(WT2, bv + kH, act1, acc, ug, sg);
    __syncthreads();  // all reads of act0 (the features) are done
    fwd_store(act0, acc, ug, sg);
    __syncthreads();
    fwd_layer<kH>(WT3, bv + 2 * kH, act0, acc, ug, sg);
    // output unit: y = b4 + sum_a W4[a] silu(z3[a]), summed over the 16 unit groups
    float y[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float v = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) v = fmaf(bv[3 * kH + 4 * ug + j], silu(acc[k][j]), v);
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      y[k] = v + bv[4 * kH];
    }
    if (ug == 0)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t gs = s0 + 8 * sg + k;
        if (gs < samples) {
          if (out) out[gs] = y[k];
          if (q0) q0[gs] = q_prev[gs] + (double)scale * (double)y[k];  // the guess, fused
        }
      }
  }
}

// Gradient of the mean squared error (1/S) sum_s (y_s - t_s)^2 over this call's samples,
// accumulated into grad (zeroed by the caller); loss_sum accumulates sum (y - t)^2.
// One block = 128 samples; activations of the block in shared memory; the parameter
// gradients are reductions over the block's samples, then one atomic add per parameter.
constexpr int kB = 128;
constexpr int kLd = kH + 1;  // padded row of a [sample][unit] array

__global__ void __launch_bounds__(kB, 1)
k_mlp_grad(const float* __restrict__ params, const float* __restrict__ norm, int bf16,
           int64_t samples, double inv_s, const float* __restrict__ feat,
           const float* __restrict__ target, float* __restrict__ grad,
           double* __restrict__ loss_sum) {
  extern __shared__ float sm[];
  float* w = sm;                       // kP
  float* X = w + kP;                   // [kB][kF + 1]
  float* Z1 = X + kB * (kF + 1);       // pre-activations, later dL/dz
  float* Z2 = Z1 + kB * kLd;
  float* Z3 = Z2 + kB * kLd;
  float* H1 = Z3 + kB * kLd;           // silu(Z1)
  float* H2 = H1 + kB * kLd;           // silu(Z2)
  float* DY = H2 + kB * kLd;           // [kB]
  load_params(params, w, bf16);
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t s = blockIdx.x * (int64_t)kB + t;
  const bool valid = s < samples;
  // ---- forward, one sample per thread
  {
    float* x = X + t * (kF + 1);
    for (int c = 0; c < kF; ++c)
      x[c] = valid ? (feat[s * kF + c] - norm[c]) * norm[kF + c] : 0.f;
    for (int a = 0; a < kH; ++a) {
      float z = w[ob1 + a];
      for (int c = 0; c < kF; ++c) z = fmaf(w[oW1 + a * kF + c], x[c], z);
      Z1[t * kLd + a] = z;
      H1[t * kLd + a] = silu(z);
    }
    for (int a = 0; a < kH; ++a) {
      float z = w[ob2 + a];
      for (int c = 0; c < kH; ++c) z = fmaf(w[oW2 + a * kH + c], H1[t * kLd + c], z);
      Z2[t * kLd + a] = z;
      H2[t * kLd + a] = silu(z);
    }
    float y = w[ob4];
    for (int a = 0; a < kH; ++a) {
      float z = w[ob3 + a];
      for (int c = 0; c < kH; ++c) z = fmaf(w[oW3 + a * kH + c], H2[t * kLd + c], z);
      Z3[t * kLd + a] = z;
      y = fmaf(w[oW4 + a], silu(z), y);
    }
    const float diff = valid ? y - target[s] : 0.f;
    DY[t] = (float)(2.0 * inv_s) * diff;
    double l = (double)diff * (double)diff;
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((t & 31) == 0) atomicAdd(loss_sum, l);
  }
  __syncthreads();
  // ---- output layer: dW4[a] = sum_s dy_s h3[s][a]; db4 = sum_s dy_s
  if (t < kH) {
    float acc = 0.f;
    for (int q = 0; q < kB; ++q) acc = fmaf(DY[q], silu(Z3[q * kLd + t]), acc);
    atomicAdd(&grad[oW4 + t], acc);
  } else if (t == kH) {
    float acc = 0.f;
    for (int q = 0; q < kB; ++q) acc += DY[q];
    atomicAdd(&grad[ob4], acc);
  }
  __syncthreads();
  // g3 = dy W4 * silu'(z3), in place of Z3
  for (int a = 0; a < kH; ++a) Z3[t * kLd + a] = DY[t] * w[oW4 + a] * silu_grad(Z3[t * kLd + a]);
  __syncthreads();
  // ---- hidden layers: dW = sum_s g_s h_in_s^T, db = sum_s g_s, then g_in = W^T g * silu'
  auto layer = [&](float* G, const float* Hin, int nin, int ow, int ob) {
    // 64 x nin outputs over kB threads
    const int per = kH * nin / kB;
    for (int u = 0; u < per; ++u) {
      const int e = t * per + u;
      const int a = e / nin, c = e % nin;
      float acc = 0.f;
      for (int q = 0; q < kB; ++q) {
        const float hv = nin == kF ? Hin[q * (kF + 1) + c] : Hin[q * kLd + c];
        acc = fmaf(G[q * kLd + a], hv, acc);
      }
      atomicAdd(&grad[ow + a * nin + c], acc);
    }
    if (t < kH) {
      float acc = 0.f;
      for (int q = 0; q < kB; ++q) acc += G[q * kLd + t];
      atomicAdd(&grad[ob + t], acc);
    }
  };
  layer(Z3, H2, kH, oW3, ob3);
  // g2 = W3^T g3 * silu'(z2), in place of Z2
  {
    float g[kH];
    for (int c = 0; c < kH; ++c) {
      float acc = 0.f;
      for (int a = 0; a < kH; ++a) acc = fmaf(w[oW3 + a * kH + c], Z3[t * kLd + a], acc);
      g[c] = acc * silu_grad(Z2[t * kLd + c]);
    }
    __syncthreads();  // every thread has finished reading Z2 through `layer`
    for (int c = 0; c < kH; ++c) Z2[t * kLd + c] = g[c];
  }
  __syncthreads();
  layer(Z2, H1, kH, oW2, ob2);
  {
    float g[kH];
    for (int c = 0; c < kH; ++c) {
      float acc = 0.f;
      for (int a = 0; a < kH; ++a) acc = fmaf(w[oW2 + a * kH + c], Z2[t * kLd + a], acc);
      g[c] = acc * silu_grad(Z1[t * kLd + c]);
    }
    __syncthreads();
    for (int c = 0; c < kH; ++c) Z1[t * kLd + c] = g[c];
  }
  __syncthreads();
  layer(Z1, X, kF, oW1, ob1);
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = 0.9f * m[k] + 0.1f * gk;
  const float vk = 0.999f * v[k] + 0.001f * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + 1e-8f);
}

__global__ void k_guess_apply(int64_t len, const float* __restrict__ y, float scale,
                              const double* __restrict__ q_prev, double* __restrict__ q0) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len;
       k += (int64_t)gridDim.x * blockDim.x)
    q0[k] = q_prev[k] + (double)scale * (double)y[k];
}

// Device memory of the context's device (or managed memory): what these kernels may use.
bool dev_ok(const Ctx* c, const void* p) { return pointer_where(c, p) == 1; }

constexpr size_t kGradSmem =
    sizeof(float) * (kP + kB * (kF + 1) + 5 * kB * kLd + kB);

}  // namespace
}  // namespace cpm

using namespace cpm;

struct cpm_ctx : public cpm::Ctx {};

namespace {

int features_async(cpm_ctx* c, int frames, const double* b, const double* b_prev,
                   const double* chi, float* feat) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_guess_features before cpm_build_E");
  if (c->solve_only)
    return set_err(c, CPM_EINVAL, "cpm_guess_features: a context built by cpm_build_E_copy");
  if (c->p.precond != CPM_PRECOND_DC || !c->nbr_off.ptr)
    return set_err(c, CPM_EINVAL, "cpm_guess_features needs the PCG-DC neighbour lists");
  if (frames < 1 || !dev_ok(c, b) || !dev_ok(c, b_prev) || !dev_ok(c, chi) || !dev_ok(c, feat))
    return set_err(c, CPM_EINVAL, "cpm_guess_features: frames >= 1 and device arrays");
  int st = CPM_OK;
  const int n = c->n;
  if (!c->shells_ready) {  // frame-independent geometry, once per electrode
    Buf codes;
    if ((st = buf_alloc(c, &codes, std::max<int64_t>(c->nnz, 1)))) return st;
    (k_shell_codes<<<(n + 127) / 128, 128, 0, c->stream>>>(
         n, (const double*)c->xyz.ptr, c->p.box[0], c->p.box[1], c->p.box[2],
         (const int64_t*)c->nbr_off.ptr, (const int*)c->nbr_idx.ptr, (uint8_t*)codes.ptr),
     note_launch());
    std::vector<double> hx(3 * (size_t)n);
    std::vector<int64_t> hoff(n + 1);
    std::vector<int> hidx(c->nnz);
    std::vector<uint8_t> hk(c->nnz);
    st = cuda_check(c, cudaMemcpyAsync(hx.data(), c->xyz.ptr, hx.size() * sizeof(double),
                                       cudaMemcpyDeviceToHost, c->stream), "xyz");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(hoff.data(), c->nbr_off.ptr,
                                                hoff.size() * sizeof(int64_t),
                                                cudaMemcpyDeviceToHost, c->stream), "off");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(hidx.data(), c->nbr_idx.ptr,
                                                hidx.size() * sizeof(int),
                                                cudaMemcpyDeviceToHost, c->stream), "idx");
    if (!st) st = cuda_check(c, cudaMemcpyAsync(hk.data(), codes.ptr, hk.size(),
                                                cudaMemcpyDeviceToHost, c->stream), "codes");
    if (!st) st = cuda_check(c, cudaStreamSynchronize(c->stream), "shell sync");
    buf_free(c, &codes);
    if (st) return st;
    // entries of atom i filed by shell: bucket (i, k) = sh_off[8 i + k] .. sh_off[8 i + k + 1]
    std::vector<int64_t> so(8 * (size_t)n + 1, 0);
    for (int i = 0; i < n; ++i)
      for (int64_t e = hoff[i]; e < hoff[i + 1]; ++e)
        if (hk[e]) ++so[8 * (size_t)i + hk[e]];
    for (size_t t = 1; t < so.size(); ++t) so[t] += so[t - 1];
    std::vector<int> sj(std::max<int64_t>(so.back(), 1));
    std::vector<int64_t> fill(so.begin(), so.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int64_t e = hoff[i]; e < hoff[i + 1]; ++e)
        if (hk[e]) sj[fill[8 * (size_t)i + hk[e] - 1]++] = hidx[e];
    double zm = 0.0;
    for (int i = 0; i < n; ++i) zm += hx[3 * i + 2];
    c->zmean = zm / n;
    if ((st = buf_alloc(c, &c->shell_off, so.size() * sizeof(int64_t))) ||
        (st = buf_alloc(c, &c->shell_members, sj.size() * sizeof(int))))
      return st;
    st = cuda_check(c, cudaMemcpy(c->shell_off.ptr, so.data(), so.size() * sizeof(int64_t),
                                  cudaMemcpyHostToDevice), "shell offsets");
    if (!st) st = cuda_check(c, cudaMemcpy(c->shell_members.ptr, sj.data(), sj.size() * sizeof(int),
                                           cudaMemcpyHostToDevice), "shell members");
    if (st) return st;
    // the preconditioner's pattern values (Eq. 36, p_gap taken back out) as floats
    if ((st = buf_alloc(c, &c->p_f32, std::max<int64_t>(c->nnz, 1) * sizeof(float)))) return st;
    (k_to_float<<<256, 256, 0, c->stream>>>((const double*)c->prow.ptr, c->nnz, c->pgap,
                                           (float*)c->p_f32.ptr), note_launch());
    if ((st = cuda_check(c, cudaGetLastError(), "P float"))) return st;
    c->shells_ready = true;
  }
  const int64_t len = (int64_t)frames * n;
  if ((st = buf_reserve(c, &c->ws_guess, len * sizeof(float2)))) return st;
  (k_guess_prep<<<(int)std::min<int64_t>((len + 255) / 256, 8192), 256, 0, c->stream>>>(
       len, b, b_prev, (float2*)c->ws_guess.ptr), note_launch());
  dim3 grid((n + kFeatThreads - 1) / kFeatThreads, (frames + kFeatFrames - 1) / kFeatFrames);
  (k_guess_features<<<grid, kFeatThreads, 0, c->stream>>>(
       n, frames, (const float2*)c->ws_guess.ptr, chi, (const double*)c->xyz.ptr, c->zmean,
       (const int64_t*)c->shell_off.ptr, (const int*)c->shell_members.ptr,
       (const int64_t*)c->nbr_off.ptr, (const int*)c->nbr_idx.ptr,
       (const float*)c->p_f32.ptr, feat), note_launch());
  return cuda_check(c, cudaGetLastError(), "features");
}

}  // namespace

extern "C" {

int cpm_guess_features(cpm_ctx* c, int frames, const double* b, const double* b_prev,
                       const double* chi, float* feat) {
  int st = features_async(c, frames, b, b_prev, chi, feat);
  if (st) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "features sync");
}

int cpm_guess(cpm_ctx* c, const float* params, const float* norm, int bf16, int frames,
              const double* b, const double* b_prev, const double* chi, float scale,
              const double* q_prev, double* q0) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_guess before cpm_build_E");
  if (frames < 1 || !dev_ok(c, params) || !dev_ok(c, norm) || !dev_ok(c, q_prev) ||
      !dev_ok(c, q0))
    return set_err(c, CPM_EINVAL, "cpm_guess: frames >= 1 and device arrays");
  const int64_t samples = (int64_t)frames * c->n;
  int st = buf_reserve(c, &c->ws_feat, samples * kF * sizeof(float));
  if (st) return st;
  float* feat = (float*)c->ws_feat.ptr;
  if ((st = features_async(c, frames, b, b_prev, chi, feat))) return st;
  if ((st = cuda_check(c, cudaFuncSetAttribute(k_mlp_forward,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kFwdSmem), "forward smem")))
    return st;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t tiles = (samples + kTs - 1) / kTs;
  const int blocks = (int)std::min<int64_t>(tiles, 2 * (int64_t)std::max(sms, 1));
  (k_mlp_forward<<<blocks, kFwdThreads, kFwdSmem, c->stream>>>(params, norm, bf16, samples,
                                                               feat, nullptr, scale, q_prev,
                                                               q0), note_launch());
  if ((st = cuda_check(c, cudaGetLastError(), "guess"))) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "guess sync");
}

int cpm_mlp_forward(cpm_ctx* c, const float* params, const float* norm, int bf16,
                    int64_t samples, const float* feat, float* out) {
  if (!c) return CPM_EINVAL;
  if (samples < 1 || !dev_ok(c, params) || !dev_ok(c, norm) || !dev_ok(c, feat) ||
      !dev_ok(c, out))
    return set_err(c, CPM_EINVAL, "cpm_mlp_forward: samples >= 1 and device arrays");
  int st = cuda_check(c, cudaFuncSetAttribute(k_mlp_forward,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kFwdSmem), "forward smem");
  if (st) return st;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t tiles = (samples + kTs - 1) / kTs;
  const int blocks = (int)std::min<int64_t>(tiles, 2 * (int64_t)std::max(sms, 1));
  (k_mlp_forward<<<blocks, kFwdThreads, kFwdSmem, c->stream>>>(params, norm, bf16, samples,
                                                               feat, out, 0.f, nullptr,
                                                               nullptr), note_launch());
  if ((st = cuda_check(c, cudaGetLastError(), "forward"))) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "forward sync");
}

int cpm_mlp_grad(cpm_ctx* c, const float* params, const float* norm, int bf16,
                 int64_t samples, const float* feat, const float* target, float* grad,
                 double* loss) {
  if (!c) return CPM_EINVAL;
  if (samples < 1 || !dev_ok(c, params) || !dev_ok(c, norm) || !dev_ok(c, feat) ||
      !dev_ok(c, target) || !dev_ok(c, grad) || !dev_ok(c, loss))
    return set_err(c, CPM_EINVAL, "cpm_mlp_grad: samples >= 1 and device arrays");
  int st = cuda_check(c, cudaMemsetAsync(grad, 0, kP * sizeof(float), c->stream), "grad zero");
  if (!st) st = cuda_check(c, cudaMemsetAsync(loss, 0, sizeof(double), c->stream), "loss zero");
  if (!st) st = cuda_check(c, cudaFuncSetAttribute(k_mlp_grad,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kGradSmem), "grad smem");
  if (st) return st;
  const int64_t blocks = (samples + kB - 1) / kB;
  (k_mlp_grad<<<(unsigned)blocks, kB, kGradSmem, c->stream>>>(
      params, norm, bf16, samples, 1.0 / (double)samples, feat, target, grad, loss), note_launch());
  if ((st = cuda_check(c, cudaGetLastError(), "grad"))) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "grad sync");
}

int cpm_mlp_adam(cpm_ctx* c, float* params, float* m, float* v, const float* grad, int step,
                 float lr) {
  if (!c) return CPM_EINVAL;
  if (step < 1 || !dev_ok(c, params) || !dev_ok(c, m) || !dev_ok(c, v) || !dev_ok(c, grad))
    return set_err(c, CPM_EINVAL, "cpm_mlp_adam: step >= 1 and device arrays");
  const float c1 = 1.0f / (1.0f - powf(0.9f, (float)step));
  const float c2 = 1.0f / (1.0f - powf(0.999f, (float)step));
  (k_adam<<<(kP + 255) / 256, 256, 0, c->stream>>>(params, m, v, grad, kP, lr, c1, c2), note_launch());
  return cuda_check(c, cudaGetLastError(), "adam");
}

int cpm_guess_train_step(cpm_ctx* c, float* params, const float* norm, int bf16,
                         int64_t samples, const float* feat, const float* target, float* m,
                         float* v, float* grad, double* loss, int step, float lr,
                         double* loss_out) {
  if (!c) return CPM_EINVAL;
  if (samples < 1 || step < 1 || !dev_ok(c, params) || !dev_ok(c, norm) ||
      !dev_ok(c, feat) || !dev_ok(c, target) || !dev_ok(c, m) || !dev_ok(c, v) ||
      !dev_ok(c, grad) || !dev_ok(c, loss))
    return set_err(c, CPM_EINVAL,
                   "cpm_guess_train_step: samples >= 1, step >= 1 and device arrays");
  int st = cuda_check(c, cudaMemsetAsync(grad, 0, kP * sizeof(float), c->stream), "grad zero");
  if (!st) st = cuda_check(c, cudaMemsetAsync(loss, 0, sizeof(double), c->stream), "loss zero");
  if (!st) st = cuda_check(c, cudaFuncSetAttribute(k_mlp_grad,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kGradSmem), "grad smem");
  if (st) return st;
  const int64_t blocks = (samples + kB - 1) / kB;
  (k_mlp_grad<<<(unsigned)blocks, kB, kGradSmem, c->stream>>>(
       params, norm, bf16, samples, 1.0 / (double)samples, feat, target, grad, loss),
   note_launch());
  const float c1 = 1.0f / (1.0f - powf(0.9f, (float)step));
  const float c2 = 1.0f / (1.0f - powf(0.999f, (float)step));
  (k_adam<<<(kP + 255) / 256, 256, 0, c->stream>>>(params, m, v, grad, kP, lr, c1, c2),
   note_launch());
  if ((st = cuda_check(c, cudaGetLastError(), "train step"))) return st;
  if (loss_out) {
    double l = 0.0;
    if ((st = cuda_check(c, cudaMemcpyAsync(&l, loss, sizeof(double), cudaMemcpyDeviceToHost,
                                            c->stream), "train step loss")))
      return st;
    if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "train step sync"))) return st;
    *loss_out = l / (double)samples;
    return CPM_OK;
  }
  return cuda_check(c, cudaStreamSynchronize(c->stream), "train step sync");
}

int cpm_guess_apply(cpm_ctx* c, int64_t len, const float* y, float scale, const double* q_prev,
                    double* q0) {
  if (!c) return CPM_EINVAL;
  if (len < 1 || !dev_ok(c, y) || !dev_ok(c, q_prev) || !dev_ok(c, q0))
    return set_err(c, CPM_EINVAL, "cpm_guess_apply: len >= 1 and device arrays");
  (k_guess_apply<<<256, 256, 0, c->stream>>>(len, y, scale, q_prev, q0), note_launch());
  int st = cuda_check(c, cudaGetLastError(), "guess apply");
  if (st) return st;
  return cuda_check(c, cudaStreamSynchronize(c->stream), "guess sync");
}

}  // extern "C"
