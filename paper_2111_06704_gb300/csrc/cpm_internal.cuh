// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cpm.h"

namespace cpm {

constexpr double kPi = 3.14159265358979323846;
constexpr double kKe = 14.399645478;  // V A / e

// sin and cos of 2 pi x for a fixed-point phase x = ph * 2^-32 (mod 1) to about one float
// ulp.  Converting the whole 32-bit phase to float would round it by up to 2^-25 of a
// turn (2e-7 rad); instead its top 24 bits, exact in float, go through sincospif and
// the low 8 bits (below 2^-24 of a turn, t <= 4e-7 rad) through first order, whose
// neglected t^2 / 2 is below 1e-13.
__device__ __forceinline__ void sincos_turns(uint32_t ph, float* s, float* c) {
  const int32_t p = (int32_t)ph;
  const float hi = (float)(p >> 8) * 5.9604644775390625e-08f;  // 2^-24, in [-1/2, 1/2)
  const float t = (float)(p & 255) * 1.4629180792671596e-09f;  // 2 pi 2^-32
  float s0, c0;
  sincospif(2.0f * hi, &s0, &c0);
  *c = fmaf(-s0, t, c0);
  *s = fmaf(c0, t, s0);
}

// sin and cos of 2 pi x for a fixed-point phase x = ph 2^-32 from the 4,096-entry table T
// of exp(2 pi i j / 4096) as float pairs (cos hi, cos lo, sin hi, sin lo; made in FP64)
// and the remaining angle t = 2 pi (ph mod 2^20) 2^-32 < 1.6e-3 rad by angle addition:
// cos = Tc - (t^2/2) Tc - t Ts and sin = Ts - (t^2/2) Ts + t Tc, the large term added last
// (t^4/24 < 3e-13 and t^3/6 are below float rounding of the result).  About one float
// ulp, as sincos_turns, in a third of the instructions.  sincos_entry takes the table
// entry t4 = T[ph >> 20] already loaded (from global or shared memory).
__device__ __forceinline__ void sincos_entry(float4 t4, uint32_t ph, float* s, float* c) {
  const float t = (float)(ph & 0xFFFFFu) * 1.462918119976564e-09f;  // 2 pi 2^-32
  const float h = -0.5f * t * t;
  *c = t4.x + fmaf(h, t4.x, fmaf(-t, t4.z, t4.y));
  *s = t4.z + fmaf(h, t4.z, fmaf(t, t4.x, t4.w));
}

__device__ __forceinline__ void sincos_table(uint32_t ph, const float4* __restrict__ T,
                                             float* s, float* c) {
  sincos_entry(__ldg(T + (ph >> 20)), ph, s, c);
}

// (h, l) += q x for a float pair (h, l) and q = qh + ql: the product qh x is split
// exactly (two-product) and added by an error-free two-sum, so the pair carries the sum
// to ~1e-14 relative however many terms are added.
__device__ __forceinline__ void pair_fma(float& h, float& l, float qh, float ql, float x) {
  const float p = qh * x;
  const float pe = fmaf(qh, x, -p);
  const float s = h + p;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (p - bb);
  l += e + fmaf(ql, x, pe);
  h = s;
}

struct Status {
  int code = CPM_OK;
  std::string msg;
};

// Device buffer owned by a context (allocated through the context's allocator).
struct Buf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Geometry {
  double L[3];
  double vol;
  double g;
  double rc;
  int slab;
  const uint32_t* sfix = nullptr;  // electrode fractional coordinates x 2^32, when built
};

struct Ctx {
  cpm_params p;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;

  bool built = false;
  bool solve_only = false;  // built by cpm_build_E_copy: E, P, d without the geometry's
                            // k-space tables (no potential, no guess features)
  int n = 0;        // electrode atoms
  int npad = 0;     // rows of A (multiple of 128), zero beyond n
  int m = 0;        // k-vectors
  int mpad = 0;     // k-vectors padded to a multiple of 64 (zero weight)
  int64_t ldE = 0;  // leading dimension of E (elements)
  double vol = 0;

  // geometry on device
  Buf xyz;      // double [n*3]
  Buf alpha;    // double [n]
  Buf sfix;     // uint32 [npad*3]: fractional coordinates in 2^-32 fixed point
  Buf hkl;      // int32 [mpad*3]
  Buf sqw;      // double [mpad]  sqrt(W_K), zero in the padding
  Buf flush;    // uint32 [(2*mpad/16 + 31)/32]: k-steps after which float partials flush
  int heavy_steps = 0;  // leading k-steps accumulated exactly in FP64
  int kh = 0;           // head k-vectors with an FP64 operand copy (float storage only)
  Buf Ahead;            // double [npad][2*kh], same column layout as A
  Buf chunk_end;        // uint32 bit per K-block of 64 columns (tensor-core build)
  Buf kexp;             // int per K-block: FP16 plane scale exponent (tensor-core build)
  bool streamed = false;  // A too large to keep: built in k-windows, potential direct
  int kwin = 0, kwin_n = 0, kwin_mpad = 0;  // the streamed build's k-window, fixed per geometry
  int kb6_end = 0, kb3_end = 0;  // tensor-core K-blocks: six products before kb6_end,
                                 // three before kb3_end, one after
  int kb8_begin = 0;             // K-blocks from here take one FP8 product
  Buf A;        // float/double [npad][2*mpad]
  Buf E;        // float/double [n][ldE]
  Buf diag;     // double [2n]: diag(E_n), then its reciprocal

  // PCG-DC preconditioner (row form: z_j = sum_tau P[j,tau] r_tau)
  Buf nbr_off;  // int64 [n+1]
  Buf nbr_idx;  // int32 [nnz]
  Buf prow;     // double [nnz]  (P - p_gap on the pattern when p_gap is on)
  int64_t nnz = 0;
  double pgap = 0;

  // learned-guess feature geometry (frame independent, made on first use)
  Buf turn;       // float4 [4096]: exp(2 pi i j / 4096) as float pairs (ion phasors)
  Buf shell_off;    // int64 [8n+1]: offsets of the (atom, shell 1..8) buckets in shell_members
  Buf shell_members;  // int32: members of the buckets (neighbours filed by shell)
  Buf p_f32;          // float [nnz]: PCG-DC pattern values (Eq. 36) for the guess feature
  double zmean = 0;
  bool shells_ready = false;

  Buf d;        // double [n] neutralising vector
  double c_ele = 0;
  int d_iters = 0;

  // fixed charge per electrode (GCD), made by cpm_gcd_setup, dropped by a rebuild
  int gcd_m = 0;       // electrodes; 0: not set up
  Buf gcd_labels;      // int32 [n]
  Buf gcd_a;           // double [m][n]: a^h = E_n^-1 b^h
  Buf gcd_c;           // double [m][m]: C_ab at [b * m + a]
  Buf gcd_cinv;        // double [m][m]: C^-1, row-major
  Buf gcd_status;      // int: singular C
  Buf gcd_scratch;        // double: per-frame sums and shifts

  // the matrix path: S = E_n^-1 (I - 1 d^T), column-major (S_ij at [j * n + i])
  bool smat_ready = false;
  Buf smat;            // double [n][n]

  // scratch (grown on demand, never shrunk)
  std::vector<Buf*> scratch;
  std::vector<double> kw;  // k-vector weights W_K of the sorted table, mpad entries (0 past m)
  std::vector<int> kv_hkl;    // the k-vector table (host), made on the first build
  std::vector<double> kv_w;
  Buf ws_solve, ws_in0, ws_in1, ws_in2, ws_out0, ws_out1, ws_pot, ws_guess, ws_feat;
  Buf ws_cluster;  // per-column results of the cluster-resident solve
  // the solver's online autotuner: per bucket of right-hand-side counts (1, 2-3, 4-7, ..,
  // 128+), the path found faster (0 not yet known, 1 host-driven kernels, 2 cluster-
  // resident) and the measured device time per iteration of each path (reset by a build)
  int tune_path[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float tune_cost[8][2] = {};
  int last_solve_path = 0;
  // tensor-core build workspace, kept for the next build: operand planes, the FP64
  // head matrix, the error flag, the head's float pairs, the per-SM hi / lo scratch
  Buf tc_planes[4], tc_head, tc_err, tc_hsplit, tc_scratch;  // planes 0-2: 16-bit, 3: FP8
  Buf tc_tiles;       // the tile kernels' tile order, for tc_tiles_nt row blocks
  int tc_tiles_nt = 0;
  Buf dc_cnt, dc_pcol, dc_status;  // PCG-DC build workspace
  int nsmid = 0;  // SM slots of tc_scratch (%nsmid), queried once

  float t_kspace_ms = 0, t_phase_ms = 0, t_precond_ms = 0, t_dsolve_ms = 0, t_tc_ms = 0;
  float t_matvec_ms = 0;  // last cpm_apply_E: the matvec launches alone
  float t_head_ms = 0;    // FP64-accurate head of the tensor-core build
  float t_light_ms = 0;   // tensor-core tail: the three- and one-product K-blocks
  float t_tc_loop_ms = 0; // the tail's window loop (streamed builds: operand planes too)
  // last PCG solve: its device time, that of its matvec launches (fast or exact), of its
  // residual replacements, and their count
  float t_solve_ms = 0, t_solve_mv_ms = 0, t_solve_rep_ms = 0, t_solve_dc_ms = 0;
  int solve_replacements = 0;
  std::vector<cudaEvent_t> ev_pool;  // timing events of the solve, made on first use
  // last cpm_potential: the ions' structure factors, the k-space contraction, the real
  // space with the finish (device time)
  float t_pot_sf_ms = 0, t_pot_kspace_ms = 0, t_pot_real_ms = 0;
  std::vector<cudaEvent_t> ev_pot;
  cudaEvent_t ev_tc[3] = {nullptr, nullptr, nullptr};

  bool fp64() const { return p.precision == CPM_PREC_FP64; }
  size_t esz() const { return fp64() ? 8 : 4; }
};

// ---- kernel launch count (every launch site calls note_launch) ---------------------
void note_launch();
long long launch_count();

// ---- allocation (ctx.cu) -----------------------------------------------------------
int buf_alloc(Ctx* c, Buf* b, size_t bytes);
void buf_free(Ctx* c, Buf* b);
int buf_reserve(Ctx* c, Buf* b, size_t bytes);  // grow-only
int set_err(Ctx* c, int code, const std::string& msg);
int cuda_check(Ctx* c, cudaError_t e, const char* what);
// Where the array at p lives: 1 in device memory of the context's device (or managed
// memory), 0 in host memory (or p is null), -1 in device memory of another device.
int pointer_where(const Ctx* c, const void* p);
// *dev = whether p is device memory the context's kernels may use; CPM_EINVAL (with a
// message) when it is device memory of another device.
int on_device(Ctx* c, const void* p, bool* dev);

// ---- kernels (launchers) -----------------------------------------------------------
// kspace.cu
void launch_fixed_point_coords(const double* xyz, int n, int npad, const double L[3],
                               uint32_t* sfix, cudaStream_t s);
// k-vectors [kbeg, kend) (multiples of 64): A (if not null) and the BF16 planes (if not
// null) over that window
void launch_structure_operand(bool fp64, const double* xyz, const uint32_t* sfix, int npad,
                              int n, const int* hkl, const double* sqw, int mpad,
                              const double L[3], void* A, void* const* planes, int kb0,
                              int kb6, int kb3, int kb8, const int* kexp, const void* turn,
                              int kbeg, int kend, cudaStream_t s);
void launch_structure_operand_head(const double* xyz, int npad, int n, const int* hkl,
                                   const double* sqw, int kh, const double L[3], double* Ahead,
                                   cudaStream_t s);
int launch_ek_simt(bool fp64, const void* A, int npad, int mpad, const double* xyz,
                   const double* alpha, int n, const Geometry& geo, void* E, int64_t ldE,
                   int heavy_steps, const uint32_t* flush_mask, cudaStream_t s);
void launch_mirror_lower(bool fp64, void* E, int n, int64_t ldE, cudaStream_t s);

int launch_ek_head_f64(const double* Ahead, int kh, int ktot, int npad, float* hi, float* lo,
                       const double* xyz, const double* alpha, int n, const Geometry& geo,
                       float2* Ehead, int64_t ldE, cudaStream_t s);

// tc_syrk.cu
int launch_ek_tc(const void* p0, const void* p1, const void* p2, const void* p8, int npad,
                 int64_t plane_cols, int kb_col0, int n, int kb_begin, int kb_end, int kb6_end,
                 int kb3_end, int kb8_begin,
                 const uint32_t* chunk_end, const int* kexp, float2* head, int64_t ldh,
                 float* E, int64_t ldE, int* err, const double* kw, float* scratch,
                 int scratch_slots, const uint32_t* tile_map, cudaEvent_t mid,
                 cudaStream_t s);
std::vector<uint32_t> ek_tile_order(int nt);  // the tile kernels' tile order (host)
int64_t ek_strip_scratch_floats();  // per SM slot of the 256 x 256 tile kernels
void launch_nsmid(int* d_out, cudaStream_t s);
void launch_extract_diag(bool fp64, const void* E, int n, int64_t ldE, double* diag,
                         cudaStream_t s);
void launch_get_E(bool fp64, const void* E, int n, int64_t ldE, const double* xyz,
                  const Geometry& geo, int paper_form, const int* rows, int nrows, double* out,
                  int64_t ld, cudaStream_t s);

// potential.cu
void launch_ion_fixed(const double* ion_xyz, int frames, int n_ion, const double L[3],
                      uint32_t* sion, cudaStream_t s);
void launch_turn_table(void* T, cudaStream_t s);
void launch_ion_structure_factor(bool fp64, const double* ion_xyz, const uint32_t* sion,
                                 const double* ion_q, int frames, int n_ion, const int* hkl,
                                 const double* sqw, int mpad, int kh, const double L[3],
                                 const void* turn, void* v, double* vhead, cudaStream_t s);
void launch_bsol_kspace(bool fp64, const void* A, const double* Ahead, int n, int mpad, int kh,
                        const void* v, const double* vhead, int frames, double* bsol,
                        const uint32_t* sfix, const int* hkl, const double* sqw,
                        const void* turn, int nsplit, double* split_part, cudaStream_t s);
// shares of the k range of a streamed build's direct k-space sum (split_part then holds
// nsplit x frames x n doubles)
int bsol_direct_splits(int n, int frames, int mpad, int kh, int sms);
void launch_bsol_real_and_finish(const double* xyz, const double* alpha, const uint32_t* sfix,
                                 int n, const double* ion_xyz, const double* ion_q,
                                 const uint32_t* sion, int frames, int n_ion,
                                 const Geometry& geo, const double* chi, const double* bsol_k,
                                 double* b_out, double* qsol, bool far_float, cudaStream_t s);

void launch_ion_forces(const double* xyz, const double* alpha, const uint32_t* sfix, int n,
                       const double* ion_xyz, const double* ion_q, const uint32_t* sion,
                       int frames, int n_ion, const double* q, const int* hkl,
                       const double* sqw, int mpad, int kh, const Geometry& geo,
                       const void* turn, const float* v, const double* vhead, double* grad,
                       double* out, cudaStream_t s);

// pcg.cu
// One system of a ragged batch: a right-hand side with its own (float) matrix, size and
// preconditioner.  Vectors of the batch are laid out [system][ld], zero past n.
struct SysCol {
  const float* E;
  int64_t ldE;
  int n;
  const int64_t* nbr_off;  // PCG-DC pattern (row form) and values, p_gap
  const int* nbr_idx;
  const double* prow;
  double pgap;
  const double* inv_diag;  // Jacobi
  const double* d;         // neutralising vector
};

struct SolveArgs {
  int nrhs;
  const double* b;   // [nrhs*n]; multiplied by bscale to give e/A
  double bscale;
  double* x;         // [nrhs*n]
  bool use_guess;
  double tol;
  int maxit;
  int* iters;        // host [nrhs]
  double* relres;    // host [nrhs]
  void* ws = nullptr;    // optional fixed device workspace (else the context's, grown)
  size_t ws_bytes = 0;
  const SysCol* sys = nullptr;  // ragged batch: device array [nrhs], one system per column
  bool timed = true;             // record the solve's device timings (events of the context)
};
int pcg_solve(Ctx* c, const SolveArgs& a);
// pcg_cluster.cu: the whole solve in one launch, one cluster per right-hand side
// (CPM_EINVAL when the context does not fit it)
int pcg_solve_cluster(Ctx* c, const SolveArgs& a);
int cluster_solve_max_atoms();
int apply_E(Ctx* c, int nrhs, const double* p, double* q);  // device arrays [nrhs][n]
void launch_neutralize(double* q, int nrhs, int n, const double* d, const double* qsol,
                       cudaStream_t s);
// ragged batch: q [count][ld], system c neutralised with its own d over its n
void launch_neutralize_ragged(double* q, int count, int64_t ld, const SysCol* sys,
                              const double* qsol, cudaStream_t s);

// dc.cu
int build_dc_preconditioner(Ctx* c);
int build_sparse_inverse(Ctx* c);  // PCG-Normal / PCG-Full
int copy_precond(Ctx* c, int64_t* off, int* idx, double* val);
int apply_p_gap(Ctx* c);
int device_sum(Ctx* c, const double* v, int64_t len, double* out);

// ---- fixed charge per electrode, GCD (gcd.cu) -------------------------------------
void launch_gcd_indicators(const int* labels, int n, int m, double* bh, cudaStream_t s);
void launch_gcd_sums(const double* x, int n, int nvec, const int* labels, int m, double* out,
                     cudaStream_t s);
void launch_gcd_invert(const double* ct, int m, double* cinv, int* status, cudaStream_t s);
void launch_gcd_shifts(const double* cinv, const double* q0, const double* sums, int nrhs,
                       int m, double* dmu, double* dmu_volts, cudaStream_t s);
void launch_gcd_apply(double* q, const double* amat, const double* dmu, int n, int nrhs, int m,
                      cudaStream_t s);

// ---- the matrix path (smatrix.cu) --------------------------------------------------
int smatrix_max_frames();
void launch_identity(double* x, int n, cudaStream_t s);
void launch_smatrix_form(double* x, const double* d, double c_ele, int n, cudaStream_t s);
void launch_smatrix_apply(const double* S, const double* b, const double* qsol, const double* d,
                          int n, int frames, double bscale, double* q, cudaStream_t s);

}  // namespace cpm
