/*
 * cpm.h -- C ABI of the GB300 SR-CPM electrode-charge library (libcpm.so).
 *
 * The library computes the electrode charges of the Siepmann-Sprik / Reed constant
 * potential method as reformulated by Li, Wang, Liu & Jiang (arXiv 2111.06704):
 *
 *   cpm_build_E     the Gaussian Ewald interaction matrix E of the electrode atoms
 *                   (Sec. II C, Eq. 22-23; slab correction Eq. 39), the PCG-DC
 *                   preconditioner (Sec. III B 2, Eq. 36-37) and the neutralising
 *                   vector d (Eq. S8-S9);
 *   cpm_potential   the extrinsic potential b = chi - b^sol on every electrode atom
 *                   (Eq. 25) for one or many electrolyte frames;
 *   cpm_solve       the first step of the two-step method, E q^b = b, by
 *                   preconditioned conjugate gradient (Sec. III B 2);
 *   cpm_neutralize  the second step q = q^b - (Q^b + Q^sol) d (Eq. 35).
 *
 * Units: positions in Angstrom, charges in e, chi and b in volts.  E is kept in
 * Gaussian units (1/A); volts convert with k_e = 14.399645478 V A / e.
 *
 * Neutral-equivalent form.  Eq. 39 expands to -(2 pi/V)(z_i^2 + z_j^2) + (4 pi/V) z_i z_j
 * - (2 pi/V) Lz^2/6 and the Ewald constant -pi/(V g^2) is the same for every pair.  The
 * library stores E_n = E + pi/(V g^2) + (2 pi/V)(z_i^2 + z_j^2 + Lz^2/6), i.e. it keeps
 * the dipole term (4 pi/V) z_i z_j and drops the rank-2 remainder u 1^T + 1 u^T + k0 1 1^T.
 * For charges with 1^T q = -Q^sol that remainder only adds a multiple of 1 (absorbed by
 * the multiplier mu_c of Eq. 29-30) and a -Q^sol u term that the matching Q^sol z_i^2
 * term of b^sol cancels, so the neutral charges of Eq. 35 are unchanged.  E_n is
 * symmetric positive definite; the literal E is indefinite along 1 for slabs, which
 * conjugate gradient cannot handle.  cpm_potential returns b in the same form.
 *
 * Pointers: every array argument may be a host pointer or a CUDA device pointer of the
 * context's device (detected with cudaPointerGetAttributes; device memory of another
 * device is rejected with CPM_EINVAL).  The caller owns them; the
 * library never keeps them past the call.  Host arrays are staged through device
 * buffers inside the call.  Layouts are row-major and contiguous.
 *
 * Synchronisation: every call is ordered on the context's stream and returns after its
 * results are complete (the call synchronises that stream before returning).
 *
 * Errors: every call returns CPM_OK (0) or a negative status; cpm_last_error() gives a
 * message.  No call aborts or exits the process.  A context is not thread safe.
 */
#ifndef CPM_H
#define CPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define CPM_OK 0
#define CPM_EINVAL (-1)      /* bad argument (size, pointer, parameter) */
#define CPM_ENOMEM (-2)      /* device allocation failed */
#define CPM_ECUDA (-3)       /* a CUDA runtime or driver call failed */
#define CPM_ENOCONV (-4)     /* maxit reached: q holds the last iterate, relres is set */
#define CPM_EBREAKDOWN (-5)  /* p^T E p <= 0 or a non-finite value in the iteration */
#define CPM_ENOTBUILT (-7)   /* cpm_build_E has not succeeded on this context */
#define CPM_EIO (-8)         /* a file could not be written or read, or is not a valid one */

/* ---- precision of the E build and of the solve ----------------------------------- */
#define CPM_PREC_FP64 0    /* FP64 phases, FP64 structure-factor GEMM, FP64 E and matvec */
#define CPM_PREC_FP32 1    /* exact fixed-point phases, FP32 SIMT GEMM with K-chunks
                              summed in FP64, FP32 E, FP32 matvec with FP64 reductions */
#define CPM_PREC_BF16X6 2  /* as FP32, but the GEMM runs on tcgen05 tensor cores: six
                              products of a three-way BF16 split of each operand for
                              the heavy k-vectors, three or one FP16 or one FP8 product
                              of scaled operands for the light ones (cpm_plan_kspace) */

/* ---- preconditioners (Sec. III B 2) ----------------------------------------------- */
#define CPM_PRECOND_NONE 0    /* conventional CG */
#define CPM_PRECOND_JACOBI 1  /* diag(E)^-1: the plain baseline */
#define CPM_PRECOND_DC 2      /* PCG-DC: columns of local inverses M_tau^-1 (Eq. 36) */
#define CPM_PRECOND_NORMAL 3  /* PCG-Normal (Fig. 6a): the entries of E^-1 for the pairs
                                 with r < rcut_dc (minimum image), zero elsewhere */
#define CPM_PRECOND_FULL 4    /* PCG-Full (Fig. 6a): the entries of E^-1 for the pairs
                                 with r <= rcut_real.  Normal and Full find E^-1 by one
                                 Jacobi-preconditioned solve over the n identity columns
                                 at build time (n <= CPM_SMATRIX_MAX_ATOMS) */

/* ---- forms for cpm_get_E ----------------------------------------------------------- */
#define CPM_E_STORED 0  /* the stored neutral-equivalent E_n */
#define CPM_E_PAPER 1   /* E of Eq. 22 with Eq. 39, rebuilt from E_n by adding the
                           rank-2 remainder back */

typedef struct cpm_params {
  double box[3];       /* orthorhombic periodic cell edges Lx, Ly, Lz (A) */
  double g_ewald;      /* Ewald splitting parameter (the paper's eta, Eq. 12), 1/A */
  double rcut_real;    /* real-space cutoff (A); every image within it is summed */
  double kspace_eps;   /* reciprocal cutoff Kc = 2 g sqrt(ln(1/eps)) */
  int slab;            /* 1: Yeh-Ballenger slab correction of Eq. 39 */
  int precision;       /* CPM_PREC_* */
  int precond;         /* CPM_PRECOND_* */
  double g_dc;         /* PCG-DC screening factor g of Eq. 36 (1/A) */
  double rcut_dc;      /* PCG-DC neighbour cutoff r_cut (A), inclusive */
  int p_gap;           /* 1: fill the zeros of P with p_gap (Eq. 37) */
  void* stream;        /* cudaStream_t for every call; NULL = the legacy default stream */
  /* Optional device allocator (e.g. the PyTorch caching allocator).  NULL = cudaMalloc.
     alloc returns NULL on failure; free receives the pointers alloc returned. */
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* alloc_user;
  /* Operand streaming (BF16X6 builds): the structure-factor operand A is kept resident
     when it fits 32 GiB, otherwise the build makes its BF16 planes k-window by k-window
     (about 12 GB of planes at a time) and cpm_potential sums the k-space part directly
     from the electrode phases.  stream_operand: 0 automatic, 1 always.  k_window:
     k-vectors per window (rounded down to a multiple of 64), 0 automatic. */
  int stream_operand;
  int k_window;
  /* Matvec of solves with two or more right-hand sides of a float-stored E:
     0 (default): the inner iterations apply E to every group of 16 columns in one pass
     with float products and sums (~1e-6 of the row's partial sums), and the true
     residual b - E x, through the error-free matvec below, replaces the recursive one
     whenever a column's residual has fallen 100-fold since its last replacement or it
     reports convergence: a column converges on its true residual only.
     1: every matvec error-free (products split exactly, float-pair sums; up to four
     columns per pass over E).  One right-hand side always takes the error-free matvec. */
  int matvec_mode;
  /* How a solve runs.  0 (default): chosen per context by its online autotuner for each
     bucket of right-hand-side counts (1, 2-3, 4-7, .., 128 and more): the first eligible
     solve of a bucket runs on the cluster path, the next on the kernel path, each timed
     per iteration on the device, and later solves take the faster (a build resets it).
     1: the kernel path: a few kernels an iteration, the host polling convergence every
     four iterations (every size, every precision, ragged batches).  2: the cluster path:
     the whole solve in one launch, one thread-block cluster of 8 CTAs per right-hand
     side, for float storage and n <= 4,096 (larger or FP64 contexts take the kernel
     path).  cpm_solve_static always takes the kernel path. */
  int solver_path;
} cpm_params;

typedef struct cpm_ctx cpm_ctx;

/* Fills p with the defaults: g 0.3, rcut 12, eps 1e-8, slab 1, BF16X6, PCG-DC with
 * g_dc 0.083 and r_cut 8 (Sec. IV A), p_gap 1, default stream, cudaMalloc.  The box
 * is left zero and must be set. */
void cpm_default_params(cpm_params* p);

/* Creates a context on the current CUDA device.  *out receives the handle. */
int cpm_create(cpm_ctx** out, const cpm_params* p);
int cpm_destroy(cpm_ctx* c);

/*
 * Builds everything that depends only on the electrode geometry (done once per
 * geometry; the electrode coefficients are invariant during MD, Sec. III A):
 *  - the half-space k-vector table: K = 2 pi (h/Lx, k/Ly, l/Lz) != 0, |K| <= Kc,
 *    weights W_K = 2 (4 pi/V) exp(-K^2/4g^2) / K^2 (Eq. 13, Eq. 20);
 *  - the structure-factor operand A = [sqrt(W) cos(K.r_i) | sqrt(W) sin(K.r_i)] and
 *    the reciprocal part of E as A A^T (Eq. 23 with cos(K.(r_i - r_j)) split by the
 *    angle-addition formula);
 *  - in the same pass, the real-space part, the diagonal self terms and the slab
 *    dipole term of Eq. 22 / Eq. 39 (neutral-equivalent form, see above);
 *  - the PCG-DC preconditioner (if selected) and d = d' / (1^T d'), E_n d' = 1.
 * n: electrode atoms (1 <= n).  xyz[n*3]: positions (A).  alpha[n]: Gaussian inverse
 * widths (1/A) of Eq. 4; INFINITY marks a point charge (no self-energy, Sec. II C).
 * Replaces any earlier build on the context.  Device buffers of the earlier build are
 * reused where large enough; the BF16X6 build's workspace (its 16-bit operand planes,
 * up to 12 bytes per electrode atom and k-vector, the FP64 head matrix of 8 N^2 bytes,
 * and a 512 KB scratch slot per SM) is kept for the next build until
 * cpm_release_workspace or cpm_destroy.
 */
int cpm_build_E(cpm_ctx* c, int n, const double* xyz, const double* alpha);

/*
 * cpm_build_E_copy: builds dst from the built E of src instead of from the geometry.  No
 * counterpart in the paper: it serves the plain FP64 PCG baseline on electrodes where an
 * FP64 k-space build is out of reach (at 106,568 atoms the FP64 E takes 91 GB and its
 * FP64 GEMM some 4e15 FLOP at the FP64 rate).  dst gets src's stored E_n in dst's
 * storage precision (float to FP64 is an exact widening; equal precisions copy), src's
 * diagonal, d and C^ele, and, when dst selects PCG-DC, src's PCG-DC preconditioner (src
 * must have one with the same g_dc, rcut_dc and p_gap).  Jacobi and no preconditioner
 * need nothing more.  Both contexts on one device, with the same box, g, r_c, eps and
 * slab setting, else CPM_EINVAL; an FP64 src cannot be narrowed (CPM_EINVAL).  dst then
 * serves cpm_solve, cpm_solve_static, cpm_neutralize, cpm_apply_E, cpm_get_E(_rows),
 * cpm_get_d, cpm_get_precond, the GCD and matrix-path calls; it has no k-space tables, so
 * cpm_potential and the learned-guess feature calls return CPM_EINVAL (compute b on src).
 * Replaces dst's earlier build; src is left as it was (its stream is synchronised first).
 * dst holds its own copies: src may be rebuilt or destroyed afterwards.
 */
int cpm_build_E_copy(cpm_ctx* dst, cpm_ctx* src);

/* Frees the context's kept workspace: the E build's (above) and the solve and potential
 * workspaces, which later calls reserve again as needed.  The built E, P, d and the
 * operand A stay.  Waits for the context's stream first.  No counterpart in the paper:
 * device-memory management of this library. */
int cpm_release_workspace(cpm_ctx* c);

/*
 * The host plan of the k-space sum of cpm_build_E for the parameters p: host arithmetic
 * only, no context, build or GPU.
 *  - The k-vector table of Eq. 13 / Eq. 20 (as above) in the build's order, decreasing
 *    weight W_K (ties keep the h, k, l loop order).
 *  - The head: the leading operand columns (cos and sin halves of 64 k-vectors per 128
 *    columns) that the build sums in float-float (BF16X6) or FP64 (FP32) arithmetic.
 *  - For BF16X6, the tail after the head in K-blocks of 64 operand columns (block b:
 *    the cos (b even) or sin (b odd) half of k-vectors 64 (b / 2) ..): each block's
 *    product format, its power-of-two operand scale 2^kexp and the blocks that end an
 *    accumulation chunk.  Each format's region is the longest run of trailing blocks
 *    whose summed bound 64 max W_K times the format's error per product stays within
 *    1e-8 (E4M3: 0.13, one FP16 product: 2^-10 + 2^-23, three: 5 x 2^-22), region ends
 *    rounded up to even blocks; six BF16 products before them.
 * out: sizes and region bounds.  hkl[3 m] (h, k, l per k-vector), w[m] (W_K, 1/A),
 * kexp[kb_end] and chunk_end[kb_end] (1 where a chunk ends): host arrays, filled when not
 * NULL (call once with NULL arrays for the sizes).  CPM_EINVAL for a NULL p or out or
 * parameters cpm_create rejects.
 */
typedef struct cpm_kspace_plan {
  int m;          /* k-vectors in the table */
  int m_pad;      /* m rounded up to 64 (the operand has 2 m_pad columns) */
  int head_cols;  /* leading operand columns summed in float-float / FP64 */
  int kb_begin;   /* first K-block of the tail: head_cols / 64 */
  int kb6_end;    /* six BF16 products in [kb_begin, kb6_end) */
  int kb3_end;    /* three FP16 products in [kb6_end, kb3_end) */
  int kb8_begin;  /* one FP16 product in [kb3_end, kb8_begin), one E4M3 product after */
  int kb_end;     /* 2 m_pad / 64 */
  int chunks;     /* accumulation chunks of the tail */
} cpm_kspace_plan;

int cpm_plan_kspace(const cpm_params* p, cpm_kspace_plan* out, int* hkl, double* w,
                    int* kexp, uint8_t* chunk_end);

/*
 * b = chi - k_e * b^sol for `frames` electrolyte frames (Eq. 25), in the
 * neutral-equivalent form: b^sol_i = sum_I q_I [real + reciprocal part of e_iI with
 * the point-Gaussian coefficient alpha_i] + (4 pi/V) z_i sum_I q_I z_I (slab).
 * ion_xyz[frames*n_ion*3] (A), ion_q[frames*n_ion] (e), chi[n] (V, shared by all
 * frames).  b_out[frames*n] (V).  qsol_out[frames] (may be NULL) receives
 * Q^sol = sum_I q_I of each frame.  n_ion may be 0.
 */
int cpm_potential(cpm_ctx* c, int frames, int n_ion, const double* ion_xyz,
                  const double* ion_q, const double* chi, double* b_out, double* qsol_out);

/*
 * Forces on the electrolyte ions from the electrode charges: F_I = -q_I d/dr_I
 * sum_i q_i e_iI(alpha_i), with e_iI the point-Gaussian coefficient of Eq. 25 in the
 * paper's form (real space with the Gaussian's own terms of Eq. S25, reciprocal space,
 * and the slab term of Eq. 39; the constants drop out).  ion_xyz[frames*n_ion*3] (A),
 * ion_q[frames*n_ion] (e), q[frames*n] the electrode charges (e, e.g. cpm_neutralize's),
 * f_out[frames*n_ion*3] in e^2/A^2 (times k_e = 14.399645478 for eV/A).  Real space in
 * FP64 over every image within r_c; the reciprocal part from the electrode's
 * charge-weighted structure factors (head k-vectors in FP64, the rest in float phasors
 * with error-free float-pair sums).  Not a step of the charge solve: what the charges do to
 * the ions in an MD step (Supplementary Note, Eq. S25).
 */
int cpm_ion_forces(cpm_ctx* c, int frames, int n_ion, const double* ion_xyz,
                   const double* ion_q, const double* q, double* f_out);

/*
 * First step of Eq. 35: solves E_n q^b = b / k_e for nrhs right-hand sides by
 * (preconditioned) conjugate gradient.  The PCG-DC preconditioner is not symmetric, so
 * the flexible (Polak-Ribiere) beta is used with it.
 * b[nrhs*n] (V).  q_inout[nrhs*n] (e): with use_guess != 0 it holds the initial guess
 * (e.g. the previous MD step, Eq. 26), else the guess is zero; on return it holds q^b.
 * Stops when ||b - E_n q||_2 / ||b||_2 <= tol for every column, or after maxit
 * iterations (CPM_ENOCONV).  iters_out[nrhs] and relres_out[nrhs] may be NULL.
 */
int cpm_solve(cpm_ctx* c, int nrhs, const double* b, double* q_inout, int use_guess,
              double tol, int maxit, int* iters_out, double* relres_out);

/*
 * cpm_solve_static: the same first-step solve as cpm_solve, but it allocates no device
 * memory.  The paper has no counterpart; this variant is for callers that cannot call
 * cudaMalloc at solve time -- an MD engine that has reserved the device for its own
 * memory pool, a host program that forbids allocation after start-up, or a time step
 * that must not stall on an allocation.  cpm_solve grows a per-context workspace on
 * demand; this call instead runs the same kernels on a fixed workspace of
 * CPM_STATIC_SCRATCH_BYTES held in a file-scope device array, which every device that
 * loads the library keeps until the process exits.
 * b[nrhs*n] and q_inout[nrhs*n] must be device pointers (staging host arrays would
 * allocate); other arguments as for cpm_solve.  Returns CPM_EINVAL when the problem
 * (n rounded up to 128, times nrhs) needs more workspace than the array holds, or when a
 * pointer is on the host.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture.  All calls share the array and each call clears what must
 * start at zero; calls whose work overlaps on the GPU race, so serialise them.
 */
#define CPM_STATIC_SCRATCH_BYTES (8u * 1024u * 1024u)
int cpm_solve_static(cpm_ctx* c, int nrhs, const double* b, double* q_inout, int use_guess,
                     double tol, int maxit, int* iters_out, double* relres_out);

/*
 * Second step of Eq. 35 for nrhs columns: q <- q - (sum_i q_i + Q^sol) d, so that
 * sum_i q_i = -Q^sol (Eq. 34).  qsol[nrhs] may be NULL (Q^sol = 0).
 */
int cpm_neutralize(cpm_ctx* c, int nrhs, double* q_inout, const double* qsol);

/* ---- fixed total charge per electrode (GCD) -------------------------------------- */
#define CPM_GCD_MAX_ELECTRODES 16

/*
 * Galvanostatic charge-discharge constraint (Supplementary Note, Eq. S14-S24): the
 * electrode atoms form m electrodes, each holding a given total charge Q_a^0 while its
 * atoms share one potential shift Delta mu_a.  An alternative second step to
 * cpm_neutralize; the first step stays cpm_solve.
 *
 * cpm_gcd_setup: labels[n] (host or device) assigns atom i to electrode labels[i] in
 * 0 .. m-1, 1 <= m <= CPM_GCD_MAX_ELECTRODES, no electrode empty.  Solves
 * E a^h = b^h (b^h one on electrode h, Eq. S22-S23) for the m electrodes by the
 * context's PCG to the relative residual tol within maxit iterations, forms the
 * capacitance coefficients C_ab = sum over the atoms of electrode a of a^b_i (Eq. S24),
 * and inverts C.  Kept until the next cpm_build_E, which drops it.  c_out[m*m] (host or
 * device, optional) receives C in e/V, row a, column b.  These are the coefficients of
 * the stored neutral-equivalent E_n.  What charges of zero net sum see of them is the
 * paper's, e.g. the joint capacitance (C_aa C_bb - C_ab^2) / sum_ab C_ab of Eq. S21;
 * C_E itself is not.  iters_out[m], relres_out[m]: optional host arrays.
 * CPM_EINVAL for bad labels or arguments, CPM_ENOCONV if a solve misses tol,
 * CPM_EBREAKDOWN if C is singular to working precision.
 *
 * cpm_gcd_charges: q_inout[nrhs*n] holds q^b = E^-1 b from cpm_solve on entry and the
 * GCD charges on exit, q = q^b + A C^-1 (Q^0 - B^T q^b) (Eq. S16-S20), with
 * A = (a^1 .. a^m) and B the indicator columns.  q0[nrhs*m] (host or device): Q_a^0 per
 * frame (e).  E_n stands in for E only for charges of the right net sum, so each frame's
 * totals must balance its electrolyte charge: |sum_a q0[f*m + a] + qsol[f]| at most 1e-9
 * of max(1, sum_a |q0[f*m + a]| + |qsol[f]|) (qsol from cpm_potential; NULL = 0), else
 * CPM_EINVAL.  dmu_out[nrhs*m] (optional, host or device) receives Delta mu_a in volts,
 * up to one constant per frame that the form of E shifts; differences between
 * electrodes are the paper's.  CPM_EINVAL before cpm_gcd_setup.
 */
int cpm_gcd_setup(cpm_ctx* c, int m, const int* labels, double tol, int maxit, double* c_out,
                  int* iters_out, double* relres_out);
int cpm_gcd_charges(cpm_ctx* c, int nrhs, double* q_inout, const double* q0,
                    const double* qsol, double* dmu_out);

/* ---- the matrix path for a small fixed electrode ---------------------------------- */
#define CPM_SMATRIX_MAX_ATOMS 8192

/*
 * The paper's matrix alternative to the iterative solve (Eq. 33 with Eq. 35): S =
 * E^-1 (I - 1 d^T), formed once per geometry, after which a frame's neutral charges are
 * one dense product, q = S b - Q^sol d, with no iteration.
 *
 * cpm_smatrix_build: forms S from the n columns E^-1 e_j, which the context's PCG solves
 * to the relative residual tol within maxit iterations (n right-hand sides at once).
 * S takes 8 n^2 bytes and is kept until the next cpm_build_E, which drops it.
 * n <= CPM_SMATRIX_MAX_ATOMS.  max_iters_out (optional): the most iterations a column
 * took.  CPM_EINVAL for n above the limit or bad arguments, CPM_ENOCONV if a column
 * misses tol.
 *
 * cpm_smatrix_charges: b[frames*n] in volts (as cpm_potential returns it), qsol[frames]
 * (NULL = 0), q_out[frames*n]: the neutral charges (e), as cpm_solve followed by
 * cpm_neutralize give them to the solve's tolerance.  All host or device.  CPM_EINVAL
 * before cpm_smatrix_build.
 */
int cpm_smatrix_build(cpm_ctx* c, double tol, int maxit, int* max_iters_out);
int cpm_smatrix_charges(cpm_ctx* c, int frames, const double* b, const double* qsol,
                        double* q_out);

/* ---- learned initial guess ------------------------------------------------------------
 * The paper has no learned component; the warm start it describes is the previous MD
 * step's charges (Eq. 26).  These calls add a small per-atom network that predicts the
 * change of the first-step charges q^b between consecutive frames from local features of
 * the potential, so PCG can start from q_prev + scale * net(features).  The converged
 * residual judges every guess, so accuracy is never traded.  All arrays are device
 * pointers.  Network: 32 -> 64 -> 64 -> 64 -> 1 with SiLU on the hidden layers;
 * parameters as one FP32 vector [W1 (64x32), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (64),
 * b4]; with bf16 != 0 the weights are used rounded to BF16, accumulation in FP32.
 * norm[64] holds a per-feature mean then inverse standard deviation. */
#define CPM_MLP_FEATURES 32
#define CPM_MLP_PARAMS 10497

/* Features of every atom of `frames` frames from their potentials b[frames*n] (V) and
 * the previous frames' b_prev[frames*n]: Delta b_i, the means of Delta b over the
 * neighbour shells k - 1/2 <= r < k + 1/2 (k = 1..8), b_i and its shell means, chi_i,
 * the side of the electrode (+1 above the mean height) and 12 zeros.
 * feat[frames*n*32] (float).  Needs a PCG-DC build (its neighbour lists, r <= rcut_dc). */
int cpm_guess_features(cpm_ctx* c, int frames, const double* b, const double* b_prev,
                       const double* chi, float* feat);

/* out[s] = net((feat[s] - mean) * inv_std) for s < samples. */
int cpm_mlp_forward(cpm_ctx* c, const float* params, const float* norm, int bf16,
                    int64_t samples, const float* feat, float* out);

/* grad[CPM_MLP_PARAMS] = gradient of (1/samples) sum_s (net(x_s) - target_s)^2 and
 * *loss = sum_s (net(x_s) - target_s)^2 (both overwritten). */
int cpm_mlp_grad(cpm_ctx* c, const float* params, const float* norm, int bf16,
                 int64_t samples, const float* feat, const float* target, float* grad,
                 double* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected for `step` >= 1). */
int cpm_mlp_adam(cpm_ctx* c, float* params, float* m, float* v, const float* grad, int step,
                 float lr);

/* The network's initial parameters into params[CPM_MLP_PARAMS] (device): the weights of a
 * layer with i inputs uniform in [-sqrt(6/i), sqrt(6/i)) (the output layer's times 0.1,
 * so that the first guesses stay near the previous step's charges), biases zero.  Weight
 * k is drawn from output number k of a SplitMix64 stream seeded with `seed` (its top 53
 * bits as a uniform in [0, 1)), so the same seed gives the same network on any device. */
int cpm_guess_init(cpm_ctx* c, uint64_t seed, float* params);

/* The feature normalisation and the target scale from `samples` training samples:
 * norm[64] (host or device) receives each feature's mean, then its inverse standard
 * deviation (0 for a feature constant over the samples); *target_scale (host) the
 * standard deviation of target[samples] (1 if it is 0).  feat[samples*32] and
 * target[samples] are device arrays; the sums run in FP64 in a fixed order. */
int cpm_guess_norm(cpm_ctx* c, int64_t samples, const float* feat, const float* target,
                   float* norm, float* target_scale);

/* A trained network to / from a file: parameters[CPM_MLP_PARAMS], norm[64] and the
 * target scale (pointers host or device), with a header (magic "CPMGUESS", version 1,
 * sizes) and an FNV-1a checksum.  CPM_EIO when the file cannot be written or read, or
 * its header, size or checksum do not match; nothing is written into the outputs then.
 * No context: host file operations only. */
int cpm_guess_save(const char* path, const float* params, const float* norm,
                   float target_scale);
int cpm_guess_load(const char* path, float* params, float* norm, float* target_scale);

/* One training step in one call: the gradient of the mean squared error on `samples`
 * samples (as cpm_mlp_grad, into the device buffers grad[CPM_MLP_PARAMS] and loss[1]),
 * then one Adam step on params with moments m, v (as cpm_mlp_adam, step >= 1).  When
 * loss_out (host) is not NULL it receives the mean squared error before the step.  All
 * other arrays are device arrays; CPM_EINVAL for host pointers, samples < 1 or step < 1. */
int cpm_guess_train_step(cpm_ctx* c, float* params, const float* norm, int bf16,
                         int64_t samples, const float* feat, const float* target, float* m,
                         float* v, float* grad, double* loss, int step, float lr,
                         double* loss_out);

/* q0[k] = q_prev[k] + scale * y[k] for k < len. */
int cpm_guess_apply(cpm_ctx* c, int64_t len, const float* y, float scale, const double* q_prev,
                    double* q0);

/* The whole guess in one call: features of `frames` frames (as cpm_guess_features, into
 * a context workspace), the network, and q0 = q_prev + scale * y, with one
 * synchronisation.  Device arrays; b, b_prev, q_prev, q0 [frames*n]. */
int cpm_guess(cpm_ctx* c, const float* params, const float* norm, int bf16, int frames,
              const double* b, const double* b_prev, const double* chi, float scale,
              const double* q_prev, double* q0);

/* q = E_n p for nrhs charge vectors p[nrhs*n] (e): the electrostatic potentials (1/A per e)
 * on the electrode atoms, through the same matvec as the solver (E streamed once per pass
 * of up to eight columns). */
int cpm_apply_E(cpm_ctx* c, int nrhs, const double* p, double* q);

/* Copies E (form CPM_E_STORED or CPM_E_PAPER) into out[n*ld] (row-major, ld >= n). */
int cpm_get_E(cpm_ctx* c, int form, double* out, int64_t ld);

/* Copies rows rows[0..nrows) of E (form as above) into out[nrows*ld]; rows host or
 * device, each in [0, n). */
int cpm_get_E_rows(cpm_ctx* c, int form, int nrows, const int* rows, double* out, int64_t ld);

typedef struct cpm_info_t {
  int n;              /* electrode atoms */
  int m;              /* half-space k-vectors */
  int64_t nnz_p;      /* stored entries of the PCG-DC preconditioner */
  double p_gap;       /* Eq. 37 value in use (0 if disabled) */
  double c_ele;       /* 1^T E_n^-1 1 */
  double t_kspace_ms; /* device time of the last build's k-space GEMM (fused epilogue) */
  double t_phase_ms;  /* structure-factor operand generation */
  double t_precond_ms;
  double t_dsolve_ms;
  int d_iters;        /* iterations of the E_n d' = 1 solve */
  int64_t launches;   /* CUDA kernels launched by the library in this process so far */
  double t_tc_ms;     /* BF16X6 builds: device time of the tensor-core tail kernel alone */
  int head_cols;      /* leading k-space operand columns summed in FP64 (heaviest weights) */
  double t_matvec_ms; /* last cpm_apply_E: device time of its matvec launches alone */
  int tc_blocks[3];   /* BF16X6 builds: 64-column K-blocks of the tensor-core tail taking
                         six, three and one BF16 products (weight-bounded schedule) */
  double t_head_ms;   /* BF16X6 builds: device time of the FP64-accurate head kernel */
  double t_tc_light_ms; /* BF16X6 builds with a resident operand: the part of t_tc_ms spent
                           on the three- and one-product K-blocks */
  int tc_blocks_fp8;    /* BF16X6 builds: of tc_blocks[2], the K-blocks taking their one
                           product in FP8 (E4M3) instead of FP16 */
  double t_tc_loop_ms;  /* BF16X6 builds: the whole k-window loop of the tail; a streamed
                           build makes each window's operand planes inside it, so there
                           t_tc_ms (the tensor-core launches alone) is the smaller */
  double t_solve_ms;         /* last PCG solve on this context: device time */
  double t_solve_matvec_ms;  /* ... of its matvec launches (inner and error-free) */
  double t_solve_replace_ms; /* ... of its residual replacements (many-column solves) */
  int solve_replacements;    /* ... and their count */
  double t_pot_sf_ms;        /* last cpm_potential: the ions' structure factors, */
  double t_pot_kspace_ms;    /* the k-space contraction with the electrode operand, */
  double t_pot_real_ms;      /* the real-space sums and b = chi - k_e b^sol (device time) */
  int solve_path;            /* path of the last solve: 1 kernels, 2 cluster-resident */
  double t_solve_dc_ms;      /* last PCG-DC solve on the kernel path: device time of its
                                preconditioner applies (z = P r) */
} cpm_info_t;

int cpm_get_info(cpm_ctx* c, cpm_info_t* out);

/* Copies the PCG-DC preconditioner P (Sec. III B 2, Eq. 36) in row form: row j holds
 * P[j, tau] for the neighbours tau of j (r <= rcut_dc, tau = j included, ascending), so
 * z_j = sum_tau P[j, tau] r_tau.  off[n+1] (int64) row offsets, idx[nnz] (int32) columns
 * tau, val[nnz] the entries as Eq. 36 gives them (column tau of M_tau^-1); the Eq. 37
 * fill p_gap (cpm_info_t.p_gap) is not added.  nnz is cpm_info_t.nnz_p.  Host or device
 * pointers, caller-owned.  CPM_EINVAL if the context was built without PCG-DC. */
int cpm_get_precond(cpm_ctx* c, int64_t* off, int* idx, double* val);

/* Copies the neutralising vector d (Eq. S8) into d_out[n]. */
int cpm_get_d(cpm_ctx* c, double* d_out);

const char* cpm_last_error(const cpm_ctx* c);

/* ---- ragged batches (no counterpart in the paper) --------------------------------------
 * Several independent electrodes of any sizes, each its own built context (float storage
 * of E: CPM_PREC_FP32 or CPM_PREC_BF16X6; same preconditioner; same device), solved by
 * one PCG over all of them: every system is a right-hand-side column with its own E,
 * preconditioner and d, so an iteration is one launch per step for the whole batch.  The
 * batch reads the systems' builds at every call (a rebuilt system is picked up) and runs
 * on the first system's stream.  It does not own the contexts; destroy the batch first. */
typedef struct cpm_batch cpm_batch;

int cpm_batch_create(cpm_batch** out, int count, cpm_ctx* const* systems);
int cpm_batch_destroy(cpm_batch* b);

/* Eq. 25 first step for every system: E_k q_k = b_k (b in V as cpm_potential gives it).
 * rhs and q_inout are the systems' vectors concatenated in batch order
 * ([n_0 + n_1 + ...], host or device); q_inout holds the guess when use_guess != 0.
 * iters_out / relres_out: host [count] or NULL.  Returns CPM_ENOCONV if any system
 * missed tol within maxit (q holds the last iterates). */
int cpm_batch_solve(cpm_batch* b, const double* rhs, double* q_inout, int use_guess,
                    double tol, int maxit, int* iters_out, double* relres_out);

/* Eq. 35 for every system with its own d: q_k -= (sum q_k + qsol[k]) d_k.  q_inout
 * concatenated as above; qsol [count] or NULL (all zero). */
int cpm_batch_neutralize(cpm_batch* b, double* q_inout, const double* qsol);

const char* cpm_batch_last_error(const cpm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* CPM_H */
