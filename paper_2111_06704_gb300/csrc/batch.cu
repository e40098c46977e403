// Ragged batches: several independent electrodes (each its own built context, of any
// size) solved together.  One PCG runs over all of them at once: every system is a
// right-hand-side column with its own matrix, preconditioner and neutralising vector, so
// each iteration is one launch per step for the whole batch instead of one per system.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "cpm_internal.cuh"

using namespace cpm;

struct cpm_ctx : public cpm::Ctx {};

struct cpm_batch {
  std::vector<cpm_ctx*> sys;
  Ctx work;       // stream, allocator and workspace of the batch solve (n = largest system)
  Buf cols;       // SysCol [count]
  Buf pad_b, pad_q, pad_s;  // [count][nmax] right-hand sides, solutions; [count] Q^sol
  std::vector<int64_t> off;  // offsets of the systems in the concatenated vectors
  int nmax = 0;
};

namespace {

int64_t round_up128(int64_t v) { return (v + 127) / 128 * 128; }

// Refreshes the per-system descriptors from the contexts (a rebuilt system is picked
// up) and the concatenated offsets.
int describe(cpm_batch* b) {
  const int count = (int)b->sys.size();
  std::vector<SysCol> h(count);
  b->off.assign(count + 1, 0);
  b->nmax = 0;
  for (int k = 0; k < count; ++k) {
    cpm_ctx* c = b->sys[k];
    if (!c->built) return set_err(&b->work, CPM_ENOTBUILT, "batch system " + std::to_string(k) +
                                                             " is not built");
    h[k].E = (const float*)c->E.ptr;
    h[k].ldE = c->ldE;
    h[k].n = c->n;
    h[k].nbr_off = (const int64_t*)c->nbr_off.ptr;
    h[k].nbr_idx = (const int*)c->nbr_idx.ptr;
    h[k].prow = (const double*)c->prow.ptr;
    h[k].pgap = c->pgap;
    h[k].inv_diag = (const double*)c->diag.ptr + c->n;
    h[k].d = (const double*)c->d.ptr;
    b->off[k + 1] = b->off[k] + c->n;
    b->nmax = std::max(b->nmax, c->n);
  }
  Ctx* w = &b->work;
  w->n = b->nmax;
  w->ldE = round_up128(b->nmax);
  w->built = true;
  int st = buf_reserve(w, &b->cols, count * sizeof(SysCol));
  if (!st) st = cuda_check(w, cudaMemcpyAsync(b->cols.ptr, h.data(), count * sizeof(SysCol),
                                              cudaMemcpyHostToDevice, w->stream), "batch cols");
  if (!st) st = cuda_check(w, cudaStreamSynchronize(w->stream), "batch cols sync");
  return st;
}

// Concatenated [sum n_k] <-> padded [count][nmax] (host or device concatenated side).
int pack(cpm_batch* b, const double* cat, double* pad, bool zero_first) {
  Ctx* w = &b->work;
  const int count = (int)b->sys.size();
  int st = CPM_OK;
  if (zero_first)
    st = cuda_check(w, cudaMemsetAsync(pad, 0, (size_t)count * b->nmax * sizeof(double),
                                       w->stream), "batch zero");
  for (int k = 0; k < count && !st; ++k)
    st = cuda_check(w, cudaMemcpyAsync(pad + (int64_t)k * b->nmax, cat + b->off[k],
                                       (b->off[k + 1] - b->off[k]) * sizeof(double),
                                       cudaMemcpyDefault, w->stream), "batch pack");
  return st;
}

int unpack(cpm_batch* b, const double* pad, double* cat) {
  Ctx* w = &b->work;
  int st = CPM_OK;
  for (int k = 0; k < (int)b->sys.size() && !st; ++k)
    st = cuda_check(w, cudaMemcpyAsync(cat + b->off[k], pad + (int64_t)k * b->nmax,
                                       (b->off[k + 1] - b->off[k]) * sizeof(double),
                                       cudaMemcpyDefault, w->stream), "batch unpack");
  if (!st) st = cuda_check(w, cudaStreamSynchronize(w->stream), "batch unpack sync");
  return st;
}

}  // namespace

extern "C" {

int cpm_batch_create(cpm_batch** out, int count, cpm_ctx* const* systems) {
  if (!out || count < 1 || !systems) return CPM_EINVAL;
  *out = nullptr;
  for (int k = 0; k < count; ++k) {
    cpm_ctx* c = systems[k];
    if (!c) return CPM_EINVAL;
    if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_batch_create: a system is not built");
    if (c->fp64())
      return set_err(c, CPM_EINVAL, "cpm_batch_create: systems must use float storage of E");
    if (c->p.precond != systems[0]->p.precond || c->device != systems[0]->device)
      return set_err(c, CPM_EINVAL,
                     "cpm_batch_create: systems must share the preconditioner and the device");
  }
  cpm_batch* b = new cpm_batch();
  b->sys.assign(systems, systems + count);
  b->work.p = systems[0]->p;
  b->work.stream = systems[0]->stream;
  b->work.device = systems[0]->device;
  *out = b;
  return CPM_OK;
}

int cpm_batch_destroy(cpm_batch* b) {
  if (!b) return CPM_EINVAL;
  cudaStreamSynchronize(b->work.stream);
  Buf* all[] = {&b->cols, &b->pad_b, &b->pad_q, &b->pad_s, &b->work.ws_solve};
  for (Buf* x : all) buf_free(&b->work, x);
  delete b;
  return CPM_OK;
}

int cpm_batch_solve(cpm_batch* b, const double* rhs, double* q_inout, int use_guess,
                    double tol, int maxit, int* iters_out, double* relres_out) {
  if (!b) return CPM_EINVAL;
  Ctx* w = &b->work;
  if (!rhs || !q_inout || !(tol > 0) || maxit < 1)
    return set_err(w, CPM_EINVAL, "cpm_batch_solve: bad arguments");
  int st = describe(b);
  if (st) return st;
  const int count = (int)b->sys.size();
  const size_t pbytes = (size_t)count * b->nmax * sizeof(double);
  if ((st = buf_reserve(w, &b->pad_b, pbytes)) || (st = buf_reserve(w, &b->pad_q, pbytes)))
    return st;
  double* pb = (double*)b->pad_b.ptr;
  double* pq = (double*)b->pad_q.ptr;
  if ((st = pack(b, rhs, pb, true))) return st;
  if (use_guess) st = pack(b, q_inout, pq, true);
  else st = cuda_check(w, cudaMemsetAsync(pq, 0, pbytes, w->stream), "batch q zero");
  if (st) return st;
  std::vector<int> it(count);
  std::vector<double> rr(count);
  SolveArgs a{count, pb, 1.0 / kKe, pq, use_guess != 0, tol, maxit, it.data(), rr.data()};
  a.sys = (const SysCol*)b->cols.ptr;
  const int solve_st = pcg_solve(w, a);
  if (solve_st != CPM_OK && solve_st != CPM_ENOCONV) return solve_st;
  if ((st = unpack(b, pq, q_inout))) return st;
  if (iters_out) memcpy(iters_out, it.data(), count * sizeof(int));
  if (relres_out) memcpy(relres_out, rr.data(), count * sizeof(double));
  return solve_st;
}

int cpm_batch_neutralize(cpm_batch* b, double* q_inout, const double* qsol) {
  if (!b) return CPM_EINVAL;
  Ctx* w = &b->work;
  if (!q_inout) return set_err(w, CPM_EINVAL, "cpm_batch_neutralize: bad arguments");
  int st = describe(b);
  if (st) return st;
  const int count = (int)b->sys.size();
  const size_t pbytes = (size_t)count * b->nmax * sizeof(double);
  if ((st = buf_reserve(w, &b->pad_q, pbytes)) ||
      (st = buf_reserve(w, &b->pad_s, count * sizeof(double))))
    return st;
  double* pq = (double*)b->pad_q.ptr;
  double* ps = (double*)b->pad_s.ptr;
  if ((st = pack(b, q_inout, pq, true))) return st;
  if (qsol && (st = cuda_check(w, cudaMemcpyAsync(ps, qsol, count * sizeof(double),
                                                  cudaMemcpyDefault, w->stream), "qsol")))
    return st;
  launch_neutralize_ragged(pq, count, b->nmax, (const SysCol*)b->cols.ptr, qsol ? ps : nullptr,
                           w->stream);
  if ((st = cuda_check(w, cudaGetLastError(), "batch neutralize"))) return st;
  return unpack(b, pq, q_inout);
}

const char* cpm_batch_last_error(const cpm_batch* b) {
  return b ? b->work.err.c_str() : "null batch";
}

}  // extern "C"
