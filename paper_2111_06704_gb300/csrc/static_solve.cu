// cpm_solve_static: the first-step charge solve with a fixed device workspace.
//
// cpm_solve grows a per-context workspace with the context's allocator the first time
// it sees a larger problem.  Some callers cannot allocate device memory at solve time:
// an MD engine that has reserved the whole device for its own pool, a plugin whose
// host forbids cudaMalloc after start-up, or a time step that must not stall on an
// allocation.  This entry point runs the same PCG kernels on a workspace that lives in
// a file-scope __device__ array, so a call allocates nothing.
//
// The array is CPM_STATIC_SCRATCH_BYTES (8 MiB) on every device that loads the library,
// held until the process exits.  Host code may not use the array's name as a device
// address (it is a host-side stand-in); its device address is looked up once per device
// with cudaGetSymbolAddress while that device is current, on the first call made there.
// That first call should therefore come before any stream capture.  Every call shares
// the one array: calls whose work overlaps on the GPU (other streams, other host
// threads) race and must be serialised by the caller.  The solver clears the parts of
// the workspace that must start at zero on every call.
#include <mutex>
#include <string>

#include "cpm_internal.cuh"

namespace cpm {

namespace {

static __device__ __align__(256) unsigned char g_solve_scratch[CPM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array on `device` (looked up once, that device current).
int scratch_address(Ctx* c, void** out) {
  if (c->device < 0 || c->device >= kMaxDevices)
    return set_err(c, CPM_EINVAL, "cpm_solve_static: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[c->device]) {
    int cur = 0;
    if (int st = cuda_check(c, cudaGetDevice(&cur), "cudaGetDevice")) return st;
    if (cur != c->device &&
        cuda_check(c, cudaSetDevice(c->device), "cudaSetDevice"))
      return CPM_ECUDA;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (cur != c->device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_addr[c->device] = p;
  }
  *out = g_scratch_addr[c->device];
  return CPM_OK;
}

}  // namespace
}  // namespace cpm

using namespace cpm;

struct cpm_ctx : public cpm::Ctx {};

extern "C" int cpm_solve_static(cpm_ctx* c, int nrhs, const double* b, double* q_inout,
                                int use_guess, double tol, int maxit, int* iters_out,
                                double* relres_out) {
  if (!c) return CPM_EINVAL;
  if (!c->built) return set_err(c, CPM_ENOTBUILT, "cpm_solve_static before cpm_build_E");
  if (nrhs < 1 || !(tol > 0) || maxit < 1)
    return set_err(c, CPM_EINVAL, "cpm_solve_static: bad arguments");
  if (pointer_where(c, b) != 1 || pointer_where(c, q_inout) != 1)
    return set_err(c, CPM_EINVAL,
                   "cpm_solve_static: b and q must be device pointers of the context's device "
                   "(staging would allocate)");
  void* ws = nullptr;
  if (int st = scratch_address(c, &ws)) return st;
  SolveArgs a{nrhs, b, 1.0 / kKe, q_inout, use_guess != 0, tol, maxit, iters_out, relres_out};
  a.ws = ws;
  a.ws_bytes = CPM_STATIC_SCRATCH_BYTES;
  a.timed = false;
  const int st = pcg_solve(c, a);
  if (st != CPM_OK && st != CPM_ENOCONV) return st;
  const int sync = cuda_check(c, cudaStreamSynchronize(c->stream), "solve_static sync");
  return sync ? sync : st;
}
