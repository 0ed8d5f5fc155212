// grmhd_rk_step_static: one method-of-lines step whose scratch lives in a
// fixed device array of this library instead of a caller-provided workspace.
//
// Why it exists: grmhd_rk_step needs a device workspace (the stage-0 copy of
// U, plus an accumulator for RK4) that the caller allocates.  Some callers
// cannot call cudaMalloc or any allocating routine: host codes whose device
// memory is owned entirely by another allocator or memory pool, plug-in or
// callback contexts where allocation is forbidden, or language bindings
// with no device allocator at all.  They pass only their state buffers and
// this entry point supplies the scratch.
//
// The scratch is a file-scope __device__ array of GRMHD_STATIC_SCRATCH_BYTES
// (64 MiB).  Every GPU on which this library's device code is loaded holds
// it until the process exits (under CUDA's default lazy module loading, from
// the first use of the library on that GPU).  Host code cannot use the
// array's name as a device address, so on the first call on each device
// (that device current) the address is looked up once with
// cudaGetSymbolAddress and cached; that first call should therefore come
// before any stream capture, and the cached address does not survive a
// cudaDeviceReset (do not call this entry point across one).  The array is
// shared by every call: overlapping calls on the GPU (different streams, no
// ordering between them) race on it.
//
// The step lays the grmhd_rk_step workspace over the array, so blocks whose
// cached workspace (grmhd_rk_workspace_bytes_cached) fits -- ncell up to
// about 42,100 points for RK2/RK3 and 40,500 for RK4, e.g. a 28^3 interior
// with 3 ghosts --
// take the cached paths, and larger blocks up to the plain workspace size the
// uncached ones, as grmhd_rk_step does with workspaces of those sizes.
// Nothing in the array has to start at zero: the step overwrites the U^n
// copy, the RK4 accumulator, the geometry caches and the RHS buffers before
// reading them.  The caches are rebuilt on every call: GRMHD_REUSE_GEOMETRY
// is cleared, because the array may hold another block's caches from the
// previous call.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = GRMHD_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_rk_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_for_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GRMHD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_rk_scratch) != cudaSuccess || !p) return GRMHD_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GRMHD_OK;
}

}  // namespace

extern "C" int grmhd_rk_step_static(const grmhd_grid* grid, const grmhd_params* params, int32_t scheme, double dt,
                                    double* cons, double* prim, const double* metric, const double* kij,
                                    int32_t* nfail, void* stream) {
  const size_t need = grmhd_rk_workspace_bytes(grid, scheme);
  if (need == 0) return GRMHD_ERR_ARG;
  if (need > kScratchBytes) return GRMHD_ERR_SIZE;
  if (!params) return GRMHD_ERR_ARG;
  void* ws = nullptr;
  const int e = scratch_for_current_device(&ws);
  if (e != GRMHD_OK) return e;
  grmhd_params p = *params;
  p.flags &= ~GRMHD_REUSE_GEOMETRY;
  return grmhd_rk_step(grid, &p, scheme, dt, cons, prim, metric, kij, ws, kScratchBytes, nfail, stream);
}
