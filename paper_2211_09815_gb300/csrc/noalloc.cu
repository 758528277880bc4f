// pm_density_noalloc: the CIC overdensity of a particle set without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: code whose device memory is owned entirely by its own pool allocator
// (a framework's caching allocator, an inference server with a fixed memory budget) so
// that a foreign cudaMalloc either fails or fragments the pool, and latency-sensitive
// loops that must not pay for cudaMalloc/cudaFree, which can synchronise the device.
// pm_op_density needs a context, and creating a context allocates its accumulators.
//
// How: the int64 fixed-point accumulator lives in a file-scope __device__ array of a
// fixed size (PM_NOALLOC_MAX_CELLS cells, 16 MiB), which every GPU that loads this
// library holds until the process exits.  Host code cannot use the array's name as a
// device address (on the host it names a host-side shadow), so the device address is
// looked up with cudaGetSymbolAddress while the device is current: once per device, and
// again when the device's CUDA context has been replaced since (cudaDeviceReset), which
// the context's unique id shows.  The first call on a device does this look-up; make that
// first call before any stream capture.  All calls share the one array and it keeps the
// previous call's contents, so each call clears the cells it uses before scattering;
// calls that overlap on the GPU (different streams, or different host threads, on the
// same device) race on it.
#include <cmath>
#include <mutex>

#include "pm_engine.h"
#include "pm_kernels.cuh"

namespace {

constexpr long long kMaxCells = PM_NOALLOC_MAX_CELLS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_density_scratch[kMaxCells];

struct DevEntry {
  unsigned long long ctx_id;   // id of the context the address belongs to
  unsigned long long* addr;
};
std::mutex g_mu;
DevEntry g_dev[kMaxDevices] = {};

// id of the calling thread's current context (0: none current yet), through the driver
// entry points of the runtime (no link against libcuda)
unsigned long long current_context_id() {
  using GetCur = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  if (!get_cur || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return 0;
    get_cur = (GetCur)f1;
    get_id = (GetId)f2;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_cur(&c) != CUDA_SUCCESS || !c) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

int scratch_address(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { pmgb::set_cuda_error(e); return PM_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) return PM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  DevEntry& d = g_dev[dev];
  const unsigned long long id = current_context_id();
  if (!d.addr || id == 0 || id != d.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_density_scratch);   // makes the device's context current
    if (e != cudaSuccess) { pmgb::set_cuda_error(e); return PM_ERR_CUDA; }
    d.addr = static_cast<unsigned long long*>(p);
    d.ctx_id = current_context_id();
  }
  *out = d.addr;
  return PM_OK;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" int pm_density_noalloc(double box, int n_mesh, int n_ptcl, const float* disp, float* dens_out,
                                  void* stream) {
  using namespace pmgb;
  if (!disp || !dens_out) return PM_ERR_ARG;
  // the checks of pm_init for these arguments (finite box, 8 <= n_mesh, power-of-two sizes)
  if (!(box > 0) || !std::isfinite(box) || !pow2(n_mesh) || !pow2(n_ptcl) || n_ptcl < 4 || n_mesh < 8 ||
      n_mesh % n_ptcl != 0)
    return PM_ERR_ARG;
  const long long M = (long long)n_mesh * n_mesh * n_mesh;
  if (M > kMaxCells) return PM_ERR_ARG;  // larger meshes need pm_op_density with a context
  unsigned long long* acc = nullptr;
  const int r = scratch_address(&acc);
  if (r != PM_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = (long long)n_ptcl * n_ptcl * n_ptcl;
  Geo<float> g;
  g.lg_np = 0;
  while ((1 << g.lg_np) < n_ptcl) ++g.lg_np;
  g.np = n_ptcl;
  g.nm = n_mesh;
  g.ratio = n_mesh / n_ptcl;
  g.inv_l = (float)(n_mesh / box);
  g.N = N;
  g.M = M;
  int lgN = 0;
  while ((1LL << lgN) < N) ++lgN;
  const int e_d = fixed_top<float>(lgN);   // the quantum of pm_op_density: equal results bit for bit
  // the array keeps the previous call's sums: clear the cells this call uses
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * M, st);
  if (e != cudaSuccess) { set_cuda_error(e); return PM_ERR_CUDA; }
  const int grid = (int)std::min<long long>((N + kPtclThreads - 1) / kPtclThreads, kMaxRedBlocks);
  k_scatter<float, 1><<<dim3(grid, 1), kPtclThreads, 0, st>>>(g, disp, nullptr, acc, e_d, nullptr);
  k_density_out<float><<<1024, 256, 0, st>>>((const long long*)acc, dens_out, M,
                                              (float)ldexp((double)M / (double)N, -e_d));
  e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e); return PM_ERR_CUDA; }
  return PM_OK;
}
