// noalloc.cu -- allocation-free variant of tns_heff_diag.
//
// Some callers cannot allocate device memory at the point where they need the
// Davidson preconditioner: code running inside a memory pool that forbids
// further cudaMalloc calls (a framework that pre-reserves all device memory,
// or a region where allocation would synchronise the device), or callers that
// must not fail with an out-of-memory error mid-iteration.  tns_heff_diag
// uploads its per-call index tables into freshly allocated device buffers;
// this variant stages them into a fixed file-scope device array instead.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tns.h"
#include "cuda_backend.h"

namespace tns {

// index tables of the diagonal work list: diag task indices followed by the
// per-block ranges; every GPU that loads the library holds this array (16 MiB)
// until the process exits
static __device__ __align__(256) int g_diag_scratch[TNS_NOALLOC_DIAG_MAX];

namespace {
std::mutex g_mu;
int* g_addr[256] = {nullptr};
void* g_ctx[256] = {nullptr};  // the CUDA context g_addr[device] was looked up in

// the current CUDA context (driver handle), through the runtime's driver entry
// point: a device reset or a new primary context loads the module again,
// possibly at another address
void* current_context() {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return (GetCurrent)f;
  }();
  void* c = nullptr;
  if (fn && fn(&c) != 0) c = nullptr;
  return c;
}
}  // namespace

// device address of the scratch array for the current device (looked up with
// that device current, once per device and CUDA context)
static int* diag_scratch(int device, std::string& err) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (device < 0 || device >= 256) {
    err = "heff_diag_noalloc: device index out of range";
    return nullptr;
  }
  void* ctx = current_context();
  if (!g_addr[device] || ctx != g_ctx[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_diag_scratch);
    if (e != cudaSuccess) {
      err = std::string("heff_diag_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_addr[device] = (int*)p;
    g_ctx[device] = ctx;
  }
  return g_addr[device];
}

int heff_diag_noalloc(CudaBackend& be, Step& st, double* diag, std::string& err) {
  const size_t nt = st.diag_tasks.size(), nr = st.diag_rng.size();
  if (nt + nr > (size_t)TNS_NOALLOC_DIAG_MAX) {
    err = "heff_diag_noalloc: the diagonal work list needs " + std::to_string(nt + nr) +
          " index entries, more than the fixed maximum TNS_NOALLOC_DIAG_MAX";
    return -1;
  }
  const DevList* dl = be.resident(st.heff);
  if (!dl) {
    err = "heff_diag_noalloc: the work list of this step is not resident on the device; call tns_heff_apply or "
          "tns_heff_diag once for this step first";
    return -2;
  }
  int* s = diag_scratch(be.device(), err);
  if (!s) return -6;
  be.note(cudaMemcpyAsync(s, st.diag_tasks.data(), nt * sizeof(int), cudaMemcpyHostToDevice, be.stream()),
          "heff_diag_noalloc");
  be.note(cudaMemcpyAsync(s + nt, st.diag_rng.data(), nr * sizeof(int), cudaMemcpyHostToDevice, be.stream()),
          "heff_diag_noalloc");
  launch_heff_diag(be, dl->tasks, s, s + nt, (int)st.heff.groups.size(), dl->groups, diag);
  be.sync();
  std::string e = be.error();
  if (!e.empty()) {
    err = e;
    return -6;
  }
  return 0;
}

}  // namespace tns
