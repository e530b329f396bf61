// cuda_backend.h -- CUDA backend of the engine (sm_103a).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "engine.h"

namespace tns {

// device memory of the library (devmem.cu): every allocation goes through
// dmalloc / dfree, which count the bytes in use per device and refuse,
// before cudaMalloc, an allocation above the device budget (0: no budget)
cudaError_t dmalloc_raw(void** p, size_t bytes);
template <class T>
inline cudaError_t dmalloc(T** p, size_t bytes) {
  return dmalloc_raw((void**)p, bytes);
}
void dfree(void* p);
struct DevMem {
  long long used = 0, peak = 0, budget = 0;
};
DevMem dmem(int device);
void dmem_set_budget(int device, long long bytes);
void dmem_reset_peak(int device);

struct Tile {  // an output tile of a group: rows [row0, row0+nrows), cols [col0, col0+ncols)
  int g;
  int row0, col0, nrows, ncols;
  int t0, t1;      // task range of this piece (a split tile has several pieces)
  long long poff;  // -1: write the output block; else element offset of this piece's partial tile
};

struct SplitRed {  // a split tile: sum of nsplit partial tiles (fixed order) -> output
  int g;
  int row0, col0, nrows, ncols;
  int nsplit;
  long long poff;
};

// schedule variants tried by the online autotuner: the split-K target is
// (total cost) / (resident CTAs x SMs x rounds) with rounds = kRounds[v];
// for the tensor-core form variant kWsVariant runs the persistent
// warp-specialised kernel (its own split, rounds 2) instead of one CTA per
// piece; the FP64 form tries the first kFp64Variants
constexpr int kNumVariants = 4;
constexpr double kRounds[kNumVariants] = {1.0, 2.0, 4.0, 2.0};
constexpr int kWsVariant = 3;
constexpr int kFp64Variants = 3;

// one schedule of a work list for the FP64 kernels: tiles split into size
// classes, long task lists cut into partial tiles summed in fixed order
struct FpVariant {
  bool planned = false;
  Tile* tiles = nullptr;
  int ncls[4] = {0, 0, 0, 0};  // tiles per size class (contiguous, class 0 first)
  double ccost[4] = {0, 0, 0, 0};  // estimated FMAs per class (the costliest runs on the launching stream)
  int ntiles = 0;
  SplitRed* reds = nullptr;  // split tiles to reduce after the product kernels
  int nreds = 0;
  long long psize = 0;       // partial-tile elements per vector
  double* part = nullptr;    // partial tiles (psize * part_nvec)
  int part_nvec = 0;
};

// online autotuner state of one (precision, nvec) use of a work list: the
// first products run the variants in turn and are timed; the fastest is kept
// for the rest of the list's life
struct Tune {
  int step = 0;   // products run so far while tuning
  int best = -1;
  float ms[kNumVariants] = {1e30f, 1e30f, 1e30f, 1e30f};  // fastest sample of each variant
};
// tuning sequence: one untimed product (default variant: first-use effects
// such as cold caches land there), then kTuneRounds timed samples of every
// variant, the fastest sample of each compared
constexpr int kTuneRounds = 2;

// captured launch sequence of one (precision, nvec) use: replayed with the
// input copied into xbuf and the output copied out of ybuf
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  double* xbuf = nullptr;
  double* ybuf = nullptr;
  long long elems = 0;  // doubles per buffer (nvec * stride)
  long long stride = 0;
  int kernels = 0;      // kernel launches inside the graph
  bool failed = false;  // capture not possible: launch directly
};

// device copy of a work list
struct DevList {
  long long gen = -1;
  unsigned long long shape = 0;  // shape signature of the list (schedule cache key)
  Task* tasks = nullptr;
  Group* groups = nullptr;
  Tile* wtiles = nullptr;    // 32 x 16 warp tiles of the FP64 tensor (DMMA) kernel
  int nwtiles = 0;
  FpVariant fv[kNumVariants];
  // FP64 output tiles per size class with their estimated FMAs (host; shared
  // by the schedule variants, which differ only in how they cut the tiles)
  bool fp_tiled = false;
  std::vector<Tile> fp_tiles[4];
  std::vector<double> fp_cost[4];
  // tensor-core form (precision != FP64)
  void* tc = nullptr;
  long long tc_gen = -1;
  std::map<int, Tune> tune;         // key: precision * 64 + nvec
  std::map<int, GraphSlot> graphs;  // same key
};

class CudaBackend : public Backend {
 public:
  CudaBackend(int device, cudaStream_t s, bool own);
  // FP64 product kernel: 0 DFMA tile classes (default: on GB300 DFMA and DMMA
  // peak at ~1.0 TFLOP/s alike and the DFMA kernel measured faster), 1 DMMA
  // (mma.sync m8n8k4 f64); environment TNS_FP64_KERNEL=dfma|dmma
  int fp64_kernel = 0;
  // bound of one wait inside the tensor-core product loop (ns); the
  // environment variable TNS_TC_WAIT_NS overrides the default 0.2 s when the
  // backend is created (a test makes the waits run out with it and checks the
  // reported error and that the context stays usable; with 0 every warp of
  // the small-block kernel first waits on a barrier that nothing completes,
  // since its copies may land before any wait could run out)
  unsigned long long tc_wait_ns = 200000000ull;
  // TNS_TC_VARIANT=v (0..kNumVariants-1) fixes the tensor-core schedule
  // variant instead of tuning it (tests run each kernel this way)
  int forced_tc_variant = -1;
  // output blocks whose dimensions, and those of every X block they read, are
  // at most tc_small go to the warp-level small-block kernel of the
  // tensor-core form (0: every block to the tile kernel; at most 32);
  // environment TNS_TC_SMALL
  int tc_small = 32;
  // destroy the CUDA graphs captured for a work list (after both streams
  // have drained): every buffer a graph reads or writes is baked into it, so
  // they go before any such buffer is freed or reallocated
  void free_graphs(DevList& d);
  ~CudaBackend() override;
  double* alloc(long long n) override;
  void release(double* p) override;
  void upload(double* dst, const double* src, long long n) override;
  void download(double* dst, const double* src, long long n) override;
  void zero(double* p, long long n) override;
  void lincomb(const LCList& l) override;
  void run(const TaskList& tl, const double* xv, double* yv, int nvec, long long xs, long long ys,
           int precision) override;
  void task_values(const TaskList& tl, const double* xv, const double* ybar, double* out) override;
  void nonzero_blocks(const std::vector<const double*>& p, const std::vector<long long>& n,
                      std::vector<char>& nz) override;
  long long mem_used() override;
  long long mem_limit() override;
  long long mem_free() override;
  void set_budget(long long bytes) override;
  double* host_alloc(long long n) override;
  void host_release(double* p) override;
  void forget(const TaskList& tl) override { drop(tl); }
  long long step_bytes(const TaskList& tl, long long psi_length) override;
  void sync() override;
  std::string error() override;

  cudaStream_t stream() const { return stream_; }
  int device() const { return device_; }
  void note(cudaError_t e, const char* what);
  // false once a failure (an allocation, a launch) has been noted in the
  // current call: later launches are skipped so that no kernel runs on a
  // buffer that does not exist
  bool ok() const { return err_.empty(); }
  // persistent device copy of a task list (uploaded when tl.gen changes)
  DevList& dev(const TaskList& tl);
  // the device copy of tl if it is resident and current, else nullptr (never uploads)
  const DevList* resident(const TaskList& tl) const {
    auto it = lists_.find(&tl);
    return (it != lists_.end() && it->second.gen == tl.gen && it->second.tasks) ? &it->second : nullptr;
  }
  void drop(const TaskList& tl);
  // CUDA graphs for persistent work lists (on by default; TNS_GRAPHS=0 turns
  // them off)
  bool use_graphs = true;
  // online schedule autotuning (on by default; TNS_AUTOTUNE=0 keeps the
  // default variant, which makes repeated runs bitwise reproducible)
  bool autotune = true;
  // launches of the FP64 product kernels of variant v (no allocation, no
  // synchronisation: capturable)
  void enqueue_fp64(const DevList& d, int v, const double* xv, double* yv, int nvec, long long xs, long long ys);
  // room for `bytes` of the backend's own allocations (the engine's hook)
  void need(long long bytes) {
    if (room && bytes > (64LL << 20)) room(bytes);
  }
  // scratch device memory owned by the backend (grows, never shrinks)
  void* scratch(size_t bytes, int slot);
  // counted launches of the engine's own kernels
  long long launches = 0;
  // schedule tuning: lists tuned, lists that took a cached choice, and how
  // often each variant ran as the chosen one (per precision: 0 FP64, 1 TF32, 2 BF16X3)
  long long tuned = 0, tune_cache_hits = 0;
  long long variant_runs[3][kNumVariants] = {};
  float last_ms = 0.f;

 private:
  int device_;
  cudaStream_t stream_;
  bool own_;
  std::string err_;
  std::map<const TaskList*, DevList> lists_;
  // best schedule variant per (precision, nvec, shape signature): work lists
  // of later steps with the same shape take it without tuning again
  std::map<std::pair<int, unsigned long long>, int> tune_cache_;
  std::vector<std::pair<void*, size_t>> scratch_ = std::vector<std::pair<void*, size_t>>(8, {nullptr, 0});
  cudaStream_t gstream_ = nullptr;  // side stream for graph capture and replay
  cudaEvent_t gev_[2] = {nullptr, nullptr};
  // forked streams: the FP64 tile classes run side by side (fork/join events)
  cudaStream_t fstream_[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fev_[4] = {nullptr, nullptr, nullptr, nullptr};
  bool fork_ready();
  void upload_list(const TaskList& tl, DevList& d);
  void plan_variant(const TaskList& tl, DevList& d, int v);
  bool ensure_part(DevList& d, FpVariant& f, int nvec);
  void free_list(DevList& d);
  template <class F>
  void launch_graphed(DevList& d, int key, const double* xv, double* yv, int nvec, long long xs, long long ys,
                      F&& enqueue);
};

// allocation-free H_eff diagonal (noalloc.cu)
int heff_diag_noalloc(CudaBackend& be, Step& st, double* diag, std::string& err);

// tensor-core form (tc.cu): prepare (plan, allocations; not capturable),
// enqueue (kernel launches only; capturable), check (reads the timeout flag,
// synchronises)
bool prepare_tasks_tc(CudaBackend& be, const TaskList& tl, DevList& d, int nvec, int variant, int precision);
void enqueue_tasks_tc(CudaBackend& be, DevList& d, const double* xv, double* yv, int nvec, long long xs,
                      long long ys, int precision, int variant);
void check_tasks_tc(CudaBackend& be, DevList& d);
void release_tc_plan(void* plan);

// kernels used by the solver (defined in kernels.cu)
void launch_heff_diag(CudaBackend& be, const Task* d_tasks, const int* d_idx, const int* d_rng, int ngroups,
                      const Group* d_groups, double* diag);
void launch_multidot(CudaBackend& be, const double* V, long long ldv, int k, const double* w, long long n,
                     double* out);
void launch_axpy_multi(CudaBackend& be, const double* V, long long ldv, int k, const double* coef, double sign,
                       double* w, long long n);
void launch_combine(CudaBackend& be, const double* V, long long ldv, int k, const double* coef, double* out,
                    long long n);
void launch_scale(CudaBackend& be, double* x, const double* num, int inv_sqrt, long long n);
void launch_precond(CudaBackend& be, const double* r, const double* diag, const double* theta, double* t,
                    long long n);
void launch_residual(CudaBackend& be, const double* AVs, const double* x, const double* theta, double* r,
                     long long n);
// batched symmetric eigensolver (cyclic Jacobi), matrices column-major == row-major (symmetric)
// A: nmat matrices at A + off[i] with size n[i]; V: eigenvectors (columns) at V + off[i]; w: eigenvalues at w + woff[i]
void launch_jacobi(CudaBackend& be, double* A, double* V, double* w, const long long* off, const int* n,
                   const int* woff, int nmat, int maxn, int* sweeps_out);
// batched symmetric eigensolver (Householder tridiagonalisation + implicit QR),
// one CTA per matrix; eigenvector p is ROW p of Z (Z + off[i], n x n); A is
// overwritten; *status (nullable) is set to 1 if a matrix hit the QR step limit
constexpr int SYEV_MAXN = 4096;
void launch_syev(CudaBackend& be, double* A, double* Z, double* w, const long long* off, const int* n,
                 const int* woff, int nmat, int maxn, int* status);
void launch_select(CudaBackend& be, const double* w, const int* sec_of, int total, int keep_max, double cut,
                   int* keep_flag, double* disc);
void launch_gather(CudaBackend& be, const double* src, const long long* so, const int* sld, double* dst,
                   const long long* dof, const int* dld, const int* rows, const int* cols, const int* trans,
                   int nblk);
void launch_argmin(CudaBackend& be, const double* x, long long n, long long* idx);
void launch_fill_unit(CudaBackend& be, double* x, long long n, const long long* idx);

}  // namespace tns
