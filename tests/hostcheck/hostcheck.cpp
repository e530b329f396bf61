// hostcheck.cpp -- test-only build of the engine's host logic.
//
// Compiles the product's symbolic layer (engine.cpp: catalogues, enlarged
// operators, work lists) against a plain-loop executor so that the CPU test
// suite can check the operator algebra and the work lists against the
// oracle without a GPU.  This library is built only by tests/ (symbols
// tnshc_*); the product library never contains or loads it, and it is not a
// fallback for anything: it has no Davidson, truncation or sweep.
#include <cstdlib>
#include <map>
#include <cstring>
#include <stdexcept>
#include <string>

#include "../../include/tns.h"
#include "../../paper_2305_05581_gb300/csrc/engine.h"

namespace {
struct HostBackend : tns::Backend {
  // allocation accounting with an optional budget, standing in for a device
  std::map<void*, long long> live;
  long long used = 0, peak = 0, budget = 0;
  double* alloc(long long n) override {
    const long long b = n * 8;
    if (budget > 0 && used + b > budget) return nullptr;
    double* p = (double*)std::calloc((size_t)n, sizeof(double));
    if (p) {
      live[p] = b;
      used += b;
      if (used > peak) peak = used;
    }
    return p;
  }
  void release(double* p) override {
    auto it = live.find(p);
    if (it != live.end()) {
      used -= it->second;
      live.erase(it);
    }
    std::free(p);
  }
  long long mem_used() override { return used; }
  long long mem_limit() override { return budget; }
  long long mem_free() override { return 1LL << 60; }
  void set_budget(long long bytes) override { budget = bytes > 0 ? bytes : 0; }
  double* host_alloc(long long n) override { return (double*)std::malloc((size_t)n * sizeof(double)); }
  void host_release(double* p) override { std::free(p); }
  void forget(const tns::TaskList&) override {}
  // the plain-loop executor allocates nothing to run a work list
  long long step_bytes(const tns::TaskList&, long long) override { return 0; }
  void upload(double* d, const double* s, long long n) override { std::memcpy(d, s, (size_t)n * 8); }
  void download(double* d, const double* s, long long n) override { std::memcpy(d, s, (size_t)n * 8); }
  void zero(double* p, long long n) override { std::memset(p, 0, (size_t)n * 8); }
  void nonzero_blocks(const std::vector<const double*>& p, const std::vector<long long>& n,
                      std::vector<char>& nz) override {
    nz.assign(p.size(), 0);
    for (size_t i = 0; i < p.size(); ++i)
      for (long long j = 0; j < n[i] && !nz[i]; ++j) nz[i] = p[i][j] != 0.0;
  }
  void lincomb(const tns::LCList& l) override {
    for (const auto& b : l.blocks)
      for (int i = 0; i < b.rows; ++i)
        for (int j = 0; j < b.cols; ++j) {
          double s = 0.0;
          for (int t = b.t0; t < b.t1; ++t) {
            const auto& tm = l.terms[t];
            if (!tm.src) s += (i == j) ? tm.c : 0.0;
            else s += tm.c * (tm.tr ? tm.src[(long long)j * b.rows + i] : tm.src[(long long)i * b.cols + j]);
          }
          b.dst[(long long)i * b.cols + j] = s;
        }
  }
  static double opL(const tns::Task& t, int i, int k) {
    if (t.flags & tns::TF_LI) return i == k ? 1.0 : 0.0;
    return (t.flags & tns::TF_LT) ? t.L[(long long)k * t.q + i] : t.L[(long long)i * t.m + k];
  }
  static double opX(const tns::Task& t, const double* X, int i, int j) {
    if (t.flags & tns::TF_XI) return i == j ? 1.0 : 0.0;
    return (t.flags & tns::TF_XT) ? X[(long long)j * t.m + i] : X[(long long)i * t.n + j];
  }
  static double opR(const tns::Task& t, int j, int k) {
    if (t.flags & tns::TF_RI) return j == k ? 1.0 : 0.0;
    return (t.flags & tns::TF_RT) ? t.R[(long long)k * t.r + j] : t.R[(long long)j * t.n + k];
  }
  void run(const tns::TaskList& tl, const double* xv, double* yv, int nvec, long long xs, long long ys,
           int precision) override {
    (void)precision;
    for (int v = 0; v < nvec; ++v)
      for (const auto& g : tl.groups) {
        double* Y = yv + (long long)v * ys + g.yoff;
        for (int i = 0; i < g.q * g.r; ++i) Y[i] = 0.0;
        for (int ti = g.t0; ti < g.t1; ++ti) {
          const tns::Task& t = tl.tasks[ti];
          const double* X = (t.flags & tns::TF_XV) ? xv + (long long)v * xs + (long long)(uintptr_t)t.X : t.X;
          for (int i = 0; i < t.q; ++i)
            for (int j = 0; j < t.r; ++j) {
              double s = 0.0;
              for (int a = 0; a < t.m; ++a) {
                double la = opL(t, i, a);
                if (la == 0.0) continue;
                for (int b = 0; b < t.n; ++b) s += la * opX(t, X, a, b) * opR(t, j, b);
              }
              Y[(long long)i * g.r + j] += t.alpha * s;
            }
        }
      }
  }
  void task_values(const tns::TaskList& tl, const double* xv, const double* ybar, double* out) override {
    for (const auto& g : tl.groups) {
      const double* Y = ybar + g.yoff;
      for (int ti = g.t0; ti < g.t1; ++ti) {
        const tns::Task& t = tl.tasks[ti];
        const double* X = (t.flags & tns::TF_XV) ? xv + (long long)(uintptr_t)t.X : t.X;
        double v = 0.0;
        for (int i = 0; i < t.q; ++i)
          for (int j = 0; j < t.r; ++j) {
            double s = 0.0;
            for (int a = 0; a < t.m; ++a) {
              double la = opL(t, i, a);
              if (la == 0.0) continue;
              for (int b = 0; b < t.n; ++b) s += la * opX(t, X, a, b) * opR(t, j, b);
            }
            v += Y[(long long)i * g.r + j] * s;
          }
        out[ti] = v;
      }
    }
  }
  void sync() override {}
  std::string error() override { return ""; }
};
}  // namespace

static tns::Backend* make_backend(int, void*, std::string&) { return new HostBackend(); }
static int backend_davidson(tns::Engine&, double*, double, int, int, double*, int*, std::string& err) {
  err = "not available in the host-logic check library";
  return -2;
}
static int backend_step(tns::Engine&, int, bool, const tns_sweep_opts*, const double*, double*, tns_step_stats*,
                        std::string& err) {
  err = "not available in the host-logic check library";
  return -2;
}
static int backend_sym_eig(tns::Engine&, int, const int*, double*, double*, double*, std::string& err) {
  err = "not available in the host-logic check library";
  return -2;
}
static int backend_diag_noalloc(tns::Engine&, double*, std::string& err) {
  err = "not available in the host-logic check library";
  return -2;
}
static int backend_psi_guess(tns::Engine&, int, double*, long long*, std::string& err) {
  err = "not available in the host-logic check library";
  return -2;
}
static int backend_sweep(tns::Engine&, const tns_sweep_opts*, double*, tns_sweep_stats*, std::string& err) {
  err = "not available in the host-logic check library";
  return -2;
}
static void backend_sched_stats(tns::Engine&, tns_sched_stats* out) { *out = tns_sched_stats{}; }

static long long backend_mem_peak(tns::Engine& e, bool reset) {
  HostBackend& b = *static_cast<HostBackend*>(e.be());
  const long long p = b.peak;
  if (reset) b.peak = b.used;
  return p;
}

static int backend_diag(tns::Engine& e, double* diag, std::string&) {
  tns::Step& st = e.step();
  std::memset(diag, 0, (size_t)st.length * 8);
  for (int ti : st.diag_tasks) {
    const tns::Task& t = st.heff.tasks[ti];
    const tns::PsiBlock& Y = st.psi[t.pad];
    for (int i = 0; i < t.q; ++i)
      for (int j = 0; j < t.r; ++j)
        diag[Y.off + (long long)i * t.r + j] += t.alpha * HostBackend::opL(t, i, i) * HostBackend::opR(t, j, j);
  }
  return 0;
}

#define PFX(name) tnshc_##name
#include "../../paper_2305_05581_gb300/csrc/api_impl.inc"
