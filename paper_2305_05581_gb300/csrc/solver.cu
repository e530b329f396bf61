// solver.cu -- Davidson eigensolver, SVD truncation and the sweep driver on
// the device, plus the C ABI instantiation of the product library.
//
// Davidson (Sec. III: the diagonalisation of H_eff, done iteratively, ~85% of
// the run time): every vector operation (matrix-vector products, projections,
// orthogonalisation, residuals, preconditioner) runs in device FP64 kernels;
// the host only reads the handful of subspace scalars it needs to decide
// convergence.  Truncation: per middle-bond symmetry sector the reduced
// density matrix is diagonalised on the device, the largest D eigenvalues over
// all sectors are kept (D sets the accuracy, Sec. III) and the new site tensor
// plus the wavefunction guess for the next step are formed on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/tns.h"
#include "cuda_backend.h"

namespace tns {

namespace {

struct DBuf {  // owned device buffer
  CudaBackend* be = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() {}
  DBuf(CudaBackend& b, size_t n) : be(&b) { alloc(n); }
  void alloc(size_t n) {
    if (p) {
      cudaStreamSynchronize(be->stream());
      dfree(p);
    }
    p = nullptr;
    bytes = 0;
    if (n == 0) n = 8;
    if (dmalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      be->note(cudaErrorMemoryAllocation, "solver buffer");
      p = nullptr;
      return;
    }
    bytes = n;
  }
  ~DBuf() {
    if (p) {
      cudaStreamSynchronize(be->stream());
      dfree(p);
    }
  }
  double* d() const { return (double*)p; }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

template <typename T>
void put(CudaBackend& be, T* dst, const std::vector<T>& v) {
  if (!v.empty())
    be.note(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, be.stream()), "upload");
}
template <typename T>
void get(CudaBackend& be, std::vector<T>& v, const T* src, size_t n) {
  v.resize(n);
  if (n) be.note(cudaMemcpyAsync(v.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, be.stream()), "download");
  be.note(cudaStreamSynchronize(be.stream()), "download");
}

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  float stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

struct Acc {
  double heff_ms = 0, env_ms = 0, svd_ms = 0;
  long long matvecs = 0;
  double flops = 0;
  int exact_products = 0;  // FP64 products of the reduced-precision form (refreshes)
  double exact_ms = 0;
};

int check(CudaBackend& be, std::string& err) {
  std::string e = be.error();
  if (!e.empty()) {
    err = e;
    return -6;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Davidson
// ---------------------------------------------------------------------------
int davidson(Engine& E, CudaBackend& be, double* X, double tol, int max_iter, int precision, double* energy,
             int* iters, Acc* acc, std::string& err, int block) {
  Step& st = E.step();
  const long long n = st.length;
  if (n <= 0) {
    err = "davidson: empty wavefunction space";
    return -1;
  }
  block = std::max(1, std::min(block, 4));
  // block form: a larger subspace and a thick restart that keeps 2*block
  // Ritz vectors (fewer restarts per correction added)
  const int kmax = (int)std::min<long long>(block > 1 ? 48 : 24, n);
  block = std::min(block, std::max(1, kmax / 8));
  DBuf V(be, sizeof(double) * kmax * n), AV(be, sizeof(double) * kmax * n);
  DBuf diag(be, sizeof(double) * n), x(be, sizeof(double) * n), r(be, sizeof(double) * n),
      avs(be, sizeof(double) * n), t(be, sizeof(double) * n);
  // reduced precision: Ritz vectors kept across a refresh (besides the refreshed one)
  const int lp_keep = precision != 0 ? std::max(0, std::min(3, kmax - 2)) : 0;
  DBuf tmp(be, sizeof(double) * std::max(block > 1 ? 4 * block : 1, 2 * lp_keep) * n);
  DBuf sm(be, sizeof(double) * (3 * 64 * 64 + 256));  // subspace matrix, eigvecs, eigvals, coefs
  DBuf aux(be, 256);
  if (!V.p || !AV.p || !diag.p || !x.p || !r.p || !avs.p || !t.p || !tmp.p || !sm.p || !aux.p) {
    err = "davidson: device allocation failed";
    return -3;
  }
  double* dA = sm.d();
  double* dVs = dA + 64 * 64;
  double* dw = dVs + 64 * 64;
  double* dcoef = dw + 64 * 64;
  double* dscal = dcoef + 128;  // [0] theta, [1] dot result, [2] scale, [8 + i] theta of pair i
  long long* didx = aux.as<long long>();
  DBuf jac_meta(be, 64);
  long long zero_off = 0;
  // diagonal
  {
    DevList& dl = be.dev(st.heff);
    std::vector<int> idx = st.diag_tasks, rng = st.diag_rng;
    DBuf di(be, sizeof(int) * (idx.size() + 1)), dr(be, sizeof(int) * rng.size());
    put(be, di.as<int>(), idx);
    put(be, dr.as<int>(), rng);
    launch_heff_diag(be, dl.tasks, di.as<int>(), dr.as<int>(), (int)st.heff.groups.size(), dl.groups, diag.d());
    be.sync();
  }
  auto dot1 = [&](const double* a, const double* b) {
    launch_multidot(be, a, 0, 1, b, n, dscal + 1);
    std::vector<double> h;
    get(be, h, dscal + 1, 1);
    return h[0];
  };
  const int lowp = precision != 0;
  // nv products in one launch (the block of Davidson vectors shares every
  // operator block read)
  auto matvec = [&](const double* in, double* out, int nv, int prec) {
    Timer tm(be.stream());
    be.run(st.heff, in, out, nv, n, n, prec);
    float ms = tm.stop();
    if (acc) {
      acc->heff_ms += ms;
      acc->matvecs += nv;
      acc->flops += st.heff.flops * nv;
      if (lowp && prec == 0) {
        acc->exact_products += nv;
        acc->exact_ms += ms;
      }
    }
  };
  auto scale_by = [&](double* v, double f) {
    std::vector<double> sc = {f};
    put(be, dscal + 2, sc);
    launch_scale(be, v, dscal + 2, 0, n);
  };
  // orthogonalise w twice against the first kk basis vectors; returns |w|^2
  auto orth = [&](double* w, int kk) {
    if (kk > 0)
      for (int pass = 0; pass < 2; ++pass) {
        launch_multidot(be, V.d(), n, kk, w, n, dcoef);
        launch_axpy_multi(be, V.d(), n, kk, dcoef, -1.0, w, n);
      }
    return dot1(w, w);
  };
  // start vector
  be.note(cudaMemcpyAsync(V.d(), X, sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()), "copy");
  double nx = dot1(V.d(), V.d());
  if (!(nx > 0.0) || !std::isfinite(nx)) {
    launch_argmin(be, diag.d(), n, didx);
    launch_fill_unit(be, V.d(), n, didx);
    nx = 1.0;
  }
  scale_by(V.d(), 1.0 / std::sqrt(nx));
  std::vector<double> H((size_t)kmax * kmax, 0.0);
  int k = 0, it = 0, nnew = 1;
  double theta = 0.0, rn = 1e300;
  bool conv = false;
  double fp64_res = 1e300;
  // reduced precision: the start vector's product is reduced too (the first
  // phase only has to cut the residual by 1e-3); V_0 carries an exact FP64
  // product from the first refresh on
  bool v0_exact = !lowp;
  while (true) {
    // expand by the nnew vectors V[k..k+nnew)
    matvec(V.d() + (long long)k * n, AV.d() + (long long)k * n, nnew, lowp ? precision : 0);
    it += nnew;
    for (int j = 0; j < nnew; ++j) {
      const int kj = k + j;
      launch_multidot(be, V.d(), n, kj + 1, AV.d() + (long long)kj * n, n, dcoef);
      std::vector<double> hc;
      get(be, hc, dcoef, kj + 1);
      if (lowp && v0_exact && kj > 0) {
        // couplings to V_0 from its exact FP64 product: <V_k, H V_0> instead of
        // <V_0, H~ V_k>; near convergence the reduced-precision error of the
        // latter exceeds the coupling itself and would stall the refinement
        hc[0] = dot1(V.d() + (long long)kj * n, AV.d());
      }
      for (int i = 0; i <= kj; ++i) H[(size_t)i * kmax + kj] = H[(size_t)kj * kmax + i] = hc[i];
    }
    k += nnew;
    // Rayleigh-Ritz on the device
    std::vector<double> Hk((size_t)k * k);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Hk[(size_t)i * k + j] = 0.5 * (H[(size_t)i * kmax + j] + H[(size_t)j * kmax + i]);
    put(be, dA, Hk);
    std::vector<long long> offv = {zero_off};
    std::vector<int> nvv = {k}, wo = {0};
    put(be, jac_meta.as<long long>(), offv);
    put(be, (int*)(jac_meta.as<long long>() + 1), nvv);
    put(be, (int*)(jac_meta.as<long long>() + 1) + 1, wo);
    launch_jacobi(be, dA, dVs, dw, jac_meta.as<long long>(), (int*)(jac_meta.as<long long>() + 1),
                  (int*)(jac_meta.as<long long>() + 1) + 1, 1, k, nullptr);
    std::vector<double> w, vs;
    get(be, w, dw, k);
    get(be, vs, dVs, (size_t)k * k);
    std::vector<int> order(k);
    for (int i = 0; i < k; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] < w[b]; });
    auto ritz_coef = [&](int i) {
      std::vector<double> s(k);
      for (int q = 0; q < k; ++q) s[q] = vs[(size_t)q * k + order[i]];
      return s;
    };
    theta = w[order[0]];
    {
      std::vector<double> s = ritz_coef(0), th = {theta};
      put(be, dcoef, s);
      put(be, dscal, th);
    }
    launch_combine(be, V.d(), n, k, dcoef, x.d(), n);
    launch_combine(be, AV.d(), n, k, dcoef, avs.d(), n);
    launch_residual(be, avs.d(), x.d(), dscal, r.d(), n);
    rn = std::sqrt(std::max(0.0, dot1(r.d(), r.d())));
    if (check(be, err)) return -6;
    bool restarted = false;
    if (lowp) {
      // FP64 residual correction: after the first refresh V_0 carries an
      // exact FP64 product, the other basis vectors reduced-precision ones;
      // the Ritz pair is accepted only on an FP64 residual, and every refresh
      // restarts the subspace from the exact pair (x, H x)
      if (k == 1) {
        fp64_res = rn;  // x = V_0: exact after a refresh, a reference residual before the first one
        if (v0_exact && (rn < tol || it >= max_iter)) {
          conv = rn < tol;
          break;
        }
      }
      bool stalled = (k > 1 || !v0_exact) &&
                     (rn < std::max(0.5 * tol, 1e-3 * fp64_res) || k + block > kmax || it >= max_iter);
      if (k == 1 && !v0_exact && !(it >= max_iter)) stalled = false;
      if (stalled) {
        matvec(x.d(), avs.d(), 1, 0);
        ++it;
        double xx = dot1(x.d(), x.d());
        double xh = dot1(x.d(), avs.d());
        theta = xh / xx;
        std::vector<double> th = {theta};
        put(be, dscal, th);
        launch_residual(be, avs.d(), x.d(), dscal, r.d(), n);
        rn = std::sqrt(std::max(0.0, dot1(r.d(), r.d())) / xx);
        fp64_res = rn;
        if (rn < tol || it >= max_iter) {
          conv = rn < tol;
          break;
        }
        // restart from the FP64-exact pair, keeping the next Ritz vectors of
        // the current subspace (their reduced-precision products; diagonal
        // block) with their couplings to the exact pair from its exact product
        const int keep = std::max(0, std::min(lp_keep, k - 1));
        for (int i = 0; i < keep; ++i) {
          std::vector<double> sc = ritz_coef(i + 1);
          put(be, dcoef, sc);
          launch_combine(be, V.d(), n, k, dcoef, tmp.d() + (long long)i * n, n);
          launch_combine(be, AV.d(), n, k, dcoef, tmp.d() + (long long)(lp_keep + i) * n, n);
        }
        v0_exact = true;
        const double f = 1.0 / std::sqrt(xx);
        scale_by(x.d(), f);
        scale_by(avs.d(), f);
        scale_by(r.d(), f);
        be.note(cudaMemcpyAsync(V.d(), x.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()), "copy");
        be.note(cudaMemcpyAsync(AV.d(), avs.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()), "copy");
        std::fill(H.begin(), H.end(), 0.0);
        H[0] = theta;
        for (int i = 0; i < keep; ++i) {
          be.note(cudaMemcpyAsync(V.d() + (long long)(i + 1) * n, tmp.d() + (long long)i * n, sizeof(double) * n,
                                  cudaMemcpyDeviceToDevice, be.stream()),
                  "copy");
          be.note(cudaMemcpyAsync(AV.d() + (long long)(i + 1) * n, tmp.d() + (long long)(lp_keep + i) * n,
                                  sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()),
                  "copy");
        }
        // orthonormal Ritz vectors: re-orthogonalise against the refreshed x
        // (x was rescaled, the others are unit and mutually orthogonal)
        for (int i = 0; i < keep; ++i) {
          double* vi = V.d() + (long long)(i + 1) * n;
          const double c0 = dot1(vi, V.d());
          std::vector<double> cc = {c0};
          put(be, dcoef, cc);
          launch_axpy_multi(be, V.d(), n, 1, dcoef, -1.0, vi, n);
          H[(size_t)(i + 1) * kmax + (i + 1)] = w[order[i + 1]];
          const double hc = dot1(vi, AV.d());  // exact coupling <u_i, A x>
          H[(size_t)(i + 1) * kmax] = H[(size_t)(i + 1)] = hc;
        }
        k = 1 + keep;
        restarted = true;
      }
    } else {
      if (rn < tol || it >= max_iter) {
        conv = rn < tol;
        break;
      }
      if (k + block > kmax) {
        // thick restart: keep the lowest 2*block Ritz vectors (H becomes diagonal)
        const int keep = block > 1 ? std::min(2 * block, k) : 1;
        if (keep == 1) {
          be.note(cudaMemcpyAsync(V.d(), x.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()), "copy");
          be.note(cudaMemcpyAsync(AV.d(), avs.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()),
                  "copy");
        } else {
          for (int i = 0; i < keep; ++i) {
            std::vector<double> s = ritz_coef(i);
            put(be, dcoef, s);
            launch_combine(be, V.d(), n, k, dcoef, tmp.d() + (long long)i * n, n);
            launch_combine(be, AV.d(), n, k, dcoef, tmp.d() + (long long)(keep + i) * n, n);
          }
          be.note(cudaMemcpyAsync(V.d(), tmp.d(), sizeof(double) * n * keep, cudaMemcpyDeviceToDevice, be.stream()),
                  "copy");
          be.note(cudaMemcpyAsync(AV.d(), tmp.d() + (long long)keep * n, sizeof(double) * n * keep,
                                  cudaMemcpyDeviceToDevice, be.stream()),
                  "copy");
        }
        std::fill(H.begin(), H.end(), 0.0);
        for (int i = 0; i < keep; ++i) H[(size_t)i * kmax + i] = w[order[i]];
        k = keep;
        restarted = true;
      }
    }
    // corrections: preconditioned residuals of the lowest Ritz pairs (block
    // form: up to `block` of them), each orthogonalised twice against the
    // basis and the corrections before it
    const int npairs = restarted ? 1 : std::min(block, k);
    nnew = 0;
    for (int i = 0; i < npairs && k + nnew < kmax; ++i) {
      double* slot = V.d() + (long long)(k + nnew) * n;
      double* thp = dscal + 8 + i;
      std::vector<double> thi = {i == 0 ? theta : w[order[i]]};
      put(be, thp, thi);
      const double* ri = r.d();
      if (i > 0) {
        std::vector<double> s = ritz_coef(i);
        put(be, dcoef, s);
        launch_combine(be, V.d(), n, k, dcoef, tmp.d(), n);
        launch_combine(be, AV.d(), n, k, dcoef, t.d(), n);
        launch_residual(be, t.d(), tmp.d(), thp, tmp.d() + n, n);
        ri = tmp.d() + n;
      }
      launch_precond(be, ri, diag.d(), thp, slot, n);
      double nt = orth(slot, k + nnew);
      if (!(nt > 1e-26) && i == 0) {
        // preconditioner gave nothing new: use the residual itself
        be.note(cudaMemcpyAsync(slot, r.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()), "copy");
        nt = orth(slot, k + nnew);
        if (!(nt > 1e-28)) continue;
      } else if (!(nt > 1e-26)) {
        continue;
      }
      scale_by(slot, 1.0 / std::sqrt(nt));
      ++nnew;
    }
    if (nnew == 0) {
      conv = rn < tol;
      break;
    }
  }
  // normalised eigenvector out
  double xx = dot1(x.d(), x.d());
  scale_by(x.d(), 1.0 / std::sqrt(xx));
  be.note(cudaMemcpyAsync(X, x.d(), sizeof(double) * n, cudaMemcpyDeviceToDevice, be.stream()), "copy");
  be.sync();
  if (check(be, err)) return -6;
  if (energy) *energy = theta + E.e_core();
  if (iters) *iters = it;
  if (!conv) {
    err = "davidson: residual " + std::to_string(rn) + " above tolerance after " + std::to_string(it) + " products";
    return -4;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// two-site guess: psi(ql,s1,s2,qr) = site_k(ql,s1) * site_{k+1}(qm,s2)
// ---------------------------------------------------------------------------
void two_site_guess(Engine& E, CudaBackend& be, double* X, int k, const std::vector<PsiBlock>& psi) {
  const Site& a = E.sites()[k];
  const Site& b = E.sites()[k + 1];
  const Basis& bm = E.bonds()[k + 1];
  const Basis& bl = E.bonds()[k];
  TaskList tl;
  for (const PsiBlock& p : psi) {
    Group g;
    g.yoff = p.off;
    g.q = p.m;
    g.r = p.n;
    g.row0 = g.col0 = 0;
    g.nrows = p.m;
    g.ncols = p.n;
    g.t0 = (int)tl.tasks.size();
    int ia = a.index[p.ql * 4 + p.s1];
    if (ia >= 0) {
      int qm = bm.find(bl.q[p.ql] + kSiteQN[p.s1]);
      int ib = qm >= 0 ? b.index[qm * 4 + p.s2] : -1;
      if (ib >= 0) {
        Task tk;
        tk.alpha = 1.0;
        tk.L = a.d + a.blocks[ia].off;
        tk.X = b.d + b.blocks[ib].off;
        tk.R = nullptr;
        tk.q = p.m;
        tk.m = a.blocks[ia].n;
        tk.n = p.n;
        tk.r = p.n;
        tk.flags = TF_RI;
        tk.pad = 0;
        tl.tasks.push_back(tk);
      }
    }
    g.t1 = (int)tl.tasks.size();
    tl.groups.push_back(g);
  }
  be.run(tl, nullptr, X, 1, 0, 0, 0);
  be.sync();
}

// ---------------------------------------------------------------------------
// truncation: split psi at bond k+1 (left_to_right: new left-canonical site k)
// ---------------------------------------------------------------------------
int truncate(Engine& E, CudaBackend& be, const double* psi, bool ltr, int Dmax, double cutoff, double* disc_out,
             std::string& err) {
  Step& st = E.step();
  const int k = st.k;
  const Basis& bl = E.bonds()[k];
  const Catalogue& Rc = E.right(k + 2);
  const QN tgt = E.target();
  struct Seg {
    int a, s, off, dim;
  };
  struct Sec {
    QN q;
    std::vector<Seg> rows, cols;
    int R = 0, C = 0;
    long long moff = 0, roff = 0;
    int woff = 0;
  };
  std::map<QN, Sec> secs;
  for (int ql = 0; ql < bl.size(); ++ql)
    for (int s1 = 0; s1 < 4; ++s1) {
      QN qm = bl.q[ql] + kSiteQN[s1];
      Sec& S = secs[qm];
      S.q = qm;
      S.rows.push_back({ql, s1, S.R, bl.dim[ql]});
      S.R += bl.dim[ql];
    }
  for (int s2 = 0; s2 < 4; ++s2)
    for (int qr = 0; qr < Rc.basis.size(); ++qr) {
      QN qm = tgt - kSiteQN[s2] - Rc.basis.q[qr];
      auto it = secs.find(qm);
      if (it == secs.end()) continue;
      Sec& S = it->second;
      S.cols.push_back({qr, s2, S.C, Rc.basis.dim[qr]});
      S.C += Rc.basis.dim[qr];
    }
  std::vector<Sec*> list;
  long long mtot = 0, rtot = 0;
  int wtot = 0, maxn = 0;
  for (auto& kv : secs) {
    Sec& S = kv.second;
    if (S.R == 0 || S.C == 0) continue;
    S.moff = mtot;
    mtot += (long long)S.R * S.C;
    int nn = ltr ? S.R : S.C;
    S.roff = rtot;
    rtot += (long long)nn * nn;
    S.woff = wtot;
    wtot += nn;
    maxn = std::max(maxn, nn);
    list.push_back(&S);
  }
  if (list.empty()) {
    err = "truncate: no middle-bond sector";
    return -1;
  }
  if (maxn > SYEV_MAXN) {
    err = "truncate: sector matrix larger than " + std::to_string(SYEV_MAXN);
    return -1;
  }
  DBuf M(be, sizeof(double) * mtot), RHO(be, sizeof(double) * rtot), EV(be, sizeof(double) * rtot),
      W(be, sizeof(double) * wtot);
  // gather psi blocks into the sector matrices
  {
    std::vector<long long> so, dof;
    std::vector<int> sld, dld, rows, cols, tr;
    std::map<std::pair<int, int>, int> rowoff, coloff;
    for (Sec* S : list) {
      for (auto& sg : S->rows) rowoff[{sg.a, sg.s}] = sg.off;
      for (auto& sg : S->cols) coloff[{sg.a, sg.s}] = sg.off;
    }
    for (const PsiBlock& p : st.psi) {
      QN qm = bl.q[p.ql] + kSiteQN[p.s1];
      Sec& S = secs[qm];
      if (S.R == 0 || S.C == 0) continue;
      so.push_back(p.off);
      sld.push_back(p.n);
      dof.push_back(S.moff + (long long)rowoff[{p.ql, p.s1}] * S.C + coloff[{p.qr, p.s2}]);
      dld.push_back(S.C);
      rows.push_back(p.m);
      cols.push_back(p.n);
      tr.push_back(0);
    }
    int nb = (int)so.size();
    DBuf a(be, 8 * nb), b(be, 8 * nb), c(be, 4 * nb), d(be, 4 * nb), e(be, 4 * nb), f(be, 4 * nb), g(be, 4 * nb);
    put(be, a.as<long long>(), so);
    put(be, b.as<long long>(), dof);
    put(be, c.as<int>(), sld);
    put(be, d.as<int>(), dld);
    put(be, e.as<int>(), rows);
    put(be, f.as<int>(), cols);
    put(be, g.as<int>(), tr);
    be.zero(M.d(), mtot);
    launch_gather(be, psi, a.as<long long>(), c.as<int>(), M.d(), b.as<long long>(), d.as<int>(), e.as<int>(),
                  f.as<int>(), g.as<int>(), nb);
    be.sync();
  }
  // reduced density matrices rho = M M^T (ltr) or M^T M
  {
    TaskList tl;
    for (Sec* S : list) {
      int nn = ltr ? S->R : S->C;
      Group g;
      g.yoff = S->roff;
      g.q = g.r = nn;
      g.row0 = g.col0 = 0;
      g.nrows = g.ncols = nn;
      g.t0 = (int)tl.tasks.size();
      Task tk;
      tk.alpha = 1.0;
      tk.L = nullptr;
      tk.X = M.d() + S->moff;
      tk.R = M.d() + S->moff;
      tk.q = nn;
      tk.m = nn;
      if (ltr) {
        tk.n = S->C;
        tk.r = nn;
        tk.flags = TF_LI;  // I * M * M^T
      } else {
        tk.n = S->R;
        tk.r = nn;
        tk.flags = TF_LI | TF_XT | TF_RT;  // I * M^T * M
      }
      tk.pad = 0;
      tl.tasks.push_back(tk);
      g.t1 = (int)tl.tasks.size();
      tl.groups.push_back(g);
    }
    be.run(tl, nullptr, RHO.d(), 1, 0, 0, 0);
  }
  // eigen-decomposition per sector
  {
    std::vector<long long> off;
    std::vector<int> nn, wo;
    for (Sec* S : list) {
      off.push_back(S->roff);
      nn.push_back(ltr ? S->R : S->C);
      wo.push_back(S->woff);
    }
    int nmat = (int)list.size();
    DBuf a(be, 8 * nmat), b(be, 4 * nmat), c(be, 4 * nmat);
    put(be, a.as<long long>(), off);
    put(be, b.as<int>(), nn);
    put(be, c.as<int>(), wo);
    DBuf stat(be, 8);
    be.note(cudaMemsetAsync(stat.p, 0, 8, be.stream()), "syev status");
    launch_syev(be, RHO.d(), EV.d(), W.d(), a.as<long long>(), b.as<int>(), c.as<int>(), nmat, maxn, stat.as<int>());
    std::vector<int> sv;
    get(be, sv, stat.as<int>(), 1);
    if (sv[0]) {
      err = "truncate: eigensolver did not converge";
      return -4;
    }
  }
  // global selection of the kept states
  DBuf keep(be, 4 * (size_t)wtot), dd(be, 8);
  launch_select(be, W.d(), nullptr, wtot, Dmax, cutoff * cutoff, keep.as<int>(), dd.d());
  std::vector<int> kf;
  std::vector<double> disc;
  get(be, kf, keep.as<int>(), wtot);
  get(be, disc, dd.d(), 1);
  if (check(be, err)) return -6;
  if (disc_out) *disc_out = disc[0];
  // new bond basis (sectors in increasing order) and the kept eigenvector columns
  Basis nb;
  std::vector<std::vector<int>> kept(list.size());
  for (size_t i = 0; i < list.size(); ++i) {
    Sec* S = list[i];
    int nn = ltr ? S->R : S->C;
    for (int j = 0; j < nn; ++j)
      if (kf[S->woff + j]) kept[i].push_back(j);
    if (!kept[i].empty()) nb.add(S->q, (int)kept[i].size());
  }
  if (nb.size() == 0) {
    err = "truncate: nothing kept";
    return -1;
  }
  // U_sel / V_sel per sector: column gather from the eigenvector matrices
  long long stot = 0;
  std::vector<long long> soff(list.size());
  for (size_t i = 0; i < list.size(); ++i) {
    int nn = ltr ? list[i]->R : list[i]->C;
    soff[i] = stot;
    stot += (long long)nn * kept[i].size();
  }
  DBuf SEL(be, sizeof(double) * std::max(stot, 1LL));
  {
    std::vector<long long> so, dof;
    std::vector<int> sld, dld, rows, cols, tr;
    for (size_t i = 0; i < list.size(); ++i) {
      int nn = ltr ? list[i]->R : list[i]->C;
      int kc = (int)kept[i].size();
      for (int c = 0; c < kc; ++c) {
        so.push_back(list[i]->roff + (long long)kept[i][c] * nn);  // eigenvector = row of EV
        sld.push_back(1);
        dof.push_back(soff[i] + c);
        dld.push_back(kc);
        rows.push_back(nn);
        cols.push_back(1);
        tr.push_back(0);
      }
    }
    int nbk = (int)so.size();
    DBuf a(be, 8 * nbk), b(be, 8 * nbk), c(be, 4 * nbk), d(be, 4 * nbk), e(be, 4 * nbk), f(be, 4 * nbk),
        g(be, 4 * nbk);
    put(be, a.as<long long>(), so);
    put(be, b.as<long long>(), dof);
    put(be, c.as<int>(), sld);
    put(be, d.as<int>(), dld);
    put(be, e.as<int>(), rows);
    put(be, f.as<int>(), cols);
    put(be, g.as<int>(), tr);
    launch_gather(be, EV.d(), a.as<long long>(), c.as<int>(), SEL.d(), b.as<long long>(), d.as<int>(), e.as<int>(),
                  f.as<int>(), g.as<int>(), nbk);
  }
  // centre matrix: C = U^T M (kept x C) for ltr, C = M V (R x kept) otherwise
  long long ctot = 0;
  std::vector<long long> coff(list.size());
  for (size_t i = 0; i < list.size(); ++i) {
    coff[i] = ctot;
    ctot += (long long)kept[i].size() * (ltr ? list[i]->C : list[i]->R);
  }
  DBuf CEN(be, sizeof(double) * std::max(ctot, 1LL));
  {
    TaskList tl;
    for (size_t i = 0; i < list.size(); ++i) {
      Sec* S = list[i];
      int kc = (int)kept[i].size();
      if (!kc) continue;
      Group g;
      g.yoff = coff[i];
      g.row0 = g.col0 = 0;
      g.t0 = (int)tl.tasks.size();
      Task tk;
      tk.alpha = 1.0;
      tk.X = M.d() + S->moff;
      tk.pad = 0;
      if (ltr) {
        g.q = kc;
        g.r = S->C;
        tk.L = SEL.d() + soff[i];
        tk.R = nullptr;
        tk.q = kc;
        tk.m = S->R;
        tk.n = S->C;
        tk.r = S->C;
        tk.flags = TF_LT | TF_RI;
      } else {
        g.q = S->R;
        g.r = kc;
        tk.L = nullptr;
        tk.R = SEL.d() + soff[i];
        tk.q = S->R;
        tk.m = S->R;
        tk.n = S->C;
        tk.r = kc;
        tk.flags = TF_LI | TF_RT;
      }
      g.nrows = g.q;
      g.ncols = g.r;
      tl.tasks.push_back(tk);
      g.t1 = (int)tl.tasks.size();
      tl.groups.push_back(g);
    }
    be.run(tl, nullptr, CEN.d(), 1, 0, 0, 0);
  }
  be.sync();
  if (check(be, err)) return -6;
  // install the new bond and the two site tensors
  E.bonds()[k + 1] = nb;
  int rc = E.alloc_site(k, err);
  if (!rc) rc = E.alloc_site(k + 1, err);
  if (rc) return rc;
  const Site& sa = E.sites()[k];
  const Site& sb = E.sites()[k + 1];
  {
    std::vector<long long> so, dof;
    std::vector<int> sld, dld, rows, cols, tr;
    std::vector<long long> srcbase;  // 0: SEL, 1: CEN
    std::vector<int> which;
    for (size_t i = 0; i < list.size(); ++i) {
      Sec* S = list[i];
      int kc = (int)kept[i].size();
      if (!kc) continue;
      int qm = nb.find(S->q);
      // left factor -> site k blocks (ql, s1) -> qm
      for (auto& sg : S->rows) {
        int bi = sa.index[sg.a * 4 + sg.s];
        if (bi < 0) continue;
        // ltr: rows of U_sel (R x kc); rtl: rows of C (R x kc)
        so.push_back((ltr ? soff[i] : coff[i]) + (long long)sg.off * kc);
        sld.push_back(kc);
        dof.push_back(sa.blocks[bi].off);
        dld.push_back(kc);
        rows.push_back(sg.dim);
        cols.push_back(kc);
        tr.push_back(0);
        which.push_back(ltr ? 0 : 1);
      }
      // right factor -> site k+1 blocks (qm, s2) -> bond k+2
      for (auto& sg : S->cols) {
        int bi = sb.index[qm * 4 + sg.s];
        if (bi < 0) continue;
        if (ltr) {  // C is kc x C: columns [off, off+dim)
          so.push_back(coff[i] + sg.off);
          sld.push_back(S->C);
          tr.push_back(0);
          which.push_back(1);
        } else {  // V_sel is C x kc: rows [off, off+dim), transposed
          so.push_back(soff[i] + (long long)sg.off * kc);
          sld.push_back(kc);
          tr.push_back(1);
          which.push_back(0);
        }
        dof.push_back(sb.blocks[bi].off);
        dld.push_back(sg.dim);
        rows.push_back(kc);
        cols.push_back(sg.dim);
      }
    }
    // two launches: from SEL and from CEN, into site k or k+1
    for (int src = 0; src < 2; ++src)
      for (int dst = 0; dst < 2; ++dst) {
        std::vector<long long> a1, b1;
        std::vector<int> c1, d1, e1, f1, g1;
        // blocks are ordered: for each sector, rows first (site k) then cols (site k+1)
        size_t idx = 0;
        for (size_t i = 0; i < list.size(); ++i) {
          Sec* S = list[i];
          int kc = (int)kept[i].size();
          if (!kc) continue;
          int qm = nb.find(S->q);
          for (auto& sg : S->rows) {
            if (sa.index[sg.a * 4 + sg.s] < 0) continue;
            if (dst == 0 && which[idx] == src) {
              a1.push_back(so[idx]);
              b1.push_back(dof[idx]);
              c1.push_back(sld[idx]);
              d1.push_back(dld[idx]);
              e1.push_back(rows[idx]);
              f1.push_back(cols[idx]);
              g1.push_back(tr[idx]);
            }
            ++idx;
          }
          for (auto& sg : S->cols) {
            if (sb.index[qm * 4 + sg.s] < 0) continue;
            if (dst == 1 && which[idx] == src) {
              a1.push_back(so[idx]);
              b1.push_back(dof[idx]);
              c1.push_back(sld[idx]);
              d1.push_back(dld[idx]);
              e1.push_back(rows[idx]);
              f1.push_back(cols[idx]);
              g1.push_back(tr[idx]);
            }
            ++idx;
          }
        }
        int nbk = (int)a1.size();
        if (!nbk) continue;
        DBuf a(be, 8 * nbk), b(be, 8 * nbk), c(be, 4 * nbk), d(be, 4 * nbk), e(be, 4 * nbk), f(be, 4 * nbk),
            g(be, 4 * nbk);
        put(be, a.as<long long>(), a1);
        put(be, b.as<long long>(), b1);
        put(be, c.as<int>(), c1);
        put(be, d.as<int>(), d1);
        put(be, e.as<int>(), e1);
        put(be, f.as<int>(), f1);
        put(be, g.as<int>(), g1);
        launch_gather(be, src == 0 ? SEL.d() : CEN.d(), a.as<long long>(), c.as<int>(),
                      dst == 0 ? sa.d : sb.d, b.as<long long>(), d.as<int>(), e.as<int>(), f.as<int>(),
                      g.as<int>(), nbk);
        be.sync();
      }
  }
  be.sync();
  return check(be, err);
}

}  // namespace

}  // namespace tns

// ---------------------------------------------------------------------------
// C ABI instantiation with the CUDA backend
// ---------------------------------------------------------------------------
static tns::Backend* make_backend(int device, void* stream, std::string& err) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    err = "no CUDA device";
    return nullptr;
  }
  if (cudaSetDevice(device) != cudaSuccess) return nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  bool own = false;
  if (!s) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    own = true;
  }
  return new tns::CudaBackend(device, s, own);
}

static int backend_sym_eig(tns::Engine& E, int nmat, const int* n, double* A, double* Z, double* w,
                           std::string& err) {
  using namespace tns;
  CudaBackend& be = *static_cast<CudaBackend*>(E.be());
  cudaSetDevice(be.device());
  if (nmat == 0) return 0;
  std::vector<long long> off(nmat);
  std::vector<int> nn(n, n + nmat), wo(nmat);
  long long o = 0;
  int wt = 0, maxn = 0;
  for (int i = 0; i < nmat; ++i) {
    off[i] = o;
    o += (long long)n[i] * n[i];
    wo[i] = wt;
    wt += n[i];
    maxn = std::max(maxn, n[i]);
  }
  if (maxn > SYEV_MAXN) {
    err = "sym_eig: matrix larger than " + std::to_string(SYEV_MAXN);
    return -1;
  }
  DBuf a(be, 8 * (size_t)nmat), b(be, 4 * (size_t)nmat), c(be, 4 * (size_t)nmat), stat(be, 8);
  put(be, a.as<long long>(), off);
  put(be, b.as<int>(), nn);
  put(be, c.as<int>(), wo);
  be.note(cudaMemsetAsync(stat.p, 0, 8, be.stream()), "sym_eig status");
  launch_syev(be, A, Z, w, a.as<long long>(), b.as<int>(), c.as<int>(), nmat, maxn, stat.as<int>());
  std::vector<int> sv;
  get(be, sv, stat.as<int>(), 1);
  if (check(be, err)) return -6;
  if (sv[0]) {
    err = "sym_eig: QR iteration limit reached";
    return -4;
  }
  return 0;
}

static int backend_diag_noalloc(tns::Engine& E, double* diag, std::string& err) {
  tns::CudaBackend& be = *static_cast<tns::CudaBackend*>(E.be());
  cudaSetDevice(be.device());
  return tns::heff_diag_noalloc(be, E.step(), diag, err);
}

static void backend_sched_stats(tns::Engine& E, tns_sched_stats* out) {
  tns::CudaBackend& be = *static_cast<tns::CudaBackend*>(E.be());
  out->tuned = be.tuned;
  out->cache_hits = be.tune_cache_hits;
  for (int p = 0; p < 3; ++p)
    for (int v = 0; v < 4; ++v) out->runs[p][v] = v < tns::kNumVariants ? be.variant_runs[p][v] : 0;
}

static long long backend_mem_peak(tns::Engine& E, bool reset) {
  tns::CudaBackend& be = *static_cast<tns::CudaBackend*>(E.be());
  const long long p = tns::dmem(be.device()).peak;
  if (reset) tns::dmem_reset_peak(be.device());
  return p;
}

static int backend_diag(tns::Engine& E, double* diag, std::string& err) {
  tns::CudaBackend& be = *static_cast<tns::CudaBackend*>(E.be());
  cudaSetDevice(be.device());
  tns::Step& st = E.step();
  tns::DevList& dl = be.dev(st.heff);
  tns::DBuf di(be, sizeof(int) * (st.diag_tasks.size() + 1)), dr(be, sizeof(int) * st.diag_rng.size());
  tns::put(be, di.as<int>(), st.diag_tasks);
  tns::put(be, dr.as<int>(), st.diag_rng);
  tns::launch_heff_diag(be, dl.tasks, di.as<int>(), dr.as<int>(), (int)st.heff.groups.size(), dl.groups, diag);
  be.sync();
  return tns::check(be, err);
}

static int backend_davidson(tns::Engine& E, double* X, double tol, int max_iter, int precision, double* energy,
                            int* iters, std::string& err) {
  tns::CudaBackend& be = *static_cast<tns::CudaBackend*>(E.be());
  cudaSetDevice(be.device());
  return tns::davidson(E, be, X, tol, max_iter, precision, energy, iters, nullptr, err, 1);
}

namespace tns {
namespace {
// one two-site step: env, guess, Davidson, truncation, renormalisation
int one_step(Engine& E, CudaBackend& be, int k, bool ltr, const tns_sweep_opts* o, const double* x0_host,
             double* psi_host, DBuf& X, Acc& acc, double* e, int* its, double* disc, bool* conv, std::string& err) {
  {
    Timer tm(be.stream());
    int rc = E.ensure_step(k, err);
    if (!rc && !(E.step().valid && E.step().k == k)) rc = E.prepare_step(k, err);
    acc.env_ms += tm.stop();
    if (rc) return rc;
  }
  Step& st = E.step();
  if ((long long)X.bytes < 8 * st.length) X.alloc(8 * st.length);
  if (!X.p) {
    err = "step: device allocation failed";
    return -3;
  }
  if (x0_host) {
    be.note(cudaMemcpyAsync(X.d(), x0_host, sizeof(double) * st.length, cudaMemcpyHostToDevice, be.stream()), "x0");
  } else {
    two_site_guess(E, be, X.d(), k, st.psi);
  }
  int rc = davidson(E, be, X.d(), o->tol, o->max_iter, o->precision, e, its, &acc, err, o->block);
  *conv = rc == 0;
  if (rc && rc != -4) return rc;
  err.clear();
  if (psi_host) {
    be.note(cudaMemcpyAsync(psi_host, X.d(), sizeof(double) * st.length, cudaMemcpyDeviceToHost, be.stream()), "psi");
    be.sync();
  }
  {
    Timer tm(be.stream());
    rc = truncate(E, be, X.d(), ltr, o->D, o->cutoff, disc, err);
    acc.svd_ms += tm.stop();
    if (rc) return rc;
  }
  {
    Timer tm(be.stream());
    E.invalidate_left_from(k + 1);
    E.invalidate_right_from(k + 1);
    rc = ltr ? E.grow_left(k, err) : E.grow_right(k, err);
    acc.env_ms += tm.stop();
    if (rc) return rc;
  }
  return check(be, err);
}
}  // namespace
}  // namespace tns

static int backend_psi_guess(tns::Engine& E, int k, double* xh, long long* len, std::string& err) {
  using namespace tns;
  CudaBackend& be = *static_cast<CudaBackend*>(E.be());
  cudaSetDevice(be.device());
  std::vector<PsiBlock> psi;
  std::vector<int> index;
  std::vector<long long> desc;
  long long length = 0;
  psi_layout_of(E.bonds()[k], E.right_basis_of_bond(k + 2), E.target(), psi, index, desc, length);
  if (len) *len = length;
  if (!xh) return 0;
  for (int b : {k, k + 1})
    if (!E.sites()[b].d) {
      err = "psi_guess: site tensor not set";
      return -2;
    }
  DBuf X(be, 8 * std::max(length, 1LL));
  two_site_guess(E, be, X.d(), k, psi);
  be.note(cudaMemcpyAsync(xh, X.d(), 8 * length, cudaMemcpyDeviceToHost, be.stream()), "psi_guess");
  be.sync();
  return check(be, err);
}

static int backend_step(tns::Engine& E, int k, bool ltr, const tns_sweep_opts* o, const double* x0, double* psi,
                        tns_step_stats* stats, std::string& err) {
  using namespace tns;
  CudaBackend& be = *static_cast<CudaBackend*>(E.be());
  cudaSetDevice(be.device());
  auto t0 = std::chrono::steady_clock::now();
  Acc acc;
  DBuf X(be, 8);
  double e = 0, disc = 0;
  int its = 0;
  bool conv = false;
  long long length = 0;
  const long long launches0 = be.launches;
  const double ef0 = E.env_flops(), eb0 = E.env_bytes();
  if (E.step().valid && E.step().k == k) length = E.step().length;
  int rc = one_step(E, be, k, ltr, o, x0, psi, X, acc, &e, &its, &disc, &conv, err);
  if (rc) return rc;
  if (stats) {
    stats->energy = e;
    stats->discarded = disc;
    stats->iters = its;
    stats->converged = conv ? 1 : 0;
    stats->heff_flops = acc.flops;
    stats->heff_seconds = acc.heff_ms * 1e-3;
    stats->env_seconds = acc.env_ms * 1e-3;
    stats->svd_seconds = acc.svd_ms * 1e-3;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->length = length ? length : (long long)(X.bytes / 8);
    stats->bond_dim = (int)E.bonds()[k + 1].total;
    stats->kernel_launches = be.launches - launches0;
    stats->exact_products = acc.exact_products;
    stats->exact_seconds = acc.exact_ms * 1e-3;
    stats->env_flops = E.env_flops() - ef0;
    stats->env_bytes = E.env_bytes() - eb0;
  }
  return 0;
}

static int backend_sweep(tns::Engine& E, const tns_sweep_opts* o, double* energy, tns_sweep_stats* stats,
                         std::string& err) {
  using namespace tns;
  CudaBackend& be = *static_cast<CudaBackend*>(E.be());
  cudaSetDevice(be.device());
  const int N = E.N();
  if (N < 3) {
    err = "sweep: needs at least 3 orbitals";
    return -1;
  }
  auto t0 = std::chrono::steady_clock::now();
  Acc acc;
  std::vector<std::pair<int, bool>> plan;  // (k, split left-to-right)
  for (int k = 0; k <= N - 3; ++k) plan.push_back({k, true});
  plan.push_back({N - 2, false});
  for (int k = N - 3; k >= 1; --k) plan.push_back({k, false});
  double e = 0.0, maxdisc = 0.0;
  int steps = 0;
  DBuf X(be, 8);
  for (int sw = 0; sw < o->nsweeps; ++sw) {
    maxdisc = 0.0;
    for (auto& pk : plan) {
      int its = 0;
      double disc = 0;
      bool conv = false;
      int rc = one_step(E, be, pk.first, pk.second, o, nullptr, nullptr, X, acc, &e, &its, &disc, &conv, err);
      if (rc) return rc;
      maxdisc = std::max(maxdisc, disc);
      ++steps;
      if (o->verbose)
        std::printf("sweep %d step %d %s E=%.12f its=%d disc=%.3e bond=%lld\n", sw, pk.first,
                    pk.second ? "->" : "<-", e, its, disc, (long long)E.bonds()[pk.first + 1].total);
    }
  }
  be.sync();
  if (check(be, err)) return -6;
  if (energy) *energy = e;
  if (stats) {
    stats->energy = e;
    stats->max_discarded = maxdisc;
    stats->matvecs = acc.matvecs;
    stats->heff_flops = acc.flops;
    stats->heff_seconds = acc.heff_ms * 1e-3;
    stats->env_seconds = acc.env_ms * 1e-3;
    stats->svd_seconds = acc.svd_ms * 1e-3;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->steps = steps;
    int mb = 0;
    for (auto& b : E.bonds()) mb = std::max(mb, (int)b.total);
    stats->max_bond = mb;
  }
  return 0;
}

#define PFX(name) tns_##name
#include "api_impl.inc"
