// engine.cpp -- integrals, MPS, operator catalogues, enlarged operators and
// the work lists of the environment build and of H_eff*psi.
//
// Derivation of the enlarged operators (blocking).  For two adjacent parts
// of the orbital chain, a product of full-space operators (X)_first (Y)_second
// equals (X P_first^{|Y|}) (x) Y with block-local operators (Jordan-Wigner
// string inside each part), P = (-1)^n and |Y| the fermionic parity of Y.
// The two-site Hamiltonian is split at the bond between LL = L + dot k and
// RR = dot k+1 + R (normal operators left, complementary right):
//   H = H_LL + H_RR + sum_{a in LL}[c+_a S_a + h.c.] + sum_{x in RR}[T_x c_x + h.c.]
//       + sum_{a<b in LL}[A_ab P_ab + h.c.] + sum_{a,b in LL} B_ab Q_ab,
// and each LL (RR) operator is expanded over L (R) operators and 4x4 dot
// operators with the same rule; the dot factors are scalars per dot block
// (Sec. III.A.2), which gives the tasks B += alpha L A R^T of Eq. (2).
#include "engine.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>

namespace tns {

const QN kSiteQN[4] = {{0, 0}, {1, 1}, {1, -1}, {2, 0}};

// ---------------------------------------------------------------------------
// dot operators (site basis |0>,|up>,|dn>,|updn>, |updn> = c+_up c+_dn |0>)
// ---------------------------------------------------------------------------
namespace {
struct DotOps {
  M4 cd[2], c[2], P, I;
  DotOps() {
    cd[0].a[1][0] = 1.0;   // c+_up |0>  = |up>
    cd[0].a[3][2] = 1.0;   // c+_up |dn> = |updn>
    cd[1].a[2][0] = 1.0;   // c+_dn |0>  = |dn>
    cd[1].a[3][1] = -1.0;  // c+_dn |up> = -|updn>
    c[0] = cd[0].T();
    c[1] = cd[1].T();
    P.a[0][0] = 1.0;
    P.a[1][1] = -1.0;
    P.a[2][2] = -1.0;
    P.a[3][3] = 1.0;
    I = M4::eye();
  }
};
const DotOps& dot() {
  static DotOps d;
  return d;
}
inline int spin2(int p) { return (p & 1) ? -1 : 1; }
inline double sgn_n(int n) { return (n & 1) ? -1.0 : 1.0; }
}  // namespace

// ---------------------------------------------------------------------------
// layouts and catalogues
// ---------------------------------------------------------------------------
void make_layout(const Basis& b, QN dq, Layout& L) {
  L.dq = dq;
  L.in.clear();
  L.out.clear();
  L.off.clear();
  L.size = 0;
  L.blk_of_in.assign(b.size(), -1);
  for (int i = 0; i < b.size(); ++i) {
    int o = b.find(b.q[i] + dq);
    if (o < 0) continue;
    L.blk_of_in[i] = (int)L.in.size();
    L.in.push_back(i);
    L.out.push_back(o);
    L.off.push_back(L.size);
    L.size += (long long)b.dim[o] * b.dim[i];
  }
}

static int blk_of_out(const Basis& b, const Layout& L, int out) {
  int in = b.find(b.q[out] - L.dq);
  return in < 0 ? -1 : L.blk_of_in[in];
}

int Catalogue::layout_for(QN dq) {
  auto it = layout_of.find(dq);
  if (it != layout_of.end()) return it->second;
  Layout L;
  make_layout(basis, dq, L);
  layouts.push_back(L);
  int id = (int)layouts.size() - 1;
  layout_of[dq] = id;
  return id;
}

int Catalogue::add_op(int kind, int i, int j, QN dq) {
  CatOp o;
  o.kind = kind;
  o.i = i;
  o.j = j;
  o.dq = dq;
  o.layout = layout_for(dq);
  o.off = 0;
  ops.push_back(o);
  int id = (int)ops.size() - 1;
  index[key(kind, i, j)] = id;
  return id;
}

void Catalogue::assign_offsets() {
  long long o = 0;
  for (auto& op : ops) {
    op.off = o;
    o += layouts[op.layout].size;
  }
  size = o;
}

static QN dq_of(int kind, int i, int j) {
  switch (kind) {
    case K_H: return {0, 0};
    case K_C: return {1, spin2(i)};
    case K_A: return {2, spin2(i) + spin2(j)};
    case K_B: return {0, spin2(i) - spin2(j)};
    case K_T: return {1, spin2(i)};
    case K_S: return {-1, -spin2(i)};
    case K_P: return {-2, -(spin2(i) + spin2(j))};
    case K_Q: return {0, spin2(j) - spin2(i)};
  }
  return {0, 0};
}

// ---------------------------------------------------------------------------
// engine basics
// ---------------------------------------------------------------------------
Engine::~Engine() {
  for (auto& c : Lcat_) free_cat(c);
  for (auto& c : Rcat_) free_cat(c);
  free_side(step_.L);
  free_side(step_.R);
  for (auto& s : sites_)
    if (s.d) be_->release(s.d);
}

void Engine::free_cat(Catalogue& c) {
  if (c.d) be_->release(c.d);
  c.d = nullptr;
  if (c.h) {
    be_->host_release(c.h);
    ms_.host_used -= std::max(c.size, 1LL) * 8;
  }
  c.h = nullptr;
  c.zero_off.clear();
  c.valid = false;
  c.ops.clear();
  c.index.clear();
  c.layouts.clear();
  c.layout_of.clear();
  c.size = 0;
}

void Engine::free_side(Side& s) {
  if (s.d) be_->release(s.d);
  s.d = nullptr;
  s.size = 0;
  s.exprs.clear();
  s.eops.clear();
  s.eop_index.clear();
  s.mats.clear();
}

int Engine::alloc_cat(Catalogue& c, std::string& err) {
  c.assign_offsets();
  if (c.d) be_->release(c.d);
  c.d = nullptr;
  int rc = make_room(std::max(c.size, 1LL) * 8, err);
  if (rc) return rc;
  c.d = be_->alloc(std::max(c.size, 1LL));
  if (!c.d) {
    err = "device allocation of " + std::to_string(c.size * 8) + " bytes failed (operator catalogue)";
    return -3;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// out-of-HBM environments: the operator catalogues a step does not read may
// leave the device, in stack order (the one needed last first: the farthest
// from the current step), to pinned host memory while the host budget lasts,
// else they are dropped and rebuilt from their neighbours when needed again
// (the tree-traversal cache of Alg. 1 applied to the left/right block chain)
// ---------------------------------------------------------------------------
void Engine::set_memory_budget(long long device_bytes, long long host_bytes) {
  be_->set_budget(device_bytes);
  host_budget_ = host_bytes > 0 ? host_bytes : 0;
}

MemStats Engine::mem_stats() {
  MemStats m = ms_;
  m.device_used = be_->mem_used();
  m.device_limit = be_->mem_limit();
  m.host_budget = host_budget_;
  return m;
}

bool Engine::movable(const Catalogue& c) const {
  if (!c.valid || !c.d) return false;
  for (const Catalogue* k : keep_)
    if (k == &c) return false;
  if (step_.valid && (&c == &Lcat_[step_.k] || &c == &Rcat_[step_.k + 2])) return false;
  return true;
}

int Engine::make_room(long long bytes, std::string& err) {
  // headroom for allocations the library does not plan (stream-ordered
  // scratch, the caller's own buffers on the same device)
  const long long reserve = 512LL << 20;
  for (;;) {
    long long avail = LLONG_MAX;
    const long long lim = be_->mem_limit();
    if (lim > 0) avail = lim - be_->mem_used();
    const long long fr = be_->mem_free() - reserve;
    if (fr < avail) avail = fr;
    if (bytes <= avail) return 0;
    // the movable catalogue farthest from the current step (L_j is read at
    // step j, R_j at step j-2)
    Catalogue* victim = nullptr;
    long long best = -1;
    for (int j = 0; j < (int)Lcat_.size(); ++j) {
      for (int side = 0; side < 2; ++side) {
        Catalogue& c = side ? Rcat_[j] : Lcat_[j];
        if (!movable(c)) continue;
        const long long dist = std::llabs((long long)(side ? j - 2 : j) - pos_) * 4 + side;
        if (dist > best) {
          best = dist;
          victim = &c;
        }
      }
    }
    if (!victim) {
      err = "device memory: " + std::to_string(bytes) + " more bytes needed, " +
            std::to_string(std::max(avail, 0LL)) + " available and no catalogue left to move off the device";
      return -3;
    }
    int rc = evict(*victim, err);
    if (rc) return rc;
  }
}

int Engine::evict(Catalogue& c, std::string& err) {
  (void)err;
  const long long n = std::max(c.size, 1LL);
  if (host_budget_ > 0 && ms_.host_used + n * 8 <= host_budget_) {
    double* h = be_->host_alloc(n);
    if (h) {
      be_->download(h, c.d, n);
      be_->release(c.d);
      c.d = nullptr;
      c.h = h;
      ms_.host_used += n * 8;
      ms_.host_peak = std::max(ms_.host_peak, ms_.host_used);
      ++ms_.staged;
      return 0;
    }
  }
  free_cat(c);  // dropped: rebuilt from its neighbours when needed again
  ++ms_.dropped;
  return 0;
}

int Engine::restore(Catalogue& c, std::string& err) {
  if (c.d) return 0;
  if (!c.valid || !c.h) {
    err = "restore: catalogue not available";
    return -2;
  }
  const long long n = std::max(c.size, 1LL);
  int rc = make_room(n * 8, err);
  if (rc) return rc;
  c.d = be_->alloc(n);
  if (!c.d) {
    err = "device allocation of " + std::to_string(n * 8) + " bytes failed (catalogue restore)";
    return -3;
  }
  be_->upload(c.d, c.h, n);
  be_->host_release(c.h);
  c.h = nullptr;
  ms_.host_used -= n * 8;
  ++ms_.restored;
  return 0;
}

double Engine::t(int p, int q) const {
  if ((p & 1) != (q & 1)) return 0.0;
  return h_[(p >> 1) * N_ + (q >> 1)];
}

double Engine::W(int p, int q, int r, int s) const {
  if ((p & 1) != (s & 1) || (q & 1) != (r & 1)) return 0.0;
  const long long N = N_;
  return v_[(((long long)(p >> 1) * N + (s >> 1)) * N + (q >> 1)) * N + (r >> 1)];
}

template <>
double Engine::tc<double>(int p, int q) const {
  return t(p, q);
}
template <>
Lin Engine::tc<Lin>(int p, int q) const {
  if ((p & 1) != (q & 1)) return Lin(0.0);
  const long long idx = (long long)(p >> 1) * N_ + (q >> 1);
  return Lin::var(h_[idx], idx);
}
template <>
double Engine::Wc<double>(int p, int q, int r, int s) const {
  return W(p, q, r, s);
}
template <>
Lin Engine::Wc<Lin>(int p, int q, int r, int s) const {
  if ((p & 1) != (s & 1) || (q & 1) != (r & 1)) return Lin(0.0);
  const long long N = N_;
  const long long idx = (((long long)(p >> 1) * N + (s >> 1)) * N + (q >> 1)) * N + (r >> 1);
  return Lin::var(v_[idx], N * N + idx);
}

// ---------------------------------------------------------------------------
// tracked scalars
// ---------------------------------------------------------------------------
void Lin::compact() {
  if (c.size() < 2) return;
  std::sort(c.begin(), c.end(), [](const std::pair<long long, double>& a, const std::pair<long long, double>& b) {
    return a.first < b.first;
  });
  size_t w = 0;
  for (size_t i = 0; i < c.size(); ++i) {
    if (w > 0 && c[w - 1].first == c[i].first)
      c[w - 1].second += c[i].second;
    else
      c[w++] = c[i];
  }
  c.resize(w);
}

Lin operator+(const Lin& a, const Lin& b) {
  Lin r;
  r.v = a.v + b.v;
  r.c.reserve(a.c.size() + b.c.size());
  r.c = a.c;
  r.c.insert(r.c.end(), b.c.begin(), b.c.end());
  if (r.c.size() > 64) r.compact();
  return r;
}
Lin operator-(const Lin& a) {
  Lin r = a;
  r.v = -r.v;
  for (auto& x : r.c) x.second = -x.second;
  return r;
}
Lin operator-(const Lin& a, const Lin& b) { return a + (-b); }
Lin operator*(double s, const Lin& a) {
  Lin r = a;
  r.v *= s;
  for (auto& x : r.c) x.second *= s;
  return r;
}
Lin operator*(const Lin& a, const Lin& b) {
  if (a.is_const()) return a.v * b;
  if (b.is_const()) return b.v * a;
  // a product of two integral-dependent coefficients cannot occur in a
  // Hamiltonian linear in the integrals; flag it with a NaN value
  Lin r(std::nan(""));
  return r;
}

int Engine::load_integrals(int N, const double* h, const double* v, double e_core, std::string& err) {
  {
    const char* ve = std::getenv("TNS_VERBOSE_ENV");
    verbose_env_ = ve && *ve && *ve != '0';
  }
  if (N < 2 || N > 128 || !h || !v) {
    err = "load_integrals: need 2 <= N <= 128 and non-null h, v";
    return -1;
  }
  const long long n = N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      if (std::fabs(h[i * N + j] - h[j * N + i]) > 1e-12) {
        err = "load_integrals: h is not symmetric";
        return -1;
      }
  auto V = [&](long long i, long long j, long long k, long long l) { return v[((i * n + j) * n + k) * n + l]; };
  for (long long i = 0; i < n; ++i)
    for (long long j = 0; j < n; ++j)
      for (long long k = 0; k < n; ++k)
        for (long long l = 0; l < n; ++l) {
          double x = V(i, j, k, l);
          if (std::fabs(x - V(j, i, k, l)) > 1e-12 || std::fabs(x - V(i, j, l, k)) > 1e-12 ||
              std::fabs(x - V(k, l, i, j)) > 1e-12) {
            err = "load_integrals: v lacks the 8-fold permutational symmetry";
            return -1;
          }
        }
  if (have_mps_ && N != N_) have_mps_ = false;
  N_ = N;
  h_.assign(h, h + n * n);
  v_.assign(v, v + n * n * n * n);
  e_core_ = e_core;
  have_ints_ = true;
  for (auto& c : Lcat_) free_cat(c);
  for (auto& c : Rcat_) free_cat(c);
  step_.valid = false;
  return 0;
}

// ---------------------------------------------------------------------------
// MPS
// ---------------------------------------------------------------------------
int Engine::mps_define(int N, int n_elec, int two_sz, int D, std::string& err) {
  if (!have_ints_) {
    err = "mps_define: load integrals first";
    return -2;
  }
  if (N != N_ || D < 1 || n_elec < 0 || n_elec > 2 * N || std::abs(two_sz) > n_elec ||
      ((n_elec + two_sz) & 1)) {
    err = "mps_define: inconsistent N / n_elec / two_sz / D";
    return -1;
  }
  for (auto& s : sites_)
    if (s.d) be_->release(s.d);
  sites_.assign(N, Site());
  bonds_.assign(N + 1, Basis());
  target_ = {n_elec, two_sz};
  D_ = D;
  for (auto& c : Lcat_) free_cat(c);
  for (auto& c : Rcat_) free_cat(c);
  Lcat_.assign(N + 1, Catalogue());
  Rcat_.assign(N + 1, Catalogue());
  step_.valid = false;
  have_mps_ = true;
  return 0;
}

void Engine::set_bond_basis(int b, const Basis& basis) { bonds_[b] = basis; }

int Engine::mps_set_bond(int b, int nsec, const int* sec, const int* dims, std::string& err) {
  if (!have_mps_ || b < 0 || b > N_ || nsec < 1 || !sec || !dims) {
    err = "mps_set_bond: bad bond index or arguments";
    return -1;
  }
  Basis B;
  for (int i = 0; i < nsec; ++i) {
    QN q{sec[2 * i], sec[2 * i + 1]};
    if (dims[i] < 1 || (i > 0 && !(B.q.back() < q))) {
      err = "mps_set_bond: sectors must be strictly increasing with positive dims";
      return -1;
    }
    B.add(q, dims[i]);
  }
  bonds_[b] = B;
  invalidate_left_from(b);
  invalidate_right_from(b);
  return 0;
}

int Engine::site_from_host(int b, const std::vector<SiteBlock>& blocks, const std::vector<double>& data,
                           std::string& err) {
  Site& S = sites_[b];
  if (S.d) be_->release(S.d);
  S.blocks = blocks;
  S.index.assign(bonds_[b].size() * 4, -1);
  long long o = 0;
  for (size_t i = 0; i < S.blocks.size(); ++i) {
    S.blocks[i].off = o;
    o += (long long)S.blocks[i].m * S.blocks[i].n;
    S.index[S.blocks[i].ql * 4 + S.blocks[i].s] = (int)i;
  }
  S.size = o;
  S.d = be_->alloc(std::max(o, 1LL));
  if (!S.d) {
    err = "device allocation failed (site tensor)";
    return -3;
  }
  if (!data.empty()) be_->upload(S.d, data.data(), o);
  return 0;
}

static void site_layout(const Basis& l, const Basis& r, std::vector<SiteBlock>& out) {
  out.clear();
  for (int i = 0; i < l.size(); ++i)
    for (int s = 0; s < 4; ++s) {
      int j = r.find(l.q[i] + kSiteQN[s]);
      if (j < 0) continue;
      SiteBlock sb;
      sb.ql = i;
      sb.s = s;
      sb.qr = j;
      sb.m = l.dim[i];
      sb.n = r.dim[j];
      sb.off = 0;
      out.push_back(sb);
    }
}

int Engine::alloc_site(int b, std::string& err) {
  std::vector<SiteBlock> blocks;
  site_layout(bonds_[b], bonds_[b + 1], blocks);
  int rc = site_from_host(b, blocks, std::vector<double>(), err);
  if (!rc) be_->zero(sites_[b].d, std::max(sites_[b].size, 1LL));
  return rc;
}

int Engine::mps_set_site(int b, const double* x, long long len, std::string& err) {
  if (!have_mps_ || b < 0 || b >= N_ || !x || bonds_[b].size() == 0 || bonds_[b + 1].size() == 0) {
    err = "mps_set_site: bad site index, or bonds b and b+1 not set";
    return -1;
  }
  std::vector<SiteBlock> blocks;
  site_layout(bonds_[b], bonds_[b + 1], blocks);
  long long tot = 0;
  for (auto& sb : blocks) tot += (long long)sb.m * sb.n;
  if (tot != len) {
    err = "mps_set_site: length " + std::to_string(len) + " != expected " + std::to_string(tot);
    return -1;
  }
  std::vector<double> data(x, x + len);
  int rc = site_from_host(b, blocks, data, err);
  invalidate_left_from(b + 1);
  invalidate_right_from(b);
  return rc;
}

int Engine::mps_get_site(int b, double* x, long long len, long long* len_out, std::string& err) {
  if (!have_mps_ || b < 0 || b >= N_ || !sites_[b].d) {
    err = "mps_get_site: site not set";
    return -1;
  }
  if (len_out) *len_out = sites_[b].size;
  if (!x) return 0;
  if (len != sites_[b].size) {
    err = "mps_get_site: wrong length";
    return -1;
  }
  be_->download(x, sites_[b].d, len);
  be_->sync();
  return 0;
}

// ---------------------------------------------------------------------------
// checkpoint / restart: integrals, MPS and sweep position in one binary file
//   "TNSCKPT1", int32 version, N, n_elec, two_sz, D, site, left_to_right,
//   double e_core, h (N^2), v (N^4), per bond: int32 nsec + nsec x (n, two_sz,
//   dim), per site: int64 len + len doubles, then the 64-bit FNV-1a hash of
//   every byte before it.  Little-endian hosts (x86-64, Arm64) only.
// ---------------------------------------------------------------------------
namespace {
struct Fnv {
  unsigned long long h = 1469598103934665603ULL;
  void add(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
  }
};
struct Writer {
  FILE* f;
  Fnv fnv;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (!n) return;
    fnv.add(p, n);
    ok = ok && std::fwrite(p, 1, n, f) == n;
  }
  template <class T>
  void val(T x) {
    put(&x, sizeof(T));
  }
};
struct Reader {
  FILE* f;
  Fnv fnv;
  bool ok = true;
  void get(void* p, size_t n) {
    if (!n) return;
    ok = ok && std::fread(p, 1, n, f) == n;
    if (ok) fnv.add(p, n);
  }
  template <class T>
  T val() {
    T x{};
    get(&x, sizeof(T));
    return x;
  }
};
const char kCkptMagic[8] = {'T', 'N', 'S', 'C', 'K', 'P', 'T', '1'};
}  // namespace

int Engine::checkpoint_save(const char* path, int site, int ltr, std::string& err) {
  if (!have_ints_ || !have_mps_) {
    err = "checkpoint_save: no integrals or MPS";
    return -2;
  }
  for (int b = 0; b < N_; ++b)
    if (!sites_[b].d) {
      err = "checkpoint_save: site tensor " + std::to_string(b) + " not set";
      return -2;
    }
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    err = std::string("checkpoint_save: cannot open ") + path;
    return -1;
  }
  Writer w{f};
  w.put(kCkptMagic, 8);
  for (int x : {1, N_, target_.n, target_.s, D_, site, ltr}) w.val<int>(x);
  w.val<double>(e_core_);
  w.put(h_.data(), h_.size() * 8);
  w.put(v_.data(), v_.size() * 8);
  for (int b = 0; b <= N_; ++b) {
    const Basis& B = bonds_[b];
    w.val<int>(B.size());
    for (int i = 0; i < B.size(); ++i) {
      w.val<int>(B.q[i].n);
      w.val<int>(B.q[i].s);
      w.val<int>(B.dim[i]);
    }
  }
  std::vector<double> buf;
  for (int b = 0; b < N_; ++b) {
    buf.resize(sites_[b].size);
    be_->download(buf.data(), sites_[b].d, sites_[b].size);
    be_->sync();
    w.val<long long>(sites_[b].size);
    w.put(buf.data(), buf.size() * 8);
  }
  const unsigned long long hash = w.fnv.h;
  w.ok = w.ok && std::fwrite(&hash, 8, 1, f) == 1;
  const bool ok = w.ok && std::fclose(f) == 0;
  if (!ok) {
    err = std::string("checkpoint_save: write to ") + path + " failed";
    return -1;
  }
  return 0;
}

int Engine::checkpoint_load(const char* path, int* site, int* ltr, std::string& err) {
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    err = std::string("checkpoint_load: cannot open ") + path;
    return -1;
  }
  struct Closer {
    FILE* f;
    ~Closer() { std::fclose(f); }
  } closer{f};
  Reader r{f};
  char magic[8];
  r.get(magic, 8);
  if (!r.ok || std::memcmp(magic, kCkptMagic, 8) != 0) {
    err = "checkpoint_load: not a checkpoint file";
    return -1;
  }
  const int version = r.val<int>(), N = r.val<int>(), ne = r.val<int>(), s2 = r.val<int>(), D = r.val<int>();
  const int st = r.val<int>(), lr = r.val<int>();
  const double ec = r.val<double>();
  if (!r.ok || version != 1 || N < 2 || N > 128 || D < 1) {
    err = "checkpoint_load: unsupported or damaged header";
    return -1;
  }
  const long long n = N;
  std::vector<double> h(n * n), v(n * n * n * n);
  r.get(h.data(), h.size() * 8);
  r.get(v.data(), v.size() * 8);
  std::vector<std::vector<int>> bonds(N + 1);
  for (int b = 0; b <= N && r.ok; ++b) {
    const int ns = r.val<int>();
    if (!r.ok || ns < 1 || ns > 100000) {
      err = "checkpoint_load: damaged bond table";
      return -1;
    }
    bonds[b].resize(3 * ns);
    r.get(bonds[b].data(), bonds[b].size() * 4);
  }
  std::vector<std::vector<double>> sites(N);
  for (int b = 0; b < N && r.ok; ++b) {
    const long long len = r.val<long long>();
    if (!r.ok || len < 0 || len > (1LL << 36)) {
      err = "checkpoint_load: damaged site tensor";
      return -1;
    }
    sites[b].resize(len);
    r.get(sites[b].data(), len * 8);
  }
  const unsigned long long expect = r.fnv.h;
  unsigned long long hash = 0;
  if (!r.ok || std::fread(&hash, 8, 1, f) != 1 || hash != expect) {
    err = "checkpoint_load: truncated or corrupted file (hash mismatch)";
    return -1;
  }
  // everything read and checked: replace the context's problem and state
  int rc = load_integrals(N, h.data(), v.data(), ec, err);
  if (!rc) rc = mps_define(N, ne, s2, D, err);
  for (int b = 0; b <= N && !rc; ++b) {
    const int ns = (int)bonds[b].size() / 3;
    std::vector<int> sec(2 * ns), dim(ns);
    for (int i = 0; i < ns; ++i) {
      sec[2 * i] = bonds[b][3 * i];
      sec[2 * i + 1] = bonds[b][3 * i + 1];
      dim[i] = bonds[b][3 * i + 2];
    }
    rc = mps_set_bond(b, ns, sec.data(), dim.data(), err);
  }
  for (int b = 0; b < N && !rc; ++b) rc = mps_set_site(b, sites[b].data(), (long long)sites[b].size(), err);
  if (rc) return rc;
  if (site) *site = st;
  if (ltr) *ltr = lr;
  return 0;
}

// splitmix64: counter-based generator (Steele, Lea, Flood 2014)
static unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

static double count_dets(int nsites, int n, int s2) {
  if ((n + s2) & 1) return 0.0;
  int nu = (n + s2) / 2, nd = (n - s2) / 2;
  if (nu < 0 || nd < 0 || nu > nsites || nd > nsites) return 0.0;
  auto binom = [](int a, int b) {
    double r = 1.0;
    for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
  };
  return binom(nsites, nu) * binom(nsites, nd);
}

int Engine::mps_init(int N, int n_elec, int two_sz, int D, unsigned long long seed, std::string& err) {
  int rc = mps_define(N, n_elec, two_sz, D, err);
  if (rc) return rc;
  // sector dims per bond: Schmidt-rank bound, proportional share of D,
  // then made consistent so every site tensor can be a right isometry
  std::vector<std::map<QN, long long>> dims(N + 1);
  for (int b = 0; b <= N; ++b) {
    std::map<QN, double> full;
    double tot = 0;
    for (int n = 0; n <= 2 * b; ++n)
      for (int s = -b; s <= b; ++s) {
        double cl = count_dets(b, n, s), cr = count_dets(N - b, n_elec - n, two_sz - s);
        if (cl > 0 && cr > 0) {
          full[{n, s}] = std::min(cl, cr);
          tot += std::min(cl, cr);
        }
      }
    if (full.empty()) {
      err = "mps_init: target sector unreachable";
      return -1;
    }
    std::map<QN, long long> d;
    if (tot <= D) {
      for (auto& kv : full) d[kv.first] = (long long)kv.second;
    } else {
      std::vector<std::pair<double, QN>> frac;
      long long used = 0;
      for (auto& kv : full) {
        double share = D * kv.second / tot;
        long long a = (long long)share;
        d[kv.first] = a;
        used += a;
        frac.push_back({-(share - a), kv.first});
      }
      std::sort(frac.begin(), frac.end(), [](const std::pair<double, QN>& x, const std::pair<double, QN>& y) {
        return x.first < y.first || (x.first == y.first && x.second < y.second);
      });
      for (long long i = 0; i < D - used && i < (long long)frac.size(); ++i) d[frac[i].second] += 1;
    }
    dims[b] = d;
  }
  for (bool changed = true; changed;) {
    changed = false;
    for (int b = N - 1; b >= 0; --b)
      for (auto& kv : dims[b]) {
        long long avail = 0;
        for (int s = 0; s < 4; ++s) {
          auto it = dims[b + 1].find(kv.first + kSiteQN[s]);
          if (it != dims[b + 1].end()) avail += it->second;
        }
        if (kv.second > avail) {
          kv.second = avail;
          changed = true;
        }
      }
    for (int b = 1; b <= N; ++b)
      for (auto& kv : dims[b]) {
        long long avail = 0;
        for (int s = 0; s < 4; ++s) {
          auto it = dims[b - 1].find(kv.first - kSiteQN[s]);
          if (it != dims[b - 1].end()) avail += it->second;
        }
        if (kv.second > avail) {
          kv.second = avail;
          changed = true;
        }
      }
  }
  for (int b = 0; b <= N; ++b) {
    Basis B;
    for (auto& kv : dims[b])
      if (kv.second > 0) B.add(kv.first, (int)kv.second);
    if (B.size() == 0) {
      err = "mps_init: empty bond after consistency (D too small)";
      return -1;
    }
    bonds_[b] = B;
  }
  // 0/1 right isometries: left state i of sector q picks the i-th column of a
  // seed-dependent ordering of the (s, right state) pairs
  for (int b = 0; b < N; ++b) {
    std::vector<SiteBlock> blocks;
    site_layout(bonds_[b], bonds_[b + 1], blocks);
    long long tot = 0;
    std::vector<long long> boff;
    for (auto& sb : blocks) {
      boff.push_back(tot);
      tot += (long long)sb.m * sb.n;
    }
    std::vector<double> data(tot, 0.0);
    const Basis& L = bonds_[b];
    for (int i = 0; i < L.size(); ++i) {
      std::vector<std::pair<unsigned long long, std::pair<int, int>>> cols;  // (key, (block, col))
      for (size_t bi = 0; bi < blocks.size(); ++bi) {
        if (blocks[bi].ql != i) continue;
        for (int c = 0; c < blocks[bi].n; ++c) {
          unsigned long long key = splitmix64(seed ^ splitmix64(((unsigned long long)b << 40) ^
                                                               ((unsigned long long)blocks[bi].s << 32) ^
                                                               (unsigned long long)c));
          cols.push_back({key, {(int)bi, c}});
        }
      }
      std::sort(cols.begin(), cols.end());
      for (int r = 0; r < L.dim[i]; ++r) {
        int bi = cols[r].second.first, c = cols[r].second.second;
        data[boff[bi] + (long long)r * blocks[bi].n + c] = 1.0;
      }
    }
    rc = site_from_host(b, blocks, data, err);
    if (rc) return rc;
  }
  return 0;
}

void Engine::invalidate_left_from(int k) {
  for (int j = std::max(k, 0); j < (int)Lcat_.size(); ++j) free_cat(Lcat_[j]);
  step_.valid = false;
}
void Engine::invalidate_right_from(int k) {
  for (int j = 0; j <= k && j < (int)Rcat_.size(); ++j) free_cat(Rcat_[j]);
  step_.valid = false;
}

// ---------------------------------------------------------------------------
// empty blocks
// ---------------------------------------------------------------------------
void Engine::empty_left(Catalogue& c) {
  c = Catalogue();
  c.left = true;
  c.len = 0;
  c.zero = true;
  c.basis.add({0, 0}, 1);
  c.add_op(K_H, -1, -1, {0, 0});
  for (int x = 0; x < 2 * N_; ++x) c.add_op(K_T, x, -1, dq_of(K_T, x, -1));
}

void Engine::empty_right(Catalogue& c) {
  c = Catalogue();
  c.left = false;
  c.len = N_;
  c.zero = true;
  c.basis.add({0, 0}, 1);
  c.add_op(K_H, -1, -1, {0, 0});
  for (int a = 0; a < 2 * N_; ++a) c.add_op(K_S, a, -1, dq_of(K_S, a, -1));
  for (int a = 0; a < 2 * N_; ++a)
    for (int b = a + 1; b < 2 * N_; ++b) c.add_op(K_P, a, b, dq_of(K_P, a, b));
  for (int a = 0; a < 2 * N_; ++a)
    for (int b = 0; b < 2 * N_; ++b) c.add_op(K_Q, a, b, dq_of(K_Q, a, b));
}

// ---------------------------------------------------------------------------
// expressions and enlarged operators
// ---------------------------------------------------------------------------
namespace {
template <class Sc>
struct Builder {
  SideT<Sc>& S;
  const Catalogue& cat;
  std::map<std::tuple<int, int, int>, int> refs;  // (op, tr, par) -> expr
  Builder(SideT<Sc>& s, const Catalogue& c) : S(s), cat(c) {}

  QN term_dq(const TermT<Sc>& t) const {
    if (t.op < 0) return {0, 0};
    QN d = cat.ops[t.op].dq;
    return t.tr ? -d : d;
  }
  int ref(int op, bool tr = false, int par = 0) {
    if (op >= 0 && cat.zero) return -1;  // an operator of an empty block
    auto key = std::make_tuple(op, (int)tr, par);
    auto it = refs.find(key);
    if (it != refs.end()) return it->second;
    ExprT<Sc> e;
    e.t.push_back({Sc(1.0), op, tr, par});
    e.dq = term_dq(e.t[0]);
    S.exprs.push_back(e);
    int id = (int)S.exprs.size() - 1;
    refs[key] = id;
    return id;
  }
  int ident(int par = 0) { return ref(-1, false, par); }
  // linear combination; returns -1 if all coefficients vanish
  int comb(const std::vector<TermT<Sc>>& ts) {
    ExprT<Sc> e;
    for (auto& t : ts)
      if (t.c != 0.0 && !(t.op >= 0 && cat.zero)) e.t.push_back(t);
    if (e.t.empty()) return -1;
    e.dq = term_dq(e.t[0]);
    S.exprs.push_back(e);
    return (int)S.exprs.size() - 1;
  }
};

QN dot_shift(const M4& y) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (y.a[i][j] != 0.0) return kSiteQN[i] - kSiteQN[j];
  return {0, 0};
}

template <class Sc, class Y>
void add_part(EOpT<Sc>& E, const Y& y, int expr) {
  M4T<Sc> yy(y);
  if (expr < 0 || yy.zero()) return;
  E.parts.push_back({yy, expr});
}
}  // namespace

template <class Sc>
static EOpT<Sc>& new_eop(SideT<Sc>& S, int kind, int i, int j) {
  EOpT<Sc> E;
  E.kind = kind;
  E.i = i;
  E.j = j;
  S.eops.push_back(E);
  S.eop_index[Catalogue::key(kind, i, j)] = (int)S.eops.size() - 1;
  return S.eops.back();
}

// LL = L (x) dot `site`; L holds orbitals 0..site-1.  Operators of LL are the
// catalogue of the left block of orbitals 0..site.
template <class Sc>
void Engine::build_left_eops(const Catalogue& L, int site, SideT<Sc>& S) {
  const DotOps& d = dot();
  Builder<Sc> B(S, L);
  const int m0 = 2 * site, m1 = 2 * site + 1;
  const int ms[2] = {m0, m1};
  const int M = 2 * N_;
  std::vector<int> inL;
  for (int a = 0; a < 2 * site; ++a) inL.push_back(a);
  auto op = [&](int kind, int i, int j) { return L.find(kind, i, j); };

  // site Hamiltonian (one- and two-body terms on the dot)
  M4T<Sc> hs;
  for (int p : ms)
    for (int q : ms) hs = hs + (d.cd[p & 1] * d.c[q & 1]).scale(tc<Sc>(p, q));
  for (int p : ms)
    for (int q : ms)
      for (int r : ms)
        for (int s : ms) {
          Sc w = Wc<Sc>(p, q, r, s);
          if (w != 0.0) hs = hs + (d.cd[p & 1] * d.cd[q & 1] * d.c[r & 1] * d.c[s & 1]).scale(0.5 * w);
        }

  {  // H
    EOpT<Sc>& E = new_eop(S, K_H, -1, -1);
    add_part(E, d.I, B.ref(op(K_H, -1, -1)));
    add_part(E, hs, B.ident());
    for (int a : inL) {
      M4T<Sc> Sa;
      for (int q : ms) {
        Sa = Sa + d.c[q & 1].scale(tc<Sc>(a, q));
        for (int r : ms)
          for (int u : ms) {
            Sc w = Wc<Sc>(a, q, r, u);
            if (w != 0.0) Sa = Sa + (d.cd[q & 1] * d.c[r & 1] * d.c[u & 1]).scale(w);
          }
      }
      int ca = op(K_C, a, -1);
      add_part(E, Sa, B.ref(ca, false, 1));
      add_part(E, Sa.T().scale(-1.0), B.ref(ca, true, 1));
    }
    for (int m : ms) {
      int Tm = op(K_T, m, -1);
      add_part(E, d.c[m & 1], B.ref(Tm, false, 1));
      add_part(E, d.cd[m & 1].scale(-1.0), B.ref(Tm, true, 1));
    }
    for (size_t ai = 0; ai < inL.size(); ++ai)
      for (size_t bi = ai + 1; bi < inL.size(); ++bi) {
        int a = inL[ai], b = inL[bi];
        M4T<Sc> Pp;
        for (int r : ms)
          for (int u : ms) {
            Sc w = Wc<Sc>(a, b, r, u);
            if (w != 0.0) Pp = Pp + (d.c[r & 1] * d.c[u & 1]).scale(w);
          }
        int Aab = op(K_A, a, b);
        add_part(E, Pp, B.ref(Aab));
        add_part(E, Pp.T(), B.ref(Aab, true));
      }
    for (int a : inL)
      for (int b : inL) {
        M4T<Sc> Q;
        for (int q : ms)
          for (int r : ms) {
            Sc w = Wc<Sc>(a, q, r, b) - Wc<Sc>(a, q, b, r);
            if (w != 0.0) Q = Q + (d.cd[q & 1] * d.c[r & 1]).scale(w);
          }
        add_part(E, Q, B.ref(op(K_B, a, b)));
      }
  }
  // creation operators
  for (int a : inL) add_part(new_eop(S, K_C, a, -1), d.I, B.ref(op(K_C, a, -1)));
  for (int m : ms) add_part(new_eop(S, K_C, m, -1), d.cd[m & 1], B.ident(1));
  // A_ab
  for (size_t ai = 0; ai < inL.size(); ++ai)
    for (size_t bi = ai + 1; bi < inL.size(); ++bi)
      add_part(new_eop(S, K_A, inL[ai], inL[bi]), d.I, B.ref(op(K_A, inL[ai], inL[bi])));
  for (int a : inL)
    for (int m : ms) add_part(new_eop(S, K_A, a, m), d.cd[m & 1], B.ref(op(K_C, a, -1), false, 1));
  add_part(new_eop(S, K_A, m0, m1), d.cd[0] * d.cd[1], B.ident());
  // B_ab
  for (int a : inL)
    for (int b : inL) add_part(new_eop(S, K_B, a, b), d.I, B.ref(op(K_B, a, b)));
  for (int a : inL)
    for (int m : ms) {
      add_part(new_eop(S, K_B, a, m), d.c[m & 1], B.ref(op(K_C, a, -1), false, 1));
      add_part(new_eop(S, K_B, m, a), d.cd[m & 1].scale(-1.0), B.ref(op(K_C, a, -1), true, 1));
    }
  for (int m : ms)
    for (int n : ms) add_part(new_eop(S, K_B, m, n), d.cd[m & 1] * d.c[n & 1], B.ident());
  // T_x for x right of LL
  for (int x = 2 * site + 2; x < M; ++x) {
    EOpT<Sc>& E = new_eop(S, K_T, x, -1);
    add_part(E, d.I, B.ref(op(K_T, x, -1)));
    for (int m : ms) {
      std::vector<TermT<Sc>> bs, as;
      for (int q : inL)
        for (int r : inL) {
          Sc w = Wc<Sc>(m, q, r, x) - Wc<Sc>(q, m, r, x);
          if (w != 0.0) bs.push_back({w, op(K_B, q, r), false, 1});
        }
      for (size_t pi = 0; pi < inL.size(); ++pi)
        for (size_t qi = pi + 1; qi < inL.size(); ++qi) {
          int p = inL[pi], q = inL[qi];
          Sc w = Wc<Sc>(p, q, m, x) - Wc<Sc>(q, p, m, x);
          if (w != 0.0) as.push_back({w, op(K_A, p, q), false, 1});
        }
      add_part(E, d.cd[m & 1], B.comb(bs));
      add_part(E, d.c[m & 1], B.comb(as));
    }
    for (int a : inL) {
      M4T<Sc> y1, y2;
      for (int p : ms)
        for (int q : ms) {
          Sc w1 = Wc<Sc>(p, q, a, x);
          if (w1 != 0.0) y1 = y1 + (d.cd[p & 1] * d.cd[q & 1]).scale(w1);
          Sc w2 = Wc<Sc>(a, p, q, x) - Wc<Sc>(p, a, q, x);
          if (w2 != 0.0) y2 = y2 + (d.cd[p & 1] * d.c[q & 1]).scale(w2);
        }
      int ca = op(K_C, a, -1);
      add_part(E, y1, B.ref(ca, true));
      add_part(E, y2, B.ref(ca));
    }
    M4T<Sc> y3;
    for (int p : ms)
      for (int q : ms)
        for (int r : ms) {
          Sc w = Wc<Sc>(p, q, r, x);
          if (w != 0.0) y3 = y3 + (d.cd[p & 1] * d.cd[q & 1] * d.c[r & 1]).scale(w);
        }
    add_part(E, y3, B.ident(1));
  }
}

// RR = dot `site` (x) R; R holds orbitals site+1..N-1.  Operators of RR are
// the catalogue of the right block of orbitals site..N-1.
template <class Sc>
void Engine::build_right_eops(const Catalogue& R, int site, SideT<Sc>& S) {
  const DotOps& d = dot();
  Builder<Sc> B(S, R);
  const int m0 = 2 * site, m1 = 2 * site + 1;
  const int ms[2] = {m0, m1};
  const int M = 2 * N_;
  std::vector<int> inR;
  for (int x = 2 * site + 2; x < M; ++x) inR.push_back(x);
  auto op = [&](int kind, int i, int j) { return R.find(kind, i, j); };
  const M4& P4 = d.P;

  M4T<Sc> hs;
  for (int p : ms)
    for (int q : ms) hs = hs + (d.cd[p & 1] * d.c[q & 1]).scale(tc<Sc>(p, q));
  for (int p : ms)
    for (int q : ms)
      for (int r : ms)
        for (int s : ms) {
          Sc w = Wc<Sc>(p, q, r, s);
          if (w != 0.0) hs = hs + (d.cd[p & 1] * d.cd[q & 1] * d.c[r & 1] * d.c[s & 1]).scale(0.5 * w);
        }
  {  // H
    EOpT<Sc>& E = new_eop(S, K_H, -1, -1);
    add_part(E, hs, B.ident());
    add_part(E, d.I, B.ref(op(K_H, -1, -1)));
    for (int m : ms) {
      int Sm = op(K_S, m, -1);
      add_part(E, d.cd[m & 1] * P4, B.ref(Sm));
      add_part(E, (d.c[m & 1] * P4).scale(-1.0), B.ref(Sm, true));
    }
    for (int x : inR) {
      M4T<Sc> Ts;
      for (int p : ms)
        for (int q : ms)
          for (int r : ms) {
            Sc w = Wc<Sc>(p, q, r, x);
            if (w != 0.0) Ts = Ts + (d.cd[p & 1] * d.cd[q & 1] * d.c[r & 1]).scale(w);
          }
      int cx = op(K_C, x, -1);
      add_part(E, Ts * P4, B.ref(cx, true));
      add_part(E, (Ts.T() * P4).scale(-1.0), B.ref(cx));
    }
    M4 As = d.cd[0] * d.cd[1];
    int Pm = op(K_P, m0, m1);
    add_part(E, As, B.ref(Pm));
    add_part(E, As.T(), B.ref(Pm, true));
    for (int m : ms)
      for (int n : ms) add_part(E, d.cd[m & 1] * d.c[n & 1], B.ref(op(K_Q, m, n)));
  }
  for (int m : ms) add_part(new_eop(S, K_C, m, -1), d.cd[m & 1], B.ident());
  for (int x : inR) add_part(new_eop(S, K_C, x, -1), P4, B.ref(op(K_C, x, -1)));
  // S_a
  for (int a = 0; a < 2 * site; ++a) {
    EOpT<Sc>& E = new_eop(S, K_S, a, -1);
    add_part(E, P4, B.ref(op(K_S, a, -1)));
    for (int m : ms) {
      add_part(E, d.cd[m & 1], B.ref(op(K_P, a, m)));
      add_part(E, d.c[m & 1], B.ref(op(K_Q, a, m)));
      if (tc<Sc>(a, m) != 0.0) add_part(E, d.c[m & 1].scale(tc<Sc>(a, m)), B.ident());
    }
    for (int x : inR) {
      M4T<Sc> y1, y3;
      for (int q : ms)
        for (int r : ms) {
          Sc w1 = Wc<Sc>(a, q, r, x) - Wc<Sc>(a, q, x, r);
          if (w1 != 0.0) y1 = y1 + (d.cd[q & 1] * d.c[r & 1]).scale(w1);
          Sc w3 = Wc<Sc>(a, x, q, r);
          if (w3 != 0.0) y3 = y3 + (d.c[q & 1] * d.c[r & 1]).scale(w3);
        }
      int cx = op(K_C, x, -1);
      add_part(E, y1 * P4, B.ref(cx, true));
      add_part(E, y3 * P4, B.ref(cx));
    }
    M4T<Sc> y;
    for (int q : ms)
      for (int r : ms)
        for (int u : ms) {
          Sc w = Wc<Sc>(a, q, r, u);
          if (w != 0.0) y = y + (d.cd[q & 1] * d.c[r & 1] * d.c[u & 1]).scale(w);
        }
    add_part(E, y, B.ident());
  }
  // P_ab, Q_ab for a, b left of RR
  for (int a = 0; a < 2 * site; ++a)
    for (int b = 0; b < 2 * site; ++b) {
      {
        EOpT<Sc>& E = new_eop(S, K_Q, a, b);
        add_part(E, d.I, B.ref(op(K_Q, a, b)));
        for (int m : ms) {
          std::vector<TermT<Sc>> cqr, crq;
          for (int x : inR) {
            Sc w1 = Wc<Sc>(a, m, x, b) - Wc<Sc>(a, m, b, x);  // c+_m c_x
            Sc w2 = Wc<Sc>(a, x, m, b) - Wc<Sc>(a, x, b, m);  // c+_x c_m
            int cx = op(K_C, x, -1);
            if (w1 != 0.0) cqr.push_back({w1, cx, true, 0});
            if (w2 != 0.0) crq.push_back({w2, cx, false, 0});
          }
          add_part(E, d.cd[m & 1] * P4, B.comb(cqr));
          add_part(E, (d.c[m & 1] * P4).scale(-1.0), B.comb(crq));
        }
        M4T<Sc> y;
        for (int q : ms)
          for (int r : ms) {
            Sc w = Wc<Sc>(a, q, r, b) - Wc<Sc>(a, q, b, r);
            if (w != 0.0) y = y + (d.cd[q & 1] * d.c[r & 1]).scale(w);
          }
        add_part(E, y, B.ident());
      }
      if (a < b) {
        EOpT<Sc>& E = new_eop(S, K_P, a, b);
        add_part(E, d.I, B.ref(op(K_P, a, b)));
        for (int m : ms) {
          std::vector<TermT<Sc>> cf;
          for (int x : inR) {
            Sc w = Wc<Sc>(a, b, m, x) - Wc<Sc>(a, b, x, m);
            if (w != 0.0) cf.push_back({w, op(K_C, x, -1), true, 0});
          }
          add_part(E, d.c[m & 1] * P4, B.comb(cf));
        }
        M4T<Sc> y;
        for (int r : ms)
          for (int u : ms) {
            Sc w = Wc<Sc>(a, b, r, u);
            if (w != 0.0) y = y + (d.c[r & 1] * d.c[u & 1]).scale(w);
          }
        add_part(E, y, B.ident());
      }
    }
}

// dot blocks of every enlarged operator; dot blocks with more than two
// expressions become one materialised expression (partial summation)
template <class Sc>
void Engine::compile_side(SideT<Sc>& S, const Catalogue& cat, bool left) {
  (void)left;
  Builder<Sc> B(S, cat);
  for (auto& E : S.eops) {
    E.dots.clear();
    E.dq = {0, 0};
    bool have_dq = false;
    for (int so = 0; so < 4; ++so)
      for (int si = 0; si < 4; ++si) {
        DotBlockT<Sc> db;
        db.so = so;
        db.si = si;
        for (auto& pr : E.parts) {
          Sc y = pr.first.a[so][si];
          if (y == 0.0) continue;
          bool merged = false;
          for (auto& dt : db.t)
            if (dt.expr == pr.second) {
              dt.s += y;
              merged = true;
            }
          if (!merged) db.t.push_back({y, pr.second});
        }
        std::vector<DotTermT<Sc>> keep;
        for (auto& dt : db.t)
          if (dt.s != 0.0) keep.push_back(dt);
        db.t = keep;
        if (db.t.empty()) continue;
        if (db.t.size() > 2) {
          std::vector<TermT<Sc>> ts;
          for (auto& dt : db.t)
            for (auto& tm : S.exprs[dt.expr].t) ts.push_back({dt.s * tm.c, tm.op, tm.tr, tm.par});
          int e = B.comb(ts);
          db.t.clear();
          if (e < 0) continue;
          db.t.push_back({Sc(1.0), e});
        }
        QN dq = S.exprs[db.t[0].expr].dq + kSiteQN[so] - kSiteQN[si];
        if (!have_dq) {
          E.dq = dq;
          have_dq = true;
        }
        E.dots.push_back(db);
      }
    if (!have_dq) {
      // structurally zero operator: shift from its catalogue kind
      E.dq = dq_of(E.kind, E.i, E.j);
    }
  }
}

constexpr long long kLincombChunk = 8LL << 20;  // terms per partial-sum launch

// the partial sums of a side: every expression with more than one term gets
// its own operator on the side's block basis (layout and offsets only)
void Engine::layout_mats(Side& S, Catalogue& cat) {
  S.mats.clear();
  for (size_t e = 0; e < S.exprs.size(); ++e) {
    Expr& x = S.exprs[e];
    x.mat = -1;
    if (x.t.size() <= 1) continue;
    Mat m;
    m.layout = cat.layout_for(x.dq);
    m.off = 0;
    m.expr = (int)e;
    x.mat = (int)S.mats.size();
    S.mats.push_back(m);
  }
  long long tot = 0;
  for (auto& m : S.mats) {
    m.off = tot;
    tot += cat.layouts[m.layout].size;
  }
  if (S.d) be_->release(S.d);
  S.d = nullptr;
  S.size = tot;
}

// allocate the partial-sum arena of a side and compute it (linear
// combinations of catalogue operators, Sec. III.A.2)
int Engine::fill_mats(Side& S, Catalogue& cat, std::string& err) {
  if (S.size == 0) return 0;
  int rc = make_room(S.size * 8, err);
  if (rc) return rc;
  S.d = be_->alloc(S.size);
  if (!S.d) {
    err = "device allocation of " + std::to_string(S.size * 8) + " bytes failed (partial sums)";
    return -3;
  }
  LCList lc;
  const Basis& bs = cat.basis;
  for (auto& m : S.mats) {
    const Expr& x = S.exprs[m.expr];
    const Layout& L = cat.layouts[m.layout];
    for (size_t b = 0; b < L.in.size(); ++b) {
      int in = L.in[b], out = L.out[b];
      LCBlock blk;
      blk.dst = S.d + m.off + L.off[b];
      blk.rows = bs.dim[out];
      blk.cols = bs.dim[in];
      blk.t0 = (int)lc.terms.size();
      for (auto& tm : x.t) {
        double sign = tm.par == 1 ? sgn_n(bs.q[in].n) : tm.par == 2 ? sgn_n(bs.q[out].n) : 1.0;
        if (tm.op < 0) {
          if (in == out) lc.terms.push_back({tm.c * sign, nullptr, 0});
          continue;
        }
        const CatOp& o = cat.ops[tm.op];
        const Layout& OL = cat.layouts[o.layout];
        int ob = tm.tr ? OL.blk_of_in[out] : OL.blk_of_in[in];
        if (ob < 0) continue;
        if (tm.tr && OL.out[ob] != in) continue;
        if (!tm.tr && OL.out[ob] != out) continue;
        lc.terms.push_back({tm.c * sign, cat.d + o.off + OL.off[ob], tm.tr ? 1 : 0});
      }
      blk.t1 = (int)lc.terms.size();
      lc.blocks.push_back(blk);
      env_bytes_ += 8.0 * blk.rows * blk.cols * (1 + (blk.t1 - blk.t0));
      // the term lists of large partial sums run to hundreds of millions of
      // entries: computed in chunks so that the host list and its device copy
      // stay bounded
      if (lc.terms.size() >= (size_t)kLincombChunk) {
        be_->lincomb(lc);
        lc.blocks.clear();
        lc.terms.clear();
      }
    }
  }
  be_->lincomb(lc);
  return 0;
}

int Engine::materialize(Side& S, Catalogue& cat, std::string& err) {
  layout_mats(S, cat);
  return fill_mats(S, cat, err);
}

// element offsets (in the side's arena) of the partial-sum blocks that are
// identically zero: every term reads a zero catalogue block or none at all
// (an identity term makes a diagonal block nonzero)
static void mats_zero(const Side& S, const Catalogue& cat, std::vector<long long>& out) {
  const Basis& bs = cat.basis;
  for (auto& m : S.mats) {
    const Expr& x = S.exprs[m.expr];
    const Layout& L = cat.layouts[m.layout];
    for (size_t b = 0; b < L.in.size(); ++b) {
      int in = L.in[b], outq = L.out[b];
      bool nz = false;
      for (auto& tm : x.t) {
        if (tm.op < 0) {
          if (in == outq) nz = true;
          continue;
        }
        const CatOp& o = cat.ops[tm.op];
        const Layout& OL = cat.layouts[o.layout];
        int ob = tm.tr ? OL.blk_of_in[outq] : OL.blk_of_in[in];
        if (ob < 0) continue;
        if (tm.tr && OL.out[ob] != in) continue;
        if (!tm.tr && OL.out[ob] != outq) continue;
        if (!cat.zero_off.count(o.off + OL.off[ob])) nz = true;
      }
      (void)bs;
      if (!nz) out.push_back(m.off + L.off[b]);
    }
  }
}

// operand of a product: expression `e` of side S used plain or transposed,
// applied to in-sector `in` of the side's basis
namespace {
struct Operand {
  const double* p;  // block address; for a partial sum whose arena is not allocated yet, its element offset
  int out;
  bool ident, trans;
  bool mat = false;  // the block is a partial sum (in the side's arena)
  double sign;
};
bool resolve(const Side& S, const Catalogue& cat, int e, bool tr, int in, Operand& r) {
  const Expr& x = S.exprs[e];
  const Basis& bs = cat.basis;
  if (x.mat >= 0) {
    const Mat& M = S.mats[x.mat];
    const Layout& L = cat.layouts[M.layout];
    int b;
    if (!tr) {
      b = L.blk_of_in[in];
      if (b < 0) return false;
      r.out = L.out[b];
    } else {
      b = blk_of_out(bs, L, in);
      if (b < 0) return false;
      r.out = L.in[b];
    }
    const long long eo = M.off + L.off[b];
    r.p = S.d ? S.d + eo : reinterpret_cast<const double*>((uintptr_t)eo);
    r.ident = false;
    r.trans = tr;
    r.mat = true;
    r.sign = 1.0;
    return true;
  }
  const Term& t = x.t[0];
  bool tt = tr != t.tr;
  int par = t.par;
  if (tr && par) par = 3 - par;
  r.mat = false;
  if (t.op < 0) {
    r.out = in;
    r.ident = true;
    r.trans = false;
    r.p = nullptr;
  } else {
    const CatOp& o = cat.ops[t.op];
    const Layout& L = cat.layouts[o.layout];
    int b;
    if (!tt) {
      b = L.blk_of_in[in];
      if (b < 0) return false;
      r.out = L.out[b];
    } else {
      b = blk_of_out(bs, L, in);
      if (b < 0) return false;
      r.out = L.in[b];
    }
    r.p = cat.d + o.off + L.off[b];
    r.ident = false;
    r.trans = tt;
  }
  r.sign = t.c * (par == 1 ? sgn_n(bs.q[in].n) : par == 2 ? sgn_n(bs.q[r.out].n) : 1.0);
  return true;
}

double chain_flops(const Task& t) {
  bool li = t.flags & TF_LI, ri = t.flags & TF_RI, xi = t.flags & TF_XI;
  double q = t.q, m = t.m, n = t.n, r = t.r;
  if (xi) {
    if (li || ri) return 2.0 * q * r;  // plain copy-scale / one product
    return 2.0 * q * m * r;
  }
  if (li && ri) return 2.0 * m * n;
  if (li) return 2.0 * m * n * r;
  if (ri) return 2.0 * q * m * n;
  return std::min(2.0 * m * r * (n + q), 2.0 * q * n * (m + r));
}

}  // namespace

// rotate the enlarged operators of a side into the new block (renormalisation)
int Engine::rotate(Side& S, const Catalogue& src, Catalogue& dst, int site, bool left, std::string& err) {
  // dst basis: left -> bond site+1 (left counted); right -> bond `site` right counted
  dst = Catalogue();
  dst.left = left;
  dst.len = left ? site + 1 : site;
  if (left) {
    dst.basis = bonds_[site + 1];
  } else {
    const Basis& b = bonds_[site];
    for (int i = 0; i < b.size(); ++i) dst.basis.add(target_ - b.q[i], b.dim[i]);
  }
  for (auto& E : S.eops) dst.add_op(E.kind, E.i, E.j, E.dq);
  dst.assign_offsets();
  TaskList tl;
  rotation_tasks(S, src, dst, site, left, tl, nullptr);
  tl.nprod = (long long)tl.tasks.size();
  // room for the work list of the renormalisation next to the new catalogue
  int rc = make_room(be_->step_bytes(tl, 0) + std::max(dst.size, 1LL) * 8, err);
  if (!rc) rc = alloc_cat(dst, err);
  if (rc) return rc;
  if (verbose_env_) {
    static const auto t_start = std::chrono::steady_clock::now();
    std::fprintf(stderr,
                 "[tns %.1fs] %s block of %d orbitals: %.2f GB catalogue, %.2f GB partial sums, %lld products, "
                 "device %.1f GB, host %.1f GB\n",
                 std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(),
                 left ? "left" : "right", left ? dst.len : N_ - dst.len, dst.size * 8e-9, S.size * 8e-9,
                 (long long)tl.tasks.size(), be_->mem_used() * 1e-9, ms_.host_used * 1e-9);
  }
  be_->run(tl, nullptr, dst.d, 1, 0, 0, 0);
  be_->forget(tl);
  env_flops_ += tl.flops;
  env_bytes_ += 8.0 * ((double)src.size + (double)S.size + (double)dst.size + (double)sites_[site].size);
  dst.valid = true;
  scan_zero(dst);
  ++ms_.built;
  return 0;
}

void Engine::rotation_tasks(const Side& S, const Catalogue& src, const Catalogue& dst, int site, bool left,
                            TaskList& tl, std::vector<std::array<int, 3>>* prov) {
  const Site& st = sites_[site];
  const Basis& sb = bonds_[site];        // site tensor left bond
  const Basis& sb1 = bonds_[site + 1];   // site tensor right bond
  for (size_t ei = 0; ei < S.eops.size(); ++ei) {
    const EOp& E = S.eops[ei];
    const CatOp& o = dst.ops[ei];
    const Layout& OL = dst.layouts[o.layout];
    for (size_t b = 0; b < OL.in.size(); ++b) {
      int qin = OL.in[b], qout = OL.out[b];  // sectors of dst basis
      Group g;
      g.yoff = o.off + OL.off[b];
      g.q = dst.basis.dim[qout];
      g.r = dst.basis.dim[qin];
      g.row0 = g.col0 = 0;
      g.nrows = g.q;
      g.ncols = g.r;
      g.t0 = (int)tl.tasks.size();
      for (size_t di = 0; di < E.dots.size(); ++di) {
        const DotBlock& db = E.dots[di];
        for (size_t ti = 0; ti < db.t.size(); ++ti) {
          const DotTerm& dt = db.t[ti];
          if (left) {
            // new op (q'' <- q) += A^{so}(ql' -> q'')^T  X(ql' <- ql)  A^{si}(ql -> q)
            QN qo = dst.basis.q[qout] - kSiteQN[db.so];
            QN qi = dst.basis.q[qin] - kSiteQN[db.si];
            int lo = sb.find(qo), li = sb.find(qi);
            if (lo < 0 || li < 0) continue;
            int bo = st.index[lo * 4 + db.so], bi = st.index[li * 4 + db.si];
            if (bo < 0 || bi < 0) continue;
            Operand X;
            if (!resolve(S, src, dt.expr, false, li, X)) continue;
            if (X.out != lo) continue;
            Task tk;
            tk.alpha = dt.s * X.sign;
            tk.L = st.d + st.blocks[bo].off;
            tk.X = X.p;
            tk.R = st.d + st.blocks[bi].off;
            tk.q = g.q;
            tk.m = sb.dim[lo];
            tk.n = sb.dim[li];
            tk.r = g.r;
            tk.flags = TF_LT | TF_RT | (X.ident ? TF_XI : 0) | (X.trans ? TF_XT : 0);
            tk.pad = 0;
            tl.flops += chain_flops(tk);
            tl.tasks.push_back(tk);
            if (prov) prov->push_back({(int)ei, (int)di, (int)ti});
          } else {
            // new op (Q' <- Q) += B^{so}(Q') X(Q'-so <- Q-si) B^{si}(Q)^T ; Q right counted
            QN Qo = dst.basis.q[qout], Qi = dst.basis.q[qin];
            int lo = sb.find(target_ - Qo), li = sb.find(target_ - Qi);  // bond `site` (left counted)
            if (lo < 0 || li < 0) continue;
            int bo = st.index[lo * 4 + db.so], bi = st.index[li * 4 + db.si];
            if (bo < 0 || bi < 0) continue;
            // R-block sectors (own content of orbitals site+1..N-1)
            int ro = src.basis.find(Qo - kSiteQN[db.so]);
            int ri = src.basis.find(Qi - kSiteQN[db.si]);
            if (ro < 0 || ri < 0) continue;
            Operand X;
            if (!resolve(S, src, dt.expr, false, ri, X)) continue;
            if (X.out != ro) continue;
            Task tk;
            tk.alpha = dt.s * X.sign;
            tk.L = st.d + st.blocks[bo].off;
            tk.X = X.p;
            tk.R = st.d + st.blocks[bi].off;
            tk.q = g.q;
            tk.m = src.basis.dim[ro];
            tk.n = src.basis.dim[ri];
            tk.r = g.r;
            tk.flags = (X.ident ? TF_XI : 0) | (X.trans ? TF_XT : 0);
            tk.pad = 0;
            tl.flops += chain_flops(tk);
            tl.tasks.push_back(tk);
            if (prov) prov->push_back({(int)ei, (int)di, (int)ti});
            (void)sb1;
          }
        }
      }
      g.t1 = (int)tl.tasks.size();
      tl.groups.push_back(g);
    }
  }
}

// ---------------------------------------------------------------------------
// environment
// ---------------------------------------------------------------------------
// the two catalogues of step k on the device (a previous step's partial sums
// and work list are released first, so that they leave room)
int Engine::ensure_step(int k, std::string& err) {
  if (step_.valid && step_.k != k) {
    be_->forget(step_.heff);
    be_->forget(step_.heff_full);
    be_->forget(step_.heff_part);
    step_.heff_part.clear();
    step_.heff_full.clear();
    step_.part_key = -1;
    free_side(step_.L);
    free_side(step_.R);
    step_.heff.clear();
    step_.valid = false;
  }
  pos_ = k;
  keep_.clear();
  if (step_.valid) return 0;  // this step's catalogues are on the device and pinned
  int rc = ensure_left(k, err);
  if (rc) return rc;
  keep_.push_back(&Lcat_[k]);
  rc = ensure_right(k + 2, err);
  if (rc) return rc;
  keep_.push_back(&Rcat_[k + 2]);
  if (!Lcat_[k].d || !Rcat_[k + 2].d) {
    err = "step " + std::to_string(k) + ": its two catalogues do not fit on the device together";
    return -3;
  }
  return 0;
}

// L_k resident on the device: restored from host memory, or rebuilt from the
// nearest catalogue below it that still exists (on the device or the host)
int Engine::ensure_left(int k, std::string& err) {
  if (Lcat_[k].valid) {
    if (Lcat_[k].d) return 0;
    std::vector<const Catalogue*> saved = keep_;
    int rc = restore(Lcat_[k], err);
    keep_ = saved;
    return rc;
  }
  int j = k;
  while (j > 0 && !Lcat_[j].valid) --j;
  const std::vector<const Catalogue*> saved = keep_;
  int rc = 0;
  if (j == 0 && !Lcat_[0].valid) {
    empty_left(Lcat_[0]);
    rc = alloc_cat(Lcat_[0], err);
    if (rc) return rc;
    be_->zero(Lcat_[0].d, Lcat_[0].size);
    Lcat_[0].valid = true;
  }
  rc = restore(Lcat_[j], err);
  if (rc) return rc;
  for (; j < k; ++j) {
    if (!sites_[j].d) {
      err = "site tensor " + std::to_string(j) + " not set";
      keep_ = saved;
      return -2;
    }
    keep_ = saved;
    keep_.push_back(&Lcat_[j]);
    const int pos_saved = pos_;
    pos_ = j;
    Side S;
    build_left_eops(Lcat_[j], j, S);
    compile_side(S, Lcat_[j], true);
    rc = materialize(S, Lcat_[j], err);
    if (!rc) rc = rotate(S, Lcat_[j], Lcat_[j + 1], j, true, err);
    be_->sync();
    free_side(S);
    pos_ = pos_saved;
    if (rc) break;
  }
  keep_ = saved;
  return rc;
}

int Engine::ensure_right(int k, std::string& err) {
  if (Rcat_[k].valid) {
    if (Rcat_[k].d) return 0;
    std::vector<const Catalogue*> saved = keep_;
    int rc = restore(Rcat_[k], err);
    keep_ = saved;
    return rc;
  }
  int j = k;
  while (j < N_ && !Rcat_[j].valid) ++j;
  const std::vector<const Catalogue*> saved = keep_;
  int rc = 0;
  if (j == N_ && !Rcat_[N_].valid) {
    empty_right(Rcat_[N_]);
    rc = alloc_cat(Rcat_[N_], err);
    if (rc) return rc;
    be_->zero(Rcat_[N_].d, Rcat_[N_].size);
    Rcat_[N_].valid = true;
  }
  rc = restore(Rcat_[j], err);
  if (rc) return rc;
  for (; j > k; --j) {
    if (!sites_[j - 1].d) {
      err = "site tensor " + std::to_string(j - 1) + " not set";
      keep_ = saved;
      return -2;
    }
    keep_ = saved;
    keep_.push_back(&Rcat_[j]);
    const int pos_saved = pos_;
    pos_ = j - 2;
    Side S;
    build_right_eops(Rcat_[j], j - 1, S);
    compile_side(S, Rcat_[j], false);
    rc = materialize(S, Rcat_[j], err);
    if (!rc) rc = rotate(S, Rcat_[j], Rcat_[j - 1], j - 1, false, err);
    be_->sync();
    free_side(S);
    pos_ = pos_saved;
    if (rc) break;
  }
  keep_ = saved;
  return rc;
}

void psi_layout_of(const Basis& L, const Basis& R, QN target, std::vector<PsiBlock>& psi, std::vector<int>& index,
                   std::vector<long long>& desc, long long& length) {
  psi.clear();
  desc.clear();
  int nqr = R.size();
  index.assign((size_t)L.size() * 16 * nqr, -1);
  long long off = 0;
  for (int ql = 0; ql < L.size(); ++ql)
    for (int s1 = 0; s1 < 4; ++s1)
      for (int s2 = 0; s2 < 4; ++s2) {
        QN need = target - L.q[ql] - kSiteQN[s1] - kSiteQN[s2];
        int qr = R.find(need);
        if (qr < 0) continue;
        PsiBlock pb;
        pb.ql = ql;
        pb.s1 = s1;
        pb.s2 = s2;
        pb.qr = qr;
        pb.m = L.dim[ql];
        pb.n = R.dim[qr];
        pb.off = off;
        off += (long long)pb.m * pb.n;
        index[((size_t)(ql * 4 + s1) * 4 + s2) * nqr + qr] = (int)psi.size();
        psi.push_back(pb);
        long long d9[9] = {L.q[ql].n, L.q[ql].s, s1, s2, R.q[qr].n, R.q[qr].s, pb.m, pb.n, pb.off};
        desc.insert(desc.end(), d9, d9 + 9);
      }
  length = off;
}

Basis Engine::right_basis_of_bond(int b) const {
  Basis R;
  const Basis& bb = bonds_[b];
  for (int i = 0; i < bb.size(); ++i) R.add(target_ - bb.q[i], bb.dim[i]);
  return R;
}

void Engine::build_psi(int k) {
  psi_layout_of(bonds_[k], Rcat_[k + 2].basis, target_, step_.psi, step_.psi_index, step_.desc, step_.length);
}

// operator-table x task-table: every pair of the LL|RR split, every dot
// block pair, every symmetry block of psi
void Engine::build_heff_tasks() {
  Step& st = step_;
  const int k = st.k;
  const Catalogue& Lc = Lcat_[k];
  const Catalogue& Rc = Rcat_[k + 2];
  const Basis& Lb = Lc.basis;
  const int nqr = Rc.basis.size();
  TaskList& tl = st.heff;
  tl.clear();
  st.heff_prov.clear();
  st.heff_row.clear();
  st.nrows = 0;

  struct Pair {
    int eL;
    bool trL;
    int eR;
    bool trR;
    double c;
    int f;
  };
  std::vector<Pair> pairs;
  auto eL = [&](int kind, int i, int j) {
    auto it = st.L.eop_index.find(Catalogue::key(kind, i, j));
    return it == st.L.eop_index.end() ? -1 : it->second;
  };
  auto eR = [&](int kind, int i, int j) {
    auto it = st.R.eop_index.find(Catalogue::key(kind, i, j));
    return it == st.R.eop_index.end() ? -1 : it->second;
  };
  const int nLL = 2 * (k + 1);
  const int M = 2 * N_;
  // H_LL (x) 1 and 1 (x) H_RR use a virtual identity operator (index -2)
  pairs.push_back({eL(K_H, -1, -1), false, -2, false, 1.0, 0});
  pairs.push_back({-2, false, eR(K_H, -1, -1), false, 1.0, 0});
  for (int a = 0; a < nLL; ++a) {
    int l = eL(K_C, a, -1), r = eR(K_S, a, -1);
    pairs.push_back({l, false, r, false, 1.0, 1});
    pairs.push_back({l, true, r, true, -1.0, 1});
  }
  for (int x = nLL; x < M; ++x) {
    int l = eL(K_T, x, -1), r = eR(K_C, x, -1);
    pairs.push_back({l, false, r, true, 1.0, 1});
    pairs.push_back({l, true, r, false, -1.0, 1});
  }
  for (int a = 0; a < nLL; ++a)
    for (int b = a + 1; b < nLL; ++b) {
      int l = eL(K_A, a, b), r = eR(K_P, a, b);
      pairs.push_back({l, false, r, false, 1.0, 0});
      pairs.push_back({l, true, r, true, 1.0, 0});
    }
  for (int a = 0; a < nLL; ++a)
    for (int b = 0; b < nLL; ++b) pairs.push_back({eL(K_B, a, b), false, eR(K_Q, a, b), false, 1.0, 0});

  // per output block task buckets (and where each coefficient comes from)
  std::vector<Operand> rres(nqr);
  std::vector<char> rok(nqr);
  std::vector<int> qr_of((size_t)Lb.size() * 16, -1);  // (q_l, s1, s2) -> the q_r of its psi block, or -1
  for (int ql = 0; ql < Lb.size(); ++ql)
    for (int s12 = 0; s12 < 16; ++s12)
      for (int qr = 0; qr < nqr; ++qr)
        if (st.psi_index[((size_t)ql * 16 + s12) * nqr + qr] >= 0) qr_of[(size_t)ql * 16 + s12] = qr;
  std::vector<std::vector<Task>> bucket(st.psi.size());
  std::vector<std::vector<std::array<int, 6>>> pbucket(st.psi.size());
  std::vector<std::vector<int>> rbucket(st.psi.size());  // operator-pair index (operator-table row) per task
  std::vector<std::vector<char>> zbucket(st.psi.size());  // 0: the task reads an identically zero block
  static const std::vector<DotBlock> kIdent = {
      {0, 0, {{1.0, -1}}}, {1, 1, {{1.0, -1}}}, {2, 2, {{1.0, -1}}}, {3, 3, {{1.0, -1}}}};
  // useful flops (Eq. 2 with the cheaper chain of Sec. III.B): one product per
  // (operator pair, left dot block, right dot block, X block), whatever the
  // number of expressions the two dot blocks hold (their sum is one operator
  // block); a factor counts as the identity only if its dot block is the
  // identity expression alone.  `counted[ql]` marks the X blocks of the
  // current dot-block pair that already have their product counted.
  std::vector<long long> counted(Lb.size(), -1);
  long long dot_pair = 0;
  // a dot block is a multiple of the block's identity when every term is an
  // identity expression (parity signs allowed) and the summed coefficient is
  // the same nonzero number on every sector of the block basis (always so on
  // a one-state basis)
  auto dot_ident = [](const Side& S, const DotBlock& db, const Basis& bs) {
    if (bs.total == 1) return true;
    double c0 = 0.0, c1 = 0.0;  // coefficient of the plain and of the parity-signed identity
    for (const DotTerm& dt : db.t) {
      if (dt.expr == -1) {
        c0 += dt.s;
        continue;
      }
      for (const Term& tm : S.exprs[dt.expr].t) {
        if (tm.op >= 0) return false;
        (tm.par ? c1 : c0) += dt.s * tm.c;
      }
    }
    const double ev = c0 + c1, od = c0 - c1;  // on sectors with even / odd particle number
    bool has_ev = false, has_od = false;
    for (const QN& q : bs.q) (q.n % 2 ? has_od : has_ev) = true;
    if (has_ev && ev == 0.0) return false;
    if (has_od && od == 0.0) return false;
    return !(has_ev && has_od) || ev == od;
  };
  double useful = 0.0;

  for (size_t pi = 0; pi < pairs.size(); ++pi) {
    const Pair& pr = pairs[pi];
    if (pr.eL == -1 || pr.eR == -1) continue;
    const std::vector<DotBlock>& dl = pr.eL == -2 ? kIdent : st.L.eops[pr.eL].dots;
    const std::vector<DotBlock>& dr = pr.eR == -2 ? kIdent : st.R.eops[pr.eR].dots;
    for (size_t ai = 0; ai < dl.size(); ++ai) {
      const auto& a = dl[ai];
      int s1o = pr.trL ? a.si : a.so, s1i = pr.trL ? a.so : a.si;
      for (size_t bi = 0; bi < dr.size(); ++bi) {
        const auto& b = dr[bi];
        int s2o = pr.trR ? b.si : b.so, s2i = pr.trR ? b.so : b.si;
        ++dot_pair;
        const bool li_u = pr.eL == -2 || dot_ident(st.L, a, Lb);
        const bool ri_u = pr.eR == -2 || dot_ident(st.R, b, Rc.basis);
        for (size_t tai = 0; tai < a.t.size(); ++tai)
          for (size_t tbi = 0; tbi < b.t.size(); ++tbi) {
            const auto& ta = a.t[tai];
            const auto& tb = b.t[tbi];
            // the right operand depends on qr only: resolved once per term
            for (int qr = 0; qr < nqr; ++qr) {
              Operand& Ro = rres[qr];
              if (tb.expr == -1) {
                Ro.p = nullptr;
                Ro.out = qr;
                Ro.ident = true;
                Ro.trans = false;
                Ro.sign = 1.0;
                rok[qr] = 1;
              } else {
                rok[qr] = resolve(st.R, Rc, tb.expr, pr.trR, qr, Ro) ? 1 : 0;
              }
            }
            for (int ql = 0; ql < Lb.size(); ++ql) {
              // the target sector fixes q_r given (q_l, s1, s2): at most one X block
              const int qr = qr_of[(ql * 4 + s1i) * 4 + s2i];
              if (qr < 0 || !rok[qr]) continue;
              Operand Lo;
              if (ta.expr == -1) {
                Lo.p = nullptr;
                Lo.out = ql;
                Lo.ident = true;
                Lo.trans = false;
                Lo.sign = 1.0;
              } else if (!resolve(st.L, Lc, ta.expr, pr.trL, ql, Lo)) {
                continue;
              }
              double pl = pr.f ? sgn_n(Lb.q[ql].n + kSiteQN[s1i].n) : 1.0;
              const int* yrow = &st.psi_index[((size_t)(Lo.out * 4 + s1o) * 4 + s2o) * nqr];
              {
                const int xb = st.psi_index[((size_t)(ql * 4 + s1i) * 4 + s2i) * nqr + qr];
                const Operand& Ro = rres[qr];
                const int yb = yrow[Ro.out];
                if (yb < 0) continue;
                const PsiBlock& X = st.psi[xb];
                const PsiBlock& Y = st.psi[yb];
                Task tk;
                tk.alpha = pr.c * ta.s * tb.s * Lo.sign * Ro.sign * pl;
                if (tk.alpha == 0.0) continue;
                tk.L = Lo.p;
                tk.X = reinterpret_cast<const double*>((uintptr_t)X.off);
                tk.R = Ro.p;
                tk.q = Y.m;
                tk.m = X.m;
                tk.n = X.n;
                tk.r = Y.n;
                tk.flags = TF_XV | (Lo.ident ? TF_LI : 0) | (Lo.trans ? TF_LT : 0) | (Ro.ident ? TF_RI : 0) |
                           (Ro.trans ? TF_RT : 0) | (Lo.mat ? TF_LM : 0) | (Ro.mat ? TF_RM : 0);
                tk.pad = xb;
                const bool nz = (Lo.ident || !st.zero_L.count(Lo.p)) && (Ro.ident || !st.zero_R.count(Ro.p));
                if (nz && counted[ql] != dot_pair) {
                  counted[ql] = dot_pair;
                  Task u = tk;
                  u.flags = TF_XV | (li_u ? TF_LI : 0) | (ri_u ? TF_RI : 0);
                  useful += chain_flops(u);
                }
                bucket[yb].push_back(tk);
                zbucket[yb].push_back(nz ? 1 : 0);
                rbucket[yb].push_back((int)pi);
                pbucket[yb].push_back({pr.eL == -2 ? -1 : pr.eL, pr.eL == -2 ? -1 : (int)ai, (int)tai,
                                       pr.eR == -2 ? -1 : pr.eR, pr.eR == -2 ? -1 : (int)bi, (int)tbi});
              }
            }
          }
      }
    }
  }
  // two lists over the same output blocks: every product (the adjoint and the
  // integral gradients differentiate with respect to every operator entry,
  // zero blocks included), and the products whose operator blocks are not
  // identically zero (the forward product: the others add exact zeros)
  TaskList& full = st.heff_full;
  full.clear();
  size_t ntot = 0, nnz = 0;
  for (size_t yb = 0; yb < bucket.size(); ++yb) {
    ntot += bucket[yb].size();
    for (char z : zbucket[yb]) nnz += z;
  }
  full.tasks.reserve(ntot);
  tl.tasks.reserve(nnz);
  st.heff_prov.reserve(ntot);
  st.heff_row.reserve(nnz);
  for (size_t yb = 0; yb < st.psi.size(); ++yb) {
    const PsiBlock& Y = st.psi[yb];
    Group g;
    g.yoff = Y.off;
    g.q = Y.m;
    g.r = Y.n;
    g.row0 = g.col0 = 0;
    g.nrows = Y.m;
    g.ncols = Y.n;
    Group gf = g;
    g.t0 = (int)tl.tasks.size();
    gf.t0 = (int)full.tasks.size();
    for (size_t i = 0; i < bucket[yb].size(); ++i) {
      full.tasks.push_back(bucket[yb][i]);
      if (zbucket[yb][i]) {
        tl.tasks.push_back(bucket[yb][i]);
        st.heff_row.push_back(rbucket[yb][i]);
      }
    }
    for (auto& pv : pbucket[yb]) st.heff_prov.push_back(pv);
    g.t1 = (int)tl.tasks.size();
    gf.t1 = (int)full.tasks.size();
    tl.groups.push_back(g);
    full.groups.push_back(gf);
  }
  full.flops = useful;
  full.nprod = (long long)full.tasks.size();
  tl.flops = useful;
  tl.nprod = (long long)tl.tasks.size();
  st.nrows = (int)pairs.size();
  st.part_key = -1;
  st.diag_tasks.clear();
  st.diag_rng.assign(1, 0);
  for (int g = 0; g < (int)tl.groups.size(); ++g) {
    for (int i = tl.groups[g].t0; i < tl.groups[g].t1; ++i)
      if (tl.tasks[i].pad == g) st.diag_tasks.push_back(i);
    st.diag_rng.push_back((int)st.diag_tasks.size());
  }
  tl.persistent = true;
}

// the operator blocks of a catalogue that are identically zero (an operator
// acting on, or into, a state it annihilates: e.g. any operator with an
// annihilator on the vacuum sector); kept as element offsets
void Engine::scan_zero(Catalogue& c) {
  c.zero_off.clear();
  if (!c.d) return;
  std::vector<const double*> p;
  std::vector<long long> n, off;
  for (const CatOp& o : c.ops) {
    const Layout& L = c.layouts[o.layout];
    for (size_t b = 0; b < L.in.size(); ++b) {
      off.push_back(o.off + L.off[b]);
      p.push_back(c.d + o.off + L.off[b]);
      n.push_back((long long)c.basis.dim[L.out[b]] * c.basis.dim[L.in[b]]);
    }
  }
  std::vector<char> nz;
  be_->nonzero_blocks(p, n, nz);
  for (size_t i = 0; i < nz.size(); ++i)
    if (!nz[i]) c.zero_off.insert(off[i]);
}

int Engine::refresh_step(std::string& err) {
  if (!step_.valid) return -2;
  // the caller may have changed the arenas: their zero blocks are found again
  scan_zero(Lcat_[step_.k]);
  scan_zero(Rcat_[step_.k + 2]);
  return prepare_step(step_.k, err);
}

int Engine::prepare_step(int k, std::string& err) {
  be_->forget(step_.heff);  // the device copy of the previous step's work list
  be_->forget(step_.heff_full);
  be_->forget(step_.heff_part);
  step_.heff_part.clear();
  step_.part_key = -1;
  free_side(step_.L);
  free_side(step_.R);
  step_.valid = false;
  step_.k = k;
  pos_ = k;
  Catalogue& Lc = Lcat_[k];
  Catalogue& Rc = Rcat_[k + 2];
  keep_ = {&Lc, &Rc};
  // host: enlarged operators, partial-sum layouts, psi blocks and the work
  // list (partial-sum operands as arena offsets); nothing is allocated yet
  build_left_eops(Lc, k, step_.L);
  compile_side(step_.L, Lc, true);
  layout_mats(step_.L, Lc);
  build_right_eops(Rc, k + 1, step_.R);
  compile_side(step_.R, Rc, false);
  layout_mats(step_.R, Rc);
  step_.zero_L.clear();
  step_.zero_R.clear();
  for (long long o : Lc.zero_off) step_.zero_L.insert(Lc.d + o);
  for (long long o : Rc.zero_off) step_.zero_R.insert(Rc.d + o);
  {
    std::vector<long long> zo;
    mats_zero(step_.L, Lc, zo);
    for (long long o : zo) step_.zero_L.insert(reinterpret_cast<const double*>((uintptr_t)o));
    zo.clear();
    mats_zero(step_.R, Rc, zo);
    for (long long o : zo) step_.zero_R.insert(reinterpret_cast<const double*>((uintptr_t)o));
  }
  build_psi(k);
  build_heff_tasks();
  // memory plan: partial sums + work list + images + Davidson vectors must fit
  // next to the step's two catalogues once every other catalogue has left the
  // device; refused before the step allocates anything
  const long long need = (step_.L.size + step_.R.size) * 8 + be_->step_bytes(step_.heff, step_.length);
  step_.plan_bytes = need;
  ms_.last_plan = need;
  {
    const long long lim = be_->mem_limit();
    const long long fixed = (long long)(std::max(Lc.size, 1LL) + std::max(Rc.size, 1LL)) * 8;
    if (lim > 0 && need + fixed > lim) {
      err = "memory plan: step " + std::to_string(k) + " needs " + std::to_string(need + fixed) +
            " device bytes (catalogues " + std::to_string(fixed) + ", partial sums " +
            std::to_string((step_.L.size + step_.R.size) * 8) + ", work list, images and vectors " +
            std::to_string(need - (step_.L.size + step_.R.size) * 8) + "), above the limit " + std::to_string(lim);
      step_.heff.clear();
      step_.heff_full.clear();
      return -3;
    }
  }
  int rc = make_room(need, err);
  if (rc) {
    err = "memory plan: " + err;
    step_.heff.clear();
    step_.heff_full.clear();
    return rc;
  }
  rc = fill_mats(step_.L, Lc, err);
  if (!rc) rc = fill_mats(step_.R, Rc, err);
  if (rc) {
    step_.heff.clear();
    step_.heff_full.clear();
    return rc;
  }
  for (TaskList* l : {&step_.heff, &step_.heff_full})
    for (Task& t : l->tasks) {
      if (t.flags & TF_LM) t.L = step_.L.d + (long long)(uintptr_t)t.L;
      if (t.flags & TF_RM) t.R = step_.R.d + (long long)(uintptr_t)t.R;
      t.flags &= ~(TF_LM | TF_RM);
    }
  be_->sync();
  std::string e = be_->error();
  if (!e.empty()) {
    err = e;
    return -6;
  }
  step_.valid = true;
  return 0;
}

int Engine::build_env(int k, std::string& err) {
  if (!have_ints_ || !have_mps_) {
    err = "build_env: load integrals and an MPS first";
    return -2;
  }
  if (k < 0 || k > N_ - 2) {
    err = "build_env: site out of range";
    return -1;
  }
  int rc = ensure_step(k, err);
  if (!rc) {
    // the caller may have changed the two arenas (tns_env_arena): their zero
    // blocks are found again before the work list is built
    scan_zero(Lcat_[k]);
    scan_zero(Rcat_[k + 2]);
    rc = prepare_step(k, err);
  }
  if (!rc) {
    std::string e = be_->error();
    if (!e.empty()) {
      err = e;
      rc = -6;
    }
  }
  return rc;
}

int Engine::grow_left(int k, std::string& err) {
  // L_{k+1} from the step's LL operators and the (new) site tensor k
  int rc = rotate(step_.L, Lcat_[k], Lcat_[k + 1], k, true, err);
  be_->sync();
  return rc;
}

int Engine::grow_right(int k, std::string& err) {
  int rc = rotate(step_.R, Rcat_[k + 2], Rcat_[k + 1], k + 1, false, err);
  be_->sync();
  return rc;
}

int Engine::heff(const double* X, double* Y, int nvec, int precision, std::string& err) {
  if (!step_.valid) {
    err = "heff: call build_env first";
    return -2;
  }
  be_->run(step_.heff, X, Y, nvec, step_.length, step_.length, precision);
  be_->sync();
  std::string e = be_->error();
  if (!e.empty()) {
    err = e;
    // a bounded device wait that gave up leaves the context usable
    return e.find("wait timed out") != std::string::npos ? -5 : -6;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// operator-row split (Sec. "Independent operational tasks": the rows of the
// operator table, i.e. the normal/complementary operator pairs, are
// distributed; every part accumulates all output blocks of its rows and the
// parts' sums add up to H_eff X)
// ---------------------------------------------------------------------------
void Engine::row_parts(int nparts, std::vector<int>& part_of_row) const {
  // cost of a row: the chain flops of its products; longest first onto the
  // least loaded part (deterministic: every caller computes the same split)
  const Step& st = step_;
  std::vector<double> cost(st.nrows, 0.0);
  for (size_t i = 0; i < st.heff.tasks.size(); ++i) cost[st.heff_row[i]] += chain_flops(st.heff.tasks[i]) + 64.0;
  std::vector<int> order(st.nrows);
  for (int r = 0; r < st.nrows; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(nparts, 0.0);
  part_of_row.assign(st.nrows, 0);
  for (int r : order) {
    int best = 0;
    for (int p = 1; p < nparts; ++p)
      if (load[p] < load[best]) best = p;
    part_of_row[r] = best;
    load[best] += cost[r];
  }
}

int Engine::heff_part(const double* X, double* Y, int nvec, int precision, int part, int nparts, std::string& err) {
  if (!step_.valid) {
    err = "heff_part: call build_env first";
    return -2;
  }
  if (nparts < 1 || part < 0 || part >= nparts) {
    err = "heff_part: part must be in [0, nparts)";
    return -1;
  }
  Step& st = step_;
  const long long key = (long long)part * 65536 + nparts;
  if (st.part_key != key) {
    std::vector<int> pr;
    row_parts(nparts, pr);
    TaskList& tl = st.heff_part;
    tl.clear();
    tl.tasks.reserve(st.heff.tasks.size() / nparts + 16);
    for (const Group& g0 : st.heff.groups) {
      Group g = g0;
      g.t0 = (int)tl.tasks.size();
      for (int i = g0.t0; i < g0.t1; ++i)
        if (pr[st.heff_row[i]] == part) tl.tasks.push_back(st.heff.tasks[i]);
      g.t1 = (int)tl.tasks.size();
      tl.groups.push_back(g);
    }
    tl.nprod = (long long)tl.tasks.size();
    tl.flops = 0.0;
    tl.persistent = true;
    st.part_key = key;
  }
  be_->run(st.heff_part, X, Y, nvec, st.length, st.length, precision);
  be_->sync();
  std::string e = be_->error();
  if (!e.empty()) {
    err = e;
    return e.find("wait timed out") != std::string::npos ? -5 : -6;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// adjoint of the grouped triple product
//
// E = <Yb, Y>, Y_blk = sum alpha op(L) op(X) op(R)^T.  For one product
//   Xb_blk        += alpha op(L)^T Yb op(R)
//   d/d op(L)      = alpha Yb op(R) op(X)^T       d/d op(R) = alpha Yb^T op(L) op(X)
// and the gradient of a stored block is the (transposed) gradient of its
// op().  Each is again a triple product, grouped by its target block, so the
// same kernels run it.  Gradients reaching a materialised partial sum flow on
// to the catalogue operators of its terms (adjoint of the linear combination).
// ---------------------------------------------------------------------------
namespace {
struct AdjTarget {
  std::vector<Task> tasks;
};
Task adj_task(double a, const double* P, int pf, const double* M, int mf, const double* S, int sf, int q, int m, int n,
              int r) {
  Task t;
  t.alpha = a;
  t.L = P;
  t.X = M;
  t.R = S;
  t.q = q;
  t.m = m;
  t.n = n;
  t.r = r;
  t.flags = pf | mf | sf;
  t.pad = 0;
  return t;
}
// flags of a stored operand used as op(.)^T given its flags as op(.)
int lflags_T(int f) { return (f & TF_LI) ? TF_LI : ((f & TF_LT) ? 0 : TF_LT); }
int rflags_T(int f) { return (f & TF_RI) ? TF_RI : ((f & TF_RT) ? 0 : TF_RT); }
}  // namespace

int Engine::heff_adjoint(const double* X, const double* Yb, double* Xb, double* Lb, double* Rb, std::string& err) {
  if (!step_.valid) {
    err = "heff_adjoint: call build_env first";
    return -2;
  }
  Step& st = step_;
  const int k = st.k;
  Catalogue& Lc = Lcat_[k];
  Catalogue& Rc = Rcat_[k + 2];
  const TaskList& fw = st.heff_full;
  const long long nL = Lc.size, nR = Rc.size, nML = st.L.size, nMR = st.R.size;
  // temporaries: direct gradients of catalogue blocks and of materialised blocks
  double* GL = Lb ? be_->alloc(std::max(nL, 1LL)) : nullptr;
  double* GR = Rb ? be_->alloc(std::max(nR, 1LL)) : nullptr;
  double* ML = (Lb && nML) ? be_->alloc(nML) : nullptr;
  double* MR = (Rb && nMR) ? be_->alloc(nMR) : nullptr;
  if ((Lb && !GL) || (Rb && !GR) || (Lb && nML && !ML) || (Rb && nMR && !MR)) {
    err = "heff_adjoint: device allocation failed";
    for (double* p : {GL, GR, ML, MR})
      if (p) be_->release(p);
    return -3;
  }
  // target maps: block pointer -> list of tasks
  std::map<const double*, std::vector<Task>> tx, tl_, tr_;
  for (size_t g = 0; g < fw.groups.size(); ++g) {
    const Group& G = fw.groups[g];
    const double* yb = Yb + G.yoff;
    for (int i = G.t0; i < G.t1; ++i) {
      const Task& t = fw.tasks[i];
      const PsiBlock& xbk = st.psi[t.pad];
      const double* xblk = X + xbk.off;
      const int lf = t.flags & (TF_LI | TF_LT), rf = t.flags & (TF_RI | TF_RT);
      const int q = t.q, m = t.m, n = t.n, r = t.r;
      if (Xb) {  // Xb (m x n) += a op(L)^T Yb op(R)
        tx[Xb + xbk.off].push_back(adj_task(t.alpha, t.L, lflags_T(lf), yb, 0, t.R, rflags_T(rf), m, q, r, n));
      }
      if (Lb && !(t.flags & TF_LI)) {
        const int mfR = (t.flags & TF_RI) ? TF_XI : ((t.flags & TF_RT) ? TF_XT : 0);
        if (!(t.flags & TF_LT))  // L (q x m) += a Yb op(R) op(X)^T
          tl_[t.L].push_back(adj_task(t.alpha, yb, 0, t.R, mfR, xblk, 0, q, r, n, m));
        else  // L stored (m x q) += a op(X) op(R)^T Yb^T
          tl_[t.L].push_back(adj_task(t.alpha, xblk, 0, t.R, (t.flags & TF_RI) ? TF_XI : ((t.flags & TF_RT) ? 0 : TF_XT),
                                      yb, 0, m, n, r, q));
      }
      if (Rb && !(t.flags & TF_RI)) {
        if (!(t.flags & TF_RT))  // R (r x n) += a Yb^T op(L) op(X)
          tr_[t.R].push_back(adj_task(t.alpha, yb, TF_LT, t.L,
                                      (t.flags & TF_LI) ? TF_XI : ((t.flags & TF_LT) ? TF_XT : 0), xblk, TF_RT, r, q,
                                      m, n));
        else  // R stored (n x r) += a op(X)^T op(L)^T Yb
          tr_[t.R].push_back(adj_task(t.alpha, xblk, TF_LT, t.L,
                                      (t.flags & TF_LI) ? TF_XI : ((t.flags & TF_LT) ? 0 : TF_XT), yb, TF_RT, n, m, q,
                                      r));
      }
    }
  }
  auto run_map = [&](std::map<const double*, std::vector<Task>>& mp, double* outbase, const double* srcbase,
                     long long srcsize, const std::vector<std::pair<long long, std::pair<int, int>>>& blocks) {
    // groups: every block of [srcbase, srcbase+srcsize) listed in `blocks` (offset, (rows, cols))
    TaskList tl;
    for (auto& b : blocks) {
      Group g;
      g.yoff = b.first;
      g.q = b.second.first;
      g.r = b.second.second;
      g.row0 = g.col0 = 0;
      g.nrows = g.q;
      g.ncols = g.r;
      g.t0 = (int)tl.tasks.size();
      auto it = mp.find(srcbase + b.first);
      if (it != mp.end())
        for (auto& t : it->second) tl.tasks.push_back(t);
      g.t1 = (int)tl.tasks.size();
      tl.groups.push_back(g);
    }
    (void)srcsize;
    be_->run(tl, nullptr, outbase, 1, 0, 0, 0);
  };
  auto cat_blocks = [&](const Catalogue& c) {
    std::vector<std::pair<long long, std::pair<int, int>>> v;
    for (auto& o : c.ops) {
      const Layout& L = c.layouts[o.layout];
      for (size_t b = 0; b < L.in.size(); ++b)
        v.push_back({o.off + L.off[b], {c.basis.dim[L.out[b]], c.basis.dim[L.in[b]]}});
    }
    return v;
  };
  auto mat_blocks = [&](const Side& s, const Catalogue& c) {
    std::vector<std::pair<long long, std::pair<int, int>>> v;
    for (auto& mt : s.mats) {
      const Layout& L = c.layouts[mt.layout];
      for (size_t b = 0; b < L.in.size(); ++b)
        v.push_back({mt.off + L.off[b], {c.basis.dim[L.out[b]], c.basis.dim[L.in[b]]}});
    }
    return v;
  };
  if (Xb) {
    std::vector<std::pair<long long, std::pair<int, int>>> v;
    for (auto& p : st.psi) v.push_back({p.off, {p.m, p.n}});
    run_map(tx, Xb, Xb, st.length, v);
  }
  // second phase: catalogue gradient = direct part + adjoint of the partial sums
  auto finish = [&](Side& S, Catalogue& C, double* G, double* M, double* out, std::map<const double*, std::vector<Task>>& mp) {
    const auto cb = cat_blocks(C);
    run_map(mp, G, C.d, C.size, cb);
    if (M) run_map(mp, M, S.d, S.size, mat_blocks(S, C));
    be_->sync();
    std::map<long long, std::vector<Task>> add;  // target offset -> tasks
    for (auto& b : cb)
      add[b.first].push_back(adj_task(1.0, nullptr, TF_LI, G + b.first, 0, nullptr, TF_RI, b.second.first,
                                      b.second.first, b.second.second, b.second.second));
    const Basis& bs = C.basis;
    for (auto& mt : S.mats) {
      const Expr& x = S.exprs[mt.expr];
      const Layout& L = C.layouts[mt.layout];
      for (size_t b = 0; b < L.in.size(); ++b) {
        const int in = L.in[b], out = L.out[b];
        const double* mb = M + mt.off + L.off[b];
        for (auto& tm : x.t) {
          if (tm.op < 0) continue;
          const double sign = tm.par == 1 ? sgn_n(bs.q[in].n) : tm.par == 2 ? sgn_n(bs.q[out].n) : 1.0;
          const CatOp& o = C.ops[tm.op];
          const Layout& OL = C.layouts[o.layout];
          int ob = tm.tr ? OL.blk_of_in[out] : OL.blk_of_in[in];
          if (ob < 0) continue;
          if (tm.tr && OL.out[ob] != in) continue;
          if (!tm.tr && OL.out[ob] != out) continue;
          const long long toff = o.off + OL.off[ob];
          const int tr = bs.dim[OL.out[ob]], tc = bs.dim[OL.in[ob]];
          add[toff].push_back(adj_task(tm.c * sign, nullptr, TF_LI, mb, tm.tr ? TF_XT : 0, nullptr, TF_RI, tr, tr, tc, tc));
        }
      }
    }
    TaskList tl;
    for (auto& b : cb) {
      Group g;
      g.yoff = b.first;
      g.q = b.second.first;
      g.r = b.second.second;
      g.row0 = g.col0 = 0;
      g.nrows = g.q;
      g.ncols = g.r;
      g.t0 = (int)tl.tasks.size();
      for (auto& t : add[b.first]) tl.tasks.push_back(t);
      g.t1 = (int)tl.tasks.size();
      tl.groups.push_back(g);
    }
    be_->run(tl, nullptr, out, 1, 0, 0, 0);
  };
  if (Lb) finish(st.L, Lc, GL, ML, Lb, tl_);
  if (Rb) finish(st.R, Rc, GR, MR, Rb, tr_);
  be_->sync();
  for (double* p : {GL, GR, ML, MR})
    if (p) be_->release(p);
  std::string e = be_->error();
  if (!e.empty()) {
    err = e;
    return -6;
  }
  return 0;
}


// ===========================================================================
// differentiation form: gradient of E = <psi|H_eff|psi>/<psi|psi> with
// respect to the integrals (1-RDM = dE/dh, 2-RDM = 2 dE/dv), MPS isometries
// fixed.  Reverse mode: per-product values <Ybar, op(L) op(X) op(R)^T> give
// the derivatives of the products' coefficients (which are linear in the
// integrals; Lin records which integrals), operand adjoints carry the
// gradient of every operator block down the renormalisation chain
// (rotation O' = U^T O U, partial sums) to the empty blocks.
// ===========================================================================
namespace {
// a used operand: ident ? I : (trans ? stored^T : stored), rows x cols as used
struct Opd {
  const double* p;
  bool ident, trans;
  int rows, cols;
};
Opd opd_T(Opd o) {
  std::swap(o.rows, o.cols);
  if (!o.ident) o.trans = !o.trans;
  return o;
}
// product a * A B C^T as a task (A rows x C rows)
Task mk(double a, const Opd& A, const Opd& B, const Opd& C) {
  Task t;
  t.alpha = a;
  t.L = A.p;
  t.X = B.p;
  t.R = C.p;
  t.q = A.rows;
  t.m = A.cols;
  t.n = B.cols;
  t.r = C.rows;
  t.flags = (A.ident ? TF_LI : A.trans ? TF_LT : 0) | (B.ident ? TF_XI : B.trans ? TF_XT : 0) |
            (C.ident ? TF_RI : C.trans ? TF_RT : 0);
  t.pad = 0;
  return t;
}

// gradient buffers mirroring forward arenas; adjoint products grouped by the
// stored block they write
struct AdjSink {
  struct Region {
    const double* base;
    long long size;
    double* grad;
    std::map<long long, std::pair<std::pair<int, int>, std::vector<Task>>> blocks;
  };
  std::vector<Region> regions;
  void region(const double* base, long long size, double* grad) { regions.push_back({base, size, grad, {}}); }
  int find(const double* p) const {
    for (size_t i = 0; i < regions.size(); ++i)
      if (p >= regions[i].base && p < regions[i].base + regions[i].size) return (int)i;
    return -1;
  }
  void add(const double* stored, int rows, int cols, const Task& t) {
    const int r = find(stored);
    if (r < 0) return;
    auto& e = regions[r].blocks[stored - regions[r].base];
    e.first = {rows, cols};
    e.second.push_back(t);
  }
  // adjoint of one forward product Y(q x r) += a A B C^T with output gradient Yb
  void adjoint(const Task& t, const double* xv, const double* Yb) {
    const Opd A{t.L, (t.flags & TF_LI) != 0, (t.flags & TF_LT) != 0, t.q, t.m};
    const double* xp = (t.flags & TF_XV) ? xv + (long long)(size_t)t.X : t.X;
    const Opd B{xp, (t.flags & TF_XI) != 0, (t.flags & TF_XT) != 0, t.m, t.n};
    const Opd C{t.R, (t.flags & TF_RI) != 0, (t.flags & TF_RT) != 0, t.r, t.n};
    const Opd Y{Yb, false, false, t.q, t.r};
    const double a = t.alpha;
    if (!A.ident && find(A.p) >= 0) {  // dA = Yb C B^T
      if (!A.trans)
        add(A.p, t.q, t.m, mk(a, Y, C, B));
      else
        add(A.p, t.m, t.q, mk(a, B, opd_T(C), Y));
    }
    if (!B.ident && find(B.p) >= 0) {  // dB = A^T Yb C
      if (!B.trans)
        add(B.p, t.m, t.n, mk(a, opd_T(A), Y, opd_T(C)));
      else
        add(B.p, t.n, t.m, mk(a, opd_T(C), opd_T(Y), opd_T(A)));
    }
    if (!C.ident && find(C.p) >= 0) {  // dC = Yb^T A B
      if (!C.trans)
        add(C.p, t.r, t.n, mk(a, opd_T(Y), A, opd_T(B)));
      else
        add(C.p, t.n, t.r, mk(a, opd_T(B), opd_T(A), opd_T(Y)));
    }
  }
  // write every region's gradient blocks (blocks without products are left as they are)
  void flush(Backend* be) {
    for (auto& R : regions) {
      TaskList tl;
      for (auto& kv : R.blocks) {
        Group g;
        g.yoff = kv.first;
        g.q = kv.second.first.first;
        g.r = kv.second.first.second;
        g.row0 = g.col0 = 0;
        g.nrows = g.q;
        g.ncols = g.r;
        g.t0 = (int)tl.tasks.size();
        for (auto& t : kv.second.second) tl.tasks.push_back(t);
        g.t1 = (int)tl.tasks.size();
        tl.groups.push_back(g);
      }
      if (!tl.groups.empty()) be->run(tl, nullptr, R.grad, 1, 0, 0, 0);
      R.blocks.clear();
    }
  }
};

// every block (offset, rows, cols) of a catalogue
std::vector<std::array<long long, 3>> blocks_of(const Catalogue& c) {
  std::vector<std::array<long long, 3>> v;
  for (auto& o : c.ops) {
    const Layout& L = c.layouts[o.layout];
    for (size_t b = 0; b < L.in.size(); ++b)
      v.push_back({o.off + L.off[b], c.basis.dim[L.out[b]], c.basis.dim[L.in[b]]});
  }
  return v;
}

void acc_lin(std::vector<double>& g, const Lin& f, double w) {
  for (auto& x : f.c) g[x.first] += w * x.second;
}
}  // namespace

int Engine::integral_gradient(const double* psi, std::vector<double>& g, std::string& err) {
  if (!step_.valid) {
    err = "integral_gradient: call build_env first";
    return -2;
  }
  Step& st = step_;
  const int k = st.k;
  const long long N = N_, len = st.length;
  g.assign(N * N + N * N * N * N, 0.0);
  std::vector<double> ph(len);
  be_->download(ph.data(), psi, len);
  be_->sync();
  double n2 = 0.0;
  for (double x : ph) n2 += x * x;
  if (!(n2 > 0.0)) {
    err = "integral_gradient: zero wavefunction";
    return -1;
  }
  std::vector<double> yh(len);
  for (long long i = 0; i < len; ++i) yh[i] = ph[i] / n2;
  double* Yb = be_->alloc(std::max(len, 1LL));
  if (!Yb) {
    err = "integral_gradient: allocation failed";
    return -3;
  }
  be_->upload(Yb, yh.data(), len);
  std::vector<double*> owned = {Yb};
  auto galloc = [&](long long n) {
    double* p = be_->alloc(std::max(n, 1LL));
    if (p) {
      be_->zero(p, std::max(n, 1LL));
      owned.push_back(p);
    }
    return p;
  };
  auto gfree = [&](double* p) {
    if (!p) return;
    for (auto& q : owned)
      if (q == p) q = nullptr;
    be_->release(p);
  };
  auto cleanup = [&]() {
    be_->sync();
    for (double* p : owned)
      if (p) be_->release(p);
  };
  auto values = [&](const TaskList& tl, const double* xv, const double* yb) {
    std::vector<double> v(tl.tasks.size(), 0.0);
    if (tl.tasks.empty()) return v;
    double* d = be_->alloc((long long)tl.tasks.size());
    be_->task_values(tl, xv, yb, d);
    be_->download(v.data(), d, (long long)v.size());
    be_->sync();
    be_->release(d);
    return v;
  };
  // coefficient derivative of one dot term (and of its expression's single
  // coefficient when the expression is not materialised): weight w = dE/d(alpha) * alpha
  auto dot_term = [&](const Side& S, const SideT<Lin>& SL, int e, int d, int t, double w) {
    const DotTerm& dt = S.eops[e].dots[d].t[t];
    const Lin& dl = SL.eops[e].dots[d].t[t].s;
    if (!dl.is_const()) acc_lin(g, dl, w / dt.s);
    const Expr& x = S.exprs[dt.expr];
    if (x.mat < 0 && !x.t.empty()) {
      const Lin& cl = SL.exprs[dt.expr].t[0].c;
      if (!cl.is_const()) acc_lin(g, cl, w / x.t[0].c);
    }
  };
  // partial sums: Gm (gradient of S's materialised arena) -> Gc (+= adjoint)
  // and the derivatives of their coefficients; Gd: direct catalogue gradient
  auto partial_sums = [&](const Side& S, const SideT<Lin>& SL, const Catalogue& C, const double* Gm, const double* Gd,
                          double* Gc) {
    const Basis& bs = C.basis;
    TaskList lc;  // forward partial sums as products (I * op(src) * I)
    std::vector<std::array<int, 2>> lprov;  // (expr, term) per product
    std::vector<double> lsign;
    AdjSink sink;
    sink.region(C.d, C.size, Gc);
    for (auto& b : blocks_of(C)) {  // carry the direct gradient
      Opd I1{nullptr, true, false, (int)b[1], (int)b[1]}, I2{nullptr, true, false, (int)b[2], (int)b[2]};
      sink.add(C.d + b[0], (int)b[1], (int)b[2], mk(1.0, I1, Opd{Gd + b[0], false, false, (int)b[1], (int)b[2]}, I2));
    }
    for (auto& mt : S.mats) {
      const Expr& x = S.exprs[mt.expr];
      const Layout& L = C.layouts[mt.layout];
      for (size_t b = 0; b < L.in.size(); ++b) {
        const int in = L.in[b], out = L.out[b];
        const int rows = bs.dim[out], cols = bs.dim[in];
        Group gr;
        gr.yoff = mt.off + L.off[b];
        gr.q = rows;
        gr.r = cols;
        gr.row0 = gr.col0 = 0;
        gr.nrows = rows;
        gr.ncols = cols;
        gr.t0 = (int)lc.tasks.size();
        for (size_t ti = 0; ti < x.t.size(); ++ti) {
          const Term& tm = x.t[ti];
          const double sign = tm.par == 1 ? sgn_n(bs.q[in].n) : tm.par == 2 ? sgn_n(bs.q[out].n) : 1.0;
          Opd I1{nullptr, true, false, rows, rows}, I2{nullptr, true, false, cols, cols};
          if (tm.op < 0) {
            if (in != out) continue;
            lc.tasks.push_back(mk(tm.c * sign, I1, Opd{nullptr, true, false, rows, cols}, I2));
          } else {
            const CatOp& o = C.ops[tm.op];
            const Layout& OL = C.layouts[o.layout];
            int ob = tm.tr ? OL.blk_of_in[out] : OL.blk_of_in[in];
            if (ob < 0) continue;
            if (tm.tr && OL.out[ob] != in) continue;
            if (!tm.tr && OL.out[ob] != out) continue;
            const double* src = C.d + o.off + OL.off[ob];
            Opd X{src, false, tm.tr, rows, cols};
            lc.tasks.push_back(mk(tm.c * sign, I1, X, I2));
            sink.adjoint(lc.tasks.back(), nullptr, Gm + gr.yoff);
          }
          lprov.push_back({mt.expr, (int)ti});
          lsign.push_back(sign);
        }
        gr.t1 = (int)lc.tasks.size();
        lc.groups.push_back(gr);
      }
    }
    const std::vector<double> v = values(lc, nullptr, Gm);
    for (size_t i = 0; i < v.size(); ++i) {
      const Lin& cl = SL.exprs[lprov[i][0]].t[lprov[i][1]].c;
      if (!cl.is_const()) acc_lin(g, cl, v[i] * lsign[i]);
    }
    sink.flush(be_);
  };
  // Lin twins of the step's sides
  SideT<Lin> SLl, SLr;
  build_left_eops<Lin>(Lcat_[k], k, SLl);
  compile_side<Lin>(SLl, Lcat_[k], true);
  build_right_eops<Lin>(Rcat_[k + 2], k + 1, SLr);
  compile_side<Lin>(SLr, Rcat_[k + 2], false);
  if (SLl.eops.size() != st.L.eops.size() || SLr.eops.size() != st.R.eops.size() ||
      SLl.exprs.size() != st.L.exprs.size() || SLr.exprs.size() != st.R.exprs.size()) {
    cleanup();
    err = "integral_gradient: tracked operator structure differs";
    return -6;
  }
  // ---- H_eff*psi: coefficients and operand adjoints ----
  {
    const TaskList& tl = st.heff_full;
    const std::vector<double> v = values(tl, psi, Yb);
    for (size_t i = 0; i < tl.tasks.size(); ++i) {
      const auto& pv = st.heff_prov[i];
      const double w = v[i] * tl.tasks[i].alpha;
      if (w == 0.0) continue;
      if (pv[0] >= 0) dot_term(st.L, SLl, pv[0], pv[1], pv[2], w);
      if (pv[3] >= 0) dot_term(st.R, SLr, pv[3], pv[4], pv[5], w);
    }
  }
  Catalogue& Lk = Lcat_[k];
  Catalogue& Rk = Rcat_[k + 2];
  double* GdL = galloc(Lk.size);
  double* GmL = galloc(st.L.size);
  double* GdR = galloc(Rk.size);
  double* GmR = galloc(st.R.size);
  if (!GdL || !GmL || !GdR || !GmR) {
    cleanup();
    err = "integral_gradient: allocation failed";
    return -3;
  }
  {
    AdjSink sink;
    sink.region(Lk.d, Lk.size, GdL);
    if (st.L.size) sink.region(st.L.d, st.L.size, GmL);
    sink.region(Rk.d, Rk.size, GdR);
    if (st.R.size) sink.region(st.R.d, st.R.size, GmR);
    for (const Group& gr : st.heff_full.groups)
      for (int i = gr.t0; i < gr.t1; ++i) sink.adjoint(st.heff_full.tasks[i], psi, Yb + gr.yoff);
    sink.flush(be_);
  }
  double* GL = galloc(Lk.size);
  double* GR = galloc(Rk.size);
  if (!GL || !GR) {
    cleanup();
    err = "integral_gradient: allocation failed";
    return -3;
  }
  partial_sums(st.L, SLl, Lk, GmL, GdL, GL);
  partial_sums(st.R, SLr, Rk, GmR, GdR, GR);
  gfree(GdL);
  gfree(GmL);
  gfree(GdR);
  gfree(GmR);
  // ---- renormalisation chain: block l+1 = U^T (block l (x) dot l) U ----
  auto level = [&](int site, bool left, double* Gnext, double*& Gout) -> int {
    // both blocks of this level must exist (staged ones come back, dropped
    // ones are rebuilt); the source's arena is read on the device
    {
      int rc0 = left ? ensure_left(site + 1, err) : ensure_right(site, err);
      if (!rc0) rc0 = left ? ensure_left(site, err) : ensure_right(site + 1, err);
      if (rc0) return rc0;
    }
    Catalogue& src = left ? Lcat_[site] : Rcat_[site + 1];
    Catalogue& dst = left ? Lcat_[site + 1] : Rcat_[site];
    struct Keep {
      std::vector<const Catalogue*>& k;
      std::vector<const Catalogue*> saved;
      Keep(std::vector<const Catalogue*>& kk, const Catalogue* a, const Catalogue* b) : k(kk), saved(kk) {
        k.push_back(a);
        k.push_back(b);
      }
      ~Keep() { k = saved; }
    } keep(keep_, &src, &dst);
    Side S;
    SideT<Lin> SL;
    if (left) {
      build_left_eops<double>(src, site, S);
      compile_side<double>(S, src, true);
      build_left_eops<Lin>(src, site, SL);
      compile_side<Lin>(SL, src, true);
    } else {
      build_right_eops<double>(src, site, S);
      compile_side<double>(S, src, false);
      build_right_eops<Lin>(src, site, SL);
      compile_side<Lin>(SL, src, false);
    }
    int rc = materialize(S, src, err);
    if (rc) return rc;
    TaskList rt;
    std::vector<std::array<int, 3>> prov;
    rotation_tasks(S, src, dst, site, left, rt, &prov);
    const std::vector<double> v = values(rt, nullptr, Gnext);
    for (size_t i = 0; i < rt.tasks.size(); ++i) {
      const double w = v[i] * rt.tasks[i].alpha;
      if (w != 0.0) dot_term(S, SL, prov[i][0], prov[i][1], prov[i][2], w);
    }
    double* Gd = galloc(src.size);
    double* Gm = galloc(S.size);
    Gout = galloc(src.size);
    if (!Gd || !Gm || !Gout) {
      free_side(S);
      err = "integral_gradient: allocation failed";
      return -3;
    }
    AdjSink sink;
    sink.region(src.d, src.size, Gd);
    if (S.size) sink.region(S.d, S.size, Gm);
    for (const Group& gr : rt.groups)
      for (int i = gr.t0; i < gr.t1; ++i) sink.adjoint(rt.tasks[i], nullptr, Gnext + gr.yoff);
    sink.flush(be_);
    partial_sums(S, SL, src, Gm, Gd, Gout);
    be_->sync();
    gfree(Gd);
    gfree(Gm);
    free_side(S);
    std::string e = be_->error();
    if (!e.empty()) {
      err = e;
      return -6;
    }
    return 0;
  };
  double* cur = GL;
  for (int site = k - 1; site >= 0; --site) {
    double* nxt = nullptr;
    int rc = level(site, true, cur, nxt);
    if (rc) {
      cleanup();
      return rc;
    }
    gfree(cur);
    cur = nxt;
  }
  gfree(cur);
  cur = GR;
  for (int site = k + 2; site <= N_ - 1; ++site) {
    double* nxt = nullptr;
    int rc = level(site, false, cur, nxt);
    if (rc) {
      cleanup();
      return rc;
    }
    gfree(cur);
    cur = nxt;
  }
  gfree(cur);
  cleanup();
  std::string e = be_->error();
  if (!e.empty()) {
    err = e;
    return -6;
  }
  return 0;
}

}  // namespace tns

namespace tns {
template void Engine::build_left_eops<double>(const Catalogue&, int, SideT<double>&);
template void Engine::build_left_eops<Lin>(const Catalogue&, int, SideT<Lin>&);
template void Engine::build_right_eops<double>(const Catalogue&, int, SideT<double>&);
template void Engine::build_right_eops<Lin>(const Catalogue&, int, SideT<Lin>&);
template void Engine::compile_side<double>(SideT<double>&, const Catalogue&, bool);
template void Engine::compile_side<Lin>(SideT<Lin>&, const Catalogue&, bool);
}  // namespace tns
