// engine.h -- symbolic layer of the two-site DMRG H_eff*psi engine.
//
// Block-sparse layout (Sec. III.A.1): an operator on a block basis is stored
// as the dense blocks (out-sector <- in-sector) allowed by its quantum-number
// shift dq, each block row-major, blocks of one operator contiguous.
//
// Operator catalogues (Sec. III.A.2, partial summation N^4 -> N^2):
//   left block  L (orbitals 0..len-1):  H, c+_a, A_ab = c+_a c+_b (a<b),
//       B_ab = c+_a c_b, T_x = sum_{pqr in L} W_pqrx c+_p c+_q c_r  (x >= 2*len)
//   right block R (orbitals len..N-1):  H, c+_x, S_a, P_ab (a<b), Q_ab  (a,b < 2*len)
//       S_a  = sum_{qru in R} W_aqru c+_q c_r c_u + sum_{x in R} t_ax c_x
//       P_ab = sum_{ru in R} W_abru c_r c_u
//       Q_ab = sum_{qr in R} (W_aqrb - W_aqbr) c+_q c_r
// with spin-orbital integrals t_pq = h_{i_p i_q} d(s_p,s_q) and
// W_pqrs = (i_p i_s | i_q i_r) d(s_p,s_s) d(s_q,s_r) of Eq. (1).
//
// Enlarged operators (blocking of a block with one dot) are sums of
// (D-basis expression) (x) (4x4 dot operator); the dot's one-dimensional
// sectors turn every dot factor into scalars (Sec. III.A.2), so an enlarged
// operator is a set of "dot blocks" (s' <- s), each a short list of
// scalar x expression.  Expressions are a catalogue operator (optionally
// transposed, optionally times the block parity), the identity, or a
// materialised linear combination (partial sum).
//
// Every product the engine executes has the form of Eq. (2):
//     Y_blk += alpha * op(L) * op(X) * op(R)^T
// (op = identity, plain or transposed), grouped by output block.
#pragma once

#include <array>
#include <functional>
#include <cstdint>
#include <map>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace tns {

struct QN {
  int n = 0, s = 0;
};
inline bool operator<(QN a, QN b) { return a.n < b.n || (a.n == b.n && a.s < b.s); }
inline bool operator==(QN a, QN b) { return a.n == b.n && a.s == b.s; }
inline bool operator!=(QN a, QN b) { return !(a == b); }
inline QN operator+(QN a, QN b) { return {a.n + b.n, a.s + b.s}; }
inline QN operator-(QN a, QN b) { return {a.n - b.n, a.s - b.s}; }
inline QN operator-(QN a) { return {-a.n, -a.s}; }

extern const QN kSiteQN[4];

struct Basis {
  std::vector<QN> q;
  std::vector<int> dim;
  std::vector<long long> off;
  long long total = 0;
  std::map<QN, int> idx;
  void clear() { q.clear(); dim.clear(); off.clear(); total = 0; idx.clear(); }
  void add(QN x, int d) {
    idx[x] = (int)q.size();
    q.push_back(x);
    dim.push_back(d);
    off.push_back(total);
    total += d;
  }
  int find(QN x) const {
    auto it = idx.find(x);
    return it == idx.end() ? -1 : it->second;
  }
  int size() const { return (int)q.size(); }
};

// blocks of an operator with shift dq on a basis: block b maps in[b] -> out[b]
struct Layout {
  QN dq;
  std::vector<int> in, out;
  std::vector<long long> off;
  std::vector<int> blk_of_in;  // in-sector index -> block index, -1 if none
  long long size = 0;
};
void make_layout(const Basis& b, QN dq, Layout& L);

enum OpKind { K_H = 0, K_C, K_A, K_B, K_T, K_S, K_P, K_Q };

struct CatOp {
  int kind, i, j;
  QN dq;
  int layout;
  long long off;  // element offset in the catalogue arena
};

struct Catalogue {
  bool left = true;
  int len = 0;   // left: orbitals 0..len-1, right: orbitals len..N-1
  Basis basis;   // own content of the block (particles inside it)
  std::vector<Layout> layouts;
  std::map<QN, int> layout_of;
  std::vector<CatOp> ops;
  std::unordered_map<long long, int> index;
  double* d = nullptr;  // arena (device for the CUDA backend)
  long long size = 0;
  bool valid = false;
  // an empty block (no orbitals): every operator is zero by definition, so
  // expressions drop its operators instead of reading them
  bool zero = false;
  // pinned host copy while the catalogue is staged off the device (d == nullptr)
  double* h = nullptr;
  // element offsets of the operator blocks that are identically zero (found
  // when the catalogue is built; used by the useful-flop count)
  std::unordered_set<long long> zero_off;
  static long long key(int kind, int i, int j) {
    return ((long long)kind << 40) | ((long long)(i + 1) << 20) | (long long)(j + 1);
  }
  int layout_for(QN dq);
  int find(int kind, int i = -1, int j = -1) const {
    auto it = index.find(key(kind, i, j));
    return it == index.end() ? -1 : it->second;
  }
  int add_op(int kind, int i, int j, QN dq);  // appends, assigns offsets later
  void assign_offsets();
};

// Scalar that carries, besides its value, its (sparse) derivative with
// respect to the integrals theta = (h_ij, v_ijkl) as independent entries:
// index i*N+j for h_ij and N^2 + ((i*N+j)*N+k)*N+l for v_ijkl.  Every
// coefficient of the operator construction is linear in theta, so running
// the same construction with this type records where each coefficient comes
// from (used by the integral gradients of the differentiation form).
struct Lin {
  double v = 0.0;
  std::vector<std::pair<long long, double>> c;
  Lin() = default;
  Lin(double x) : v(x) {}
  static Lin var(double x, long long idx) {
    Lin r(x);
    r.c.push_back({idx, 1.0});
    return r;
  }
  bool is_const() const { return c.empty(); }
  void compact();
};
Lin operator+(const Lin& a, const Lin& b);
Lin operator-(const Lin& a);
Lin operator-(const Lin& a, const Lin& b);
Lin operator*(double s, const Lin& a);
inline Lin operator*(const Lin& a, double s) { return s * a; }
Lin operator*(const Lin& a, const Lin& b);  // one factor must be constant
inline Lin& operator+=(Lin& a, const Lin& b) { return a = a + b; }
inline bool operator==(const Lin& a, double x) { return a.v == x; }
inline bool operator!=(const Lin& a, double x) { return a.v != x; }
inline double value(double x) { return x; }
inline double value(const Lin& x) { return x.v; }

template <class S>
struct M4T {
  S a[4][4];
  M4T() {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) a[i][j] = S(0.0);
  }
  template <class S2>
  explicit M4T(const M4T<S2>& o) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) a[i][j] = S(o.a[i][j]);
  }
  static M4T eye() {
    M4T m;
    for (int i = 0; i < 4; ++i) m.a[i][i] = S(1.0);
    return m;
  }
  // product with a plain (or same-type) 4x4 on the right
  template <class S2>
  M4T operator*(const M4T<S2>& b) const {
    M4T r;
    for (int i = 0; i < 4; ++i)
      for (int k = 0; k < 4; ++k)
        if (a[i][k] != 0.0)
          for (int j = 0; j < 4; ++j)
            if (b.a[k][j] != 0.0) r.a[i][j] += a[i][k] * b.a[k][j];
    return r;
  }
  M4T operator+(const M4T& b) const {
    M4T r;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) r.a[i][j] = a[i][j] + b.a[i][j];
    return r;
  }
  // c * this, c a plain or a tracked scalar
  template <class C>
  auto scale(const C& c) const -> M4T<decltype(c * a[0][0])> {
    M4T<decltype(c * a[0][0])> r;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (a[i][j] != 0.0) r.a[i][j] = c * a[i][j];
    return r;
  }
  M4T T() const {
    M4T r;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) r.a[i][j] = a[j][i];
    return r;
  }
  bool zero() const {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (a[i][j] != 0.0) return false;
    return true;
  }
};
using M4 = M4T<double>;

// one term of an expression: c * op^(T) * P^(par)
//   op = -1: identity; par: 0 none, 1 parity of the in-sector, 2 of the out-sector
template <class S>
struct TermT {
  S c;
  int op;
  bool tr;
  int par;
};
using Term = TermT<double>;

template <class S>
struct ExprT {
  std::vector<TermT<S>> t;
  QN dq;          // shift of the expression (in -> in + dq)
  int mat = -1;   // materialised: index into Step::mats
};
using Expr = ExprT<double>;

// enlarged operator = sum_parts (expr (x) y) ; dot blocks compiled from it
template <class S>
struct DotTermT {
  S s;
  int expr;
};
using DotTerm = DotTermT<double>;
template <class S>
struct DotBlockT {
  int so, si;
  std::vector<DotTermT<S>> t;
};
using DotBlock = DotBlockT<double>;
template <class S>
struct EOpT {
  int kind, i, j;   // catalogue key of the enlarged block this operator belongs to
  QN dq;            // total shift (expr dq + dot shift)
  std::vector<std::pair<M4T<S>, int>> parts;  // (dot operator, expr id)
  std::vector<DotBlockT<S>> dots;
};
using EOp = EOpT<double>;

// a materialised expression: its own operator on the block basis
struct Mat {
  int layout;      // index into the owning side's catalogue layouts
  long long off;   // element offset in the step scratch arena
  int expr;
};

// ---------------------------------------------------------------------------
// work lists
// ---------------------------------------------------------------------------
enum TaskFlags {
  TF_LI = 1,      // L is the identity
  TF_LT = 2,      // L stored transposed (m x q)
  TF_XI = 4,      // X is the identity (m == n)
  TF_XT = 8,      // X stored transposed (n x m)
  TF_XV = 16,     // X pointer is an element offset into the launch's X vector
  TF_RI = 32,     // R is the identity
  TF_RT = 64,     // R stored transposed (n x r)
  TF_LM = 128,    // while a step is planned: L is an element offset into the left partial-sum arena
  TF_RM = 256,    // the same for R and the right partial-sum arena
};

struct Task {
  double alpha;
  const double* L;
  const double* X;  // pointer, or element offset cast to pointer when TF_XV
  const double* R;
  int q, m, n, r;
  int flags;
  int pad;
};

struct Group {  // one output block (or tile of it) and its task range
  long long yoff;  // element offset (H_eff: into Y vector; env: into the arena given at launch)
  int q, r;        // full block dims (row-major q x r)
  int row0, col0, nrows, ncols;
  int t0, t1;
};

struct TaskList {
  std::vector<Task> tasks;
  std::vector<Group> groups;
  double flops = 0.0;
  long long nprod = 0;
  long long gen = 0;        // bumped on every rebuild (device copies keyed on it)
  bool persistent = false;  // kept on the device between runs
  void clear() { tasks.clear(); groups.clear(); flops = 0; nprod = 0; ++gen; }
};

struct LCTerm {
  double c;
  const double* src;  // nullptr: identity
  int tr;             // source block stored transposed (cols x rows)
};
struct LCBlock {
  double* dst;
  int rows, cols;
  int t0, t1;
};
struct LCList {
  std::vector<LCBlock> blocks;
  std::vector<LCTerm> terms;
};

// ---------------------------------------------------------------------------
// backend: device memory and the kernels (CUDA in the product library)
// ---------------------------------------------------------------------------
struct Backend {
  virtual ~Backend() {}
  virtual double* alloc(long long n) = 0;  // nullptr on failure
  virtual void release(double* p) = 0;
  virtual void upload(double* dst, const double* src, long long n) = 0;
  virtual void download(double* dst, const double* src, long long n) = 0;
  virtual void zero(double* p, long long n) = 0;
  virtual void lincomb(const LCList& l) = 0;
  // run a task list: each group's output (tile) is overwritten with the sum of
  // its tasks.  xv/yv: bases for TF_XV offsets and group yoff.
  virtual void run(const TaskList& tl, const double* xv, double* yv, int nvec,
                   long long xstride, long long ystride, int precision) = 0;
  // out[t] = < Ybar_g, op(L_t) op(X_t) op(R_t)^T > for every task t of group g
  // (alpha not included); out is backend memory of tl.tasks.size() doubles
  virtual void task_values(const TaskList& tl, const double* xv, const double* ybar, double* out) = 0;
  // nz[i] = 1 if any element of block i (p[i], n[i] doubles in backend
  // memory) is nonzero, else 0
  virtual void nonzero_blocks(const std::vector<const double*>& p, const std::vector<long long>& n,
                              std::vector<char>& nz) = 0;
  // memory of the backend's device: bytes in use by the library, the most it
  // may hold (the budget, else the device's size; 0 = no limit known) and the
  // bytes the device reports free
  virtual long long mem_used() = 0;
  virtual long long mem_limit() = 0;
  virtual long long mem_free() = 0;
  virtual void set_budget(long long bytes) = 0;  // 0: no budget
  // pinned host memory for catalogues staged off the device (nullptr on failure)
  virtual double* host_alloc(long long n) = 0;
  virtual void host_release(double* p) = 0;
  // release the device copy of a work list (if any)
  virtual void forget(const TaskList& tl) = 0;
  // device bytes the backend will allocate to run a step's H_eff work list on
  // vectors of psi_length (work-list copy, operand images, solver vectors)
  virtual long long step_bytes(const TaskList& tl, long long psi_length) = 0;
  // called by the backend before a large allocation of its own: the engine
  // moves catalogues it does not need off the device to make room
  std::function<int(long long)> room;
  virtual void sync() = 0;
  virtual std::string error() = 0;  // "" if fine
};

// ---------------------------------------------------------------------------
// MPS
// ---------------------------------------------------------------------------
struct SiteBlock {
  int ql, s, qr;  // bond-b sector index, site state, bond-(b+1) sector index
  int m, n;
  long long off;  // element offset in the site array
};
struct Site {
  std::vector<SiteBlock> blocks;
  std::vector<int> index;  // ql*4+s -> block or -1
  double* d = nullptr;
  long long size = 0;
};

// ---------------------------------------------------------------------------
// per two-site step state
// ---------------------------------------------------------------------------
template <class S>
struct SideT {  // enlarged operators of one side for a step
  std::vector<ExprT<S>> exprs;
  std::vector<EOpT<S>> eops;
  std::map<long long, int> eop_index;  // catalogue key -> eop
  std::vector<Mat> mats;
  double* d = nullptr;  // materialised arena
  long long size = 0;
};
using Side = SideT<double>;

struct PsiBlock {
  int ql, s1, s2, qr;  // ql: bond-k sector index; qr: index in the right block basis
  int m, n;
  long long off;
};

struct Step {
  int k = -1;
  Side L, R;
  std::vector<PsiBlock> psi;
  std::vector<int> psi_index;  // ((ql*4+s1)*4+s2)*nqr+qr -> block
  std::vector<long long> desc;
  long long length = 0;
  TaskList heff;       // products whose operator blocks are not identically zero (the forward product)
  TaskList heff_full;  // every product (adjoint and integral gradients; heff_prov is aligned with it)
  // per H_eff task, where its coefficient comes from: (eop, dot block, dot
  // term) on the left side and on the right side; -1 for an identity side
  std::vector<std::array<int, 6>> heff_prov;
  std::vector<int> heff_row;  // per forward H_eff task: its operator-table row (operator pair)
  int nrows = 0;              // operator-table rows of the step
  TaskList heff_part;         // the tasks of one part of an operator-row split
  long long part_key = -1;    // (part, nparts) heff_part was built for
  // operand blocks of the step that are identically zero, per side (catalogue
  // blocks by address, partial-sum blocks by their arena offset while the
  // step is planned); products reading one are not counted as useful flops
  std::unordered_set<const double*> zero_L, zero_R;
  long long plan_bytes = 0;  // device bytes the memory plan reserved for the step
  std::vector<int> diag_tasks;  // tasks contributing to the diagonal, in group order
  std::vector<int> diag_rng;    // per group: range [diag_rng[g], diag_rng[g+1]) of diag_tasks
  bool valid = false;
};

// two-site wavefunction layout: blocks (ql, s1, s2, qr) ordered by (ql, s1, s2, qr)
void psi_layout_of(const Basis& L, const Basis& R, QN target, std::vector<PsiBlock>& psi, std::vector<int>& index,
                   std::vector<long long>& desc, long long& length);

// memory management of the operator catalogues (out-of-HBM environments)
struct MemStats {
  long long device_used = 0, device_peak = 0, device_limit = 0;
  long long host_used = 0, host_peak = 0, host_budget = 0;
  long long staged = 0, restored = 0, dropped = 0, built = 0;  // catalogue moves and renormalisations
  long long last_plan = 0;  // bytes of the last step's memory plan
};

class Engine {
 public:
  explicit Engine(Backend* be) : be_(be) {
    be_->room = [this](long long bytes) {
      std::string e;
      return make_room(bytes, e);
    };
  }
  ~Engine();

  int load_integrals(int N, const double* h, const double* v, double e_core, std::string& err);
  int mps_define(int N, int n_elec, int two_sz, int D, std::string& err);
  int mps_set_bond(int b, int nsec, const int* sec, const int* dims, std::string& err);
  int mps_set_site(int b, const double* x, long long len, std::string& err);
  int mps_get_site(int b, double* x, long long len, long long* len_out, std::string& err);
  int mps_init(int N, int n_elec, int two_sz, int D, unsigned long long seed, std::string& err);
  // checkpoint / restart of a sweep: integrals, MPS and position in one file
  int checkpoint_save(const char* path, int site, int ltr, std::string& err);
  int checkpoint_load(const char* path, int* site, int* ltr, std::string& err);

  int build_env(int k, std::string& err);        // L_k, R_{k+2}, step k tables
  int heff(const double* X, double* Y, int nvec, int precision, std::string& err);
  // the part `part` of an nparts-way operator-row split of Y = H_eff X: Y is
  // overwritten with the sum over the operator pairs assigned to that part
  // (balanced by flops, the same split on every caller); the parts add up to H_eff X
  int heff_part(const double* X, double* Y, int nvec, int precision, int part, int nparts, std::string& err);
  void row_parts(int nparts, std::vector<int>& part_of_row) const;
  // adjoint of Y = H_eff X for the cotangent Yb: Xb = H_eff^T Yb and the
  // gradients of <Yb, H_eff X> w.r.t. the arenas of L_k (Lb) and R_{k+2} (Rb);
  // any output may be null.  All pointers in the backend's memory space.
  int heff_adjoint(const double* X, const double* Yb, double* Xb, double* Lb, double* Rb, std::string& err);
  // gradient of E = <psi|H_eff|psi>/<psi|psi> at the current step with respect
  // to every stored integral (h_ij at i*N+j, (ij|kl) at N^2+((i*N+j)*N+k)*N+l),
  // the MPS isometries fixed: reverse mode through H_eff*psi and through the
  // renormalisation chain of both blocks.  psi: backend memory, step layout.
  int integral_gradient(const double* psi, std::vector<double>& g, std::string& err);
  // refresh the step's partial sums after the catalogue arenas were changed
  int refresh_step(std::string& err);
  // algorithmic work of the environment build so far: FP64 flops of the
  // renormalisation products and bytes of the partial sums (terms read,
  // result written) and renormalisations (source catalogue and partial sums
  // read, site tensor read, new catalogue written)
  double env_flops() const { return env_flops_; }
  double env_bytes() const { return env_bytes_; }
  // device budget (bytes; 0 = none) and pinned host memory for staged
  // catalogues (bytes; 0 = none: catalogues that must leave the device are
  // dropped and rebuilt when needed)
  void set_memory_budget(long long device_bytes, long long host_bytes);
  MemStats mem_stats();
  double e_core() const { return e_core_; }

  // accessors for the API layer
  Step& step() { return step_; }
  int N() const { return N_; }
  QN target() const { return target_; }
  int D() const { return D_; }
  std::vector<Basis>& bonds() { return bonds_; }
  std::vector<Site>& sites() { return sites_; }
  Backend* be() { return be_; }
  Catalogue& left(int k) { return Lcat_[k]; }
  Catalogue& right(int k) { return Rcat_[k]; }

  // pieces used by the sweep driver
  int ensure_step(int k, std::string& err);  // L_k and R_{k+2} on the device
  int ensure_left(int k, std::string& err);
  int ensure_right(int k, std::string& err);
  int prepare_step(int k, std::string& err);
  int grow_left(int k, std::string& err);   // L_{k+1} from L_k, site k (needs step k)
  int grow_right(int k, std::string& err);  // R_{k+1} from R_{k+2}, site k+1 (needs step k)
  void invalidate_left_from(int k);
  void invalidate_right_from(int k);  // R_j for j <= k
  int site_from_host(int b, const std::vector<SiteBlock>& blocks, const std::vector<double>& data,
                     std::string& err);
  int alloc_site(int b, std::string& err);  // layout from bonds b, b+1; zeroed device storage
  Basis right_basis_of_bond(int b) const;    // right-counted basis of bond b (bond order)
  void set_bond_basis(int b, const Basis& basis);

  // integrals
  double t(int p, int q) const;
  double W(int p, int q, int r, int s) const;
  // the same integrals as plain (double) or tracked (Lin) scalars
  template <class Sc>
  Sc tc(int p, int q) const;
  template <class Sc>
  Sc Wc(int p, int q, int r, int s) const;

 private:
  Backend* be_;
  int N_ = 0;
  std::vector<double> h_, v_;
  double e_core_ = 0.0;
  bool have_ints_ = false;
  QN target_;
  int D_ = 0;
  bool have_mps_ = false;
  std::vector<Basis> bonds_;  // left counted, 0..N
  std::vector<Site> sites_;
  std::vector<Catalogue> Lcat_;  // Lcat_[k]: orbitals 0..k-1
  std::vector<Catalogue> Rcat_;  // Rcat_[k]: orbitals k..N-1
  Step step_;
  // catalogue staging: the position of the current work (eviction order is
  // the distance from it: the catalogue needed last leaves first), the
  // catalogues in use (never moved), pinned host memory in use and budget
  int pos_ = 0;
  std::vector<const Catalogue*> keep_;
  long long host_budget_ = 0;
  MemStats ms_;
  double env_flops_ = 0.0, env_bytes_ = 0.0;
  bool verbose_env_ = false;  // TNS_VERBOSE_ENV=1: one line per renormalisation on stderr

  int make_room(long long bytes, std::string& err);
  int evict(Catalogue& c, std::string& err);
  int restore(Catalogue& c, std::string& err);
  bool movable(const Catalogue& c) const;
  void scan_zero(Catalogue& c);
  void layout_mats(Side& S, Catalogue& cat);
  int fill_mats(Side& S, Catalogue& cat, std::string& err);

  void free_cat(Catalogue& c);
  void free_side(Side& s);
  int alloc_cat(Catalogue& c, std::string& err);
  void empty_left(Catalogue& c);
  void empty_right(Catalogue& c);
  template <class Sc>
  void build_left_eops(const Catalogue& L, int site, SideT<Sc>& S);
  template <class Sc>
  void build_right_eops(const Catalogue& R, int site, SideT<Sc>& S);
  template <class Sc>
  void compile_side(SideT<Sc>& S, const Catalogue& cat, bool left);
  int materialize(Side& S, Catalogue& cat, std::string& err);
  int rotate(Side& S, const Catalogue& src, Catalogue& dst, int site, bool left, std::string& err);
  // the renormalisation task list of rotate() into an existing dst layout;
  // prov (optional) receives (eop, dot block, dot term) per task
  void rotation_tasks(const Side& S, const Catalogue& src, const Catalogue& dst, int site, bool left, TaskList& tl,
                      std::vector<std::array<int, 3>>* prov);

  void build_psi(int k);
  void find_zero_blocks();
  void build_heff_tasks();
};

}  // namespace tns
