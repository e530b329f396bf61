// plancheck.cu -- host-side checks of the tensor-core product planning
// (test-only; compiled on the CPU with nvcc and linked against the library;
// no CUDA call is made).
//
// The planning code of tc.cu is included as it is and driven with seeded
// synthetic work lists of output blocks and products of 1 to 100 states:
//   * routing: an output block whose dimensions and those of every X block it
//     reads are <= 16 (<= 32) goes to the 16-state (32-state) warp kernel when
//     the routing limit allows it, every other block to the tile kernel, whose
//     128 x 64 tiles cover it;
//   * chunks: every product of a block in exactly one chunk of each of its
//     tiles, a chunk's products sharing one X block and fitting the stacked
//     GEMM1 (tile kernel) or at most 8 long (warp kernels);
//   * splits for every schedule variant (rounds 1, 2, 4): the pieces of a tile
//     cover its chunks once, in order; unsplit tiles write the output block;
//     split pieces own disjoint partial tiles inside the arena; every split
//     reduction sums exactly its tile's pieces, stored one after the other;
//   * the launch checks accept the plans and reject a corrupted product record.
// Prints one line per configuration and "ALL OK" at the end; exit status 1 on
// the first failure.
#include "../../paper_2305_05581_gb300/csrc/tc.cu"

#include <cmath>
#include <cstdint>
#include <random>
#include <set>

using namespace tns;

namespace {

int g_fail = 0;
#define CHECK(cond, ...)                                \
  do {                                                  \
    if (!(cond)) {                                      \
      std::printf("FAIL %s:%d: ", __FILE__, __LINE__);  \
      std::printf(__VA_ARGS__);                         \
      std::printf("\n");                                \
      g_fail = 1;                                       \
      return false;                                     \
    }                                                   \
  } while (0)

struct XDef {
  long long off;
  int m, n;
};

TaskList make_list(unsigned seed, int ngroups, std::vector<XDef>& xdefs) {
  std::mt19937 rng(seed);
  const int dims[] = {1, 2, 3, 5, 7, 8, 9, 12, 15, 16, 17, 20, 24, 31, 32, 33, 40, 64, 100};
  const int nd = sizeof(dims) / sizeof(dims[0]);
  auto pick = [&](int hi) { return dims[rng() % hi]; };
  // X blocks: mostly small, some large
  xdefs.clear();
  long long xoff = 0;
  for (int i = 0; i < 40; ++i) {
    const int lim = (i % 5 == 0) ? nd : 15;  // dims[14] = 32
    XDef x{xoff, pick(lim), pick(lim)};
    xoff += (long long)x.m * x.n;
    xdefs.push_back(x);
  }
  TaskList tl;
  tl.persistent = true;
  long long yoff = 0;
  long long ptr = 0x100000;
  for (int g = 0; g < ngroups; ++g) {
    Group G{};
    const int lim = (g % 4 == 0) ? nd : (g % 4 == 1 ? 10 : 15);  // dims[9] = 16
    G.q = pick(lim);
    G.r = pick(lim);
    G.yoff = yoff;
    G.row0 = G.col0 = 0;
    G.nrows = G.q;
    G.ncols = G.r;
    yoff += (long long)G.q * G.r;
    G.t0 = (int)tl.tasks.size();
    // the X blocks this block reads: small ones for most blocks
    const int nt = 1 + (int)(rng() % 200);
    for (int t = 0; t < nt; ++t) {
      int xi = (int)(rng() % xdefs.size());
      if (g % 4 == 1) {  // blocks meant for the 16-state kernel read X blocks <= 16 only
        for (int tries = 0; tries < 100 && (xdefs[xi].m > 16 || xdefs[xi].n > 16); ++tries)
          xi = (int)(rng() % xdefs.size());
        if (xdefs[xi].m > 16 || xdefs[xi].n > 16) continue;
      }
      const XDef& X = xdefs[xi];
      Task k{};
      k.alpha = std::ldexp((double)(rng() % 2001) - 1000.0, -10);
      k.q = G.q;
      k.m = X.m;
      k.n = X.n;
      k.r = G.r;
      k.flags = TF_XV;
      k.X = (const double*)(size_t)X.off;
      if (k.q == k.m && rng() % 5 == 0)
        k.flags |= TF_LI;
      else
        k.L = (const double*)(uintptr_t)(ptr += 64 * (1 + rng() % 3));
      if (k.r == k.n && rng() % 5 == 0)
        k.flags |= TF_RI;
      else
        k.R = (const double*)(uintptr_t)(ptr += 64);
      if (rng() % 3 == 0) k.flags |= TF_LT;
      if (rng() % 3 == 0) k.flags |= TF_RT;
      tl.tasks.push_back(k);
    }
    G.t1 = (int)tl.tasks.size();
    tl.groups.push_back(G);
  }
  return tl;
}

// a copy of a list's products in chunk order must be the group's products
bool check_chunks(const TcPlan& P, const TcTile& T, const Group& G, int cap, int base) {
  std::vector<int> seen;
  for (int c = T.c0; c < T.c1; ++c) {
    const TcChunk& C = P.chunks_h[c];
    CHECK(C.t1 > C.t0 && C.t1 - C.t0 <= cap, "chunk size %d (cap %d)", C.t1 - C.t0, cap);
    for (int t = C.t0; t < C.t1; ++t) {
      CHECK(P.tasks_h[t].xb == C.xb, "chunk X block");
      seen.push_back(t);
    }
  }
  CHECK((int)seen.size() == G.t1 - G.t0, "tile of group covers %zu of %d products", seen.size(), G.t1 - G.t0);
  for (size_t i = 0; i < seen.size(); ++i) CHECK(seen[i] == base + (int)i, "products out of order");
  return true;
}

bool check_split(const std::vector<TcTile>& orig, const std::vector<TcTile>& pieces,
                 const std::vector<SplitRed>& reds, long long psize) {
  // pieces of each original tile, in chunk order
  std::map<std::tuple<int, int, int>, std::vector<TcTile>> by;
  for (const TcTile& p : pieces) by[std::make_tuple(p.g, p.row0, p.col0)].push_back(p);
  CHECK(by.size() == orig.size(), "pieces of %zu tiles for %zu tiles", by.size(), orig.size());
  std::set<std::tuple<int, int, int>> split;
  for (const SplitRed& R : reds) {
    const auto key = std::make_tuple(R.g, R.row0, R.col0);
    CHECK(split.insert(key).second, "two reductions of one tile");
    auto it = by.find(key);
    CHECK(it != by.end(), "reduction of an unknown tile");
    std::vector<TcTile> ps = it->second;
    CHECK((int)ps.size() == R.nsplit, "reduction sums %d pieces of %zu", R.nsplit, ps.size());
    std::sort(ps.begin(), ps.end(), [](const TcTile& a, const TcTile& b) { return a.poff < b.poff; });
    for (int i = 0; i < R.nsplit; ++i)
      CHECK(ps[i].poff == R.poff + (long long)i * R.nrows * R.ncols, "partial tile %d not in place", i);
  }
  std::vector<std::pair<long long, long long>> spans;
  for (auto& kv : by) {
    std::vector<TcTile> ps = kv.second;
    std::sort(ps.begin(), ps.end(), [](const TcTile& a, const TcTile& b) { return a.c0 < b.c0; });
    const TcTile* o = nullptr;
    for (const TcTile& t : orig)
      if (std::make_tuple(t.g, t.row0, t.col0) == kv.first) o = &t;
    CHECK(o, "piece of an unknown tile");
    CHECK(ps.front().c0 == o->c0 && ps.back().c1 == o->c1, "pieces do not span the tile's chunks");
    for (size_t i = 1; i < ps.size(); ++i) CHECK(ps[i].c0 == ps[i - 1].c1, "gap or overlap between pieces");
    if (!split.count(kv.first)) {
      CHECK(ps.size() == 1 && ps[0].poff == -1, "unsplit tile writes a partial tile");
    } else {
      for (const TcTile& p : ps) {
        CHECK(p.poff >= 0 && p.poff + (long long)p.nrows * p.ncols <= psize, "partial tile outside the arena");
        spans.push_back({p.poff, p.poff + (long long)p.nrows * p.ncols});
      }
    }
  }
  std::sort(spans.begin(), spans.end());
  for (size_t i = 1; i < spans.size(); ++i) CHECK(spans[i].first >= spans[i - 1].second, "partial tiles overlap");
  return true;
}

bool run(unsigned seed, int small, int es) {
  std::vector<XDef> xdefs;
  TaskList tl = make_list(seed, 80, xdefs);
  TcPlan P;
  std::vector<ImgJob> jobs;
  std::vector<XBlock> xbs;
  build_plan(tl, es, small, P, jobs, xbs);
  CHECK(P.tasks_h.size() == tl.tasks.size(), "products lost");
  // routing and chunks per group
  std::map<int, std::vector<const TcTile*>> tiles_of;
  for (const TcTile& T : P.tiles_h) tiles_of[T.g].push_back(&T);
  std::map<int, int> wkind;
  for (int w = 0; w < 2; ++w)
    for (const TcTile& T : P.wtiles_h[w]) {
      CHECK(!wkind.count(T.g), "block routed twice");
      wkind[T.g] = w;
    }
  int n16 = 0, n32 = 0, ntile = 0;
  for (int g = 0; g < (int)tl.groups.size(); ++g) {
    const Group& G = tl.groups[g];
    int dmax = std::max(G.q, G.r);
    for (int t = G.t0; t < G.t1; ++t) dmax = std::max(dmax, std::max(tl.tasks[t].m, tl.tasks[t].n));
    const int want = (small > 0 && dmax <= small && dmax <= SW_MAXD) ? (dmax <= 16 ? 0 : 1) : 2;
    const int base = tl.groups[g].t0;  // build_plan keeps a group's products together, X-ordered
    if (want < 2) {
      CHECK(wkind.count(g) && wkind[g] == want && !tiles_of.count(g), "block %d (max dim %d) routed wrongly", g,
            dmax);
      const TcTile* T = nullptr;
      for (const TcTile& t : P.wtiles_h[want])
        if (t.g == g) T = &t;
      CHECK(T->row0 == 0 && T->col0 == 0 && T->nrows == G.q && T->ncols == G.r, "small tile shape");
      if (!check_chunks(P, *T, G, 8, base)) return false;
      (want == 0 ? n16 : n32)++;
    } else {
      CHECK(!wkind.count(g), "block %d (max dim %d) on a small kernel", g, dmax);
      const auto& ts = tiles_of[g];
      CHECK((int)ts.size() == ((G.q + TC_M - 1) / TC_M) * ((G.r + TC_NC - 1) / TC_NC), "tiles of block %d", g);
      for (const TcTile* T : ts) {
        CHECK(T->row0 % TC_M == 0 && T->col0 % TC_NC == 0 && T->nrows == std::min(TC_M, G.q - T->row0) &&
                  T->ncols == std::min(TC_NC, G.r - T->col0),
              "tile shape");
        const int rp = (T->ncols + 15) & ~15;
        if (!check_chunks(P, *T, G, std::max(1, TC_M / rp), base)) return false;
      }
      ++ntile;
    }
  }
  // X-ordered products inside a group
  for (const Group& G : tl.groups)
    for (int t = G.t0 + 1; t < G.t1; ++t)
      CHECK(xbs[P.tasks_h[t - 1].xb].src <= xbs[P.tasks_h[t].xb].src, "products not ordered by X block");
  // splits of every variant, and the launch checks
  // chunk costs computed once per plan, as the launch path does, equal the
  // direct estimates of each chunk's kernel
  plan_chunk_costs(P, es);
  const std::vector<TcTask>& tk = P.tasks_h;
  for (const TcTile& T : P.tiles_h)
    for (int c = T.c0; c < T.c1; ++c) CHECK(P.ccost_h[c] == chunk_cost(tk, P.chunks_h[c], T), "chunk cost");
  for (int w = 0; w < 2; ++w)
    for (const TcTile& T : P.wtiles_h[w])
      for (int c = T.c0; c < T.c1; ++c) CHECK(P.ccost_h[c] == sw_chunk_cost(tk, P.chunks_h[c], T, es), "chunk cost");
  auto cost = [&](const TcChunk& C, const TcTile&) { return P.ccost_h[&C - P.chunks_h.data()]; };
  size_t nsplit = 0;  // split tiles at rounds 4
  for (double rounds : {1.0, 2.0, 4.0}) {
    std::vector<TcTile> tiles = P.tiles_h, w16 = P.wtiles_h[0], w32 = P.wtiles_h[1];
    std::vector<SplitRed> r0, r1, r2;
    long long p0 = 0, p1 = 0, p2 = 0;
    split_plan(tiles, P.chunks_h, r0, p0, (double)TC_CTAS * 152, rounds, cost);
    split_plan(w16, P.chunks_h, r1, p1, (double)SwCfg<16>::WARPS * SwCfg<16>::CTAS * 152, rounds, cost);
    split_plan(w32, P.chunks_h, r2, p2, (double)SwCfg<32>::WARPS * SwCfg<32>::CTAS * 152, rounds, cost);
    if (!check_split(P.tiles_h, tiles, r0, p0) || !check_split(P.wtiles_h[0], w16, r1, p1) ||
        !check_split(P.wtiles_h[1], w32, r2, p2))
      return false;
    nsplit = r0.size() + r1.size() + r2.size();
    std::string why;
    CHECK(check_plan(P, tiles, xbs, es, why), "tile plan rejected: %s", why.c_str());
    CHECK(check_small_plan<16>(P, w16, xbs, tl.groups, es, why), "16-state plan rejected: %s", why.c_str());
    CHECK(check_small_plan<32>(P, w32, xbs, tl.groups, es, why), "32-state plan rejected: %s", why.c_str());
    // a corrupted product record is refused
    int wt = -1;
    for (size_t i = 0; i < w16.size() && wt < 0; ++i)
      if (w16[i].c1 > w16[i].c0) wt = (int)i;
    if (wt >= 0) {
      TcPlan Q = P;
      const int t = Q.chunks_h[w16[wt].c0].t0;
      Q.tasks_h[t].R.kb += 32;
      CHECK(!check_small_plan<16>(Q, w16, xbs, tl.groups, es, why), "wrong K width accepted");
      Q = P;
      Q.tasks_h[t].L.off += 16;
      CHECK(!check_small_plan<16>(Q, w16, xbs, tl.groups, es, why), "misaligned image accepted");
    }
  }
  std::printf("ok seed %u limit %d %s: %d blocks on the 16-state kernel, %d on the 32-state kernel, %d on the tile "
              "kernel, %zu products, %zu images, %zu split tiles\n",
              seed, small, es == 2 ? "bf16x3" : "tf32", n16, n32, ntile, P.tasks_h.size(), jobs.size(), nsplit);
  return true;
}

}  // namespace

int main() {
  for (unsigned seed : {1u, 2u, 3u})
    for (int small : {32, 16, 24, 0})
      for (int es : {2, 4})
        if (!run(seed, small, es)) return 1;
  std::printf("ALL OK\n");
  return g_fail;
}
