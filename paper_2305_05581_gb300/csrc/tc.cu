// tc.cu -- reduced-precision form of the grouped triple product on the
// 5th-generation tensor cores (tcgen05, accumulators in TMEM).
//
// The products of one output tile that read the same input block X are
// fused the way Alg. 2 fuses the position sum (Sec. II.C): with
// p products sharing X,
//     GEMM1:  [T_1 | ... | T_p] = X [R_1; ...; R_p]^T        (N = p*r, one MMA chain)
//     GEMM2:  Y += [a_1 L_1 | ... | a_p L_p] [T_1; ...; T_p]   (K = p*m, accumulated in TMEM)
// so the sum over positions, operator pairs and dot blocks is the K loop of
// one accumulation, as SBMM4S does with cuBLAS, but without leaving the SM:
// T goes TMEM -> registers -> shared memory (re-split) -> GEMM2.
//
// Precisions: TNS_TF32 (kind::tf32, operands rounded to TF32) and TNS_BF16X3
// (x = x_hi + x_lo in bf16, three products hi*hi + hi*lo + lo*hi, FP32
// accumulation).  Operands are converted from the FP64 arenas while staged
// into shared memory in the no-swizzle K-major layout (8 x 16-byte core
// matrices, consecutive along K).  One CTA of 128 threads per output tile
// (<= 128 rows x <= 64 columns); thread 0 issues the MMAs; every wait on the
// MMA-completion mbarrier is bounded and reports a timeout flag instead of
// hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "cuda_backend.h"

namespace tns {

namespace {

// two CTAs of 8 warps per SM: ~105 KB shared memory and 256 TMEM columns each
constexpr int TC_NT = 256;
constexpr int TC_M = 128;    // MMA M (rows of a tile / of an X chunk)
constexpr int TC_RMAX = 64;  // tile columns
constexpr int TC_N1 = 128;   // GEMM1 N limit (p * r_pad) = TMEM columns of D1
constexpr int TC_K1 = 32;    // GEMM1 K chunk (elements)
constexpr int TC_K2 = 96;    // GEMM2 K limit per chunk (p * mc16)
constexpr long long TC_SPIN = 20000000;

struct TcTile {
  int g;
  int row0, col0, nrows, ncols;
  int c0, c1;      // chunk range of this piece
  long long poff;  // -1: write the output block; else offset of this piece's partial tile
};
struct TcChunk {
  int t0, t1;  // tasks (indices into the permuted task array)
  int kind;    // 0: T = X R^T (GEMM1 + GEMM2); 1: T = X directly (R identity)
  int pad;
};

struct TcPlan {
  Task* tasks = nullptr;
  TcTile* tiles = nullptr;
  TcChunk* chunks = nullptr;
  int ntiles = 0;
  int* flag = nullptr;
  SplitRed* reds = nullptr;  // split tiles (pieces summed in order afterwards)
  int nreds = 0;
  long long psize = 0;
  double* part = nullptr;
  int part_nvec = 0;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, LBO = 128 B between
// core matrices along K, SBO between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D f32, A/B format fmt (1 bf16, 2 tf32), K-major, M=128
__device__ __forceinline__ uint32_t idesc(int fmt, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}

template <int TF32>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (TF32)
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
                     tmem),
                 "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                     tmem),
                 "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

// bounded wait for phase `ph`; returns false on timeout
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t ph) {
  uint32_t done = 0;
  for (long long it = 0; it < TC_SPIN && !done; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(ph));
  }
  return done != 0;
}

// element (row, k) of a K-major no-swizzle operand with kc elements per row
template <int ES>
__device__ __forceinline__ int coff(int row, int k, int kc) {
  constexpr int KPC = 16 / ES;
  return (row >> 3) * (kc / KPC) * 128 + (k / KPC) * 128 + (row & 7) * 16 + (k % KPC) * ES;
}

template <int TF32>
__device__ __forceinline__ void put(unsigned char* hi, unsigned char* lo, int off, float x) {
  if (TF32) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    *(uint32_t*)(hi + off) = r;
  } else {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    *(__nv_bfloat16*)(hi + off) = h;
    *(__nv_bfloat16*)(lo + off) = l;
  }
}

__device__ __forceinline__ double g_opL(const Task& t, int i, int k) {
  if (t.flags & TF_LI) return i == k ? 1.0 : 0.0;
  return (t.flags & TF_LT) ? __ldg(t.L + (long long)k * t.q + i) : __ldg(t.L + (long long)i * t.m + k);
}
__device__ __forceinline__ double g_opR(const Task& t, int j, int k) {
  if (t.flags & TF_RI) return j == k ? 1.0 : 0.0;
  return (t.flags & TF_RT) ? __ldg(t.R + (long long)k * t.r + j) : __ldg(t.R + (long long)j * t.n + k);
}

template <int TF32>
__global__ void __launch_bounds__(TC_NT, 2) k_tasks_tc(const Task* __restrict__ tasks, const Group* __restrict__ groups,
                                                        const TcTile* __restrict__ tiles,
                                                        const TcChunk* __restrict__ chunks, const double* xv,
                                                        double* yv, long long xs, long long ys, int* flag,
                                                        double* part_all, long long psize) {
  constexpr int ES = TF32 ? 4 : 2;
  constexpr int NPROD = TF32 ? 1 : 3;
  constexpr int KSTEP = 16 / ES * 2;  // elements per MMA k-step (32 bytes)
  constexpr int SZ_A1 = TC_M * TC_K1 * ES, SZ_B1 = TC_N1 * TC_K1 * ES;
  constexpr int SZ_A2 = TC_M * TC_K2 * ES, SZ_B2 = TC_RMAX * TC_K2 * ES;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A1h = smem;
  unsigned char* A1l = A1h + SZ_A1;
  unsigned char* B1h = A1l + (TF32 ? 0 : SZ_A1);
  unsigned char* B1l = B1h + SZ_B1;
  unsigned char* A2h = B1l + (TF32 ? 0 : SZ_B1);
  unsigned char* A2l = A2h + SZ_A2;
  unsigned char* B2h = A2l + (TF32 ? 0 : SZ_A2);
  unsigned char* B2l = B2h + SZ_B2;
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ int bad;
  const int tid = threadIdx.x;
  const TcTile TL = tiles[blockIdx.x];
  const Group G = groups[TL.g];
  const int vec = blockIdx.y;
  const double* X0 = xv + (long long)vec * xs;
  const int rpad = (TL.ncols + 15) & ~15;
  double* part = TL.poff >= 0 ? part_all : nullptr;  // split piece: write the partial tile

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    bad = 0;
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tbase)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tD1 = tbase, tD2 = tbase + TC_N1;
  uint32_t phase = 0;
  bool d2 = false;

  for (int c = TL.c0; c < TL.c1 && !bad; ++c) {
    const TcChunk C = chunks[c];
    const int pc = C.t1 - C.t0;
    const Task t0 = tasks[C.t0];
    const double* Xp = X0 + (long long)(size_t)t0.X;
    const int m = t0.m, n = t0.n;
    const long long sXi = (t0.flags & TF_XT) ? 1 : n, sXk = (t0.flags & TF_XT) ? m : 1;
    for (int m0 = 0; m0 < m && !bad; m0 += TC_M) {
      const int mc = min(TC_M, m - m0);
      const int mc16 = (mc + 15) & ~15;
      if (C.kind == 0) {
        // GEMM1: D1[128 x pc*rpad] = X[m0.., :] * [R_t]^T
        const int N1 = pc * rpad;
        for (int n0 = 0; n0 < n && !bad; n0 += TC_K1) {
          // only rows that reach the output are staged: D1 rows >= mc and
          // columns of j >= ncols are never read back (K padding is zeroed)
          for (int e = tid; e < mc * TC_K1; e += TC_NT) {
            const int i = e / TC_K1, k = e % TC_K1;
            float x = (n0 + k < n) ? (float)__ldg(Xp + (m0 + i) * sXi + (n0 + k) * sXk) : 0.f;
            put<TF32>(A1h, A1l, coff<ES>(i, k, TC_K1), x);
          }
          for (int e = tid; e < pc * TL.ncols * TC_K1; e += TC_NT) {
            const int tj = e / TC_K1, k = e % TC_K1;
            const int t = tj / TL.ncols, j = tj % TL.ncols;
            const Task tk = tasks[C.t0 + t];
            float x = (n0 + k < n) ? (float)g_opR(tk, TL.col0 + j, n0 + k) : 0.f;
            put<TF32>(B1h, B1l, coff<ES>(t * rpad + j, k, TC_K1), x);
          }
          asm volatile("fence.proxy.async.shared::cta;");
          __syncthreads();
          if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t id = idesc(TF32 ? 2 : 1, N1);
            const uint32_t sboA = (TC_K1 / (16 / ES)) * 128, sboB = sboA;
            for (int ks = 0; ks < TC_K1 / KSTEP; ++ks)
              for (int pr = 0; pr < NPROD; ++pr) {
                const unsigned char* a = (pr == 2) ? A1l : A1h;
                const unsigned char* b = (pr == 1) ? B1l : B1h;
                uint32_t acc = (n0 > 0 || ks > 0 || pr > 0) ? 1u : 0u;
                mma<TF32>(tD1, sdesc(smem_u32(a) + ks * 256, sboA), sdesc(smem_u32(b) + ks * 256, sboB), id, acc);
              }
            commit(&bar);
          }
          if (!wait_bar(&bar, phase)) {
            bad = 1;
          }
          phase ^= 1;
          asm volatile("tcgen05.fence::after_thread_sync;");
          __syncthreads();
        }
        if (bad) break;
      }
      // stage A2 = [a_t L_t] (128 x pc*mc16) and B2 = [T_t]^T (rpad x pc*mc16)
      const int K2 = pc * mc16;
      for (int e = tid; e < TL.nrows * K2; e += TC_NT) {  // D2 rows >= nrows are never read back
        const int i = e / K2, kk = e % K2;
        const int t = kk / mc16, k = kk % mc16;
        const Task tk = tasks[C.t0 + t];
        float x = (k < mc) ? (float)(tk.alpha * g_opL(tk, TL.row0 + i, m0 + k)) : 0.f;
        put<TF32>(A2h, A2l, coff<ES>(i, kk, TC_K2), x);
      }
      if (C.kind == 0) {
        // from TMEM: warp w reads lane quarter w%4 (rows 32(w%4)..+31 of D1,
        // row = k index inside a task's slot); the two warpgroups split the
        // column chunks
        const int warp = tid >> 5, row = ((warp & 3) << 5) | (tid & 31), wg = warp >> 2;
        for (int t = 0; t < pc; ++t)
          for (int j0 = 8 * wg; j0 < rpad; j0 += 16) {
            uint32_t r[8];
            const uint32_t addr = tD1 + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(t * rpad + j0);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row < mc16)
              for (int q = 0; q < 8; ++q) {
                float x = (row < mc && j0 + q < TL.ncols) ? __uint_as_float(r[q]) : 0.f;
                put<TF32>(B2h, B2l, coff<ES>(j0 + q, t * mc16 + row, TC_K2), x);
              }
          }
      } else {
        // T = X directly (product with R = identity)
        for (int e = tid; e < rpad * K2; e += TC_NT) {
          const int j = e / K2, kk = e % K2;
          const int t = kk / mc16, k = kk % mc16;
          const Task tk = tasks[C.t0 + t];
          const double* Xt = X0 + (long long)(size_t)tk.X;
          const long long si = (tk.flags & TF_XT) ? 1 : tk.n, sk = (tk.flags & TF_XT) ? tk.m : 1;
          float x = (k < mc && j < TL.ncols) ? (float)__ldg(Xt + (m0 + k) * si + (TL.col0 + j) * sk) : 0.f;
          put<TF32>(B2h, B2l, coff<ES>(j, kk, TC_K2), x);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t id = idesc(TF32 ? 2 : 1, rpad);
        const uint32_t sboA = (TC_K2 / (16 / ES)) * 128, sboB = sboA;
        for (int ks = 0; ks < K2 / KSTEP; ++ks)
          for (int pr = 0; pr < NPROD; ++pr) {
            const unsigned char* a = (pr == 2) ? A2l : A2h;
            const unsigned char* b = (pr == 1) ? B2l : B2h;
            uint32_t acc = (d2 || ks > 0 || pr > 0) ? 1u : 0u;
            mma<TF32>(tD2, sdesc(smem_u32(a) + ks * 256, sboA), sdesc(smem_u32(b) + ks * 256, sboB), id, acc);
          }
        commit(&bar);
      }
      if (!wait_bar(&bar, phase)) bad = 1;
      phase ^= 1;
      d2 = true;
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();
    }
  }
  // epilogue: D2 -> Y (FP64)
  double* Y = yv + (long long)vec * ys + G.yoff;
  const int warp = tid >> 5, row = ((warp & 3) << 5) | (tid & 31), wg = warp >> 2;
  for (int j0 = 8 * wg; j0 < rpad; j0 += 16) {
    uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (d2 && !bad) {
      const uint32_t addr = tD2 + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)j0;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                   : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
    }
    if (row < TL.nrows)
      for (int q = 0; q < 8; ++q)
        if (j0 + q < TL.ncols) {
          if (part)
            part[(long long)vec * psize + TL.poff + row * TL.ncols + j0 + q] = (double)__uint_as_float(r[q]);
          else
            Y[(long long)(TL.row0 + row) * G.r + TL.col0 + j0 + q] = (double)__uint_as_float(r[q]);
        }
  }
  if (bad && tid == 0) {
    // let any MMA still in flight finish (bounded) before the TMEM is released
    wait_bar(&bar, phase);
    atomicExch(flag, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase));
}

template <int TF32>
constexpr int tc_smem() {
  constexpr int ES = TF32 ? 4 : 2;
  constexpr int mult = TF32 ? 1 : 2;
  return mult * (TC_M * TC_K1 + TC_N1 * TC_K1 + TC_M * TC_K2 + TC_RMAX * TC_K2) * ES + 1024;
}

void build_plan(const TaskList& tl, std::vector<Task>& perm, std::vector<TcTile>& tiles, std::vector<TcChunk>& chunks) {
  perm.clear();
  tiles.clear();
  chunks.clear();
  for (int g = 0; g < (int)tl.groups.size(); ++g) {
    const Group& G = tl.groups[g];
    // tasks of the group ordered by (kind, X block)
    std::vector<int> idx;
    for (int t = G.t0; t < G.t1; ++t) idx.push_back(t);
    auto kind = [&](int t) { return (tl.tasks[t].flags & TF_RI) ? 1 : 0; };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
      int ka = kind(a), kb = kind(b);
      if (ka != kb) return ka < kb;
      return (size_t)tl.tasks[a].X < (size_t)tl.tasks[b].X;
    });
    const int base = (int)perm.size();
    for (int t : idx) perm.push_back(tl.tasks[t]);
    for (int r0 = 0; r0 < G.q; r0 += TC_M)
      for (int c0 = 0; c0 < G.r; c0 += TC_RMAX) {
        TcTile T;
        T.g = g;
        T.row0 = r0;
        T.col0 = c0;
        T.nrows = std::min(TC_M, G.q - r0);
        T.ncols = std::min(TC_RMAX, G.r - c0);
        T.c0 = (int)chunks.size();
        const int rpad = (T.ncols + 15) & ~15;
        int i = 0;
        const int nt = (int)idx.size();
        while (i < nt) {
          const Task& a = perm[base + i];
          const int kd = (a.flags & TF_RI) ? 1 : 0;
          const int mc16 = ((std::min(a.m, TC_M) + 15) & ~15);
          int cap = TC_K2 / mc16;
          if (kd == 0) cap = std::min(cap, TC_N1 / rpad);
          cap = std::max(cap, 1);
          int j = i + 1;
          while (j < nt && j - i < cap) {
            const Task& b = perm[base + j];
            const int kb = (b.flags & TF_RI) ? 1 : 0;
            if (kb != kd || (kd == 0 && b.X != a.X) || b.m != a.m) break;
            ++j;
          }
          TcChunk C;
          C.t0 = base + i;
          C.t1 = base + j;
          C.kind = kd;
          C.pad = 0;
          chunks.push_back(C);
          i = j;
        }
        T.c1 = (int)chunks.size();
        T.poff = -1;
        tiles.push_back(T);
      }
  }
}

// cut tiles whose chunk lists are long into pieces of similar cost (each piece
// accumulates its own TMEM tile and writes a partial tile; the pieces are
// summed in order afterwards), so the CTAs of one launch finish together
void split_plan(const TaskList& tl, const std::vector<Task>& perm, std::vector<TcTile>& tiles,
                const std::vector<TcChunk>& chunks, std::vector<SplitRed>& reds, long long& psize, int sms) {
  auto ccost = [&](const TcChunk& C) {
    double s = 4.0e4;  // fixed cost of one chunk (staging passes and two MMA round trips)
    for (int t = C.t0; t < C.t1; ++t) {
      const Task& k = perm[t];
      s += 2.0 * k.m * k.n * std::min(k.r, TC_RMAX) + 2.0 * std::min(k.q, TC_M) * k.m * std::min(k.r, TC_RMAX);
    }
    return s;
  };
  std::vector<double> tcost(tiles.size(), 0.0);
  double tot = 0;
  for (size_t i = 0; i < tiles.size(); ++i) {
    for (int c = tiles[i].c0; c < tiles[i].c1; ++c) tcost[i] += ccost(chunks[c]);
    tot += tcost[i];
  }
  const double target = std::max(tot / (2.0 * sms * 2.0), 1.0);
  std::vector<TcTile> out;
  psize = 0;
  reds.clear();
  for (size_t i = 0; i < tiles.size(); ++i) {
    const TcTile& T = tiles[i];
    const int nch = T.c1 - T.c0;
    int ns = (int)std::min<double>(nch, std::ceil(tcost[i] / target));
    ns = std::max(1, std::min(ns, 64));
    if (ns == 1) {
      out.push_back(T);
      continue;
    }
    SplitRed R;
    R.g = T.g;
    R.row0 = T.row0;
    R.col0 = T.col0;
    R.nrows = T.nrows;
    R.ncols = T.ncols;
    R.poff = psize;
    int start = T.c0, made = 0;
    double acc = 0;
    for (int c = T.c0; c < T.c1 && made < ns - 1; ++c) {
      acc += ccost(chunks[c]);
      if (acc >= tcost[i] * (made + 1) / ns) {
        TcTile p = T;
        p.c0 = start;
        p.c1 = c + 1;
        p.poff = psize;
        psize += (long long)T.nrows * T.ncols;
        out.push_back(p);
        ++made;
        start = c + 1;
      }
    }
    TcTile p = T;
    p.c0 = start;
    p.c1 = T.c1;
    p.poff = psize;
    psize += (long long)T.nrows * T.ncols;
    out.push_back(p);
    R.nsplit = made + 1;
    reds.push_back(R);
  }
  tiles.swap(out);
  (void)tl;
}

}  // namespace

void launch_reduce_splits(CudaBackend& be, const SplitRed* reds, int nreds, const Group* groups, const double* part,
                          long long psize, double* yv, long long ys, int nvec);

void release_tc_plan(void* p);

void launch_tasks_tc(CudaBackend& be, const TaskList& tl, DevList& d, const double* xv, double* yv, int nvec,
                     long long xs, long long ys, int precision) {
  TcPlan* plan = (TcPlan*)d.tc;
  if (!plan || d.tc_gen != tl.gen) {
    if (plan) {
      cudaStreamSynchronize(be.stream());
      release_tc_plan(plan);
    }
    std::vector<Task> perm;
    std::vector<TcTile> tiles;
    std::vector<TcChunk> chunks;
    std::vector<SplitRed> reds;
    long long psize = 0;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, be.device());
    build_plan(tl, perm, tiles, chunks);
    split_plan(tl, perm, tiles, chunks, reds, psize, sms);
    plan = new TcPlan();
    bool ok = cudaMalloc(&plan->tasks, sizeof(Task) * std::max<size_t>(perm.size(), 1)) == cudaSuccess &&
              cudaMalloc(&plan->tiles, sizeof(TcTile) * std::max<size_t>(tiles.size(), 1)) == cudaSuccess &&
              cudaMalloc(&plan->chunks, sizeof(TcChunk) * std::max<size_t>(chunks.size(), 1)) == cudaSuccess &&
              cudaMalloc(&plan->flag, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&plan->reds, sizeof(SplitRed) * std::max<size_t>(reds.size(), 1)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      be.note(cudaErrorMemoryAllocation, "tensor-core plan");
      release_tc_plan(plan);
      d.tc = nullptr;
      return;
    }
    if (!perm.empty()) cudaMemcpyAsync(plan->tasks, perm.data(), sizeof(Task) * perm.size(), cudaMemcpyHostToDevice, be.stream());
    if (!tiles.empty()) cudaMemcpyAsync(plan->tiles, tiles.data(), sizeof(TcTile) * tiles.size(), cudaMemcpyHostToDevice, be.stream());
    if (!chunks.empty()) cudaMemcpyAsync(plan->chunks, chunks.data(), sizeof(TcChunk) * chunks.size(), cudaMemcpyHostToDevice, be.stream());
    if (!reds.empty()) cudaMemcpyAsync(plan->reds, reds.data(), sizeof(SplitRed) * reds.size(), cudaMemcpyHostToDevice, be.stream());
    plan->ntiles = (int)tiles.size();
    plan->nreds = (int)reds.size();
    plan->psize = psize;
    d.tc = plan;
    d.tc_gen = tl.gen;
    be.note(cudaStreamSynchronize(be.stream()), "tensor-core plan upload");
  }
  if (plan->ntiles == 0) return;
  if (plan->psize > 0 && plan->part_nvec < nvec) {
    if (plan->part) {
      cudaStreamSynchronize(be.stream());
      cudaFree(plan->part);
    }
    plan->part = nullptr;
    plan->part_nvec = 0;
    if (cudaMalloc(&plan->part, sizeof(double) * plan->psize * nvec) != cudaSuccess) {
      cudaGetLastError();
      be.note(cudaErrorMemoryAllocation, "tensor-core partial tiles");
      plan->part = nullptr;
      return;
    }
    plan->part_nvec = nvec;
  }
  cudaMemsetAsync(plan->flag, 0, sizeof(int), be.stream());
  dim3 grid(plan->ntiles, nvec);
  if (precision == 1) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_tasks_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<1>());
      attr = true;
    }
    k_tasks_tc<1><<<grid, TC_NT, tc_smem<1>(), be.stream()>>>(plan->tasks, d.groups, plan->tiles, plan->chunks, xv,
                                                             yv, xs, ys, plan->flag, plan->part, plan->psize);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_tasks_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<0>());
      attr = true;
    }
    k_tasks_tc<0><<<grid, TC_NT, tc_smem<0>(), be.stream()>>>(plan->tasks, d.groups, plan->tiles, plan->chunks, xv,
                                                             yv, xs, ys, plan->flag, plan->part, plan->psize);
  }
  be.launches++;
  be.note(cudaGetLastError(), "k_tasks_tc");
  if (plan->nreds > 0)
    launch_reduce_splits(be, plan->reds, plan->nreds, d.groups, plan->part, plan->psize, yv, ys, nvec);
  int h = 0;
  cudaMemcpyAsync(&h, plan->flag, sizeof(int), cudaMemcpyDeviceToHost, be.stream());
  be.note(cudaStreamSynchronize(be.stream()), "k_tasks_tc");
  if (h) be.note(cudaErrorLaunchTimeout, "k_tasks_tc: MMA completion wait timed out");
}

void release_tc_plan(void* p) {
  TcPlan* plan = (TcPlan*)p;
  if (!plan) return;
  if (plan->reds) cudaFree(plan->reds);
  if (plan->part) cudaFree(plan->part);
  cudaFree(plan->tasks);
  cudaFree(plan->tiles);
  cudaFree(plan->chunks);
  cudaFree(plan->flag);
  delete plan;
}

}  // namespace tns
