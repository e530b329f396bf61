// tc.cu -- reduced-precision form of the grouped triple product on the
// 5th-generation tensor cores (tcgen05, accumulators in TMEM).
//
// Every product of H_eff*psi is Y += a op(L) X op(R)^T (Eq. 2); an identity
// operator is a small identity image, so all products take one path.  The
// products of one output tile that read the same X block are fused the way
// Alg. 2 fuses the position sum (Sec. II.C):
//     GEMM1:  [T_1^T; ...; T_p^T] = [R_1; ...; R_p] X^T    (R rows stacked into M = 128)
//     GEMM2:  Y += sum_t (a_t L_t) T_t                       (one TMEM accumulator)
// The TMEM rows of GEMM1 are rows of T_t^T, so in the T pass each thread
// holds eight consecutive K elements of GEMM2's B operand and writes them,
// scaled by a_t and re-split, as one 16-byte vector.
//
// Operands: the L/R operator blocks are fixed during the ~50 products of a
// two-site step, so they are converted once per step into images -- bf16 hi +
// bf16 lo (TNS_BF16X3: x = hi + lo, three products hi*hi + hi*lo + lo*hi) or
// tf32 (TNS_TF32) -- already in the K-major, no-swizzle core-matrix layout the
// MMA reads: K in chunks of 64 bytes per row; inside a chunk, groups of 8 rows
// of 16-byte core matrices.  X is converted once per product call.  Staging
// is a few cp.async.bulk copies per chunk with mbarrier completion; the FP64
// pipe stays out of the product loop.
//
// One CTA (256 threads) per output tile piece (128 rows x <= 64 columns);
// thread 0 issues copies and MMAs from the chunk's product metadata, which
// all threads stage in shared memory one chunk ahead; GEMM2's first copies
// are issued while the T pass runs; all threads do the T pass and the
// epilogue.  Steps of 32 X rows and one staging region shared by the two
// GEMMs keep a CTA at 56 KB of shared memory, three per SM.
// Every wait is bounded; a timeout sets a flag the host reads, after the CTA
// has drained (bounded) its own copies and MMAs and released its TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/tns.h"
#include "cuda_backend.h"

namespace tns {

namespace {

constexpr int TC_NT = 256;
constexpr int TC_M = 128;     // MMA M: output tile rows; stacked R rows of GEMM1
constexpr int TC_NC = 64;     // output tile columns (GEMM2 N <= 64)
constexpr int TC_MC = 32;     // X rows per GEMM1 step (GEMM1 N <= 32, GEMM2 K <= 32)
constexpr int TC_CTAS = 3;    // resident CTAs per SM (shared memory and registers are sized for it)
constexpr int CH_BYTES = 64;  // bytes of one K chunk of one row (4 core matrices)
constexpr unsigned long long TC_WAIT_NS = 200000000ull;  // bound of one wait: 0.2 s

// operand image: rows padded to 8, K padded to 32 bytes, K chunks of 64 bytes
struct Img {
  long long off;  // byte offset in the image arena (hi; lo at the same offset)
  int rg;         // row groups (rows / 8, rounded up)
  int kb;         // padded K in bytes (multiple of 32)
};

struct TcTask {
  float alpha;
  int xb;  // X block index (its image is converted per call)
  Img L, R;
  int m, n;  // X block m x n (= columns of op(L), columns of op(R))
};

struct TcTile {
  int g;
  int row0, col0, nrows, ncols;
  int c0, c1;      // chunk range of this piece
  long long poff;  // -1: write the output block; else offset of this piece's partial tile
};

struct TcChunk {
  int t0, t1;  // products sharing one X block
  int xb;      // that X block
  int pad;
};

struct XBlock {
  long long src;  // element offset of the block in the psi vector
  int m, n;
  Img img;
};

struct ImgJob {  // convert one operand block into its image
  const double* src;
  int rows, cols;  // op(M) is rows x cols
  int trans;       // op(M)[i][k] = trans ? M[k * rows + i] : M[i * cols + k]; identity if src == null
  Img img;
};

struct TcVariant {
  bool planned = false;
  TcTile* tiles = nullptr;  // pieces of the tile kernel
  int ntiles = 0;
  TcTile* wtiles[2] = {nullptr, nullptr};  // pieces of the small-block warp kernel (blocks <= 16, <= 32)
  int nwtiles[2] = {0, 0};
  // persistent kernel: pieces of CTA b are ws_order[ws_off[b] .. ws_off[b+1])
  int* ws_order = nullptr;
  int* ws_off = nullptr;
  int ws_ctas = 0;
  SplitRed* reds = nullptr;
  int nreds = 0;
  long long psize = 0;
  double* part = nullptr;
  int part_nvec = 0;
};

struct SwRec;

struct TcPlan {
  int precision = 0;
  TcTask* tasks = nullptr;
  SwRec* swrec = nullptr;  // the products as 16-byte records of the small-block kernel
  TcChunk* chunks = nullptr;
  XBlock* xblocks = nullptr;
  int nxb = 0;
  int* flag = nullptr;
  unsigned char* ops_hi = nullptr;  // L/R images (built once per plan)
  unsigned char* ops_lo = nullptr;
  long long ops_bytes = 0;
  unsigned char* x_hi = nullptr;  // X images (per product call, per vector)
  unsigned char* x_lo = nullptr;
  long long x_bytes = 0;  // per vector
  int x_nvec = 0;
  std::vector<TcTask> tasks_h;
  std::vector<TcTile> tiles_h;   // tiles of the tile kernel
  std::vector<TcTile> wtiles_h[2];  // output blocks of the small-block warp kernel (<= 16, <= 32)
  std::vector<TcChunk> chunks_h;
  std::vector<double> ccost_h;  // estimated cost of each chunk (its tile's kernel), shared by every variant's split
  std::vector<XBlock> xbs_h;
  TcVariant var[kNumVariants];
  int sms = 152;
};

__host__ __device__ inline long long img_bytes(const Img& g) { return (long long)g.rg * 8 * g.kb; }
// bytes per row of K chunk c, and the chunk's offset
__host__ __device__ inline int chunk_w(const Img& g, int c) {
  const int w = g.kb - c * CH_BYTES;
  return w < CH_BYTES ? w : CH_BYTES;
}
__host__ __device__ inline long long chunk_off(const Img& g, int c) {
  return g.off + (long long)g.rg * 8 * c * CH_BYTES;
}

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

__device__ __forceinline__ void bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bulk global -> shared copy completing on `bar` (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// wait for phase `ph`, bounded in time (bound_ns); returns false on timeout
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t ph, unsigned long long bound_ns) {
  uint32_t done = 0;
  const unsigned long long t0 = gtimer();
  while (!done) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(ph)
                 : "memory");
    if (!done && gtimer() - t0 > bound_ns) break;
  }
  return done != 0;
}

// ---------------------------------------------------------------------------
// image conversion: one thread per 16-byte unit of the destination
// ---------------------------------------------------------------------------
template <int TF32>
__device__ __forceinline__ void convert_unit(const double* v, unsigned char* hi, unsigned char* lo, long long off) {
  if (TF32) {
    uint32_t r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r[e]) : "f"((float)v[e]));
    *(uint4*)(hi + off) = make_uint4(r[0], r[1], r[2], r[3]);
  } else {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float x = (float)v[e];
      h[e] = __float2bfloat16_rn(x);
      l[e] = __float2bfloat16_rn(x - __bfloat162float(h[e]));
    }
    *(uint4*)(hi + off) = *(const uint4*)h;
    *(uint4*)(lo + off) = *(const uint4*)l;
  }
}

// 16-byte unit u of an image (units in byte order: chunk, row group, core
// matrix, row) -> its row, first K element and byte offset
template <int TF32>
__device__ __forceinline__ void unit_pos(const Img& g, long long u, int& row, int& k0, long long& off) {
  constexpr int ES = TF32 ? 4 : 2;
  long long rem = u;
  int c = 0;
  for (;; ++c) {
    const long long cu = (long long)g.rg * 8 * chunk_w(g, c) / 16;
    if (rem < cu) break;
    rem -= cu;
  }
  const int kcm = chunk_w(g, c) / 16;
  const int r8 = (int)(rem % 8);
  const long long t = rem / 8;
  const int kk = (int)(t % kcm);
  const int rgi = (int)(t / kcm);
  row = rgi * 8 + r8;
  k0 = (c * CH_BYTES + kk * 16) / ES;
  off = chunk_off(g, c) + ((long long)rgi * kcm + kk) * 128 + r8 * 16;
}

template <int TF32>
__global__ void __launch_bounds__(256) k_img_ops(const ImgJob* __restrict__ jobs, unsigned char* hi,
                                                 unsigned char* lo) {
  constexpr int EPU = TF32 ? 4 : 8;  // elements per 16-byte unit
  const ImgJob J = jobs[blockIdx.x];
  const long long units = img_bytes(J.img) / 16;
  for (long long u = threadIdx.x; u < units; u += blockDim.x) {
    int row, k0;
    long long off;
    unit_pos<TF32>(J.img, u, row, k0, off);
    double v[EPU];
#pragma unroll
    for (int e = 0; e < EPU; ++e) {
      const int k = k0 + e;
      double x = 0.0;
      if (row < J.rows && k < J.cols) {
        if (!J.src)
          x = row == k ? 1.0 : 0.0;
        else
          x = J.trans ? J.src[(long long)k * J.rows + row] : J.src[(long long)row * J.cols + k];
      }
      v[e] = x;
    }
    convert_unit<TF32>(v, hi, lo, off);
  }
}

template <int TF32>
__global__ void __launch_bounds__(256) k_img_x(const XBlock* __restrict__ xb, const double* xv, long long xs,
                                               unsigned char* hi, unsigned char* lo, long long xbytes) {
  constexpr int EPU = TF32 ? 4 : 8;
  const XBlock B = xb[blockIdx.x];
  const int vec = blockIdx.y;
  const double* X = xv + (long long)vec * xs + B.src;
  unsigned char* h = hi + (long long)vec * xbytes;
  unsigned char* l = TF32 ? nullptr : lo + (long long)vec * xbytes;
  const long long units = img_bytes(B.img) / 16;
  for (long long u = threadIdx.x; u < units; u += blockDim.x) {
    int row, k0;
    long long off;
    unit_pos<TF32>(B.img, u, row, k0, off);
    double v[EPU];
#pragma unroll
    for (int e = 0; e < EPU; ++e) {
      const int k = k0 + e;
      v[e] = (row < B.m && k < B.n) ? X[(long long)row * B.n + k] : 0.0;
    }
    convert_unit<TF32>(v, h, l, off);
  }
}

// ---------------------------------------------------------------------------
// the product kernel
// ---------------------------------------------------------------------------
template <int TF32>
struct TcSmem {
  static constexpr int ES = TF32 ? 4 : 2;
  static constexpr int NS = TF32 ? 1 : 2;       // planes: hi (+ lo)
  static constexpr int A1 = TC_M * CH_BYTES;    // stacked R rows, one K chunk
  static constexpr int B1 = TC_MC * CH_BYTES;   // X rows, one K chunk
  static constexpr int CB2 = TC_M * CH_BYTES;   // one K chunk of B2 (all 128 rows)
  static constexpr int B2 = TC_MC * ES / CH_BYTES * CB2;  // T^T of all products, K = TC_MC
  static constexpr int A2 = TC_M * CH_BYTES;    // L rows, one K chunk (two buffers)
  // GEMM1's two operand buffers and GEMM2's two L buffers share one region
  // (they are never live together: GEMM2's copies start once D1 is
  // complete, GEMM1's once the previous GEMM2's MMAs are done), which keeps
  // a CTA at 56 KB (split-BF16) so that three fit on an SM
  static constexpr int G1 = 2 * NS * (A1 + B1), G2 = 2 * NS * A2;
  static constexpr int R1 = G1 > G2 ? G1 : G2;
  static constexpr int total = R1 + NS * B2;
};

template <int TF32>
__global__ void __launch_bounds__(TC_NT, TC_CTAS)
    k_tasks_tc(const TcTask* __restrict__ tasks, const Group* __restrict__ groups, const TcTile* __restrict__ tiles,
               const TcChunk* __restrict__ chunks, const unsigned char* __restrict__ ops_hi,
               const unsigned char* __restrict__ ops_lo, const unsigned char* __restrict__ x_hi,
               const unsigned char* __restrict__ x_lo, long long x_bytes, const XBlock* __restrict__ xblocks,
               double* yv, long long ys, int* flag, double* part_all, long long psize, int nv,
               unsigned long long wait_ns) {
  using S = TcSmem<TF32>;
  constexpr int ES = S::ES;
  constexpr int NPROD = TF32 ? 1 : 3;
  constexpr int EPC = CH_BYTES / ES;              // elements per K chunk
  constexpr uint32_t SBO_FULL = (CH_BYTES / 16) * 128;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* const sG1 = smem;                    // GEMM1 operand buffers, or
  unsigned char* const sA2 = smem;                    // GEMM2 L buffers: buffer b, plane p at + (b * NS + p) * S::A2
  unsigned char* const sB2 = smem + S::R1;            // planes at + p * S::B2
  auto sA1 = [&](int b) { return sG1 + b * S::NS * (S::A1 + S::B1); };          // plane p at + p * S::A1
  auto sB1 = [&](int b) { return sG1 + b * S::NS * (S::A1 + S::B1) + S::NS * S::A1; };  // plane p at + p * S::B1
  __shared__ uint64_t lbar1[2], mbar1[2], lbar2[2], mbar2[2];
  __shared__ uint32_t tbase;
  __shared__ int bad;
  // metadata of the products of a chunk (at most TC_M / 16 share one X
  // block), double-buffered by chunk parity: thread 0's copy and MMA issue
  // reads it from here instead of from global memory
  struct MetaT {
    Img L, R;
    float alpha;
  };
  struct Meta {
    MetaT t[TC_M / 16];
    XBlock xb;
    int pc;
  };
  __shared__ Meta meta[2];
  const int tid = threadIdx.x;
  // the vectors of one tile piece are adjacent CTAs (they read the same operator blocks)
  const TcTile TL = tiles[blockIdx.x / nv];
  const Group G = groups[TL.g];
  const int vec = blockIdx.x % nv;
  const unsigned char* xh = x_hi + (long long)vec * x_bytes;
  const unsigned char* xl = TF32 ? nullptr : x_lo + (long long)vec * x_bytes;
  const int rp = (TL.ncols + 15) & ~15;  // GEMM2 N; rows of one product in the GEMM1 stack
  const bool has_work = TL.c1 > TL.c0;   // uniform: this piece issues at least one GEMM2 chain
  double* part = TL.poff >= 0 ? part_all : nullptr;

  if (tid == 0) {
    bar_init(&lbar1[0]);
    bar_init(&lbar1[1]);
    bar_init(&mbar1[0]);
    bar_init(&mbar1[1]);
    bar_init(&lbar2[0]);
    bar_init(&lbar2[1]);
    bar_init(&mbar2[0]);
    bar_init(&mbar2[1]);
    asm volatile("fence.mbarrier_init.release.cluster;");
    bad = 0;
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&tbase)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tD1 = tbase, tD2 = tbase + 64;
  // barrier bookkeeping (thread 0 only): phases and outstanding completions
  uint32_t pl1[2] = {0, 0}, pm1[2] = {0, 0}, pl2[2] = {0, 0}, pm2[2] = {0, 0};
  int l1_out[2] = {0, 0}, m1_out[2] = {0, 0}, l2_out[2] = {0, 0}, m2_out[2] = {0, 0};
  int g2_steps = 0;
  bool d2 = false;
  int where_c = -1, where_m0 = -1, where_s = -1;
  // waits inside the product loop give up after wait_ns; the final drain
  // before TMEM is released always allows the full TC_WAIT_NS, so that no copy
  // or MMA of this CTA is still in flight when it exits
  auto drain = [&](uint64_t* bar, uint32_t& ph, int& out, unsigned long long bound = 0) {
    if (!out) return;
    if (wait_bar(bar, ph, bound ? bound : wait_ns)) {
      ph ^= 1;
      out = 0;
    } else {
      if (!bad && atomicCAS(flag, 0, 1) == 0) {
        const int which = (bar == &lbar1[0] || bar == &lbar1[1]) ? 1 : (bar == &mbar1[0] || bar == &mbar1[1]) ? 2
                        : bar == &lbar2[0] ? 3 : bar == &lbar2[1] ? 4 : bar == &mbar2[0] ? 5 : 6;
        flag[1] = blockIdx.x;
        flag[2] = which;
        flag[3] = where_c;
        flag[4] = where_m0;
        flag[5] = where_s;
        flag[6] = (int)ph;
      }
      bad = 1;
    }
  };

  // thread 0's copy issue for the steps (chunk c, X rows m0..m0+TC_MC-1) of this
  // piece; GEMM1 chunk kc of a step goes to G1 buffer kc & 1, GEMM2 slice st
  // (product st / nch2, K chunk st % nch2) to G2 buffer (g2_steps + st) & 1
  // all threads: metadata of chunk c into meta[c & 1]
  auto load_meta = [&](int c) {
    const TcChunk C = chunks[c];
    Meta& M = meta[c & 1];
    const int pc = C.t1 - C.t0;
    if (tid < pc) {
      const TcTask& k = tasks[C.t0 + tid];
      M.t[tid].L = k.L;
      M.t[tid].R = k.R;
      M.t[tid].alpha = k.alpha;
    }
    if (tid == 0) {
      M.pc = pc;
      M.xb = xblocks[C.xb];
    }
  };
  auto issue1 = [&](int c, int m0, int kc, int b) {
    const Meta& M = meta[c & 1];
    const int pc = M.pc;
    const XBlock& XB = M.xb;
    const int mc16 = (min(TC_MC, XB.m - m0) + 15) & ~15;
    const int xg0 = m0 / 8, xng = min(mc16 / 8, XB.img.rg - xg0);
    const uint32_t rowb = (chunk_w(XB.img, kc) / 16) * 128;  // bytes of one row group in this chunk
    uint32_t bytes = (xng > 0 ? xng * rowb : 0) * S::NS;
    for (int t = 0; t < pc; ++t) {
      const int ng = min(rp / 8, M.t[t].R.rg - TL.col0 / 8);
      if (ng > 0) bytes += ng * rowb * S::NS;
    }
    expect_tx(&lbar1[b], bytes);
    l1_out[b] = 1;
    if (xng > 0) {
      const long long xo = chunk_off(XB.img, kc) + (long long)xg0 * rowb;
      bulk_g2s(sB1(b), xh + xo, xng * rowb, &lbar1[b]);
      if (!TF32) bulk_g2s(sB1(b) + S::B1, xl + xo, xng * rowb, &lbar1[b]);
    }
    for (int t = 0; t < pc; ++t) {
      const Img R = M.t[t].R;
      const int ng = min(rp / 8, R.rg - TL.col0 / 8);
      if (ng <= 0) continue;
      const long long ro = chunk_off(R, kc) + (long long)(TL.col0 / 8) * rowb;
      const uint32_t dst = (uint32_t)(t * rp / 8) * rowb;
      bulk_g2s(sA1(b) + dst, ops_hi + ro, ng * rowb, &lbar1[b]);
      if (!TF32) bulk_g2s(sA1(b) + S::A1 + dst, ops_lo + ro, ng * rowb, &lbar1[b]);
    }
  };
  // the first (up to) two GEMM1 chunks of a step, into free G1 buffers
  auto prefetch1 = [&](int c, int m0) {
    const int nch = (meta[c & 1].xb.img.kb + CH_BYTES - 1) / CH_BYTES;
    for (int kc = 0; kc < 2 && kc < nch; ++kc) issue1(c, m0, kc, kc);
  };
  auto issue2 = [&](int c, int m0, int st, int nch2, int b) {
    const int t = st / nch2, c2 = st % nch2;
    const Img Lm = meta[c & 1].t[t].L;
    const int lg0 = TL.row0 / 8, lng = min(TC_M / 8, Lm.rg - lg0);
    const int lc = (m0 * ES) / CH_BYTES + c2;  // chunk of L's K (= X rows)
    const uint32_t rowb = (chunk_w(Lm, lc) / 16) * 128;
    unsigned char* a2 = sA2 + b * S::NS * S::A2;
    expect_tx(&lbar2[b], lng * rowb * S::NS);
    l2_out[b] = 1;
    const long long lo_ = chunk_off(Lm, lc) + (long long)lg0 * rowb;
    bulk_g2s(a2, ops_hi + lo_, lng * rowb, &lbar2[b]);
    if (!TF32) bulk_g2s(a2 + S::A2, ops_lo + lo_, lng * rowb, &lbar2[b]);
  };
  if (has_work) load_meta(TL.c0);
  __syncthreads();
  if (tid == 0 && has_work) prefetch1(TL.c0, 0);
  bool first_step = true;  // thread 0: the first step's GEMM1 chunks are already in flight

  for (int c = TL.c0; c < TL.c1 && !bad; ++c) {
    // the next chunk's metadata goes to the other buffer, free since the last
    // step of chunk c-1 ended (thread 0 reads it for its prefetch at the end
    // of this chunk, after the barriers of this chunk's steps)
    if (c + 1 < TL.c1) load_meta(c + 1);
    const Meta& M = meta[c & 1];
    const int pc = M.pc;
    const XBlock XB = M.xb;
    const int m = XB.m;
    where_c = c;
    for (int m0 = 0; m0 < m && !bad; m0 += TC_MC) {
      where_m0 = m0;
      const int mc = min(TC_MC, m - m0);
      const int mc16 = (mc + 15) & ~15;
      const int nch2 = (mc16 * ES + CH_BYTES - 1) / CH_BYTES;
      const int nsteps = pc * nch2;
      if (tid == 0) {
        // ---- GEMM1: D1[t*rp + j][i] = sum_k R_t[col0 + j][k] X[m0 + i][k] ----
        // the previous step's GEMM2 MMAs read the shared region and B2: done
        // first; then chunks 0 and 1 of this step (the first step's were
        // issued before the loop); chunk kc+1 >= 2 is copied once chunk
        // kc-1's MMAs have released its buffer
        drain(&mbar2[0], pm2[0], m2_out[0]);
        drain(&mbar2[1], pm2[1], m2_out[1]);
        if (!first_step && !bad) prefetch1(c, m0);
        first_step = false;
        const int nch = (XB.img.kb + CH_BYTES - 1) / CH_BYTES;
        for (int kc = 0; kc < nch && !bad; ++kc) {
          where_s = kc;
          const int b = kc & 1, bn = (kc + 1) & 1;
          if (kc + 1 < nch && kc + 1 >= 2) {
            drain(&mbar1[bn], pm1[bn], m1_out[bn]);
            if (bad) break;
            issue1(c, m0, kc + 1, bn);
          }
          drain(&lbar1[b], pl1[b], l1_out[b]);
          if (bad) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int kcm = chunk_w(XB.img, kc) / 16;
          const uint32_t rowb = kcm * 128;
          const uint32_t id = idesc(TF32 ? 2 : 1, mc16);
          for (int ks = 0; ks < kcm / 2; ++ks)
            for (int pr = 0; pr < NPROD; ++pr) {
              const unsigned char* a = sA1(b) + (pr == 2 ? S::A1 : 0);
              const unsigned char* bb = sB1(b) + (pr == 1 ? S::B1 : 0);
              const uint32_t acc = (kc > 0 || ks > 0 || pr > 0) ? 1u : 0u;
              mma<TF32>(tD1, sdesc(smem_u32(a) + ks * 256, rowb), sdesc(smem_u32(bb) + ks * 256, rowb), id, acc);
            }
          commit(&mbar1[b]);
          m1_out[b] = 1;
        }
        // D1 complete before the T pass; the shared region is then free and
        // this step's first two L slices are copied while the T pass runs
        drain(&mbar1[0], pm1[0], m1_out[0]);
        drain(&mbar1[1], pm1[1], m1_out[1]);
        for (int st = 0; st < 2 && st < nsteps && !bad; ++st) issue2(c, m0, st, nch2, (g2_steps + st) & 1);
      }
      __syncthreads();
      if (bad) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      // ---- T pass: D1 (fp32) -> B2 = a_t T_t^T in the K-major operand layout ----
      {
        const int warp = tid >> 5, wg = warp >> 2;
        const int row = (warp & 3) * 32 + (tid & 31);  // TMEM lane = stacked R row = B2 row
        const int t = row / rp;
        const float al = (t < pc) ? M.t[t].alpha : 0.f;
        for (int i0 = 8 * wg; i0 < mc16; i0 += 16) {
          uint32_t r[8];
          const uint32_t addr = tD1 + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)i0;
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                         "=r"(r[7])
                       : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          if (t >= pc) continue;
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = (i0 + e < mc) ? al * __uint_as_float(r[e]) : 0.f;
          if (TF32) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int i = i0 + 4 * h;
              const int off = (i / EPC) * S::CB2 + ((row >> 3) * (CH_BYTES / 16) + (i % EPC) * ES / 16) * 128 +
                              (row & 7) * 16;
              uint32_t q[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(q[e]) : "f"(v[4 * h + e]));
              *(uint4*)(sB2 + off) = make_uint4(q[0], q[1], q[2], q[3]);
            }
          } else {
            const int off = (i0 / EPC) * S::CB2 + ((row >> 3) * (CH_BYTES / 16) + (i0 % EPC) * ES / 16) * 128 +
                            (row & 7) * 16;
            __align__(16) __nv_bfloat16 hh[8], ll[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              hh[e] = __float2bfloat16_rn(v[e]);
              ll[e] = __float2bfloat16_rn(v[e] - __bfloat162float(hh[e]));
            }
            *(uint4*)(sB2 + off) = *(const uint4*)hh;
            *(uint4*)(sB2 + S::B2 + off) = *(const uint4*)ll;
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      // ---- GEMM2: D2 += sum_t L_t[row0.., m0 + k] * B2_t^T (thread 0) ----
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int nk2 = mc16 * ES / 32;  // 32-byte MMA k-steps over this X row range
        const uint32_t id = idesc(TF32 ? 2 : 1, rp);
        // two-stage pipeline over the steps s = (product t, K chunk c2): the
        // L slice of step s+1 is copied while step s's MMAs run
        for (int st = 0; st < nsteps && !bad; ++st) {
          const int b = (g2_steps + st) & 1, bn = (g2_steps + st + 1) & 1;
          where_s = 1000 + st;
          if (st + 1 < nsteps && st + 1 >= 2) {
            drain(&mbar2[bn], pm2[bn], m2_out[bn]);  // the MMAs of step st-1 read buffer bn
            if (bad) break;
            issue2(c, m0, st + 1, nch2, bn);
          }
          drain(&lbar2[b], pl2[b], l2_out[b]);
          if (bad) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const int t = st / nch2, c2 = st % nch2;
          const Img Lm = M.t[t].L;
          const int lc = (m0 * ES) / CH_BYTES + c2;
          const int kcm = chunk_w(Lm, lc) / 16;
          const uint32_t rowb = kcm * 128;
          const unsigned char* a2 = sA2 + b * S::NS * S::A2;
          const uint32_t bt = (uint32_t)(t * rp / 8) * SBO_FULL;  // product t's rows inside a B2 chunk
          const int ks_here = min(kcm / 2, nk2 - c2 * (CH_BYTES / 32));
          for (int ks = 0; ks < ks_here; ++ks)
            for (int pr = 0; pr < NPROD; ++pr) {
              const unsigned char* a = a2 + (pr == 2 ? S::A2 : 0);
              const unsigned char* bb = sB2 + (pr == 1 ? S::B2 : 0) + c2 * S::CB2 + bt;
              const uint32_t acc = (d2 || ks > 0 || pr > 0) ? 1u : 0u;
              mma<TF32>(tD2, sdesc(smem_u32(a) + ks * 256, rowb), sdesc(smem_u32(bb) + ks * 256, SBO_FULL), id,
                        acc);
            }
          d2 = true;
          commit(&mbar2[b]);
          m2_out[b] = 1;
        }
        g2_steps += nsteps;
      }
      __syncthreads();
    }
  }
  // every copy and MMA of this CTA done (bounded) before TMEM is read or released
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      drain(&lbar1[b], pl1[b], l1_out[b], TC_WAIT_NS);
      drain(&mbar1[b], pm1[b], m1_out[b], TC_WAIT_NS);
    }
    for (int b = 0; b < 2; ++b) {
      drain(&lbar2[b], pl2[b], l2_out[b], TC_WAIT_NS);
      drain(&mbar2[b], pm2[b], m2_out[b], TC_WAIT_NS);
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue: D2 -> Y (FP64) or the partial tile
  double* Y = yv + (long long)vec * ys + G.yoff;
  {
    const int warp = tid >> 5, row = ((warp & 3) << 5) | (tid & 31), wg = warp >> 2;
    for (int j0 = 8 * wg; j0 < rp; j0 += 16) {
      uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      // warp-collective load: the condition must be uniform over the CTA (d2 is
      // thread 0's own bookkeeping; a tile with chunks always issued GEMM2)
      if (has_work && !bad) {
        const uint32_t addr = tD2 + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)j0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tbase));
}

// ---------------------------------------------------------------------------
// the same product, warp-specialised and persistent
//
// One CTA per SM walks its share of the tile pieces (static stride over the
// costliest-first list).  The steps (chunk c, X rows m0..m0+TC_MC-1) of all
// its pieces form one stream that three roles pipeline through mbarriers:
//   warp 0 (one lane)  copies: GEMM1 operand chunks into a ring of WS_S1
//                      slots, the L slices of GEMM2 into a ring of WS_S2 slots;
//   warp 1 (one lane)  MMAs: GEMM1 of step s into TMEM buffer D1[s & 1], then
//                      GEMM2 of step s-1 into D2[piece & 1];
//   warps 2-5          the T pass of step s (D1 -> B2[s & 1], scaled and
//                      re-split) while GEMM1 of step s+1 runs, and the
//                      epilogue of a piece (D2 -> Y) while the next piece's
//                      first steps run.
// The L ring holds every slice of one step (pc * K chunks <= WS_S2), so the
// copy role never waits on a slot that only a later step's MMAs free.  Every
// wait is bounded; after a timeout every role stops, the copy and MMA roles
// wait (with the full bound) for their own copies and MMAs, and the CTA
// releases its tensor memory before it exits.
// ---------------------------------------------------------------------------
constexpr int WS_NT = 192;
constexpr int WS_S1 = 3;

template <int TF32>
struct WsSmem {
  static constexpr int NS = TF32 ? 1 : 2;
  static constexpr int ES = TF32 ? 4 : 2;
  static constexpr int S2 = TF32 ? 16 : 8;                  // pc (<= 8) x K chunks of GEMM2 per step
  static constexpr int A1 = TC_M * CH_BYTES, B1 = TC_MC * CH_BYTES;
  static constexpr int G1 = NS * (A1 + B1);                 // one GEMM1 slot (all planes)
  static constexpr int CB2 = TC_M * CH_BYTES;
  static constexpr int B2 = TC_MC * ES / CH_BYTES * CB2;    // one plane of one T buffer
  static constexpr int A2 = TC_M * CH_BYTES;
  static constexpr int off_b2 = WS_S1 * G1;
  static constexpr int off_l = off_b2 + 2 * NS * B2;
  static constexpr int total = off_l + S2 * NS * A2;
};

__device__ __forceinline__ void bar_init_n(uint64_t* bar, int n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(n));
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int TF32>
__global__ void __launch_bounds__(WS_NT, 1)
    k_tasks_tc_ws(const TcTask* __restrict__ tasks, const Group* __restrict__ groups, const TcTile* __restrict__ tiles,
                  const int* __restrict__ order, const int* __restrict__ order_off,
                  const TcChunk* __restrict__ chunks, const unsigned char* __restrict__ ops_hi,
                  const unsigned char* __restrict__ ops_lo, const unsigned char* __restrict__ x_hi,
                  const unsigned char* __restrict__ x_lo, long long x_bytes, const XBlock* __restrict__ xblocks,
                  double* yv, long long ys, int* flag, double* part_all, long long psize, int nv,
                  unsigned long long wait_ns) {
  using S = WsSmem<TF32>;
  constexpr int ES = S::ES, NS = S::NS;
  constexpr int NPROD = TF32 ? 1 : 3;
  constexpr int EPC = CH_BYTES / ES;
  constexpr uint32_t SBO_FULL = (CH_BYTES / 16) * 128;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full1[WS_S1], empty1[WS_S1], full2[S::S2], empty2[S::S2];
  __shared__ uint64_t d1_full[2], d1_empty[2], b2_full[2], b2_empty[2], d2_full[2], d2_empty[2], drain_bar;
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this CTA's items: its pieces (balanced on the host by estimated cost) x vectors
  const int it0 = order_off[blockIdx.x] * nv, it1 = order_off[blockIdx.x + 1] * nv;
  auto item_tile = [&](int w) { return tiles[order[w / nv]]; };

  if (tid == 0) {
    for (int i = 0; i < WS_S1; ++i) {
      bar_init_n(&full1[i], 1);
      bar_init_n(&empty1[i], 1);
    }
    for (int i = 0; i < S::S2; ++i) {
      bar_init_n(&full2[i], 1);
      bar_init_n(&empty2[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      bar_init_n(&d1_full[i], 1);
      bar_init_n(&d1_empty[i], 128);
      bar_init_n(&b2_full[i], 128);
      bar_init_n(&b2_empty[i], 1);
      bar_init_n(&d2_full[i], 1);
      bar_init_n(&d2_empty[i], 128);
    }
    bar_init_n(&drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tbase)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tD1[2] = {tbase, tbase + 32}, tD2[2] = {tbase + 64, tbase + 128};

  // bounded wait on phase parity ph; on timeout the first role to give up
  // records where and every role stops at its next wait
  auto wait = [&](uint64_t* bar, uint32_t ph, int where, unsigned long long bound) -> bool {
    if (abort_flag) return false;
    if (wait_bar(bar, ph, bound)) return true;
    if (atomicCAS(flag, 0, 1) == 0) {
      flag[1] = blockIdx.x;
      flag[2] = where;
      flag[3] = warp;
    }
    abort_flag = 1;
    return false;
  };

  if (warp == 0) {
    // ------------------------------ copies ------------------------------
    if (lane == 0) {
      long long i1 = 0, i2 = 0;  // running slot counters of the two rings
      int armed1[WS_S1], armed2[S::S2];
      for (int i = 0; i < WS_S1; ++i) armed1[i] = 0;
      for (int i = 0; i < S::S2; ++i) armed2[i] = 0;
      bool go = true;
      for (int w = it0; w < it1 && go; ++w) {
        const TcTile TL = item_tile(w);
        const int vec = w % nv;
        const unsigned char* xh = x_hi + (long long)vec * x_bytes;
        const unsigned char* xl = TF32 ? nullptr : x_lo + (long long)vec * x_bytes;
        const int rp = (TL.ncols + 15) & ~15;
        for (int c = TL.c0; c < TL.c1 && go; ++c) {
          const TcChunk C = chunks[c];
          const int pc = C.t1 - C.t0;
          const XBlock XB = xblocks[C.xb];
          // the operand images of the chunk's products, loaded together
          Img Rs[TC_M / 16], Ls[TC_M / 16];
#pragma unroll
          for (int t = 0; t < TC_M / 16; ++t)
            if (t < pc) {
              Rs[t] = tasks[C.t0 + t].R;
              Ls[t] = tasks[C.t0 + t].L;
            }
          const int nch = (XB.img.kb + CH_BYTES - 1) / CH_BYTES;
          for (int m0 = 0; m0 < XB.m && go; m0 += TC_MC) {
            const int mc16 = (min(TC_MC, XB.m - m0) + 15) & ~15;
            const int xg0 = m0 / 8, xng = min(mc16 / 8, XB.img.rg - xg0);
            for (int kc = 0; kc < nch; ++kc, ++i1) {
              const int sl = (int)(i1 % WS_S1);
              if (!wait(&empty1[sl], (uint32_t)(((i1 / WS_S1) & 1) ^ 1), 1, wait_ns)) {
                go = false;
                break;
              }
              unsigned char* a = smem + sl * S::G1;
              unsigned char* b = a + NS * S::A1;
              const uint32_t rowb = (chunk_w(XB.img, kc) / 16) * 128;
              uint32_t bytes = (xng > 0 ? xng * rowb : 0) * NS;
#pragma unroll
              for (int t = 0; t < TC_M / 16; ++t)
                if (t < pc) {
                  const int ng = min(rp / 8, Rs[t].rg - TL.col0 / 8);
                  if (ng > 0) bytes += ng * rowb * NS;
                }
              expect_tx(&full1[sl], bytes);
              armed1[sl] = (int)(i1 / WS_S1) + 1;
              if (xng > 0) {
                const long long xo = chunk_off(XB.img, kc) + (long long)xg0 * rowb;
                bulk_g2s(b, xh + xo, xng * rowb, &full1[sl]);
                if (!TF32) bulk_g2s(b + S::B1, xl + xo, xng * rowb, &full1[sl]);
              }
#pragma unroll
              for (int t = 0; t < TC_M / 16; ++t) {
                if (t >= pc) continue;
                const Img R = Rs[t];
                const int ng = min(rp / 8, R.rg - TL.col0 / 8);
                if (ng <= 0) continue;
                const long long ro = chunk_off(R, kc) + (long long)(TL.col0 / 8) * rowb;
                const uint32_t dst = (uint32_t)(t * rp / 8) * rowb;
                bulk_g2s(a + dst, ops_hi + ro, ng * rowb, &full1[sl]);
                if (!TF32) bulk_g2s(a + S::A1 + dst, ops_lo + ro, ng * rowb, &full1[sl]);
              }
            }
            if (!go) break;
            const int nch2 = (mc16 * ES + CH_BYTES - 1) / CH_BYTES;
#pragma unroll
            for (int t = 0; t < TC_M / 16; ++t) {
              if (t >= pc || !go) continue;
              const Img Lm = Ls[t];
              const int lg0 = TL.row0 / 8, lng = min(TC_M / 8, Lm.rg - lg0);
              for (int c2 = 0; c2 < nch2; ++c2, ++i2) {
                const int sl = (int)(i2 % S::S2);
                if (!wait(&empty2[sl], (uint32_t)(((i2 / S::S2) & 1) ^ 1), 2, wait_ns)) {
                  go = false;
                  break;
                }
                const int lc = (m0 * ES) / CH_BYTES + c2;
                const uint32_t rowb = (chunk_w(Lm, lc) / 16) * 128;
                unsigned char* a2 = smem + S::off_l + sl * NS * S::A2;
                expect_tx(&full2[sl], lng * rowb * NS);
                armed2[sl] = (int)(i2 / S::S2) + 1;
                const long long lo_ = chunk_off(Lm, lc) + (long long)lg0 * rowb;
                bulk_g2s(a2, ops_hi + lo_, lng * rowb, &full2[sl]);
                if (!TF32) bulk_g2s(a2 + S::A2, ops_lo + lo_, lng * rowb, &full2[sl]);
              }
            }
          }
        }
      }
      // every copy issued by this role has landed (the last arm of a slot
      // completing implies the earlier ones did) before the CTA can exit
      for (int i = 0; i < WS_S1; ++i)
        if (armed1[i]) wait_bar(&full1[i], (uint32_t)((armed1[i] - 1) & 1), TC_WAIT_NS);
      for (int i = 0; i < S::S2; ++i)
        if (armed2[i]) wait_bar(&full2[i], (uint32_t)((armed2[i] - 1) & 1), TC_WAIT_NS);
    }
  } else if (warp == 1) {
    // ------------------------------- MMAs -------------------------------
    if (lane == 0) {
      long long i1 = 0, i2 = 0, s = 0;
      int piece = 0;  // pieces with work of this CTA so far (D2 buffer and its phase)
      bool go = true;
      // the GEMM2 of the previous step, issued after the GEMM1 of the current one
      struct Prev {
        bool valid;
        int c, m0, mc16, rp, first, last, piece;
        long long s;
      } prev = {false, 0, 0, 0, 0, 0, 0, 0, 0};
      auto gemm2 = [&](const Prev& P) -> bool {
        const TcChunk C = chunks[P.c];
        const int pc = C.t1 - C.t0;
        const int bb = (int)(P.s & 1);
        if (!wait(&b2_full[bb], (uint32_t)((P.s >> 1) & 1), 3, wait_ns)) return false;
        if (P.first && !wait(&d2_empty[P.piece & 1], (uint32_t)(((P.piece >> 1) & 1) ^ 1), 4, wait_ns)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int nch2 = (P.mc16 * ES + CH_BYTES - 1) / CH_BYTES;
        const int nk2 = P.mc16 * ES / 32;
        const uint32_t id = idesc(TF32 ? 2 : 1, P.rp);
        const unsigned char* b2 = smem + S::off_b2 + bb * NS * S::B2;
        bool acc_any = !P.first;
        Img Ls[TC_M / 16];
#pragma unroll
        for (int t = 0; t < TC_M / 16; ++t)
          if (t < pc) Ls[t] = tasks[C.t0 + t].L;
#pragma unroll
        for (int t = 0; t < TC_M / 16; ++t) {
          if (t >= pc) continue;
          for (int c2 = 0; c2 < nch2; ++c2, ++i2) {
            const int sl = (int)(i2 % S::S2);
            if (!wait(&full2[sl], (uint32_t)((i2 / S::S2) & 1), 5, wait_ns)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const Img Lm = Ls[t];
            const int lc = (P.m0 * ES) / CH_BYTES + c2;
            const int kcm = chunk_w(Lm, lc) / 16;
            const uint32_t rowb = kcm * 128;
            const unsigned char* a2 = smem + S::off_l + sl * NS * S::A2;
            const uint32_t bt = (uint32_t)(t * P.rp / 8) * SBO_FULL;
            const int ks_here = min(kcm / 2, nk2 - c2 * (CH_BYTES / 32));
            for (int ks = 0; ks < ks_here; ++ks)
              for (int pr = 0; pr < NPROD; ++pr) {
                const unsigned char* a = a2 + (pr == 2 ? S::A2 : 0);
                const unsigned char* bbp = b2 + (pr == 1 ? S::B2 : 0) + c2 * S::CB2 + bt;
                mma<TF32>(tD2[P.piece & 1], sdesc(smem_u32(a) + ks * 256, rowb),
                          sdesc(smem_u32(bbp) + ks * 256, SBO_FULL), id, acc_any ? 1u : 0u);
                acc_any = true;
              }
            commit(&empty2[sl]);
          }
        }
        commit(&b2_empty[bb]);
        if (P.last) commit(&d2_full[P.piece & 1]);
        return true;
      };
      for (int w = it0; w < it1 && go; ++w) {
        const TcTile TL = item_tile(w);
        const int rp = (TL.ncols + 15) & ~15;
        if (TL.c1 <= TL.c0) continue;
        for (int c = TL.c0; c < TL.c1 && go; ++c) {
          const TcChunk C = chunks[c];
          const XBlock XB = xblocks[C.xb];
          const int nch = (XB.img.kb + CH_BYTES - 1) / CH_BYTES;
          for (int m0 = 0; m0 < XB.m && go; m0 += TC_MC, ++s) {
            const int mc16 = (min(TC_MC, XB.m - m0) + 15) & ~15;
            // GEMM1 of step s into D1[s & 1] (free once the T pass of s-2 read it)
            const int db = (int)(s & 1);
            if (!wait(&d1_empty[db], (uint32_t)(((s >> 1) & 1) ^ 1), 6, wait_ns)) {
              go = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t id = idesc(TF32 ? 2 : 1, mc16);
            for (int kc = 0; kc < nch; ++kc, ++i1) {
              const int sl = (int)(i1 % WS_S1);
              if (!wait(&full1[sl], (uint32_t)((i1 / WS_S1) & 1), 7, wait_ns)) {
                go = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
              const unsigned char* a = smem + sl * S::G1;
              const unsigned char* b = a + NS * S::A1;
              const int kcm = chunk_w(XB.img, kc) / 16;
              const uint32_t rowb = kcm * 128;
              for (int ks = 0; ks < kcm / 2; ++ks)
                for (int pr = 0; pr < NPROD; ++pr) {
                  const unsigned char* aa = a + (pr == 2 ? S::A1 : 0);
                  const unsigned char* bbp = b + (pr == 1 ? S::B1 : 0);
                  const uint32_t acc = (kc > 0 || ks > 0 || pr > 0) ? 1u : 0u;
                  mma<TF32>(tD1[db], sdesc(smem_u32(aa) + ks * 256, rowb), sdesc(smem_u32(bbp) + ks * 256, rowb),
                            id, acc);
                }
              commit(&empty1[sl]);
            }
            if (!go) break;
            commit(&d1_full[db]);
            // GEMM2 of the previous step
            if (prev.valid && !gemm2(prev)) {
              go = false;
              break;
            }
            prev.valid = true;
            prev.c = c;
            prev.m0 = m0;
            prev.mc16 = mc16;
            prev.rp = rp;
            prev.first = (c == TL.c0 && m0 == 0) ? 1 : 0;
            prev.last = (c == TL.c1 - 1 && m0 + TC_MC >= XB.m) ? 1 : 0;
            prev.piece = piece;
            prev.s = s;
          }
        }
        ++piece;
      }
      if (go && prev.valid) gemm2(prev);
      // every MMA of this role completed before the CTA can exit
      commit(&drain_bar);
      wait_bar(&drain_bar, 0, TC_WAIT_NS);
    }
  } else {
    // ------------------------ T pass and epilogue ------------------------
    const int q = warp & 3;               // TMEM lane quadrant of this warp
    const int row = q * 32 + lane;        // TMEM lane = stacked R row (T pass) = tile row (epilogue)
    // the warp-collective TMEM loads below need the whole warp: a wait that
    // gives up on any lane stops all of them
    auto wait_w = [&](uint64_t* bar, uint32_t ph, int where) -> bool {
      const bool ok = __all_sync(0xffffffffu, wait(bar, ph, where, wait_ns) ? 1 : 0);
      if (!ok) abort_flag = 1;
      return ok;
    };
    long long s = 0;
    int piece = 0;  // pieces with work so far (as counted by the MMA role)
    bool go = true;
    for (int w = it0; w < it1 && go; ++w) {
      const TcTile TL = item_tile(w);
      const Group G = groups[TL.g];
      const int vec = w % nv;
      const int rp = (TL.ncols + 15) & ~15;
      const bool has_work = TL.c1 > TL.c0;
      for (int c = TL.c0; c < TL.c1 && go; ++c) {
        const TcChunk C = chunks[c];
        const int pc = C.t1 - C.t0;
        const XBlock XB = xblocks[C.xb];
        const int t = row / rp;
        const float al = t < pc ? tasks[C.t0 + t].alpha : 0.f;
        for (int m0 = 0; m0 < XB.m && go; m0 += TC_MC, ++s) {
          const int mc = min(TC_MC, XB.m - m0), mc16 = (mc + 15) & ~15;
          const int db = (int)(s & 1);
          if (!wait_w(&d1_full[db], (uint32_t)((s >> 1) & 1), 8)) {
            go = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          uint32_t r[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = 0u;
#pragma unroll
          for (int i0 = 0; i0 < 32; i0 += 8) {
            if (i0 < mc16) {
              const uint32_t addr = tD1[db] + ((uint32_t)(q * 32) << 16) + (uint32_t)i0;
              asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                           : "=r"(r[i0]), "=r"(r[i0 + 1]), "=r"(r[i0 + 2]), "=r"(r[i0 + 3]), "=r"(r[i0 + 4]),
                             "=r"(r[i0 + 5]), "=r"(r[i0 + 6]), "=r"(r[i0 + 7])
                           : "r"(addr));
            }
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          asm volatile("tcgen05.fence::before_thread_sync;");
          bar_arrive(&d1_empty[db]);
          if (!wait_w(&b2_empty[db], (uint32_t)(((s >> 1) & 1) ^ 1), 9)) {
            go = false;
            break;
          }
          unsigned char* b2 = smem + S::off_b2 + db * NS * S::B2;
#pragma unroll
          for (int i0 = 0; i0 < 32; i0 += 8) {
            if (i0 >= mc16) continue;
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = (t < pc && i0 + e < mc) ? al * __uint_as_float(r[i0 + e]) : 0.f;
            if (TF32) {
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const int i = i0 + 4 * hh;
                const int off = (i / EPC) * S::CB2 + ((row >> 3) * (CH_BYTES / 16) + (i % EPC) * ES / 16) * 128 +
                                (row & 7) * 16;
                uint32_t qq[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(qq[e]) : "f"(v[4 * hh + e]));
                *(uint4*)(b2 + off) = make_uint4(qq[0], qq[1], qq[2], qq[3]);
              }
            } else {
              const int off = (i0 / EPC) * S::CB2 + ((row >> 3) * (CH_BYTES / 16) + (i0 % EPC) * ES / 16) * 128 +
                              (row & 7) * 16;
              __align__(16) __nv_bfloat16 hh[8], ll[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                hh[e] = __float2bfloat16_rn(v[e]);
                ll[e] = __float2bfloat16_rn(v[e] - __bfloat162float(hh[e]));
              }
              *(uint4*)(b2 + off) = *(const uint4*)hh;
              *(uint4*)(b2 + S::B2 + off) = *(const uint4*)ll;
            }
          }
          asm volatile("fence.proxy.async.shared::cta;");
          bar_arrive(&b2_full[db]);
        }
      }
      if (!go) break;
      // epilogue of the piece: D2 -> Y (or its partial tile)
      double* Y = yv + (long long)vec * ys + G.yoff;
      double* part = TL.poff >= 0 ? part_all + (long long)vec * psize + TL.poff : nullptr;
      const int pb = piece & 1;
      if (has_work) {
        if (!wait_w(&d2_full[pb], (uint32_t)((piece >> 1) & 1), 10)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
      for (int j0 = 0; j0 < rp; j0 += 8) {
        uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (has_work) {
          const uint32_t addr = tD2[pb] + ((uint32_t)(q * 32) << 16) + (uint32_t)j0;
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                         "=r"(r[7])
                       : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
        }
        if (row < TL.nrows)
          for (int e = 0; e < 8; ++e)
            if (j0 + e < TL.ncols) {
              const double val = (double)__uint_as_float(r[e]);
              if (part)
                part[row * TL.ncols + j0 + e] = val;
              else
                Y[(long long)(TL.row0 + row) * G.r + TL.col0 + j0 + e] = val;
            }
      }
      if (has_work) {
        asm volatile("tcgen05.fence::before_thread_sync;");
        bar_arrive(&d2_empty[pb]);
        ++piece;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase));
}

#include "tc_small.inc"

// ---------------------------------------------------------------------------
// host planning
// ---------------------------------------------------------------------------
Img make_img(int rows, int cols, int es, long long& arena) {
  Img g;
  g.off = arena;
  g.rg = (rows + 7) / 8;
  g.kb = ((cols * es + 31) / 32) * 32;
  arena += img_bytes(g);
  return g;
}

// products of a group ordered by X block; tiles of 128 rows x 64 columns;
// chunks of products sharing X with (products x padded tile columns) <= 128.
// A group whose block and X blocks all have dimensions <= small is one tile
// of the small-block warp kernel instead (its chunks only delimit pieces).
// operand image key: (source block, stored transposed, rows, cols of op(M))
struct ImgKey {
  const double* src;
  int trans, rows, cols;
  bool operator==(const ImgKey& o) const {
    return src == o.src && trans == o.trans && rows == o.rows && cols == o.cols;
  }
};
struct ImgKeyHash {
  size_t operator()(const ImgKey& k) const {
    unsigned long long h = (unsigned long long)(uintptr_t)k.src * 0x9E3779B97F4A7C15ull;
    h ^= ((unsigned long long)k.trans << 62) ^ ((unsigned long long)(unsigned)k.rows << 32) ^ (unsigned)k.cols;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    return (size_t)(h ^ (h >> 32));
  }
};

// stable sort of (X offset, product) pairs by X offset: least-significant-digit
// radix sort, 8 bits per pass over the bits the largest offset uses (a
// group's products number thousands, its X offsets fit in ~20 bits)
void stable_sort_by_x(std::vector<std::pair<size_t, int>>& v, std::vector<std::pair<size_t, int>>& tmp) {
  const size_t n = v.size();
  if (n < 64) {
    std::stable_sort(v.begin(), v.end(),
                     [](const std::pair<size_t, int>& a, const std::pair<size_t, int>& b) { return a.first < b.first; });
    return;
  }
  size_t mx = 0;
  for (const auto& e : v) mx = std::max(mx, e.first);
  tmp.resize(n);
  for (int shift = 0; shift < 64 && (mx >> shift) != 0; shift += 8) {
    size_t cnt[257] = {};
    for (const auto& e : v) ++cnt[((e.first >> shift) & 255) + 1];
    for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
    for (const auto& e : v) tmp[cnt[(e.first >> shift) & 255]++] = e;
    v.swap(tmp);
  }
}

void build_plan(const TaskList& tl, int es, int small, TcPlan& P, std::vector<ImgJob>& jobs,
                std::vector<XBlock>& xbs) {
  // hashed lookups (two per product) with a one-entry memo per operand:
  // products of a group come X-ordered and often repeat an operator block;
  // images and X blocks get their offsets in first-use order
  std::unordered_map<ImgKey, Img, ImgKeyHash> imgs;
  std::unordered_map<long long, int> xidx;
  imgs.reserve(1 << 16);
  xidx.reserve(1 << 12);
  long long arena = 0, xarena = 0;
  ImgKey lastk[2] = {{nullptr, -1, -1, -1}, {nullptr, -1, -1, -1}};
  Img lastg[2] = {};
  auto image = [&](int side, const double* src, int trans, int rows, int cols) {
    const ImgKey key{src, trans, rows, cols};
    if (key == lastk[side]) return lastg[side];
    auto it = imgs.find(key);
    Img g;
    if (it != imgs.end()) {
      g = it->second;
    } else {
      g = make_img(rows, cols, es, arena);
      imgs.emplace(key, g);
      jobs.push_back({src, rows, cols, trans, g});
    }
    lastk[side] = key;
    lastg[side] = g;
    return g;
  };
  P.tasks_h.clear();
  P.tiles_h.clear();
  P.wtiles_h[0].clear();
  P.wtiles_h[1].clear();
  P.chunks_h.clear();
  P.tasks_h.reserve(tl.tasks.size());
  std::vector<std::pair<size_t, int>> idx, tmp;  // (X offset, product): sorted by X, stable
  long long last_xo = -1;
  int last_xb = -1;
  for (int g = 0; g < (int)tl.groups.size(); ++g) {
    const Group& G = tl.groups[g];
    idx.clear();
    for (int t = G.t0; t < G.t1; ++t) idx.push_back({(size_t)tl.tasks[t].X, t});
    stable_sort_by_x(idx, tmp);
    const int base = (int)P.tasks_h.size();
    for (const auto& e : idx) {
      const Task& k = tl.tasks[e.second];
      TcTask c;
      c.alpha = (float)k.alpha;
      c.m = k.m;
      c.n = k.n;
      // op(L): q x m ; op(R): r x n ; identities become identity images
      c.L = (k.flags & TF_LI) ? image(0, nullptr, 0, k.q, k.m) : image(0, k.L, (k.flags & TF_LT) ? 1 : 0, k.q, k.m);
      c.R = (k.flags & TF_RI) ? image(1, nullptr, 0, k.r, k.n) : image(1, k.R, (k.flags & TF_RT) ? 1 : 0, k.r, k.n);
      const long long xo = (long long)(size_t)k.X;
      if (xo != last_xo) {
        auto it = xidx.find(xo);
        if (it == xidx.end()) {
          XBlock B;
          B.src = xo;
          B.m = k.m;
          B.n = k.n;
          B.img = make_img(k.m, k.n, es, xarena);
          xidx.emplace(xo, (int)xbs.size());
          xbs.push_back(B);
          last_xb = (int)xbs.size() - 1;
        } else {
          last_xb = it->second;
        }
        last_xo = xo;
      }
      c.xb = last_xb;
      P.tasks_h.push_back(c);
    }
    const int nt = (int)idx.size();
    int dmax = std::max(G.q, G.r);
    for (int i = 0; i < nt; ++i) dmax = std::max(dmax, std::max(P.tasks_h[base + i].m, P.tasks_h[base + i].n));
    if (small > 0 && dmax <= small && dmax <= SW_MAXD) {
      TcTile T;
      T.g = g;
      T.row0 = T.col0 = 0;
      T.nrows = G.q;
      T.ncols = G.r;
      T.c0 = (int)P.chunks_h.size();
      int i = 0;
      while (i < nt) {
        const TcTask& a = P.tasks_h[base + i];
        int j = i + 1;
        while (j < nt && j - i < 8 && P.tasks_h[base + j].xb == a.xb) ++j;
        P.chunks_h.push_back({base + i, base + j, a.xb, 0});
        i = j;
      }
      T.c1 = (int)P.chunks_h.size();
      T.poff = -1;
      P.wtiles_h[dmax <= 16 ? 0 : 1].push_back(T);
      continue;
    }
    for (int r0 = 0; r0 < G.q; r0 += TC_M)
      for (int c0 = 0; c0 < G.r; c0 += TC_NC) {
        TcTile T;
        T.g = g;
        T.row0 = r0;
        T.col0 = c0;
        T.nrows = std::min(TC_M, G.q - r0);
        T.ncols = std::min(TC_NC, G.r - c0);
        T.c0 = (int)P.chunks_h.size();
        const int rp = (T.ncols + 15) & ~15;
        const int cap = std::max(1, TC_M / rp);
        int i = 0;
        while (i < nt) {
          const TcTask& a = P.tasks_h[base + i];
          int j = i + 1;
          while (j < nt && j - i < cap && P.tasks_h[base + j].xb == a.xb) ++j;
          P.chunks_h.push_back({base + i, base + j, a.xb, 0});
          i = j;
        }
        T.c1 = (int)P.chunks_h.size();
        T.poff = -1;
        P.tiles_h.push_back(T);
      }
  }
  P.ops_bytes = arena;
  P.x_bytes = xarena;
}

// cut tiles whose chunk lists are long into pieces of similar cost (each piece
// accumulates its own TMEM tile and writes a partial tile; the pieces are
// summed in order afterwards), so the CTAs of one launch finish together
// estimated cost of one chunk of a tile piece (MMA work with padding, plus a
// fixed cost for its copies, T pass and barriers)
double chunk_cost(const std::vector<TcTask>& tasks, const TcChunk& C, const TcTile& T) {
  double s = 1.5e4;
  const TcTask& a = tasks[C.t0];
  const int p = C.t1 - C.t0;
  const int rp = (T.ncols + 15) & ~15;
  const double mm = ((a.m + 15) / 16) * 16.0, nn = ((a.n + 15) / 16) * 16.0;
  s += 2.0 * TC_M * mm * nn + p * 2.0 * TC_M * mm * rp;
  return s;
}

// pieces of the persistent kernel per CTA: longest first onto the least
// loaded of `ctas` CTAs (the kernel walks each CTA's list in order)
void ws_assign(const std::vector<TcTask>& tasks, const std::vector<TcTile>& tiles, const std::vector<TcChunk>& chunks,
               int ctas, std::vector<int>& order, std::vector<int>& off) {
  const int n = (int)tiles.size();
  std::vector<double> cost(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int c = tiles[i].c0; c < tiles[i].c1; ++c) cost[i] += chunk_cost(tasks, chunks[c], tiles[i]);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> per(ctas);
  std::vector<std::pair<double, int>> heap;  // (load, cta), min-heap
  for (int b = 0; b < ctas; ++b) heap.push_back({0.0, b});
  auto cmp = [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first > y.first || (x.first == y.first && x.second > y.second);
  };
  std::make_heap(heap.begin(), heap.end(), cmp);
  for (int i : idx) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    auto& h = heap.back();
    per[h.second].push_back(i);
    h.first += cost[i];
    std::push_heap(heap.begin(), heap.end(), cmp);
  }
  order.clear();
  off.assign(1, 0);
  for (int b = 0; b < ctas; ++b) {
    for (int i : per[b]) order.push_back(i);
    off.push_back((int)order.size());
  }
}

// estimated cost of one chunk of the small-block warp kernel: its MMAs and a
// fixed cost per product (metadata, copies, waits)
double sw_chunk_cost(const std::vector<TcTask>& tasks, const TcChunk& C, const TcTile& T, int es) {
  const int nprod = es == 2 ? 3 : 1;
  const int MT = (T.ncols + 15) / 16, QT = (T.nrows + 7) / 8;
  double s = 0.0;
  for (int t = C.t0; t < C.t1; ++t) {
    const TcTask& k = tasks[t];
    const int NT1 = (k.m + 7) / 8, K1 = k.R.kb / 32, K2 = es == 2 ? (k.m + 15) / 16 : NT1;
    s += 120.0 + 8.0 * nprod * (MT * NT1 * K1 + MT * QT * K2);
  }
  return s;
}

// the estimated cost of every chunk, once per plan (chunks belong to one tile each)
void plan_chunk_costs(TcPlan& P, int es) {
  P.ccost_h.assign(P.chunks_h.size(), 0.0);
  for (const TcTile& T : P.tiles_h)
    for (int c = T.c0; c < T.c1; ++c) P.ccost_h[c] = chunk_cost(P.tasks_h, P.chunks_h[c], T);
  for (int w = 0; w < 2; ++w)
    for (const TcTile& T : P.wtiles_h[w])
      for (int c = T.c0; c < T.c1; ++c) P.ccost_h[c] = sw_chunk_cost(P.tasks_h, P.chunks_h[c], T, es);
}

// cut tiles into pieces of similar estimated cost: the split target is the
// total cost over (resident units x rounds); pieces costliest first
template <class Cost>
void split_plan(std::vector<TcTile>& tiles, const std::vector<TcChunk>& chunks, std::vector<SplitRed>& reds,
                long long& psize, double units, double rounds, Cost ccost) {
  std::vector<double> tcost(tiles.size(), 0.0);
  double tot = 0;
  for (size_t i = 0; i < tiles.size(); ++i) {
    for (int c = tiles[i].c0; c < tiles[i].c1; ++c) tcost[i] += ccost(chunks[c], tiles[i]);
    tot += tcost[i];
  }
  const double target = std::max(tot / (units * rounds), 1.0);
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
      acc += ccost(chunks[c], T);
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
  // costliest pieces first: CTAs are dispatched in index order, so the long
  // pieces start in the first wave and the short ones fill in behind them
  {
    std::vector<double> pc(out.size(), 0.0);
    for (size_t i = 0; i < out.size(); ++i)
      for (int c = out[i].c0; c < out[i].c1; ++c) pc[i] += ccost(chunks[c], out[i]);
    std::vector<int> ord(out.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return pc[a] > pc[b]; });
    std::vector<TcTile> sorted(out.size());
    for (size_t i = 0; i < ord.size(); ++i) sorted[i] = out[ord[i]];
    out.swap(sorted);
  }
  tiles.swap(out);
}

// Walk every tile piece the way k_tasks_tc does and check each bulk copy and
// operand range against its image and its shared-memory region; a plan that
// fails is never launched.
bool check_plan(const TcPlan& P, const std::vector<TcTile>& tiles, const std::vector<XBlock>& xbs, int es,
                std::string& why) {
  const int ns = es == 2 ? 2 : 1;
  const long long A1 = TC_M * CH_BYTES, B1 = TC_MC * CH_BYTES, CB2 = TC_M * CH_BYTES;
  const long long B2 = (long long)TC_MC * es / CH_BYTES * CB2, A2 = TC_M * CH_BYTES;
  auto inside = [&](const Img& g, long long off, long long bytes, long long arena) {
    return off >= g.off && bytes >= 0 && off + bytes <= g.off + img_bytes(g) && g.off + img_bytes(g) <= arena &&
           off % 16 == 0 && bytes % 16 == 0;
  };
  for (const TcTile& T : tiles) {
    const int rp = (T.ncols + 15) & ~15;
    if (T.col0 % 64 || T.row0 % TC_M || rp > TC_NC) {
      why = "tile shape";
      return false;
    }
    for (int c = T.c0; c < T.c1; ++c) {
      const TcChunk& C = P.chunks_h[c];
      const int pc = C.t1 - C.t0;
      if (pc < 1 || pc * rp > TC_M || pc > TC_M / 16) {
        why = "chunk capacity";
        return false;
      }
      const TcTask& t0 = P.tasks_h[C.t0];
      if (C.xb != t0.xb) {
        why = "chunk X block";
        return false;
      }
      const XBlock& XB = xbs[t0.xb];
      for (int t = C.t0; t < C.t1; ++t) {
        const TcTask& k = P.tasks_h[t];
        if (k.xb != t0.xb || k.m != XB.m || k.n != XB.n || k.R.kb != XB.img.kb ||
            k.L.kb != ((XB.m * es + 31) / 32) * 32 || k.R.rg * 8 < T.col0 + 1 || k.L.rg * 8 < T.row0 + 1) {
          why = "operand shapes";
          return false;
        }
      }
      for (int m0 = 0; m0 < XB.m; m0 += TC_MC) {
        const int mc = std::min(TC_MC, XB.m - m0), mc16 = (mc + 15) & ~15;
        const int nch = (XB.img.kb + CH_BYTES - 1) / CH_BYTES;
        const int xg0 = m0 / 8, xng = std::min(mc16 / 8, XB.img.rg - xg0);
        for (int kc = 0; kc < nch; ++kc) {
          const int w = chunk_w(XB.img, kc);
          if (w <= 0 || w % 32) {
            why = "chunk width";
            return false;
          }
          const long long rowb = (w / 16) * 128;
          if (xng > 0 && (!inside(XB.img, chunk_off(XB.img, kc) + xg0 * rowb, xng * rowb, P.x_bytes) ||
                          xng * rowb > B1)) {
            why = "input image copy";
            return false;
          }
          for (int t = C.t0; t < C.t1; ++t) {
            const Img& R = P.tasks_h[t].R;
            const int ng = std::min(rp / 8, R.rg - T.col0 / 8);
            const long long dst = (long long)((t - C.t0) * rp / 8) * rowb;
            if (ng > 0 && (chunk_w(R, kc) != w || !inside(R, chunk_off(R, kc) + (T.col0 / 8) * rowb, ng * rowb,
                                                          P.ops_bytes) ||
                           dst + ng * rowb > A1)) {
              why = "operator image copy (GEMM1)";
              return false;
            }
          }
          if (16 * rowb > A1 || (mc16 / 8) * rowb > B1) {
            why = "GEMM1 operand extent";
            return false;
          }
        }
        const int nk2 = mc16 * es / 32, nch2 = (mc16 * es + CH_BYTES - 1) / CH_BYTES;
        if ((long long)nch2 * CB2 > B2) {
          why = "T pass extent";
          return false;
        }
        for (int t = C.t0; t < C.t1; ++t) {
          const Img& Lm = P.tasks_h[t].L;
          const int lg0 = T.row0 / 8, lng = std::min(TC_M / 8, Lm.rg - lg0);
          for (int c2 = 0; c2 < nch2; ++c2) {
            const int lc = (m0 * es) / CH_BYTES + c2;
            const int w = chunk_w(Lm, lc);
            if (w <= 0 || w % 32) {
              why = "operator chunk";
              return false;
            }
            const long long rowb = (w / 16) * 128;
            const int ks_here = std::min((int)(w / 32), nk2 - c2 * (CH_BYTES / 32));
            if (lng <= 0 || !inside(Lm, chunk_off(Lm, lc) + lg0 * rowb, lng * rowb, P.ops_bytes) ||
                lng * rowb > A2 || ks_here <= 0) {
              why = "operator image copy (GEMM2)";
              return false;
            }
          }
        }
      }
    }
  }
  (void)ns;
  return true;
}

// The small-block warp kernel's assumptions, checked for every product of
// every piece before a launch: whole-block images with the row groups and K
// widths it indexes, a product's images within its ring, an X image within
// one X buffer, all copies inside their arenas and 16-byte aligned.
template <int D>
bool check_small_plan(const TcPlan& P, const std::vector<TcTile>& tiles, const std::vector<XBlock>& xbs,
                      const std::vector<Group>& groups, int es, std::string& why) {
  const int ns = es == 2 ? 2 : 1;
  auto kbw = [&](int cols) { return ((cols * es + 31) / 32) * 32; };
  auto fits = [&](const Img& g, long long arena) {
    return g.off >= 0 && g.off % 16 == 0 && img_bytes(g) % 16 == 0 && g.off + img_bytes(g) <= arena;
  };
  for (const TcTile& T : tiles) {
    const Group& G = groups[T.g];
    if (T.row0 != 0 || T.col0 != 0 || T.nrows != G.q || T.ncols != G.r || G.q > D || G.r > D ||
        G.q < 1 || G.r < 1) {
      why = "small tile shape";
      return false;
    }
    for (int c = T.c0; c < T.c1; ++c) {
      const TcChunk& C = P.chunks_h[c];
      for (int t = C.t0; t < C.t1; ++t) {
        const TcTask& k = P.tasks_h[t];
        if (k.xb < 0 || k.xb >= (int)xbs.size()) {
          why = "small: X block index";
          return false;
        }
        const XBlock& X = xbs[k.xb];
        if (k.m < 1 || k.n < 1 || k.m > D || k.n > D || X.m != k.m || X.n != k.n ||
            X.img.rg != (k.m + 7) / 8 || X.img.kb != kbw(k.n) || k.L.rg != (G.q + 7) / 8 || k.L.kb != kbw(k.m) ||
            k.R.rg != (G.r + 7) / 8 || k.R.kb != kbw(k.n)) {
          why = "small: operand shapes";
          return false;
        }
        if (k.L.off % 256 || k.R.off % 256 || (k.L.off >> 8) > 0xFFFFFFFFll || (k.R.off >> 8) > 0xFFFFFFFFll ||
            k.xb >= (1 << 20)) {
          why = "small: product record fields";
          return false;
        }
        if ((img_bytes(k.L) + img_bytes(k.R)) * ns > SwCfg<D>::RING || img_bytes(X.img) * ns > SwCfg<D>::XBUF) {
          why = "small: staging capacity";
          return false;
        }
        if (!fits(k.L, P.ops_bytes) || !fits(k.R, P.ops_bytes) || !fits(X.img, P.x_bytes)) {
          why = "small: image copy";
          return false;
        }
      }
    }
  }
  return true;
}

template <class T>
T* upload_vec(CudaBackend& be, const std::vector<T>& v, bool& ok) {
  T* p = nullptr;
  if (dmalloc(&p, sizeof(T) * std::max<size_t>(v.size(), 1)) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
    return nullptr;
  }
  if (!v.empty()) cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, be.stream());
  return p;
}

}  // namespace

void launch_reduce_splits(CudaBackend& be, const SplitRed* reds, int nreds, const Group* groups, const double* part,
                          long long psize, double* yv, long long ys, int nvec);

void release_tc_plan(void* p);

bool prepare_tasks_tc(CudaBackend& be, const TaskList& tl, DevList& d, int nvec, int variant, int precision) {
  if (!be.ok()) return false;
  TcPlan* plan = (TcPlan*)d.tc;
  if (plan && (d.tc_gen != tl.gen || plan->precision != precision)) {
    be.free_graphs(d);  // they hold the plan's buffers
    cudaStreamSynchronize(be.stream());
    release_tc_plan(plan);
    d.tc = nullptr;
    plan = nullptr;
  }
  const int es = precision == TNS_TF32 ? 4 : 2;
  if (!plan) {
    for (const Task& t : tl.tasks)
      if (!(t.flags & TF_XV) || (t.flags & (TF_XT | TF_XI))) {
        be.note(cudaErrorInvalidValue, "tensor-core form: work list is not an H_eff*psi list");
        return false;
      }
    plan = new TcPlan();
    plan->precision = precision;
    cudaDeviceGetAttribute(&plan->sms, cudaDevAttrMultiProcessorCount, be.device());
    std::vector<ImgJob> jobs;
    std::vector<XBlock> xbs;
    build_plan(tl, es, be.tc_small, *plan, jobs, xbs);
    plan_chunk_costs(*plan, es);
    if (const char* vp = std::getenv("TNS_VERBOSE_PLAN")) {
      if (*vp && *vp != '0') {
        // products and useful flops by the output block's larger dimension
        // (<= 16, <= 32, larger) and the X block's larger dimension
        double cnt[3][3] = {}, fl[3][3] = {};
        auto cls = [](int d) { return d <= 16 ? 0 : d <= 32 ? 1 : 2; };
        for (const Group& G : tl.groups)
          for (int t = G.t0; t < G.t1; ++t) {
            const Task& k = tl.tasks[t];
            const int a = cls(std::max(G.q, G.r)), b = cls(std::max(k.m, k.n));
            cnt[a][b] += 1;
            fl[a][b] += 2.0 * k.r * k.m * k.n + 2.0 * k.q * k.m * k.r;
          }
        std::fprintf(stderr, "[tns plan] groups %zu products %zu: tile kernel %zu tiles, small kernels %zu + %zu blocks\n",
                     tl.groups.size(), tl.tasks.size(), plan->tiles_h.size(), plan->wtiles_h[0].size(),
                     plan->wtiles_h[1].size());
        const char* nm[3] = {"<=16", "<=32", ">32"};
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            if (cnt[a][b] > 0)
              std::fprintf(stderr, "[tns plan]   output %s, X %s: %.0f products, %.3g flops\n", nm[a], nm[b],
                           cnt[a][b], fl[a][b]);
      }
    }
    // each kernel's product records go up only if that kernel has blocks
    const bool any_tile = !plan->tiles_h.empty();
    const bool any_small = !plan->wtiles_h[0].empty() || !plan->wtiles_h[1].empty();
    be.need(plan->ops_bytes * (es == 2 ? 2 : 1) +
            (long long)plan->tasks_h.size() *
                ((any_tile ? (long long)sizeof(TcTask) : 0) + (any_small ? (long long)sizeof(SwRec) : 0)) +
            (long long)plan->chunks_h.size() * (long long)sizeof(TcChunk) +
            (long long)jobs.size() * (long long)sizeof(ImgJob));
    bool ok = true;
    if (any_tile) plan->tasks = upload_vec(be, plan->tasks_h, ok);
    if (any_small) {
      std::vector<SwRec> recs(plan->tasks_h.size());
      for (size_t i = 0; i < recs.size(); ++i) {
        const TcTask& k = plan->tasks_h[i];
        recs[i].loff = (uint32_t)(k.L.off >> 8);
        recs[i].roff = (uint32_t)(k.R.off >> 8);
        recs[i].alpha = k.alpha;
        recs[i].pk = ((uint32_t)k.xb & 0xFFFFFu) | ((uint32_t)((k.m - 1) & 31) << 20) |
                     ((uint32_t)((k.n - 1) & 31) << 25);
      }
      plan->swrec = upload_vec(be, recs, ok);
    }
    plan->chunks = upload_vec(be, plan->chunks_h, ok);
    plan->xblocks = upload_vec(be, xbs, ok);
    plan->nxb = (int)xbs.size();
    plan->xbs_h = xbs;
    ImgJob* djobs = upload_vec(be, jobs, ok);
    ok = ok && dmalloc(&plan->flag, 8 * sizeof(int)) == cudaSuccess;
    ok = ok && dmalloc(&plan->ops_hi, std::max<long long>(plan->ops_bytes, 16)) == cudaSuccess;
    if (es == 2) ok = ok && dmalloc(&plan->ops_lo, std::max<long long>(plan->ops_bytes, 16)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      if (djobs) {
        cudaStreamSynchronize(be.stream());
        dfree(djobs);
      }
      be.note(cudaErrorMemoryAllocation, "tensor-core plan / operand images");
      release_tc_plan(plan);
      return false;
    }
    if (!jobs.empty()) {
      if (es == 4)
        k_img_ops<1><<<(unsigned)jobs.size(), 256, 0, be.stream()>>>(djobs, plan->ops_hi, nullptr);
      else
        k_img_ops<0><<<(unsigned)jobs.size(), 256, 0, be.stream()>>>(djobs, plan->ops_hi, plan->ops_lo);
      be.launches++;
      be.note(cudaGetLastError(), "operand images");
    }
    be.note(cudaStreamSynchronize(be.stream()), "operand images");
    dfree(djobs);
    d.tc = plan;
    d.tc_gen = tl.gen;
  }
  if (plan->x_nvec < nvec) {
    if (plan->x_hi) {
      be.free_graphs(d);  // graphs captured with the smaller images would write through freed pointers
      cudaStreamSynchronize(be.stream());
      dfree(plan->x_hi);
      if (plan->x_lo) dfree(plan->x_lo);
    }
    plan->x_hi = plan->x_lo = nullptr;
    plan->x_nvec = 0;
    const size_t xb = (size_t)std::max<long long>(plan->x_bytes, 16) * nvec;
    be.need((long long)xb * (es == 2 ? 2 : 1));
    bool ok = dmalloc(&plan->x_hi, xb) == cudaSuccess;
    if (es == 2) ok = ok && dmalloc(&plan->x_lo, xb) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      be.note(cudaErrorMemoryAllocation, "tensor-core input images");
      return false;
    }
    plan->x_nvec = nvec;
  }
  TcVariant& V = plan->var[variant];
  if (!V.planned) {
    std::vector<TcTile> tiles = plan->tiles_h;
    std::vector<TcTile> wtiles[2] = {plan->wtiles_h[0], plan->wtiles_h[1]};
    std::vector<SplitRed> reds;
    long long psize = 0;
    const std::vector<TcChunk>& ch = plan->chunks_h;
    const std::vector<double>& cc = plan->ccost_h;
    auto cost = [&](const TcChunk& C, const TcTile&) { return cc[&C - ch.data()]; };
    split_plan(tiles, plan->chunks_h, reds, psize, (double)TC_CTAS * plan->sms, kRounds[variant], cost);
    const double wunits[2] = {(double)SwCfg<16>::WARPS * SwCfg<16>::CTAS * plan->sms,
                              (double)SwCfg<32>::WARPS * SwCfg<32>::CTAS * plan->sms};
    for (int w = 0; w < 2; ++w) {
      // one partial-tile arena: each kernel's partial tiles after the previous ones
      std::vector<SplitRed> wreds;
      long long wpsize = 0;
      split_plan(wtiles[w], plan->chunks_h, wreds, wpsize, wunits[w], kRounds[variant], cost);
      for (TcTile& T : wtiles[w])
        if (T.poff >= 0) T.poff += psize;
      for (SplitRed& R : wreds) {
        R.poff += psize;
        reds.push_back(R);
      }
      psize += wpsize;
    }
    std::string why;
    if (!check_plan(*plan, tiles, plan->xbs_h, es, why) ||
        !check_small_plan<16>(*plan, wtiles[0], plan->xbs_h, tl.groups, es, why) ||
        !check_small_plan<32>(*plan, wtiles[1], plan->xbs_h, tl.groups, es, why)) {
      be.note(cudaErrorInvalidValue, ("tensor-core plan check failed: " + why).c_str());
      return false;
    }
    bool ok = true;
    V.tiles = upload_vec(be, tiles, ok);
    for (int w = 0; w < 2; ++w) {
      V.wtiles[w] = upload_vec(be, wtiles[w], ok);
      V.nwtiles[w] = (int)wtiles[w].size();
    }
    V.reds = upload_vec(be, reds, ok);
    if (variant == kWsVariant) {
      std::vector<int> order, off;
      V.ws_ctas = std::max(1, std::min((int)tiles.size(), plan->sms));
      ws_assign(plan->tasks_h, tiles, plan->chunks_h, V.ws_ctas, order, off);
      V.ws_order = upload_vec(be, order, ok);
      V.ws_off = upload_vec(be, off, ok);
    }
    if (!ok) {
      be.note(cudaErrorMemoryAllocation, "tensor-core schedule");
      return false;
    }
    V.ntiles = (int)tiles.size();
    V.nreds = (int)reds.size();
    V.psize = psize;
    V.planned = true;
    be.note(cudaStreamSynchronize(be.stream()), "tensor-core schedule upload");
  }
  if (V.psize > 0 && V.part_nvec < nvec) {
    if (V.part) {
      be.free_graphs(d);  // the same for the partial tiles
      cudaStreamSynchronize(be.stream());
      dfree(V.part);
    }
    V.part = nullptr;
    V.part_nvec = 0;
    be.need((long long)sizeof(double) * V.psize * nvec);
    if (dmalloc(&V.part, sizeof(double) * V.psize * nvec) != cudaSuccess) {
      cudaGetLastError();
      be.note(cudaErrorMemoryAllocation, "tensor-core partial tiles");
      return false;
    }
    V.part_nvec = nvec;
  }
  // kernel attributes once, outside any stream capture: the dynamic shared
  // memory, and the largest shared-memory carve-out (the kernel stages all
  // operands in shared memory and does not rely on L1)
  static bool attr = false;
  if (!attr) {
    be.note(cudaFuncSetAttribute(k_tasks_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<0>::total),
            "k_tasks_tc shared memory");
    be.note(cudaFuncSetAttribute(k_tasks_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<1>::total),
            "k_tasks_tc shared memory");
    be.note(cudaFuncSetAttribute(k_tasks_tc<0>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared),
            "k_tasks_tc carve-out");
    be.note(cudaFuncSetAttribute(k_tasks_tc<1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared),
            "k_tasks_tc carve-out");
    be.note(cudaFuncSetAttribute(k_tasks_tc_ws<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, WsSmem<0>::total),
            "k_tasks_tc_ws shared memory");
    be.note(cudaFuncSetAttribute(k_tasks_tc_ws<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, WsSmem<1>::total),
            "k_tasks_tc_ws shared memory");
    auto sw_attr = [&](const void* f, int bytes) {
      be.note(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes), "k_tasks_sw shared memory");
      be.note(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared),
              "k_tasks_sw carve-out");
    };
    sw_attr((const void*)k_tasks_sw<0, 16>, (int)sizeof(SwWarp<16>) * SwCfg<16>::WARPS);
    sw_attr((const void*)k_tasks_sw<1, 16>, (int)sizeof(SwWarp<16>) * SwCfg<16>::WARPS);
    sw_attr((const void*)k_tasks_sw<0, 32>, (int)sizeof(SwWarp<32>) * SwCfg<32>::WARPS);
    sw_attr((const void*)k_tasks_sw<1, 32>, (int)sizeof(SwWarp<32>) * SwCfg<32>::WARPS);
    attr = true;
  }
  return be.ok();
}

void enqueue_tasks_tc(CudaBackend& be, DevList& d, const double* xv, double* yv, int nvec, long long xs,
                      long long ys, int precision, int variant) {
  TcPlan* plan = (TcPlan*)d.tc;
  if (!plan || !be.ok()) return;
  TcVariant& V = plan->var[variant];
  if (V.ntiles == 0 && V.nwtiles[0] == 0 && V.nwtiles[1] == 0) return;
  be.note(cudaMemsetAsync(plan->flag, 0, 8 * sizeof(int), be.stream()), "tensor-core flag");
  if (plan->nxb > 0) {
    dim3 gx(plan->nxb, nvec);
    if (precision == TNS_TF32)
      k_img_x<1><<<gx, 256, 0, be.stream()>>>(plan->xblocks, xv, xs, plan->x_hi, nullptr, plan->x_bytes);
    else
      k_img_x<0><<<gx, 256, 0, be.stream()>>>(plan->xblocks, xv, xs, plan->x_hi, plan->x_lo, plan->x_bytes);
    be.launches++;
    be.note(cudaGetLastError(), "input images");
  }
  // small blocks: one warp per (piece, vector), the vectors of a piece in adjacent warps
  auto launch_sw = [&](auto kern, int warps, int bytes, const TcTile* wt, int nwt) {
    if (nwt <= 0) return;
    const long long nw = (long long)nwt * nvec;
    const unsigned grid = (unsigned)((nw + warps - 1) / warps);
    kern<<<grid, 32 * warps, bytes, be.stream()>>>(plan->swrec, d.groups, wt, nwt, plan->chunks, plan->ops_hi,
                                                    plan->ops_lo, plan->x_hi, plan->x_lo, plan->x_bytes,
                                                    plan->xblocks, yv, ys, plan->flag, V.part, V.psize, nvec,
                                                    be.tc_wait_ns);
    be.launches++;
    be.note(cudaGetLastError(), "k_tasks_sw");
  };
  const int b16 = (int)sizeof(SwWarp<16>) * SwCfg<16>::WARPS, b32 = (int)sizeof(SwWarp<32>) * SwCfg<32>::WARPS;
  if (precision == TNS_TF32) {
    launch_sw(k_tasks_sw<1, 16>, SwCfg<16>::WARPS, b16, V.wtiles[0], V.nwtiles[0]);
    launch_sw(k_tasks_sw<1, 32>, SwCfg<32>::WARPS, b32, V.wtiles[1], V.nwtiles[1]);
  } else {
    launch_sw(k_tasks_sw<0, 16>, SwCfg<16>::WARPS, b16, V.wtiles[0], V.nwtiles[0]);
    launch_sw(k_tasks_sw<0, 32>, SwCfg<32>::WARPS, b32, V.wtiles[1], V.nwtiles[1]);
  }
  if (V.ntiles == 0) {
    if (V.nreds > 0) launch_reduce_splits(be, V.reds, V.nreds, d.groups, V.part, V.psize, yv, ys, nvec);
    return;
  }
  if (variant == kWsVariant) {
    // persistent warp-specialised kernel: one CTA per SM, each over its list
    // of pieces (balanced by estimated cost) and all vectors
    const unsigned grid = (unsigned)V.ws_ctas;
    if (precision == TNS_TF32)
      k_tasks_tc_ws<1><<<grid, WS_NT, WsSmem<1>::total, be.stream()>>>(
          plan->tasks, d.groups, V.tiles, V.ws_order, V.ws_off, plan->chunks, plan->ops_hi, plan->ops_lo, plan->x_hi,
          plan->x_lo, plan->x_bytes, plan->xblocks, yv, ys, plan->flag, V.part, V.psize, nvec, be.tc_wait_ns);
    else
      k_tasks_tc_ws<0><<<grid, WS_NT, WsSmem<0>::total, be.stream()>>>(
          plan->tasks, d.groups, V.tiles, V.ws_order, V.ws_off, plan->chunks, plan->ops_hi, plan->ops_lo, plan->x_hi,
          plan->x_lo, plan->x_bytes, plan->xblocks, yv, ys, plan->flag, V.part, V.psize, nvec, be.tc_wait_ns);
    be.launches++;
    be.note(cudaGetLastError(), "k_tasks_tc_ws");
    if (V.nreds > 0) launch_reduce_splits(be, V.reds, V.nreds, d.groups, V.part, V.psize, yv, ys, nvec);
    return;
  }
  const unsigned grid = (unsigned)V.ntiles * (unsigned)nvec;
  if (precision == TNS_TF32)
    k_tasks_tc<1><<<grid, TC_NT, TcSmem<1>::total, be.stream()>>>(plan->tasks, d.groups, V.tiles, plan->chunks,
                                                                   plan->ops_hi, plan->ops_lo, plan->x_hi, plan->x_lo,
                                                                   plan->x_bytes, plan->xblocks, yv, ys, plan->flag,
                                                                   V.part, V.psize, nvec, be.tc_wait_ns);
  else
    k_tasks_tc<0><<<grid, TC_NT, TcSmem<0>::total, be.stream()>>>(plan->tasks, d.groups, V.tiles, plan->chunks,
                                                                   plan->ops_hi, plan->ops_lo, plan->x_hi, plan->x_lo,
                                                                   plan->x_bytes, plan->xblocks, yv, ys, plan->flag,
                                                                   V.part, V.psize, nvec, be.tc_wait_ns);
  be.launches++;
  be.note(cudaGetLastError(), "k_tasks_tc");
  if (V.nreds > 0) launch_reduce_splits(be, V.reds, V.nreds, d.groups, V.part, V.psize, yv, ys, nvec);
}

void check_tasks_tc(CudaBackend& be, DevList& d) {
  TcPlan* plan = (TcPlan*)d.tc;
  if (!plan) return;
  int h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  cudaMemcpyAsync(h, plan->flag, sizeof(h), cudaMemcpyDeviceToHost, be.stream());
  be.note(cudaStreamSynchronize(be.stream()), "k_tasks_tc");
  if (h[0] && h[2] == 20) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "k_tasks_sw: wait timed out (piece %d, product %d, %d issued)", h[1], h[3], h[4]);
    be.note(cudaErrorLaunchTimeout, msg);
  } else if (h[0]) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "k_tasks_tc: wait timed out (tile piece %d, barrier %d, chunk %d, row offset %d, step %d, phase %d)",
                  h[1], h[2], h[3], h[4], h[5], h[6]);
    be.note(cudaErrorLaunchTimeout, msg);
  }
}

void release_tc_plan(void* p) {
  TcPlan* plan = (TcPlan*)p;
  if (!plan) return;
  for (TcVariant& V : plan->var) {
    for (TcTile* w : V.wtiles)
      if (w) dfree(w);
    if (V.ws_order) dfree(V.ws_order);
    if (V.ws_off) dfree(V.ws_off);
    if (V.tiles) dfree(V.tiles);
    if (V.reds) dfree(V.reds);
    if (V.part) dfree(V.part);
  }
  if (plan->tasks) dfree(plan->tasks);
  if (plan->swrec) dfree(plan->swrec);
  if (plan->chunks) dfree(plan->chunks);
  if (plan->xblocks) dfree(plan->xblocks);
  if (plan->flag) dfree(plan->flag);
  if (plan->ops_hi) dfree(plan->ops_hi);
  if (plan->ops_lo) dfree(plan->ops_lo);
  if (plan->x_hi) dfree(plan->x_hi);
  if (plan->x_lo) dfree(plan->x_lo);
  delete plan;
}

}  // namespace tns
