// kernels.cu -- FP64 kernels of the engine and the CUDA backend (sm_103a).
//
// The grouped triple product (Eq. 2, Alg. 2):
//     Y_tile = sum_{tasks of the tile's output block} alpha * op(L) op(X) op(R)^T
// One CTA owns one output tile (<= 64 x 64) of one output block and walks
// that block's task list in a fixed order, so every run is bitwise
// reproducible and no atomics are needed.  The position sum of Eq. (2) (and
// the sum over all operator pairs and dot blocks that hit the block) is the
// K loop of the accumulation, as in Alg. 2 where the sum over i becomes the
// inner dimension of one GEMM.  Each task is evaluated in the cheaper chain
// order: L (X R^T) or (L X) R^T, with the intermediate chunk in shared
// memory.  FP64 on GB300 is DFMA-issue bound, so the kernel keeps every
// DFMA useful (loops run to the exact block sizes, no zero padding) and
// sizes its CTA to the tile so that few lanes idle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <unordered_set>

#include "cuda_backend.h"

namespace tns {

// ---------------------------------------------------------------------------
// operand access
// ---------------------------------------------------------------------------
__device__ __forceinline__ double opL(const Task& t, int i, int k) {
  if (t.flags & TF_LI) return i == k ? 1.0 : 0.0;
  return (t.flags & TF_LT) ? __ldg(t.L + (long long)k * t.q + i) : __ldg(t.L + (long long)i * t.m + k);
}
__device__ __forceinline__ double opX(const Task& t, const double* X, int i, int j) {
  if (t.flags & TF_XI) return i == j ? 1.0 : 0.0;
  return (t.flags & TF_XT) ? __ldg(X + (long long)j * t.m + i) : __ldg(X + (long long)i * t.n + j);
}
__device__ __forceinline__ double opR(const Task& t, int j, int k) {
  if (t.flags & TF_RI) return j == k ? 1.0 : 0.0;
  return (t.flags & TF_RT) ? __ldg(t.R + (long long)k * t.r + j) : __ldg(t.R + (long long)j * t.n + k);
}

constexpr int CH = 32;  // chunk of the contracted middle dimension

// tile classes: (threads, outputs per thread, max tile rows, max tile cols);
// a group's output block is cut into tall (<= 128 x 32) or wide (<= 32 x 128)
// tiles, whichever executes fewer FMAs for its products; tiles of at most
// 32 x 32 (16 x 16) run in the small classes, which keep many CTAs per SM
constexpr int C0_NT = 32, C0_ACC = 8, C0_TR = 16, C0_TC = 16;
constexpr int C1_NT = 128, C1_ACC = 8, C1_TR = 32, C1_TC = 32;
constexpr int C2_NT = 256, C2_ACC = 16, C2_TR = 128, C2_TC = 32;  // tall
constexpr int C3_NT = 256, C3_ACC = 16, C3_TR = 32, C3_TC = 128;  // wide
constexpr int kFpClasses = 4;
constexpr int kTallR = 128, kTallC = 32, kWideR = 32, kWideC = 128;

// dynamic shared memory of a class: max(SA, SB) + SR doubles (see the kernel)
constexpr int fp64_smem(int TR, int TC) {
  return 8 * ((CH * (TC + 1) > TR * (CH + 1) ? CH * (TC + 1) : TR * (CH + 1)) + CH * (TC + 1));
}

// FMAs of one product on an nr x nc tile of its output block.  With no
// identity factor the kernel evaluates L (X R^T) or (L X) R^T, whichever is
// cheaper on this tile (the intermediate is recomputed per tile: X R^T per
// row tile, L X per column tile); *ordb tells which
__host__ __device__ inline long long tile_fmas(const Task& t, int nr, int nc, bool* ordb) {
  const long long a = nr, b = nc;
  if (ordb) *ordb = false;
  if ((t.flags & TF_LI) && (t.flags & TF_RI)) return a * b;
  if (t.flags & TF_LI) return a * b * t.n;
  if (t.flags & (TF_RI | TF_XI)) return a * b * t.m;
  const long long ca = b * t.m * (t.n + a);  // L (X R^T)
  const long long cb = a * t.n * (t.m + b);  // (L X) R^T
  if (ordb) *ordb = cb < ca;
  return cb < ca ? cb : ca;
}

template <int NT, int ACC, int TR, int TC>
__global__ void __launch_bounds__(NT, NT >= 256 ? 2 : NT >= 128 ? 4 : 16) k_tasks_fp64(const Task* __restrict__ tasks, const Group* __restrict__ groups,
                                                   const Tile* __restrict__ tiles, int tile0, const double* xv,
                                                   double* yv, long long xs, long long ys, double* part,
                                                   long long psize, int nv) {
  constexpr int SA = CH * (TC + 1);  // L (X R^T): CH rows of X R^T, TC columns
  constexpr int SB = TR * (CH + 1);  // (L X) R^T: TR rows of L X, CH columns
  constexpr int TE = CH * TC / NT;   // elements of X R^T per thread and chunk (upper bound)
  extern __shared__ double S[];      // max(SA, SB) + SR doubles, SR = CH * (TC + 1)
  double* const Rt = S + (SA > SB ? SA : SB);  // L (X R^T): a K slice of the tile's R rows, transposed
  // the vectors of one tile piece are adjacent CTAs (they read the same operator blocks)
  const Tile T = tiles[tile0 + blockIdx.x / nv];
  const Group G = groups[T.g];
  const int vec = blockIdx.x % nv;
  const double* X0 = xv ? xv + (long long)vec * xs : nullptr;
  double* Y = yv + (long long)vec * ys + G.yoff;
  const int nc = T.ncols, nr = T.nrows;
  const int nout = nr * nc;
  const int tid = threadIdx.x;
  double* P = T.poff >= 0 ? part + (long long)vec * psize + T.poff : nullptr;  // split piece
  int ri[ACC], cj[ACC];
  double acc[ACC];
#pragma unroll
  for (int u = 0; u < ACC; ++u) {
    const int e = tid + u * NT;
    ri[u] = e < nout ? e / nc : -1;
    cj[u] = e < nout ? e % nc : 0;
    acc[u] = 0.0;
  }
  // phase-1 thread maps (no division inside the task loop)
  const int a_j = tid % nc, a_i0 = tid / nc, a_st = NT / nc;
  const bool a_ok = tid < a_st * nc;
  const int b_j = tid % CH, b_i0 = tid / CH, b_st = NT / CH;

  for (int ti = T.t0; ti < T.t1; ++ti) {
    const Task tk = tasks[ti];
    const int f = tk.flags;
    const double a = tk.alpha;
    // element (i,k) of op(L) = pL[i*sLi + k*sLk]; op(X)(i,k) = pX[i*sXi + k*sXk]; op(R)(j,k) = pR[j*sRj + k*sRk]
    const double* pL = tk.L;
    const long long sLi = (f & TF_LT) ? 1 : tk.m, sLk = (f & TF_LT) ? tk.q : 1;
    const double* pX = (f & TF_XV) ? X0 + (long long)(size_t)tk.X : tk.X;
    const long long sXi = (f & TF_XT) ? 1 : tk.n, sXk = (f & TF_XT) ? tk.m : 1;
    const double* pR = tk.R;
    const long long sRj = (f & TF_RT) ? 1 : tk.n, sRk = (f & TF_RT) ? tk.r : 1;
    bool ordb;
    tile_fmas(tk, nr, nc, &ordb);
    if ((f & TF_LI) && (f & TF_RI)) {
#pragma unroll
      for (int u = 0; u < ACC; ++u)
        if (ri[u] >= 0) acc[u] = fma(a, __ldg(pX + (T.row0 + ri[u]) * sXi + (T.col0 + cj[u]) * sXk), acc[u]);
    } else if (f & TF_LI) {  // Y += X R^T
#pragma unroll
      for (int u = 0; u < ACC; ++u) {
        if (ri[u] < 0) continue;
        const double* xr = pX + (T.row0 + ri[u]) * sXi;
        const double* rr = pR + (T.col0 + cj[u]) * sRj;
        double s = 0.0;
        for (int k = 0; k < tk.n; ++k) s = fma(__ldg(xr + k * sXk), __ldg(rr + k * sRk), s);
        acc[u] = fma(a, s, acc[u]);
      }
    } else if (f & TF_RI) {  // Y += L X
#pragma unroll
      for (int u = 0; u < ACC; ++u) {
        if (ri[u] < 0) continue;
        const double* lr = pL + (T.row0 + ri[u]) * sLi;
        const double* xc = pX + (T.col0 + cj[u]) * sXk;
        double s = 0.0;
        for (int k = 0; k < tk.m; ++k) s = fma(__ldg(lr + k * sLk), __ldg(xc + k * sXi), s);
        acc[u] = fma(a, s, acc[u]);
      }
    } else if (f & TF_XI) {  // Y += L R^T
#pragma unroll
      for (int u = 0; u < ACC; ++u) {
        if (ri[u] < 0) continue;
        const double* lr = pL + (T.row0 + ri[u]) * sLi;
        const double* rr = pR + (T.col0 + cj[u]) * sRj;
        double s = 0.0;
        for (int k = 0; k < tk.m; ++k) s = fma(__ldg(lr + k * sLk), __ldg(rr + k * sRk), s);
        acc[u] = fma(a, s, acc[u]);
      }
    } else if (!ordb) {
      // L (X R^T): chunks of CH rows of X
      for (int m0 = 0; m0 < tk.m; m0 += CH) {
        const int mc = min(CH, tk.m - m0);
        // T = X[m0.., :] R[tile cols, :]^T in K slices of CH; the slice of R
        // is staged transposed so that consecutive threads read consecutive
        // columns (a strided row read per thread otherwise)
        double tacc[TE];
#pragma unroll
        for (int e = 0; e < TE; ++e) tacc[e] = 0.0;
        for (int k0 = 0; k0 < tk.n; k0 += CH) {
          const int kc = min(CH, tk.n - k0);
          for (int e = tid; e < nc * kc; e += NT) {
            const int j = e / kc, kk = e % kc;
            Rt[kk * (TC + 1) + j] = __ldg(pR + (T.col0 + j) * sRj + (k0 + kk) * sRk);
          }
          __syncthreads();
          if (a_ok) {
#pragma unroll
            for (int e = 0; e < TE; ++e) {
              const int i = a_i0 + e * a_st;
              if (i < mc) {
                const double* xr = pX + (m0 + i) * sXi + k0 * sXk;
                double s = tacc[e];
                for (int kk = 0; kk < kc; ++kk) s = fma(__ldg(xr + kk * sXk), Rt[kk * (TC + 1) + a_j], s);
                tacc[e] = s;
              }
            }
          }
          __syncthreads();
        }
        if (a_ok) {
#pragma unroll
          for (int e = 0; e < TE; ++e) {
            const int i = a_i0 + e * a_st;
            if (i < mc) S[i * (TC + 1) + a_j] = tacc[e];
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < ACC; ++u) {
          if (ri[u] < 0) continue;
          const double* lr = pL + (T.row0 + ri[u]) * sLi + m0 * sLk;
          double s = 0.0;
          for (int k = 0; k < mc; ++k) s = fma(__ldg(lr + k * sLk), S[k * (TC + 1) + cj[u]], s);
          acc[u] = fma(a, s, acc[u]);
        }
        __syncthreads();
      }
    } else {
      // (L X) R^T: chunks of CH columns of X
      for (int n0 = 0; n0 < tk.n; n0 += CH) {
        const int ncc = min(CH, tk.n - n0);
        if (b_j < ncc) {
          const double* xc = pX + (n0 + b_j) * sXk;
          for (int i = b_i0; i < nr; i += b_st) {
            const double* lr = pL + (T.row0 + i) * sLi;
            double s = 0.0;
            for (int k = 0; k < tk.m; ++k) s = fma(__ldg(lr + k * sLk), __ldg(xc + k * sXi), s);
            S[i * (CH + 1) + b_j] = s;
          }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < ACC; ++u) {
          if (ri[u] < 0) continue;
          const double* rr = pR + (T.col0 + cj[u]) * sRj + n0 * sRk;
          double s = 0.0;
          for (int k = 0; k < ncc; ++k) s = fma(S[ri[u] * (CH + 1) + k], __ldg(rr + k * sRk), s);
          acc[u] = fma(a, s, acc[u]);
        }
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int u = 0; u < ACC; ++u)
    if (ri[u] >= 0) {
      if (P) P[ri[u] * nc + cj[u]] = acc[u];
      else Y[(long long)(T.row0 + ri[u]) * G.r + T.col0 + cj[u]] = acc[u];
    }
}

// ---------------------------------------------------------------------------
// FP64 tensor path: the same grouped triple product on DMMA
// (mma.sync m8n8k4 f64).  One warp owns a 32 x 16 output tile; per product it
// streams the contracted dimension in chunks of 8 through a warp-private
// shared-memory slab: L (X R^T) (T chunk 8 x 16) or (L X) R^T (U chunk
// 32 x 8), whichever is cheaper for the tile.  Ragged edges are predicated
// loads returning zero.  Fragment layout of m8n8k4 f64 (g = lane/4,
// t = lane%4): A(g, t), B(t, g), C(g, 2t), C(g, 2t+1).
// ---------------------------------------------------------------------------
constexpr int DM_WR = 32, DM_WC = 16, DM_WARPS = 4;
constexpr int DM_SLAB = 32 * 9;  // max(8 x 17, 32 x 9)

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(32 * DM_WARPS) k_tasks_dmma(const Task* __restrict__ tasks,
                                                              const Group* __restrict__ groups,
                                                              const Tile* __restrict__ tiles, int ntiles,
                                                              const double* xv, double* yv, long long xs,
                                                              long long ys) {
  __shared__ double slab[DM_WARPS][DM_SLAB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti_ = blockIdx.x * DM_WARPS + warp;
  if (ti_ >= ntiles) return;  // whole warp
  double* S = slab[warp];
  const int g = lane >> 2, t = lane & 3;
  const Tile T = tiles[ti_];
  const Group G = groups[T.g];
  const int vec = blockIdx.y;
  const double* X0 = xv ? xv + (long long)vec * xs : nullptr;
  double* Y = yv + (long long)vec * ys + G.yoff;
  const int nr = T.nrows, nc = T.ncols;
  const int nrt = (nr + 7) >> 3, nct = (nc + 7) >> 3;  // used 8x8 tiles
  double acc[4][2][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b][0] = acc[a][b][1] = 0.0;

  for (int k = T.t0; k < T.t1; ++k) {
    const Task tk = tasks[k];
    const int f = tk.flags;
    const double al = tk.alpha;
    const int m = tk.m, n = tk.n;
    const double* pL = tk.L;
    const long long sLi = (f & TF_LT) ? 1 : m, sLk = (f & TF_LT) ? tk.q : 1;
    const double* pX = (f & TF_XV) ? X0 + (long long)(size_t)tk.X : tk.X;
    const long long sXi = (f & TF_XT) ? 1 : n, sXk = (f & TF_XT) ? m : 1;
    const double* pR = tk.R;
    const long long sRj = (f & TF_RT) ? 1 : n, sRk = (f & TF_RT) ? tk.r : 1;
    // predicated operand loads (tile-local row/col)
    auto Lv = [&](int i, int kk) -> double {
      if (i >= nr || kk >= m) return 0.0;
      if (f & TF_LI) return (T.row0 + i == kk) ? 1.0 : 0.0;
      return __ldg(pL + (T.row0 + i) * sLi + kk * sLk);
    };
    auto Rv = [&](int j, int kk) -> double {  // op(R)(col, kk)
      if (j >= nc || kk >= n) return 0.0;
      if (f & TF_RI) return (T.col0 + j == kk) ? 1.0 : 0.0;
      return __ldg(pR + (T.col0 + j) * sRj + kk * sRk);
    };
    auto Xv = [&](int i, int kk) -> double {  // op(X)(i, kk), absolute indices
      if (i >= m || kk >= n) return 0.0;
      if (f & TF_XI) return (i == kk) ? 1.0 : 0.0;
      return __ldg(pX + i * sXi + kk * sXk);
    };
    if ((f & TF_LI) && (f & TF_RI)) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int i = 8 * a + g, j = 8 * b + 2 * t + e;
            if (i < nr && j < nc) acc[a][b][e] = fma(al, Xv(T.row0 + i, T.col0 + j), acc[a][b][e]);
          }
      continue;
    }
    if (f & (TF_LI | TF_RI | TF_XI)) {
      // two-factor product P Q^T with P rows = tile rows, Q rows = tile cols
      const int K = (f & TF_LI) ? n : m;
      for (int k0 = 0; k0 < K; k0 += 4) {
        double bq[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int j = 8 * b + g, kk = k0 + t;
          bq[b] = (f & TF_RI) ? Xv(kk, (j < nc) ? T.col0 + j : n) : Rv(j, kk);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (a >= nrt) break;
          const int i = 8 * a + g, kk = k0 + t;
          const double av = al * ((f & TF_LI) ? ((i < nr) ? Xv(T.row0 + i, kk) : 0.0) : Lv(i, kk));
#pragma unroll
          for (int b = 0; b < 2; ++b)
            if (b < nct) dmma(acc[a][b], av, bq[b]);
        }
      }
      continue;
    }
    // three-factor product: choose the chain order for this tile
    const double ca = (double)m * n * nc + (double)nr * m * nc;
    const double cb = (double)nr * m * n + (double)nr * n * nc;
    if (ca <= cb) {
      // L (X R^T): T chunk (8 x 16) = X[k0..k0+8, :] R[cols, :]^T
      for (int k0 = 0; k0 < m; k0 += 8) {
        double tc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int b0 = 0; b0 < n; b0 += 4) {
          const double av = Xv(k0 + g, b0 + t);
#pragma unroll
          for (int b = 0; b < 2; ++b)
            if (b < nct) dmma(tc[b], av, Rv(8 * b + g, b0 + t));
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          S[g * 17 + 8 * b + 2 * t] = tc[b][0];
          S[g * 17 + 8 * b + 2 * t + 1] = tc[b][1];
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          double bq[2];
#pragma unroll
          for (int b = 0; b < 2; ++b) bq[b] = S[(4 * s + t) * 17 + 8 * b + g];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (a >= nrt) break;
            const double av = al * Lv(8 * a + g, k0 + 4 * s + t);
#pragma unroll
            for (int b = 0; b < 2; ++b)
              if (b < nct) dmma(acc[a][b], av, bq[b]);
          }
        }
        __syncwarp();
      }
    } else {
      // (L X) R^T: U chunk (32 x 8) = L[rows, :] X[:, n0..n0+8]
      for (int n0 = 0; n0 < n; n0 += 8) {
        double uc[4][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        for (int k0 = 0; k0 < m; k0 += 4) {
          const double bx = Xv(k0 + t, n0 + g);
#pragma unroll
          for (int a = 0; a < 4; ++a)
            if (a < nrt) dmma(uc[a], Lv(8 * a + g, k0 + t), bx);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          S[(8 * a + g) * 9 + 2 * t] = uc[a][0];
          S[(8 * a + g) * 9 + 2 * t + 1] = uc[a][1];
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          double bq[2];
#pragma unroll
          for (int b = 0; b < 2; ++b) bq[b] = Rv(8 * b + g, n0 + 4 * s + t);
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (a >= nrt) break;
            const double av = al * S[(8 * a + g) * 9 + 4 * s + t];
#pragma unroll
            for (int b = 0; b < 2; ++b)
              if (b < nct) dmma(acc[a][b], av, bq[b]);
          }
        }
        __syncwarp();
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int i = 8 * a + g, j = 8 * b + 2 * t + e;
        if (i < nr && j < nc) Y[(long long)(T.row0 + i) * G.r + T.col0 + j] = acc[a][b][e];
      }
}

// split tiles: output = sum of the pieces' partial tiles in piece order
__global__ void k_reduce_splits(const SplitRed* __restrict__ reds, int nreds, const Group* __restrict__ groups,
                                const double* __restrict__ part, long long psize, double* yv, long long ys) {
  const int vec = blockIdx.y;
  for (int b = blockIdx.x; b < nreds; b += gridDim.x) {
    const SplitRed R = reds[b];
    const Group G = groups[R.g];
    const int nel = R.nrows * R.ncols;
    const double* p = part + (long long)vec * psize + R.poff;
    double* Y = yv + (long long)vec * ys + G.yoff;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q < R.nsplit; ++q) s += p[(long long)q * nel + e];
      Y[(long long)(R.row0 + e / R.ncols) * G.r + R.col0 + e % R.ncols] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// partial sums (materialised linear combinations of operator blocks)
// ---------------------------------------------------------------------------
__global__ void k_lincomb(const LCBlock* __restrict__ blocks, int nb, const LCTerm* __restrict__ terms) {
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const LCBlock B = blocks[b];
    const int n = B.rows * B.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int i = e / B.cols, j = e % B.cols;
      double s = 0.0;
      for (int t = B.t0; t < B.t1; ++t) {
        const LCTerm T = terms[t];
        double x;
        if (!T.src) x = (i == j) ? 1.0 : 0.0;
        else x = T.tr ? __ldg(T.src + (long long)j * B.rows + i) : __ldg(T.src + e);
        s = fma(T.c, x, s);
      }
      B.dst[e] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// H_eff diagonal: diag(Y_blk)_{ij} = sum alpha op(L)_ii op(R)_jj over the
// tasks mapping a block onto itself (fixed order per block)
// ---------------------------------------------------------------------------
__global__ void k_heff_diag(const Task* __restrict__ tasks, const int* __restrict__ idx, const int* __restrict__ rng,
                            int ngroups, const Group* __restrict__ groups, double* diag) {
  for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const Group G = groups[g];
    const int n = G.q * G.r;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int i = e / G.r, j = e % G.r;
      double s = 0.0;
      for (int t = rng[g]; t < rng[g + 1]; ++t) {
        const Task tk = tasks[idx[t]];
        s = fma(tk.alpha, opL(tk, i, i) * opR(tk, j, j), s);
      }
      diag[G.yoff + e] = s;
    }
  }
}

void launch_reduce_splits(CudaBackend& be, const SplitRed* reds, int nreds, const Group* groups, const double* part,
                          long long psize, double* yv, long long ys, int nvec) {
  if (!be.ok()) return;
  if (nreds <= 0) return;
  dim3 grid(std::min(nreds, 65535), nvec);
  k_reduce_splits<<<grid, 128, 0, be.stream()>>>(reds, nreds, groups, part, psize, yv, ys);
  be.launches++;
  be.note(cudaGetLastError(), "k_reduce_splits");
}

void launch_heff_diag(CudaBackend& be, const Task* d_tasks, const int* d_idx, const int* d_rng, int ngroups,
                      const Group* d_groups, double* diag) {
  if (!be.ok()) return;
  if (ngroups <= 0) return;
  k_heff_diag<<<std::min(ngroups, 65535), 128, 0, be.stream()>>>(d_tasks, d_idx, d_rng, ngroups, d_groups, diag);
  be.launches++;
  be.note(cudaGetLastError(), "k_heff_diag");
}

// ---------------------------------------------------------------------------
// FP64 vector kernels for the Davidson step (deterministic reductions)
// ---------------------------------------------------------------------------
constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
constexpr int RED_NT = 256;
constexpr int MAXK = 40;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partial[i * gridDim.x + blk] = sum over this block's slice of V_i . w
__global__ void __launch_bounds__(RED_NT) k_multidot(const double* __restrict__ V, long long ldv, int k,
                                                     const double* __restrict__ w, long long n,
                                                     double* __restrict__ partial) {
  __shared__ double red[RED_NT / 32][MAXK];
  double acc[MAXK];
  for (int i = 0; i < k; ++i) acc[i] = 0.0;
  for (long long j = blockIdx.x * (long long)RED_NT + threadIdx.x; j < n; j += (long long)gridDim.x * RED_NT) {
    const double x = w[j];
    for (int i = 0; i < k; ++i) acc[i] = fma(V[i * ldv + j], x, acc[i]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < k; ++i) {
    double s = warp_sum(acc[i]);
    if (lane == 0) red[wid][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int q = 0; q < RED_NT / 32; ++q) s += red[q][threadIdx.x];
    partial[threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_reduce_partials(const double* __restrict__ partial, int nb, int k, double* out) {
  // one warp per output, fixed order
  const int i = blockIdx.x;
  if (i >= k) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += partial[i * nb + b];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[i] = s;
}

void launch_multidot(CudaBackend& be, const double* V, long long ldv, int k, const double* w, long long n,
                     double* out) {
  if (!be.ok()) return;
  // in chunks of at most MAXK vectors (the kernel keeps one accumulator per vector)
  double* partial = (double*)be.scratch(sizeof(double) * MAXK * RED_BLOCKS, 0);
  for (int i0 = 0; i0 < k; i0 += MAXK) {
    const int kc = std::min(MAXK, k - i0);
    k_multidot<<<RED_BLOCKS, RED_NT, 0, be.stream()>>>(V + (long long)i0 * ldv, ldv, kc, w, n, partial);
    k_reduce_partials<<<kc, 32, 0, be.stream()>>>(partial, RED_BLOCKS, kc, out + i0);
    be.launches += 2;
    be.note(cudaGetLastError(), "multidot");
  }
}

// w += sign * sum_i coef[i] V_i
__global__ void k_axpy_multi(const double* __restrict__ V, long long ldv, int k, const double* __restrict__ coef,
                             double sign, double* w, long long n) {
  __shared__ double c[MAXK];
  if (threadIdx.x < k) c[threadIdx.x] = sign * coef[threadIdx.x];
  __syncthreads();
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    double s = w[j];
    for (int i = 0; i < k; ++i) s = fma(c[i], V[i * ldv + j], s);
    w[j] = s;
  }
}

void launch_axpy_multi(CudaBackend& be, const double* V, long long ldv, int k, const double* coef, double sign,
                       double* w, long long n) {
  if (!be.ok()) return;
  for (int i0 = 0; i0 < k; i0 += MAXK) {
    const int kc = std::min(MAXK, k - i0);
    k_axpy_multi<<<RED_BLOCKS * 2, 256, 0, be.stream()>>>(V + (long long)i0 * ldv, ldv, kc, coef + i0, sign, w, n);
    be.launches++;
    be.note(cudaGetLastError(), "axpy_multi");
  }
}

__global__ void k_combine(const double* __restrict__ V, long long ldv, int k, const double* __restrict__ coef,
                          double* out, long long n) {
  __shared__ double c[MAXK];
  if (threadIdx.x < k) c[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(c[i], V[i * ldv + j], s);
    out[j] = s;
  }
}

void launch_combine(CudaBackend& be, const double* V, long long ldv, int k, const double* coef, double* out,
                    long long n) {
  if (!be.ok()) return;
  if (k <= 0) return;
  const int kc = std::min(MAXK, k);
  k_combine<<<RED_BLOCKS * 2, 256, 0, be.stream()>>>(V, ldv, kc, coef, out, n);
  be.launches++;
  be.note(cudaGetLastError(), "combine");
  if (k > kc) launch_axpy_multi(be, V + (long long)kc * ldv, ldv, k - kc, coef + kc, 1.0, out, n);
}

// x *= f(num): inv_sqrt ? 1/sqrt(num) : num
__global__ void k_scale(double* x, const double* num, int inv_sqrt, long long n) {
  const double v = *num;
  const double s = inv_sqrt ? (v > 0.0 ? 1.0 / sqrt(v) : 0.0) : v;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    x[j] *= s;
}

void launch_scale(CudaBackend& be, double* x, const double* num, int inv_sqrt, long long n) {
  if (!be.ok()) return;
  k_scale<<<RED_BLOCKS * 2, 256, 0, be.stream()>>>(x, num, inv_sqrt, n);
  be.launches++;
  be.note(cudaGetLastError(), "scale");
}

// Davidson correction t = r / (theta - d), denominator floored at 1e-12
__global__ void k_precond(const double* r, const double* diag, const double* theta, double* t, long long n) {
  const double th = *theta;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    double den = th - diag[j];
    if (fabs(den) < 1e-12) den = den < 0 ? -1e-12 : 1e-12;
    t[j] = r[j] / den;
  }
}

void launch_precond(CudaBackend& be, const double* r, const double* diag, const double* theta, double* t,
                    long long n) {
  if (!be.ok()) return;
  k_precond<<<RED_BLOCKS * 2, 256, 0, be.stream()>>>(r, diag, theta, t, n);
  be.launches++;
  be.note(cudaGetLastError(), "precond");
}

// r = AVs - theta x
__global__ void k_residual(const double* AVs, const double* x, const double* theta, double* r, long long n) {
  const double th = *theta;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    r[j] = fma(-th, x[j], AVs[j]);
}

void launch_residual(CudaBackend& be, const double* AVs, const double* x, const double* theta, double* r,
                     long long n) {
  if (!be.ok()) return;
  k_residual<<<RED_BLOCKS * 2, 256, 0, be.stream()>>>(AVs, x, theta, r, n);
  be.launches++;
  be.note(cudaGetLastError(), "residual");
}

__global__ void k_argmin(const double* x, long long n, long long* idx) {
  __shared__ double bv[1024];
  __shared__ long long bi[1024];
  double v = 1e300;
  long long id = 0;
  for (long long j = threadIdx.x; j < n; j += blockDim.x)
    if (x[j] < v) {
      v = x[j];
      id = j;
    }
  bv[threadIdx.x] = v;
  bi[threadIdx.x] = id;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double v2 = bv[threadIdx.x + s];
      long long i2 = bi[threadIdx.x + s];
      if (v2 < bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *idx = bi[0];
}

void launch_argmin(CudaBackend& be, const double* x, long long n, long long* idx) {
  if (!be.ok()) return;
  k_argmin<<<1, 1024, 0, be.stream()>>>(x, n, idx);
  be.launches++;
  be.note(cudaGetLastError(), "argmin");
}

__global__ void k_fill_unit(double* x, long long n, const long long* idx) {
  const long long id = *idx;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    x[j] = (j == id) ? 1.0 : 0.0;
}

void launch_fill_unit(CudaBackend& be, double* x, long long n, const long long* idx) {
  if (!be.ok()) return;
  k_fill_unit<<<RED_BLOCKS * 2, 256, 0, be.stream()>>>(x, n, idx);
  be.launches++;
  be.note(cudaGetLastError(), "fill_unit");
}

// ---------------------------------------------------------------------------
// batched symmetric eigensolver: parallel cyclic Jacobi (round-robin pairs),
// one CTA per matrix, matrices in global memory; bounded number of sweeps
// ---------------------------------------------------------------------------
constexpr int JAC_NT = 256;
constexpr int JAC_MAXSWEEP = 40;
constexpr int JAC_MAXPAIR = 1024;  // n <= 2048

__global__ void __launch_bounds__(JAC_NT) k_jacobi(double* A, double* V, double* w, const long long* off,
                                                   const int* nn, const int* woff, int* sweeps_out) {
  __shared__ double cs[JAC_MAXPAIR], sn[JAC_MAXPAIR];
  __shared__ int pp[JAC_MAXPAIR], qq[JAC_MAXPAIR];
  __shared__ double red[JAC_NT / 32];
  __shared__ int done;
  const int mi = blockIdx.x;
  const int n = nn[mi];
  double* a = A + off[mi];
  double* v = V + off[mi];
  for (long long e = threadIdx.x; e < (long long)n * n; e += JAC_NT) v[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
  __syncthreads();
  const int ne = n + (n & 1);
  const int np = ne / 2;
  int sweep = 0;
  for (; sweep < JAC_MAXSWEEP && n > 1; ++sweep) {
    // convergence test: off-diagonal vs diagonal Frobenius norm
    double off2 = 0.0, dia2 = 0.0;
    for (long long e = threadIdx.x; e < (long long)n * n; e += JAC_NT) {
      double x = a[e];
      if ((e / n) == (e % n)) dia2 += x * x;
      else off2 += x * x;
    }
    off2 = warp_sum(off2);
    dia2 = warp_sum(dia2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = off2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int q = 0; q < JAC_NT / 32; ++q) s += red[q];
      red[0] = s;
    }
    __syncthreads();
    off2 = red[0];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dia2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int q = 0; q < JAC_NT / 32; ++q) s += red[q];
      done = (off2 <= 1e-30 * (s + off2)) || off2 < 1e-300;
    }
    __syncthreads();
    if (done) break;
    for (int round = 0; round < ne - 1; ++round) {
      for (int k = threadIdx.x; k < np; k += JAC_NT) {
        int p, q;
        if (k == 0) {
          p = round;
          q = ne - 1;
        } else {
          p = (round + k) % (ne - 1);
          q = (round - k + (ne - 1)) % (ne - 1);
        }
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = a[(long long)p * n + q];
          if (apq != 0.0) {
            double app = a[(long long)p * n + p], aqq = a[(long long)q * n + q];
            double tau = (aqq - app) / (2.0 * apq);
            double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[k] = c;
        sn[k] = s;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (long long e = threadIdx.x; e < (long long)np * n; e += JAC_NT) {
        int k = (int)(e / n), j = (int)(e % n);
        int p = pp[k], q = qq[k];
        if (q >= n || sn[k] == 0.0) continue;
        double c = cs[k], s = sn[k];
        double x = a[(long long)p * n + j], y = a[(long long)q * n + j];
        a[(long long)p * n + j] = c * x - s * y;
        a[(long long)q * n + j] = s * x + c * y;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (long long e = threadIdx.x; e < (long long)np * n; e += JAC_NT) {
        int k = (int)(e / n), i = (int)(e % n);
        int p = pp[k], q = qq[k];
        if (q >= n || sn[k] == 0.0) continue;
        double c = cs[k], s = sn[k];
        double x = a[(long long)i * n + p], y = a[(long long)i * n + q];
        a[(long long)i * n + p] = c * x - s * y;
        a[(long long)i * n + q] = s * x + c * y;
        x = v[(long long)i * n + p];
        y = v[(long long)i * n + q];
        v[(long long)i * n + p] = c * x - s * y;
        v[(long long)i * n + q] = s * x + c * y;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += JAC_NT) w[woff[mi] + i] = a[(long long)i * n + i];
  if (threadIdx.x == 0 && sweeps_out) sweeps_out[mi] = sweep;
}

void launch_jacobi(CudaBackend& be, double* A, double* V, double* w, const long long* off, const int* n,
                   const int* woff, int nmat, int maxn, int* sweeps_out) {
  if (!be.ok()) return;
  if (nmat <= 0) return;
  if (maxn > 2 * JAC_MAXPAIR) {
    be.note(cudaErrorInvalidValue, "jacobi: matrix too large");
    return;
  }
  k_jacobi<<<nmat, JAC_NT, 0, be.stream()>>>(A, V, w, off, n, woff, sweeps_out);
  be.launches++;
  be.note(cudaGetLastError(), "jacobi");
}

// ---------------------------------------------------------------------------
// global truncation: keep the `keep_max` largest eigenvalues (> cut) over all
// sectors; ties broken by (sector, index).  One CTA, bitonic sort in global
// scratch.  keep_flag[i] = 1 for kept entries, disc = discarded weight.
// ---------------------------------------------------------------------------
__global__ void k_select(const double* w, const int* sec_of, int total, int P, int keep_max, double cut,
                         double* kv, int* ki, int* keep_flag, double* disc) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    kv[i] = i < total ? w[i] : -1e300;
    ki[i] = i < total ? i : 0x7fffffff;
  }
  __syncthreads();
  // sort descending by value, ascending by index on ties (index order = (sector, in-sector))
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          bool desc = ((i & k) == 0);
          double a = kv[i], b = kv[l];
          int ia = ki[i], ib = ki[l];
          bool a_first = (a > b) || (a == b && ia < ib);
          if (desc ? !a_first : a_first) {
            kv[i] = b;
            kv[l] = a;
            ki[i] = ib;
            ki[l] = ia;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < total; i += blockDim.x) keep_flag[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < total; i += blockDim.x)
    if (i < keep_max && kv[i] > cut) keep_flag[ki[i]] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int i = 0; i < total; ++i)
      if (!(i < keep_max && kv[i] > cut)) d += fmax(kv[i], 0.0);
    *disc = d;
  }
  (void)sec_of;
}

void launch_select(CudaBackend& be, const double* w, const int* sec_of, int total, int keep_max, double cut,
                   int* keep_flag, double* disc) {
  if (!be.ok()) return;
  int P = 1;
  while (P < total) P <<= 1;
  double* kv = (double*)be.scratch(sizeof(double) * P + 64, 1);
  int* ki = (int*)be.scratch(sizeof(int) * P + 64, 2);
  k_select<<<1, 1024, 0, be.stream()>>>(w, sec_of, total, P, keep_max, cut, kv, ki, keep_flag, disc);
  be.launches++;
  be.note(cudaGetLastError(), "select");
}

// strided block copies: dst[i*dld + j] = trans ? src[j*sld + i] : src[i*sld + j]
__global__ void k_gather(const double* src, const long long* so, const int* sld, double* dst, const long long* dof,
                         const int* dld, const int* rows, const int* cols, const int* trans, int nblk) {
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const double* s = src + so[b];
    double* d = dst + dof[b];
    const int R = rows[b], Cn = cols[b], ls = sld[b], ld = dld[b], tr = trans[b];
    for (int e = threadIdx.x; e < R * Cn; e += blockDim.x) {
      int i = e / Cn, j = e % Cn;
      d[(long long)i * ld + j] = tr ? s[(long long)j * ls + i] : s[(long long)i * ls + j];
    }
  }
}

void launch_gather(CudaBackend& be, const double* src, const long long* so, const int* sld, double* dst,
                   const long long* dof, const int* dld, const int* rows, const int* cols, const int* trans,
                   int nblk) {
  if (!be.ok()) return;
  if (nblk <= 0) return;
  k_gather<<<std::min(nblk, 65535), 128, 0, be.stream()>>>(src, so, sld, dst, dof, dld, rows, cols, trans, nblk);
  be.launches++;
  be.note(cudaGetLastError(), "gather");
}

// ---------------------------------------------------------------------------
// backend
// ---------------------------------------------------------------------------
CudaBackend::CudaBackend(int device, cudaStream_t s, bool own) : device_(device), stream_(s), own_(own) {
  const char* gr = std::getenv("TNS_GRAPHS");
  if (gr && std::strcmp(gr, "0") == 0) use_graphs = false;
  const char* at = std::getenv("TNS_AUTOTUNE");
  if (at && std::strcmp(at, "0") == 0) autotune = false;
  const char* k = std::getenv("TNS_FP64_KERNEL");
  if (k && std::strcmp(k, "dfma") == 0) fp64_kernel = 0;
  if (k && std::strcmp(k, "dmma") == 0) fp64_kernel = 1;
  const char* w = std::getenv("TNS_TC_WAIT_NS");
  if (w && *w) tc_wait_ns = std::strtoull(w, nullptr, 10);
  const char* tv = std::getenv("TNS_TC_VARIANT");
  if (tv && *tv) {
    const int x = std::atoi(tv);
    if (x >= 0 && x < kNumVariants) forced_tc_variant = x;
  }
  const char* sm = std::getenv("TNS_TC_SMALL");
  if (sm && *sm) tc_small = std::max(0, std::min(32, std::atoi(sm)));
}

CudaBackend::~CudaBackend() {
  for (auto& kv : lists_) free_list(kv.second);
  for (auto& s : scratch_)
    if (s.first) dfree(s.first);
  if (gstream_) cudaStreamDestroy(gstream_);
  for (cudaEvent_t e : gev_)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t f : fstream_)
    if (f) cudaStreamDestroy(f);
  for (cudaEvent_t e : fev_)
    if (e) cudaEventDestroy(e);
  if (own_ && stream_) cudaStreamDestroy(stream_);
}

bool CudaBackend::fork_ready() {
  if (fstream_[0]) return true;
  bool good = true;
  for (int i = 0; i < 3 && good; ++i) good = cudaStreamCreateWithFlags(&fstream_[i], cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < 4 && good; ++i) good = cudaEventCreateWithFlags(&fev_[i], cudaEventDisableTiming) == cudaSuccess;
  if (!good) {
    cudaGetLastError();
    for (cudaStream_t& f : fstream_)
      if (f) {
        cudaStreamDestroy(f);
        f = nullptr;
      }
    for (cudaEvent_t& e : fev_)
      if (e) {
        cudaEventDestroy(e);
        e = nullptr;
      }
  }
  return good;
}

void CudaBackend::note(cudaError_t e, const char* what) {
  if (e != cudaSuccess && err_.empty()) err_ = std::string(what) + ": " + cudaGetErrorString(e);
}

std::string CudaBackend::error() {
  std::string e = err_;
  err_.clear();
  return e;
}

double* CudaBackend::alloc(long long n) {
  void* p = nullptr;
  if (dmalloc(&p, (size_t)n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (double*)p;
}

void CudaBackend::release(double* p) {
  if (p) {
    cudaStreamSynchronize(stream_);
    dfree(p);
  }
}

// the device memory of a step beyond its catalogues and partial sums: the
// work list with its schedules, the tensor-core product records (48 bytes
// for the tile kernel, 16 for the small-block kernels, chunk records), the
// operand images (every distinct operator block, rows padded to 8 and K to
// 32 bytes, 4 bytes per element) and the vectors of a block Davidson
// (subspace, products, X images, graph buffers: about 120 vectors)
long long CudaBackend::step_bytes(const TaskList& tl, long long psi_length) {
  long long b = (long long)tl.tasks.size() * ((long long)sizeof(Task) * 3 / 2 + 48 + 16 + 8) +
                (long long)tl.groups.size() * (long long)sizeof(Group) * 4;
  std::unordered_set<uintptr_t> seenL, seenR;
  auto pad = [](long long rows, long long cols) { return ((rows + 7) / 8 * 8) * ((cols * 4 + 31) / 32 * 32); };
  // an operator block used plain and transposed gets two images
  for (const Task& t : tl.tasks) {
    if (!(t.flags & TF_LI) && seenL.insert((uintptr_t)t.L ^ ((t.flags & TF_LT) ? 1u : 0u)).second) b += pad(t.q, t.m);
    if (!(t.flags & TF_RI) && seenR.insert((uintptr_t)t.R ^ ((t.flags & TF_RT) ? 1u : 0u)).second) b += pad(t.r, t.n);
  }
  // + split-K partial tiles and scratch
  return b + psi_length * 8LL * 120 + (1LL << 30);
}

long long CudaBackend::mem_used() { return dmem(device_).used; }

long long CudaBackend::mem_limit() {
  const long long b = dmem(device_).budget;
  if (b > 0) return b;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (long long)tot;
}

long long CudaBackend::mem_free() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (long long)fr;
}

void CudaBackend::set_budget(long long bytes) { dmem_set_budget(device_, bytes); }

double* CudaBackend::host_alloc(long long n) {
  void* p = nullptr;
  if (cudaMallocHost(&p, (size_t)n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (double*)p;
}

void CudaBackend::host_release(double* p) {
  if (p) {
    cudaStreamSynchronize(stream_);
    cudaFreeHost(p);
  }
}

void CudaBackend::upload(double* dst, const double* src, long long n) {
  note(cudaMemcpyAsync(dst, src, (size_t)n * 8, cudaMemcpyHostToDevice, stream_), "upload");
  note(cudaStreamSynchronize(stream_), "upload");
}

void CudaBackend::download(double* dst, const double* src, long long n) {
  note(cudaMemcpyAsync(dst, src, (size_t)n * 8, cudaMemcpyDeviceToHost, stream_), "download");
  note(cudaStreamSynchronize(stream_), "download");
}

void CudaBackend::zero(double* p, long long n) { note(cudaMemsetAsync(p, 0, (size_t)n * 8, stream_), "zero"); }

void CudaBackend::sync() { note(cudaStreamSynchronize(stream_), "sync"); }

void* CudaBackend::scratch(size_t bytes, int slot) {
  auto& s = scratch_[slot];
  if (s.second < bytes) {
    if (s.first) {
      cudaStreamSynchronize(stream_);
      dfree(s.first);
    }
    s.first = nullptr;
    s.second = 0;
    if (dmalloc(&s.first, bytes) != cudaSuccess) {
      cudaGetLastError();
      note(cudaErrorMemoryAllocation, "scratch");
      return nullptr;
    }
    s.second = bytes;
  }
  return s.first;
}

template <typename T>
static T* dev_copy(const std::vector<T>& v, CudaBackend& be) {
  if (v.empty()) return nullptr;
  void* p = nullptr;
  if (dmalloc(&p, v.size() * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    be.note(cudaErrorMemoryAllocation, "work list upload");
    return nullptr;
  }
  be.note(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, be.stream()), "work list upload");
  return (T*)p;
}

void CudaBackend::free_graphs(DevList& d) {
  if (d.graphs.empty()) return;
  cudaStreamSynchronize(stream_);
  if (gstream_) cudaStreamSynchronize(gstream_);
  for (auto& kv : d.graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.xbuf) dfree(kv.second.xbuf);
    if (kv.second.ybuf) dfree(kv.second.ybuf);
  }
  d.graphs.clear();
}

void CudaBackend::free_list(DevList& d) {
  cudaStreamSynchronize(stream_);
  if (gstream_) cudaStreamSynchronize(gstream_);
  free_graphs(d);
  if (d.tasks) dfree(d.tasks);
  if (d.groups) dfree(d.groups);
  if (d.wtiles) dfree(d.wtiles);
  for (FpVariant& f : d.fv) {
    if (f.tiles) dfree(f.tiles);
    if (f.reds) dfree(f.reds);
    if (f.part) dfree(f.part);
  }
  if (d.tc) release_tc_plan(d.tc);
  d = DevList();
}

// shape signature of a work list: the number of products (octave), the
// product-weighted mean output-block size q*r (octave) and the share of
// products on blocks larger than 64 x 64 (quarters) -- lists of one bond in
// successive sweeps and of neighbouring bonds share it, lists of a very
// different sector structure do not
static unsigned long long shape_signature(const TaskList& tl) {
  unsigned long long h = 1469598103934665603ULL;
  auto mix = [&](long long x) { h = (h ^ (unsigned long long)x) * 1099511628211ULL; };
  const double n = std::max<double>(1.0, (double)tl.tasks.size());
  double wsum = 0.0, big = 0.0;
  for (const Group& g : tl.groups) {
    const double c = g.t1 - g.t0, a = (double)g.q * g.r;
    wsum += c * a;
    if (a > 4096.0) big += c;
  }
  mix((long long)std::floor(std::log2(n)));
  mix((long long)std::floor(std::log2(wsum / n + 1.0)));
  mix((long long)std::floor(4.0 * big / n));
  return h;
}

void CudaBackend::upload_list(const TaskList& tl, DevList& d) {
  free_list(d);
  need((long long)tl.tasks.size() * (long long)sizeof(Task) * 3 / 2 +
       (long long)tl.groups.size() * (long long)sizeof(Group) * 4);
  d.tasks = dev_copy(tl.tasks, *this);
  d.groups = dev_copy(tl.groups, *this);
  std::vector<Tile> wt;
  for (int g = 0; g < (int)tl.groups.size(); ++g) {
    const Group& G = tl.groups[g];
    for (int r0 = 0; r0 < G.q; r0 += DM_WR)
      for (int c0 = 0; c0 < G.r; c0 += DM_WC) {
        Tile t;
        t.g = g;
        t.row0 = r0;
        t.col0 = c0;
        t.nrows = std::min(DM_WR, G.q - r0);
        t.ncols = std::min(DM_WC, G.r - c0);
        t.t0 = G.t0;
        t.t1 = G.t1;
        t.poff = -1;
        wt.push_back(t);
      }
  }
  d.nwtiles = (int)wt.size();
  d.wtiles = dev_copy(wt, *this);
  d.gen = tl.gen;
  d.shape = shape_signature(tl);
  note(cudaStreamSynchronize(stream_), "work list upload");
}

// estimated fixed cost of one product on one tile (loads, barriers), in FMAs
constexpr double kTaskOverhead = 512.0;

// cut an extent into p near-equal parts of at most mx
static std::vector<std::pair<int, int>> cut_extent(int len, int mx) {
  std::vector<std::pair<int, int>> out;
  const int p = (len + mx - 1) / mx;
  for (int i = 0, o = 0; i < p; ++i) {
    const int w = len / p + (i < len % p ? 1 : 0);
    out.push_back({o, w});
    o += w;
  }
  return out;
}

// FP64 output tiles of every group: tall or wide, whichever executes fewer
// FMAs over the group's products (fixed overhead per product and tile
// included), each tile in the smallest class it fits
static void fp64_tiles(const TaskList& tl, DevList& d) {
  for (int c = 0; c < kFpClasses; ++c) {
    d.fp_tiles[c].clear();
    d.fp_cost[c].clear();
  }
  for (int g = 0; g < (int)tl.groups.size(); ++g) {
    const Group& G = tl.groups[g];
    if (G.q <= 0 || G.r <= 0) continue;
    std::vector<std::pair<int, int>> rows[2] = {cut_extent(G.q, kTallR), cut_extent(G.q, kWideR)};
    std::vector<std::pair<int, int>> cols[2] = {cut_extent(G.r, kTallC), cut_extent(G.r, kWideC)};
    double best = -1;
    int pick = 0;
    for (int o = 0; o < 2; ++o) {
      double c = 0;
      for (auto& rr : rows[o])
        for (auto& cc : cols[o])
          for (int t = G.t0; t < G.t1; ++t) c += (double)tile_fmas(tl.tasks[t], rr.second, cc.second, nullptr) + kTaskOverhead;
      if (best < 0 || c < best) {
        best = c;
        pick = o;
      }
    }
    for (auto& rr : rows[pick])
      for (auto& cc : cols[pick]) {
        Tile t;
        t.g = g;
        t.row0 = rr.first;
        t.col0 = cc.first;
        t.nrows = rr.second;
        t.ncols = cc.second;
        t.t0 = G.t0;
        t.t1 = G.t1;
        t.poff = -1;
        double w = 0;
        for (int k = G.t0; k < G.t1; ++k) w += (double)tile_fmas(tl.tasks[k], t.nrows, t.ncols, nullptr) + kTaskOverhead;
        const int c = (t.nrows <= C0_TR && t.ncols <= C0_TC)   ? 0
                      : (t.nrows <= C1_TR && t.ncols <= C1_TC) ? 1
                      : (t.ncols <= C2_TC)                     ? 2
                                                               : 3;
        d.fp_tiles[c].push_back(t);
        d.fp_cost[c].push_back(w);
      }
  }
  d.fp_tiled = true;
}

// schedule variant v of the FP64 kernels: the tiles of each class, a tile
// whose task list is long cut into pieces of similar cost (split-K), each
// written to a partial tile and summed afterwards in piece order, so that
// every class fills the GPU and no CTA walks a much longer list than the rest
void CudaBackend::plan_variant(const TaskList& tl, DevList& d, int v) {
  FpVariant& f = d.fv[v];
  if (f.planned) return;
  // kernel attribute once, outside any stream capture: the wide class needs
  // more than 48 KB of dynamic shared memory
  static bool attr = false;
  if (!attr) {
    note(cudaFuncSetAttribute(k_tasks_fp64<C3_NT, C3_ACC, C3_TR, C3_TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              fp64_smem(C3_TR, C3_TC)),
         "k_tasks_fp64 shared memory");
    attr = true;
  }
  if (!d.fp_tiled) fp64_tiles(tl, d);
  double ctot[kFpClasses] = {0, 0, 0, 0};
  for (int c = 0; c < kFpClasses; ++c)
    for (double w : d.fp_cost[c]) ctot[c] += w;
  // resident CTAs per SM of each class (registers) x SMs x rounds
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device_);
  const double rounds = kRounds[v];
  const double slots[kFpClasses] = {16.0 * sms * rounds, 4.0 * sms * rounds, 2.0 * sms * rounds,
                                    2.0 * sms * rounds};
  std::vector<Tile> all;
  std::vector<SplitRed> reds;
  long long poff = 0;
  for (int c = 0; c < kFpClasses; ++c) {
    const double target = std::max(ctot[c] / slots[c], 1.0);
    int count = 0;
    const size_t first = all.size();
    std::vector<double> pcost;  // estimated cost of each piece of this class
    for (size_t i = 0; i < d.fp_tiles[c].size(); ++i) {
      const Tile t = d.fp_tiles[c][i];
      const double tc = d.fp_cost[c][i];
      const int ntask = t.t1 - t.t0;
      int ns = (int)std::min<double>(ntask, std::ceil(tc / target));
      ns = std::max(1, std::min(ns, 64));
      if (ns == 1) {
        all.push_back(t);
        pcost.push_back(tc);
        ++count;
        continue;
      }
      // cut the task range at equal shares of its cost on this tile
      std::vector<double> kc(ntask);
      double tot = 0;
      for (int k = t.t0; k < t.t1; ++k)
        tot += kc[k - t.t0] = (double)tile_fmas(tl.tasks[k], t.nrows, t.ncols, nullptr) + kTaskOverhead;
      SplitRed R;
      R.g = t.g;
      R.row0 = t.row0;
      R.col0 = t.col0;
      R.nrows = t.nrows;
      R.ncols = t.ncols;
      R.poff = poff;
      int start = t.t0, made = 0;
      double acc = 0, last = 0;
      for (int k = t.t0; k < t.t1 && made < ns - 1; ++k) {
        acc += kc[k - t.t0];
        if (acc >= tot * (made + 1) / ns) {
          Tile p = t;
          p.t0 = start;
          p.t1 = k + 1;
          p.poff = poff;
          poff += (long long)t.nrows * t.ncols;
          all.push_back(p);
          pcost.push_back(acc - last);
          last = acc;
          ++made;
          ++count;
          start = k + 1;
        }
      }
      Tile p = t;
      p.t0 = start;
      p.t1 = t.t1;
      p.poff = poff;
      poff += (long long)t.nrows * t.ncols;
      all.push_back(p);
      pcost.push_back(tot - last);
      ++count;
      R.nsplit = made + 1;
      reds.push_back(R);
    }
    // costliest pieces first: CTAs are dispatched in index order, so the long
    // pieces start in the first wave and the short ones fill in behind them
    std::vector<int> ord(pcost.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return pcost[a] > pcost[b]; });
    std::vector<Tile> sorted(ord.size());
    for (size_t i = 0; i < ord.size(); ++i) sorted[i] = all[first + ord[i]];
    std::copy(sorted.begin(), sorted.end(), all.begin() + first);
    f.ncls[c] = count;
    f.ccost[c] = ctot[c];
  }
  f.psize = poff;
  f.nreds = (int)reds.size();
  f.reds = dev_copy(reds, *this);
  f.ntiles = (int)all.size();
  f.tiles = dev_copy(all, *this);
  f.planned = true;
  note(cudaStreamSynchronize(stream_), "schedule upload");
}

bool CudaBackend::ensure_part(DevList& d, FpVariant& f, int nvec) {
  if (f.psize == 0 || f.part_nvec >= nvec) return true;
  if (f.part) {
    // graphs captured with the smaller buffer would write through a freed pointer
    free_graphs(d);
    cudaStreamSynchronize(stream_);
    if (gstream_) cudaStreamSynchronize(gstream_);
    dfree(f.part);
  }
  f.part = nullptr;
  f.part_nvec = 0;
  if (dmalloc(&f.part, sizeof(double) * f.psize * nvec) != cudaSuccess) {
    cudaGetLastError();
    note(cudaErrorMemoryAllocation, "split partial tiles");
    f.part = nullptr;
    return false;
  }
  f.part_nvec = nvec;
  return true;
}

DevList& CudaBackend::dev(const TaskList& tl) {
  DevList& d = lists_[&tl];
  if (d.gen != tl.gen) upload_list(tl, d);
  return d;
}

void CudaBackend::drop(const TaskList& tl) {
  auto it = lists_.find(&tl);
  if (it != lists_.end()) {
    free_list(it->second);
    lists_.erase(it);
  }
}

void CudaBackend::enqueue_fp64(const DevList& d, int v, const double* xv, double* yv, int nvec, long long xs,
                               long long ys) {
  if (!ok()) return;
  const FpVariant& f = d.fv[v];
  // the classes write disjoint tiles and partial tiles: the costliest class
  // runs on the launching stream and the others on forked streams beside it
  // (they fill its tail), joined before the split reduction
  int order[kFpClasses] = {0, 1, 2, 3};
  std::stable_sort(order, order + kFpClasses, [&](int a, int b) { return f.ccost[a] > f.ccost[b]; });
  const int nact = (f.ncls[0] > 0) + (f.ncls[1] > 0) + (f.ncls[2] > 0) + (f.ncls[3] > 0);
  const bool fork = nact > 1 && fork_ready();
  if (fork) {
    note(cudaEventRecord(fev_[0], stream_), "fork");
    for (int i = 0; i < 3; ++i) note(cudaStreamWaitEvent(fstream_[i], fev_[0], 0), "fork");
  }
  int tbeg[kFpClasses];
  for (int c = 0, t = 0; c < kFpClasses; ++c) {
    tbeg[c] = t;
    t += f.ncls[c];
  }
  int side = 0;
  for (int oi = 0; oi < kFpClasses; ++oi) {
    const int c = order[oi];
    const int n = f.ncls[c];
    if (n == 0) continue;
    const unsigned grid = (unsigned)n * (unsigned)nvec;
    cudaStream_t s = stream_;
    if (fork && oi > 0) s = fstream_[side++];
    const int t0 = tbeg[c];
    if (c == 0)
      k_tasks_fp64<C0_NT, C0_ACC, C0_TR, C0_TC><<<grid, C0_NT, fp64_smem(C0_TR, C0_TC), s>>>(
          d.tasks, d.groups, f.tiles, t0, xv, yv, xs, ys, f.part, f.psize, nvec);
    else if (c == 1)
      k_tasks_fp64<C1_NT, C1_ACC, C1_TR, C1_TC><<<grid, C1_NT, fp64_smem(C1_TR, C1_TC), s>>>(
          d.tasks, d.groups, f.tiles, t0, xv, yv, xs, ys, f.part, f.psize, nvec);
    else if (c == 2)
      k_tasks_fp64<C2_NT, C2_ACC, C2_TR, C2_TC><<<grid, C2_NT, fp64_smem(C2_TR, C2_TC), s>>>(
          d.tasks, d.groups, f.tiles, t0, xv, yv, xs, ys, f.part, f.psize, nvec);
    else
      k_tasks_fp64<C3_NT, C3_ACC, C3_TR, C3_TC><<<grid, C3_NT, fp64_smem(C3_TR, C3_TC), s>>>(
          d.tasks, d.groups, f.tiles, t0, xv, yv, xs, ys, f.part, f.psize, nvec);
    launches++;
    note(cudaGetLastError(), "k_tasks_fp64");
  }
  if (fork) {
    for (int i = 0; i < 3; ++i) {
      note(cudaEventRecord(fev_[1 + i], fstream_[i]), "join");
      note(cudaStreamWaitEvent(stream_, fev_[1 + i], 0), "join");
    }
  }
  if (f.nreds > 0) {
    dim3 grid(std::min(f.nreds, 65535), nvec);
    k_reduce_splits<<<grid, 128, 0, stream_>>>(f.reds, f.nreds, d.groups, f.part, f.psize, yv, ys);
    launches++;
    note(cudaGetLastError(), "k_reduce_splits");
  }
}

// Replay (capturing it first if needed) the launch sequence `enqueue` of one
// (precision, nvec) use of a persistent list as a CUDA graph on the side
// stream, ordered after the context stream's prior work and before its next:
// input copied into the graph's fixed buffer, output copied out.  Falls back
// to direct launches where capture is not possible.
template <class F>
void CudaBackend::launch_graphed(DevList& d, int key, const double* xv, double* yv, int nvec, long long xs,
                                 long long ys, F&& enqueue) {
  GraphSlot& gs = d.graphs[key];
  if (!gs.exec && !gs.failed) need(2LL * (long long)sizeof(double) * nvec * std::max(xs, ys));
  const long long elems = (long long)nvec * xs;
  if (!use_graphs || gs.failed || xs != ys) {
    enqueue(xv, yv);
    return;
  }
  if (!gstream_) {
    if (cudaStreamCreateWithFlags(&gstream_, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&gev_[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&gev_[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      gs.failed = true;
      enqueue(xv, yv);
      return;
    }
  }
  if (!gs.exec) {
    if (dmalloc(&gs.xbuf, sizeof(double) * elems) != cudaSuccess ||
        dmalloc(&gs.ybuf, sizeof(double) * elems) != cudaSuccess) {
      cudaGetLastError();
      gs.failed = true;
      enqueue(xv, yv);
      return;
    }
    gs.elems = elems;
    gs.stride = xs;
    cudaStream_t saved = stream_;
    stream_ = gstream_;
    const long long l0 = launches;
    const std::string saved_err = err_;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(gstream_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      enqueue(gs.xbuf, gs.ybuf);
      ok = cudaStreamEndCapture(gstream_, &g) == cudaSuccess && g;
    }
    stream_ = saved;
    if (ok) ok = cudaGraphInstantiate(&gs.exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    gs.kernels = (int)(launches - l0);
    launches = l0;
    if (!ok) {
      cudaGetLastError();
      err_ = saved_err;
      gs.failed = true;
      gs.exec = nullptr;
      enqueue(xv, yv);
      return;
    }
  }
  note(cudaEventRecord(gev_[0], stream_), "graph order");
  note(cudaStreamWaitEvent(gstream_, gev_[0], 0), "graph order");
  note(cudaMemcpyAsync(gs.xbuf, xv, sizeof(double) * elems, cudaMemcpyDeviceToDevice, gstream_), "graph input");
  note(cudaGraphLaunch(gs.exec, gstream_), "graph launch");
  note(cudaMemcpyAsync(yv, gs.ybuf, sizeof(double) * elems, cudaMemcpyDeviceToDevice, gstream_), "graph output");
  note(cudaEventRecord(gev_[1], gstream_), "graph order");
  note(cudaStreamWaitEvent(stream_, gev_[1], 0), "graph order");
  launches += gs.kernels;
}

void CudaBackend::run(const TaskList& tl, const double* xv, double* yv, int nvec, long long xs, long long ys,
                      int precision) {
  if (!ok()) return;
  if (tl.groups.empty()) return;
  if (!tl.persistent) {
    // one-off list (rotations, truncation products): default schedule, direct launches
    DevList tmp;
    upload_list(tl, tmp);
    if (precision != 0) {
      if (prepare_tasks_tc(*this, tl, tmp, nvec, 1, precision)) {
        enqueue_tasks_tc(*this, tmp, xv, yv, nvec, xs, ys, precision, 1);
        check_tasks_tc(*this, tmp);
      }
    } else if (fp64_kernel == 1) {
      if (tmp.nwtiles > 0) {
        dim3 grid((tmp.nwtiles + DM_WARPS - 1) / DM_WARPS, nvec);
        k_tasks_dmma<<<grid, 32 * DM_WARPS, 0, stream_>>>(tmp.tasks, tmp.groups, tmp.wtiles, tmp.nwtiles, xv, yv, xs,
                                                           ys);
        launches++;
        note(cudaGetLastError(), "k_tasks_dmma");
      }
    } else {
      plan_variant(tl, tmp, 1);
      if (ok() && tmp.tasks && tmp.groups && ensure_part(tmp, tmp.fv[1], nvec)) enqueue_fp64(tmp, 1, xv, yv, nvec, xs, ys);
    }
    free_list(tmp);
    return;
  }
  DevList& d = dev(tl);
  if (!ok() || !d.tasks || !d.groups) return;
  if (precision == 0 && fp64_kernel == 1) {
    if (d.nwtiles > 0) {
      dim3 grid((d.nwtiles + DM_WARPS - 1) / DM_WARPS, nvec);
      k_tasks_dmma<<<grid, 32 * DM_WARPS, 0, stream_>>>(d.tasks, d.groups, d.wtiles, d.nwtiles, xv, yv, xs, ys);
      launches++;
      note(cudaGetLastError(), "k_tasks_dmma");
    }
    return;
  }
  // online autotuner: after one untimed product, the next products of this
  // (precision, nvec) use run the schedule variants in turn, timed with
  // events; the variant with the fastest sample is kept
  const int key = precision * 64 + nvec;
  Tune& tu = d.tune[key];
  if (!autotune && tu.best < 0) tu.best = 1;
  const int nvar = precision != 0 ? kNumVariants : kFp64Variants;
  if (precision != 0 && forced_tc_variant >= 0) tu.best = forced_tc_variant;
  const auto ckey = std::make_pair(key, d.shape);
  if (tu.best < 0 && tu.step == 0 && autotune) {
    auto it = tune_cache_.find(ckey);
    if (it != tune_cache_.end()) {
      tu.best = it->second;
      ++tune_cache_hits;
    }
  }
  const bool tuning = tu.best < 0;
  const bool timing = tuning && tu.step > 0;
  const int v = !tuning ? tu.best : timing ? (tu.step - 1) % nvar : 1;
  if (precision != 0) {
    if (!prepare_tasks_tc(*this, tl, d, nvec, v, precision)) return;
  } else {
    plan_variant(tl, d, v);
    if (!ok() || !ensure_part(d, d.fv[v], nvec)) return;
  }
  auto enqueue = [&](const double* x, double* y) {
    if (precision != 0)
      enqueue_tasks_tc(*this, d, x, y, nvec, xs, ys, precision, v);
    else
      enqueue_fp64(d, v, x, y, nvec, xs, ys);
  };
  if (tuning && !timing) {
    enqueue(xv, yv);
    ++tu.step;
  } else if (timing) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, stream_);
    enqueue(xv, yv);
    cudaEventRecord(b, stream_);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    tu.ms[v] = std::min(tu.ms[v], ms);
    if (++tu.step == 1 + kTuneRounds * nvar) {
      tu.best = 0;
      for (int i = 1; i < nvar; ++i)
        if (tu.ms[i] < tu.ms[tu.best]) tu.best = i;
      tune_cache_[ckey] = tu.best;
      ++tuned;
    }
  } else {
    launch_graphed(d, key, xv, yv, nvec, xs, ys, enqueue);
    if (precision >= 0 && precision < 3) ++variant_runs[precision][v];
  }
  if (precision != 0) check_tasks_tc(*this, d);
}

// out[t] = < Ybar_g, op(L) op(X) op(R)^T > for every task t (alpha excluded):
// one CTA per task; each thread takes elements (k, j) of the m x r product
// P = op(L)^T Ybar and T = op(X) op(R)^T and accumulates P_kj T_kj
__global__ void __launch_bounds__(128) k_task_values(const Task* __restrict__ tasks, const int* __restrict__ tgroup,
                                                     const Group* __restrict__ groups, const double* xv,
                                                     const double* __restrict__ ybar, double* out) {
  const Task T = tasks[blockIdx.x];
  const Group G = groups[tgroup[blockIdx.x]];
  const double* Y = ybar + G.yoff;
  const double* X = (T.flags & TF_XV) ? xv + (long long)(size_t)T.X : T.X;
  double s = 0.0;
  for (long long e = threadIdx.x; e < (long long)T.m * T.r; e += blockDim.x) {
    const int k = (int)(e / T.r), j = (int)(e % T.r);
    double P = 0.0;
    if (T.flags & TF_LI)
      P = Y[(long long)k * G.r + j];
    else
      for (int i = 0; i < T.q; ++i) P = fma(opL(T, i, k), Y[(long long)i * G.r + j], P);
    double V = 0.0;
    if (T.flags & TF_RI)
      V = opX(T, X, k, j);
    else if (T.flags & TF_XI)
      V = opR(T, j, k);
    else
      for (int l = 0; l < T.n; ++l) V = fma(opX(T, X, k, l), opR(T, j, l), V);
    s = fma(P, V, s);
  }
  __shared__ double red[4];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) out[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

void CudaBackend::task_values(const TaskList& tl, const double* xv, const double* ybar, double* out) {
  if (!ok()) return;
  if (tl.tasks.empty()) return;
  std::vector<int> tg(tl.tasks.size(), 0);
  for (int g = 0; g < (int)tl.groups.size(); ++g)
    for (int i = tl.groups[g].t0; i < tl.groups[g].t1; ++i) tg[i] = g;
  Task* dt = dev_copy(tl.tasks, *this);
  Group* dg = dev_copy(tl.groups, *this);
  int* dtg = dev_copy(tg, *this);
  if (dt && dg && dtg) {
    k_task_values<<<(unsigned)tl.tasks.size(), 128, 0, stream_>>>(dt, dtg, dg, xv, ybar, out);
    launches++;
    note(cudaGetLastError(), "k_task_values");
  }
  cudaStreamSynchronize(stream_);
  for (void* p : {(void*)dt, (void*)dg, (void*)dtg})
    if (p) dfree(p);
}

// one warp per block: nz[i] = any element of block i nonzero (HBM-bound read)
__global__ void k_nonzero(const double* const* __restrict__ p, const long long* __restrict__ n, int nb,
                          char* __restrict__ nz) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = w0; i < nb; i += nw) {
    const double* x = p[i];
    const long long len = n[i];
    int any = 0;
    for (long long j = lane; j < len && !any; j += 32) any = x[j] != 0.0;
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) nz[i] = (char)any;
  }
}

void CudaBackend::nonzero_blocks(const std::vector<const double*>& p, const std::vector<long long>& n,
                                 std::vector<char>& nz) {
  nz.assign(p.size(), 1);  // on any failure every block counts as nonzero
  if (!ok() || p.empty()) return;
  const double** dp = dev_copy(p, *this);
  long long* dn = dev_copy(n, *this);
  char* dz = nullptr;
  if (dp && dn && dmalloc(&dz, p.size()) == cudaSuccess) {
    const int nb = (int)p.size();
    const int grid = std::min((nb + 7) / 8, 152 * 16);
    k_nonzero<<<grid, 256, 0, stream_>>>(dp, dn, nb, dz);
    launches++;
    note(cudaGetLastError(), "k_nonzero");
    std::vector<char> h(p.size());
    if (cudaMemcpyAsync(h.data(), dz, p.size(), cudaMemcpyDeviceToHost, stream_) == cudaSuccess &&
        cudaStreamSynchronize(stream_) == cudaSuccess)
      nz = h;
  }
  cudaStreamSynchronize(stream_);
  for (void* q : {(void*)dp, (void*)dn, (void*)dz})
    if (q) dfree(q);
}

void CudaBackend::lincomb(const LCList& l) {
  if (!ok()) return;
  if (l.blocks.empty()) return;
  LCBlock* b = dev_copy(l.blocks, *this);
  LCTerm* t = dev_copy(l.terms, *this);
  if (!b) return;
  int nb = (int)l.blocks.size();
  k_lincomb<<<std::min(nb, 65535), 128, 0, stream_>>>(b, nb, t);
  launches++;
  note(cudaGetLastError(), "k_lincomb");
  cudaStreamSynchronize(stream_);
  dfree(b);
  if (t) dfree(t);
}

}  // namespace tns
