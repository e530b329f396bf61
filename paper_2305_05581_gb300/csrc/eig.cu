// Batched symmetric eigen-decomposition for the truncation (reduced density
// matrix of each sector of the new bond).
//   k_tridiag, one CTA per matrix: Householder tridiagonalisation
//      T = Q^T A Q (Golub & Van Loan, "Matrix Computations", Sec. 8.3.1);
//      reflectors kept in the rows of A (beta on the diagonal), (d, e) to a
//      scratch array.
//   k_tqr, one CTA per (matrix, slice of 32 columns of Z):
//      1. its columns of Z = Q^T, column j = H_{n-3} ... H_0 e_j;
//      2. implicit symmetric QR steps with the Wilkinson shift and deflation
//         (Golub & Van Loan Sec. 8.3.3-8.3.5) on its own copy of (d, e): lane 0
//         computes the Givens rotations of a bulge chase, every lane applies
//         them to one column (rows i, i+1 rotate).  Every slice runs the same
//         chase on the same data, so the slices agree bit for bit and need no
//         communication; the rotation work, which dominates, is spread over
//         ceil(n / 32) SMs instead of one.
// Output: eigenvalues w[woff + p] and eigenvector p as ROW p of Z
// (Z[p * n + i], n x n row-major at off).  A is overwritten.
#include <cuda_runtime.h>

#include <string>

#include "cuda_backend.h"

namespace tns {
namespace {

constexpr int SY_NT = 512;
constexpr int SY_WARPS = SY_NT / 32;

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; every thread gets the result
__device__ double bsum(double v, double* red) {
  v = wsum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < SY_WARPS; ++q) s += red[q];
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(SY_NT) k_tridiag(double* A, double* DE, const long long* off, const int* nn,
                                                   const int* woff, int maxn) {
  extern __shared__ double sm[];
  double* v = sm;              // Householder vector
  double* p = sm + maxn;       // work vector
  double* d = sm + 2 * maxn;   // diagonal of T
  double* e = sm + 3 * maxn;   // sub-diagonal of T (e[i] couples i, i+1)
  __shared__ double red[SY_WARPS];
  const int mi = blockIdx.x;
  const int n = nn[mi];
  if (n <= 0) return;
  double* a = A + off[mi];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k = 0; k + 2 < n; ++k) {
    const long long rk = (long long)k * n;
    // x = a[k][k+1 .. n-1] (row k = column k by symmetry)
    double sg = 0.0;
    for (int j = k + 2 + tid; j < n; j += SY_NT) sg += a[rk + j] * a[rk + j];
    sg = bsum(sg, red);
    const double alpha = a[rk + k + 1];
    double beta = 0.0, mu = alpha, v0 = 1.0;
    if (sg > 0.0) {
      mu = sqrt(alpha * alpha + sg);
      v0 = alpha <= 0.0 ? alpha - mu : -sg / (alpha + mu);
      beta = 2.0 * v0 * v0 / (sg + v0 * v0);
    }
    if (tid == 0) {
      d[k] = a[rk + k];
      e[k] = sg > 0.0 ? mu : alpha;
    }
    for (int j = k + 1 + tid; j < n; j += SY_NT) v[j] = j == k + 1 ? 1.0 : a[rk + j] / v0;
    __syncthreads();
    if (beta != 0.0) {
      // p = beta * A_sub v (one warp per row, coalesced)
      for (int i = k + 1 + wid; i < n; i += SY_WARPS) {
        const long long ri = (long long)i * n;
        double s = 0.0;
        for (int j = k + 1 + lane; j < n; j += 32) s += a[ri + j] * v[j];
        s = wsum(s);
        if (lane == 0) p[i] = beta * s;
      }
      __syncthreads();
      double pv = 0.0;
      for (int j = k + 1 + tid; j < n; j += SY_NT) pv += p[j] * v[j];
      pv = bsum(pv, red);
      const double K = 0.5 * beta * pv;
      for (int j = k + 1 + tid; j < n; j += SY_NT) p[j] -= K * v[j];
      __syncthreads();
      // A_sub -= v p^T + p v^T
      const int m = n - k - 1;
      for (long long t = tid; t < (long long)m * m; t += SY_NT) {
        const int i = k + 1 + (int)(t / m), j = k + 1 + (int)(t % m);
        a[(long long)i * n + j] -= v[i] * p[j] + p[i] * v[j];
      }
    }
    // keep the reflector: v (without its leading 1) in row k, beta on the diagonal
    for (int j = k + 2 + tid; j < n; j += SY_NT) a[rk + j] = v[j];
    __syncthreads();
    if (tid == 0) a[rk + k] = beta;
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = a[(long long)(n - 2) * n + n - 2];
      e[n - 2] = a[(long long)(n - 2) * n + n - 1];
    }
    d[n - 1] = a[(long long)(n - 1) * n + n - 1];
  }
  __syncthreads();
  // (d, e) of matrix mi at DE + 2 * woff: d[0..n), e[0..n-1)
  double* de = DE + 2 * (long long)woff[mi];
  for (int i = tid; i < n; i += SY_NT) {
    de[i] = d[i];
    de[n + i] = i + 1 < n ? e[i] : 0.0;
  }
}

constexpr int TQ_COLS = 32;   // columns of Z per CTA (one per lane of warp 0)
constexpr int TQ_NT = 128;    // 4 row phases x 32 columns while building Q^T
constexpr int TQ_PH = TQ_NT / TQ_COLS;

__global__ void __launch_bounds__(TQ_NT) k_tqr(const double* A, double* Zall, double* w, const double* DE,
                                               const long long* off, const int* nn, const int* woff, int maxn,
                                               int* status) {
  extern __shared__ double sm[];
  double* v = sm;              // reflector; then two slots of rotations (cos, sin) in sm[0, 4 maxn)
  double* d = sm + 4 * maxn;
  double* e = sm + 5 * maxn;
  __shared__ double red[TQ_PH][TQ_COLS];
  __shared__ int ctl[9];       // lo, hi, done; per slot: lo, hi, done
  const int mi = blockIdx.x;
  const int n = nn[mi];
  const int j0 = blockIdx.y * TQ_COLS;
  if (n <= 0 || j0 >= n) return;
  const int cw = min(TQ_COLS, n - j0);
  const double* a = A + off[mi];
  double* Z = Zall + off[mi];
  const int tid = threadIdx.x, lane = tid & 31, ph = tid / TQ_COLS;
  const double eps = 2.220446049250313e-16;
  const double* de = DE + 2 * (long long)woff[mi];
  for (int i = tid; i < n; i += TQ_NT) {
    d[i] = de[i];
    e[i] = de[n + i];
  }
  // ---- 1. columns j0 .. j0+cw of Z = Q^T = H_{n-3} ... H_0 ----------------
  const int jc = j0 + lane;  // this thread's column (lane < cw)
  for (int r = ph; r < n; r += TQ_PH)
    if (lane < cw) Z[(long long)r * n + jc] = r == jc ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const long long rk = (long long)k * n;
    const double beta = a[rk + k];
    if (beta == 0.0) continue;  // uniform across the block
    for (int r = k + 1 + tid; r < n; r += TQ_NT) v[r] = r == k + 1 ? 1.0 : a[rk + r];
    __syncthreads();
    double s = 0.0;
    if (lane < cw)
      for (int r = k + 1 + ph; r < n; r += TQ_PH) s += v[r] * Z[(long long)r * n + jc];
    red[ph][lane] = s;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < TQ_PH; ++q) t += red[q][lane];
    t *= beta;
    if (lane < cw)
      for (int r = k + 1 + ph; r < n; r += TQ_PH) Z[(long long)r * n + jc] -= t * v[r];
    __syncthreads();
  }
  // ---- 2. implicit symmetric QR with Wilkinson shift -----------------------
  // warp 1 (lane 0) computes the bulge chases, warp 0 applies them to the
  // columns: chase t+1 is computed while chase t is applied (rotations
  // double-buffered in cs[t & 1], one 64-thread named barrier per chase)
  if (tid >= 64) return;  // only named barriers over warps 0 and 1 below
  double* cs[2] = {v, v + 2 * maxn};  // cos at [i], sin at [maxn + i]
  const int max_steps = 40 * n + 40;
  int hi_state = n - 1;  // producer: bottom of the unreduced part
  for (int t = 0;; ++t) {
    if (tid == 32) {
      double* cc = cs[t & 1];
      double* ss = cc + maxn;
      int hi = hi_state, lo = 0, done = 0;
      // deflate from the bottom
      while (hi > 0) {
        const double b = fabs(e[hi - 1]);
        if (b <= eps * (fabs(d[hi - 1]) + fabs(d[hi])) || b < 1e-300) {
          e[hi - 1] = 0.0;
          --hi;
        } else {
          break;
        }
      }
      if (hi == 0) {
        done = 1;
      } else {
        lo = hi - 1;
        while (lo > 0) {
          const double b = fabs(e[lo - 1]);
          if (b <= eps * (fabs(d[lo - 1]) + fabs(d[lo])) || b < 1e-300) {
            e[lo - 1] = 0.0;
            break;
          }
          --lo;
        }
        // Wilkinson shift from the trailing 2x2 of the block
        const double dl = 0.5 * (d[hi - 1] - d[hi]);
        const double bb = e[hi - 1] * e[hi - 1];
        const double den = dl + (dl >= 0.0 ? 1.0 : -1.0) * sqrt(dl * dl + bb);
        const double mu = den != 0.0 ? d[hi] - bb / den : d[hi];
        // the chase with d[i], e[i] carried in registers and the next
        // diagonal / off-diagonal entries loaded one step ahead
        double ai = d[lo], b = e[lo];
        double x = ai - mu, z = b;
        double aj_n = d[lo + 1], e_n = lo + 1 < hi ? e[lo + 1] : 0.0;
        for (int i = lo; i < hi; ++i) {
          const double aj = aj_n, en = e_n;
          if (i + 1 < hi) {
            aj_n = d[i + 2];
            e_n = i + 2 < hi ? e[i + 2] : 0.0;
          }
          // Givens rotation zeroing z against x
          double c = 1.0, sn = 0.0, r = 0.0;
          const double q = x * x + z * z;
          if (q >= 1e-280 && q <= 1e280) {
            const double ri = rsqrt(q);
            c = x * ri;
            sn = z * ri;
            r = q * ri;
          } else if (x != 0.0 || z != 0.0) {
            const double ri = rhypot(x, z);
            c = x * ri;
            sn = z * ri;
            r = c * x + sn * z;
          }
          if (i > lo) e[i - 1] = r;
          const double cs2 = 2.0 * c * sn * b;
          d[i] = c * c * ai + cs2 + sn * sn * aj;
          const double dj = sn * sn * ai - cs2 + c * c * aj;
          const double ei = c * sn * (aj - ai) + (c * c - sn * sn) * b;
          e[i] = ei;
          x = ei;
          if (i + 1 < hi) {
            z = sn * en;  // bulge at (i, i+2)
            b = c * en;
          }
          ai = dj;
          cc[i] = c;
          ss[i] = sn;
        }
        d[hi] = ai;
      }
      hi_state = hi;
      ctl[0] = lo;
      ctl[1] = hi;
      ctl[2] = done;
      ctl[3 + (t & 1)] = lo;  // slot copies for the consumer
      ctl[5 + (t & 1)] = hi;
      ctl[7 + (t & 1)] = done;
    }
    // chase t is in cs[t & 1]; chase t-1 has been applied
    asm volatile("bar.sync 1, 64;" ::: "memory");
    if (ctl[7 + (t & 1)]) break;
    if (t > max_steps) {
      if (tid == 0 && status) atomicExch(status, 1);
      break;
    }
    if (tid < 32 && lane < cw) {
      const int lo = ctl[3 + (t & 1)], hi = ctl[5 + (t & 1)];
      const double* cc = cs[t & 1];
      const double* ss = cc + maxn;
      double carry = Z[(long long)lo * n + jc];
      int i = lo;
      // every original row is read once (as y) before its row is written, so
      // the loads of the next 8 rows are issued together ahead of the stores
      for (; i + 8 <= hi; i += 8) {
        double y[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) y[q] = Z[(long long)(i + 1 + q) * n + jc];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const double c = cc[i + q], sn = ss[i + q];
          Z[(long long)(i + q) * n + jc] = c * carry + sn * y[q];
          carry = -sn * carry + c * y[q];
        }
      }
      for (; i < hi; ++i) {
        const double y = Z[(long long)(i + 1) * n + jc];
        const double c = cc[i], sn = ss[i];
        Z[(long long)i * n + jc] = c * carry + sn * y;
        carry = -sn * carry + c * y;
      }
      Z[(long long)hi * n + jc] = carry;
    }
  }
  if (blockIdx.y == 0 && tid >= 32)
    for (int i = lane; i < n; i += 32) w[woff[mi] + i] = d[i];
}

}  // namespace

void launch_syev(CudaBackend& be, double* A, double* Z, double* w, const long long* off, const int* n,
                 const int* woff, int nmat, int maxn, int* status) {
  if (nmat <= 0 || maxn <= 0 || !be.ok()) return;
  {
    // an error left pending by an earlier call would otherwise be reported
    // as this launch's
    const cudaError_t pending = cudaGetLastError();
    if (pending != cudaSuccess) {
      be.note(pending, "pending CUDA error before the truncation eigensolver");
      return;
    }
  }
  if (maxn > SYEV_MAXN) {
    be.note(cudaErrorInvalidValue, "syev: matrix too large");
    return;
  }
  // (d, e) of every matrix: 2 * sum(n) doubles, sum(n) <= nmat * maxn
  double* DE = (double*)be.scratch(sizeof(double) * 2 * (size_t)nmat * maxn + 64, 3);
  if (!DE) return;
  const size_t smem = sizeof(double) * 4 * (size_t)maxn, smem_q = sizeof(double) * 6 * (size_t)maxn;
  // the dynamic shared memory of both kernels is set on every call: with the
  // kernels' static shared memory a request just below 48 KB can already
  // exceed the default limit
  {
    cudaError_t e = cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tqr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_q);
    if (e != cudaSuccess) {
      cudaGetLastError();
      be.note(e, "syev: shared memory attribute");
      return;
    }
  }
  k_tridiag<<<nmat, SY_NT, smem, be.stream()>>>(A, DE, off, n, woff, maxn);
  be.launches++;
  be.note(cudaGetLastError(), "syev tridiagonalisation");
  dim3 grid(nmat, (maxn + TQ_COLS - 1) / TQ_COLS);
  k_tqr<<<grid, TQ_NT, smem_q, be.stream()>>>(A, Z, w, DE, off, n, woff, maxn, status);
  be.launches++;
  {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      const std::string what = "syev QR (" + std::to_string(nmat) + " matrices, largest " + std::to_string(maxn) +
                               ", " + std::to_string(smem_q) + " bytes of shared memory)";
      be.note(e, what.c_str());
    }
  }
}

}  // namespace tns
