// Device kernels of the H^2 product: segmented batched small GEMM (float64), the
// batched normalised-Gram eigen-decomposition with truncation (Sec. III-C, IV-C),
// and the permutations between user order and padded tree order.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "internal.hpp"

namespace h2 {

struct Arenas {
  double* p[kArenas];
};

__device__ __forceinline__ double* resolve(const Arenas& a, int64_t t) {
  return a.p[(t >> kTagShift) & 7] + (t & kOffMask);
}

// ------------------------------------------------------------ segmented GEMM
// One CTA per segment (blockIdx.x) and 64-column slice (blockIdx.y); the CTA
// walks 64 x 64 output tiles, each thread owning rows ty + 16 i, cols tx + 16 j.
constexpr int GT = 64, GK = 32, GPAD = 65;

__global__ void __launch_bounds__(256) seg_gemm_kernel(const Seg* __restrict__ segs,
                                                       const Item* __restrict__ items, int64_t first,
                                                       Arenas ar) {
  __shared__ double sA[GK * GPAD];
  __shared__ double sB[GK * GPAD];
  const Seg s = segs[first + blockIdx.x];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool ta = s.flags & SF_TA, tb = s.flags & SF_TB, accum = s.flags & SF_ACC;
  double* out = resolve(ar, s.out);
  const Item* it = items + s.first;
  for (int n0 = blockIdx.y * GT; n0 < s.n; n0 += gridDim.y * GT) {
    for (int m0 = 0; m0 < s.m; m0 += GT) {
      double acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
      if (s.flags & SF_SUM) {
        for (int q = 0; q < s.count; ++q) {
          const double* A = resolve(ar, it[q].a);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              int r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
              if (r < s.m && c < s.n) acc[i][j] += A[(int64_t)r * s.lda + c];
            }
        }
      } else {
        for (int q = 0; q < s.count; ++q) {
          const double* A = resolve(ar, it[q].a);
          const double* B = resolve(ar, it[q].b);
          for (int k0 = 0; k0 < s.k; k0 += GK) {
            for (int e = tid; e < GT * GK; e += 256) {
              int r, kk;
              if (ta) { r = e % GT; kk = e / GT; } else { kk = e % GK; r = e / GK; }
              int gr = m0 + r, gk = k0 + kk;
              double v = 0.0;
              if (gr < s.m && gk < s.k) v = ta ? A[(int64_t)gk * s.lda + gr] : A[(int64_t)gr * s.lda + gk];
              sA[kk * GPAD + r] = v;
              int c;
              if (tb) { kk = e % GK; c = e / GK; } else { c = e % GT; kk = e / GT; }
              int gc = n0 + c;
              gk = k0 + kk;
              double w = 0.0;
              if (gc < s.n && gk < s.k) w = tb ? B[(int64_t)gc * s.ldb + gk] : B[(int64_t)gk * s.ldb + gc];
              sB[kk * GPAD + c] = w;
            }
            __syncthreads();
            const int kl = min(GK, s.k - k0);
            for (int kk = 0; kk < kl; ++kk) {
              double a[4], b[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) a[i] = sA[kk * GPAD + ty + 16 * i];
#pragma unroll
              for (int j = 0; j < 4; ++j) b[j] = sB[kk * GPAD + tx + 16 * j];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
          if (r < s.m && c < s.n) {
            double* o = out + (int64_t)r * s.ldc + c;
            *o = accum ? *o + acc[i][j] : acc[i][j];
          }
        }
    }
  }
}

void launch_gemm(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, double* const arenas[kArenas],
                 int maxn, void* stream) {
  Arenas ar;
  for (int i = 0; i < kArenas; ++i) ar.p[i] = arenas[i];
  const int64_t kMaxGrid = 2147483647LL;
  int gy = (maxn + GT - 1) / GT;
  if (gy < 1) gy = 1;
  if (gy > 256) gy = 256;
  for (int64_t off = 0; off < count; off += kMaxGrid) {
    int64_t c = count - off < kMaxGrid ? count - off : kMaxGrid;
    dim3 grid((unsigned)c, (unsigned)gy);
    seg_gemm_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_segs, d_items, first + off, ar);
  }
}

// ------------------------------------------------------------ eigen + truncation
// Cyclic two-sided Jacobi with the round-robin (tournament) ordering: each step
// applies n/2 disjoint rotations in parallel; a sweep is n-1 steps.  The rotation
// zeroing a_pq is the symmetric 2 x 2 Schur rotation: tau = (a_qq - a_pp)/(2 a_pq),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c.
constexpr int kEigSmemMax = 112;

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

__global__ void __launch_bounds__(256) eig_kernel(const EigTask* __restrict__ tasks, int64_t first, Arenas ar,
                                                  int32_t* kr, int32_t* kc, double eps, int trunc,
                                                  unsigned long long* cap_hits, double* scratch,
                                                  int64_t scratch_stride) {
  extern __shared__ double smem[];
  __shared__ int act[256];
  __shared__ double red[8];
  __shared__ double cs[128], sn[128];
  __shared__ int pp[128], qq[128];
  __shared__ int order[256];
  __shared__ double lam[256];
  __shared__ int s_n, s_rank;
  const EigTask t = tasks[first + blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x;
  int32_t* ranks = t.col ? kc : kr;
  if (tid == 0) {
    int n = 0;
    if (t.child1 < 0) {
      for (int a = 0; a < t.nleaf; ++a) act[n++] = a;
    } else {
      int k1 = ranks[t.child1], k2 = ranks[t.child2];
      for (int a = 0; a < k1; ++a) act[n++] = a;
      for (int a = 0; a < k2; ++a) act[n++] = t.half + a;
    }
    s_n = n;
  }
  __syncthreads();
  const int n = s_n;
  const int nn = n + (n & 1);
  double *A, *V;
  if (nn <= kEigSmemMax) {
    A = smem;
    V = smem + nn * nn;
  } else {
    A = scratch + blockIdx.x * scratch_stride;
    V = A + (int64_t)nn * nn;
  }
  // normalised sum of the Gram matrices over the active rows/cols
  for (int e = tid; e < nn * nn; e += nt) A[e] = 0.0;
  __syncthreads();
  for (int m = 0; m < 3; ++m) {
    if (t.g[m] < 0) continue;
    const double* G = resolve(ar, t.g[m]);
    double loc = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      double v = G[(int64_t)act[e / n] * t.n_pad + act[e % n]];
      loc += v * v;
    }
    double nrm2 = block_sum(loc, red);
    if (nrm2 > 0.0) {
      double inv = 1.0 / sqrt(nrm2);
      for (int e = tid; e < n * n; e += nt) A[(e / n) * nn + (e % n)] += G[(int64_t)act[e / n] * t.n_pad + act[e % n]] * inv;
    }
    __syncthreads();
  }
  // symmetrise (the Grams are symmetric up to rounding of their products)
  for (int e = tid; e < nn * nn; e += nt) {
    int a = e / nn, b = e % nn;
    V[e] = (a == b) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < nn * nn; e += nt) {
    int a = e / nn, b = e % nn;
    if (a < b) {
      double v = 0.5 * (A[a * nn + b] + A[b * nn + a]);
      A[a * nn + b] = v;
      A[b * nn + a] = v;
    }
  }
  __syncthreads();
  const int np = nn / 2;
  for (int sweep = 0; sweep < 30 && nn > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < nn * nn; e += nt) {
      double v = A[e] * A[e];
      tot += v;
      if (e / nn != e % nn) off += v;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (!(off > 1e-30 * tot)) break;
    for (int step = 0; step < nn - 1; ++step) {
      for (int k = tid; k < np; k += nt) {
        int pa = (k == 0) ? 0 : ((k - 1 + step) % (nn - 1)) + 1;
        int pb = ((nn - 1 - k - 1 + step) % (nn - 1)) + 1;
        int p = min(pa, pb), q = max(pa, pb);
        double apq = A[p * nn + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          double tau = (A[q * nn + q] - A[p * nn + p]) / (2.0 * apq);
          double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
        }
        pp[k] = p;
        qq[k] = q;
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      for (int e = tid; e < np * nn; e += nt) {  // rows p, q
        int k = e / nn, j = e % nn;
        if (sn[k] == 0.0) continue;
        int p = pp[k], q = qq[k];
        double x = A[p * nn + j], y = A[q * nn + j];
        A[p * nn + j] = cs[k] * x - sn[k] * y;
        A[q * nn + j] = sn[k] * x + cs[k] * y;
      }
      __syncthreads();
      for (int e = tid; e < np * nn; e += nt) {  // columns p, q of A and V
        int k = e / nn, i = e % nn;
        if (sn[k] == 0.0) continue;
        int p = pp[k], q = qq[k];
        double x = A[i * nn + p], y = A[i * nn + q];
        A[i * nn + p] = cs[k] * x - sn[k] * y;
        A[i * nn + q] = sn[k] * x + cs[k] * y;
        double vx = V[i * nn + p], vy = V[i * nn + q];
        V[i * nn + p] = cs[k] * vx - sn[k] * vy;
        V[i * nn + q] = sn[k] * vx + cs[k] * vy;
      }
      __syncthreads();
    }
  }
  // order by decreasing eigenvalue (ties by index); only the n active ones
  for (int a = tid; a < n; a += nt) lam[a] = A[a * nn + a];
  __syncthreads();
  for (int a = tid; a < n; a += nt) {
    int pos = 0;
    for (int b = 0; b < n; ++b)
      if (lam[b] > lam[a] || (lam[b] == lam[a] && b < a)) ++pos;
    order[pos] = a;
  }
  __syncthreads();
  if (tid == 0) {
    int r = 0;
    if (n > 0) {
      if (trunc == H2_TRUNC_FULL) {
        r = n;
      } else {
        double l1 = lam[order[0]];
        double thr = trunc == H2_TRUNC_SV ? eps * eps : eps;
        if (l1 > 0.0)
          while (r < n && lam[order[r]] > thr * l1) ++r;
      }
    }
    if (r > t.kcap) {
      r = t.kcap;
      atomicAdd(cap_hits, 1ull);
    }
    s_rank = r;
    ranks[t.rank_out] = r;
  }
  __syncthreads();
  const int rank = s_rank;
  double* out = resolve(ar, t.out);
  for (int e = tid; e < t.n_pad * t.kcap; e += nt) out[e] = 0.0;
  __syncthreads();
  // sign: the entry of largest magnitude (first such) is positive
  for (int c = tid; c < rank; c += nt) {
    int col = order[c];
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < n; ++a) {
      double v = fabs(V[a * nn + col]);
      if (v > bv) { bv = v; best = a; }
    }
    double sg = V[best * nn + col] < 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < n; ++a) out[(int64_t)act[a] * t.kcap + c] = sg * V[a * nn + col];
  }
}

void launch_eig(const EigTask* d_eigs, int64_t first, int64_t count, double* const arenas[kArenas], int32_t* kr,
                int32_t* kc, double eps, int trunc, unsigned long long* cap_hits, int max_npad, double* scratch,
                void* stream) {
  Arenas ar;
  for (int i = 0; i < kArenas; ++i) ar.p[i] = arenas[i];
  int nn = max_npad + (max_npad & 1);
  size_t smem = 0;
  int64_t stride = 0;
  if (nn <= kEigSmemMax) {
    smem = (size_t)2 * nn * nn * sizeof(double);
  } else {
    smem = (size_t)2 * kEigSmemMax * kEigSmemMax * sizeof(double);
    stride = (int64_t)2 * nn * nn;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * kEigSmemMax * kEigSmemMax * sizeof(double)));
    attr = true;
  }
  eig_kernel<<<(unsigned)count, 256, smem, (cudaStream_t)stream>>>(d_eigs, first, ar, kr, kc, eps, trunc, cap_hits,
                                                                     scratch, stride);
}

// ------------------------------------------------------------ permutations
// padded tree row pr = leaf * LS + local <-> user index user[pr] (-1 for padding)
__global__ void to_tree_kernel(const double* __restrict__ x, double* __restrict__ xt, const int64_t* __restrict__ user,
                               int64_t rows, int64_t n, int64_t nrhs) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * nrhs) return;
  int64_t pr = e / nrhs, c = e % nrhs;
  int64_t u = user[pr];
  xt[e] = u >= 0 ? x[u + c * n] : 0.0;
}

__global__ void from_tree_kernel(const double* __restrict__ yt, double* __restrict__ y, const int64_t* __restrict__ user,
                                 int64_t rows, int64_t n, int64_t nrhs) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * nrhs) return;
  int64_t pr = e / nrhs, c = e % nrhs;
  int64_t u = user[pr];
  if (u >= 0) y[u + c * n] = yt[e];
}

__global__ void identity_kernel(double* out, int64_t n) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  out[e] = (e / n == e % n) ? 1.0 : 0.0;
}

void launch_identity(double* out, int64_t n, void* stream) {
  identity_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(out, n);
}

void launch_permute(const double* src, double* dst, const int64_t* user, int64_t rows, int64_t n, int64_t nrhs,
                    bool to_tree, void* stream) {
  int64_t tot = rows * nrhs;
  unsigned blocks = (unsigned)((tot + 255) / 256);
  if (to_tree)
    to_tree_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(src, dst, user, rows, n, nrhs);
  else
    from_tree_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(src, dst, user, rows, n, nrhs);
}

}  // namespace h2
