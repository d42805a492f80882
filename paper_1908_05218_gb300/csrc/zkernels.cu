// Complex kernels of the product for complex kernel functions (the Helmholtz kernel
// exp(-j k r) / (4 pi r) of the scattering workloads, Sec. VI-B): the segmented batched
// GEMM with a conjugation flag per operand (complex float64, and complex float32 for
// the mixed product), the Hermitian eigen-decomposition with truncation (Sec. III-C,
// IV-C; float64, reading float32 or float64 Gram matrices), and the permutations of
// complex vectors.
//
// Complex numbers are double2 / float2 (x = real part, y = imaginary part); arenas of a
// complex matrix hold complex elements at the same offsets as a real matrix holds reals
// (an arena's float32 bit selects float2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "device.cuh"
#include "internal.hpp"

namespace h2 {

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a * b
__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ const double2* zptr(const Arenas* a, int64_t t) {
  return (const double2*)a->p[arena_idx(t)] + (t & kOffMask);
}
__device__ __forceinline__ double2* zptr_w(const Arenas* a, int64_t t) {
  return (double2*)a->p[arena_idx(t)] + (t & kOffMask);
}
// element i of a complex matrix in float32 or float64 storage, as double2
__device__ __forceinline__ double2 zld(const Arenas* a, int64_t t, int64_t i) {
  const int ai = arena_idx(t);
  if ((a->f32 >> ai) & 1) {
    const float2 v = ((const float2*)a->p[ai] + (t & kOffMask))[i];
    return make_double2((double)v.x, (double)v.y);
  }
  return ((const double2*)a->p[ai] + (t & kOffMask))[i];
}
__device__ __forceinline__ float2 cmul_add(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}

// ------------------------------------------------------------ complex segmented GEMM
// The segments of the product program (plan.cpp) over complex operands: out (=|+=)
// sum over items of op(A) op(B), op = optional transpose (SF_TA / SF_TB) and optional
// complex conjugation (SF_CA / SF_CB, which the program sets from the paper's formulas:
// V^H for row bases, V^T and conj(V) for column bases, Z Z^H and Z^T conj(Z) for Gram
// matrices).  One CTA of 64 threads per segment walks 32 x 32 output tiles; thread (tx,
// ty) owns a 4 x 4 block; k slices of 16 complex values are staged in shared memory.
constexpr int ZK = 16, ZT = 32, ZPAD = ZT + 1, ZNT = 64;

__global__ void __launch_bounds__(ZNT) seg_zgemm_kernel(const Seg* __restrict__ segs, const Item* __restrict__ items,
                                                        int64_t first, const Arenas* __restrict__ ars) {
  __shared__ double2 sA[ZK][ZPAD];
  __shared__ double2 sB[ZK][ZPAD];
  const Seg s = segs[first + blockIdx.x];
  const Arenas* ar = ars + s.inst;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const bool ta = s.flags & SF_TA, tb = s.flags & SF_TB, accum = s.flags & SF_ACC;
  const bool ca = s.flags & SF_CA, cb = s.flags & SF_CB;
  const int M = bound(ar, s.mref, s.m), N = bound(ar, s.nref, s.n);
  double2* out = zptr_w(ar, s.out);
  const Item* it = items + s.first;
  unsigned long long work = 0;
  for (int n0 = blockIdx.y * ZT; n0 < N; n0 += gridDim.y * ZT) {
    const int nc = min(ZT, N - n0);
    for (int m0 = 0; m0 < M; m0 += ZT) {
      const int mc = min(ZT, M - m0);
      double2 acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
      if (s.flags & SF_SUM) {
        for (int q = 0; q < s.count; ++q) {
          const double2* A = zptr(ar, it[q].a);
          for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
              const int r = 4 * ty + i, c = 4 * tx + j;
              if (r < mc && c < nc) {
                const double2 v = A[(int64_t)(m0 + r) * s.lda + n0 + c];
                acc[i][j].x += v.x;
                acc[i][j].y += v.y;
              }
            }
        }
      } else {
        for (int q = 0; q < s.count; ++q) {
          const Item iq = it[q];
          const int K = bound(ar, iq.kref, iq.kpad ? iq.kpad : s.k);
          const double2* A = zptr(ar, iq.a);
          const double2* B = zptr(ar, iq.b);
          const int lda = iq.lda ? iq.lda : s.lda, ldb = iq.ldb ? iq.ldb : s.ldb;
          for (int k0 = 0; k0 < K; k0 += ZK) {
            const int kc = min(ZK, K - k0);
            for (int e = tid; e < ZK * ZT; e += ZNT) {
              const int kk = e / ZT, r = e % ZT;
              double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
              if (kk < kc && r < mc) va = ta ? A[(int64_t)(k0 + kk) * lda + m0 + r] : A[(int64_t)(m0 + r) * lda + k0 + kk];
              if (kk < kc && r < nc) vb = tb ? B[(int64_t)(n0 + r) * ldb + k0 + kk] : B[(int64_t)(k0 + kk) * ldb + n0 + r];
              sA[kk][r] = ca ? zconj(va) : va;
              sB[kk][r] = cb ? zconj(vb) : vb;
            }
            __syncthreads();
            for (int kk = 0; kk < kc; ++kk) {
              double2 a[4], b[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) a[i] = sA[kk][4 * ty + i];
#pragma unroll
              for (int j = 0; j < 4; ++j) b[j] = sB[kk][4 * tx + j];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = zfma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
            work += 8ull * mc * nc * kc;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = 4 * ty + i, c = 4 * tx + j;
          if (r < mc && c < nc) {
            double2* p = out + (int64_t)(m0 + r) * s.ldc + n0 + c;
            if (accum) {
              double2 v = *p;
              v.x += acc[i][j].x;
              v.y += acc[i][j].y;
              *p = v;
            } else {
              *p = acc[i][j];
            }
          }
        }
    }
  }
  if (ar->flops && tid == 0 && work) atomicAdd(ar->flops, work);
}

// The same segments in complex float32 (the mixed product): every operand is float2
// (float copies of A and B, float work regions, the float shadow of C's bases); sums
// in float32; the output is float2 or, in C's arena, double2.
__global__ void __launch_bounds__(ZNT) seg_zgemm32_kernel(const Seg* __restrict__ segs, const Item* __restrict__ items,
                                                          int64_t first, const Arenas* __restrict__ ars) {
  __shared__ float2 sA[ZK][ZPAD];
  __shared__ float2 sB[ZK][ZPAD];
  const Seg s = segs[first + blockIdx.x];
  const Arenas* ar = ars + s.inst;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const bool ta = s.flags & SF_TA, tb = s.flags & SF_TB, accum = s.flags & SF_ACC;
  const bool ca = s.flags & SF_CA, cb = s.flags & SF_CB;
  const int M = bound(ar, s.mref, s.m), N = bound(ar, s.nref, s.n);
  const int oa = arena_idx(s.out);
  const bool out32 = (ar->f32 >> oa) & 1;
  char* obase = ar->p[oa];
  const int64_t ooff = s.out & kOffMask;
  const Item* it = items + s.first;
  unsigned long long work = 0;
  for (int n0 = blockIdx.y * ZT; n0 < N; n0 += gridDim.y * ZT) {
    const int nc = min(ZT, N - n0);
    for (int m0 = 0; m0 < M; m0 += ZT) {
      const int mc = min(ZT, M - m0);
      float2 acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
      if (s.flags & SF_SUM) {
        for (int q = 0; q < s.count; ++q) {
          const float2* A = (const float2*)ar->p[arena_idx(it[q].a)] + (it[q].a & kOffMask);
          for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
              const int r = 4 * ty + i, c = 4 * tx + j;
              if (r < mc && c < nc) {
                const float2 v = A[(int64_t)(m0 + r) * s.lda + n0 + c];
                acc[i][j].x += v.x;
                acc[i][j].y += v.y;
              }
            }
        }
      } else {
        for (int q = 0; q < s.count; ++q) {
          const Item iq = it[q];
          const int K = bound(ar, iq.kref, iq.kpad ? iq.kpad : s.k);
          const float2* A = (const float2*)ar->p[arena_idx(iq.a)] + (iq.a & kOffMask);
          const float2* B = (const float2*)ar->p[arena_idx(iq.b)] + (iq.b & kOffMask);
          const int lda = iq.lda ? iq.lda : s.lda, ldb = iq.ldb ? iq.ldb : s.ldb;
          for (int k0 = 0; k0 < K; k0 += ZK) {
            const int kc = min(ZK, K - k0);
            for (int e = tid; e < ZK * ZT; e += ZNT) {
              const int kk = e / ZT, r = e % ZT;
              float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
              if (kk < kc && r < mc) va = ta ? A[(int64_t)(k0 + kk) * lda + m0 + r] : A[(int64_t)(m0 + r) * lda + k0 + kk];
              if (kk < kc && r < nc) vb = tb ? B[(int64_t)(n0 + r) * ldb + k0 + kk] : B[(int64_t)(k0 + kk) * ldb + n0 + r];
              if (ca) va.y = -va.y;
              if (cb) vb.y = -vb.y;
              sA[kk][r] = va;
              sB[kk][r] = vb;
            }
            __syncthreads();
            for (int kk = 0; kk < kc; ++kk) {
              float2 a[4], b[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) a[i] = sA[kk][4 * ty + i];
#pragma unroll
              for (int j = 0; j < 4; ++j) b[j] = sB[kk][4 * tx + j];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = cmul_add(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
            work += 8ull * mc * nc * kc;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = 4 * ty + i, c = 4 * tx + j;
          if (r < mc && c < nc) {
            const int64_t o = ooff + (int64_t)(m0 + r) * s.ldc + n0 + c;
            if (out32) {
              float2* p = (float2*)obase + o;
              float2 v = accum ? *p : make_float2(0.f, 0.f);
              v.x += acc[i][j].x;
              v.y += acc[i][j].y;
              *p = v;
            } else {
              double2* p = (double2*)obase + o;
              double2 v = accum ? *p : make_double2(0.0, 0.0);
              v.x += (double)acc[i][j].x;
              v.y += (double)acc[i][j].y;
              *p = v;
            }
          }
        }
    }
  }
  if (ar->flops && tid == 0 && work) atomicAdd(ar->flops, work);
}

// ------------------------------------------------------------ Hermitian eigen + truncation
// Cyclic two-sided complex Jacobi with round-robin pairs.  For a pair (p, q) with
// a_pq = |a_pq| e^{i phi}, the unitary U = diag(1, e^{-i phi}) R, R the real rotation
// (c, s) that zeroes |a_pq| (tau = (a_qq - a_pp) / (2 |a_pq|), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c), updates A <- U^H A U and V <- V U:
//   rows:    a_p. <- c a_p. - s e^{i phi} a_q.,   a_q. <- s a_p. + c e^{i phi} a_q.
//   columns: a_.p <- c a_.p - s e^{-i phi} a_.q,  a_.q <- s a_.p + c e^{-i phi} a_.q
// Shared memory holds A and V (nn x (nn + 1) double2 each) up to nn = kZeigSmemMax;
// larger Gram matrices use the product's global eigen work space.
constexpr int kZeigSmemMax = 80;

__device__ double zblock_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

__device__ void zjacobi(double2* A, double2* V, int nn, int lds, double* red, double* cs, double* sn, double2* ph,
                        int* pp, int* qq) {
  const int tid = threadIdx.x, nt = blockDim.x, np = nn / 2;
  const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  for (int sweep = 0; sweep < 30 && nn > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = w; i < nn; i += nw)
      for (int j = lane; j < nn; j += 32) {
        const double2 a = A[i * lds + j];
        const double v = a.x * a.x + a.y * a.y;
        tot += v;
        if (i != j) off += v;
      }
    off = zblock_sum(off, red);
    tot = zblock_sum(tot, red);
    if (!(off > 1e-30 * tot)) break;
    for (int step = 0; step < nn - 1; ++step) {
      for (int k = tid; k < np; k += nt) {
        const int pa = (k == 0) ? 0 : ((k - 1 + step) % (nn - 1)) + 1;
        const int pb = ((nn - 1 - k - 1 + step) % (nn - 1)) + 1;
        const int p = min(pa, pb), q = max(pa, pb);
        const double2 apq = A[p * lds + q];
        const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
        double c = 1.0, s = 0.0;
        double2 e = make_double2(1.0, 0.0);
        if (mag != 0.0) {
          e = make_double2(apq.x / mag, apq.y / mag);  // e^{i phi}
          const double tau = (A[q * lds + q].x - A[p * lds + p].x) / (2.0 * mag);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        pp[k] = p;
        qq[k] = q;
        cs[k] = c;
        sn[k] = s;
        ph[k] = e;
      }
      __syncthreads();
      for (int k = w; k < np; k += nw) {  // rows p, q
        if (sn[k] == 0.0) continue;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double2 e = ph[k];
        for (int j = lane; j < nn; j += 32) {
          const double2 x = A[p * lds + j], y = zmul(e, A[q * lds + j]);
          A[p * lds + j] = make_double2(c * x.x - s * y.x, c * x.y - s * y.y);
          A[q * lds + j] = make_double2(s * x.x + c * y.x, s * x.y + c * y.y);
        }
      }
      __syncthreads();
      for (int k = w; k < np; k += nw) {  // columns p, q of A and V
        if (sn[k] == 0.0) continue;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double2 e = zconj(ph[k]);
        for (int i = lane; i < nn; i += 32) {
          const double2 x = A[i * lds + p], y = zmul(e, A[i * lds + q]);
          A[i * lds + p] = make_double2(c * x.x - s * y.x, c * x.y - s * y.y);
          A[i * lds + q] = make_double2(s * x.x + c * y.x, s * x.y + c * y.y);
          const double2 vx = V[i * lds + p], vy = zmul(e, V[i * lds + q]);
          V[i * lds + p] = make_double2(c * vx.x - s * vy.x, c * vx.y - s * vy.y);
          V[i * lds + q] = make_double2(s * vx.x + c * vy.x, s * vx.y + c * vy.y);
        }
      }
      __syncthreads();
    }
  }
}

// loads the Hermitian part of sum_m scale[m] G_m (active rows/cols) into A (nn x lds),
// zero padding; V = I
__device__ void zload_sum(const EigTask& t, const Arenas* ar, const int* act, int n, int nn, int lds,
                          const double* scale, double2* A, double2* V) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < nn * lds; e += nt) {
    const int a = e / lds, b = e % lds;
    double2 v = make_double2(0.0, 0.0);
    if (a < n && b < n)
      for (int m = 0; m < 3; ++m)
        if (scale[m] != 0.0) {
          const double2 g = zld(ar, t.g[m], (int64_t)act[a] * t.n_pad + act[b]);
          v.x += g.x * scale[m];
          v.y += g.y * scale[m];
        }
    A[e] = v;
    V[e] = make_double2(a == b ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int e = tid; e < nn * nn; e += nt) {  // Hermitian part (the Grams are Hermitian up to rounding)
    const int a = e / nn, b = e % nn;
    if (a < b) {
      const double2 x = A[a * lds + b], y = A[b * lds + a];
      const double2 h = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
      A[a * lds + b] = h;
      A[b * lds + a] = zconj(h);
    } else if (a == b) {
      A[a * lds + a].y = 0.0;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) zeig_kernel(const EigTask* __restrict__ tasks, int64_t first,
                                                   const Arenas* __restrict__ ars, double eps, int trunc, int norm,
                                                   double2* scratch, int64_t scratch_stride) {
  extern __shared__ double2 zsm[];
  __shared__ int act[256];
  __shared__ double red[8];
  __shared__ double cs[128], sn[128];
  __shared__ double2 ph[128];
  __shared__ int pp[128], qq[128];
  __shared__ int order[256];
  __shared__ double lam[256];
  __shared__ double s_scale[3];
  __shared__ int s_n, s_rank;
  const EigTask t = tasks[first + blockIdx.x];
  const Arenas* ar = ars + t.inst;
  const int tid = threadIdx.x, nt = blockDim.x;
  int32_t* ranks = t.col ? ar->kc : ar->kr;
  if (tid == 0) {
    int n = 0;
    if (t.child1 < 0) {
      for (int a = 0; a < t.nleaf; ++a) act[n++] = a;
    } else {
      const int k1 = ranks[t.child1], k2 = ranks[t.child2];
      for (int a = 0; a < k1; ++a) act[n++] = a;
      for (int a = 0; a < k2; ++a) act[n++] = t.half + a;
    }
    s_n = n;
  }
  __syncthreads();
  const int n = s_n, nn = n + (n & 1), lds = nn + 1;
  double2 *A, *V;
  if (nn <= kZeigSmemMax) {
    A = zsm;
    V = zsm + nn * lds;
  } else {
    A = scratch + blockIdx.x * scratch_stride;
    V = A + nn * lds;
  }
  // scale of each Gram matrix: 1 / ||G_m||_F, or 1 / lambda_max(G_m) for the spectral norm
  for (int m = 0; m < 3; ++m) {
    double loc = 0.0;
    if (t.g[m] >= 0) {
      for (int e = tid; e < n * n; e += nt) {
        const double2 g = zld(ar, t.g[m], (int64_t)act[e / n] * t.n_pad + act[e % n]);
        loc += g.x * g.x + g.y * g.y;
      }
    }
    const double nrm2 = zblock_sum(loc, red);
    if (tid == 0) s_scale[m] = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
    __syncthreads();
    if (norm == H2_NORM_SPECTRAL && s_scale[m] != 0.0) {
      double one[3] = {0.0, 0.0, 0.0};
      one[m] = 1.0;
      zload_sum(t, ar, act, n, nn, lds, one, A, V);
      zjacobi(A, V, nn, lds, red, cs, sn, ph, pp, qq);
      double mx = 0.0;
      for (int a = 0; a < n; ++a) mx = fmax(mx, A[a * lds + a].x);
      __syncthreads();
      if (tid == 0) s_scale[m] = mx > 0.0 ? 1.0 / mx : 0.0;
      __syncthreads();
    }
  }
  double scale[3] = {s_scale[0], s_scale[1], s_scale[2]};
  zload_sum(t, ar, act, n, nn, lds, scale, A, V);
  zjacobi(A, V, nn, lds, red, cs, sn, ph, pp, qq);
  for (int a = tid; a < n; a += nt) lam[a] = A[a * lds + a].x;
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
        const double l1 = lam[order[0]];
        const double thr = trunc == H2_TRUNC_SV ? eps * eps : eps;
        if (l1 > 0.0)
          while (r < n && lam[order[r]] > thr * l1) ++r;
      }
    }
    if (r > t.klim) {
      r = t.klim;
      atomicAdd(ar->cap_hits, 1ull);
    }
    s_rank = r;
    ranks[t.rank_out] = r;
  }
  __syncthreads();
  const int rank = s_rank;
  double2* out = zptr_w(ar, t.out);
  // the float copy of C's new bases for the GEMMs of the mixed product (arena X mirrors
  // C's basis region; absent in float64)
  float2* out32 = ar->p[AR_X] ? (float2*)ar->p[AR_X] + (t.out & kOffMask) : nullptr;
  for (int e = tid; e < t.n_pad * t.kcap; e += nt) {
    out[e] = make_double2(0.0, 0.0);
    if (out32) out32[e] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  // phase: the entry of largest magnitude (first such) is made real and positive
  for (int c = tid; c < rank; c += nt) {
    const int col = order[c];
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < n; ++a) {
      const double2 v = V[a * lds + col];
      const double m2 = v.x * v.x + v.y * v.y;
      if (m2 > bv) {
        bv = m2;
        best = a;
      }
    }
    const double2 pv = V[best * lds + col];
    const double mag = sqrt(pv.x * pv.x + pv.y * pv.y);
    const double2 f = mag > 0.0 ? make_double2(pv.x / mag, -pv.y / mag) : make_double2(1.0, 0.0);
    for (int a = 0; a < n; ++a) {
      const double2 v = zmul(V[a * lds + col], f);
      out[(int64_t)act[a] * t.kcap + c] = v;
      if (out32) out32[(int64_t)act[a] * t.kcap + c] = make_float2((float)v.x, (float)v.y);
    }
  }
}

__global__ void zto_tree_kernel(const double2* __restrict__ x, double2* __restrict__ xt, const int64_t* __restrict__ user,
                                int64_t rows, int64_t n, int64_t nrhs) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * nrhs) return;
  const int64_t pr = e / nrhs, c = e % nrhs, u = user[pr];
  xt[e] = u >= 0 ? x[u + c * n] : make_double2(0.0, 0.0);
}

__global__ void zfrom_tree_kernel(const double2* __restrict__ yt, double2* __restrict__ y,
                                  const int64_t* __restrict__ user, int64_t rows, int64_t n, int64_t nrhs) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows * nrhs) return;
  const int64_t pr = e / nrhs, c = e % nrhs, u = user[pr];
  if (u >= 0) y[u + c * n] = yt[e];
}

__global__ void zidentity_kernel(double2* out, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  out[e] = make_double2(e / n == e % n ? 1.0 : 0.0, 0.0);
}

}  // namespace

void launch_zgemm(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars, int maxn,
                  void* stream) {
  const int64_t kMaxGrid = 2147483647LL;
  int gy = std::max(1, std::min(256, (maxn + ZT - 1) / ZT));
  for (int64_t off = 0; off < count; off += kMaxGrid) {
    const int64_t c = std::min(count - off, kMaxGrid);
    seg_zgemm_kernel<<<dim3((unsigned)c, (unsigned)gy), ZNT, 0, (cudaStream_t)stream>>>(d_segs, d_items, first + off,
                                                                                      d_ars);
    add_kernel_launches(1);
  }
}

void launch_zgemm32(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars,
                    int maxn, void* stream) {
  const int64_t kMaxGrid = 2147483647LL;
  int gy = std::max(1, std::min(256, (maxn + ZT - 1) / ZT));
  for (int64_t off = 0; off < count; off += kMaxGrid) {
    const int64_t c = std::min(count - off, kMaxGrid);
    seg_zgemm32_kernel<<<dim3((unsigned)c, (unsigned)gy), ZNT, 0, (cudaStream_t)stream>>>(d_segs, d_items,
                                                                                        first + off, d_ars);
    add_kernel_launches(1);
  }
}

int64_t zeig_scratch_elems(int max_npad, int64_t count) {
  const int nn = max_npad + (max_npad & 1);
  return nn > kZeigSmemMax ? count * 2LL * nn * (nn + 1) * 2 : 0;  // in doubles
}

void launch_zeig(const EigTask* d_eigs, int64_t first, int64_t count, const Arenas* d_ars, double eps, int trunc,
                 int norm, int max_npad, double* scratch, void* stream) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(zeig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * kZeigSmemMax * (kZeigSmemMax + 1) * sizeof(double2)));
  });
  const int nn = max_npad + (max_npad & 1);
  size_t smem = 0;
  int64_t stride = 0;
  if (nn <= kZeigSmemMax) {
    smem = (size_t)2 * nn * (nn + 1) * sizeof(double2);
  } else {
    smem = (size_t)2 * kZeigSmemMax * (kZeigSmemMax + 1) * sizeof(double2);
    stride = (int64_t)2 * nn * (nn + 1);
  }
  zeig_kernel<<<(unsigned)count, 256, smem, (cudaStream_t)stream>>>(d_eigs, first, d_ars, eps, trunc, norm,
                                                                    (double2*)scratch, stride);
  add_kernel_launches(1);
}

void launch_zpermute(const double* src, double* dst, const int64_t* user, int64_t rows, int64_t n, int64_t nrhs,
                     bool to_tree, void* stream) {
  const int64_t tot = rows * nrhs;
  const unsigned blocks = (unsigned)((tot + 255) / 256);
  if (to_tree)
    zto_tree_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const double2*)src, (double2*)dst, user, rows, n, nrhs);
  else
    zfrom_tree_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const double2*)src, (double2*)dst, user, rows, n,
                                                                nrhs);
  add_kernel_launches(1);
}

void launch_zidentity(double* out, int64_t n, void* stream) {
  zidentity_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((double2*)out, n);
  add_kernel_launches(1);
}

}  // namespace h2
