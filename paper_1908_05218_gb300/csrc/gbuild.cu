// H^2 construction on the GPU (the step before the product; the paper, Sec. V-A and
// Sec. VI, cites its construction method without describing it).  The same sampled
// nested far-field compression as the host builder (builder.cpp: the same samples,
// skeleton rows and truncation), batched level by level with one CTA per cluster or
// per block, and written straight into the device arena:
//   * far(t): for t and each of its ancestors, every admissible partner s, sampled with
//     at most kBuildSamples points spread evenly over s in tree order;
//   * the Gram matrix G_t = W_t W_t^T of W_t = K(t, far(t)) (leaf t) or
//     [Q_t1 K(I_t1, far(t)); Q_t2 K(I_t2, far(t))] (non-leaf t; I_c are the skeleton
//     rows of child c, Q_c maps samples on I_c to coefficients).  The kernel values are
//     float32, taken from float64 coordinate differences (relative error ~1e-7, far
//     below eps); the Gram sums must resolve eigenvalues down to eps^2 lambda_1, so each
//     product is split exactly into two float32 values (x y = p + e, e = fma(x, y, -p))
//     and summed in double-float arithmetic (an unevaluated sum hi + lo of two float32
//     values, Knuth's TwoSum; relative error ~1e-13), on the float32 pipes;
//   * a float64 Jacobi decomposition of G_t: the eigenvectors with lambda > eps^2
//     lambda_1 (at most kBuildMaxRank) are the leaf basis V_t or the stacked transfer
//     E_t;
//   * skeleton rows I_t (all candidate rows while |t| <= kBuildAllRows, else k_t +
//     kBuildOver rows by greedy pivoted Gram-Schmidt on the rows of V_t), Q_t =
//     pinv(V_t[I_t, :]) (leaf: V_t^T) in float64, couplings Q_t K(I_t, I_s) Q_s^T in
//     float32 (stored as float64; relative error ~1e-6, far below eps) and dense blocks
//     K(t, s) in float64;
//   * symmetric kernel and partition: the column bases equal the row bases.
// Real kernels only (1/(4 pi r), 1/r^2); the complex Helmholtz kernel is built on the
// host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "internal.hpp"
#include "jacobi.cuh"

namespace h2 {

namespace {

constexpr int kCW = 32;          // sampled far-field columns per chunk of the Gram kernel
constexpr int kSmemMax = 200 * 1024;

// kernel value at squared distance r2 (float32; far field: r2 > 0)
__device__ __forceinline__ float kfar32(int kind, float r2) {
  if (kind == H2_K_LAPLACE) return 0.0795774715459476679f * rsqrtf(r2);  // 1 / (4 pi r)
  return 1.f / r2;                                                       // 1 / r^2
}

// kernel value between tree positions a and b, float64 (the host builder's formula)
__device__ __forceinline__ double kval64(int kind, double diag, const double* pts, int64_t a, int64_t b) {
  if (a == b) return diag;
  const double dx = pts[3 * a] - pts[3 * b], dy = pts[3 * a + 1] - pts[3 * b + 1], dz = pts[3 * a + 2] - pts[3 * b + 2];
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  if (r == 0.0) return diag;
  if (kind == H2_K_LAPLACE) return 1.0 / (4.0 * 3.14159265358979323846 * r);
  return 1.0 / (r * r);
}

// one partner block of a cluster's column stream: its first point (tree position), its
// points, and the stream position of its first sample
struct Part {
  int32_t start, size, cum;
};

struct GramTask {
  int32_t m;       // rows of W: leaf: its points; non-leaf: k1 + k2
  int32_t nr;      // kernel rows: leaf: m; non-leaf: ns1 + ns2
  int32_t k1, ns1; // non-leaf: child 1's rank and skeleton size
  int32_t ncol;    // sampled far-field columns
  int32_t nseg;    // partner blocks in the column stream
  int64_t seg0;    // first of them
  int64_t row0;    // leaf: first point
  int32_t c1, c2;  // non-leaf: the children
};

// (h, l) += x y in double-float arithmetic: the product split exactly (x y = p + e),
// p added to h by Knuth's TwoSum, the rounding errors gathered in l
// (the _rn intrinsics keep the compiler from contracting these steps into FMAs)
__device__ __forceinline__ void df_fma(float x, float y, float& h, float& l) {
  const float p = __fmul_rn(x, y);
  const float e = fmaf(x, y, -p);
  const float s = __fadd_rn(h, p);
  const float bp = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, e));
}

// the sample point of column c of a cluster's stream (binary search over its partners)
__device__ __forceinline__ int64_t column_point(const Part* parts, int32_t nseg, int32_t c) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (parts[mid].cum <= c) lo = mid;
    else hi = mid - 1;
  }
  const Part pt = parts[lo];
  const int q = c - pt.cum;
  if (pt.size <= kBuildSamples) return pt.start + q;
  return pt.start + (int64_t)((q + 0.5) * (double)pt.size / kBuildSamples);
}

// G_t = W_t W_t^T (m x m, float64, row stride m) for one cluster per CTA; U = lower-
// triangle entries per thread (256 U >= m (m + 1) / 2)
template <int U>
__global__ void __launch_bounds__(256) gb_gram_kernel(const GramTask* __restrict__ tasks, const Part* __restrict__ parts,
                                                      const double* __restrict__ pts, const int32_t* __restrict__ cskel,
                                                      int cskel_stride, const double* __restrict__ cq,
                                                      int64_t cq_stride, int kind, double* __restrict__ G,
                                                      int64_t g_stride, int nr_max, int m_max, int q_max) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const GramTask tk = tasks[blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = tk.m, nr = tk.nr;
  const bool leaf = tk.c1 < 0;
  double* rp = (double*)gsm;                    // nr_max x 4 (x, y, z; 32-byte rows)
  double* cp = rp + 4 * nr_max;                 // kCW x 4
  float* Kc = (float*)(cp + 4 * kCW);           // nr_max x kCW (16-byte aligned rows)
  float* Wc = Kc + (size_t)nr_max * kCW;        // m_max x kCW (non-leaf)
  float* Qs = Wc + (size_t)m_max * kCW;         // k1 x ns1, then k2 x ns2 (non-leaf)
  int* cok = (int*)(Qs + q_max);                // kCW: column valid
  const int k2 = m - tk.k1, ns2 = nr - tk.ns1;
  // rows: leaf points, or the children's skeleton points; the children's Q in float32
  for (int r = tid; r < nr; r += nt) {
    int64_t pr;
    if (leaf) pr = tk.row0 + r;
    else pr = r < tk.ns1 ? cskel[(int64_t)tk.c1 * cskel_stride + r] : cskel[(int64_t)tk.c2 * cskel_stride + r - tk.ns1];
    rp[4 * r] = pts[3 * pr];
    rp[4 * r + 1] = pts[3 * pr + 1];
    rp[4 * r + 2] = pts[3 * pr + 2];
  }
  if (!leaf) {
    for (int e = tid; e < tk.k1 * tk.ns1; e += nt) Qs[e] = (float)cq[(int64_t)tk.c1 * cq_stride + e];
    for (int e = tid; e < k2 * ns2; e += nt) Qs[tk.k1 * tk.ns1 + e] = (float)cq[(int64_t)tk.c2 * cq_stride + e];
  }
  // the lower-triangle entries (i, j), i >= j, this thread sums
  const int ne = m * (m + 1) / 2;
  int gi[U], gj[U];
  float hi[U], lo[U];  // G_ij = hi + lo (double-float)
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int e = tid + 256 * u;
    int i = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    gi[u] = i;
    gj[u] = e - i * (i + 1) / 2;
    hi[u] = 0.f;
    lo[u] = 0.f;
  }
  const Part* pp = parts + tk.seg0;
  const float* W = leaf ? Kc : Wc;
  for (int c0 = 0; c0 < tk.ncol; c0 += kCW) {
    __syncthreads();  // the previous chunk's values are no longer read
    if (tid < kCW) {
      const int c = c0 + tid;
      cok[tid] = c < tk.ncol;
      if (c < tk.ncol) {
        const int64_t q = column_point(pp, tk.nseg, c);
        cp[4 * tid] = pts[3 * q];
        cp[4 * tid + 1] = pts[3 * q + 1];
        cp[4 * tid + 2] = pts[3 * q + 2];
      }
    }
    __syncthreads();
    for (int e = tid; e < nr * kCW; e += nt) {
      const int r = e / kCW, c = e % kCW;
      float v = 0.f;
      if (cok[c]) {
        const float dx = (float)(rp[4 * r] - cp[4 * c]), dy = (float)(rp[4 * r + 1] - cp[4 * c + 1]),
                    dz = (float)(rp[4 * r + 2] - cp[4 * c + 2]);
        v = kfar32(kind, dx * dx + dy * dy + dz * dz);
      }
      Kc[r * kCW + c] = v;
    }
    __syncthreads();
    if (!leaf) {
      for (int e = tid; e < m * kCW; e += nt) {
        const int i = e / kCW, c = e % kCW;
        float s = 0.f;
        if (i < tk.k1) {
          const float* q = Qs + i * tk.ns1;
          for (int r = 0; r < tk.ns1; ++r) s = fmaf(q[r], Kc[r * kCW + c], s);
        } else {
          const float* q = Qs + tk.k1 * tk.ns1 + (i - tk.k1) * ns2;
          for (int r = 0; r < ns2; ++r) s = fmaf(q[r], Kc[(tk.ns1 + r) * kCW + c], s);
        }
        Wc[i * kCW + c] = s;
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (tid + 256 * u < ne) {
        const float4* a = reinterpret_cast<const float4*>(W + gi[u] * kCW);
        const float4* b = reinterpret_cast<const float4*>(W + gj[u] * kCW);
        float h = hi[u], l = lo[u];
#pragma unroll 8
        for (int c = 0; c < kCW / 4; ++c) {
          const float4 x = a[c], y = b[c];
          df_fma(x.x, y.x, h, l);
          df_fma(x.y, y.y, h, l);
          df_fma(x.z, y.z, h, l);
          df_fma(x.w, y.w, h, l);
        }
        // renormalise (Fast2Sum: |h| >= |l|)
        const float sum = __fadd_rn(h, l);
        lo[u] = __fsub_rn(l, __fsub_rn(sum, h));
        hi[u] = sum;
      }
    }
  }
  double* g = G + (int64_t)blockIdx.x * g_stride;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (tid + 256 * u < ne) {
      const double v = (double)hi[u] + (double)lo[u];
      g[gi[u] * m + gj[u]] = v;
      g[gj[u] * m + gi[u]] = v;
    }
  }
}

// shared memory of a Jacobi of an nn x nn matrix and its eigenvectors
inline size_t jac_smem(int nn) { return (size_t)2 * nn * (nn + 1) * sizeof(double); }

// the dominant eigenvectors of G_t (m x m): E_t (m x k, row-major, k = #{lambda >
// eps2 lambda_1} <= kmax); for a leaf also Q_t = E_t^T (k x m).  A and V in shared
// memory up to nn_smem, else in scratch (2 nn (nn + 1) doubles per cluster).
__global__ void __launch_bounds__(256) gb_eig_kernel(const int32_t* __restrict__ mdim, const double* __restrict__ G,
                                                     int64_t g_stride, double eps2, int kmax, double* __restrict__ E,
                                                     int64_t e_stride, int32_t* __restrict__ kout, double* __restrict__ Q,
                                                     int64_t q_stride, double* __restrict__ scratch, int nn_smem) {
  extern __shared__ __align__(16) unsigned char esm2[];
  __shared__ double red[8];
  __shared__ double cs[kBuildMaxRank + 1], sn[kBuildMaxRank + 1];
  __shared__ int pq[2 * kBuildMaxRank + 2];
  __shared__ int idx[2 * kBuildMaxRank + 2];
  __shared__ int s_k;
  const int t = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int m = mdim[t], nn = m + (m & 1), ld = nn + 1;
  if (m == 0) {
    if (tid == 0) kout[t] = 0;
    return;
  }
  double* A = nn <= nn_smem ? (double*)esm2 : scratch + (int64_t)t * 2 * nn * ld;
  double* V = A + (size_t)nn * ld;
  const double* g = G + (int64_t)t * g_stride;
  for (int e = tid; e < nn * ld; e += nt) {
    const int i = e / ld, j = e % ld;
    A[e] = (i < m && j < m) ? g[i * m + j] : 0.0;
    V[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sweeps<double>(A, V, nn, ld, 40, 1e-30, red, cs, sn, pq, pq + kBuildMaxRank + 1);
  __syncthreads();
  // eigenvalues in decreasing order, ties by index (a stable sort)
  for (int a = tid; a < m; a += nt) {
    const double la = A[a * ld + a];
    int pos = 0;
    for (int b = 0; b < m; ++b) {
      const double lb = A[b * ld + b];
      if (lb > la || (lb == la && b < a)) ++pos;
    }
    idx[pos] = a;
  }
  __syncthreads();
  if (tid == 0) {
    const double l1 = A[idx[0] * ld + idx[0]];
    int k = 0;
    if (l1 > 0)
      while (k < m && k < kmax && A[idx[k] * ld + idx[k]] > eps2 * l1) ++k;
    s_k = k;
    kout[t] = k;
  }
  __syncthreads();
  const int k = s_k;
  double* e = E + (int64_t)t * e_stride;
  for (int x = tid; x < m * k; x += nt) {
    const int r = x / k, c = x % k;
    const double v = V[r * ld + idx[c]];
    e[r * k + c] = v;
    if (Q) Q[(int64_t)t * q_stride + c * m + r] = v;
  }
}

struct SkelTask {
  int32_t k1, k2, ns1, ns2, c1, c2, k, p;  // p: skeleton rows of t
  int32_t all;                             // all candidate rows are skeleton rows
};

// skeleton rows of a non-leaf cluster: the rows of V_t at the candidate rows I_t1 u
// I_t2 are vc = [R_t1 E_t(top); R_t2 E_t(bottom)]; all of them, or k + kBuildOver
// chosen by greedy pivoted Gram-Schmidt (the largest remaining norm, first such), in
// increasing order.  Out: skel_t (p points) and R_t = vc[pick] (p x k).
__global__ void __launch_bounds__(256) gb_skel_kernel(const SkelTask* __restrict__ tasks, const double* __restrict__ crows,
                                                      int64_t cr_stride, const int32_t* __restrict__ cskel,
                                                      int cskel_stride, const double* __restrict__ E, int64_t e_stride,
                                                      int32_t* __restrict__ skel, int skel_stride,
                                                      double* __restrict__ rows, int64_t r_stride) {
  extern __shared__ __align__(16) unsigned char ssm[];
  __shared__ int chosen[kBuildMaxRank + kBuildOver + 8];
  __shared__ double qv[kBuildMaxRank + 1];
  __shared__ double bv[8];
  __shared__ int bi[8];
  __shared__ int s_best;
  const SkelTask tk = tasks[blockIdx.x];
  const int t = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5;
  const int nc2 = tk.ns1 + tk.ns2, k = tk.k;
  const double* e = E + (int64_t)t * e_stride;
  // vc row r (candidate r) into dst (k entries)
  auto vc_row = [&](int r, double* dst) {
    const double* cr;
    int kc, off;
    if (r < tk.ns1) {
      cr = crows + (int64_t)tk.c1 * cr_stride + (int64_t)r * tk.k1;
      kc = tk.k1;
      off = 0;
    } else {
      cr = crows + (int64_t)tk.c2 * cr_stride + (int64_t)(r - tk.ns1) * tk.k2;
      kc = tk.k2;
      off = tk.k1;
    }
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int i = 0; i < kc; ++i) s += cr[i] * e[(off + i) * k + j];
      dst[j] = s;
    }
  };
  auto cand = [&](int r) -> int32_t {
    return r < tk.ns1 ? cskel[(int64_t)tk.c1 * cskel_stride + r] : cskel[(int64_t)tk.c2 * cskel_stride + r - tk.ns1];
  };
  if (tk.all) {
    for (int r = tid; r < tk.p; r += nt) {
      skel[(int64_t)t * skel_stride + r] = cand(r);
      vc_row(r, rows + (int64_t)t * r_stride + (int64_t)r * k);
    }
    return;
  }
  double* R = (double*)ssm;              // nc2 x k
  double* nrm = R + (size_t)nc2 * k;     // nc2
  int* used = (int*)(nrm + nc2);         // nc2
  for (int r = tid; r < nc2; r += nt) {
    vc_row(r, R + (size_t)r * k);
    double a = 0.0;
    for (int c = 0; c < k; ++c) a += R[(size_t)r * k + c] * R[(size_t)r * k + c];
    nrm[r] = a;
    used[r] = 0;
  }
  __syncthreads();
  for (int step = 0; step < tk.p; ++step) {
    // the unused row of largest norm, the first such
    double b = -1.0;
    int bidx = nc2;
    for (int r = tid; r < nc2; r += nt)
      if (!used[r] && (nrm[r] > b || (nrm[r] == b && r < bidx))) {
        b = nrm[r];
        bidx = r;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, b, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > b || (ob == b && oi < bidx)) {
        b = ob;
        bidx = oi;
      }
    }
    if (lane == 0) {
      bv[w] = b;
      bi[w] = bidx;
    }
    __syncthreads();
    if (tid == 0) {
      double bb = bv[0];
      int ii = bi[0];
      for (int x = 1; x < (nt >> 5); ++x)
        if (bv[x] > bb || (bv[x] == bb && bi[x] < ii)) {
          bb = bv[x];
          ii = bi[x];
        }
      s_best = ii;
      used[ii] = 1;
      chosen[step] = ii;
    }
    __syncthreads();
    const int best = s_best;
    const double nb = sqrt(nrm[best]);
    if (nb > 0) {
      for (int c = tid; c < k; c += nt) qv[c] = R[(size_t)best * k + c] / nb;
      __syncthreads();
      for (int r = tid; r < nc2; r += nt) {
        if (used[r]) continue;
        double* x = R + (size_t)r * k;
        double d = 0.0;
        for (int c = 0; c < k; ++c) d += x[c] * qv[c];
        double a = 0.0;
        for (int c = 0; c < k; ++c) {
          x[c] -= d * qv[c];
          a += x[c] * x[c];
        }
        nrm[r] = a;
      }
    }
    __syncthreads();
  }
  // in increasing order
  if (tid == 0)
    for (int i = 1; i < tk.p; ++i) {
      const int v = chosen[i];
      int j = i - 1;
      while (j >= 0 && chosen[j] > v) {
        chosen[j + 1] = chosen[j];
        --j;
      }
      chosen[j + 1] = v;
    }
  __syncthreads();
  for (int r = tid; r < tk.p; r += nt) {
    skel[(int64_t)t * skel_stride + r] = cand(chosen[r]);
    vc_row(chosen[r], rows + (int64_t)t * r_stride + (int64_t)r * k);
  }
}

// Q_t = pinv(R_t) = (R^T R)^-1 R^T for R_t (p x k): the eigen-decomposition U L U^T of
// R^T R, eigenvalues below 1e-14 lambda_1 left out, Q = U L^-1 U^T R^T (k x p)
__global__ void __launch_bounds__(256) gb_pinv_kernel(const SkelTask* __restrict__ tasks, const double* __restrict__ rows,
                                                      int64_t r_stride, double* __restrict__ Q, int64_t q_stride) {
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ double red[8];
  __shared__ double cs[kBuildMaxRank / 2 + 1], sn[kBuildMaxRank / 2 + 1];
  __shared__ int pq[kBuildMaxRank + 2];
  __shared__ int idx[kBuildMaxRank + 1];
  __shared__ double lam[kBuildMaxRank + 1];
  const SkelTask tk = tasks[blockIdx.x];
  const int t = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int k = tk.k, p = tk.p, nn = k + (k & 1), ld = nn + 1;
  if (k == 0) return;
  const double* R = rows + (int64_t)t * r_stride;
  double* A = (double*)psm;
  double* V = A + (size_t)nn * ld;
  for (int e = tid; e < nn * ld; e += nt) {
    const int i = e / ld, j = e % ld;
    double s = 0.0;
    if (i < k && j < k)
      for (int r = 0; r < p; ++r) s += R[r * k + i] * R[r * k + j];
    A[e] = s;
    V[e] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sweeps<double>(A, V, nn, ld, 40, 1e-30, red, cs, sn, pq, pq + kBuildMaxRank / 2 + 1);
  __syncthreads();
  for (int a = tid; a < k; a += nt) {
    const double la = A[a * ld + a];
    int pos = 0;
    for (int b = 0; b < k; ++b) {
      const double lb = A[b * ld + b];
      if (lb > la || (lb == la && b < a)) ++pos;
    }
    idx[pos] = a;
    lam[a] = la;
  }
  __syncthreads();
  // T = U L^-1 U^T (k x k) into A (no longer read)
  const double l0 = lam[idx[0]];
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e % k;
    double s = 0.0;
    for (int c = 0; c < k; ++c) {
      const int ci = idx[c];
      if (lam[ci] > 1e-14 * l0) s += V[i * ld + ci] * V[j * ld + ci] / lam[ci];
    }
    A[i * k + j] = s;
  }
  __syncthreads();
  double* q = Q + (int64_t)t * q_stride;
  for (int e = tid; e < k * p; e += nt) {
    const int i = e / p, r = e % p;
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += A[i * k + j] * R[r * k + j];
    q[i * p + r] = s;
  }
}

struct CoupTask {
  int32_t t, s;
  int64_t off;  // arena offset of S_ts (row stride ld)
};

// S_ts = Q_t K(I_t, I_s) Q_s^T (kt x ks) into the arena, one block per CTA, in float32
// (kernel values from float64 coordinate differences)
__global__ void __launch_bounds__(128) gb_coup_kernel(const CoupTask* __restrict__ tasks, const double* __restrict__ pts,
                                                      int kind, double diag, const int32_t* __restrict__ skel,
                                                      int skel_stride, const int32_t* __restrict__ np,
                                                      const int32_t* __restrict__ kk, const double* __restrict__ Q,
                                                      int64_t q_stride, double* __restrict__ arena, int ld) {
  extern __shared__ __align__(16) unsigned char csm[];
  const CoupTask tk = tasks[blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int kt = kk[tk.t], ks = kk[tk.s], nt_ = np[tk.t], ns = np[tk.s];
  if (kt == 0 || ks == 0) return;
  float* K = (float*)csm;                    // nt_ x ns
  float* T = K + (size_t)nt_ * ns;           // kt x ns
  float* Qt = T + (size_t)kt * ns;           // kt x nt_
  float* Qs = Qt + (size_t)kt * nt_;         // ks x ns
  const int32_t* it = skel + (int64_t)tk.t * skel_stride;
  const int32_t* is = skel + (int64_t)tk.s * skel_stride;
  for (int e = tid; e < nt_ * ns; e += nt) {
    const int64_t a = it[e / ns], b = is[e % ns];
    const float dx = (float)(pts[3 * a] - pts[3 * b]), dy = (float)(pts[3 * a + 1] - pts[3 * b + 1]),
                dz = (float)(pts[3 * a + 2] - pts[3 * b + 2]);
    K[e] = kfar32(kind, dx * dx + dy * dy + dz * dz);
  }
  const double* qt = Q + (int64_t)tk.t * q_stride;
  const double* qs = Q + (int64_t)tk.s * q_stride;
  for (int e = tid; e < kt * nt_; e += nt) Qt[e] = (float)qt[e];
  for (int e = tid; e < ks * ns; e += nt) Qs[e] = (float)qs[e];
  __syncthreads();
  for (int e = tid; e < kt * ns; e += nt) {
    const int a = e / ns, j = e % ns;
    float s = 0.f;
    for (int i = 0; i < nt_; ++i) s = fmaf(Qt[a * nt_ + i], K[i * ns + j], s);
    T[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < kt * ks; e += nt) {
    const int a = e / ks, c = e % ks;
    float s = 0.f;
    for (int j = 0; j < ns; ++j) s = fmaf(T[a * ns + j], Qs[c * ns + j], s);
    arena[tk.off + (int64_t)a * ld + c] = (double)s;
  }
}

struct DenseTask {
  int64_t t0, s0;  // first points
  int32_t mt, ms;
  int64_t off;     // arena offset (row stride ld)
};

__global__ void __launch_bounds__(256) gb_dense_kernel(const DenseTask* __restrict__ tasks, const double* __restrict__ pts,
                                                       int kind, double diag, double* __restrict__ arena, int ld) {
  const DenseTask tk = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < tk.mt * tk.ms; e += blockDim.x) {
    const int i = e / tk.ms, j = e % tk.ms;
    arena[tk.off + (int64_t)i * ld + j] = kval64(kind, diag, pts, tk.t0 + i, tk.s0 + j);
  }
}

void set_smem(const void* f, size_t bytes) {
  if (bytes > 48 * 1024) cuda_check(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes), "smem");
}

// device buffer that frees itself
struct DBuf {
  void* p = nullptr;
  DBuf() = default;
  explicit DBuf(size_t bytes) { p = dev_alloc(bytes); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p) { o.p = nullptr; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (p) cudaFree(p);
    p = o.p;
    o.p = nullptr;
    return *this;
  }
  ~DBuf() {
    if (p) cudaFree(p);
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

template <typename T>
DBuf upload(const std::vector<T>& v) {
  DBuf b(std::max<size_t>(1, v.size()) * sizeof(T));
  if (!v.empty()) cuda_check(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return b;
}

// what a level keeps for its parent, its couplings and the arena
struct Level {
  int n = 0;
  std::vector<int32_t> k, p;  // ranks, skeleton sizes
  int sc = 0;                 // skeleton stride
  int64_t e_stride = 0, r_stride = 0, q_stride = 0;
  DBuf skel, E, rows, Q, dk, dp;
  bool leaf = false;
};

template <int U>
void launch_gram(const GramTask* t, int n, const Part* parts, const double* pts, const int32_t* cskel, int csc,
                 const double* cq, int64_t cqs, int kind, double* G, int64_t gs, int nr_max, int m_max, int q_max) {
  const size_t smem = (size_t)4 * nr_max * 8 + 4 * kCW * 8 + (size_t)nr_max * kCW * 4 + (size_t)m_max * kCW * 4 +
                      (size_t)q_max * 4 + kCW * 4;
  if (smem > (size_t)kSmemMax) throw Error(H2_EINTERNAL, "construction: Gram tile too large");
  set_smem((const void*)gb_gram_kernel<U>, smem);
  gb_gram_kernel<U><<<n, 256, smem>>>(t, parts, pts, cskel, csc, cq, cqs, kind, G, gs, nr_max, m_max, q_max);
  add_kernel_launches(1);
}

}  // namespace

void build_h2_device(const Structure& st, const h2_kernel& kern, double eps, Mat& m) {
  if (kern.kind != H2_K_LAPLACE && kern.kind != H2_K_INV_R2)
    throw Error(H2_EUNSUPPORTED, "the GPU construction takes the real kernels");
  const int L = st.L, LS = st.LS, kind = kern.kind;
  const double diag = kern.diag_re, eps2 = eps * eps;
  DBuf d_pts = upload(st.pts);
  // admissible partners per level, by row cluster, in block order
  std::vector<std::vector<std::vector<int32_t>>> partners(L + 1);
  for (int l = 0; l <= L; ++l) {
    partners[l].assign(1LL << l, {});
    for (auto& b : st.blocks[l])
      if (b.kind == KR) partners[l][b.t].push_back(b.s);
  }
  std::vector<Level> lv(L + 1);
  for (int l = L; l >= 0; --l) {
    const int n = 1 << l;
    Level& cur = lv[l];
    cur.n = n;
    cur.leaf = l == L;
    const Level* ch = l < L ? &lv[l + 1] : nullptr;
    // the column streams and the Gram tasks
    std::vector<GramTask> gt(n);
    std::vector<Part> parts;
    int nr_max = 1, m_max = 1, q_max = 1;
    for (int64_t t = 0; t < n; ++t) {
      GramTask& g = gt[t];
      g.seg0 = (int64_t)parts.size();
      int32_t cum = 0;
      for (int a = l; a >= 0; --a)
        for (int32_t s : partners[a][t >> (l - a)]) {
          const int32_t sz = (int32_t)st.size[a][s];
          parts.push_back({(int32_t)st.start[a][s], sz, cum});
          cum += std::min(sz, kBuildSamples);
        }
      g.nseg = (int32_t)(parts.size() - g.seg0);
      g.ncol = cum;
      if (cur.leaf) {
        g.m = g.nr = (int32_t)st.size[L][t];
        g.k1 = g.ns1 = 0;
        g.row0 = st.start[L][t];
        g.c1 = g.c2 = -1;
      } else {
        g.c1 = (int32_t)(2 * t);
        g.c2 = (int32_t)(2 * t + 1);
        g.k1 = ch->k[2 * t];
        g.ns1 = ch->p[2 * t];
        g.m = g.k1 + ch->k[2 * t + 1];
        g.nr = g.ns1 + ch->p[2 * t + 1];
        g.row0 = 0;
        q_max = std::max(q_max, g.k1 * g.ns1 + ch->k[2 * t + 1] * ch->p[2 * t + 1]);
      }
      if (g.ncol == 0) g.m = 0;  // no far field: rank 0
      nr_max = std::max(nr_max, g.nr);
      m_max = std::max(m_max, g.m);
    }
    if (parts.empty()) parts.push_back({0, 0, 0});
    DBuf d_gt = upload(gt), d_parts = upload(parts);
    // G, then the dominant eigenvectors
    const int64_t gs = (int64_t)m_max * m_max;
    DBuf G((size_t)n * gs * sizeof(double));
    const int ne = m_max * (m_max + 1) / 2;
    const int32_t* cskel = ch ? ch->skel.as<int32_t>() : nullptr;
    const double* cq = ch ? ch->Q.as<double>() : nullptr;
    const int csc = ch ? ch->sc : 0;
    const int64_t cqs = ch ? ch->q_stride : 0;
    if (ne <= 256 * 4)
      launch_gram<4>(d_gt.as<GramTask>(), n, d_parts.as<Part>(), d_pts.as<double>(), cskel, csc, cq, cqs, kind,
                     G.as<double>(), gs, nr_max, m_max, q_max);
    else if (ne <= 256 * 9)
      launch_gram<9>(d_gt.as<GramTask>(), n, d_parts.as<Part>(), d_pts.as<double>(), cskel, csc, cq, cqs, kind,
                     G.as<double>(), gs, nr_max, m_max, q_max);
    else if (ne <= 256 * 20)
      launch_gram<20>(d_gt.as<GramTask>(), n, d_parts.as<Part>(), d_pts.as<double>(), cskel, csc, cq, cqs, kind,
                      G.as<double>(), gs, nr_max, m_max, q_max);
    else if (ne <= 256 * 33)
      launch_gram<33>(d_gt.as<GramTask>(), n, d_parts.as<Part>(), d_pts.as<double>(), cskel, csc, cq, cqs, kind,
                      G.as<double>(), gs, nr_max, m_max, q_max);
    else
      throw Error(H2_EINTERNAL, "construction: Gram matrix above 128 x 128");
    cuda_check(cudaGetLastError(), "construction Gram");
    std::vector<int32_t> mdim(n);
    for (int t = 0; t < n; ++t) mdim[t] = gt[t].m;
    DBuf d_m = upload(mdim);
    const int kcap = std::min(m_max, kBuildMaxRank);
    cur.e_stride = (int64_t)m_max * kcap;
    cur.E = DBuf((size_t)n * cur.e_stride * sizeof(double));
    cur.dk = DBuf((size_t)n * sizeof(int32_t));
    if (cur.leaf) {
      cur.q_stride = (int64_t)kcap * LS;
      cur.Q = DBuf((size_t)n * cur.q_stride * sizeof(double));
    }
    {
      const int nn = m_max + (m_max & 1);
      const int nn_smem = 110;
      DBuf scratch(nn > nn_smem ? (size_t)n * 2 * nn * (nn + 1) * sizeof(double) : 8);
      const size_t smem = nn <= nn_smem ? jac_smem(nn) : 0;
      set_smem((const void*)gb_eig_kernel, jac_smem(nn_smem));
      gb_eig_kernel<<<n, 256, smem>>>(d_m.as<int32_t>(), G.as<double>(), gs, eps2, kBuildMaxRank, cur.E.as<double>(),
                                      cur.e_stride, cur.dk.as<int32_t>(), cur.leaf ? cur.Q.as<double>() : nullptr,
                                      cur.q_stride, scratch.as<double>(), nn_smem);
      add_kernel_launches(1);
      cuda_check(cudaGetLastError(), "construction eigen");
      cur.k.resize(n);
      cuda_check(cudaMemcpy(cur.k.data(), cur.dk.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost), "ranks");
    }
    G = DBuf();
    if (cur.leaf) {
      // skeleton = every point; rows of V at them = V
      cur.sc = LS;
      cur.p.resize(n);
      std::vector<int32_t> sk((size_t)n * LS, 0);
      for (int t = 0; t < n; ++t) {
        cur.p[t] = (int32_t)st.size[L][t];
        for (int r = 0; r < cur.p[t]; ++r) sk[(size_t)t * LS + r] = (int32_t)(st.start[L][t] + r);
      }
      cur.skel = upload(sk);
      cur.dp = upload(cur.p);
      cur.r_stride = cur.e_stride;  // rows alias E
    } else {
      // skeleton rows and Q
      std::vector<SkelTask> sk(n);
      int pmax = 1, kmax = 1;
      size_t ssm = 0;
      for (int t = 0; t < n; ++t) {
        SkelTask& s = sk[t];
        s.k1 = ch->k[2 * t];
        s.k2 = ch->k[2 * t + 1];
        s.ns1 = ch->p[2 * t];
        s.ns2 = ch->p[2 * t + 1];
        s.c1 = 2 * t;
        s.c2 = 2 * t + 1;
        s.k = cur.k[t];
        const int nc2 = s.ns1 + s.ns2;
        s.all = (st.size[l][t] <= kBuildAllRows || nc2 <= s.k + kBuildOver) ? 1 : 0;
        s.p = s.all ? nc2 : std::min(s.k + kBuildOver, nc2);
        if (gt[t].m == 0) {  // no far field: rank 0 (the host builder's k = 0 case)
          s.k = 0;
        }
        pmax = std::max(pmax, s.p);
        kmax = std::max(kmax, s.k);
        if (!s.all) ssm = std::max(ssm, (size_t)nc2 * s.k * 8 + (size_t)nc2 * 12);
      }
      cur.p.resize(n);
      for (int t = 0; t < n; ++t) cur.p[t] = sk[t].p;
      cur.sc = pmax;
      cur.r_stride = (int64_t)pmax * kmax;
      cur.q_stride = (int64_t)kmax * pmax;
      cur.skel = DBuf((size_t)n * pmax * sizeof(int32_t));
      cur.rows = DBuf((size_t)n * cur.r_stride * sizeof(double));
      cur.Q = DBuf((size_t)n * cur.q_stride * sizeof(double));
      cur.dp = upload(cur.p);
      DBuf d_sk = upload(sk);
      if (ssm > (size_t)kSmemMax) throw Error(H2_EINTERNAL, "construction: skeleton selection too large");
      set_smem((const void*)gb_skel_kernel, std::max<size_t>(ssm, 16));
      const double* crows = ch->leaf ? ch->E.as<double>() : ch->rows.as<double>();
      gb_skel_kernel<<<n, 256, ssm>>>(d_sk.as<SkelTask>(), crows, ch->r_stride, ch->skel.as<int32_t>(), ch->sc,
                                      cur.E.as<double>(), cur.e_stride, cur.skel.as<int32_t>(), cur.sc,
                                      cur.rows.as<double>(), cur.r_stride);
      add_kernel_launches(1);
      cuda_check(cudaGetLastError(), "construction skeleton");
      const int nn = kmax + (kmax & 1);
      set_smem((const void*)gb_pinv_kernel, jac_smem(nn));
      gb_pinv_kernel<<<n, 256, jac_smem(nn)>>>(d_sk.as<SkelTask>(), cur.rows.as<double>(), cur.r_stride,
                                               cur.Q.as<double>(), cur.q_stride);
      add_kernel_launches(1);
      cuda_check(cudaGetLastError(), "construction pinv");
    }
  }
  // ranks, caps and the zeroed arena
  const int nn = st.nnodes();
  std::vector<int32_t> kr(nn, 0);
  for (int l = 0; l <= L; ++l)
    for (int t = 0; t < (1 << l); ++t) kr[Structure::node(l, t)] = lv[l].k[t];
  m.Kr.assign(L + 1, 0);
  for (int l = 0; l <= L; ++l) {
    int mx = 0;
    for (int t = 0; t < (1 << l); ++t) mx = std::max(mx, lv[l].k[t]);
    m.Kr[l] = cap_round(mx);
  }
  m.Kc = m.Kr;
  alloc_mat(m);
  // bases and transfers: copy tasks from each level's E into the arena (rows and columns)
  for (int l = 0; l <= L; ++l) {
    std::vector<CopyTask> tk;
    for (int64_t t = 0; t < (1LL << l); ++t) {
      const int k = lv[l].k[t];
      if (!k) continue;
      const int64_t src = t * lv[l].e_stride;
      if (l == L) {
        const int rows = (int)st.size[L][t];
        tk.push_back({m.Vr(t), src, rows, k, m.Kr[L], 0});
        tk.push_back({m.Vc(t), src, rows, k, m.Kc[L], 0});
      } else {
        const int k1 = lv[l + 1].k[2 * t], k2 = lv[l + 1].k[2 * t + 1];
        if (k1) {
          tk.push_back({m.Er(l, t), src, k1, k, m.Kr[l], 0});
          tk.push_back({m.Ec(l, t), src, k1, k, m.Kc[l], 0});
        }
        if (k2) {
          tk.push_back({m.Er(l, t) + (int64_t)m.Kr[l + 1] * m.Kr[l], src + (int64_t)k1 * k, k2, k, m.Kr[l], 0});
          tk.push_back({m.Ec(l, t) + (int64_t)m.Kc[l + 1] * m.Kc[l], src + (int64_t)k1 * k, k2, k, m.Kc[l], 0});
        }
      }
    }
    if (tk.empty()) continue;
    DBuf d_tk = upload(tk);
    launch_copy_tasks(d_tk.as<CopyTask>(), (int64_t)tk.size(), lv[l].E.as<double>(), m.arena, true, nullptr);
    cuda_check(cudaGetLastError(), "construction bases");
    cuda_check(cudaDeviceSynchronize(), "construction bases");
  }
  // couplings
  for (int l = 0; l <= L; ++l) {
    std::vector<CoupTask> ct;
    size_t smem = 16;
    for (auto& b : st.blocks[l])
      if (b.kind == KR) {
        ct.push_back({b.t, b.s, m.S(l, b.idx)});
        const size_t need = ((size_t)lv[l].p[b.t] * lv[l].p[b.s] + (size_t)lv[l].k[b.t] * lv[l].p[b.s] +
                             (size_t)lv[l].k[b.t] * lv[l].p[b.t] + (size_t)lv[l].k[b.s] * lv[l].p[b.s]) * 4;
        smem = std::max(smem, need);
      }
    if (ct.empty()) continue;
    if (smem > (size_t)kSmemMax) throw Error(H2_EINTERNAL, "construction: coupling tile too large");
    set_smem((const void*)gb_coup_kernel, smem);
    DBuf d_ct = upload(ct);
    const int64_t nct = (int64_t)ct.size();
    for (int64_t off = 0; off < nct; off += 2147483647LL) {
      const unsigned g = (unsigned)std::min<int64_t>(nct - off, 2147483647LL);
      gb_coup_kernel<<<g, 128, smem>>>(d_ct.as<CoupTask>() + off, d_pts.as<double>(), kind, diag,
                                       lv[l].skel.as<int32_t>(), lv[l].sc, lv[l].dp.as<int32_t>(),
                                       lv[l].dk.as<int32_t>(), lv[l].Q.as<double>(), lv[l].q_stride, m.arena,
                                       m.Kc[l]);
      add_kernel_launches(1);
    }
    cuda_check(cudaGetLastError(), "construction couplings");
  }
  // dense leaf blocks
  {
    std::vector<DenseTask> dt;
    for (auto& b : st.blocks[L])
      if (b.kind == KF)
        dt.push_back({st.start[L][b.t], st.start[L][b.s], (int32_t)st.size[L][b.t], (int32_t)st.size[L][b.s],
                      m.F(b.idx)});
    if (!dt.empty()) {
      DBuf d_dt = upload(dt);
      gb_dense_kernel<<<(unsigned)dt.size(), 256>>>(d_dt.as<DenseTask>(), d_pts.as<double>(), kind, diag, m.arena,
                                                    LS);
      add_kernel_launches(1);
      cuda_check(cudaGetLastError(), "construction dense blocks");
    }
  }
  cuda_check(cudaDeviceSynchronize(), "construction");
  cuda_check(cudaMemcpy(m.d_kr, kr.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice), "upload ranks");
  cuda_check(cudaMemcpy(m.d_kc, kr.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice), "upload ranks");
  m.h_kr = kr;
  m.h_kc = kr;
  m.ranks_on_host = true;
}

}  // namespace h2
