// Device kernels of the H^2 product: segmented batched small GEMM (float64), the
// batched normalised-Gram eigen-decomposition with truncation (Sec. III-C, IV-C),
// and the permutations between user order and padded tree order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>
#include <cstdint>
#include <cstdio>

#include "device.cuh"
#include "jacobi.cuh"
#include "internal.hpp"

namespace h2 {

// kernel launches made by this library in this process (every launch site below adds)
static std::atomic<unsigned long long> g_launches{0};
unsigned long long kernel_launches() { return g_launches.load(); }
void add_kernel_launches(long long d) { g_launches += (unsigned long long)d; }

// ------------------------------------------------------------ segmented GEMM
// (float64 products; the float32 ones take seg_gemm32_kernel below)
// One CTA (64 threads) per segment (blockIdx.x) and 32-column slice (blockIdx.y);
// the CTA walks 32 x 32 output tiles; thread (tx, ty) owns the contiguous 4 x 4
// block rows 4 ty.., cols 4 tx.. and reads it from shared memory with vector
// loads.  The items of a segment are packed along k into shared-memory slices of
// depth GK (several short items share a slice, a long one spans several), loading
// only the actual extents: rows < M, cols < N, k < the item's rank.  Slices are
// double-buffered: cp.async fills slice s+1 while slice s is multiplied.  All
// operands of a product have the element type T (the output may be float64); a
// warp whose rows all lie beyond M skips the arithmetic; rows/cols beyond M/N hold
// stale values whose products are never stored.
constexpr int GK = 32, TILE = 32, GPAD = TILE + 4, GNT = 64;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void load(const float* p, float v[4]) {
    float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
};
template <>
struct Vec4<double> {
  __device__ static void load(const double* p, double v[4]) {
    double2 x = *reinterpret_cast<const double2*>(p);
    double2 y = *reinterpret_cast<const double2*>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
};

template <typename T>
__device__ __forceinline__ void cp_async(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }


template <typename T>
__global__ void __launch_bounds__(GNT, 12) seg_gemm_kernel(const Seg* __restrict__ segs, const Item* __restrict__ items,
                                                       int64_t first, const Arenas* __restrict__ ars) {
  __shared__ __align__(16) T sA[2][GK * GPAD];
  __shared__ __align__(16) T sB[2][GK * GPAD];
  const Seg s = segs[first + blockIdx.x];
  const Arenas* ar = ars + s.inst;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  const bool ta = s.flags & SF_TA, tb = s.flags & SF_TB, accum = s.flags & SF_ACC;
  const int M = bound(ar, s.mref, s.m), N = bound(ar, s.nref, s.n);
  const View out = view(ar, s.out);
  const Item* it = items + s.first;
  unsigned long long work = 0;
  for (int n0 = blockIdx.y * TILE; n0 < N; n0 += gridDim.y * TILE) {
    const int nc = min(TILE, N - n0);
    for (int m0 = 0; m0 < M; m0 += TILE) {
      const int mc = min(TILE, M - m0);
      const bool live = (tid >> 5) * 16 < mc;  // this warp owns rows 16 w .. 16 w + 15
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
      if (s.flags & SF_SUM) {
        for (int q = 0; q < s.count; ++q) {
          const T* A = ptr_of<T>(ar, it[q].a);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              int r = 4 * ty + i, c = 4 * tx + j;
              if (r < mc && c < nc)  // (SF_TA: the input is read transposed)
                acc[i][j] += ta ? A[(int64_t)(n0 + c) * s.lda + m0 + r] : A[(int64_t)(m0 + r) * s.lda + n0 + c];
            }
        }
      } else {
        int q = 0, koff = 0, K = s.count ? bound(ar, it[0].kref, it[0].kpad ? it[0].kpad : s.k) : 0;
        // issue the copies of the next slice into buffer `buf`; returns its depth
        auto fill = [&](int buf) -> int {
          int kfill = 0;
          T* a_s = sA[buf];
          T* b_s = sB[buf];
          while (q < s.count && kfill < GK) {
            if (K == 0) {
              ++q;
              if (q < s.count) K = bound(ar, it[q].kref, it[q].kpad ? it[q].kpad : s.k);
              continue;
            }
            const int take = min(K - koff, GK - kfill);
            const Item iq = it[q];
            const T* A = ptr_of<T>(ar, iq.a);
            const T* B = ptr_of<T>(ar, iq.b);
            const int lda = iq.lda ? iq.lda : s.lda, ldb = iq.ldb ? iq.ldb : s.ldb;
            if (ta) {
              for (int kk = tid / TILE; kk < take; kk += GNT / TILE) {
                const int r = tid % TILE;
                if (r < mc) cp_async(&a_s[(kfill + kk) * GPAD + r], A + (int64_t)(koff + kk) * lda + (m0 + r));
              }
            } else {
              for (int r = tid / GK; r < mc; r += GNT / GK) {
                const int kk = tid % GK;
                if (kk < take) cp_async(&a_s[(kfill + kk) * GPAD + r], A + (int64_t)(m0 + r) * lda + (koff + kk));
              }
            }
            if (tb) {
              for (int c = tid / GK; c < nc; c += GNT / GK) {
                const int kk = tid % GK;
                if (kk < take) cp_async(&b_s[(kfill + kk) * GPAD + c], B + (int64_t)(n0 + c) * ldb + (koff + kk));
              }
            } else {
              for (int kk = tid / TILE; kk < take; kk += GNT / TILE) {
                const int c = tid % TILE;
                if (c < nc) cp_async(&b_s[(kfill + kk) * GPAD + c], B + (int64_t)(koff + kk) * ldb + (n0 + c));
              }
            }
            kfill += take;
            koff += take;
            work += 2ull * mc * nc * take;
            if (koff == K) {
              koff = 0;
              ++q;
              if (q < s.count) K = bound(ar, it[q].kref, it[q].kpad ? it[q].kpad : s.k);
            }
          }
          return kfill;
        };
        int buf = 0;
        int kf = fill(0);
        cp_commit();
        while (kf > 0) {
          const int kf_next = fill(buf ^ 1);
          cp_commit();
          cp_wait1();
          __syncthreads();
          if (live) {
            const T* a_s = sA[buf];
            const T* b_s = sB[buf];
            for (int kk = 0; kk < kf; ++kk) {
              T a[4], b[4];
              Vec4<T>::load(&a_s[kk * GPAD + 4 * ty], a);
              Vec4<T>::load(&b_s[kk * GPAD + 4 * tx], b);
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
          }
          __syncthreads();
          buf ^= 1;
          kf = kf_next;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int r = 4 * ty + i, c = 4 * tx + j;
          if (r < mc && c < nc) st<T>(out, (int64_t)(m0 + r) * s.ldc + n0 + c, acc[i][j], accum);
        }
    }
  }
  if (ar->flops && tid == 0 && work) atomicAdd(ar->flops, work);
}

// ------------------------------------------------------------ segmented GEMM, float32
// The float32 products of the mixed-precision product.  Same segments, tiles and
// thread layout as seg_gemm_kernel, with the operand traffic cut to what the tile
// needs:
//   * each warp holds the metadata of 32 items at a time, one item per lane (its
//     operand pointers, leading dims and k bound, the rank read once), and the fill
//     loop takes an item's fields by shuffle: no dependent global loads per item;
//   * A is staged in the layout it has in memory: row-major (m x k) as rows of k,
//     transposed (k x m) as rows of m; B (k x n) as rows of n; each row is copied in
//     16-byte pieces when the item's pointer and leading dim allow it (else element by
//     element), so a 32 x 32 slice takes four copies per thread and operand;
//   * items are packed along k in steps of four; k from an item's bound up to the
//     next multiple of four is zero in both operands (cp.async zero-fills the tail
//     of a piece, whole padded rows are written as zeros).
constexpr int LDK = GK + 4;  // row stride of a row-major A slice (16-byte rows)
constexpr int kSliceA = (TILE * LDK > GK * GPAD) ? TILE * LDK : GK * GPAD;

__device__ __forceinline__ void cp_async16(float* dst, const float* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes));
}

template <bool AMK>
__device__ __forceinline__ void slice_fma(const float* __restrict__ a_s, const float* __restrict__ b_s, int kf,
                                          int tx, int ty, float acc[4][4], int k0, int kstep) {
  for (int kk = k0; kk < kf; kk += kstep) {
    float a[4][4], b[4][4];  // a[i][q]: row 4 ty + i, k kk + q;  b[q][j]: k kk + q, col 4 tx + j
    if (AMK) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v = *reinterpret_cast<const float4*>(&a_s[(4 * ty + i) * LDK + kk]);
        a[i][0] = v.x; a[i][1] = v.y; a[i][2] = v.z; a[i][3] = v.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 v = *reinterpret_cast<const float4*>(&a_s[(kk + q) * GPAD + 4 * ty]);
        a[0][q] = v.x; a[1][q] = v.y; a[2][q] = v.z; a[3][q] = v.w;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(&b_s[(kk + q) * GPAD + 4 * tx]);
      b[q][0] = v.x; b[q][1] = v.y; b[q][2] = v.z; b[q][3] = v.w;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i][q], b[q][j], acc[i][j]);
  }
}

__global__ void __launch_bounds__(GNT, 12) seg_gemm32_kernel(const Seg* __restrict__ segs,
                                                             const Item* __restrict__ items, int64_t first,
                                                             const Arenas* __restrict__ ars) {
  __shared__ __align__(16) float sA[2][kSliceA];
  __shared__ __align__(16) float sB[2][GK * GPAD];
  const Seg s = segs[first + blockIdx.x];
  const Arenas* ar = ars + s.inst;
  const int tid = threadIdx.x, lane = tid & 31, tx = tid & 7, ty = tid >> 3;
  const bool ta = s.flags & SF_TA, tb = s.flags & SF_TB, accum = s.flags & SF_ACC;
  const int M = bound(ar, s.mref, s.m), N = bound(ar, s.nref, s.n);
  const View out = view(ar, s.out);
  const Item* it = items + s.first;
  unsigned long long work = 0;
  if (s.flags & SF_SUM) {
    for (int n0 = blockIdx.y * TILE; n0 < N; n0 += gridDim.y * TILE) {
      const int nc = min(TILE, N - n0);
      for (int m0 = 0; m0 < M; m0 += TILE) {
        const int mc = min(TILE, M - m0);
        float acc[4][4] = {};
        const bool tiled = s.flags & SF_TILE, tt = s.flags & SF_TILE_T;
        for (int q = 0; q < s.count; ++q) {
          const float* A = ptr_of<float>(ar, it[q].a);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int r = 4 * ty + i, c = 4 * tx + j;
              if (r < mc && c < nc) {
                if (tiled)  // an operand tile of the BF16 split product (its lda: the tile's k)
                  acc[i][j] += tile_load((const char*)A, s.trows, s.lda, tt ? n0 + c : m0 + r, tt ? m0 + r : n0 + c);
                else
                  acc[i][j] += ta ? A[(int64_t)(n0 + c) * s.lda + m0 + r] : A[(int64_t)(m0 + r) * s.lda + n0 + c];
              }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = 4 * ty + i, c = 4 * tx + j;
            if (r < mc && c < nc) st<float>(out, (int64_t)(m0 + r) * s.ldc + n0 + c, acc[i][j], accum);
          }
      }
    }
    return;
  }
  // a diagonal block of a symmetric matrix: its lower tiles and, in a tile on the
  // diagonal, its lower 4 x 4 blocks only; every off-diagonal value is also written to
  // the transposed position
  const bool sym = s.flags2 & SF2_SYM;
  for (int n0 = blockIdx.y * TILE; n0 < N; n0 += gridDim.y * TILE) {
    const int nc = min(TILE, N - n0);
    for (int m0 = 0; m0 < M; m0 += TILE) {
      if (sym && n0 > m0) continue;
      const int mc = min(TILE, M - m0);
      const bool tri = sym && m0 == n0;  // (then mc == nc)
      // the tile's live 4 x 4 blocks go to threads 0 .. nthr-1 (row-major; a triangle on
      // a symmetric diagonal tile); idle threads read block 0.  A tile of at most 32 live
      // blocks (e.g. 20 x 24) is computed by both warps on the same blocks, each over
      // every other k-chunk of four, and the two partial sums are added in a fixed order
      // at the end; otherwise a warp whose threads all lie beyond the blocks skips the
      // arithmetic
      const int ncq = (nc + 3) >> 2, nthr = tri ? ncq * (ncq + 1) / 2 : ((mc + 3) >> 2) * ncq;
      const bool split = nthr <= 32;
      const int me = split ? lane : tid;
      const bool mine = me < nthr;
      int qy = 0, qx = 0;
      if (mine && tri) {
        while ((qy + 1) * (qy + 2) / 2 <= me) ++qy;
        qx = me - qy * (qy + 1) / 2;
      } else if (mine) {
        qy = me / ncq;
        qx = me - qy * ncq;
      }
      const bool live = split || (tid & ~31) < nthr;
      const int k0 = split ? 4 * (tid >> 5) : 0, kstep = split ? 8 : 4;
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      // this lane's item of the current group of 32
      const float* pa = nullptr;
      const float* pb = nullptr;
      int la_ = 0, lb_ = 0, kb = 0, va = 0, vb = 0;
      int base = -32;
      auto stage = [&](int b0) {
        base = b0;
        const int qi = b0 + lane;
        if (qi < s.count) {
          const Item iq = it[qi];
          pa = ptr_of<float>(ar, iq.a);
          pb = ptr_of<float>(ar, iq.b);
          la_ = iq.lda ? iq.lda : s.lda;
          lb_ = iq.ldb ? iq.ldb : s.ldb;
          kb = bound(ar, iq.kref, iq.kpad ? iq.kpad : s.k);
          va = ((((uintptr_t)pa) & 15) == 0 && (la_ & 3) == 0);
          vb = ((((uintptr_t)pb) & 15) == 0 && (lb_ & 3) == 0);
        } else {
          kb = 0;
        }
      };
      int q = 0, koff = 0;
      // fields of item q (uniform across the CTA)
      const float *A = nullptr, *B = nullptr;
      int lda = 0, ldb = 0, K = 0, K4 = 0;
      bool vecA = false, vecB = false;
      auto fetch = [&]() {
        if (q >= base + 32) stage(q & ~31);
        const int src = q - base;
        A = (const float*)__shfl_sync(0xffffffffu, (unsigned long long)pa, src);
        B = (const float*)__shfl_sync(0xffffffffu, (unsigned long long)pb, src);
        lda = __shfl_sync(0xffffffffu, la_, src);
        ldb = __shfl_sync(0xffffffffu, lb_, src);
        K = __shfl_sync(0xffffffffu, kb, src);
        vecA = __shfl_sync(0xffffffffu, va, src);
        vecB = __shfl_sync(0xffffffffu, vb, src);
        K4 = (K + 3) & ~3;
      };
      if (s.count > 0) fetch();
      auto fill = [&](int buf) -> int {
        int kfill = 0;
        float* a_s = sA[buf];
        float* b_s = sB[buf];
        while (q < s.count && kfill < GK) {
          if (K == 0) {
            ++q;
            if (q < s.count) fetch();
            continue;
          }
          const int take = min(K4 - koff, GK - kfill);  // a multiple of four
          if (!ta) {  // A row-major: rows of k into a_s[r * LDK + k]
            if (vecA) {
              for (int e = tid; e < TILE * (GK / 4); e += GNT) {
                const int r = e >> 3, c4 = (e & 7) * 4;
                if (r < mc && c4 < take) {
                  const int kr = K - (koff + c4);
                  cp_async16(&a_s[r * LDK + kfill + c4], A + (int64_t)(m0 + r) * lda + koff + c4,
                             (kr >= 4 ? 4 : kr) * 4);
                }
              }
            } else {
              for (int e = tid; e < TILE * GK; e += GNT) {
                const int r = e >> 5, kk = e & 31;
                if (r < mc && kk < take) {
                  if (koff + kk < K) cp_async(&a_s[r * LDK + kfill + kk], A + (int64_t)(m0 + r) * lda + koff + kk);
                  else a_s[r * LDK + kfill + kk] = 0.f;
                }
              }
            }
          } else {  // A transposed (k x m): rows of m into a_s[k * GPAD + r]
            for (int e = tid; e < GK * (TILE / 4); e += GNT) {
              const int kk = e >> 3, r4 = (e & 7) * 4;
              if (kk < take && r4 < mc) {
                float* d = &a_s[(kfill + kk) * GPAD + r4];
                const float* src = A + (int64_t)(koff + kk) * lda + m0 + r4;
                if (koff + kk >= K) {
                  *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
                } else if (vecA) {
                  cp_async16(d, src, 16);
                } else {
                  for (int u = 0; u < 4 && r4 + u < mc; ++u) cp_async(d + u, src + u);
                }
              }
            }
          }
          if (!tb) {  // B row-major (k x n): rows of n into b_s[k * GPAD + c]
            for (int e = tid; e < GK * (TILE / 4); e += GNT) {
              const int kk = e >> 3, c4 = (e & 7) * 4;
              if (kk < take && c4 < nc) {
                float* d = &b_s[(kfill + kk) * GPAD + c4];
                const float* src = B + (int64_t)(koff + kk) * ldb + n0 + c4;
                if (koff + kk >= K) {
                  *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
                } else if (vecB) {
                  cp_async16(d, src, 16);
                } else {
                  for (int u = 0; u < 4 && c4 + u < nc; ++u) cp_async(d + u, src + u);
                }
              }
            }
          } else {  // B transposed (n x k): element by element
            for (int e = tid; e < TILE * GK; e += GNT) {
              const int c = e >> 5, kk = e & 31;
              if (c < nc && kk < take) {
                if (koff + kk < K) cp_async(&b_s[(kfill + kk) * GPAD + c], B + (int64_t)(n0 + c) * ldb + koff + kk);
                else b_s[(kfill + kk) * GPAD + c] = 0.f;
              }
            }
          }
          const int kact = min(take, K - koff);
          work += 2ull * mc * nc * (kact > 0 ? kact : 0);
          kfill += take;
          koff += take;
          if (koff == K4) {
            koff = 0;
            ++q;
            if (q < s.count) fetch();
          }
        }
        return kfill;
      };
      int buf = 0;
      int kf = fill(0);
      cp_commit();
      while (kf > 0) {
        const int kf_next = fill(buf ^ 1);
        cp_commit();
        cp_wait1();
        __syncthreads();
        if (live) {
          if (!ta) slice_fma<true>(sA[buf], sB[buf], kf, qx, qy, acc, k0, kstep);
          else slice_fma<false>(sA[buf], sB[buf], kf, qx, qy, acc, k0, kstep);
        }
        __syncthreads();
        buf ^= 1;
        kf = kf_next;
      }
      if (split) {  // warp 0 adds warp 1's partial sums (the slices are done: sA is free)
        float* red = sA[0];
        if (tid >= 32) {
#pragma unroll
          for (int e = 0; e < 16; ++e) red[e * 32 + lane] = acc[e >> 2][e & 3];
        }
        __syncthreads();
        if (tid < 32) {
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[e >> 2][e & 3] += red[e * 32 + lane];
        }
        __syncthreads();
      }
      if (mine && (!split || tid < 32)) {
        if (s.flags & SF_TILE) {  // an operand tile of the BF16 split product (ldc: the tile's k)
          const bool tt = s.flags & SF_TILE_T;
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int r = m0 + 4 * qy + i, c = n0 + 4 * qx + j;
              if (r - m0 < mc && c - n0 < nc) tile_store(out.base, s.trows, s.ldc, tt ? c : r, tt ? r : c, acc[i][j]);
            }
        } else {
          const bool mirror = sym && !(tri && qx == qy);  // (a diagonal block holds both halves)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int r = 4 * qy + i, c = 4 * qx + j;
              if (r < mc && c < nc) {
                st<float>(out, (int64_t)(m0 + r) * s.ldc + n0 + c, acc[i][j], accum);
                if (mirror) st<float>(out, (int64_t)(n0 + c) * s.ldc + m0 + r, acc[i][j], accum);
              }
            }
        }
      }
    }
  }
  if (ar->flops && tid == 0 && work) atomicAdd(ar->flops, work);
}


template <typename Acc>
static void gemm_launch(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* ar,
                        int maxn, int variant, void* stream) {
  const int64_t kMaxGrid = 2147483647LL;
  // variant 0: one CTA per 32-column slice of a segment; 1: one CTA per segment (it walks
  // all column tiles).  Every output element is summed in the same order either way.
  int gy = variant == 1 ? 1 : (maxn + TILE - 1) / TILE;
  if (gy < 1) gy = 1;
  if (gy > 256) gy = 256;
  for (int64_t off = 0; off < count; off += kMaxGrid) {
    int64_t c = count - off < kMaxGrid ? count - off : kMaxGrid;
    dim3 grid((unsigned)c, (unsigned)gy);
    if constexpr (sizeof(Acc) == 4)
      seg_gemm32_kernel<<<grid, GNT, 0, (cudaStream_t)stream>>>(d_segs, d_items, first + off, ar);
    else
      seg_gemm_kernel<Acc><<<grid, GNT, 0, (cudaStream_t)stream>>>(d_segs, d_items, first + off, ar);
    g_launches += 1;
  }
}

void launch_gemm(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars,
                 int maxn, int maxdim, bool fp32, void* stream, int variant) {
  (void)maxdim;
  if (fp32) gemm_launch<float>(d_segs, d_items, first, count, d_ars, maxn, variant, stream);
  else gemm_launch<double>(d_segs, d_items, first, count, d_ars, maxn, variant, stream);
}

// ------------------------------------------------------------ plain sums
// A launch group whose segments are all plain sums of matrices (the collects of Eq.
// nonleafA / nonleafB, the split's additions): out (=|+=) sum over the items of A_q (m x n,
// leading dim lda; or operand tiles, SF_TILE), one warp per segment, each output element
// summed from zero in item order as in the GEMM kernels' sum path, four elements per lane
// in flight.
template <typename T>
__global__ void __launch_bounds__(256) seg_sum_kernel(const Seg* __restrict__ segs, const Item* __restrict__ items,
                                                      int64_t first, int64_t count, const Arenas* __restrict__ ars) {
  const int64_t si = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (si >= count) return;
  const int lane = threadIdx.x & 31;
  const Seg s = segs[first + si];
  const Arenas* ar = ars + s.inst;
  const View out = view(ar, s.out);
  const bool accum = s.flags & SF_ACC, tiled = s.flags & SF_TILE, tt = s.flags & SF_TILE_T;
  const int M = bound(ar, s.mref, s.m), N = bound(ar, s.nref, s.n), total = M * N;
  const Item* it = items + s.first;
  for (int e0 = 0; e0 < total; e0 += 128) {
    T acc[4];
    int r[4], c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + 32 * u + lane;
      r[u] = e / N;
      c[u] = e - r[u] * N;
      acc[u] = T(0);
    }
    for (int q = 0; q < s.count; ++q) {
      const T* A = ptr_of<T>(ar, it[q].a);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (e0 + 32 * u + lane < total)
          acc[u] += tiled ? (T)tile_load((const char*)A, s.trows, s.lda, tt ? c[u] : r[u], tt ? r[u] : c[u])
                          : (s.flags & SF_TA) ? A[(int64_t)c[u] * s.lda + r[u]] : A[(int64_t)r[u] * s.lda + c[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (e0 + 32 * u + lane < total) st<T>(out, (int64_t)r[u] * s.ldc + c[u], acc[u], accum);
  }
}

void launch_sum(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars, bool fp32,
                void* stream) {
  const int64_t kMaxGrid = 2147483647LL;
  for (int64_t off = 0; off < count; off += 8 * kMaxGrid) {
    const int64_t c = std::min(count - off, 8 * kMaxGrid);
    const unsigned grid = (unsigned)((c + 7) / 8);
    if (fp32)
      seg_sum_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>(d_segs, d_items, first + off, c, d_ars);
    else
      seg_sum_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(d_segs, d_items, first + off, c, d_ars);
    g_launches += 1;
  }
}

// The operand tiles of a matrix's dense leaf blocks (LS x LS, float64 in the arena) for the
// tensor-core dense products: block f as an A operand (tile position (r, c) = F[r][c]) at
// dst + f T and as a B operand (position (r, c) = F[c][r]) at dst + (nF + f) T, BF16 hi / lo
// parts of the float32 value; every position of the tiles is written (zeros past LS).
__global__ void f_tiles_kernel(const double* __restrict__ arena, int64_t off_F, int64_t nF, int LS, int tr, int kp,
                               char* __restrict__ dst) {
  const int64_t f = blockIdx.x;
  const double* F = arena + off_F + f * (int64_t)LS * LS;
  const int64_t T = (int64_t)tr * kp;  // floats per tile
  char* ta = dst + (size_t)(f * T) * 4;
  char* tb = dst + (size_t)((nF + f) * T) * 4;
  for (int e = threadIdx.x; e < tr * kp; e += blockDim.x) {
    const int r = e / kp, c = e - r * kp;
    const float xa = (r < LS && c < LS) ? (float)F[(int64_t)r * LS + c] : 0.f;
    const float xb = (r < LS && c < LS) ? (float)F[(int64_t)c * LS + r] : 0.f;
    tile_store(ta, tr, kp, r, c, xa);
    tile_store(tb, tr, kp, r, c, xb);
  }
}

void launch_f_tiles(const double* arena, int64_t off_F, int64_t nF, int LS, float* dst, void* stream) {
  if (nF <= 0) return;
  if (nF > 2147483647LL) throw Error(H2_EUNSUPPORTED, "more dense blocks than one launch covers");
  const int tr = (LS + 7) & ~7, kp = (LS + 15) & ~15;
  f_tiles_kernel<<<(unsigned)nF, 256, 0, (cudaStream_t)stream>>>(arena, off_F, nF, LS, tr, kp, (char*)dst);
  g_launches += 1;
}

__global__ void set_arenas_kernel(Arenas* dst, Arenas a) { *dst = a; }

void upload_arenas(Arenas* dst, const Arenas& a, void* stream) {
  set_arenas_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(dst, a);
  g_launches += 1;
}

Arenas to_arenas(const ArenaSet& a) {
  Arenas d;
  for (int i = 0; i < kArenas; ++i) d.p[i] = (char*)a.p[i];
  d.f32 = a.f32;
  for (int i = 0; i < 6; ++i) d.rk[i] = a.rk[i];
  d.flops = a.flops;
  d.kr = a.kr;
  d.kc = a.kc;
  d.cap_hits = a.cap_hits;
  return d;
}

__global__ void copy_ranks_kernel(const Arenas* __restrict__ ars, int inst, int64_t n) {
  const Arenas* a = ars + inst;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a->kr[i] = a->rk[RK_AR][i];
    a->kc[i] = a->rk[RK_BC][i];
  }
}

void launch_copy_ranks(const Arenas* d_ars, int inst, int64_t n, void* stream) {
  copy_ranks_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024)), 256, 0,
                      (cudaStream_t)stream>>>(d_ars, inst, n);
  g_launches += 1;
}

__global__ void to_f32_kernel(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) d[i] = (float)s[i];
}

void launch_to_f32(const double* src, float* dst, int64_t n, void* stream) {
  to_f32_kernel<<<4 * 152, 256, 0, (cudaStream_t)stream>>>(src, dst, n);
  g_launches += 1;
}

// ------------------------------------------------------------ eigen + truncation
// (the round-robin Jacobi sweeps and block sums are in jacobi.cuh)
constexpr int kEigSmemMax = 112;



__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = red[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
  return t;
}

// norm: H2_NORM_FROBENIUS scales each Gram matrix by 1 / ||G_m||_F, H2_NORM_SPECTRAL by
// 1 / lambda_max(G_m), the largest eigenvalue from a Jacobi decomposition of G_m alone
__global__ void __launch_bounds__(256) eig_kernel(const EigTask* __restrict__ tasks, int64_t first,
                                                  const Arenas* __restrict__ ars, double eps, int trunc,
                                                  int norm, double* scratch, int64_t scratch_stride) {
  extern __shared__ double smem[];
  __shared__ int act[256];
  __shared__ double red[8];
  __shared__ double cs[128], sn[128];
  __shared__ int pp[128], qq[128];
  __shared__ int order[256];
  __shared__ double lam[256];
  __shared__ int s_n, s_rank;
  const EigTask t = tasks[first + blockIdx.x];
  const Arenas* ar = ars + t.inst;  // the task's product instance
  int32_t* const kr = ar->kr;
  int32_t* const kc = ar->kc;
  unsigned long long* const cap_hits = ar->cap_hits;
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
  const int nn = n + (n & 1), lds = nn + 1, sz = nn * lds;
  double *A, *V;
  if (nn <= kEigSmemMax) {
    A = smem;
    V = smem + sz;
  } else {
    A = scratch + blockIdx.x * scratch_stride;
    V = A + sz;
  }
  // spectral norms of the Gram matrices (H2_NORM_SPECTRAL): each one decomposed alone
  __shared__ double s_lmax[3];
  if (norm == H2_NORM_SPECTRAL) {
    for (int m = 0; m < 3; ++m) {
      if (t.g[m] < 0) continue;
      const View G = view(ar, t.g[m]);
      for (int e = tid; e < sz; e += nt) {
        A[e] = 0.0;
        V[e] = (e / lds == e % lds) ? 1.0 : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += nt)
        A[(e / n) * lds + (e % n)] = ld<double>(G, (int64_t)act[e / n] * t.n_pad + act[e % n]);
      __syncthreads();
      for (int e = tid; e < nn * nn; e += nt) {
        const int a = e / nn, b = e % nn;
        if (a < b) {
          const double v = 0.5 * (A[a * lds + b] + A[b * lds + a]);
          A[a * lds + b] = v;
          A[b * lds + a] = v;
        }
      }
      __syncthreads();
      jacobi_sweeps<double>(A, V, nn, lds, 30, 1e-30, red, cs, sn, pp, qq);
      double mx = 0.0;
      for (int a = tid; a < n; a += nt) mx = fmax(mx, A[a * lds + a]);
      mx = block_max(mx, red);
      if (tid == 0) s_lmax[m] = mx;
      __syncthreads();
    }
  }
  // normalised sum of the Gram matrices over the active rows/cols
  for (int e = tid; e < sz; e += nt) A[e] = 0.0;
  __syncthreads();
  for (int m = 0; m < 3; ++m) {
    if (t.g[m] < 0) continue;
    const View G = view(ar, t.g[m]);
    double loc = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      double v = ld<double>(G, (int64_t)act[e / n] * t.n_pad + act[e % n]);
      loc += v * v;
    }
    double nrm2 = block_sum(loc, red);
    if (nrm2 > 0.0 && (norm != H2_NORM_SPECTRAL || s_lmax[m] > 0.0)) {
      double inv = norm == H2_NORM_SPECTRAL ? 1.0 / s_lmax[m] : 1.0 / sqrt(nrm2);
      for (int e = tid; e < n * n; e += nt)
        A[(e / n) * lds + (e % n)] += ld<double>(G, (int64_t)act[e / n] * t.n_pad + act[e % n]) * inv;
    }
    __syncthreads();
  }
  // symmetrise (the Grams are symmetric up to rounding of their products)
  for (int e = tid; e < sz; e += nt) V[e] = (e / lds == e % lds) ? 1.0 : 0.0;
  for (int e = tid; e < nn * nn; e += nt) {
    int a = e / nn, b = e % nn;
    if (a < b) {
      double v = 0.5 * (A[a * lds + b] + A[b * lds + a]);
      A[a * lds + b] = v;
      A[b * lds + a] = v;
    }
  }
  __syncthreads();
  jacobi_sweeps<double>(A, V, nn, lds, 30, 1e-30, red, cs, sn, pp, qq);
  // order by decreasing eigenvalue (ties by index); only the n active ones
  for (int a = tid; a < n; a += nt) lam[a] = A[a * lds + a];
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
    if (r > t.klim) {
      r = t.klim;
      atomicAdd(cap_hits, 1ull);
    }
    s_rank = r;
    ranks[t.rank_out] = r;
  }
  __syncthreads();
  const int rank = s_rank;
  double* out = (double*)view(ar, t.out).base;  // the new bases are float64 (arena C)
  // float copy for the GEMMs of the mixed product (arena X mirrors C's basis region)
  float* out32 = ar->p[AR_X] ? (float*)ar->p[AR_X] + (t.out & kOffMask) : nullptr;
  for (int e = tid; e < t.n_pad * t.kcap; e += nt) {
    out[e] = 0.0;
    if (out32) out32[e] = 0.f;
  }
  __syncthreads();
  // sign: the entry of largest magnitude (first such) is positive
  for (int c = tid; c < rank; c += nt) {
    int col = order[c];
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < n; ++a) {
      double v = fabs(V[a * lds + col]);
      if (v > bv) { bv = v; best = a; }
    }
    double sg = V[best * lds + col] < 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < n; ++a) {
      const double v = sg * V[a * lds + col];
      out[(int64_t)act[a] * t.kcap + c] = v;
      if (out32) out32[(int64_t)act[a] * t.kcap + c] = (float)v;
    }
  }
}

// ------------------------------------------------------------ mixed eigen kernel
// Same task as eig_kernel for the mixed-precision product, with the float64 work
// cut to what decides the result: (1) cyclic round-robin Jacobi in float32 on the
// normalised Gram sum G (eigenvalue errors ~1e-7 lambda_1, far below the truncation
// thresholds); (2) the float32 eigenvectors are re-orthonormalised in float64 by one
// Newton-Schulz step V <- V (3 I - V^T V) / 2 (1e-7 -> 1e-14); (3) the eigenvalues
// that decide the ranks are the float64 Rayleigh quotients v_j^T G v_j, or, for
// thresholds below 5e-5 lambda_1, the eigenvalues of V^T G V after float64 Jacobi
// refinement.  The new bases are V's leading columns (float64, orthonormal to
// ~1e-14).  Shared memory: G, V, T, each n x n float64 (n <= 96).
constexpr int kMixMax = 96;

// C = op(X) op(Y) for nn x nn float64 matrices in shared memory, row stride lds
// (C distinct from X, Y); each thread computes four outputs of one row with
// independent accumulators
__device__ void smem_gemm(const double* X, bool tx, const double* Y, bool ty, double* C, int nn, int lds) {
  const int nq = (nn + 3) / 4;
  for (int e = threadIdx.x; e < nn * nq; e += blockDim.x) {
    const int i = e / nq, j0 = (e % nq) * 4;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int k = 0; k < nn; ++k) {
      const double x = tx ? X[k * lds + i] : X[i * lds + k];
      double y0 = ty ? Y[j0 * lds + k] : Y[k * lds + j0];
      double y1 = (j0 + 1 < nn) ? (ty ? Y[(j0 + 1) * lds + k] : Y[k * lds + j0 + 1]) : 0.0;
      double y2 = (j0 + 2 < nn) ? (ty ? Y[(j0 + 2) * lds + k] : Y[k * lds + j0 + 2]) : 0.0;
      double y3 = (j0 + 3 < nn) ? (ty ? Y[(j0 + 3) * lds + k] : Y[k * lds + j0 + 3]) : 0.0;
      a0 = fma(x, y0, a0);
      a1 = fma(x, y1, a1);
      a2 = fma(x, y2, a2);
      a3 = fma(x, y3, a3);
    }
    C[i * lds + j0] = a0;
    if (j0 + 1 < nn) C[i * lds + j0 + 1] = a1;
    if (j0 + 2 < nn) C[i * lds + j0 + 2] = a2;
    if (j0 + 3 < nn) C[i * lds + j0 + 3] = a3;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) eig_mixed_kernel(const EigTask* __restrict__ tasks, int64_t first,
                                                        const Arenas* __restrict__ ars, double eps, int trunc) {
  extern __shared__ double smem[];
  __shared__ int act[kMixMax + 2];
  __shared__ double red[8];
  __shared__ double cs[kMixMax / 2 + 1], sn[kMixMax / 2 + 1];
  __shared__ float cs32[kMixMax / 2 + 1], sn32[kMixMax / 2 + 1];
  __shared__ int pp[kMixMax / 2 + 1], qq[kMixMax / 2 + 1];
  __shared__ int order[kMixMax + 2];
  __shared__ double lam[kMixMax + 2];
  __shared__ double rowbuf[4 * kMixMax];
  __shared__ int s_n, s_rank;
  const EigTask t = tasks[first + blockIdx.x];
  const Arenas* ar = ars + t.inst;  // the task's product instance
  int32_t* const kr = ar->kr;
  int32_t* const kc = ar->kc;
  unsigned long long* const cap_hits = ar->cap_hits;
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
  const int n = s_n, nn = n + (n & 1), lds = nn + 1, sz = nn * lds;
  double* G = smem;               // normalised Gram sum (row stride lds)
  double* V = smem + sz;          // eigenvectors (float64)
  double* T = smem + 2 * sz;      // work: float32 A and V during step (1), products later
  float* A32 = (float*)T;
  float* V32 = A32 + sz;
  for (int e = tid; e < sz; e += nt) G[e] = 0.0;
  __syncthreads();
  for (int m = 0; m < 3; ++m) {
    if (t.g[m] < 0) continue;
    const View Gm = view(ar, t.g[m]);
    double loc = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      double v = ld<double>(Gm, (int64_t)act[e / n] * t.n_pad + act[e % n]);
      loc += v * v;
    }
    double nrm2 = block_sum(loc, red);
    if (nrm2 > 0.0) {
      double inv = 1.0 / sqrt(nrm2);
      for (int e = tid; e < n * n; e += nt)
        G[(e / n) * lds + (e % n)] += ld<double>(Gm, (int64_t)act[e / n] * t.n_pad + act[e % n]) * inv;
    }
    __syncthreads();
  }
  for (int e = tid; e < nn * nn; e += nt) {
    int a = e / nn, b = e % nn;
    if (a < b) {
      double v = 0.5 * (G[a * lds + b] + G[b * lds + a]);
      G[a * lds + b] = v;
      G[b * lds + a] = v;
    }
  }
  __syncthreads();
  // (1) float32 Jacobi
  for (int e = tid; e < sz; e += nt) {
    A32[e] = (float)G[e];
    V32[e] = (e / lds == e % lds) ? 1.f : 0.f;
  }
  __syncthreads();
  // float32 sweeps until the off-diagonal is below 1e-5 of the total (a looser stop
  // moves the mixed product by more than 2 eps at eps = 1e-4)
  const double thr_rel = trunc == H2_TRUNC_SV ? eps * eps : eps;
  const bool refine = trunc != H2_TRUNC_FULL && thr_rel < 5e-5;
  jacobi_sweeps<float>(A32, V32, nn, lds, 12, 1e-10, red, cs32, sn32, pp, qq);
  for (int e = tid; e < sz; e += nt) V[e] = (double)V32[e];
  __syncthreads();
  // (2) one Newton-Schulz step: V <- V (3 I - V^T V) / 2, computed as T = V W
  {
    smem_gemm(V, true, V, false, T, nn, lds);          // T = V^T V
    for (int e = tid; e < sz; e += nt) {
      int i = e / lds, j = e % lds;
      T[e] = ((i == j) ? 1.5 : 0.0) - 0.5 * T[e];
    }
    __syncthreads();
    // V <- V T, four rows at a time through a small buffer
    for (int i0 = 0; i0 < nn; i0 += 4) {
      const int ni = min(4, nn - i0);
      for (int e = tid; e < ni * nn; e += nt) {
        int i = i0 + e / nn, j = e % nn;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
        for (; k + 1 < nn; k += 2) {
          a0 = fma(V[i * lds + k], T[k * lds + j], a0);
          a1 = fma(V[i * lds + k + 1], T[(k + 1) * lds + j], a1);
        }
        if (k < nn) a0 = fma(V[i * lds + k], T[k * lds + j], a0);
        rowbuf[e] = a0 + a1;
      }
      __syncthreads();
      for (int e = tid; e < ni * nn; e += nt) V[(i0 + e / nn) * lds + e % nn] = rowbuf[e];
      __syncthreads();
    }
  }
  // (3) float64 Rayleigh quotients lambda_j = v_j^T G v_j decide the ranks.  When the
  // truncation threshold is below what float32 eigenvectors resolve (< 5e-5 of
  // lambda_1), the float64 Rayleigh-Ritz matrix B = V^T G V is diagonalised by float64
  // Jacobi sweeps first (rotations accumulated into V).
  smem_gemm(G, false, V, false, T, nn, lds);   // T = G V
  if (refine) {
    smem_gemm(V, true, T, false, G, nn, lds);  // G <- V^T T = B
    for (int e = tid; e < nn * nn; e += nt) {
      int a = e / nn, b = e % nn;
      if (a < b) {
        double v = 0.5 * (G[a * lds + b] + G[b * lds + a]);
        G[a * lds + b] = v;
        G[b * lds + a] = v;
      }
    }
    __syncthreads();
    jacobi_sweeps<double>(G, V, nn, lds, 8, 1e-24, red, cs, sn, pp, qq);
    for (int j = tid; j < n; j += nt) lam[j] = G[j * lds + j];
  } else {
    for (int j = tid; j < n; j += nt) {
      double a0 = 0.0, a1 = 0.0;
      int i = 0;
      for (; i + 1 < nn; i += 2) {
        a0 = fma(V[i * lds + j], T[i * lds + j], a0);
        a1 = fma(V[(i + 1) * lds + j], T[(i + 1) * lds + j], a1);
      }
      if (i < nn) a0 = fma(V[i * lds + j], T[i * lds + j], a0);
      lam[j] = a0 + a1;
    }
  }
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
    if (r > t.klim) {
      r = t.klim;
      atomicAdd(cap_hits, 1ull);
    }
    s_rank = r;
    ranks[t.rank_out] = r;
  }
  __syncthreads();
  const int rank = s_rank;
  double* out = (double*)view(ar, t.out).base;  // the new bases are float64 (arena C)
  // float copy for the GEMMs of the mixed product (arena X mirrors C's basis region)
  float* out32 = ar->p[AR_X] ? (float*)ar->p[AR_X] + (t.out & kOffMask) : nullptr;
  for (int e = tid; e < t.n_pad * t.kcap; e += nt) {
    out[e] = 0.0;
    if (out32) out32[e] = 0.f;
  }
  __syncthreads();
  for (int c = tid; c < rank; c += nt) {
    int col = order[c];
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < n; ++a) {
      double v = fabs(V[a * lds + col]);
      if (v > bv) { bv = v; best = a; }
    }
    double sg = V[best * lds + col] < 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < n; ++a) {
      const double v = sg * V[a * lds + col];
      out[(int64_t)act[a] * t.kcap + c] = v;
      if (out32) out32[(int64_t)act[a] * t.kcap + c] = (float)v;
    }
  }
}

// ------------------------------------------------------------ mixed eigen kernel, kept columns only
// The same result as eig_mixed_kernel for truncation thresholds of 5e-5 lambda_1 and
// above (and the full mode), with the work cut where it does not decide the result:
//   (1) float32 round-robin Jacobi on G padded with zero rows and columns to a
//       multiple of four (pad indices are never rotated).  G is summed straight from the
//       three Gram matrices in global memory into float32 (no float64 copy of G is
//       kept).  One step rotates rows and columns together: a thread takes the 2 x 2
//       block (pair k, pair l), k <= l, of A, forms M_k X M_l^T and writes the block and
//       its mirror image; eigenvectors are the ROWS of Vt, so their update is a float4
//       row rotation.  The (k, l) and (pair, row piece) tasks of a step are read from
//       tables built once per CTA.  Rotations with |a_pq| <= 2^-24 sqrt(|a_pp a_qq|) are
//       skipped (below float32 resolution of their 2 x 2 problem; together they keep
//       off(A)^2 far below the 1e-10 stop);
//   (2) a_jj is v_j^T G v_j to float32 accuracy: the columns with a_jj above a
//       quarter of the threshold are the only ones whose quotient can pass it, and for
//       the decisive ones (the top cluster and those within 2e-5 lambda_1 of the
//       threshold) the float64 Rayleigh quotient v^T G v / v^T v is formed, G read from
//       the Gram matrices in global memory; these decide the rank (sorted decreasing,
//       ties by index);
//   (3) the kept columns go to float64, in place in the output (rows act[a]), and one
//       Newton-Schulz step on those columns, V <- V (3 I - V^T V) / 2, makes them
//       orthonormal to the square of their float32 error (V^T V in float64; the small
//       correction V (V^T V - I) / 2 in float32).
// Every sum whose rounding could change a decision (the norms of the Gram matrices, the
// stopping sums) is taken over 128 fixed partial sums, so the result does not depend on
// the block size (128 or 256 threads: a launch parameter).
// Float64 work: n^2 per decisive candidate plus n r^2 / 2, against 3 n^3 in eig_mixed_kernel.
// Shared memory: buffer 1 holds A (float32, nn x (nn+1)) and later V^T V - I (float32,
// packed lower triangle); buffer 2 holds Vt (float32, nn x (nn+4)) and
// later a few new rows of the kept columns; then the step's task tables.
constexpr int kKeptRows = 4;
constexpr int kFixedParts = 128;
constexpr int kEigTiers = 6;  // size tiers of the mixed eigen step (up to 32, 48, 56, 64, 80, 96)

__host__ __device__ inline int round4(int n) { return (n + 3) & ~3; }

__host__ __device__ inline size_t eig_kept_buf1(int nn) { return ((size_t)nn * (nn + 1) * sizeof(float) + 15) & ~(size_t)15; }
__host__ __device__ inline size_t eig_kept_buf2(int nn) { return (size_t)nn * (nn + 4) * sizeof(float); }
__host__ __device__ inline int eig_kept_nblk(int nn) { return (nn / 4) * (nn / 2 + 1); }
__host__ __device__ inline int eig_kept_nvt(int nn) { return (nn / 2) * (nn / 4); }
__host__ __device__ inline size_t eig_kept_smem(int nn) {
  return eig_kept_buf1(nn) + eig_kept_buf2(nn) +
         (((size_t)(eig_kept_nblk(nn) + eig_kept_nvt(nn)) * sizeof(uint16_t) + 15) & ~(size_t)15);
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// the sum of parts[0 .. kFixedParts) in a fixed order, returned to every thread
__device__ double fixed_total(const double* parts, double* bc) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = 0.0;
    for (int u = threadIdx.x; u < kFixedParts; u += 32) r += parts[u];
    r = warp_sum_d(r);
    if (threadIdx.x == 0) *bc = r;
  }
  __syncthreads();
  return *bc;
}

__global__ void __launch_bounds__(256) eig_mixed_kept_kernel(const EigTask* __restrict__ tasks, int64_t first,
                                                             const Arenas* __restrict__ ars, double eps, int trunc,
                                                             int nn_lo, int nn_hi) {
  extern __shared__ __align__(16) unsigned char esm[];
  __shared__ int act[kMixMax + 4];
  __shared__ double parts[kFixedParts];
  __shared__ float2 parts2[kFixedParts];
  __shared__ double s_bc;
  __shared__ float2 csn[kMixMax / 2];  // (c, s) of pair k
  __shared__ int pq[kMixMax / 2];      // p | q << 16 of pair k
  __shared__ int cand[kMixMax], order[kMixMax];
  __shared__ double rq[kMixMax], rqs[kMixMax];
  __shared__ float lam32[kMixMax];
  __shared__ double s_inv[3];
  __shared__ int s_nc, s_rank;
  const EigTask t = tasks[first + blockIdx.x];
  const Arenas* ar = ars + t.inst;  // the task's product instance
  int32_t* const kr = ar->kr;
  int32_t* const kc = ar->kc;
  unsigned long long* const cap_hits = ar->cap_hits;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  int32_t* ranks = t.col ? kc : kr;
  // the task's size first: one launch per size tier (nn_lo, nn_hi], shared memory sized
  // for nn_hi; a task whose size is outside the tier returns at once (another launch
  // does it)
  const int k1 = t.child1 < 0 ? t.nleaf : ranks[t.child1], k2 = t.child1 < 0 ? 0 : ranks[t.child2];
  const int n = k1 + k2, nn = round4(n), np = nn / 2, la = nn + 1, lv = nn + 4;
  if (nn <= nn_lo || nn > nn_hi) return;
  // active rows: child 1's kept rows, then child 2's (at offset half)
  for (int a = tid; a < n; a += nt) act[a] = a < k1 ? a : t.half + (a - k1);
  __syncthreads();
  float* A = (float*)esm;                                  // row stride la (buffer 1)
  float* Vt = (float*)(esm + eig_kept_buf1(nn_hi));        // row stride lv; 16-byte aligned rows (buffer 2)
  uint16_t* blk = (uint16_t*)(esm + eig_kept_buf1(nn_hi) + eig_kept_buf2(nn_hi));
  const int half = np / 2, nq = nn / 4, nblk = half * (np + 1), nvt = np * nq;
  uint16_t* vtk = blk + nblk;
  // step tasks: the triangle k <= l of 2 x 2 blocks folded into half x (np + 1), as
  // k | l << 8; the Vt row pieces as pair | piece << 8
  for (int e = tid; e < nblk; e += nt) {
    const int r = e / (np + 1), cc = e - r * (np + 1);
    int k, l;
    if (cc < np - r) {
      k = r;
      l = r + cc;
    } else {
      k = np - 1 - r;
      l = k + cc - (np - r);
    }
    blk[e] = (uint16_t)(k | (l << 8));
  }
  for (int e = tid; e < nvt; e += nt) vtk[e] = (uint16_t)((e / nq) | ((e % nq) << 8));
  // scale of each Gram matrix: 1 / ||G_m||_F (0: absent or zero, left out of the sum)
  for (int m = 0; m < 3; ++m) {
    for (int v = tid; v < kFixedParts; v += nt) {
      double loc = 0.0;
      if (t.g[m] >= 0) {
        const View Gm = view(ar, t.g[m]);
        for (int e = v; e < n * n; e += kFixedParts) {
          const double x = ld<double>(Gm, (int64_t)act[e / n] * t.n_pad + act[e % n]);
          loc += x * x;
        }
      }
      parts[v] = loc;
    }
    const double nrm2 = fixed_total(parts, &s_bc);
    if (tid == 0) s_inv[m] = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
  }
  __syncthreads();
  // A = the normalised sum (float32), zero padding, symmetrised; Vt = I
  for (int e = tid; e < nn * la; e += nt) {
    const int a = e / la, b = e - a * la;
    float v = 0.f;
    if (a < n && b < n)
      for (int m = 0; m < 3; ++m)
        if (s_inv[m] > 0.0) v = fmaf(ld<float>(view(ar, t.g[m]), (int64_t)act[a] * t.n_pad + act[b]), (float)s_inv[m], v);
    A[e] = v;
  }
  for (int e = tid; e < nn * lv; e += nt) Vt[e] = (e / lv == e % lv) ? 1.f : 0.f;
  __syncthreads();
  for (int e = tid; e < nn * nn; e += nt) {
    const int a = e / nn, b = e % nn;
    if (a < b) {
      const float v = 0.5f * (A[a * la + b] + A[b * la + a]);
      A[a * la + b] = v;
      A[b * la + a] = v;
    }
  }
  __syncthreads();
  // (1) float32 Jacobi, stop when off(A)^2 <= 1e-10 |A|^2 (as eig_mixed_kernel)
  for (int sweep = 0; sweep < 12 && n > 1; ++sweep) {
    // (sums of squares in float32: they only decide a stop at a 1e-10 ratio)
    for (int v = tid; v < kFixedParts; v += nt) {
      float offf = 0.f, totf = 0.f;
      for (int e = v; e < nn * nn; e += kFixedParts) {
        const int i = e / nn, j = e - i * nn;
        const float x = A[i * la + j] * A[i * la + j];
        totf += x;
        if (i != j) offf += x;
      }
      parts2[v] = make_float2(offf, totf);
    }
    __syncthreads();
    if (tid < 32) {
      double o = 0.0, tt = 0.0;
      for (int u = tid; u < kFixedParts; u += 32) {
        o += (double)parts2[u].x;
        tt += (double)parts2[u].y;
      }
      o = warp_sum_d(o);
      tt = warp_sum_d(tt);
      if (tid == 0) s_bc = (o > 1e-10 * tt) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (!(s_bc > 0.0)) break;
    for (int step = 0; step < nn - 1; ++step) {
      if (tid < np) {
        int pa = 0;
        if (tid > 0) {
          pa = tid - 1 + step;
          if (pa >= nn - 1) pa -= nn - 1;
          pa += 1;
        }
        int pb = nn - 2 - tid + step;
        if (pb >= nn - 1) pb -= nn - 1;
        pb += 1;
        const int p = min(pa, pb), q = max(pa, pb);
        const float apq = A[p * la + q], app = A[p * la + p], aqq = A[q * la + q];
        float c = 1.f, s = 0.f;
        if (apq != 0.f && fabsf(apq) > 5.9604645e-8f * sqrtf(fabsf(app) * fabsf(aqq))) {
          const float tau = (aqq - app) / (2.f * apq);
          const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = 1.f / sqrtf(1.f + tt * tt);
          s = tt * c;
        }
        pq[tid] = p | (q << 16);
        csn[tid] = make_float2(c, s);
      }
      __syncthreads();
      // A <- M A M^T by 2 x 2 blocks (k, l), k <= l, and their mirror images
      for (int e = tid; e < nblk; e += nt) {
        const int kl = blk[e], k = kl & 255, l = kl >> 8;
        const float2 rk = csn[k], rl = csn[l];
        if (rk.y == 0.f && rl.y == 0.f) continue;
        const float ck = rk.x, sk = rk.y, cl = rl.x, sl = rl.y;
        const int pqk = pq[k], pql = pq[l];
        const int pk = pqk & 0xffff, qk = pqk >> 16, pl = pql & 0xffff, ql = pql >> 16;
        const float x = A[pk * la + pl], y = A[pk * la + ql], z = A[qk * la + pl], u = A[qk * la + ql];
        const float r00 = ck * x - sk * z, r01 = ck * y - sk * u;  // rows: M_k X
        const float r10 = sk * x + ck * z, r11 = sk * y + ck * u;
        const float b00 = cl * r00 - sl * r01, b10 = cl * r10 - sl * r11;  // columns: (M_k X) M_l^T
        float b01 = sl * r00 + cl * r01, b11 = sl * r10 + cl * r11;
        if (k == l) {
          A[pk * la + pk] = b00;
          A[qk * la + qk] = b11;
          A[pk * la + qk] = 0.f;
          A[qk * la + pk] = 0.f;
        } else {
          A[pk * la + pl] = b00;
          A[pk * la + ql] = b01;
          A[qk * la + pl] = b10;
          A[qk * la + ql] = b11;
          A[pl * la + pk] = b00;
          A[ql * la + pk] = b01;
          A[pl * la + qk] = b10;
          A[ql * la + qk] = b11;
        }
      }
      // Vt <- M Vt (rows p, q of each pair)
      for (int e = tid; e < nvt; e += nt) {
        const int kj = vtk[e], k = kj & 255, j = (kj >> 8) * 4;
        const float2 r = csn[k];
        const float s = r.y;
        if (s == 0.f) continue;
        const float c = r.x;
        const int pqk = pq[k];
        float4* rp = reinterpret_cast<float4*>(Vt + (pqk & 0xffff) * lv + j);
        float4* rr = reinterpret_cast<float4*>(Vt + (pqk >> 16) * lv + j);
        const float4 x = *rp, y = *rr;
        *rp = make_float4(c * x.x - s * y.x, c * x.y - s * y.y, c * x.z - s * y.z, c * x.w - s * y.w);
        *rr = make_float4(s * x.x + c * y.x, s * x.y + c * y.y, s * x.z + c * y.z, s * x.w + c * y.w);
      }
      __syncthreads();
    }
  }
  for (int j = tid; j < n; j += nt) lam32[j] = A[j * la + j];
  __syncthreads();
  // (2) candidates and their float64 Rayleigh quotients
  const double thr = trunc == H2_TRUNC_SV ? eps * eps : eps;
  // a_jj differs from the float64 quotient of v_j by ~1e-6 lambda_1 (float32 rounding
  // of the accumulated rotations); the quotient is formed in float64 only where that
  // can change the result: the top cluster (lambda_1) and the columns within
  // 2e-5 lambda_1 of the threshold; elsewhere a_jj stands in for it
  __shared__ int s_nd;
  __shared__ int dq[kMixMax];
  if (tid == 0) {
    float mx = 0.f;
    for (int j = 0; j < n; ++j) mx = fmaxf(mx, lam32[j]);
    const float del = 1e-5f * mx, tau = (float)thr * mx;
    int nc = 0, nd = 0;
    for (int j = 0; j < n; ++j)
      if (trunc == H2_TRUNC_FULL || (mx > 0.f && lam32[j] > 0.25f * tau)) {
        rq[nc] = (double)lam32[j];
        if (trunc != H2_TRUNC_FULL && (lam32[j] >= mx - del || fabsf(lam32[j] - tau) <= 2.f * del)) dq[nd++] = nc;
        cand[nc++] = j;
      }
    s_nc = nc;
    s_nd = nd;
  }
  __syncthreads();
  const int nc = s_nc, nd = s_nd;
  for (int di = w; di < nd; di += nw) {
    const int ci = dq[di];
    const float* v = Vt + cand[ci] * lv;
    double num = 0.0, den = 0.0;
    for (int a = lane; a < n; a += 32) {
      double ga = 0.0;
      for (int m = 0; m < 3; ++m) {
        if (!(s_inv[m] > 0.0)) continue;
        const View Gm = view(ar, t.g[m]);
        const int64_t row = (int64_t)act[a] * t.n_pad;
        double a0 = 0.0, a1 = 0.0;
        int b = 0;
        for (; b + 1 < n; b += 2) {
          a0 = fma(ld<double>(Gm, row + act[b]), (double)v[b], a0);
          a1 = fma(ld<double>(Gm, row + act[b + 1]), (double)v[b + 1], a1);
        }
        if (b < n) a0 = fma(ld<double>(Gm, row + act[b]), (double)v[b], a0);
        ga = fma(a0 + a1, s_inv[m], ga);
      }
      const double va = (double)v[a];
      num = fma(va, ga, num);
      den = fma(va, va, den);
    }
    num = warp_sum_d(num);
    den = warp_sum_d(den);
    if (lane == 0) rq[ci] = den > 0.0 ? num / den : 0.0;
  }
  __syncthreads();
  for (int a = tid; a < nc; a += nt) {
    int pos = 0;
    for (int b = 0; b < nc; ++b)
      if (rq[b] > rq[a] || (rq[b] == rq[a] && b < a)) ++pos;
    order[pos] = cand[a];
    rqs[pos] = rq[a];
  }
  __syncthreads();
  if (tid == 0) {
    int r = 0;
    if (trunc == H2_TRUNC_FULL) {
      r = nc;
    } else if (nc > 0 && rqs[0] > 0.0) {
      const double l1 = rqs[0];
      while (r < nc && rqs[r] > thr * l1) ++r;
    }
    if (r > t.klim) {
      r = t.klim;
      atomicAdd(cap_hits, 1ull);
    }
    s_rank = r;
    ranks[t.rank_out] = r;
  }
  __syncthreads();
  // (3) kept columns in float64 in the output (the new bases are float64, arena C): row
  // act[a] holds v_a; everything else is zero
  const int rank = s_rank;
  double* out = (double*)view(ar, t.out).base;
  float* out32 = ar->p[AR_X] ? (float*)ar->p[AR_X] + (t.out & kOffMask) : nullptr;
  const int ko = t.kcap;
  for (int e = tid; e < t.n_pad * ko; e += nt) out[e] = 0.0;
  __syncthreads();
  for (int e = tid; e < n * rank; e += nt) {
    const int a = e / rank, c = e - a * rank;
    out[(int64_t)act[a] * ko + c] = (double)Vt[order[c] * lv + a];
  }
  __syncthreads();
  if (rank > 0) {
    // the Newton-Schulz step V <- V (3 I - V^T V) / 2 = V - V E / 2 with E = V^T V - I:
    // E (~1e-6: the float32 rotations' drift) is summed in float64 and kept in float32
    // (absolute error ~1e-13), so that V E can be formed in float32; E is symmetric:
    // lower triangle, packed, in buffer 1 (A is no longer read)
    float* E = reinterpret_cast<float*>(esm);
    for (int e = tid; e < rank * rank; e += nt) {
      const int i = e / rank, j = e - i * rank;
      if (j > i) continue;
      double a0 = 0.0, a1 = 0.0;
      int a = 0;
      for (; a + 1 < n; a += 2) {
        const double* r0 = out + (int64_t)act[a] * ko;
        const double* r1 = out + (int64_t)act[a + 1] * ko;
        a0 = fma(r0[i], r0[j], a0);
        a1 = fma(r1[i], r1[j], a1);
      }
      if (a < n) {
        const double* r0 = out + (int64_t)act[a] * ko;
        a0 = fma(r0[i], r0[j], a0);
      }
      E[i * (i + 1) / 2 + j] = (float)((a0 + a1) - (i == j ? 1.0 : 0.0));
    }
    __syncthreads();
    // V <- V - V E / 2, a few rows at a time through buffer 2 (Vt is no longer read)
    double* rowbuf = reinterpret_cast<double*>(Vt);
    for (int r0 = 0; r0 < n; r0 += kKeptRows) {
      const int na = min(kKeptRows, n - r0);
      for (int e = tid; e < na * rank; e += nt) {
        const int a = r0 + e / rank, j = e % rank;
        const double* row = out + (int64_t)act[a] * ko;
        float s0 = 0.f, s1 = 0.f;
        int i = 0;
        for (; i + 1 < rank; i += 2) {
          const float e0 = i >= j ? E[i * (i + 1) / 2 + j] : E[j * (j + 1) / 2 + i];
          const float e1 = i + 1 >= j ? E[(i + 1) * (i + 2) / 2 + j] : E[j * (j + 1) / 2 + i + 1];
          s0 = fmaf((float)row[i], e0, s0);
          s1 = fmaf((float)row[i + 1], e1, s1);
        }
        if (i < rank) s0 = fmaf((float)row[i], i >= j ? E[i * (i + 1) / 2 + j] : E[j * (j + 1) / 2 + i], s0);
        rowbuf[e] = row[j] - 0.5 * (double)(s0 + s1);
      }
      __syncthreads();
      for (int e = tid; e < na * rank; e += nt) out[(int64_t)act[r0 + e / rank] * ko + e % rank] = rowbuf[e];
      __syncthreads();
    }
  }
  // sign: the entry of largest magnitude (first such) is positive; the float copy for the
  // GEMMs of the mixed product (arena X mirrors C's basis region)
  if (out32)
    for (int e = tid; e < t.n_pad * ko; e += nt) out32[e] = 0.f;
  for (int c = tid; c < rank; c += nt) {
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < n; ++a) {
      const double v = fabs(out[(int64_t)act[a] * ko + c]);
      if (v > bv) {
        bv = v;
        best = a;
      }
    }
    const double sg = out[(int64_t)act[best] * ko + c] < 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < n; ++a) {
      const int64_t o = (int64_t)act[a] * ko + c;
      const double v = sg * out[o];
      out[o] = v;
      if (out32) out32[o] = (float)v;
    }
  }
}

// the eigen kernels' shared-memory limits, set once per process (before any launch or
// stream capture)
void init_kernel_attributes() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(eig_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(3 * kMixMax * (kMixMax + 1) * sizeof(double)));
    cudaFuncSetAttribute(eig_mixed_kept_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)eig_kept_smem(kMixMax));
    cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * kEigSmemMax * (kEigSmemMax + 1) * sizeof(double)));
  });
  init_coup_tc_attributes();
}

// auxiliary streams of the concurrent eigen tiers, one set per (device, calling stream);
// nullptr if they cannot be made (the tiers then run in order on the calling stream)
struct TierStreams {
  cudaStream_t s[kEigTiers];
  cudaEvent_t fork, join[kEigTiers];
};

static std::mutex g_tier_mu;
static std::map<std::pair<int, cudaStream_t>, TierStreams*> g_tier_sets;  // by (device, calling stream)
static std::map<int, std::vector<TierStreams*>> g_tier_free;            // released sets, by device

static const TierStreams* tier_streams(cudaStream_t caller) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_tier_mu);
  auto key = std::make_pair(dev, caller);
  auto f = g_tier_sets.find(key);
  if (f != g_tier_sets.end()) return f->second;
  TierStreams* t = nullptr;
  auto& fr = g_tier_free[dev];
  if (!fr.empty()) {
    t = fr.back();
    fr.pop_back();
  } else {
    t = new TierStreams();
    bool ok = cudaEventCreateWithFlags(&t->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < kEigTiers && ok; ++i)
      ok = cudaStreamCreateWithFlags(&t->s[i], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&t->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      delete t;  // (a partly made set is left to the process's end)
      t = nullptr;
    }
  }
  g_tier_sets[key] = t;
  return t;
}

void prepare_eig_streams(void* stream) { tier_streams((cudaStream_t)stream); }

void release_eig_streams(void* stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(g_tier_mu);
  auto f = g_tier_sets.find(std::make_pair(dev, (cudaStream_t)stream));
  if (f == g_tier_sets.end()) return;
  if (f->second) g_tier_free[dev].push_back(f->second);
  g_tier_sets.erase(f);
}

void launch_eig_mixed(const EigTask* d_eigs, int64_t first, int64_t count, const Arenas* ar, double eps,
                      int trunc, int max_npad, int variant, void* stream) {
  init_kernel_attributes();
  const double thr = trunc == H2_TRUNC_SV ? eps * eps : eps;
  if (trunc != H2_TRUNC_FULL && thr < 5e-5) {
    // thresholds below float32 eigenvector resolution: float64 Rayleigh-Ritz refinement
    const int nn = max_npad + (max_npad & 1);
    const size_t smem = (size_t)3 * nn * (nn + 1) * sizeof(double);
    eig_mixed_kernel<<<(unsigned)count, 256, smem, (cudaStream_t)stream>>>(d_eigs, first, ar, eps, trunc);
    g_launches += 1;
  } else {
    // the level's padded size comes from the rank caps; the actual sizes (children's
    // ranks) are only known on the device and are mostly far smaller, so tasks are
    // launched in size tiers, each with the shared memory of its largest size (more
    // CTAs per SM for the small ones).  Threads per tier by variant (results are
    // identical): 0: 128 up to 48, 256 above; 1: 128 up to 64; 2: 64 up to 32, 128 up
    // to 64; 3: 64 up to 32, 128 up to 48
    auto threads = [&](int h) {
      if (variant >= 2 && h <= 32) return 64;
      if (h <= 48 || (h <= 64 && (variant == 1 || variant == 2))) return 128;
      return 256;
    };
    const int top = round4(max_npad);
    // a level with fewer tasks than a few CTAs per SM is one launch: its tiers would run
    // one after the other, each as long as its slowest task
    if (count < 4 * 152) {
      eig_mixed_kept_kernel<<<(unsigned)count, threads(top), eig_kept_smem(top), (cudaStream_t)stream>>>(
          d_eigs, first, ar, eps, trunc, -1, top);
      g_launches += 1;
      return;
    }
    // the tiers are independent (each task belongs to one), so they run concurrently on
    // auxiliary streams forked from the calling stream and joined back to it
    const TierStreams* ts = tier_streams((cudaStream_t)stream);
    if (ts) cudaEventRecord(ts->fork, (cudaStream_t)stream);
    int lo = -1, ti = 0;
    for (int hi : {32, 48, 56, 64, 80, kMixMax}) {
      const int h = hi < top ? hi : top;
      if (h > lo) {
        cudaStream_t st = (cudaStream_t)stream;
        if (ts) {
          st = ts->s[ti];
          cudaStreamWaitEvent(st, ts->fork, 0);
        }
        eig_mixed_kept_kernel<<<(unsigned)count, threads(h), eig_kept_smem(h), st>>>(d_eigs, first, ar, eps, trunc,
                                                                                    lo, h);
        g_launches += 1;
        if (ts) {
          cudaEventRecord(ts->join[ti], st);
          cudaStreamWaitEvent((cudaStream_t)stream, ts->join[ti], 0);
        }
        ++ti;
      }
      lo = h;
      if (h == top) break;
    }
  }
}

void launch_eig(const EigTask* d_eigs, int64_t first, int64_t count, const Arenas* ar, double eps, int trunc,
                int norm, int max_npad, double* scratch, void* stream) {
  int nn = max_npad + (max_npad & 1);
  size_t smem = 0;
  int64_t stride = 0;
  if (nn <= kEigSmemMax) {
    smem = (size_t)2 * nn * (nn + 1) * sizeof(double);
  } else {
    smem = (size_t)2 * kEigSmemMax * (kEigSmemMax + 1) * sizeof(double);
    stride = (int64_t)2 * nn * (nn + 1);
  }
  init_kernel_attributes();
  eig_kernel<<<(unsigned)count, 256, smem, (cudaStream_t)stream>>>(d_eigs, first, ar, eps, trunc, norm, scratch,
                                                                  stride);
  g_launches += 1;
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
  g_launches += 1;
}

void launch_permute(const double* src, double* dst, const int64_t* user, int64_t rows, int64_t n, int64_t nrhs,
                    bool to_tree, void* stream) {
  int64_t tot = rows * nrhs;
  unsigned blocks = (unsigned)((tot + 255) / 256);
  if (to_tree)
    to_tree_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(src, dst, user, rows, n, nrhs);
  else
    from_tree_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(src, dst, user, rows, n, nrhs);
  g_launches += 1;
}

}  // namespace h2
