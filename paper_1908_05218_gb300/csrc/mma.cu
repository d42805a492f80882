// Segmented batched GEMM on the fifth-generation tensor cores (tcgen05) for the float32
// products of the mixed-precision product (H2_MIXED_TF32X3).
//
// The work is the same program as the CUDA-core kernel (kernels.cu, seg_gemm32_kernel):
// one output matrix per segment, the sum of its items' products op(A) op(B) in a fixed
// order.  A persistent CTA of 128 threads walks segments at a stride of the grid; for
// each 128 x 128 output tile:
//   * the items are packed along k in 16-byte chunks (four k each; an item's k is
//     rounded up to a multiple of four with zeros); a stage holds eight chunks (k = 32),
//     two stages alternate;
//   * all threads stage A (rows of the tile x 8 chunks) and B (columns x 8 chunks) into
//     shared memory in the K-major core-matrix layout of tcgen05 without swizzle
//     (a core matrix is 8 rows x 16 bytes; chunk (r, c) of a tile sits at
//     (r / 8) * 1024 + c * 128 + (r % 8) * 16), each float32 value x split into two
//     TF32 values hi = tf32(x), lo = tf32(x - hi);
//   * one thread issues, for each k-step of eight, the three products hi*hi, hi*lo and
//     lo*hi (tcgen05.mma kind::tf32, M = 64 for tiles of at most 64 rows, else 128;
//     N = the tile's columns rounded up to 8 or 16; float32 accumulation in tensor
//     memory) and commits them to the stage's mbarrier; the threads stage the next
//     chunks meanwhile;
//   * the accumulator is read back with tcgen05.ld (warp w reads its lanes 32 w ..
//     32 w + 31, which hold rows 32 w .. (M = 128) or 16 w .. 16 w + 15 (M = 64)) and
//     stored (or added) to the output.
// Rows of A beyond the tile's rows and columns of B beyond its columns are never written
// for the tile: the MMA reads whatever lies there (inside this CTA's shared memory) into
// rows / columns of the accumulator that are never stored.  The k padding of live rows
// is written as zeros, so it adds nothing.
//
// Split precision: |x - hi - lo| <= 2^-22 |x|; the dropped lo*lo term and the float32
// accumulation keep each product within a few float32 roundings of the exact one.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records an error in the
// product's counter block (read by h2_info / h2_export as H2_ETIMEOUT), drains its own
// products with a second bounded wait, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

#include "device.cuh"
#include "internal.hpp"

namespace h2 {

namespace {

constexpr int kThreads = 128;
constexpr int kChunks = 8;            // 16-byte chunks of k per stage (k = 32 for TF32)
constexpr int kBatch = 64;            // items whose metadata sit in shared memory at once
constexpr int kTileM = 128, kTileN = 128;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz: an mbarrier wait gives up after this

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance of the two
// k-adjacent core matrices of one MMA k-step, sbo = byte distance of 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: float32 accumulator, TF32 A and B, both K-major
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t b;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(x));
  return b;
}

__device__ __forceinline__ void split4(const float v[4], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = tf32_rna(v[q]);
    l[q] = tf32_rna(v[q] - __uint_as_float(h[q]));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// bounded wait for the given phase parity of an mbarrier; false if it gave up.  Each
// try_wait may suspend the thread until the phase completes (at most ~0.1 ms per try).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(100000)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// one thread waits for the phase, the others at the barrier (no issue slots spent on
// polling); the barrier hands its outcome to every thread, so all give up together
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity) {
  int ok = 1;
  if (threadIdx.x == 0) ok = mbar_wait(bar, parity) ? 1 : 0;
  return !__syncthreads_or(!ok);
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// shared-memory layout: two stages of A_hi, A_lo (a_bytes each: the launch's largest tile
// rows, rounded up to 8, x kChunks x 16 bytes per row) and B_hi, B_lo (b_bytes each)
struct StageLayout {
  int a_bytes, b_bytes, stage_bytes, total, tmem_cols;
};

constexpr int kRowGroupBytes = kChunks * 128;  // 8 rows x kChunks 16-byte chunks

inline StageLayout stage_layout(int maxm, int maxn) {
  StageLayout s;
  const int mr = std::min(kTileM, std::max(8, maxm)), nr = std::min(kTileN, std::max(16, maxn));
  s.a_bytes = ((mr + 7) / 8) * kRowGroupBytes;
  s.b_bytes = ((nr + 15) / 16) * 2 * kRowGroupBytes;
  s.stage_bytes = 2 * s.a_bytes + 2 * s.b_bytes;
  // tensor memory: 64 columns when every tile has at most 64 columns, else 128; at most
  // 512 / cols CTAs of this kernel fit an SM's 512 columns, so the shared memory is padded
  // until one more CTA would not fit (a CTA without columns would stall in tcgen05.alloc
  // until another retires)
  s.tmem_cols = nr <= 64 ? 64 : 128;
  const int per_sm = 512 / s.tmem_cols;
  const int floor_bytes = (228 * 1024) / (per_sm + 1) - 3 * 1024;
  // an A descriptor spans the M = 128 (or 64) rows of its tile from its start: keep that
  // inside the buffer
  const int span = (mr > 64 ? 16 : 8) * kRowGroupBytes;
  s.total = std::max(std::max(2 * s.stage_bytes, s.stage_bytes + s.a_bytes + span), floor_bytes);
  return s;
}

// one 16-byte chunk of k of a stage: the item's operands at the chunk's first k, their
// leading dims, and whether 16-byte loads (K-major and aligned) and unmasked loads (the
// item's padded k a multiple of four: entries past its rank are zero) apply
struct Slot {
  const float* a;
  const float* b;
  int lda, ldb;
  int kv;     // k of the item left from the chunk's start (<= 0: a zero chunk)
  int flags;  // 1: A 16-byte loads, 2: B 16-byte loads, 4: unmasked
};

__global__ void __launch_bounds__(kThreads) seg_mma_tf32x3_kernel(const Seg* __restrict__ segs,
                                                                  const Item* __restrict__ items, int64_t first,
                                                                  int64_t count, const Arenas* __restrict__ ars,
                                                                  StageLayout lay, unsigned int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ const float* it_a[kBatch];
  __shared__ const float* it_b[kBatch];
  __shared__ int it_lda[kBatch], it_ldb[kBatch], it_k[kBatch], it_c0[kBatch + 1], it_fl[kBatch];
  __shared__ Slot tab[2][kChunks];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(lay.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  uint32_t phase[2] = {0u, 0u};
  bool pend[2] = {false, false};
  int buf = 0;
  bool fail = false;

  // threads 0 .. kChunks-1 fill the slot table of the stage starting at chunk c0 of the
  // current item batch (items nb, chunk prefix it_c0)
  auto fill_slots = [&](int t, int c0, int nb, int nch) {
    if (tid < kChunks) {
      const int g = c0 + tid;
      Slot sl{nullptr, nullptr, 0, 0, 0, 0};
      if (g < nch) {
        int q = 0;
        while (q + 1 < nb && it_c0[q + 1] <= g) ++q;
        const int k0 = (g - it_c0[q]) * 4;
        sl.lda = it_lda[q];
        sl.ldb = it_ldb[q];
        sl.kv = it_k[q] - k0;
        sl.flags = it_fl[q];
        sl.a = it_a[q];
        sl.b = it_b[q];
        // A row-major / B transposed: k runs along the row; else k selects the row
        sl.a += (sl.flags & 8) ? (int64_t)k0 * sl.lda : k0;
        sl.b += (sl.flags & 16) ? k0 : (int64_t)k0 * sl.ldb;
      }
      tab[t][tid] = sl;
    }
  };

  for (int64_t si = blockIdx.x; si < count && !fail; si += gridDim.x) {
    const Seg s = segs[first + si];
    const Arenas* ar = ars + s.inst;
    const int M = bound(ar, s.mref, s.m), N = bound(ar, s.nref, s.n);
    const View out = view(ar, s.out);
    const bool ta = s.flags & SF_TA, tb = s.flags & SF_TB, accum = s.flags & SF_ACC;
    if (s.flags & SF_SUM) {  // plain sums of matrices (collects): CUDA cores
      const Item* it = items + s.first;
      for (int e = tid; e < M * N; e += kThreads) {
        const int r = e / N, c = e - r * N;
        float acc = 0.f;
        for (int q = 0; q < s.count; ++q) acc += ptr_of<float>(ar, it[q].a)[(int64_t)r * s.lda + c];
        st<float>(out, (int64_t)r * s.ldc + c, acc, accum);
      }
      continue;
    }
    unsigned long long work = 0;
    for (int m0 = 0; m0 < M && !fail; m0 += kTileM) {
      const int mc = min(kTileM, M - m0);
      for (int n0 = 0; n0 < N && !fail; n0 += kTileN) {
        // MMA shape: M = 64 for tiles of at most 64 rows (row r of the accumulator in
        // tensor-memory lane 32 (r / 16) + r % 16), else M = 128 (row r in lane r); N = the
        // tile's columns rounded up to 8 (M = 64) or 16 (M = 128)
        const int nc = min(kTileN, N - n0);
        const bool m64 = mc <= 64;
        const int nmma = m64 ? max(8, (nc + 7) & ~7) : max(16, (nc + 15) & ~15);
        const uint32_t idesc = idesc_tf32(m64 ? 64 : 128, nmma);
        const int mrows = (mc + 7) & ~7, nrows = (nc + 7) & ~7;
        bool issued = false;  // an MMA of this tile has been issued
        for (int b0 = 0; b0 < s.count && !fail; b0 += kBatch) {
          const int nb = min(kBatch, s.count - b0);
          __syncthreads();  // the previous batch's metadata and slots are no longer read
          if (tid < nb) {
            const Item iq = items[s.first + b0 + tid];
            const float* pa = ptr_of<float>(ar, iq.a);
            const float* pb = ptr_of<float>(ar, iq.b);
            const int la = iq.lda ? iq.lda : s.lda, lb = iq.ldb ? iq.ldb : s.ldb;
            const int kp = iq.kpad ? iq.kpad : s.k;
            // operand views of the tile: A at row m0, B at column n0
            it_a[tid] = ta ? pa + m0 : pa + (int64_t)m0 * la;
            it_b[tid] = tb ? pb + (int64_t)n0 * lb : pb + n0;
            it_lda[tid] = la;
            it_ldb[tid] = lb;
            it_k[tid] = bound(ar, iq.kref, kp);
            const bool pad4 = (kp & 3) == 0;
            it_fl[tid] = (!ta && pad4 && (((uintptr_t)pa) & 15) == 0 && (la & 3) == 0 ? 1 : 0) |
                         (tb && pad4 && (((uintptr_t)pb) & 15) == 0 && (lb & 3) == 0 ? 2 : 0) | (pad4 ? 4 : 0) |
                         (ta ? 8 : 0) | (tb ? 16 : 0);
          }
          __syncthreads();
          if (tid == 0) {
            int c = 0;
            for (int q = 0; q < nb; ++q) {
              it_c0[q] = c;
              c += (it_k[q] + 3) >> 2;
              work += 2ull * mc * nc * (unsigned long long)it_k[q];
            }
            it_c0[nb] = c;
          }
          __syncthreads();
          const int nch = it_c0[nb];
          fill_slots(buf, 0, nb, nch);
          // (the slots of a stage are read after the barrier that ends the wait below or
          // the one that precedes the first stage's staging)
          __syncthreads();
          for (int c0 = 0; c0 < nch && !fail; c0 += kChunks) {
            if (pend[buf]) {
              if (!cta_wait(&bar[buf], phase[buf])) {
                fail = true;
                break;
              }
              phase[buf] ^= 1u;
              pend[buf] = false;
            }
            unsigned char* base = smem + buf * lay.stage_bytes;
            unsigned char* a_hi = base;
            unsigned char* a_lo = base + lay.a_bytes;
            unsigned char* b_hi = base + 2 * lay.a_bytes;
            unsigned char* b_lo = b_hi + lay.b_bytes;
            const Slot* sl = tab[buf];
            // chunks of this stage, rounded up to whole MMA k-steps of two chunks
            const int live = min(kChunks, (nch - c0 + 1) & ~1);
            // chunk tasks: e -> (row group, slot, row in group), row in group fastest, so
            // that each quarter warp stores 128 contiguous bytes
            for (int e = tid; e < mrows * kChunks; e += kThreads) {
              const int rr = e & 7, slot = (e >> 3) & (kChunks - 1), rg = e / (8 * kChunks);
              const int row = rg * 8 + rr;
              if (row >= mc || slot >= live) continue;
              const Slot& q = sl[slot];
              float v[4] = {0.f, 0.f, 0.f, 0.f};
              if (q.kv > 0) {
                if (q.flags & 1) {
                  const float4 x = *reinterpret_cast<const float4*>(q.a + (int64_t)row * q.lda);
                  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
                } else if (!(q.flags & 8)) {
                  const float* p = q.a + (int64_t)row * q.lda;
                  for (int u = 0; u < 4; ++u) v[u] = ((q.flags & 4) || u < q.kv) ? p[u] : 0.f;
                } else {
                  const float* p = q.a + row;
                  for (int u = 0; u < 4; ++u) v[u] = ((q.flags & 4) || u < q.kv) ? p[(int64_t)u * q.lda] : 0.f;
                }
              }
              uint4 hi, lo;
              split4(v, hi, lo);
              const int off = rg * kRowGroupBytes + slot * 128 + rr * 16;
              *reinterpret_cast<uint4*>(a_hi + off) = hi;
              *reinterpret_cast<uint4*>(a_lo + off) = lo;
            }
            for (int e = tid; e < nrows * kChunks; e += kThreads) {
              const int rr = e & 7, slot = (e >> 3) & (kChunks - 1), rg = e / (8 * kChunks);
              const int col = rg * 8 + rr;
              if (col >= nc || slot >= live) continue;
              const Slot& q = sl[slot];
              float v[4] = {0.f, 0.f, 0.f, 0.f};
              if (q.kv > 0) {
                if (q.flags & 2) {
                  const float4 x = *reinterpret_cast<const float4*>(q.b + (int64_t)col * q.ldb);
                  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
                } else if (q.flags & 16) {
                  const float* p = q.b + (int64_t)col * q.ldb;
                  for (int u = 0; u < 4; ++u) v[u] = ((q.flags & 4) || u < q.kv) ? p[u] : 0.f;
                } else {
                  const float* p = q.b + col;
                  for (int u = 0; u < 4; ++u) v[u] = ((q.flags & 4) || u < q.kv) ? p[(int64_t)u * q.ldb] : 0.f;
                }
              }
              uint4 hi, lo;
              split4(v, hi, lo);
              const int off = rg * kRowGroupBytes + slot * 128 + rr * 16;
              *reinterpret_cast<uint4*>(b_hi + off) = hi;
              *reinterpret_cast<uint4*>(b_lo + off) = lo;
            }
            // the next stage's slots (the other table: last read before the previous barrier)
            if (c0 + kChunks < nch) fill_slots(buf ^ 1, c0 + kChunks, nb, nch);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
              const int steps = live / 2;
              for (int ks = 0; ks < steps; ++ks) {
                const uint32_t o = ks * 256;
                mma_tf32(tmem, smem_desc(ah + o, 128, kRowGroupBytes), smem_desc(bh + o, 128, kRowGroupBytes), idesc,
                         issued ? 1u : 0u);
                issued = true;
                mma_tf32(tmem, smem_desc(ah + o, 128, kRowGroupBytes), smem_desc(bl + o, 128, kRowGroupBytes), idesc, 1u);
                mma_tf32(tmem, smem_desc(al + o, 128, kRowGroupBytes), smem_desc(bh + o, 128, kRowGroupBytes), idesc, 1u);
              }
              mma_commit(&bar[buf]);
            }
            issued = true;  // (uniform: every thread tracks the same state)
            pend[buf] = true;
            buf ^= 1;
          }
        }
        // epilogue: wait for the tile's products, read the accumulator, store
        for (int b = 0; b < 2 && !fail; ++b)
          if (pend[b]) {
            if (!cta_wait(&bar[b], phase[b])) {
              fail = true;
              break;
            }
            phase[b] ^= 1u;
            pend[b] = false;
          }
        if (fail) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // warp w reads tensor-memory lanes 32 w .. 32 w + 31 (its sub-partition)
        const int rows_w = m64 ? 16 : 32;
        if (warp * rows_w < mc) {
          const int row = warp * rows_w + lane;
          const bool mine = lane < rows_w && row < mc;
          for (int c = 0; c < nmma; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (mine) {
              const int jn = min(16, nc - c);
              const int64_t o = (int64_t)(m0 + row) * s.ldc + n0 + c;
              if (out.f32) {
                float* po = (float*)out.base + o;
                for (int j = 0; j < jn; ++j) po[j] = (accum ? po[j] : 0.f) + (issued ? v[j] : 0.f);
              } else {
                double* po = (double*)out.base + o;
                for (int j = 0; j < jn; ++j) po[j] = (accum ? po[j] : 0.0) + (double)(issued ? v[j] : 0.f);
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
      }
    }
    if (ar->flops && tid == 0 && work) atomicAdd(ar->flops, work);
  }
  if (fail) {
    if (tid == 0 && err) atomicOr(err, 1u);
    // drain: the products this CTA issued must finish before its tensor memory is freed
    if (tid == 0)
      for (int b = 0; b < 2; ++b)
        if (pend[b]) mbar_wait(&bar[b], phase[b]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(lay.tmem_cols));
}

}  // namespace

void launch_gemm_mma(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars,
                     int maxm, int maxn, unsigned int* err, int ctas_per_sm, void* stream) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(seg_mma_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const StageLayout lay = stage_layout(maxm, maxn);
  // resident CTAs per SM: the tensor-memory limit (512 / columns), the shared-memory limit
  // and the requested count (the autotuner's candidates scale the requested count)
  const int tm_cap = 512 / lay.tmem_cols;
  const int sm_cap = (int)((227 * 1024) / (lay.total + 4096));
  const int want = ctas_per_sm * (lay.tmem_cols == 64 ? 2 : 1);
  const int per_sm = std::max(1, std::min(want, std::min(tm_cap, sm_cap)));
  const int64_t grid = std::min<int64_t>(count, 152LL * per_sm);
  if (grid <= 0) return;
  seg_mma_tf32x3_kernel<<<(unsigned)grid, kThreads, lay.total, (cudaStream_t)stream>>>(d_segs, d_items, first, count,
                                                                                       d_ars, lay, err);
  add_kernel_launches(1);
}

}  // namespace h2
