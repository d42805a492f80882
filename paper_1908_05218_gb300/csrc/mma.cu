// Segmented batched GEMM on the fifth-generation tensor cores (tcgen05) for the float32
// products of the mixed-precision product (H2_MIXED_TF32X3).
//
// The work is the same program as the CUDA-core kernel (kernels.cu, seg_gemm32_kernel):
// one output matrix per segment, the sum of its items' products op(A) op(B) in a fixed
// order.  A persistent CTA of 128 threads walks segments at a stride of the grid; for
// each output tile of at most 128 x 128:
//   * the items are packed along k in 16-byte chunks (four k each; an item's k is
//     rounded up to a multiple of four with zeros); a stage holds kc chunks (k = 16 or 32,
//     a launch parameter);
//   * the stages' operands are copied with cp.async into a ring of three raw float32
//     stages, two stages ahead of the one being used, in the layout they have in global
//     memory (16-byte copies where the operand allows, zero-filled past the item's k);
//   * once a stage has landed, the threads split each value x into two TF32 values
//     hi = tf32(x), lo = tf32(x - hi), written in the K-major core-matrix layout of
//     tcgen05 without swizzle (a core matrix is 8 rows x 16 bytes; chunk (r, c) of a tile
//     sits at (r / 8) * kc * 128 + c * 128 + (r % 8) * 16) into one of two operand slots;
//   * one thread issues, for each k-step of eight, the three products hi*hi, hi*lo and
//     lo*hi (tcgen05.mma kind::tf32, M = 64 for tiles of at most 64 rows, else 128;
//     N = the tile's columns rounded up to 8 or 16; float32 accumulation in tensor
//     memory) and commits them to the slot's mbarrier, which is waited on only when the
//     slot is filled again two stages later;
//   * the accumulator is read back with tcgen05.ld (warp w reads its lanes 32 w ..
//     32 w + 31, which hold rows 32 w .. (M = 128) or 16 w .. 16 w + 15 (M = 64)) and
//     stored (or added) to the output.
// Rows of A beyond the tile's rows and columns of B beyond its columns are never written
// for the tile: the MMA reads whatever lies there (inside this CTA's shared memory) into
// rows / columns of the accumulator that are never stored.  The k padding of live rows
// is written as zeros, so it adds nothing.  The products and their order are those of
// the register-staged form of this kernel, so results do not depend on the pipeline.
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

// Shared memory of one CTA (bytes, runtime sizes of the launch's largest tile):
//   * two operand slots, each A_hi, A_lo, B_hi, B_lo in the K-major core-matrix layout:
//     A_hi / A_lo: (rows / 8) row groups of kc 16-byte chunks (kc * 128 bytes per group),
//     B_hi / B_lo the same for the tile's columns (rounded up to 16);
//   * a ring of kRawStages raw stages, float32 as copied from global memory: A either as
//     rows of the tile (k contiguous, row stride 4 kc + 4 floats) or, when A is stored
//     k x m, as kc * 4 rows of k (m contiguous, row stride rows + 4 floats); B likewise.
struct StageLayout {
  int kc;          // 16-byte chunks of k per stage (4 or 8: k = 16 or 32)
  int mr, nr;      // tile rows / columns held (multiples of 8; nr of 16)
  int rs_a, rt_a;  // raw A row strides (floats): tile rows of k / rows of k holding m
  int rs_b, rt_b;
  int raw_a, raw_stage;  // bytes: raw A of a stage, one raw stage (A then B)
  int hl_a, hl_b;        // bytes of A_hi (= A_lo) and of B_hi (= B_lo)
  int slot_bytes;        // one operand slot
  int raw_off;           // offset of the raw ring
  int total, tmem_cols;
};

constexpr int kRawStages = 3;   // raw stages: the one being split and two in flight
constexpr int kMaxSmem = 200 * 1024;
constexpr int kMaxChunks = 8;

inline StageLayout stage_layout(int maxm, int maxn, int kc) {
  StageLayout s;
  s.kc = kc;
  s.mr = std::min(kTileM, (std::max(8, maxm) + 7) & ~7);
  s.nr = std::min(kTileN, (std::max(16, maxn) + 15) & ~15);
  s.rs_a = 4 * kc + 4;
  s.rt_a = s.mr + 4;
  s.rs_b = 4 * kc + 4;
  s.rt_b = s.nr + 4;
  s.raw_a = 4 * std::max(s.mr * s.rs_a, 4 * kc * s.rt_a);
  const int raw_b = 4 * std::max(s.nr * s.rs_b, 4 * kc * s.rt_b);
  s.raw_stage = s.raw_a + raw_b;
  s.hl_a = (s.mr / 8) * kc * 128;
  s.hl_b = (s.nr / 8) * kc * 128;
  s.slot_bytes = 2 * s.hl_a + 2 * s.hl_b;
  s.raw_off = 2 * s.slot_bytes;
  // an A descriptor spans the M = 64 or 128 rows of the MMA from the start of A_hi / A_lo,
  // a B descriptor the N columns (rounded up to 16): keep both spans inside the buffer
  const int m_mma = s.mr > 64 ? 128 : 64;
  const int span_a = s.slot_bytes + s.hl_a + (m_mma / 8) * kc * 128;
  const int span_b = s.slot_bytes + 2 * s.hl_a + s.hl_b + (s.nr / 8) * kc * 128;
  s.total = std::max(std::max(s.raw_off + kRawStages * s.raw_stage, span_a), span_b);
  s.total = (s.total + 1023) & ~1023;
  s.tmem_cols = s.nr <= 32 ? 32 : (s.nr <= 64 ? 64 : 128);
  return s;
}

// one 16-byte chunk of k of a stage: the item's operands at the chunk's first k, their
// leading dims, the k of the item left from the chunk's start (<= 0: a zero chunk) and
// whether 16-byte copies apply (1: A, 2: B; the operand's start and leading dim are
// 16-byte multiples)
struct Slot {
  const float* a;
  const float* b;
  int lda, ldb;
  int kv;
  int flags;
};

__device__ __forceinline__ void cp_async16z(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// copy one operand of a stage into its raw buffer.  Row layout (kmajor: the operand
// stores k contiguously for each of the tile's rows / columns): chunk c of row r to
// raw[r * rs + 4 c].  Column layout (k selects the stored row): k-row kk of the stage
// (chunk kk / 4, k kk % 4 of it), 16 bytes of the tile's rows r4 .. r4 + 3, to
// raw[kk * rt + r4].  Entries past the item's k, or past the tile's rows in a column
// chunk, are written as zeros.
template <bool kVecBit2>
__device__ __forceinline__ void stage_copy(float* raw, const Slot* sl, int kc, int rows, bool kmajor, int rs, int rt,
                                           int tid) {
  constexpr int vbit = kVecBit2 ? 2 : 1;
  if (kmajor) {
    const int c = tid & (kc - 1);
    const Slot q = sl[c];
    const float* base = kVecBit2 ? q.b : q.a;
    const int ld = kVecBit2 ? q.ldb : q.lda;
    const int kv = q.kv;
    const bool vec = q.flags & vbit;
    for (int r = tid / kc; r < rows; r += kThreads / kc) {
      float* d = raw + r * rs + 4 * c;
      if (kv <= 0) {
        *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      const float* src = base + (int64_t)r * ld;
      if (vec) {
        cp_async16z(d, src, (kv < 4 ? kv : 4) * 4);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < kv) cp_async4(d + u, src + u);
          else d[u] = 0.f;
        }
      }
    }
  } else {
    const int kk = tid & (4 * kc - 1), c = kk >> 2, u = kk & 3;
    const Slot q = sl[c];
    const float* base = kVecBit2 ? q.b : q.a;
    const int ld = kVecBit2 ? q.ldb : q.lda;
    const bool live = u < q.kv;
    const bool vec = q.flags & vbit;
    const float* src0 = base + (int64_t)u * ld;
    const int step = 4 * (kThreads / (4 * kc));
    for (int r4 = 4 * (tid / (4 * kc)); r4 < rows; r4 += step) {
      float* d = raw + kk * rt + r4;
      if (!live) {
        *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      const int cnt = rows - r4 < 4 ? rows - r4 : 4;
      if (vec) {
        cp_async16z(d, src0 + r4, cnt * 4);
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if (v < cnt) cp_async4(d + v, src0 + r4 + v);
          else d[v] = 0.f;
        }
      }
    }
  }
}

// split one operand of a stage from its raw buffer into hi / lo in the core-matrix
// layout: chunk (r, c) to (r / 8) * kc * 128 + c * 128 + (r % 8) * 16.  Threads take
// consecutive rows (rpow: the rows rounded up to a power of two), so that each quarter
// warp writes 128 contiguous bytes and reads conflict-free.  Rows past the tile's are
// not written.
__device__ __forceinline__ void stage_split(const float* raw, unsigned char* hi, unsigned char* lo, int kc, int rows,
                                            int rpow, bool kmajor, int rs, int rt, int tid) {
  const int r = tid & (rpow - 1);
  if (r >= rows) return;
  const int cstep = kThreads / rpow > 0 ? kThreads / rpow : 1;
  const int rgo = (r >> 3) * kc * 128 + (r & 7) * 16;
  for (int c = tid / rpow; c < kc; c += cstep) {
    float v[4];
    if (kmajor) {
      const float4 x = *reinterpret_cast<const float4*>(raw + r * rs + 4 * c);
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = raw[(4 * c + u) * rt + r];
    }
    uint4 h, l;
    split4(v, h, l);
    *reinterpret_cast<uint4*>(hi + rgo + c * 128) = h;
    *reinterpret_cast<uint4*>(lo + rgo + c * 128) = l;
  }
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 8;
  while (p < x) p <<= 1;
  return p;
}

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
  __shared__ Slot tab[kRawStages][kMaxChunks];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc = lay.kc, rg_bytes = kc * 128;

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
  int hs = 0;  // operand slot of the next stage
  bool fail = false;

  // threads 0 .. kc-1 fill the slot table t for the stage starting at chunk c0 of the
  // current item batch (nb items, chunk prefix it_c0, nch chunks)
  auto fill_slots = [&](int t, int c0, int nb, int nch) {
    if (tid < kc) {
      const int g = c0 + tid;
      Slot sl{nullptr, nullptr, 0, 0, 0, 0};
      if (g < nch) {
        int lo = 0, hi = nb - 1;  // the last item whose first chunk is <= g
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (it_c0[mid] <= g) lo = mid;
          else hi = mid - 1;
        }
        const int q = lo;
        const int k0 = (g - it_c0[q]) * 4;
        sl.lda = it_lda[q];
        sl.ldb = it_ldb[q];
        sl.kv = it_k[q] - k0;
        sl.flags = it_fl[q];
        sl.a = it_a[q];
        sl.b = it_b[q];
        // A stored m x k / B stored n x k: k runs along the row; else k selects the row
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
        for (int q = 0; q < s.count; ++q)  // (SF_TA: the input is read transposed)
          acc += ptr_of<float>(ar, it[q].a)[ta ? (int64_t)c * s.lda + r : (int64_t)r * s.lda + c];
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
        const int mpow = pow2_at_least(mc), npow = pow2_at_least(nc);
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
            const float* ta0 = ta ? pa + m0 : pa + (int64_t)m0 * la;
            const float* tb0 = tb ? pb + (int64_t)n0 * lb : pb + n0;
            it_a[tid] = ta0;
            it_b[tid] = tb0;
            it_lda[tid] = la;
            it_ldb[tid] = lb;
            it_k[tid] = bound(ar, iq.kref, kp);
            it_fl[tid] = ((((uintptr_t)ta0) & 15) == 0 && (la & 3) == 0 ? 1 : 0) |
                         ((((uintptr_t)tb0) & 15) == 0 && (lb & 3) == 0 ? 2 : 0) | (ta ? 8 : 0) | (tb ? 16 : 0);
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
          const int nst = (nch + kc - 1) / kc;  // stages of this batch
          // prologue: slot tables of stages 0 .. 2, copies of stages 0 and 1
          for (int p = 0; p < kRawStages; ++p) fill_slots(p, p * kc, nb, nch);
          __syncthreads();
          for (int p = 0; p < 2; ++p) {
            if (p < nst) {
              float* rA = (float*)(smem + lay.raw_off + p * lay.raw_stage);
              float* rB = (float*)(smem + lay.raw_off + p * lay.raw_stage + lay.raw_a);
              stage_copy<false>(rA, tab[p], kc, mc, !ta, lay.rs_a, lay.rt_a, tid);
              stage_copy<true>(rB, tab[p], kc, nc, tb, lay.rs_b, lay.rt_b, tid);
            }
            cp_commit();
          }
          for (int j = 0; j < nst && !fail; ++j) {
            cp_wait1();  // this thread's copies of stage j have landed
            // the operand slot hs was last read by the products committed to bar[hs]
            int ok = 1;
            if (pend[hs] && tid == 0) ok = mbar_wait(&bar[hs], phase[hs]) ? 1 : 0;
            if (__syncthreads_or(!ok)) {
              fail = true;
              break;
            }
            if (pend[hs]) {
              phase[hs] ^= 1u;
              pend[hs] = false;
            }
            // copies of stage j + 2 into the raw stage last split at j - 1
            if (j + 2 < nst) {
              const int rsl = (j + 2) % kRawStages;
              float* rA = (float*)(smem + lay.raw_off + rsl * lay.raw_stage);
              float* rB = (float*)(smem + lay.raw_off + rsl * lay.raw_stage + lay.raw_a);
              stage_copy<false>(rA, tab[rsl], kc, mc, !ta, lay.rs_a, lay.rt_a, tid);
              stage_copy<true>(rB, tab[rsl], kc, nc, tb, lay.rs_b, lay.rt_b, tid);
            }
            cp_commit();
            // the slot table of stage j + 3 (its table slot held stage j's, read at j - 2)
            if (j + 3 < nst) fill_slots((j + 3) % kRawStages, (j + 3) * kc, nb, nch);
            // split stage j into the operand slot
            {
              const int rsl = j % kRawStages;
              const float* rA = (const float*)(smem + lay.raw_off + rsl * lay.raw_stage);
              const float* rB = (const float*)(smem + lay.raw_off + rsl * lay.raw_stage + lay.raw_a);
              unsigned char* a_hi = smem + hs * lay.slot_bytes;
              unsigned char* a_lo = a_hi + lay.hl_a;
              unsigned char* b_hi = a_hi + 2 * lay.hl_a;
              unsigned char* b_lo = b_hi + lay.hl_b;
              stage_split(rA, a_hi, a_lo, kc, mc, mpow, !ta, lay.rs_a, lay.rt_a, tid);
              stage_split(rB, b_hi, b_lo, kc, nc, npow, tb, lay.rs_b, lay.rt_b, tid);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t ah = smem_u32(smem + hs * lay.slot_bytes);
              const uint32_t al = ah + lay.hl_a, bh = ah + 2 * lay.hl_a, bl = bh + lay.hl_b;
              // k-steps of eight: the stage's live chunks rounded up to an even count (the
              // chunks past the batch's end hold zeros)
              const int live = min(kc, nch - j * kc);
              const int steps = (live + 1) >> 1;
              for (int ks = 0; ks < steps; ++ks) {
                const uint32_t o = ks * 256;
                mma_tf32(tmem, smem_desc(ah + o, 128, rg_bytes), smem_desc(bh + o, 128, rg_bytes), idesc,
                         issued ? 1u : 0u);
                issued = true;
                mma_tf32(tmem, smem_desc(ah + o, 128, rg_bytes), smem_desc(bl + o, 128, rg_bytes), idesc, 1u);
                mma_tf32(tmem, smem_desc(al + o, 128, rg_bytes), smem_desc(bh + o, 128, rg_bytes), idesc, 1u);
              }
              mma_commit(&bar[hs]);
            }
            issued = true;  // (uniform: every thread tracks the same state)
            pend[hs] = true;
            hs ^= 1;
          }
          cp_wait0();
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
  cp_wait0();
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
                     int maxm, int maxn, unsigned int* err, int variant, void* stream) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(seg_mma_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  });
  // variants: 0: k = 16 per stage, as many CTAs per SM as fit; 1: k = 32 per stage (k = 16
  // where that does not fit); 2: k = 16, at most half as many CTAs
  StageLayout lay = stage_layout(maxm, maxn, variant == 1 ? 8 : 4);
  if (lay.total > kMaxSmem) lay = stage_layout(maxm, maxn, 4);
  // resident CTAs per SM: the tensor-memory limit (512 / columns) and the shared-memory
  // limit (each CTA also has ~3 KB of static shared memory)
  const int tm_cap = 512 / lay.tmem_cols;
  const int sm_cap = (int)((227 * 1024) / (lay.total + 4096));
  int per_sm = std::max(1, std::min(tm_cap, sm_cap));
  if (variant == 2) per_sm = std::max(1, per_sm / 2);
  const int64_t grid = std::min<int64_t>(count, 152LL * per_sm);
  if (grid <= 0) return;
  seg_mma_tf32x3_kernel<<<(unsigned)grid, kThreads, lay.total, (cudaStream_t)stream>>>(d_segs, d_items, first, count,
                                                                                       d_ars, lay, err);
  add_kernel_launches(1);
}

}  // namespace h2
