// Coupling sums on the fifth-generation tensor cores (tcgen05) for H2_MIXED_BF16X3: the
// main coupling pass of every level (Eq. leafcoup_simple / nonleafcoup_simple: leaf case 1,
// cases 2/4 and case 3, summed per target), S_ik += sum over items of A_item B_item.
//
// The operands were written by their producers (the projections and R images of the
// level) as BF16 split tiles (device.cuh): an A operand (rows of the target, k) as an
// rp x kp tile, a B operand transposed (columns of the target, k) as an np x kp tile, each
// in the K-major core-matrix layout of tcgen05 without swizzle, high parts then low parts.
// So an item's operands reach shared memory by two bulk copies (cp.async.bulk, completing
// on an mbarrier), and the tensor cores read them there without any rearrangement.
//
// A persistent CTA of six warps walks the launch's segments (one per target) at a stride
// of the grid:
//   * warp 4 copies the items' tiles into a ring of shared-memory stages (its lanes read
//     the metadata of 32 items at a time, lane 0 issues), a stage being reused once the
//     products reading it have completed; each stage's slot tells the issuing thread the
//     item's k and whether it starts or ends its target's sum;
//   * warp 5 (one thread) issues, per k-step of 16, the three products hi*hi, hi*lo and
//     lo*hi (tcgen05.mma kind::f16 with BF16 A and B, M = 64, N = np, float32 accumulation
//     in tensor memory; the dropped lo*lo term is below 2^-16 of the product) into one of
//     nacc accumulators, commits each stage to its "empty" mbarrier and the target's last
//     product to the accumulator's "full" mbarrier;
//   * warps 0-3 read the finished accumulator (tcgen05.ld; the M = 64 layout puts row r in
//     lane 32 (r / 16) + r % 16, so warp w holds rows 16 w .. 16 w + 15) and add it to the
//     target's coupling in its arena (or store it, for the target's first contribution),
//     then release the accumulator; a target's metadata is read before its products are
//     waited for.
// Rows of the A stage beyond the tile (the MMA reads 64) lie inside the stage and only
// reach accumulator rows that are never stored; k beyond an item's rank is zero in both
// tiles, so it adds nothing.  The products of a target run in item order, so results are
// bitwise reproducible.
//
// The executed-flop counter of tracing (Arenas::flops) counts the CUDA-core kernels only.
//
// Every mbarrier wait is bounded (about 2 s); on expiry the CTA records an error in the
// product's error word (H2_ETIMEOUT through h2_info / h2_export), every role leaves its
// loop, the copies and products in flight are waited for (bounded again), and the tensor
// memory is freed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "device.cuh"
#include "internal.hpp"

namespace h2 {

namespace {

constexpr int kMaxStages = 8;  // shared-memory stages of the copy ring (TcLayout::nst of them)
constexpr int kMaxAcc = 4;     // accumulators in tensor memory (TcLayout::nacc of them)
constexpr int kEpiWarps = 4;
constexpr int kThreads = 32 * (kEpiWarps + 2);  // warps 0-3 epilogue, 4 copies, 5 products
constexpr int kProducer = kEpiWarps, kIssuer = kEpiWarps + 1;
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz
constexpr int kMaxSmem = 200 * 1024;

struct TcLayout {
  int rp, np;      // A tile rows (a multiple of 8, at most 64), B tile rows = the MMA's N
  int nst;         // stages of the copy ring
  int nacc;        // accumulators
  int trim;        // copy only the rows up to the target's ranks (four copies per item; else two)
  int kpmax;       // largest tile k of the launch (a multiple of 16)
  int stage_bytes;  // a stage: the item's A tile, then its B tile (offset rp * kp * 4)
  int ncols;       // tensor-memory columns of one accumulator (np rounded up to 16)
  int tmem_cols;   // allocated columns: nacc accumulators, a power of two >= 32
  int total;       // dynamic shared memory
};

// launch configurations (stages, accumulators), all with the same products in the same
// order: the autotuner picks one per launch group
constexpr int kTcConfigs[kTcVariants][3] = {{4, 2, 1}, {4, 2, 0}, {6, 2, 1}, {6, 2, 0}};

TcLayout tc_layout(int rp, int np, int kpmax, int variant) {
  TcLayout t;
  t.rp = rp;
  t.np = np;
  t.kpmax = kpmax;
  const int kc = kpmax / 8;  // 16-byte k-chunks
  // the stage holds both tiles; the M = 64 descriptor of A's low part spans 8 row groups
  // from its start, which may reach into the B tile (rows that only feed accumulator
  // rows never stored) but must stay inside the stage
  t.stage_bytes = std::max((rp + np) * kpmax * 4, (rp / 8 + 8) * kc * 128);
  t.stage_bytes = (t.stage_bytes + 1023) & ~1023;
  t.ncols = (np + 15) & ~15;
  t.nst = kTcConfigs[variant][0];
  t.nacc = kTcConfigs[variant][1];
  t.trim = kTcConfigs[variant][2];
  int c = 32;
  while (c < t.nacc * t.ncols) c <<= 1;
  t.tmem_cols = c;
  t.total = t.nst * t.stage_bytes;
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major without swizzle: lbo = byte distance of the two
// k-adjacent core matrices of a k-step, sbo = byte distance of 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: float32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bulk copy global -> shared, completing `bytes` on the mbarrier (16-byte aligned, a
// multiple of 16 bytes)
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// bounded wait for the phase of the given parity; gives up after kWaitCycles or when
// another role has given up (abort flag); false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(20000)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
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

// what the copying warp tells the issuing thread about the item in a stage
enum : int { kFirst = 1, kLast = 2, kEnd = 4 };

__global__ void __launch_bounds__(kThreads, 6) coup_tc_kernel(const Seg* __restrict__ segs, const Item* __restrict__ items,
                                                           int64_t first, int64_t count, const Arenas* __restrict__ ars,
                                                           TcLayout lay, unsigned int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], accf[kMaxAcc], acce[kMaxAcc], done;
  // per stage: the item's tile k and k-steps, kFirst | kLast | kEnd
  __shared__ int slot_k[kMaxStages], slot_s[kMaxStages], slot_f[kMaxStages];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int st = 0; st < lay.nst; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    for (int b = 0; b < lay.nacc; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], kEpiWarps);
    }
    mbar_init(&done, 1);
    s_abort = 0;
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
  const uint32_t nst = (uint32_t)lay.nst;

  if (warp == kProducer) {
    // the copying warp: its lanes read the metadata of 32 items at once; lane 0 waits for
    // a free stage, describes the item in the stage's slot and starts the two copies
    uint32_t it = 0;  // items copied by this CTA
    bool ok = true;
    int64_t si = blockIdx.x;
    Seg sn{};
    if (si < count) sn = segs[first + si];
    while (si < count && ok) {
      const Seg s = sn;
      const int64_t si2 = si + gridDim.x;
      if (si2 < count) sn = segs[first + si2];  // the next segment's, while this one is copied
      const Arenas* ar = ars + s.inst;
      // only the tiles' rows up to the target's ranks (rounded up to 8) are copied: the
      // rest are zeros that only reach accumulator rows / columns never stored
      const int m8 = lay.trim ? max(8, (bound(ar, s.mref, s.m) + 7) & ~7) : lay.rp;
      const int n8 = lay.trim ? max(8, (bound(ar, s.nref, s.n) + 7) & ~7) : lay.np;
      for (int b0 = 0; b0 < s.count && ok; b0 += 32) {
        const int nb = min(32, s.count - b0);
        unsigned long long pa = 0, pb = 0;
        int kp = 0, ks = 0;
        if (lane < nb) {
          const Item iq = items[s.first + b0 + lane];
          pa = (unsigned long long)ptr_of<float>(ar, iq.a);
          pb = (unsigned long long)ptr_of<float>(ar, iq.b);
          kp = iq.kpad;
          // k-steps of 16 up to the item's rank: the tiles hold zeros beyond it
          ks = max(1, (bound(ar, iq.kref, kp) + 15) >> 4);
        }
        for (int q = 0; q < nb; ++q, ++it) {
          const unsigned long long a = __shfl_sync(0xffffffffu, pa, q), b = __shfl_sync(0xffffffffu, pb, q);
          const int k = __shfl_sync(0xffffffffu, kp, q), ksteps = __shfl_sync(0xffffffffu, ks, q);
          int good = 1;
          if (lane == 0) {
            const int st = (int)(it % nst);
            const uint32_t use = it / nst;
            if (use > 0 && !mbar_wait(&empty[st], (use - 1) & 1u, &s_abort)) {
              good = 0;
            } else {
              // hi and lo parts of A (rp rows each in the tile) and of B (np rows): the
              // first m8 / n8 rows of each part
              const uint32_t ha = (uint32_t)lay.rp * k * 2, hb = (uint32_t)lay.np * k * 2;
              const uint32_t ca = (uint32_t)m8 * k * 2, cb = (uint32_t)n8 * k * 2;
              unsigned char* sa = smem + st * lay.stage_bytes;
              unsigned char* sb = sa + 2 * ha;
              const unsigned char* ga = (const unsigned char*)a;
              const unsigned char* gb = (const unsigned char*)b;
              slot_k[st] = k;
              slot_s[st] = ksteps;
              slot_f[st] = (b0 + q == 0 ? kFirst : 0) | (b0 + q == s.count - 1 ? kLast : 0);
              mbar_expect_tx(&full[st], 2 * (ca + cb));
              if (m8 == lay.rp) {  // whole tiles: one copy each
                bulk_copy(sa, ga, 2 * ca, &full[st]);
              } else {
                bulk_copy(sa, ga, ca, &full[st]);
                bulk_copy(sa + ha, ga + ha, ca, &full[st]);
              }
              if (n8 == lay.np) {
                bulk_copy(sb, gb, 2 * cb, &full[st]);
              } else {
                bulk_copy(sb, gb, cb, &full[st]);
                bulk_copy(sb + hb, gb + hb, cb, &full[st]);
              }
            }
          }
          if (!__shfl_sync(0xffffffffu, good, 0)) {
            ok = false;
            break;
          }
        }
      }
      si = si2;
    }
    if (lane == 0) {
      if (ok) {  // the end marker: a stage with no copies
        const int st = (int)(it % nst);
        const uint32_t use = it / nst;
        if (use == 0 || mbar_wait(&empty[st], (use - 1) & 1u, &s_abort)) {
          slot_k[st] = 0;
          slot_f[st] = kEnd;
          mbar_arrive(&full[st]);
        }
      } else {
        // the copies in flight land before the CTA leaves: wait for the last use of each
        // stage (stage st served items st, st + nst, ...: its last use is (it - 1 - st) / nst)
        for (uint32_t st = 0; st < nst && st < it; ++st) {
          volatile int never = 0;
          mbar_wait(&full[st], ((it - 1 - st) / nst) & 1u, &never);
        }
      }
    }
  } else if (warp == kIssuer) {
    if (lane == 0) {
      // the issuing thread: stages in order until the end marker
      uint32_t it = 0, seg_i = 0, use_acc[kMaxAcc];
      for (int b = 0; b < kMaxAcc; ++b) use_acc[b] = 0u;
      const uint32_t idesc = idesc_bf16(64, lay.np);
      int b = 0;
      bool issued = false;
      for (;; ++it) {
        const int st = (int)(it % nst);
        if (!mbar_wait(&full[st], (it / nst) & 1u, &s_abort)) break;
        const int kp = slot_k[st], nks = slot_s[st], fl = slot_f[st];
        if (fl & kEnd) break;
        if (fl & kFirst) {
          b = (int)(seg_i % (uint32_t)lay.nacc);
          if (use_acc[b] > 0 && !mbar_wait(&acce[b], (use_acc[b] - 1) & 1u, &s_abort)) break;
          // (the accumulator's last reads by the epilogue come before these products)
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          issued = false;
        }
        const uint32_t d = tmem + (uint32_t)(b * lay.ncols);
        const uint32_t sbo = (uint32_t)(kp / 8) * 128;
        const uint32_t a_hi = smem_u32(smem + st * lay.stage_bytes), a_lo = a_hi + (uint32_t)(lay.rp / 8) * sbo;
        const uint32_t b_hi = a_hi + (uint32_t)(lay.rp / 4) * sbo, b_lo = b_hi + (uint32_t)(lay.np / 8) * sbo;
        for (int ks = 0; ks < nks; ++ks) {
          const uint32_t o = (uint32_t)ks * 256;
          mma_bf16(d, smem_desc(a_hi + o, 128, sbo), smem_desc(b_hi + o, 128, sbo), idesc, issued ? 1u : 0u);
          issued = true;
          mma_bf16(d, smem_desc(a_hi + o, 128, sbo), smem_desc(b_lo + o, 128, sbo), idesc, 1u);
          mma_bf16(d, smem_desc(a_lo + o, 128, sbo), smem_desc(b_hi + o, 128, sbo), idesc, 1u);
        }
        mma_commit(&empty[st]);
        if (fl & kLast) {
          mma_commit(&accf[b]);
          use_acc[b] += 1;
          seg_i += 1;
        }
      }
      // every product issued above has finished once this commit's phase completes
      mma_commit(&done);
      volatile int never = 0;
      mbar_wait(&done, 0u, &never);
    }
  } else {
    // epilogue: warp w holds accumulator rows 16 w .. 16 w + 15 in its lanes 0 .. 15; the
    // segment's metadata and rank bounds are read before its products are waited for
    uint32_t seg_i = 0, use_acc[kMaxAcc];
    for (int b = 0; b < kMaxAcc; ++b) use_acc[b] = 0u;
    const int row = 16 * warp + lane;
    for (int64_t si = blockIdx.x; si < count; si += gridDim.x, ++seg_i) {
      const Seg s = segs[first + si];
      const Arenas* ar = ars + s.inst;
      const int M = bound(ar, s.mref, s.m), N = bound(ar, s.nref, s.n);
      const View out = view(ar, s.out);
      const bool accum = s.flags & SF_ACC;
      const int b = (int)(seg_i % (uint32_t)lay.nacc);
      if (!mbar_wait(&accf[b], use_acc[b] & 1u, &s_abort)) break;
      use_acc[b] += 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (16 * warp < M) {
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * lay.ncols + c0), v);
          if (lane < 16 && row < M) {
            const int64_t o = (int64_t)row * s.ldc + c0;
            if (out.f32) {
              float* po = (float*)out.base + o;
              if (accum) {  // all loads first, then the stores
                float old[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) old[j] = c0 + j < N ? po[j] : 0.f;
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += old[j];
              }
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (c0 + j < N) po[j] = v[j];
            } else {
              double* po = (double*)out.base + o;
              double w[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) w[j] = accum && c0 + j < N ? po[j] : 0.0;
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (c0 + j < N) po[j] = w[j] + (double)v[j];
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
  }
  __syncthreads();
  if (tid == 0 && s_abort && err) atomicOr(err, 1u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(lay.tmem_cols));
}

}  // namespace

void launch_coup_tc(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars,
                    int rp, int np, int kpmax, unsigned int* err, int variant, void* stream) {
  if (count <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(coup_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  });
  const TcLayout lay = tc_layout(rp, np, kpmax, variant % kTcVariants);
  if (rp > 64 || rp % 8 || np > 64 || np % 8 || np == 0 || kpmax % 16 || kpmax > 64 || lay.total > kMaxSmem)
    throw Error(H2_EINTERNAL, "tensor-core coupling launch outside its tile limits");
  // resident CTAs per SM: shared memory (227 KB, ~1 KB static and 1 KB reserved per CTA),
  // registers, threads, and tensor memory (512 columns: every resident CTA must get its
  // columns)
  static int regs = 0;
  if (!regs) {
    cudaFuncAttributes fa{};
    cuda_check(cudaFuncGetAttributes(&fa, coup_tc_kernel), "kernel attributes");
    regs = std::max(1, (fa.numRegs + 7) & ~7);
  }
  const int sm_cap = (227 * 1024) / (lay.total + 2048);
  const int reg_cap = 65536 / (kThreads * regs), thr_cap = 2048 / kThreads;
  const int per_sm = std::max(1, std::min(std::min(sm_cap, reg_cap), std::min(thr_cap, 512 / lay.tmem_cols)));
  const int64_t grid = std::min<int64_t>(count, 152LL * per_sm);
  coup_tc_kernel<<<(unsigned)grid, kThreads, lay.total, (cudaStream_t)stream>>>(d_segs, d_items, first, count, d_ars,
                                                                                lay, err);
  add_kernel_launches(1);
}

}  // namespace h2
