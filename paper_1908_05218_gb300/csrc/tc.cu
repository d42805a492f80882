// Sums of small products on the fifth-generation tensor cores (tcgen05) for
// H2_MIXED_BF16X3: the main coupling pass of every level (Eq. leafcoup_simple /
// nonleafcoup_simple: leaf case 1, cases 2/4 and case 3, summed per target), S_ik (=|+=)
// sum over the terms of A_t B_t, and the dense leaf products of the dense targets (Sec.
// III-A), F^C_ik = sum over j of F^A_ij F^B_jk (the tiles of the input matrices' dense
// blocks follow their float copies).
//
// The coupling operands were written by their producers (the projections and R images of
// the level) as BF16 split tiles (device.cuh): an A operand (rows of the target, k) as an
// rp x kp tile, a B operand transposed (columns of the target, k) as an np x kp tile, each
// in the K-major core-matrix layout of tcgen05 without swizzle, high parts then low parts.
// So a term's operands reach shared memory by bulk copies (cp.async.bulk, completing on
// an mbarrier), and the tensor cores read them there without any rearrangement.
//
// Targets are summed in pairs (TcGroup): the targets (i, k) and (i', k) of two sibling row
// clusters share the B operand of every term with a common middle cluster, so one step
// multiplies the two stacked A tiles (slot 0 in rows 0 .. sr-1, slot 1 in rows sr ..
// 2 sr - 1) by one B tile with an MMA of M = 2 sr rows: sr = 32 when both targets' ranks
// fit 32 rows (decided per pair from the ranks on the device), else 64, and such a step
// takes two consecutive stages of the ring (which is sized for M = 64).  A slot without a
// term in a step gets zero rows (copied from a zero block).  The MMA reads operands from
// shared memory, and this stacking halves the operand traffic of a term.
//
// A persistent CTA of six warps walks the launch's groups at a stride of the grid:
//   * warp 4 copies the steps' tiles into a ring of shared-memory stages (its lanes read
//     the metadata of 32 steps at a time, lane 0 issues), only the rows up to each
//     target's rank (rounded up to 8), a stage being reused once the products reading it
//     have completed; each stage's slot tells the issuing thread the step's k, its k-steps
//     (the rank of the middle cluster, rounded up to 16: the tiles hold zeros beyond it)
//     and whether it starts or ends the group;
//   * warp 5 (one thread) issues, per k-step of 16, the three products hi*hi, hi*lo and
//     lo*hi (tcgen05.mma kind::f16 with BF16 A and B, M = 2 sr, N = np rounded up to 16
//     for M = 128, float32 accumulation in tensor memory; the dropped lo*lo term is below
//     2^-16 of the product) into one of nacc accumulators, commits each stage to its
//     "empty" mbarrier and the group's last product to the accumulator's "full" mbarrier;
//   * warps 0-3 read the finished accumulator (tcgen05.ld) and store or add each slot's
//     rows to its target's coupling (warps 0, 1: slot 0; warps 2, 3: slot 1: with M = 64
//     row r sits in lane 32 (r / 16) + r % 16, with M = 128 in lane r), then release the
//     accumulator; a group's metadata is read before its products are waited for.
// Rows of a stage beyond the copied ones hold stale data: they only reach accumulator rows
// or columns that are never stored.  The products of a group run in step order, so results
// are bitwise reproducible.
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

// zero rows for a slot without a term in a step: 64 rows x 64 k of BF16
__device__ __align__(128) unsigned char g_zero_rows[64 * 64 * 2];

struct TcLayout {
  int rp, np;      // A tile rows, B tile rows (multiples of 8, at most 64)
  int sr, m;       // rows per slot (32 or 64) and the MMA's M (2 sr)
  int nm;          // the MMA's N: np, rounded up to 16 when M = 128
  int kpmax;       // largest tile k of the launch (a multiple of 16)
  int nst;         // stages of the copy ring
  int nacc;        // accumulators
  int trim;        // copy only the rows up to the targets' ranks (else whole tiles)
  int dynm;        // M = 64 for the groups whose ranks fit 32 rows per slot
  int stage_bytes; // a stage: A hi (64 rows), A lo, B hi (np rows), B lo, at the step's k;
                   // a step of M = 128 takes two consecutive stages
  int ncols;       // tensor-memory columns of one accumulator (np rounded up to 16)
  int tmem_cols;   // allocated columns: nacc accumulators, a power of two >= 32
  int total;       // dynamic shared memory
};

// launch configurations (stages, accumulators, trimmed copies, M per group), all with the
// same products in the same order: the autotuner picks one per launch group
constexpr int kTcConfigs[kTcVariants][4] = {{4, 2, 1, 1}, {3, 2, 1, 1}, {6, 2, 1, 1}, {4, 4, 1, 1}};

TcLayout tc_layout(int rp, int np, int kpmax, int variant) {
  TcLayout t;
  t.rp = rp;
  t.np = np;
  t.sr = rp <= 32 ? 32 : 64;
  t.m = 2 * t.sr;
  t.kpmax = kpmax;
  t.nst = kTcConfigs[variant][0];
  t.nacc = kTcConfigs[variant][1];
  t.trim = kTcConfigs[variant][2];
  t.dynm = kTcConfigs[variant][3];
  t.nm = t.m == 128 ? (np + 15) & ~15 : np;
  // (the MMA reads nm rows from B's lo part, which starts np rows into B: the stage holds
  // m + nm rows of each part)
  t.stage_bytes = ((64 + (t.sr == 64 ? t.nm : np)) * kpmax * 4 + 1023) & ~1023;
  t.ncols = (np + 15) & ~15;
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

// what the copying warp tells the issuing thread about the step in a stage
// kDouble: the step (M = 128) takes this stage and the next; kCont: the second stage of
// such a step; kSkip: a stage passed over (a double step does not wrap around the ring)
enum : int { kFirst = 1, kLast = 2, kEnd = 4, kM128 = 8, kDouble = 16, kCont = 32, kSkip = 64 };

// a group's rows per slot: 32 when both targets' ranks fit (M = 64), else the launch's
__device__ __forceinline__ int group_sr(const TcLayout& lay, const int m8[2]) {
  return lay.sr == 32 || (lay.dynm && m8[0] <= 32 && m8[1] <= 32) ? 32 : 64;
}

__global__ void __launch_bounds__(kThreads, 6) coup_tc_kernel(const TcGroup* __restrict__ groups,
                                                              const TcStep* __restrict__ steps, int64_t first,
                                                              int64_t count, const Arenas* __restrict__ ars,
                                                              TcLayout lay, unsigned int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], accf[kMaxAcc], acce[kMaxAcc], done;
  // per stage: the step's tile k and k-steps, kFirst | kLast | kEnd
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
    // the copying warp
    uint32_t it = 0;  // steps copied by this CTA
    bool ok = true;
    int64_t gi = blockIdx.x;
    TcGroup gn{};
    if (gi < count) gn = groups[first + gi];
    while (gi < count && ok) {
      const TcGroup g = gn;
      const int64_t gi2 = gi + gridDim.x;
      if (gi2 < count) gn = groups[first + gi2];  // the next group's, while this one is copied
      const Arenas* ar = ars + g.inst;
      // rows copied per slot (0: no target) and of B: up to the ranks, rounded up to 8
      int m8[2];
      for (int sl = 0; sl < 2; ++sl)
        m8[sl] = g.out[sl] < 0 ? 0 : (lay.trim ? max(8, (bound(ar, g.mref[sl], g.m) + 7) & ~7) : lay.rp);
      const int n8 = lay.trim ? max(8, (bound(ar, g.nref, g.n) + 7) & ~7) : lay.np;
      const int sr = group_sr(lay, m8), mm = 2 * sr;  // this group's rows per slot and M
      for (int b0 = 0; b0 < g.count && ok; b0 += 32) {
        const int nb = min(32, g.count - b0);
        unsigned long long pa0 = 0, pa1 = 0, pb = 0;
        int kp = 0, ks = 0;
        if (lane < nb) {
          const TcStep sp = steps[g.first + b0 + lane];
          pa0 = sp.a[0] >= 0 ? (unsigned long long)ptr_of<float>(ar, sp.a[0]) : 0ull;
          pa1 = sp.a[1] >= 0 ? (unsigned long long)ptr_of<float>(ar, sp.a[1]) : 0ull;
          pb = (unsigned long long)ptr_of<float>(ar, sp.b);
          kp = sp.kpad;
          ks = max(1, (bound(ar, sp.kref, kp) + 15) >> 4);
        }
        for (int q = 0; q < nb; ++q) {
          const unsigned long long a0 = __shfl_sync(0xffffffffu, pa0, q), a1 = __shfl_sync(0xffffffffu, pa1, q);
          const unsigned long long b = __shfl_sync(0xffffffffu, pb, q);
          const int k = __shfl_sync(0xffffffffu, kp, q), ksteps = __shfl_sync(0xffffffffu, ks, q);
          int good = 1;
          if (lane == 0) {
            // a stage is taken once its previous use's products have completed
            auto take = [&](uint32_t i) {
              const uint32_t use = i / nst;
              return use == 0 || mbar_wait(&empty[i % nst], (use - 1) & 1u, &s_abort);
            };
            const bool dbl = mm == 128;
            if (dbl && it % nst == nst - 1) {  // no room for two stages before the ring's end
              if (!take(it)) {
                good = 0;
              } else {
                const int st = (int)(it % nst);
                slot_k[st] = 0;
                slot_s[st] = 0;
                slot_f[st] = kSkip;
                mbar_arrive(&full[st]);
                ++it;
              }
            }
            const int st = (int)(it % nst);
            if (!good || !take(it) || (dbl && !take(it + 1))) {
              good = 0;
            } else {
              // stage: A hi (M rows), A lo (M rows), B hi (np rows), B lo (np rows); a tile
              // holds its hi part, then its lo part rows x k further
              const uint32_t part_a = (uint32_t)mm * k * 2, tile_a = (uint32_t)lay.rp * k * 2;
              const uint32_t part_b = (uint32_t)lay.np * k * 2, cb = (uint32_t)n8 * k * 2;
              unsigned char* sa = smem + st * lay.stage_bytes;
              unsigned char* sb = sa + 2 * part_a;
              uint32_t tx = 2 * cb;
              for (int sl = 0; sl < 2; ++sl) tx += 4u * m8[sl] * k;
              slot_k[st] = k;
              slot_s[st] = ksteps;
              slot_f[st] = (b0 + q == 0 ? kFirst : 0) | (b0 + q == g.count - 1 ? kLast : 0) | (dbl ? kM128 | kDouble : 0);
              mbar_expect_tx(&full[st], tx);
              for (int sl = 0; sl < 2; ++sl) {
                if (!m8[sl]) continue;
                const unsigned long long a = sl ? a1 : a0;
                const uint32_t ca = (uint32_t)m8[sl] * k * 2;
                unsigned char* d = sa + (uint32_t)sl * sr * k * 2;
                if (a) {
                  bulk_copy(d, (const void*)a, ca, &full[st]);
                  bulk_copy(d + part_a, (const void*)(a + tile_a), ca, &full[st]);
                } else {  // no term for this slot: zero rows
                  bulk_copy(d, g_zero_rows, ca, &full[st]);
                  bulk_copy(d + part_a, g_zero_rows, ca, &full[st]);
                }
              }
              if (n8 == lay.np) {
                bulk_copy(sb, (const void*)b, 2 * cb, &full[st]);
              } else {
                bulk_copy(sb, (const void*)b, cb, &full[st]);
                bulk_copy(sb + part_b, (const void*)(b + part_b), cb, &full[st]);
              }
              if (dbl) {  // the second stage of the step: no copies of its own
                slot_k[st + 1] = 0;
                slot_s[st + 1] = 0;
                slot_f[st + 1] = kCont;
                mbar_arrive(&full[st + 1]);
              }
              it += dbl ? 2 : 1;
            }
          }
          it = __shfl_sync(0xffffffffu, it, 0);
          if (!__shfl_sync(0xffffffffu, good, 0)) {
            ok = false;
            break;
          }
        }
      }
      gi = gi2;
    }
    if (lane == 0) {
      if (ok) {  // the end marker: a stage with no copies
        const int st = (int)(it % nst);
        const uint32_t use = it / nst;
        if (use == 0 || mbar_wait(&empty[st], (use - 1) & 1u, &s_abort)) {
          slot_k[st] = 0;
          slot_s[st] = 0;
          slot_f[st] = kEnd;
          mbar_arrive(&full[st]);
        }
      } else {
        // the copies in flight land before the CTA leaves: wait for the last use of each
        // stage (stage st served steps st, st + nst, ...: its last use is (it - 1 - st) / nst)
        for (uint32_t st = 0; st < nst && st < it; ++st) {
          volatile int never = 0;
          mbar_wait(&full[st], ((it - 1 - st) / nst) & 1u, &never);
        }
      }
    }
  } else if (warp == kIssuer) {
    if (lane == 0) {
      // the issuing thread: stages in order until the end marker
      uint32_t it = 0, grp_i = 0, use_acc[kMaxAcc];
      for (int b = 0; b < kMaxAcc; ++b) use_acc[b] = 0u;
      const uint32_t idesc64 = idesc_bf16(64, lay.np), idesc128 = idesc_bf16(128, (lay.np + 15) & ~15);
      int b = 0;
      bool issued = false;
      for (;; ++it) {
        const int st = (int)(it % nst);
        if (!mbar_wait(&full[st], (it / nst) & 1u, &s_abort)) break;
        const int kp = slot_k[st], nks = slot_s[st], fl = slot_f[st];
        if (fl & kEnd) break;
        if (fl & (kSkip | kCont)) {  // (a continuation's stage is free once the step's products are)
          mma_commit(&empty[st]);
          continue;
        }
        if (fl & kFirst) {
          b = (int)(grp_i % (uint32_t)lay.nacc);
          if (use_acc[b] > 0 && !mbar_wait(&acce[b], (use_acc[b] - 1) & 1u, &s_abort)) break;
          // (the accumulator's last reads by the epilogue come before these products)
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          issued = false;
        }
        const uint32_t d = tmem + (uint32_t)(b * lay.ncols);
        const int mm = (fl & kM128) ? 128 : 64;
        const uint32_t idesc = mm == 128 ? idesc128 : idesc64;
        const uint32_t sbo = (uint32_t)(kp / 8) * 128;
        const uint32_t a_hi = smem_u32(smem + st * lay.stage_bytes), a_lo = a_hi + (uint32_t)(mm / 8) * sbo;
        const uint32_t b_hi = a_hi + (uint32_t)(mm / 4) * sbo, b_lo = b_hi + (uint32_t)(lay.np / 8) * sbo;
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
          grp_i += 1;
        }
      }
      // every product issued above has finished once this commit's phase completes
      mma_commit(&done);
      volatile int never = 0;
      mbar_wait(&done, 0u, &never);
    }
  } else {
    // epilogue: warps 2 sl and 2 sl + 1 hold slot sl's rows; with M = 64 warp w holds rows
    // 16 w .. 16 w + 15 of the accumulator in its lanes 0 .. 15, with M = 128 rows 32 w ..
    // 32 w + 31
    const int sl = warp >> 1;
    uint32_t grp_i = 0, use_acc[kMaxAcc];
    for (int b = 0; b < kMaxAcc; ++b) use_acc[b] = 0u;
    for (int64_t gi = blockIdx.x; gi < count; gi += gridDim.x, ++grp_i) {
      const TcGroup g = groups[first + gi];
      const Arenas* ar = ars + g.inst;
      const bool have = g.out[sl] >= 0;
      const int M = have ? bound(ar, g.mref[sl], g.m) : 0, N = bound(ar, g.nref, g.n);
      // the group's M, decided from the slots' ranks as the copying warp did
      int m8[2];
      for (int s2 = 0; s2 < 2; ++s2)
        m8[s2] = g.out[s2] < 0 ? 0 : (lay.trim ? max(8, (bound(ar, g.mref[s2], g.m) + 7) & ~7) : lay.rp);
      const int rows_w = group_sr(lay, m8) == 32 ? 16 : 32;
      const int row = rows_w * (warp & 1) + lane;  // row within the slot
      const View out = view(ar, have ? g.out[sl] : g.out[sl ^ 1]);
      const bool accum = (g.acc >> sl) & 1;
      const int b = (int)(grp_i % (uint32_t)lay.nacc);
      if (!mbar_wait(&accf[b], use_acc[b] & 1u, &s_abort)) break;
      use_acc[b] += 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (rows_w * (warp & 1) < M) {
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * lay.ncols + c0), v);
          if (lane < rows_w && row < M) {
            const int64_t o = (int64_t)row * g.ldc + c0;
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

// registers per thread of the kernel (allocation granularity 8), read once
int g_tc_regs = 0;

}  // namespace

void init_coup_tc_attributes() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(coup_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    cudaFuncAttributes fa{};
    g_tc_regs = cudaFuncGetAttributes(&fa, coup_tc_kernel) == cudaSuccess ? std::max(8, (fa.numRegs + 7) & ~7) : 64;
  });
}

void launch_coup_tc(const TcGroup* d_groups, const TcStep* d_steps, int64_t first, int64_t count,
                    const Arenas* d_ars, int rp, int np, int kpmax, unsigned int* err, int variant, void* stream) {
  if (count <= 0) return;
  init_coup_tc_attributes();
  const TcLayout lay = tc_layout(rp, np, kpmax, variant % kTcVariants);
  if (rp > 64 || rp % 8 || np > 64 || np % 8 || np == 0 || kpmax % 16 || kpmax > 64 || lay.total > kMaxSmem)
    throw Error(H2_EINTERNAL, "tensor-core coupling launch outside its tile limits");
  // resident CTAs per SM: shared memory (227 KB, ~1 KB static and 1 KB reserved per CTA),
  // registers, threads, and tensor memory (512 columns: every resident CTA must get its
  // columns)
  const int regs = g_tc_regs;
  const int sm_cap = (227 * 1024) / (lay.total + 2048);
  const int reg_cap = 65536 / (kThreads * regs), thr_cap = 2048 / kThreads;
  const int per_sm = std::max(1, std::min(std::min(sm_cap, reg_cap), std::min(thr_cap, 512 / lay.tmem_cols)));
  const int64_t grid = std::min<int64_t>(count, 152LL * per_sm);
  coup_tc_kernel<<<(unsigned)grid, kThreads, lay.total, (cudaStream_t)stream>>>(d_groups, d_steps, first, count, d_ars,
                                                                                lay, err);
  add_kernel_launches(1);
}

}  // namespace h2
