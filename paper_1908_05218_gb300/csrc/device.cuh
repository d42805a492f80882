// Device-side views of the arena tables shared by the kernels of the product (kernels.cu,
// mma.cu): a tagged offset selects one of the eight arenas of a product instance
// (Arenas, internal.hpp) and its element type (float or double).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.hpp"

namespace h2 {

__device__ __forceinline__ int arena_idx(int64_t t) { return (int)((t >> kTagShift) & 7); }

// typed view of one tagged matrix: float or double storage, read/written as Acc
struct View {
  char* base;
  bool f32;
};

// (a points at the instance's table in device memory; a.flops, if set, collects the
// executed multiply-add flops)
__device__ __forceinline__ View view(const Arenas* a, int64_t t) {
  int ai = arena_idx(t);
  bool f = (a->f32 >> ai) & 1;
  return View{a->p[ai] + (t & kOffMask) * (f ? 4 : 8), f};
}

template <typename Acc>
__device__ __forceinline__ Acc ld(const View& v, int64_t i) {
  return v.f32 ? (Acc)((const float*)v.base)[i] : (Acc)((const double*)v.base)[i];
}

template <typename Acc>
__device__ __forceinline__ void st(const View& v, int64_t i, Acc x, bool acc) {
  if (v.f32) {
    float* p = (float*)v.base + i;
    *p = acc ? (float)(*p + x) : (float)x;
  } else {
    double* p = (double*)v.base + i;
    *p = acc ? *p + (double)x : (double)x;
  }
}

__device__ __forceinline__ int bound(const Arenas* a, int32_t ref, int padded) {
  if (ref < 0) return padded;
  int r = a->rk[ref >> kRefShift][ref & ((1 << kRefShift) - 1)];
  return r < padded ? r : padded;
}

template <typename T>
__device__ __forceinline__ const T* ptr_of(const Arenas* a, int64_t t) {
  return (const T*)a->p[arena_idx(t)] + (t & kOffMask);
}

// Tensor-core operand tiles of the BF16 split product (H2_MIXED_BF16X3): a matrix of tr
// rows and kp columns (tr a multiple of 8, kp of 16) stored as core matrices of 8 rows x
// 8 BF16 values (16 bytes per row, 128 bytes each), the one of row group g and k-chunk c
// at element (g * kp / 8 + c) * 64; the high parts first, the low parts tr * kp elements
// further: x = hi + lo with hi = bf16(x), lo = bf16(x - hi).  The tile takes the place of
// tr * kp float32 values in a float arena.
__device__ __forceinline__ int64_t tile_idx(int row, int k, int kp) {
  return ((int64_t)(row >> 3) * (kp >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}
__device__ __forceinline__ void tile_store(char* base, int tr, int kp, int row, int k, float x) {
  __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(base);
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  const int64_t i = tile_idx(row, k, kp);
  p[i] = hi;
  p[(int64_t)tr * kp + i] = lo;
}
__device__ __forceinline__ float tile_load(const char* base, int tr, int kp, int row, int k) {
  const __nv_bfloat16* p = reinterpret_cast<const __nv_bfloat16*>(base);
  const int64_t i = tile_idx(row, k, kp);
  return __bfloat162float(p[i]) + __bfloat162float(p[(int64_t)tr * kp + i]);
}

}  // namespace h2
