// Device-side views of the arena tables shared by the kernels of the product (kernels.cu,
// mma.cu): a tagged offset selects one of the eight arenas of a product instance
// (Arenas, internal.hpp) and its element type (float or double).
#pragma once
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

}  // namespace h2
