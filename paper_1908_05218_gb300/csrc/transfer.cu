// Moves between the packed host layout of an H^2 matrix (h2_import / h2_export: the
// arrays vr, vc, er, ec, s, f at the actual ranks, back to back) and its padded device
// arena.  The host copies only the packed bytes; the padding and unpadding are done
// here, one warp per block (leaf basis, transfer half, coupling, dense block).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.hpp"

namespace h2 {

__global__ void scatter_kernel(const CopyTask* __restrict__ tasks, int64_t ntasks, const double* __restrict__ packed,
                               double* __restrict__ arena) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = w; t < ntasks; t += nw) {
    const CopyTask c = tasks[t];
    const int64_t n = (int64_t)c.rows * c.cols;
    for (int64_t e = lane; e < n; e += 32) {
      const int64_t r = e / c.cols, q = e - r * c.cols;
      arena[c.arena_off + r * c.ld + q] = packed[c.packed_off + e];
    }
  }
}

__global__ void gather_kernel(const CopyTask* __restrict__ tasks, int64_t ntasks, const double* __restrict__ arena,
                              double* __restrict__ packed) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = w; t < ntasks; t += nw) {
    const CopyTask c = tasks[t];
    const int64_t n = (int64_t)c.rows * c.cols;
    for (int64_t e = lane; e < n; e += 32) {
      const int64_t r = e / c.cols, q = e - r * c.cols;
      packed[c.packed_off + e] = arena[c.arena_off + r * c.ld + q];
    }
  }
}

void launch_copy_tasks(const CopyTask* d_tasks, int64_t ntasks, double* packed, double* arena, bool to_arena,
                       void* stream) {
  if (ntasks == 0) return;
  const int64_t blocks = std::min<int64_t>((ntasks + 7) / 8, 152 * 64);
  if (to_arena)
    scatter_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_tasks, ntasks, packed, arena);
  else
    gather_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_tasks, ntasks, arena, packed);
  add_kernel_launches(1);
}

}  // namespace h2
