// Block-wide helpers of the Jacobi eigen-decompositions (kernels.cu: the product's
// eigen step; gbuild.cu: the construction on the GPU).
#pragma once
#include <cuda_runtime.h>

namespace h2 {

// sum of v over the block (red: one double per warp), returned to every thread
static __device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// Cyclic two-sided Jacobi with the round-robin (tournament) ordering on an nn x nn
// symmetric matrix A (row stride lds, nn even; padded rows and columns zero) with the
// rotations accumulated into the columns of V: each step applies nn/2 disjoint
// rotations, a sweep is nn - 1 steps; stops when off(A)^2 <= tol |A|^2 or after
// max_sweeps.  The rotation zeroing a_pq is the symmetric 2 x 2 Schur rotation
// tau = (a_qq - a_pp)/(2 a_pq), t = sign(tau)/(|tau| + sqrt(1 + tau^2)),
// c = 1/sqrt(1 + t^2), s = t c.  cs, sn, pp, qq: nn/2 entries of shared memory.
template <typename T>
__device__ void jacobi_sweeps(T* A, T* V, int nn, int lds, int max_sweeps, double tol, double* red, T* cs, T* sn,
                              int* pp, int* qq) {
  const int tid = threadIdx.x, nt = blockDim.x, np = nn / 2;
  const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  for (int sweep = 0; sweep < max_sweeps && nn > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = w; i < nn; i += nw)
      for (int j = lane; j < nn; j += 32) {
        double v = (double)A[i * lds + j] * (double)A[i * lds + j];
        tot += v;
        if (i != j) off += v;
      }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (!(off > tol * tot)) break;
    for (int step = 0; step < nn - 1; ++step) {
      for (int k = tid; k < np; k += nt) {
        int pa = (k == 0) ? 0 : ((k - 1 + step) % (nn - 1)) + 1;
        int pb = ((nn - 1 - k - 1 + step) % (nn - 1)) + 1;
        int p = min(pa, pb), q = max(pa, pb);
        T apq = A[p * lds + q];
        T c = T(1), s = T(0);
        if (apq != T(0)) {
          T tau = (A[q * lds + q] - A[p * lds + p]) / (T(2) * apq);
          T tt = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          c = T(1) / sqrt(T(1) + tt * tt);
          s = tt * c;
        }
        pp[k] = p;
        qq[k] = q;
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      for (int k = w; k < np; k += nw) {  // rows p, q
        if (sn[k] == T(0)) continue;
        const int p = pp[k], q = qq[k];
        const T c = cs[k], s = sn[k];
        for (int j = lane; j < nn; j += 32) {
          T x = A[p * lds + j], y = A[q * lds + j];
          A[p * lds + j] = c * x - s * y;
          A[q * lds + j] = s * x + c * y;
        }
      }
      __syncthreads();
      for (int k = w; k < np; k += nw) {  // columns p, q of A and V
        if (sn[k] == T(0)) continue;
        const int p = pp[k], q = qq[k];
        const T c = cs[k], s = sn[k];
        for (int i = lane; i < nn; i += 32) {
          T x = A[i * lds + p], y = A[i * lds + q];
          A[i * lds + p] = c * x - s * y;
          A[i * lds + q] = s * x + c * y;
          T vx = V[i * lds + p], vy = V[i * lds + q];
          V[i * lds + p] = c * vx - s * vy;
          V[i * lds + q] = s * vx + c * vy;
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace h2
