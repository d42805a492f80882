// y = H x without any allocation: the matvec's work space (tree-ordered copies
// of x and y, the per-level coefficient vectors and the block lists) lives in one
// file-scope device array of fixed size instead of memory obtained from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory during the call, for
// example code running under a memory budget fixed up front, or a host that has
// handed all free device memory to another allocator.  Limits: the array holds
// kScratchBytes (32 MiB); the call returns H2_EINVAL when a matrix and nrhs need
// more.  Every device that loads the library keeps the array until the process
// exits.  All calls share the one array: calls that overlap on the GPU (two streams,
// two threads) race and give wrong results; the first call on a device looks up the
// array's device address (cudaGetSymbolAddress) and should therefore come before
// any stream capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "internal.hpp"

namespace h2 {

constexpr int64_t kScratchBytes = 32ll << 20;
static __device__ __align__(256) unsigned char g_mv_scratch[kScratchBytes];

namespace {

// device addresses of g_mv_scratch, per device (set once, with that device current)
void* g_scratch_ptr[64] = {nullptr};

constexpr int kThreads = 128;

// leaf forward transform: xh[t][a][c] = sum_r Vc_t[r][a] xt[t LS + r][c], with the
// gather of x into padded tree order done on the fly
__global__ void na_forward_leaf(const double* __restrict__ x, const int64_t* __restrict__ user,
                                const double* __restrict__ Vc, double* __restrict__ xt,
                                double* __restrict__ xh, int LS, int K, int64_t n, int nrhs) {
  const int64_t t = blockIdx.x;
  for (int e = threadIdx.x; e < LS * nrhs; e += blockDim.x) {
    int r = e / nrhs, c = e % nrhs;
    int64_t u = user[t * LS + r];
    xt[(t * LS + r) * nrhs + c] = u >= 0 ? x[u + (int64_t)c * n] : 0.0;
  }
  __syncthreads();
  const double* V = Vc + t * (int64_t)LS * K;
  for (int e = threadIdx.x; e < K * nrhs; e += blockDim.x) {
    int a = e / nrhs, c = e % nrhs;
    double acc = 0.0;
    for (int r = 0; r < LS; ++r) acc += V[r * K + a] * xt[(t * LS + r) * nrhs + c];
    xh[(t * K + a) * nrhs + c] = acc;
  }
}

// forward transform one level up: xh_l[t] = E_t^T [xh_{l+1}[2t]; xh_{l+1}[2t+1]]
__global__ void na_forward_up(const double* __restrict__ E, const double* __restrict__ xc,
                              double* __restrict__ xp, int Kc, int Kp, int nrhs) {
  const int64_t t = blockIdx.x;
  const double* Et = E + t * 2LL * Kc * Kp;
  const double* xs = xc + 2 * t * (int64_t)Kc * nrhs;
  for (int e = threadIdx.x; e < Kp * nrhs; e += blockDim.x) {
    int a = e / nrhs, c = e % nrhs;
    double acc = 0.0;
    for (int r = 0; r < 2 * Kc; ++r) acc += Et[r * Kp + a] * xs[r * nrhs + c];
    xp[(t * Kp + a) * nrhs + c] = acc;
  }
}

// coupling of one level: yh[t] = sum over admissible (t, s) of S_ts xh[s]; on the
// leaf level also the near field yt[t] = sum over dense (t, s) of F_ts xt[s]
__global__ void na_coupling(const Block* __restrict__ blocks, const int32_t* __restrict__ row_ptr,
                            const double* __restrict__ S, const double* __restrict__ F,
                            const double* __restrict__ xh, double* __restrict__ yh,
                            const double* __restrict__ xt, double* __restrict__ yt, int Kr, int Kc, int LS,
                            int nrhs, int leaf) {
  const int64_t t = blockIdx.x;
  const int32_t p0 = row_ptr[t], p1 = row_ptr[t + 1];
  for (int e = threadIdx.x; e < Kr * nrhs; e += blockDim.x) {
    int a = e / nrhs, c = e % nrhs;
    double acc = 0.0;
    for (int32_t p = p0; p < p1; ++p) {
      const Block b = blocks[p];
      if (b.kind != KR) continue;
      const double* Sb = S + b.idx * (int64_t)Kr * Kc;
      for (int q = 0; q < Kc; ++q) acc += Sb[a * Kc + q] * xh[((int64_t)b.s * Kc + q) * nrhs + c];
    }
    yh[(t * Kr + a) * nrhs + c] = acc;
  }
  if (!leaf) return;
  for (int e = threadIdx.x; e < LS * nrhs; e += blockDim.x) {
    int r = e / nrhs, c = e % nrhs;
    double acc = 0.0;
    for (int32_t p = p0; p < p1; ++p) {
      const Block b = blocks[p];
      if (b.kind != KF) continue;
      const double* Fb = F + b.idx * (int64_t)LS * LS;
      for (int q = 0; q < LS; ++q) acc += Fb[r * LS + q] * xt[((int64_t)b.s * LS + q) * nrhs + c];
    }
    yt[(t * LS + r) * nrhs + c] = acc;
  }
}

// backward transform one level down: [yh_{l+1}[2t]; yh_{l+1}[2t+1]] += E_t yh_l[t]
__global__ void na_backward(const double* __restrict__ E, const double* __restrict__ yp,
                            double* __restrict__ yc, int Kc, int Kp, int nrhs) {
  const int64_t t = blockIdx.x;
  const double* Et = E + t * 2LL * Kc * Kp;
  double* ys = yc + 2 * t * (int64_t)Kc * nrhs;
  for (int e = threadIdx.x; e < 2 * Kc * nrhs; e += blockDim.x) {
    int r = e / nrhs, c = e % nrhs;
    double acc = 0.0;
    for (int a = 0; a < Kp; ++a) acc += Et[r * Kp + a] * yp[(t * Kp + a) * nrhs + c];
    ys[r * nrhs + c] += acc;
  }
}

// leaf backward transform and scatter to user order: y = yt + Vr yh
__global__ void na_backward_leaf(const double* __restrict__ Vr, const double* __restrict__ yh,
                                 const double* __restrict__ yt, const int64_t* __restrict__ user,
                                 double* __restrict__ y, int LS, int K, int64_t n, int nrhs) {
  const int64_t t = blockIdx.x;
  const double* V = Vr + t * (int64_t)LS * K;
  for (int e = threadIdx.x; e < LS * nrhs; e += blockDim.x) {
    int r = e / nrhs, c = e % nrhs;
    int64_t u = user[t * LS + r];
    if (u < 0) continue;
    double acc = yt[(t * LS + r) * nrhs + c];
    for (int a = 0; a < K; ++a) acc += V[r * K + a] * yh[(t * K + a) * nrhs + c];
    y[u + (int64_t)c * n] = acc;
  }
}

int64_t align256(int64_t b) { return (b + 255) & ~int64_t(255); }

}  // namespace

// Entry point body (declared in capi.cu's extern "C" block via h2_matvec_noalloc).
h2_status matvec_noalloc(const Mat& m, const int64_t* d_user, const double* x, double* y, int64_t nrhs,
                         std::string& err) {
  const Structure& st = *m.st;
  const int L = st.L, LS = st.LS;
  const int64_t nl = 1LL << L;
  if (nrhs < 1 || nrhs > 64) {
    err = "h2_matvec_noalloc: nrhs must lie in [1, 64]";
    return H2_EINVAL;
  }
  // layout of the static array: xt, yt, xh[0..L], yh[0..L], blocks and row pointers
  int64_t off = 0;
  const int64_t o_xt = off;
  off = align256(off + nl * LS * nrhs * 8);
  const int64_t o_yt = off;
  off = align256(off + nl * LS * nrhs * 8);
  int64_t o_xh[32], o_yh[32], o_bl[32], o_rp[32];
  for (int l = 0; l <= L; ++l) {
    o_xh[l] = off;
    off = align256(off + (1LL << l) * m.Kc[l] * nrhs * 8);
    o_yh[l] = off;
    off = align256(off + (1LL << l) * m.Kr[l] * nrhs * 8);
  }
  for (int l = 0; l <= L; ++l) {
    o_bl[l] = off;
    off = align256(off + (int64_t)st.blocks[l].size() * (int64_t)sizeof(Block));
    o_rp[l] = off;
    off = align256(off + (int64_t)st.row_ptr[l].size() * 4);
  }
  if (off > kScratchBytes) {
    err = "h2_matvec_noalloc: needs " + std::to_string(off) + " bytes of static scratch, the limit is " +
          std::to_string(kScratchBytes) + " (32 MiB)";
    return H2_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    err = std::string("h2_matvec_noalloc: cudaGetDevice: ") + cudaGetErrorString(e);
    return H2_ECUDA;
  }
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mv_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("h2_matvec_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return H2_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_scratch_ptr[dev];
  cudaStream_t s = (cudaStream_t)m.stream;
  for (int l = 0; l <= L; ++l) {
    e = cudaMemcpyAsync(base + o_bl[l], st.blocks[l].data(), st.blocks[l].size() * sizeof(Block),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + o_rp[l], st.row_ptr[l].data(), st.row_ptr[l].size() * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      err = std::string("h2_matvec_noalloc: copy of the block lists: ") + cudaGetErrorString(e);
      return H2_ECUDA;
    }
  }
  double* xt = (double*)(base + o_xt);
  double* yt = (double*)(base + o_yt);
  auto xh = [&](int l) { return (double*)(base + o_xh[l]); };
  auto yh = [&](int l) { return (double*)(base + o_yh[l]); };
  const int nr = (int)nrhs;
  na_forward_leaf<<<(unsigned)nl, kThreads, 0, s>>>(x, d_user, m.arena + m.off_Vc, xt, xh(L), LS, m.Kc[L], st.n, nr);
  for (int l = L - 1; l >= 0; --l)
    na_forward_up<<<(unsigned)(1LL << l), kThreads, 0, s>>>(m.arena + m.off_Ec[l], xh(l + 1), xh(l), m.Kc[l + 1],
                                                           m.Kc[l], nr);
  for (int l = 0; l <= L; ++l)
    na_coupling<<<(unsigned)(1LL << l), kThreads, 0, s>>>((const Block*)(base + o_bl[l]), (const int32_t*)(base + o_rp[l]),
                                                         m.arena + m.off_S[l], m.arena + m.off_F, xh(l), yh(l), xt, yt,
                                                         m.Kr[l], m.Kc[l], LS, nr, l == L);
  for (int l = 0; l < L; ++l)
    na_backward<<<(unsigned)(1LL << l), kThreads, 0, s>>>(m.arena + m.off_Er[l], yh(l), yh(l + 1), m.Kr[l + 1],
                                                         m.Kr[l], nr);
  na_backward_leaf<<<(unsigned)nl, kThreads, 0, s>>>(m.arena + m.off_Vr, yh(L), yt, d_user, y, LS, m.Kr[L], st.n, nr);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("h2_matvec_noalloc: launch: ") + cudaGetErrorString(e);
    return H2_ECUDA;
  }
  return H2_OK;
}

}  // namespace h2
