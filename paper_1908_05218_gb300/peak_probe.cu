// Arithmetic throughput probe of one GPU: float64 FMA (DFMA), float32 FMA (FFMA)
// and the float64 mma.sync m8n8k4 instruction, each from 8 independent chains per
// thread on 8 CTAs of 256 threads per SM.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o peak_probe peak_probe.cu && ./peak_probe
#include <cstdio>
#include <cuda_runtime.h>
__global__ void dfma_k(double* out, int iters) {
  double a0 = threadIdx.x * 1e-9, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4=a0+4,a5=a0+5,a6=a0+6,a7=a0+7;
  const double b = 0.999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
__global__ void ffma_k(float* out, int iters) {
  float a0 = threadIdx.x * 1e-9f, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4=a0+4,a5=a0+5,a6=a0+6,a7=a0+7;
  const float b = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
    a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
    a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
__global__ void dmma_k(double* out, int iters) {
  double a = threadIdx.x * 1e-9, b = 1.0 - a;
  double c0 = 0, c1 = 0, d0 = 0, d1 = 0, e0=0,e1=0,f0=0,f1=0;
  for (int i = 0; i < iters; ++i) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(d0), "+d"(d1) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(e0), "+d"(e1) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(f0), "+d"(f1) : "d"(a), "d"(b));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + d0 + d1+e0+e1+f0+f1;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  printf("%s SMs=%d cc=%d.%d smem/blk optin=%zu\n", p.name, p.multiProcessorCount, p.major, p.minor, p.sharedMemPerBlockOptin);
  int blocks = p.multiProcessorCount * 8, threads = 256, iters = 1 << 16;
  double* d; cudaMalloc(&d, sizeof(double) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0); dfma_k<<<blocks, threads>>>(d, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("DFMA: %.2f TFLOP/s (%.2f ms)\n", 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12, ms);
    cudaEventRecord(e0); ffma_k<<<blocks, threads>>>((float*)d, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("FFMA: %.2f TFLOP/s (%.2f ms)\n", 2.0 * 8 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12, ms);
    int it2 = iters / 16;
    cudaEventRecord(e0); dmma_k<<<blocks, threads>>>(d, it2); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    // one m8n8k4 = 2*8*8*4 = 512 flops per warp
    printf("DMMA: %.2f TFLOP/s (%.2f ms)\n", 4.0 * 512.0 * it2 * (double)blocks * threads / 32 / (ms * 1e-3) / 1e12, ms);
  }
  printf("err=%s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
