// fp64_peak.cu -- FP64 throughput of this GPU: DFMA (8 independent FMA chains
// per thread), DMMA (mma.sync.aligned.m8n8k4 f64, 4 independent accumulators
// per warp) and FFMA for comparison.  Grid: 8 CTAs x 256 threads per SM.
// Build and run: python bench.py --measure-fp64-peak
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

__global__ void dfma_kernel(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void ffma_kernel(float* out, int iters, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < iters; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void dmma_kernel(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-9, b = 1.0 - threadIdx.x * 1e-9;
  double c[4][2] = {{0,0},{0,0},{0,0},{0,0}};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[j][0]), "+d"(c[j][1]) : "d"(a), "d"(b));
  }
  double s = 0; for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int nsm = p.multiProcessorCount;
  const int threads = 256, blocks = nsm * 8;
  double* dout; float* fout;
  CK(cudaMalloc(&dout, sizeof(double) * threads * blocks));
  CK(cudaMalloc(&fout, sizeof(float) * threads * blocks));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms; int it;
  // DFMA
  it = 20000;
  dfma_kernel<<<blocks, threads>>>(dout, 100, 0.999, 1e-3); CK(cudaDeviceSynchronize());
  cudaEventRecord(e0); dfma_kernel<<<blocks, threads>>>(dout, it, 0.999, 1e-3); cudaEventRecord(e1);
  CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms, e0, e1);
  double dfma_tf = 2.0 * 8 * (double)it * threads * blocks / (ms * 1e-3) / 1e12;
  // FFMA
  it = 200000;
  ffma_kernel<<<blocks, threads>>>(fout, 100, 0.999f, 1e-3f); CK(cudaDeviceSynchronize());
  cudaEventRecord(e0); ffma_kernel<<<blocks, threads>>>(fout, it, 0.999f, 1e-3f); cudaEventRecord(e1);
  CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms, e0, e1);
  double ffma_tf = 2.0 * 8 * (double)it * threads * blocks / (ms * 1e-3) / 1e12;
  // DMMA: each mma = 8x8x4 FMA = 512 flops per warp
  it = 20000;
  dmma_kernel<<<blocks, threads>>>(dout, 100); CK(cudaDeviceSynchronize());
  cudaEventRecord(e0); dmma_kernel<<<blocks, threads>>>(dout, it); cudaEventRecord(e1);
  CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms, e0, e1);
  double dmma_tf = 512.0 * 4 * (double)it * (threads / 32) * blocks / (ms * 1e-3) / 1e12;
  int clk; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("{\"gpu\": \"%s\", \"sms\": %d, \"clock_khz\": %d, \"dfma_tflops\": %.4f, \"dmma_tflops\": %.4f, \"ffma_tflops\": %.3f}\n",
         p.name, nsm, clk, dfma_tf, dmma_tf, ffma_tf);
  return 0;
}
