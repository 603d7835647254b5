// Throughput probe for the roofline denominators of the ALU-bound kernels:
// FP32 FMA, MUFU lg2, FP32 logf, FP64 FMA, FP64 log and FP64 tensor (m8n8k4) rates.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/pp peaks_probe.cu && /tmp/pp
#include <cstdio>
#include <cuda_runtime.h>
#include <cmath>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA error %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__global__ void k_ffma(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = fmaf(x[i], a, b);
  }
  float s = 0; for (int i = 0; i < 8; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_lg2(float* out, int iters) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = 2.0f + threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) {
      float y; asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
      x[i] = y + 2.0f;
    }
  }
  float s = 0; for (int i = 0; i < 8; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_logf(float* out, int iters) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = 2.0f + threadIdx.x * 1e-3f + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = logf(x[i]) + 2.0f;
  }
  float s = 0; for (int i = 0; i < 8; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; i++) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = fma(x[i], a, b);
  }
  double s = 0; for (int i = 0; i < 8; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dlog(double* out, int iters) {
  double x[4];
#pragma unroll
  for (int i = 0; i < 4; i++) x[i] = 2.0 + threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 4; i++) x[i] = log(x[i]) + 2.0;
  }
  double s = 0; for (int i = 0; i < 4; i++) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dmma(double* out, int iters) {
  // 4 independent accumulator sets per warp; each mma: 8x8x4 => 512 flops per warp.
  double a = 1.0 + threadIdx.x * 1e-6, b = 0.999;
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; i++) { c[i][0] = 0; c[i][1] = 0; }
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
    }
  }
  double s = 0; for (int i = 0; i < 4; i++) s += c[i][0] + c[i][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  int dev = 0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, dev));
  int sms = p.multiProcessorCount;
  int blocks = sms * 8, threads = 256;
  size_t n = (size_t)blocks * threads;
  float* of; double* od;
  CK(cudaMalloc(&of, n * sizeof(float))); CK(cudaMalloc(&od, n * sizeof(double)));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  float ms;
  printf("{\"gpu\": \"%s\", \"sms\": %d, \"cc\": \"%d.%d\", \"clock_khz\": %d", p.name, sms, p.major, p.minor, 0);
#define TIME(launch, ops_expr, name) \
  { launch; CK(cudaDeviceSynchronize()); float best = 1e30f; \
    for (int r = 0; r < 5; r++) { CK(cudaEventRecord(e0)); launch; CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1)); \
      CK(cudaEventElapsedTime(&ms, e0, e1)); if (ms < best) best = ms; } \
    double ops = (ops_expr); printf(", \"%s\": %.4g", name, ops / (best * 1e-3)); }
  int it = 4096;
  TIME((k_ffma<<<blocks, threads>>>(of, it, 0.9999f, 1e-4f)), 2.0 * 8 * it * (double)n, "ffma_flops");
  TIME((k_lg2<<<blocks, threads>>>(of, it / 4)), 8.0 * (it / 4) * (double)n, "mufu_lg2_per_s");
  TIME((k_logf<<<blocks, threads>>>(of, it / 8)), 8.0 * (it / 8) * (double)n, "logf_per_s");
  TIME((k_dfma<<<blocks, threads>>>(od, it / 16, 0.9999, 1e-4)), 2.0 * 8 * (it / 16) * (double)n, "dfma_flops");
  TIME((k_dlog<<<blocks, threads>>>(od, it / 64)), 4.0 * (it / 64) * (double)n, "dlog_per_s");
  TIME((k_dmma<<<blocks, threads>>>(od, it / 16)), 512.0 * 4 * (it / 16) * (double)(n / 32), "dmma_flops");
  printf("}\n");
  CK(cudaGetLastError());
  return 0;
}
