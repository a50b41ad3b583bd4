// Arithmetic-throughput probe for the roofline denominators that
// MEASURED_PEAKS.json does not carry: float64 and float32 SIMT FMA rate and
// the float64 tensor-core (DMMA m8n8k4) rate of the GPU it runs on.
// Bounded loops on register operands only.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_peaks probe_peaks.cu && ./probe_peaks
#include <cstdio>

#include <cuda_runtime.h>

template <typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void dmma_loop(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-6, b = 0.5;
  double c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0, c6 = 0, c7 = 0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c2), "+d"(c3) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c4), "+d"(c5) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c6), "+d"(c7) : "d"(a), "d"(b));
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3 + c4 + c5 + c6 + c7;
}

template <typename F>
float best_ms(F launch) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  return best;
}

int main() {
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, 0);
  const int sms = p.multiProcessorCount, blocks = sms * 8, threads = 256;
  printf("%s sm_%d%d SMs=%d\n", p.name, p.major, p.minor, sms);
  double* d;
  float* f;
  cudaMalloc(&d, sizeof(double) * blocks * threads);
  cudaMalloc(&f, sizeof(float) * blocks * threads);
  float ms = best_ms([&]() { fma_loop<double><<<blocks, threads>>>(d, 2000, 0.999, 0.001); });
  printf("fp64 FMA: %.3f TFLOP/s\n", 2.0 * 32 * 2000.0 * blocks * threads / (ms * 1e-3) / 1e12);
  ms = best_ms([&]() { fma_loop<float><<<blocks, threads>>>(f, 20000, 0.999f, 0.001f); });
  printf("fp32 FMA: %.3f TFLOP/s\n", 2.0 * 32 * 20000.0 * blocks * threads / (ms * 1e-3) / 1e12);
  ms = best_ms([&]() { dmma_loop<<<blocks, threads>>>(d, 2000); });
  printf("fp64 DMMA m8n8k4: %.3f TFLOP/s\n", 512.0 * 16 * 2000.0 * (blocks * threads / 32.0) / (ms * 1e-3) / 1e12);
  printf("status: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
