// Float64-pipe probe: issue cost of a warp-level DFMA with 32, 8 or 1 active
// lanes and 1, 4 or 8 warps per CTA, latency of a dependent DFMA chain, and
// the cost of a dependent float64 / float32 divide.  Bounded loops on
// register operands only; clock64() brackets each loop.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_fp64_pipe probe_fp64_pipe.cu && ./probe_fp64_pipe
#include <cstdio>
#include <cuda_runtime.h>
__global__ void k_tp(int iters, int active, double* out, long long* cyc) {
  const int lane = threadIdx.x & 31;
  if (lane >= active) return;
  double a0 = 1.0 + threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
  double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
  const double m = 0.999999999, c = 1e-12;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (lane == 0) cyc[blockIdx.x * 32 + threadIdx.x / 32] = t1 - t0;
}
__global__ void k_lat(int iters, double* out, long long* cyc) {
  if (threadIdx.x != 0) return;
  double a = 1.0;
  const double m = 0.999999999, c = 1e-12;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) a = fma(a, m, c);
  long long t1 = clock64();
  out[0] = a;
  cyc[0] = t1 - t0;
}
__global__ void k_div(int iters, int active, double* out, long long* cyc) {
  const int lane = threadIdx.x & 31;
  if (lane >= active) return;
  double a = 1.0 + lane * 1e-3, b = 3.0;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) { a = b / a + 0.5; }
  long long t1 = clock64();
  out[threadIdx.x] = a;
  if (lane == 0) cyc[threadIdx.x / 32] = t1 - t0;
}
__global__ void k_f32div(int iters, int active, double* out, long long* cyc) {
  const int lane = threadIdx.x & 31;
  if (lane >= active) return;
  float a = 1.0f + lane * 1e-3f, b = 3.0f;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) { a = b / a + 0.5f; }
  long long t1 = clock64();
  out[threadIdx.x] = a;
  if (lane == 0) cyc[threadIdx.x / 32] = t1 - t0;
}
int main() {
  double* out; long long* cyc; long long h[64];
  cudaMalloc(&out, 1 << 20); cudaMalloc(&cyc, 64 * 8);
  const int iters = 20000;
  int warps_list[3] = {1, 4, 8};
  for (int wi = 0; wi < 3; ++wi) {
    int w = warps_list[wi];
    for (int active : {32, 8, 1}) {
      k_tp<<<1, 32 * w>>>(iters, active, out, cyc); cudaDeviceSynchronize();
      k_tp<<<1, 32 * w>>>(iters, active, out, cyc); cudaDeviceSynchronize();
      cudaMemcpy(h, cyc, 8 * w, cudaMemcpyDeviceToHost);
      printf("throughput: warps=%d active=%2d  cycles per warp-DFMA = %.2f\n", w, active, (double)h[0] / (iters * 8.0));
    }
  }
  k_lat<<<1, 32>>>(iters, out, cyc); cudaDeviceSynchronize();
  cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
  printf("latency: dependent DFMA chain = %.2f cycles\n", (double)h[0] / iters);
  for (int active : {32, 1}) {
    k_div<<<1, 32>>>(2000, active, out, cyc); cudaDeviceSynchronize();
    cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
    printf("f64 divide chain: active=%2d  cycles per step = %.1f\n", active, (double)h[0] / 2000);
    k_f32div<<<1, 32>>>(2000, active, out, cyc); cudaDeviceSynchronize();
    cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
    printf("f32 divide chain: active=%2d  cycles per step = %.1f\n", active, (double)h[0] / 2000);
  }
  cudaError_t e = cudaGetLastError();
  printf("status %s\n", cudaGetErrorString(e));
  return 0;
}
