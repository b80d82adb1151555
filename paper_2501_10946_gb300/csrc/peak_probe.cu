// Throughput probe of the GB300 execution units used by the rooflines: independent
// dependency chains per thread, timed with CUDA events.  Standalone program, not part
// of the library:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o peak_probe paper_2501_10946_gb300/csrc/peak_probe.cu
//   ./peak_probe
#include <cstdio>
#include <cuda_runtime.h>
#define CH 8
template<int KIND>
__global__ void k_probe(float* out, int iters, float seed) {
  float a[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) a[c] = seed + 0.001f * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (KIND == 0) { float r; asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c])); a[c] = r; }
      if (KIND == 1) { float r; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c])); a[c] = r; }
      if (KIND == 2) { a[c] = fmaf(a[c], 0.999f, 0.0001f); }
      if (KIND == 3) { int i = __float_as_int(a[c]) ^ 0x5; a[c] = (float)i; }
      if (KIND == 4) { float r; asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c])); a[c] = r; }
      if (KIND == 5) { float s, co; __sincosf(a[c], &s, &co); a[c] = s + co; }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_dfma(double* out, int iters, double seed) {
  double a[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) a[c] = seed + 0.001 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] = fma(a[c], 0.999, 0.0001);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_clock(long long* o) {
  long long t0 = clock64(); unsigned long long g0; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  while (clock64() - t0 < 200000000LL) {}
  long long t1 = clock64(); unsigned long long g1; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  o[0] = t1 - t0; o[1] = (long long)(g1 - g0);
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  int nsm = p.multiProcessorCount;
  printf("device %s sms %d cc %d.%d\n", p.name, nsm, p.major, p.minor);
  const int threads = 256, blocks = nsm * 8, iters = 4096;
  float* out; double* dout; long long* clk;
  cudaMalloc(&out, sizeof(float) * threads * blocks);
  cudaMalloc(&dout, sizeof(double) * threads * blocks);
  cudaMalloc(&clk, 2 * sizeof(long long));
  k_clock<<<1, 1>>>(clk); cudaDeviceSynchronize();
  long long hc[2]; cudaMemcpy(hc, clk, sizeof(hc), cudaMemcpyDeviceToHost);
  double mhz = (double)hc[0] / (double)hc[1] * 1e3;
  printf("sm clock during spin: %.1f MHz\n", mhz);
  const char* names[] = {"sin.approx", "ex2.approx", "ffma", "i2f(+lop)", "rsqrt.approx", "__sincosf(+fadd)"};
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int kind = 0; kind < 7; ++kind) {
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0);
      switch (kind) {
        case 0: k_probe<0><<<blocks, threads>>>(out, iters, 0.5f); break;
        case 1: k_probe<1><<<blocks, threads>>>(out, iters, 0.5f); break;
        case 2: k_probe<2><<<blocks, threads>>>(out, iters, 0.5f); break;
        case 3: k_probe<3><<<blocks, threads>>>(out, iters, 0.5f); break;
        case 4: k_probe<4><<<blocks, threads>>>(out, iters, 0.5f); break;
        case 5: k_probe<5><<<blocks, threads>>>(out, iters, 0.5f); break;
        case 6: k_dfma<<<blocks, threads>>>(dout, iters / 8, 0.5); break;
      }
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      double ops = (double)blocks * threads * (kind == 6 ? iters / 8 : iters) * CH;
      double rate = ops / (ms * 1e-3);
      if (rep == 2) printf("%-18s %8.3f ms  %10.1f Gop/s  %6.2f op/clk/SM (at %.0f MHz)\n",
                           kind == 6 ? "dfma" : names[kind], ms, rate * 1e-9, rate / (nsm * mhz * 1e6), mhz);
    }
  }
  cudaError_t err = cudaGetLastError();
  printf("status: %s\n", cudaGetErrorString(err));
  return err == cudaSuccess ? 0 : 1;
}
