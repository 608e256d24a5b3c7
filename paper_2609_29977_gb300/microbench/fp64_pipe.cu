// FP64 / FP32 pipe microbenchmark for the GB300 (sm_103a).
//
// Measures the rates the FP64 kernels are designed around: DFMA throughput
// with 32, 8 and 1 active lanes, FP32 FFMA throughput, the cost of the
// FP64 rsqrt / sqrt / divide and of double<->float conversion, DMMA
// (mma.sync m8n8k4 f64), and per-warp cycles per FP64 instruction (clock64)
// for 1..8 resident warps per SM. Every launch is in bounds and every loop
// is bounded.
//
// Build and run (one GPU):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_pipe fp64_pipe.cu && ./fp64_pipe
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("ERR %s line %d\n", cudaGetErrorString(e), __LINE__); return 1;}}while(0)

template<int ACTIVE>
__global__ void dfma_k(double* out, int iters, double a, double b) {
  int lane = threadIdx.x & 31;
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  if (lane < ACTIVE) {
    for (int i = 0; i < iters; ++i) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void ffma_k(float* out, int iters, float a, float b) {
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < iters; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void drsqrt_k(double* out, int iters) {
  double x0=threadIdx.x+1.5, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i = 0; i < iters; ++i) { x0 = rsqrt(x0)+2.0; x1 = rsqrt(x1)+2.0; x2 = rsqrt(x2)+2.0; x3 = rsqrt(x3)+2.0; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3;
}
__global__ void dsqrt_k(double* out, int iters) {
  double x0=threadIdx.x+1.5, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i = 0; i < iters; ++i) { x0 = sqrt(x0)+2.0; x1 = sqrt(x1)+2.0; x2 = sqrt(x2)+2.0; x3 = sqrt(x3)+2.0; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3;
}
__global__ void ddiv_k(double* out, int iters) {
  double x0=threadIdx.x+1.5, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i = 0; i < iters; ++i) { x0 = 1.0/x0+2.0; x1 = 1.0/x1+2.0; x2 = 1.0/x2+2.0; x3 = 1.0/x3+2.0; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3;
}
__global__ void f2f_k(double* out, int iters) {
  double x0=threadIdx.x+1.5, x1=x0+1, x2=x0+2, x3=x0+3;
  for (int i = 0; i < iters; ++i) {
    x0 = (double)((float)x0 * 1.0001f); x1 = (double)((float)x1 * 1.0001f);
    x2 = (double)((float)x2 * 1.0001f); x3 = (double)((float)x3 * 1.0001f); }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3;
}
__global__ void dmma_k(double* out, int iters) {
  double a = threadIdx.x * 1e-3, b = 1.0 - threadIdx.x * 1e-4;
  double c0=0, c1=0, d0=0, d1=0, e0=0, e1=0, f0=0, f1=0;
  for (int i = 0; i < iters; ++i) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(d0), "+d"(d1) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(e0), "+d"(e1) : "d"(a), "d"(b));
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(f0), "+d"(f1) : "d"(a), "d"(b));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0+c1+d0+d1+e0+e1+f0+f1;
}


// Even warps run DFMA chains, odd warps DMMA chains (MODE 0), or only the
// even (MODE 1) or only the odd ones (MODE 2): if the two share one pipe,
// MODE 0 takes the sum of the MODE 1 and MODE 2 times; if not, their maximum.
template <int MODE>
__global__ void mix_k(double* out, int iters, double a, double b) {
  const int w = threadIdx.x >> 5;
  double acc = 0.0;
  if ((w & 1) == 0) {
    if (MODE != 2) {
      double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
      for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
      }
      acc = x0+x1+x2+x3+x4+x5+x6+x7;
    }
  } else if (MODE != 1) {
    double ma = threadIdx.x * 1e-3, mb = 1.0 - threadIdx.x * 1e-4;
    double c0=0, c1=0, d0=0, d1=0, e0=0, e1=0, f0=0, f1=0;
    for (int i = 0; i < 2 * iters; ++i) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c0), "+d"(c1) : "d"(ma), "d"(mb));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(d0), "+d"(d1) : "d"(ma), "d"(mb));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(e0), "+d"(e1) : "d"(ma), "d"(mb));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(f0), "+d"(f1) : "d"(ma), "d"(mb));
    }
    acc = c0+c1+d0+d1+e0+e1+f0+f1;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void dep_chain(double* out, long long* cyc, int iters, double a, double b) {
  double x = threadIdx.x;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) { x = fma(x, a, b); x = fma(x, a, b); x = fma(x, a, b); x = fma(x, a, b); }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
__global__ void ind8(double* out, long long* cyc, int iters, double a, double b) {
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3+x4+x5+x6+x7;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
__global__ void rsqrt_chain(double* out, long long* cyc, int iters) {
  double x = threadIdx.x + 1.5;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) { x = rsqrt(x) + 1.5; }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
__global__ void f2f_chain(double* out, long long* cyc, int iters) {
  double x = threadIdx.x + 1.5;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    float f = __double2float_rn(x);
    f = fmaf(f, 0.999f, 0.5f);
    x = (double)f;
    x = __longlong_as_double(__double_as_longlong(x) ^ 1ll);
  }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}
__global__ void f2f_thr(double* out, long long* cyc, int iters) {
  double x0 = threadIdx.x + 1.5, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    float f0 = __double2float_rn(x0), f1 = __double2float_rn(x1), f2 = __double2float_rn(x2), f3 = __double2float_rn(x3);
    x0 = __longlong_as_double(__double_as_longlong((double)f0) ^ 1ll);
    x1 = __longlong_as_double(__double_as_longlong((double)f1) ^ 1ll);
    x2 = __longlong_as_double(__double_as_longlong((double)f2) ^ 1ll);
    x3 = __longlong_as_double(__double_as_longlong((double)f3) ^ 1ll);
  }
  long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0+x1+x2+x3;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

static int part_throughput() {
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, 0));
  printf("device %s SMs %d cc %d.%d l2 %d MB smemPerBlockOptin %zu regsPerSM %d\n", p.name, p.multiProcessorCount, p.major, p.minor, p.l2CacheSize>>20, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor);
  int sms = p.multiProcessorCount;
  int blocks = sms * 8, threads = 256;
  size_t n = (size_t)blocks * threads;
  double* dout; float* fout;
  CK(cudaMalloc(&dout, n * sizeof(double))); CK(cudaMalloc(&fout, n * sizeof(float)));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  float ms;
  auto run = [&](const char* name, auto launch, double ops_per_thread_iter, int iters, double active_frac) {
    launch(iters / 10); cudaDeviceSynchronize();
    cudaEventRecord(e0); launch(iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    double ops = ops_per_thread_iter * iters * n * active_frac;
    double wi = ops_per_thread_iter * iters * (n / 32.0);
    printf("%-12s %8.3f ms  lane-ops/s %.4e  warp-instr/s %.4e  per-SM-clk(@1.9GHz) lane-ops %.3f\n", name, ms, ops / (ms * 1e-3), wi / (ms * 1e-3), ops / (ms * 1e-3) / sms / 1.9e9);
  };
  int it = 4000;
  run("dfma32", [&](int i){ dfma_k<32><<<blocks, threads>>>(dout, i, 1.0000001, 1e-9); }, 8, it, 1.0);
  run("dfma8", [&](int i){ dfma_k<8><<<blocks, threads>>>(dout, i, 1.0000001, 1e-9); }, 8, it, 0.25);
  run("dfma1", [&](int i){ dfma_k<1><<<blocks, threads>>>(dout, i, 1.0000001, 1e-9); }, 8, it, 1.0/32);
  run("ffma32", [&](int i){ ffma_k<<<blocks, threads>>>(fout, i, 1.0000001f, 1e-9f); }, 8, it * 16, 1.0);
  run("drsqrt", [&](int i){ drsqrt_k<<<blocks, threads>>>(dout, i); }, 4, it / 8, 1.0);
  run("dsqrt", [&](int i){ dsqrt_k<<<blocks, threads>>>(dout, i); }, 4, it / 8, 1.0);
  run("ddiv", [&](int i){ ddiv_k<<<blocks, threads>>>(dout, i); }, 4, it / 8, 1.0);
  run("f2f", [&](int i){ f2f_k<<<blocks, threads>>>(dout, i); }, 4, it, 1.0);
  // dmma: 8x8x4 per warp-instr = 256 FMA = 512 flop per warp; report as lane-ops = 8 FMA per thread per mma
  run("dmma", [&](int i){ dmma_k<<<blocks, threads>>>(dout, i); }, 4 * 8, it / 4, 1.0);
  // DFMA and DMMA side by side (8 DFMA vs 8 DMMA warp-instructions per warp and iteration)
  run("mix:dfma+dmma", [&](int i){ mix_k<0><<<blocks, threads>>>(dout, i, 1.0000001, 1e-9); }, 8, it / 4, 1.0);
  run("mix:dfma only", [&](int i){ mix_k<1><<<blocks, threads>>>(dout, i, 1.0000001, 1e-9); }, 8, it / 4, 1.0);
  run("mix:dmma only", [&](int i){ mix_k<2><<<blocks, threads>>>(dout, i, 1.0000001, 1e-9); }, 8, it / 4, 1.0);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  printf("done\n");
  return 0;
}

static int part_latency() {
  int sms = 152;
  double* dout; long long* cyc; long long h[2048];
  CK(cudaMalloc(&dout, 2048 * 1024 * sizeof(double))); CK(cudaMalloc(&cyc, 2048 * sizeof(long long)));
  auto report = [&](const char* name, int blocks, double instr_per_thread) {
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(h, cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost));
    double s = 0; for (int i = 0; i < blocks; ++i) s += h[i];
    printf("%-36s cycles/instr per warp %.2f\n", name, s / blocks / instr_per_thread);
    return 0;
  };
  int it = 2000;
  dep_chain<<<sms, 32>>>(dout, cyc, it, 1.0000001, 1e-9); report("dep DFMA chain, 1 warp/SM", sms, 4.0 * it);
  ind8<<<sms, 32>>>(dout, cyc, it, 1.0000001, 1e-9); report("8 indep DFMA, 1 warp/SM", sms, 8.0 * it);
  ind8<<<sms, 64>>>(dout, cyc, it, 1.0000001, 1e-9); report("8 indep DFMA, 2 warps/SM", sms, 8.0 * it);
  ind8<<<sms, 128>>>(dout, cyc, it, 1.0000001, 1e-9); report("8 indep DFMA, 4 warps/SM", sms, 8.0 * it);
  ind8<<<sms, 256>>>(dout, cyc, it, 1.0000001, 1e-9); report("8 indep DFMA, 8 warps/SM", sms, 8.0 * it);
  dep_chain<<<sms, 128>>>(dout, cyc, it, 1.0000001, 1e-9); report("dep DFMA chain, 4 warps/SM", sms, 4.0 * it);
  rsqrt_chain<<<sms, 32>>>(dout, cyc, it / 4); report("rsqrt(+dadd) chain, 1 warp/SM", sms, it / 4);
  rsqrt_chain<<<sms, 128>>>(dout, cyc, it / 4); report("rsqrt(+dadd) chain, 4 warps/SM", sms, it / 4);
  f2f_chain<<<sms, 32>>>(dout, cyc, it); report("f2f d->f->d chain, 1 warp/SM", sms, it);
  f2f_thr<<<sms, 256>>>(dout, cyc, it); report("f2f pairs indep, 8 warps/SM (per pair)", sms, 4.0 * it);
  CK(cudaGetLastError());
  printf("done\n");
  return 0;
}

int main() {
  if (part_throughput()) return 1;
  return part_latency();
}
