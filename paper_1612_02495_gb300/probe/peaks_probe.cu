// Throughput probes of the GB300 units the stencil kernels use: FP64 and FP32
// issue rates for different operand sources, the KS update's exact FP64
// instruction mix, shared-memory load bandwidth, barrier cost and launch
// latency.  Prints one JSON object.  Every loop has a fixed trip count.
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x)                                                                              \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) {                                                               \
      printf("{\"error\": \"%s: %s\"}\n", #x, cudaGetErrorString(e_));                      \
      return 1;                                                                            \
    }                                                                                      \
  } while (0)

// FP64 FMA with both other operands from kernel parameters (constant bank)
__global__ void k_dfma_const(double* out, int iters, double a, double b) {
  double x[4];
  for (int h = 0; h < 4; ++h) x[h] = threadIdx.x + h;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int h = 0; h < 4; ++h) x[h] = __fma_rn(x[h], a, b);
  if (x[0] + x[1] + x[2] + x[3] == 12345.0) out[0] = 1;
}
// FP64 FMA with three vector-register operands
__global__ void k_dfma_reg(double* out, int iters) {
  double x[4], y[4];
  for (int h = 0; h < 4; ++h) x[h] = threadIdx.x + h, y[h] = 1e-7 * (h + 1);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int h = 0; h < 4; ++h) x[h] = __fma_rn(x[h], y[h], x[(h + 1) & 3]);
  if (x[0] + x[1] + x[2] + x[3] == 12345.0) out[0] = 1;
}
__global__ void k_dadd_reg(double* out, int iters) {
  double x[4], y[4];
  for (int h = 0; h < 4; ++h) x[h] = threadIdx.x + h, y[h] = 1e-7 * (h + 1);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int h = 0; h < 4; ++h) x[h] = __dadd_rn(x[h], y[h]);
  if (x[0] + x[1] + x[2] + x[3] == 12345.0) out[0] = 1;
}
// the KS update's 11 FP64 instructions (2 add, 2 mul, 7 fma), 4 independent chains
__device__ __forceinline__ double ks_mix(double a, double b, double c, double d, double e, double ca, double c2,
                                         double c4, double mdt) {
  const double sp1 = __dadd_rn(d, b), sp2 = __dadd_rn(e, a);
  const double nl = __fma_rn(d, d, -__dmul_rn(b, b));
  const double d2 = __fma_rn(-2.0, c, sp1);
  const double d4 = __fma_rn(6.0, c, __fma_rn(-4.0, sp1, sp2));
  return __fma_rn(mdt, __fma_rn(c4, d4, __fma_rn(c2, d2, __dmul_rn(ca, nl))), c);
}
__global__ void k_ks_mix(double* out, int iters, double ca, double c2, double c4, double mdt) {
  double v[4][5];
  for (int h = 0; h < 4; ++h)
    for (int k = 0; k < 5; ++k) v[h][k] = 1.0 + 1e-3 * (threadIdx.x + h + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double r = ks_mix(v[h][0], v[h][1], v[h][2], v[h][3], v[h][4], ca, c2, c4, mdt);
      v[h][0] = v[h][1], v[h][1] = v[h][2], v[h][2] = v[h][3], v[h][3] = v[h][4], v[h][4] = r;
    }
  if (v[0][4] + v[1][4] + v[2][4] + v[3][4] == 12345.0) out[0] = 1;
}
__global__ void k_ffma_reg(float* out, int iters) {
  float x[8], y[8];
  for (int h = 0; h < 8; ++h) x[h] = threadIdx.x + h, y[h] = 1e-7f * (h + 1);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int h = 0; h < 8; ++h) x[h] = __fmaf_rn(x[h], y[h], x[(h + 1) & 7]);
  float s = 0;
  for (int h = 0; h < 8; ++h) s += x[h];
  if (s == 12345.f) out[0] = s;
}
// shared-memory 32-bit loads, conflict-free, summed with integer adds
__global__ void k_smem(int* out, int iters) {
  __shared__ int sm[4096];
  for (int i = threadIdx.x; i < 4096; i += blockDim.x) sm[i] = i;
  __syncthreads();
  int acc = 0, idx = threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += sm[(idx + k * 256) & 4095];
    idx = (idx + 32) & 4095;
  }
  if (acc == -1) out[0] = acc;
}
__global__ void k_sync(float* out, int iters) {
  float a = threadIdx.x;
  for (int i = 0; i < iters; ++i) {
    a = a * 1.0001f;
    __syncthreads();
  }
  if (a == -1.f) out[0] = a;
}
__global__ void k_empty(float* out) {
  if (threadIdx.x == 9999) out[0] = 1.f;
}

// cycles one warp FP64 FMA holds the SMSP when only `active` lanes run it (one
// warp alone on an SM, 4 independent chains): masked lanes may or may not be free
__global__ void k_dfma_lanes(int active, int iters, double a, double b, double* out, long long* cyc) {
  const int lane = threadIdx.x;
  double x0 = lane, x1 = lane + 1, x2 = lane + 2, x3 = lane + 3;
  const long long t0 = clock64();
  if (lane < active)
    for (int i = 0; i < iters; ++i) {
      x0 = __fma_rn(x0, a, b);
      x1 = __fma_rn(x1, a, b);
      x2 = __fma_rn(x2, a, b);
      x3 = __fma_rn(x3, a, b);
    }
  __syncwarp();
  const long long t1 = clock64();
  out[lane] = x0 + x1 + x2 + x3;
  if (lane == 0) *cyc = t1 - t0;
}

int main() {
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, 0));
  const int sms = p.multiProcessorCount;
  int clk_khz = 0;
  CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0));
  double* d;
  CK(cudaMalloc(&d, 1024));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float ms = 0;
  const int blocks = sms * 8, thr = 256;
  auto best = [&](auto launch) {
    float m = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(a);
      launch();
      cudaEventRecord(b);
      cudaEventSynchronize(b);
      float t;
      cudaEventElapsedTime(&t, a, b);
      if (t < m) m = t;
    }
    return m;
  };
  const double thr_total = (double)blocks * thr;
  printf("{\"device\": \"%s\", \"sms\": %d, \"clock_mhz_attr\": %.0f", p.name, sms, clk_khz / 1e3);
  ms = best([&] { k_dfma_const<<<blocks, thr>>>(d, 400, 0.999999, 1e-7); });
  printf(", \"fp64_fma_const_operands_per_s\": %.4e", thr_total * 400 * 32 / (ms * 1e-3));
  ms = best([&] { k_dfma_reg<<<blocks, thr>>>(d, 400); });
  printf(", \"fp64_fma_reg_operands_per_s\": %.4e", thr_total * 400 * 32 / (ms * 1e-3));
  ms = best([&] { k_dadd_reg<<<blocks, thr>>>(d, 400); });
  printf(", \"fp64_add_reg_operands_per_s\": %.4e", thr_total * 400 * 32 / (ms * 1e-3));
  ms = best([&] { k_ks_mix<<<blocks, thr>>>(d, 400, 0.3, 1.6, 2.6, -0.005); });
  printf(", \"fp64_ks_mix_instr_per_s\": %.4e", thr_total * 400 * 4 * 11 / (ms * 1e-3));
  ms = best([&] { k_ffma_reg<<<blocks, thr>>>((float*)d, 2000); });
  printf(", \"fp32_fma_reg_operands_per_s\": %.4e", thr_total * 2000 * 64 / (ms * 1e-3));
  ms = best([&] { k_smem<<<blocks, thr>>>((int*)d, 4000); });
  printf(", \"smem_load_bytes_per_s\": %.4e", thr_total * 4000 * 8 * 4 / (ms * 1e-3));
  for (int bpsm : {1, 4}) {
    ms = best([&] { k_sync<<<sms * bpsm, 256>>>((float*)d, 20000); });
    printf(", \"syncthreads_ns_256thr_%dblk_per_sm\": %.2f", bpsm, ms * 1e6 / 20000);
  }
  cudaStream_t s;
  CK(cudaStreamCreate(&s));
  for (int i = 0; i < 50; ++i) k_empty<<<1, 32, 0, s>>>((float*)d);
  CK(cudaStreamSynchronize(s));
  cudaEventRecord(a, s);
  for (int i = 0; i < 2000; ++i) k_empty<<<sms, 256, 0, s>>>((float*)d);
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b);
  printf(", \"stream_launch_us\": %.3f", ms * 1e3 / 2000);
  cudaGraph_t g;
  cudaGraphExec_t ge;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < 1000; ++i) k_empty<<<sms, 256, 0, s>>>((float*)d);
  CK(cudaStreamEndCapture(s, &g));
  CK(cudaGraphInstantiate(&ge, g, 0));
  CK(cudaGraphLaunch(ge, s));
  CK(cudaStreamSynchronize(s));
  cudaEventRecord(a, s);
  for (int i = 0; i < 4; ++i) cudaGraphLaunch(ge, s);
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b);
  printf(", \"graph_node_us\": %.3f", ms * 1e3 / 4000);
  long long* cyc;
  CK(cudaMalloc(&cyc, sizeof(long long)));
  for (int active : {32, 8, 1}) {
    long long c = 0;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
      k_dfma_lanes<<<1, 32>>>(active, 4096, 0.999999, 1e-9, d, cyc);
      CK(cudaMemcpy(&c, cyc, sizeof c, cudaMemcpyDeviceToHost));
    }
    printf(", \"fp64_fma_cycles_per_warp_instr_%d_lanes\": %.2f", active, (double)c / (4.0 * 4096));
  }
  printf("}\n");
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  return 0;
}
