// pipe_peaks.cu -- measured peaks of the arithmetic pipes the hot path is
// bound by, for the roofline denominators of bench.py: float32 FMA (the
// fused L2P + P2P evaluation), the paired float32 FMA (the same evaluation's
// two-rays-per-instruction loop), float64 FMA (M2M, M2L, L2L) and the MUFU
// reciprocal (one per ray-star pair).
//
// Each kernel runs independent dependency chains per thread (enough to hide
// the pipe latency), one block of 256 threads per SM slot, over a grid of
// SMs x 8 blocks; the result is the work done over the CUDA-event time of
// the best of several launches.  The chains' final values are stored so that
// nothing is optimised away.  Output: one JSON line.
//
// Build and run (bench.py --measure-peaks does both):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_peaks pipe_peaks.cu
//   ./pipe_peaks
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#define CK(x)                                                              \
  do {                                                                     \
    cudaError_t e_ = (x);                                                  \
    if (e_ != cudaSuccess) {                                               \
      std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));        \
      std::exit(1);                                                        \
    }                                                                      \
  } while (0)

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void k_ffma(float* out, float a, float b) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3f + c;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma2(float* out, float a, float b) {
  float2 v[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = make_float2(threadIdx.x * 1e-3f + c, c * 0.5f);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c].x + v[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double* out, double a, double b) {
  double v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3 + c;
  for (int it = 0; it < kIters / 16; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rcp(float* out, float a) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = 1.0f + threadIdx.x * 1e-3f + c;
  for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float r;
      asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v[c]));
      v[c] = r + a;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class F>
float best_ms(F launch, int reps) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  launch();  // warm-up
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    CK(cudaEventRecord(e0));
    launch();
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return best;
}

int main() {
  int dev = 0, sms = 0, clk = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
  const int blocks = sms * 8;
  const double threads = (double)blocks * kThreads;
  float* of = nullptr;
  double* od = nullptr;
  CK(cudaMalloc(&of, sizeof(float) * (size_t)blocks * kThreads));
  CK(cudaMalloc(&od, sizeof(double) * (size_t)blocks * kThreads));
  const int reps = 5;
  const float t_ffma = best_ms([&] { k_ffma<<<blocks, kThreads>>>(of, 0.999f, 1e-3f); }, reps);
  const float t_ffma2 = best_ms([&] { k_ffma2<<<blocks, kThreads>>>(of, 0.999f, 1e-3f); }, reps);
  const float t_dfma = best_ms([&] { k_dfma<<<blocks, kThreads>>>(od, 0.999, 1e-3); }, reps);
  const float t_rcp = best_ms([&] { k_rcp<<<blocks, kThreads>>>(of, 1e-3f); }, reps);
  CK(cudaGetLastError());
  // flops: 2 per FMA (4 per paired FMA); reciprocals: 1 per rcp
  const double ffma = threads * kIters * kChains * 2.0 / (t_ffma * 1e-3) / 1e12;
  const double ffma2 = threads * kIters * kChains * 4.0 / (t_ffma2 * 1e-3) / 1e12;
  const double dfma = threads * (kIters / 16) * kChains * 2.0 / (t_dfma * 1e-3) / 1e12;
  const double rcp = threads * (kIters / 4) * kChains / (t_rcp * 1e-3) / 1e12;
  std::printf("{\"sms\": %d, \"clock_mhz_attr\": %.0f, \"ffma_tflops\": %.3f, "
              "\"ffma2_tflops\": %.3f, \"dfma_tflops\": %.4f, \"mufu_rcp_tops\": %.3f, "
              "\"ms\": {\"ffma\": %.4f, \"ffma2\": %.4f, \"dfma\": %.4f, \"rcp\": %.4f}}\n",
              sms, clk / 1000.0, ffma, ffma2, dfma, rcp, t_ffma, t_ffma2, t_dfma, t_rcp);
  CK(cudaFree(of));
  CK(cudaFree(od));
  return 0;
}
