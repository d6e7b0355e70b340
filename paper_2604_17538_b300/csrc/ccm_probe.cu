// Throughput probes for the ALU roofline of the contact kernels: FP32 FMA
// (scalar and packed f32x2) and the SFU's ex2.approx, each timed with CUDA
// events over a grid that fills every SM.
#include <cuda_runtime.h>

#include "../../include/ccm.h"

namespace ccm {

constexpr int kProbeIters = 4096;

__global__ void probe_ffma(float* out, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
  float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
  for (int i = 0; i < kProbeIters; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  if (x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7 == 12345.f) out[0] = x0;
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long x, unsigned long long a,
                                                   unsigned long long b) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(x), "l"(a), "l"(b));
  return d;
}

__global__ void probe_ffma2(float* out, float a, float b) {
  const unsigned long long A =
      ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
  const unsigned long long B =
      ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
  unsigned long long x[8];
  for (int k = 0; k < 8; ++k) x[k] = (unsigned long long)(threadIdx.x + k) * 0x100000001ull;
  for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma2(x[k], A, B);
  }
  unsigned long long s = 0;
  for (int k = 0; k < 8; ++k) s ^= x[k];
  if (s == 12345ull) out[0] = 1.f;
}

__global__ void probe_ex2(float* out) {
  float x0 = threadIdx.x * 1e-4f, x1 = x0 + .1f, x2 = x0 + .2f, x3 = x0 + .3f;
  float x4 = x0 + .4f, x5 = x0 + .5f, x6 = x0 + .6f, x7 = x0 + .7f;
  for (int i = 0; i < kProbeIters; ++i) {
    asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x0)); asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x1));
    asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x2)); asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x3));
    asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x4)); asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x5));
    asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x6)); asm("ex2.approx.ftz.f32 %0, %0;" : "+f"(x7));
    x0 = -x0; x1 = -x1; x2 = -x2; x3 = -x3; x4 = -x4; x5 = -x5; x6 = -x6; x7 = -x7;
  }
  if (x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7 == 12345.f) out[0] = x0;
}

}  // namespace ccm

using namespace ccm;

extern "C" ccm_status ccm_peak_probe(int device, double* ffma_tflops, double* ffma2_tflops,
                                     double* ex2_tops) {
  if (cudaSetDevice(device) != cudaSuccess) return CCM_ERR_INVALID;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return CCM_ERR_CUDA;
  const int blocks = prop.multiProcessorCount * 8, threads = 256;
  float* out = nullptr;
  if (cudaMalloc(&out, 16) != cudaSuccess) return CCM_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double n_thr = (double)blocks * threads;
  float best[3] = {1e30f, 1e30f, 1e30f};
  for (int rep = 0; rep < 4; ++rep) {
    for (int k = 0; k < 3; ++k) {
      cudaEventRecord(e0);
      if (k == 0) probe_ffma<<<blocks, threads>>>(out, 0.999f, 1e-3f);
      if (k == 1) probe_ffma2<<<blocks, threads>>>(out, 0.999f, 1e-3f);
      if (k == 2) probe_ex2<<<blocks, threads>>>(out);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best[k]) best[k] = ms;   // first round warms up
    }
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return CCM_ERR_CUDA;
  const double ops = n_thr * kProbeIters * 8;
  if (ffma_tflops) *ffma_tflops = 2.0 * ops / (best[0] * 1e-3) / 1e12;
  if (ffma2_tflops) *ffma2_tflops = 4.0 * ops / (best[1] * 1e-3) / 1e12;
  if (ex2_tops) *ex2_tops = ops / (best[2] * 1e-3) / 1e12;
  return CCM_OK;
}
