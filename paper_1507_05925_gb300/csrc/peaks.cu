// Measured arithmetic peaks of the current GPU, the denominators of the
// pair-sum rooflines (the pair sums run on the FP32 FMA pipe, the MUFU
// reciprocal unit and, for FP64 solves, the FP64 pipe; none of them is a
// tensor-core or memory-bound kernel).
//
// Each kernel runs independent dependency chains per thread (enough of them,
// and enough warps per SM, that latency never limits issue), all SMs busy
// (4 CTAs of 256 threads per SM), timed with CUDA events, the fastest of five
// runs after two warm-ups.  A sum of the chains is written conditionally so
// that nothing is optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/bie2d.h"
#include "bie_internal.cuh"

namespace bie {
namespace {

constexpr int kPT = 256;     // threads per CTA
constexpr int kChains = 8;   // independent chains per thread
constexpr int kUnroll = 16;  // operations per chain per loop trip

__global__ void __launch_bounds__(kPT) k_peak_ffma(float* out, int iters, float b) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], b, 1e-7f);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.2345f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kPT) k_peak_ffma2(float* out, int iters, float b) {
  float2 a[kChains / 2];
  const float2 bb = make_float2(b, b), cc = make_float2(1e-7f, 1e-7f);
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) a[c] = make_float2(1e-3f * (threadIdx.x + c), 2e-3f * c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains / 2; ++c) a[c] = __ffma2_rn(a[c], bb, cc);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) s += a[c].x + a[c].y;
  if (s == -1.2345f) out[blockIdx.x] = s;
}

// volatile, and an add between reciprocals, so that rcp(rcp(x)) is never folded
__device__ __forceinline__ float rcp_kept(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__global__ void __launch_bounds__(kPT) k_peak_mufu(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = rcp_kept(a[c] + 0.5f);  // x -> 1/(x + 1/2): nothing folds
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.2345f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kPT) k_peak_dfma(double* out, int iters, double b) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, 1e-13);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.2345) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace bie

using namespace bie;

extern "C" int bie_measure_alu_peaks(int device, double* out) {
  if (!out) return BIE_ERR_INVALID;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  int sms = 0;
  double* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BIE_OK;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&buf, 4096 * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = BIE_ERR_CUDA;
  }
  const int grid = 4 * sms;
  const double threads = (double)grid * kPT;
  // operations per thread per loop trip (one lane operation each; FFMA2: two)
  const double per_trip = (double)kUnroll * kChains;
  auto best_ms = [&](auto launch) -> double {
    double best = 1e300;
    for (int r = 0; r < 7; ++r) {
      cudaEventRecord(e0);
      launch();
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r >= 2) best = std::min(best, (double)ms);
    }
    return best;
  };
  if (rc == BIE_OK) {
    float* fb = reinterpret_cast<float*>(buf);
    const int it_f = 4096, it_m = 512, it_d = 64;
    const double t_f = best_ms([&] { k_peak_ffma<<<grid, kPT>>>(fb, it_f, 1.0000001f); });
    const double t_f2 = best_ms([&] { k_peak_ffma2<<<grid, kPT>>>(fb, it_f, 1.0000001f); });
    const double t_m = best_ms([&] { k_peak_mufu<<<grid, kPT>>>(fb, it_m); });
    const double t_d = best_ms([&] { k_peak_dfma<<<grid, kPT>>>(buf, it_d, 1.0000000001); });
    note_launches(28);
    if (t_f <= 0 || t_f2 <= 0 || t_m <= 0 || t_d <= 0 || cudaGetLastError() != cudaSuccess) {
      rc = BIE_ERR_CUDA;
    } else {
      out[0] = 2.0 * threads * it_f * per_trip / (t_f * 1e-3) / 1e12;   // FFMA, TFLOP/s
      out[1] = 2.0 * threads * it_f * per_trip / (t_f2 * 1e-3) / 1e12;  // FFMA2, TFLOP/s
      out[2] = threads * it_m * per_trip / (t_m * 1e-3) / 1e12;         // MUFU rcp (+ one FADD), T op/s
      out[3] = 2.0 * threads * it_d * per_trip / (t_d * 1e-3) / 1e12;   // DFMA, TFLOP/s
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  cudaSetDevice(prev);
  return rc;
}
