// Measured throughput of the FP64 and FP32 fused multiply-add pipes (FP32 also in packed pairs).
//
// The multipole interactions are bound by arithmetic, not by memory, so their roofline is the
// rate at which the GPU retires fused multiply-adds of the kernel's precision.  This file measures
// that rate on the device at hand: every thread of a fully occupied grid runs independent FMA
// chains long enough (tens of milliseconds per launch) for launch overhead to vanish, and the
// fastest of a few launches, timed with CUDA events, gives FMAs per second.  A flop count of 2 per
// FMA makes it comparable with the algorithmic flop counts of the interaction kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "../../include/octo_fmm.h"

// records the calling thread's error message (fmm.cu) and returns the code
int fmm_record_error(int code, const char* msg);

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;  // 2048 threads: every warp slot of an SM
constexpr int kChains = 8;       // independent chains per thread (latency x issue rate covered)
constexpr int kUnroll = 16;      // FMAs per chain per loop trip

// v <- v a + b on kChains chains; a = 1 - eps and b = eps keep every value near 1 (no overflow,
// no subnormals).  The per-thread sums are stored, so no chain can be removed.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(int trips, T a, T b, T* __restrict__ out) {
  T v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = T(1) + T(k + (threadIdx.x & 7)) * b;
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) v[k] = fma(v[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k];
  out[size_t(blockIdx.x) * kThreads + threadIdx.x] = s;
}

// The same chains on packed FP32 pairs: one fma.rn.f32x2 instruction (sm_100 and later) performs
// two FP32 fused multiply-adds, so this kernel issues half the instructions of k_fma_rate<float>
// for the same arithmetic, and measures whether the packed form retires FMAs faster.
struct Packed2 {};
__global__ void __launch_bounds__(kThreads) k_fma2_rate(int trips, float a, float b, float* __restrict__ out) {
  float2 v[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    v[k] = make_float2(1.0f + float(k + (threadIdx.x & 7)) * b, 1.0f + float(k + 8 + (threadIdx.x & 7)) * b);
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) v[k] = __ffma2_rn(v[k], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k].x + v[k].y;
  out[size_t(blockIdx.x) * kThreads + threadIdx.x] = s;
}

template <typename T>
int measure(int reps, double* tflops, double* ms_out, cudaStream_t st) {
  constexpr bool kPacked = std::is_same<T, Packed2>::value;
  using E = typename std::conditional<kPacked, float, T>::type;  // element type
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fmm_record_error(FMM_ERR_CUDA, "fma rate: no current device");
  const int blocks = sms * kBlocksPerSm;
  E* out = nullptr;
  if (cudaMalloc(&out, sizeof(E) * size_t(blocks) * kThreads) != cudaSuccess)
    return fmm_record_error(FMM_ERR_NOMEM, "fma rate: device allocation failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FMM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FMM_ERR_CUDA;
  const E a = E(1) - E(1.0 / 4096), b = E(1.0 / 4096);
  auto time_one = [&](int trips, float* ms) -> int {
    if (cudaEventRecord(e0, st) != cudaSuccess) return FMM_ERR_CUDA;
    if constexpr (kPacked) k_fma2_rate<<<blocks, kThreads, 0, st>>>(trips, a, b, out);
    else k_fma_rate<E><<<blocks, kThreads, 0, st>>>(trips, a, b, out);
    if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return FMM_ERR_CUDA;
    return FMM_OK;
  };
  // calibrate the trip count to about 40 ms per launch, then keep the fastest of `reps` launches
  int trips = 16;
  float ms = 0.0f;
  for (int k = 0; rc == FMM_OK && k < 24; ++k) {
    rc = time_one(trips, &ms);
    if (rc || ms >= 20.0f) break;
    const double grow = ms > 0.5f ? 40.0 / ms : 16.0;
    trips = int(std::min(double(trips) * grow, 1e8));
  }
  double best = 0.0, best_ms = 0.0;
  for (int r = 0; rc == FMM_OK && r < reps; ++r) {
    rc = time_one(trips, &ms);
    const double fmas = double(blocks) * kThreads * kChains * kUnroll * double(trips) * (kPacked ? 2 : 1);
    const double rate = 2.0 * fmas / (double(ms) * 1e-3) / 1e12;
    if (rc == FMM_OK && rate > best) {
      best = rate;
      best_ms = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) return fmm_record_error(rc, "fma rate: a CUDA launch, event or synchronisation failed");
  *tflops = best;
  if (ms_out) *ms_out = best_ms;
  return FMM_OK;
}

}  // namespace

extern "C" int fmm_measure_fma_rate(int bits, int reps, double* tflops, double* ms_per_launch,
                                    void* stream) {
  if ((bits != 32 && bits != 64 && bits != FMM_FMA_F32X2) || reps < 1 || !tflops)
    return fmm_record_error(FMM_ERR_ARG,
                            "fma rate: bits must be 32, 64 or FMM_FMA_F32X2, reps >= 1, tflops not null");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (bits == 64) return measure<double>(reps, tflops, ms_per_launch, st);
  if (bits == 32) return measure<float>(reps, tflops, ms_per_launch, st);
  return measure<Packed2>(reps, tflops, ms_per_launch, st);
}
