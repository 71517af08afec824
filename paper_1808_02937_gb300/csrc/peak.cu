// ALU peak measurement (measurement support for the roofline fractions the
// benchmark reports; the paper has no counterpart): independent fused
// multiply-add chains in FP64 or FP32, timed with CUDA events, on every SM.
// Nothing else runs on the stream; clocks are whatever the GPU runs at.
#include "hfsem_internal.h"

namespace hf {
namespace {

constexpr int kChains = 8;       // independent FMA chains per thread
constexpr int kPeakThreads = 256;

template <class T>
__global__ void k_fma_peak(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)12345.678) out[blockIdx.x] = s;   // keeps the chains live
}

template <class T>
double run(int iters, int blocks, float* ms_out) {
  DevBuf<T> out;
  out.alloc(blocks);
  cudaEvent_t e0, e1;
  HF_CHECK(cudaEventCreate(&e0));
  HF_CHECK(cudaEventCreate(&e1));
  k_fma_peak<T><<<blocks, kPeakThreads>>>(out.p, 16, (T)0.999999, (T)1e-7);   // warm-up
  HF_LAUNCH_CHECK();
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    HF_CHECK(cudaEventRecord(e0));
    k_fma_peak<T><<<blocks, kPeakThreads>>>(out.p, iters, (T)0.999999, (T)1e-7);
    HF_LAUNCH_CHECK();
    HF_CHECK(cudaEventRecord(e1));
    HF_CHECK(cudaEventSynchronize(e1));
    float ms = 0;
    HF_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
  return flops / (best * 1e-3) / 1e12;
}

}  // namespace
}  // namespace hf

using namespace hf;

extern "C" int hfsem_alu_peak(int32_t kind, double* tflops, double* ms, int32_t* sms) {
  try {
    if (!tflops || (kind != 0 && kind != 1)) throw Error(HFSEM_ERR_INVALID_ARG, "kind 0 (FP64) or 1 (FP32)");
    int dev = 0, nsm = 0;
    HF_CHECK(cudaGetDevice(&dev));
    HF_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * 8;               // 64 warps per SM
    float t = 0;
    *tflops = kind == 0 ? run<double>(1 << 13, blocks, &t) : run<float>(1 << 16, blocks, &t);
    if (ms) *ms = t;
    if (sms) *sms = nsm;
    return HFSEM_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.code;
  } catch (...) {
    set_last_error("unknown error");
    return HFSEM_ERR_DEVICE;
  }
}
