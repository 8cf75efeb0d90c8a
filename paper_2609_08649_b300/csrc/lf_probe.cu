// Arithmetic-rate probes: the measured denominators of the lens-equation kernels' roofline
// (FP32 FMA issue, MUFU reciprocal square root, FP64 FMA).  Each kernel runs independent
// dependency chains per thread (enough to hide the pipes' latencies) over a grid that fills
// every SM, and the host times it with CUDA events.
#include "lf_internal.h"

namespace lf {

constexpr int LF_PROBE_ITERS = 2048;

__global__ void k_probe_fma(float* out, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
  float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
  for (int i = 0; i < LF_PROBE_ITERS; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
      x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// The same FMA chains on packed f32x2 operands (fma.rn.f32x2): each instruction does two lanes'
// work, so its lane-operation rate shows whether packing adds FP32 throughput or only saves
// issue slots.
__global__ void k_probe_fma2(float* out, float a, float b) {
  const float2 A = make_float2(a, a), B = make_float2(b, b);
  float2 x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = make_float2(threadIdx.x * 1e-3f + k, k + 0.5f);
  for (int i = 0; i < LF_PROBE_ITERS / 2; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = __ffma2_rn(x[k], A, B);
  }
  float r = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) r += x[k].x + x[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_probe_rsqrt(float* out, float a) {
  float x0 = threadIdx.x * 1e-3f + 1.f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
  float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
  for (int i = 0; i < LF_PROBE_ITERS / 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x0 = rsqrtf(x0 + a); x1 = rsqrtf(x1 + a); x2 = rsqrtf(x2 + a); x3 = rsqrtf(x3 + a);
      x4 = rsqrtf(x4 + a); x5 = rsqrtf(x5 + a); x6 = rsqrtf(x6 + a); x7 = rsqrtf(x7 + a);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_probe_dfma(double* out, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < LF_PROBE_ITERS / 32; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

// Failure-detection self-test: one thread arms an mbarrier for 16 bytes of bulk-copy
// transactions and issues no copy, so the phase can never complete; the bounded wait gives
// up after `polls` polls and records LF_DEVERR_TIMEOUT in the device error word, exactly as
// a staging wait of the lens kernels does.  Nothing asynchronous is in flight when the block
// exits.
__global__ void k_selftest_wait_timeout(uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16u);
    if (!mbar_wait(&bar, 0u, polls)) lf_flag_error(LF_DEVERR_TIMEOUT);
  }
}

}  // namespace lf

using namespace lf;

extern "C" lf_status lf_selftest_wait_timeout(uint32_t polls, void* stream) {
  if (polls < 1 || polls > 65536) return fail(LF_EINVAL, "polls must be in 1..65536");
  k_selftest_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(polls);
  LF_CUDA(cudaGetLastError());
  return LF_OK;
}

extern "C" lf_status lf_probe_alu(double* fp32_fma_per_s, double* mufu_rsqrt_per_s,
                                  double* fp64_fma_per_s, void* stream) {
  return lf_probe_alu2(fp32_fma_per_s, nullptr, mufu_rsqrt_per_s, fp64_fma_per_s, stream);
}

extern "C" lf_status lf_probe_alu2(double* fp32_fma_per_s, double* fp32_fma2_lanes_per_s,
                                   double* mufu_rsqrt_per_s, double* fp64_fma_per_s, void* stream) {
  if (!fp32_fma_per_s || !mufu_rsqrt_per_s || !fp64_fma_per_s) return fail(LF_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  LF_CUDA(cudaGetDevice(&dev));
  LF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256, blocks = nsm * 8;
  const size_t n = (size_t)threads * blocks;
  void* buf = nullptr;
  LF_CUDA(cudaMalloc(&buf, n * sizeof(double)));
  cudaEvent_t e0, e1;
  LF_CUDA(cudaEventCreate(&e0));
  LF_CUDA(cudaEventCreate(&e1));
  lf_status status = LF_OK;
  float ms = 0.f;
  auto timed = [&](auto launch, double ops, double* rate) {
    launch();                                                  // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess) {
      status = fail(LF_ECUDA, "probe kernel failed");
      return;
    }
    *rate = ops / (ms * 1e-3);
  };
  timed([&] { k_probe_fma<<<blocks, threads, 0, st>>>((float*)buf, 0.999f, 0.001f); },
        (double)n * LF_PROBE_ITERS * 64, fp32_fma_per_s);
  if (status == LF_OK && fp32_fma2_lanes_per_s)
    timed([&] { k_probe_fma2<<<blocks, threads, 0, st>>>((float*)buf, 0.999f, 0.001f); },
          (double)n * (LF_PROBE_ITERS / 2) * 128, fp32_fma2_lanes_per_s);
  if (status == LF_OK)
    timed([&] { k_probe_rsqrt<<<blocks, threads, 0, st>>>((float*)buf, 0.5f); },
          (double)n * (LF_PROBE_ITERS / 4) * 32, mufu_rsqrt_per_s);
  if (status == LF_OK)
    timed([&] { k_probe_dfma<<<blocks, threads, 0, st>>>((double*)buf, 0.999, 0.001); },
          (double)n * (LF_PROBE_ITERS / 32) * 32, fp64_fma_per_s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  return status;
}
