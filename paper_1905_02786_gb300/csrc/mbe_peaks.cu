// mbe_measure_peaks: arithmetic peaks of the device measured by this library
// (no counterpart in the paper).  The roofline of the FP64 contraction and of
// the FP32 vector arithmetic is quoted against these figures rather than
// nominal ones.
//
// Each probe kernel runs 8 independent fused multiply-add chains per thread
// (enough to cover the FMA latency) over a fixed number of steps, on a grid of
// 8 CTAs of 256 threads per SM; the chains are folded into one store per
// thread so that the compiler keeps them.  Timed with CUDA events on a
// private stream after one warm-up launch; the best of three launches counts.
#include "mbe_internal.cuh"

namespace {

constexpr int PK_THREADS = 256, PK_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_fma_probe(T a, T b, int steps, T* __restrict__ out) {
  T x[PK_CHAINS];
#pragma unroll
  for (int i = 0; i < PK_CHAINS; i++) x[i] = (T)(threadIdx.x + i);
  for (int s = 0; s < steps; s++) {
#pragma unroll
    for (int i = 0; i < PK_CHAINS; i++) x[i] = x[i] * a + b;
  }
  T acc = 0;
#pragma unroll
  for (int i = 0; i < PK_CHAINS; i++) acc += x[i];
  out[(int64_t)blockIdx.x * PK_THREADS + threadIdx.x] = acc;
}

template <typename T>
double probe(int nsm, int steps, cudaStream_t st) {
  const int grid = 8 * nsm;
  T* out = nullptr;
  CU_CHECK(cudaMalloc(&out, sizeof(T) * (size_t)grid * PK_THREADS));
  cudaEvent_t e0, e1;
  CU_CHECK(cudaEventCreate(&e0));
  CU_CHECK(cudaEventCreate(&e1));
  double best = 0.0;
  // a = 1 - 2^-20, b = 2^-10: the chains stay finite and non-trivial
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1024.0);
  for (int rep = 0; rep < 4; rep++) {
    CU_CHECK(cudaEventRecord(e0, st));
    k_fma_probe<T><<<grid, PK_THREADS, 0, st>>>(a, b, steps, out);
    CU_LAUNCH_CHECK();
    CU_CHECK(cudaEventRecord(e1, st));
    CU_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CU_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    const double flops = 2.0 * PK_CHAINS * (double)steps * grid * PK_THREADS;
    if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return best;
}

}  // namespace

extern "C" int mbe_measure_peaks(int device, double* fp64_tflops, double* fp32_tflops) {
  if (device < 0 || device >= MBE_MAX_DEVICES) return MBE_EINVAL;
  try {
    CU_CHECK(cudaSetDevice(device));
    int nsm = 0;
    CU_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    cudaStream_t st;
    CU_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    // FP64 runs at a small fraction of the FP32 rate: fewer steps keep both
    // probes near a few tens of milliseconds
    const double p64 = probe<double>(nsm, 1 << 12, st);
    const double p32 = probe<float>(nsm, 1 << 16, st);
    cudaStreamDestroy(st);
    if (fp64_tflops) *fp64_tflops = p64;
    if (fp32_tflops) *fp32_tflops = p32;
    return MBE_OK;
  } catch (const MbeError& e) {
    return e.code;
  }
}
