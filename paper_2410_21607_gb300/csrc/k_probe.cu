// Arithmetic-rate probe (sem_peak_probe): the float32 and float64 FMA rates of
// the current GPU, measured with this library's own kernel, so that the
// fractions of the element kernels' ALU rooflines rest on a number measured
// on the part (GB300 has no published float64 vector rate to take instead).
//
// Every thread runs kChains independent FMA chains x <- x a + b for `iters`
// iterations (a, b kernel arguments, so nothing folds); the chains are
// independent, so the FMA pipe sees kChains instructions in flight per warp.
// The grid is a whole number of waves: blocks_per_sm x SMs blocks of 256.
// FLOP count: 2 x kChains x iters per thread.
#include "sem_internal.h"

namespace sem {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // one store per block keeps the chains live (every thread's chains feed
  // the sum the compiler must assume thread 0 stores)
  if (threadIdx.x == 0 || s == (T)-12345.0) out[blockIdx.x] = s;
}

template <typename T>
int run_probe(double* tflops, cudaStream_t st) {
  int dev = 0, nsm = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  SEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = 8;                                  // 2048 resident threads per SM
  const int blocks = nsm * per_sm;
  // about 2e11 (float32) or 5e9 (float64) FMAs: a few ms at the expected rates
  const int iters = sizeof(T) == 4 ? 12000 : 300;
  T* out = nullptr;
  SEM_CUDA_TRY(cudaMallocAsync((void**)&out, sizeof(T) * blocks, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, st);
    fma_probe<T><<<blocks, 256, 0, st>>>(out, iters, (T)0.999999, (T)1e-6);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("peak probe: ") + cudaGetErrorString(e));
  const double flop = 2.0 * kChains * (double)iters * 256.0 * blocks;
  *tflops = flop / (best * 1e-3) / 1e12;
  return SEM_OK;
}

}  // namespace
}  // namespace sem

extern "C" int sem_peak_probe(int precision, double* tflops, cudaStream_t st) {
  using namespace sem;
  if (!tflops) return fail(SEM_ERR_ARG, "tflops is NULL");
  if (precision == SEM_PREC_MIXED) return run_probe<float>(tflops, st);
  if (precision == SEM_PREC_FP64) return run_probe<double>(tflops, st);
  return fail(SEM_ERR_ARG, "precision must be SEM_PREC_FP64 or SEM_PREC_MIXED");
}
