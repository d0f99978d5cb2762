// Throughput probe of the FP64 and FP32 fused multiply-add pipes, the
// denominators of the arithmetic rooflines of the solve kernels (the FD
// Jacobian and the multigrid are bound by FP64 issue, not by memory).
//
// Every thread runs `iters` rounds of kChains independent FMA chains
// x <- x * a + b with a, b kernel arguments, so that nothing folds at compile
// time and each round issues kChains FMAs whose inputs do not depend on the
// round before them within a chain group; the chain results are summed and
// stored, so no chain is dead code. The caller times the launch with CUDA
// events on `stream`: flops = blocks * threads * iters * kChains * 2.
#include "nswe_internal.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void k_probe_fma(int iters, T a, T b, T *sink) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + 1 + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" nswe_status nswe_probe_fma(void *stream, int precision, int blocks, int threads, int iters, void *sink,
                                      double *flops) {
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !sink ||
      (precision != NSWE_PREC_FP64 && precision != NSWE_PREC_MIXED))
    return NSWE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // a < 1 and b > 0 keep every chain bounded (it tends to b / (1 - a))
  if (precision == NSWE_PREC_FP64)
    k_probe_fma<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-6, static_cast<double *>(sink));
  else
    k_probe_fma<float><<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-3f, static_cast<float *>(sink));
  if (cudaGetLastError() != cudaSuccess) return NSWE_ECUDA;
  if (flops) *flops = 2.0 * kChains * (double)blocks * threads * (double)iters;
  return NSWE_OK;
}
