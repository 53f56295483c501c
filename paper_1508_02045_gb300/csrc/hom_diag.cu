// hom_measure_fp64: the FP64 throughput of the device, measured with a kernel of this library.
//
// The operator's FP64 passes are bound by the FP64 pipe, not by HBM, so their roofline needs
// the pipe's rate on this device and clock. The kernel below issues long chains of
// independent FP64 fused multiply-adds (or adds) from every resident warp, enough of them in
// flight per SM to cover the pipe latency, and is timed with CUDA events on the caller's
// stream. Nothing here belongs to the method of the paper.
#include <cuda_runtime.h>

#include "../../include/hom.h"
#include "ops.h"

using namespace hom;

namespace {

constexpr int kChains = 8;   // independent dependency chains per thread
constexpr int kDiagThreads = 256;

// kind 0: x = fma(x, a, b) (2 flops an instruction); kind 1: x = x + b (1 flop). a = 1 - 2^-40
// and |b| tiny keep every value bounded; the sum is stored only if it equals a value it never
// takes, so the chains cannot be removed but nothing is written.
template <int KIND>
__global__ void __launch_bounds__(kDiagThreads)
k_fp64_chain(double* __restrict__ sink, double a, double b, int iters) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1.0 + 1e-3 * (double)(threadIdx.x * kChains + i);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if (KIND == 0) x[i] = fma(x[i], a, b);
        else x[i] = x[i] + ((u & 1) ? -b : b);
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int hom_measure_fp64(int kind, int iters, void* stream, double* ms, double* ops) {
  if ((kind != 0 && kind != 1) || iters < 1 || !ms || !ops) return HOM_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HOM_ERR_CUDA;
  cudaError_t e = kind == 0
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_chain<0>, kDiagThreads, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_chain<1>, kDiagThreads, 0);
  if (e != cudaSuccess || per_sm < 1) return HOM_ERR_CUDA;
  const int blocks = sms * per_sm;  // one full wave: every SM holds its resident maximum
  const double a = 1.0 - 9.094947017729282e-13, b = 1e-300;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return HOM_ERR_CUDA;
  }
  // one untimed launch (clocks up, code resident), then the timed one
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) cudaEventRecord(e0, st);
    if (kind == 0) k_fp64_chain<0><<<blocks, kDiagThreads, 0, st>>>(nullptr, a, b, iters);
    else k_fp64_chain<1><<<blocks, kDiagThreads, 0, st>>>(nullptr, a, b, iters);
    ++launch_counter();
  }
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return HOM_ERR_CUDA;
  const double instr = (double)blocks * kDiagThreads * kChains * 16.0 * (double)iters;
  *ms = (double)t;
  *ops = instr * (kind == 0 ? 2.0 : 1.0);
  return HOM_OK;
}
