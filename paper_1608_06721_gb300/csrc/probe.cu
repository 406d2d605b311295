// probe.cu -- measured FP64 issue rate of the current GPU (a measurement
// utility, not part of the method).
//
// The residual, Jacobian and BLU-SGS kernels are bound by the FP64 pipe, not
// by memory, so their roofline needs this GPU's FP64 rate.  The probe runs
// eight independent chains per thread of either fused multiply-adds or
// plain additions (the flux code is built without contraction, so its
// arithmetic is additions and multiplications issued one by one), on eight
// blocks of 256 threads per SM, and times the launch with CUDA events.
#include <cstdio>

#include "common.cuh"
#include "../../include/swnmg.h"

namespace {

template <int OP>
__global__ void __launch_bounds__(256) k_fp64_rate(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + 37 * k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = OP == 0 ? fma(x[k], a, b) : __dadd_rn(x[k], b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == -1.0) out[0] = s;   // never true: keeps the chains live
}

}  // namespace

SWNMG_API swnmg_status swnmg_fp64_rate(int32_t op, double* lane_ops_per_s) {
  if (!lane_ops_per_s || (op != 0 && op != 1)) {
    swnmg::set_static_error("fp64_rate: bad argument");
    return SWNMG_ERR_ARG;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = 8 * nsm, threads = 256, iters = 2048;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    swnmg::set_static_error("fp64_rate: cudaEventCreate failed");
    return SWNMG_ERR_CUDA;
  }
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch is a warm-up
    cudaEventRecord(e0, 0);
    if (op == 0) k_fp64_rate<0><<<blocks, threads>>>(nullptr, iters, 0.9999999, 1e-7);
    else k_fp64_rate<1><<<blocks, threads>>>(nullptr, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double rate = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
    if (rep > 0 && rate > best) best = rate;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof msg, "fp64_rate: %s", cudaGetErrorString(e));
    swnmg::set_static_error(msg);
    return SWNMG_ERR_CUDA;
  }
  *lane_ops_per_s = best;
  return SWNMG_OK;
}
