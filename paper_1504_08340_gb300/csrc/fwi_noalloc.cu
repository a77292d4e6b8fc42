// fwi_noalloc.cu -- misfit of device-resident traces without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a host callback or
// a memory-pool-constrained serving process, plug-ins loaded into a host
// application that owns the device memory budget, or code that must not
// allocate between two calls of a latency-critical loop. For them this file
// offers fwi_trace_misfit_noalloc: the misfit (7) of traces that already live
// on the GPU, computed by the same two-level FP64 reduction as fwi_misfit but
// with its scratch in a fixed file-scope device array instead of memory from
// cudaMalloc. The caller passes inputs and outputs; the call allocates nothing.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/fwi.h"

namespace {

// Scratch: one FP64 partial sum per time sample (at most kMaxSamples samples,
// i.e. nsteps <= kMaxSamples - 1), then the total and a non-finite flag.
// 64 Ki samples * 8 bytes = 512 KiB, held by every GPU that loads the library
// until the process exits.
constexpr int kMaxSamples = 65536;
constexpr int kThreads = 256;
static __device__ __align__(256) double g_misfit_scratch[kMaxSamples + 2];

// Per-sample sums sum_r sum_c (tr - ob)^2 in FP64, one block per sample (grid-stride
// over samples), fixed-order tree reduction: deterministic.
__global__ void __launch_bounds__(kThreads) sample_sums(const float *tr, const float *ob, int64_t per_sample,
                                                        int nsamples, double *part, double *flag) {
  __shared__ double sh[kThreads];
  for (int n = blockIdx.x; n < nsamples; n += gridDim.x) {
    double acc = 0.0;
    bool bad = false;
    for (int64_t i = threadIdx.x; i < per_sample; i += kThreads) {
      const float t = tr[(int64_t)n * per_sample + i];
      const float o = ob[(int64_t)n * per_sample + i];
      if (!isfinite(t) || !isfinite(o)) bad = true;
      const float e = t - o;  // as fwi_misfit: FP32 residual, FP64 sum
      acc += (double)e * (double)e;
    }
    if (bad) *flag = 1.0;
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[n] = sh[0];
    __syncthreads();
  }
}

// J = 1/2 dt sum_n w_n part[n], trapezoid weights w_0 = w_N = 1/2; one block.
__global__ void __launch_bounds__(kThreads) trapezoid_total(const double *part, int nsamples, double dt,
                                                            double *out) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int n = threadIdx.x; n < nsamples; n += kThreads) {
    const double wn = (n == 0 || n == nsamples - 1) ? 0.5 : 1.0;
    acc += wn * part[n];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * dt * sh[0];
}

// Device address of the scratch array in the current context. In host code the
// name g_misfit_scratch is only a host-side stand-in, not a device address, so
// every call asks the runtime for the address in the context that is current
// now. The lookup is a cheap host call; not caching it means a context that was
// torn down and created again never sees a stale address.
cudaError_t scratch_for_current_device(double **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_misfit_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double *>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" fwi_status fwi_trace_misfit_noalloc(const float *traces, const float *observed, int nsteps, int nrec,
                                               double dt, void *cuda_stream, double *J) {
  if (!traces || !observed || !J || nrec < 1 || nsteps < 0 || !(dt > 0)) return FWI_E_INVAL;
  if (nsteps >= kMaxSamples) return FWI_E_INVAL;  // more time samples than the scratch holds
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double *scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return FWI_E_CUDA;
  const int nsamples = nsteps + 1;
  double *part = scratch, *total = scratch + kMaxSamples, *flag = scratch + kMaxSamples + 1;
  // every call shares the array: clear the flag that must start at zero
  if (cudaMemsetAsync(flag, 0, sizeof(double), s) != cudaSuccess) return FWI_E_CUDA;
  const int blocks = nsamples < 4096 ? nsamples : 4096;
  sample_sums<<<blocks, kThreads, 0, s>>>(traces, observed, (int64_t)nrec * 3, nsamples, part, flag);
  trapezoid_total<<<1, kThreads, 0, s>>>(part, nsamples, dt, total);
  if (cudaGetLastError() != cudaSuccess) return FWI_E_CUDA;
  double host[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(host, total, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FWI_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FWI_E_CUDA;
  if (host[1] != 0.0 || !std::isfinite(host[0])) return FWI_E_NONFINITE;
  *J = host[0];
  return FWI_OK;
}
