// Arithmetic peak of the current device, measured: the denominator of the ALU
// roofline of the per-atom kernel (all its work is FP32/INT32 issue, with FP64
// only on the fallback paths).  Not part of the method.
//
// Every thread runs 8 independent FMA chains, 16 deep per loop trip, so the
// FMA pipes never wait on a dependency; one launch fills every SM with 1024
// threads.  x <- x * a + b with a just below 1 stays bounded, and the result is
// stored only when it equals an impossible value, so nothing is optimised away.

namespace ptm {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T *sink, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-7, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 16; u++) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == (T)-12345.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static cudaError_t fma_peak_run(cudaStream_t st, int blocks, int iters, T *sink, float &ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  cudaEventRecord(e0, st);
  k_fma_peak<T><<<blocks, 256, 0, st>>>(sink, iters, (T)0.9999999, (T)1e-7);
  e = cudaGetLastError();
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace ptm

extern "C" ptm_status ptm_measure_fma_peak(int kind, void *stream, double *flops_per_s) {
  using namespace ptm;
  if ((kind != 0 && kind != 1) || !flops_per_s) return PTM_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PTM_ERR_CUDA;
  cudaGetLastError();
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = 4 * sms;                     // 1024 threads per SM
  void *sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * 256 * 8) != cudaSuccess) return PTM_ERR_OUT_OF_MEMORY;
  // calibrate on a short run, then time a run of about 50 ms (best of 3)
  int iters = kind == 0 ? 2048 : 64;
  float ms = 0.f, best = 0.f;
  cudaError_t e = kind == 0 ? fma_peak_run<float>(st, blocks, iters, (float *)sink, ms)
                            : fma_peak_run<double>(st, blocks, iters, (double *)sink, ms);
  if (e == cudaSuccess) {
    const double scale = ms > 0.f ? 50.0 / ms : 16.0;
    iters = (int)std::min(std::max(iters * scale, 1.0), 1e7);
    for (int r = 0; r < 3 && e == cudaSuccess; r++) {
      e = kind == 0 ? fma_peak_run<float>(st, blocks, iters, (float *)sink, ms)
                    : fma_peak_run<double>(st, blocks, iters, (double *)sink, ms);
      if (e == cudaSuccess && (r == 0 || ms < best)) best = ms;
    }
  }
  cudaFree(sink);
  if (e != cudaSuccess || best <= 0.f) return PTM_ERR_CUDA;
  const double fmas = (double)blocks * 256.0 * (double)iters * 128.0;
  *flops_per_s = 2.0 * fmas / (best * 1e-3);
  return PTM_OK;
}
