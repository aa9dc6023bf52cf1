// FMA-pipe peak of the GPU, measured: the denominators of the benchmark's
// roofline fractions for the ALU-bound kernels.  Not part of the FD-CGKS
// library (built as its own shared object and loaded only by the benchmark).
//
// Each thread runs NCHAIN independent fused multiply-add chains
// x <- x * a + b, enough independent work per warp to keep the FP64 or FP32
// pipe issuing every cycle; a grid of many resident blocks per SM covers all
// SMs.  A launch counts 2 flops per FMA.  The chain values are written out so
// that the compiler keeps every FMA.
#include <cuda_runtime.h>

namespace {

const int NCHAIN = 8;
const int THREADS = 256;

template <class T>
__global__ void __launch_bounds__(THREADS) fma_chains(T* out, int iters, T a, T b) {
  T x[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll 8
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int k = 0; k < NCHAIN; ++k) x[k] = fma(x[k], a, b);
    }
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += x[k];
  out[(long)blockIdx.x * THREADS + threadIdx.x] = s;
}

template <class T>
int run(int blocks_per_sm, int iters, int reps, double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  const int blocks = sms * blocks_per_sm;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * THREADS) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // contraction factor below 1 and a small offset: the chains stay bounded
  const T a = (T)0.999999, b = (T)1e-7;
  fma_chains<T><<<blocks, THREADS>>>(out, iters, a, b);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    fma_chains<T><<<blocks, THREADS>>>(out, iters, a, b);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return 2;
  const double flops = 2.0 * NCHAIN * 8.0 * (double)iters * (double)blocks * THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  *ms_out = best;
  return 0;
}

}  // namespace

// precision 0: FP64 FMA, 1: FP32 FMA.  Best of reps timed launches (after one
// warm-up) of blocks_per_sm x SM-count blocks of 256 threads, each thread
// doing 64 x iters FMAs.  Returns 0 on success.
extern "C" int pipe_peak_tflops(int precision, int blocks_per_sm, int iters, int reps, double* tflops, double* ms) {
  if (!tflops || !ms || blocks_per_sm < 1 || iters < 1 || reps < 1) return 1;
  return precision == 0 ? run<double>(blocks_per_sm, iters, reps, tflops, ms)
                        : run<float>(blocks_per_sm, iters, reps, tflops, ms);
}
