// Throughput probes of the FP64 units (the denominators of the FP64 rooflines): every
// thread keeps independent dependency chains in registers so that issue, not latency,
// limits the rate, and the result of every chain is stored so that nothing is removed.
//   DFMA: fma.rn.f64 on 8 chains per thread.
//   DMMA: mma.sync m8n8k4 f64 (the FP64 tensor instruction of this architecture) on 4
//         accumulator fragments per warp; 512 flops per warp instruction.
#include "dense.h"

namespace gks {

__global__ void __launch_bounds__(256) peak_dfma_kernel(double x, double y, long long iters, double* out) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; c++) a[c] = x * (threadIdx.x + c + 1);
  for (long long it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < 8; c++) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; c++) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) peak_dmma_kernel(double x, long long iters, double* out) {
  double av = x * (threadIdx.x + 1), bv = x * (threadIdx.x + 2);
  double d[4][2];
#pragma unroll
  for (int c = 0; c < 4; c++) d[c][0] = d[c][1] = 0.0;
  for (long long it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < 4; c++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(d[c][0]), "+d"(d[c][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; c++) s += d[c][0] + d[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Runs one probe on `sms` x 4 CTAs of 256 threads; returns the flops it executes and
// enqueues it on s (the caller times it with events).
double peak_probe(int which, int sms, long long iters, double* out, cudaStream_t s) {
  const int blocks = sms * 4, threads = 256;
  count_launch();
  if (which == 0) {
    peak_dfma_kernel<<<blocks, threads, 0, s>>>(0.9999999, 1e-9, iters, out);
    return 2.0 * 8.0 * (double)iters * blocks * threads;
  }
  peak_dmma_kernel<<<blocks, threads, 0, s>>>(0.5, iters, out);
  return 512.0 * 4.0 * (double)iters * blocks * (threads / 32);
}

}  // namespace gks
