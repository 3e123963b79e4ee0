// FP64 (real and complex) grouped/batched GEMM on the DFMA pipe.
//
// On GB300 the FP64 pipe delivers about 1 TFLOP/s (one DFMA lane-op per SM clock, 70x
// below FP32 FFMA), so every FP64 contraction is bound by that pipe and needs very
// little memory bandwidth: a 64 x 64 register-tiled CTA at K-step 16 asks for under one
// byte of shared memory per DFMA.  The kernel therefore favours many independent CTAs
// (grouped problems of different shapes in one launch) over deep software pipelining.
#include <atomic>
#include <cstdio>

#include "launch.h"

namespace gks {

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_issued() { return g_launches.load(std::memory_order_relaxed); }

template <typename T> struct GemmTile;
template <> struct GemmTile<double> {
  static constexpr int TM = 4, TN = 4, BK = 16;
};
template <> struct GemmTile<zc> {
  static constexpr int TM = 2, TN = 2, BK = 16;
};
// single precision (panel updates of the FP32 tridiagonalization): the FP32 pipe is ~60x
// the FP64 one, so larger register tiles pay
template <> struct GemmTile<float> {
  static constexpr int TM = 4, TN = 4, BK = 16;
};
template <> struct GemmTile<cf> {
  static constexpr int TM = 4, TN = 4, BK = 16;
};

template <typename T>
__device__ __forceinline__ T ld_op(const T* p, int op) {
  T v = *p;
  return op == OP_C ? conjg(v) : v;
}

template <typename T>
__global__ void __launch_bounds__(256) gemm_kernel(GemmBatch gb) {
  constexpr int TM = GemmTile<T>::TM, TN = GemmTile<T>::TN, BK = GemmTile<T>::BK;
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];

  const int z = blockIdx.z;
  GemmDesc d;
  if (gb.list) {
    d = gb.list[z];
  } else {
    d = gb.base;
    d.A = static_cast<const T*>(d.A) + item_off(z, gb.sA, gb.sA2, gb.nb2);
    d.B = static_cast<const T*>(d.B) + item_off(z, gb.sB, gb.sB2, gb.nb2);
    d.C = static_cast<T*>(d.C) + item_off(z, gb.sC, gb.sC2, gb.nb2);
    if (d.kscale) d.kscale += z * gb.sK;
  }
  int K = d.K;
  if (gb.kdev) K = min(K, gb.kdev[z]);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= d.M || n0 >= d.N) return;
  if (gb.lower && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal

  const T* A = static_cast<const T*>(d.A);
  const T* B = static_cast<const T*>(d.B);
  T* C = static_cast<T*>(d.C);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < TN; j++) acc[i][j] = zero<T>();

  for (int k0 = 0; k0 < K; k0 += BK) {
    // ---- A tile: op(A)[m0 + r][k0 + c] -> As[c][r]
    for (int e = tid; e < BM * BK; e += 256) {
      int r, c;
      if (gb.opA == OP_N) { r = e / BK; c = e % BK; } else { c = e / BM; r = e % BM; }
      int gm = m0 + r, gk = k0 + c;
      T v = zero<T>();
      if (gm < d.M && gk < K) {
        v = (gb.opA == OP_N) ? A[(size_t)gm * d.lda + gk] : ld_op(A + (size_t)gk * d.lda + gm, gb.opA);
        if (d.kscale) v = v * d.kscale[gk];
      }
      As[c][r] = v;
    }
    // ---- B tile: op(B)[k0 + c][n0 + r] -> Bs[c][r]
    for (int e = tid; e < BN * BK; e += 256) {
      int r, c;
      if (gb.opB == OP_N) { c = e / BN; r = e % BN; } else { r = e / BK; c = e % BK; }
      int gn = n0 + r, gk = k0 + c;
      T v = zero<T>();
      if (gn < d.N && gk < K)
        v = (gb.opB == OP_N) ? B[(size_t)gk * d.ldb + gn] : ld_op(B + (size_t)gn * d.ldb + gk, gb.opB);
      Bs[c][r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  // ---- epilogue: C = alpha * acc + beta * C
#pragma unroll
  for (int i = 0; i < TM; i++) {
    int gm = m0 + ty + 16 * i;
    if (gm >= d.M) continue;
#pragma unroll
    for (int j = 0; j < TN; j++) {
      int gn = n0 + tx + 16 * j;
      if (gn >= d.N) continue;
      if (gb.lower && gn > gm) continue;
      T* cp = C + (size_t)gm * d.ldc + gn;
      T v = gb.alpha * acc[i][j];
      if (gb.beta != 0.0) v = v + gb.beta * (*cp);
      *cp = v;
    }
  }
}

template <typename T>
void gemm(const GemmBatch& b, int maxM, int maxN, cudaStream_t s) {
  constexpr int BM = 16 * GemmTile<T>::TM, BN = 16 * GemmTile<T>::TN;
  if (maxM <= 0 || maxN <= 0 || b.count <= 0) return;
  dim3 grid((maxN + BN - 1) / BN, (maxM + BM - 1) / BM, b.count);
  count_launch();
  gemm_kernel<T><<<grid, 256, 0, s>>>(b);
}

template <typename T>
__global__ void copy2d_kernel(T* dst, int ldd, long long sd, const T* src, int lds, long long ss,
                              int rows, int cols) {
  const int z = blockIdx.z;
  dst += z * sd;
  src += z * ss;
  for (int i = blockIdx.y; i < rows; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += gridDim.x * blockDim.x)
      dst[(size_t)i * ldd + j] = src[(size_t)i * lds + j];
}

template <typename T>
void copy2d(T* dst, int ldd, long long sd, const T* src, int lds, long long ss, int rows, int cols,
            int count, cudaStream_t s) {
  if (rows <= 0 || cols <= 0 || count <= 0) return;
  dim3 grid((cols + 255) / 256 < 8 ? (cols + 255) / 256 : 8, rows < 1024 ? rows : 1024, count);
  count_launch();
  copy2d_kernel<T><<<grid, 256, 0, s>>>(dst, ldd, sd, src, lds, ss, rows, cols);
}

template void gemm<double>(const GemmBatch&, int, int, cudaStream_t);
template void gemm<zc>(const GemmBatch&, int, int, cudaStream_t);
template void gemm<float>(const GemmBatch&, int, int, cudaStream_t);
template void gemm<cf>(const GemmBatch&, int, int, cudaStream_t);
template void copy2d<double>(double*, int, long long, const double*, int, long long, int, int, int,
                             cudaStream_t);
template void copy2d<zc>(zc*, int, long long, const zc*, int, long long, int, int, int, cudaStream_t);
template void copy2d<float>(float*, int, long long, const float*, int, long long, int, int, int, cudaStream_t);
template void copy2d<cf>(cf*, int, long long, const cf*, int, long long, int, int, int, cudaStream_t);

}  // namespace gks
