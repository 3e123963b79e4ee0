// Host-side launchers shared between the kernel translation units and the runtime.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gks_common.cuh"

namespace gks {

enum Op : int { OP_N = 0, OP_T = 1, OP_C = 2 };

// One GEMM problem: C = alpha * op(A) * diag(kscale) * op(B) + beta * C.
// Row-major operands; op(A) is M x K, op(B) is K x N, C is M x N.
struct GemmDesc {
  const void* A;
  const void* B;
  void* C;
  const double* kscale;   // nullable; length K
  int M, N, K;
  int lda, ldb, ldc;
};

// A batch of GEMMs sharing ops/scalars.  Either `list` (device array of `count`
// descriptors, grouped problems of different shapes) or `base` plus element strides.
struct GemmBatch {
  GemmDesc base;
  const GemmDesc* list;   // device pointer or nullptr
  long long sA, sB, sC, sK;  // strides (elements) between batch items when list == nullptr
  const int* kdev;        // nullable: per-item K read on the device (K = min(K, kdev[z]))
  int count;
  int opA, opB;
  int lower;              // 1: only tiles/elements with row >= col are written
  double alpha, beta;
};

template <typename T> void gemm(const GemmBatch& b, int maxM, int maxN, cudaStream_t s);

// 2D strided copy with batch: dst[b][i][j] = src[b][i][j] (rows x cols).
template <typename T>
void copy2d(T* dst, int ldd, long long sd, const T* src, int lds, long long ss, int rows, int cols,
            int count, cudaStream_t s);

}  // namespace gks
