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
  int nb2;                // > 0: two-level batch, item z at (z / nb2) sX + (z % nb2) sX2
  long long sA2, sB2, sC2;
};

template <typename T> void gemm(const GemmBatch& b, int maxM, int maxN, cudaStream_t s);

// Number of kernel launches issued by this library (process-wide).
void count_launch(int n = 1);
long long launches_issued();

// Kernel classes and stages for the optional event profiler.
enum ProfClass : int {
  PC_GEMM = 0, PC_POTF2, PC_TRSM, PC_HEGST_DIAG, PC_HETRD_HEMV, PC_HETRD_RANK2, PC_HETRD_VEC, PC_DC_LEAF,
  PC_DC_SECULAR, PC_DC_GEMM, PC_BACKTR_AUX, PC_OCC, PC_MISC, PC_OZAKI, PC_NCLASS
};
enum ProfStage : int {
  PS_COPY = 0, PS_POTRF, PS_HEGST, PS_HETRD, PS_STEDC, PS_BACKTR, PS_UNREDUCE, PS_OCC, PS_RHO, PS_ADJOINT, PS_REFINE,
  PS_NSTAGE
};
// Records CUDA events around launch groups (no-op when profiling is off).
struct Prof {
  virtual ~Prof() {}
  virtual int begin() = 0;
  virtual void end(int tok, int cls, double flops, double bytes) = 0;
};

// 2D strided copy with batch: dst[b][i][j] = src[b][i][j] (rows x cols).
template <typename T>
void copy2d(T* dst, int ldd, long long sd, const T* src, int lds, long long ss, int rows, int cols,
            int count, cudaStream_t s);

}  // namespace gks
