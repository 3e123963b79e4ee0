// Ogita-Aishima refinement of the eigenpairs of the standard Hermitian problem H' X = X L
// (the mixed-precision path: eigenvectors from a single-precision tridiagonalization,
// refined with FP64-accurate products; Ogita & Aishima 2018).  One sweep, per item:
//   T = X^H H' X,  R = I - X^H X                         (products, FP64-accurate)
//   l_i = t_ii / (1 - r_ii)
//   w   = 2 (||T - diag(l)|| + ||H'|| ||R||)              (cluster threshold)
//   E_ii = r_ii / 2,
//   E_ij = (t_ij + l_j r_ij) / (l_j - l_i)   if |l_i - l_j| > w, else r_ij / 2
//   X  <- X + X E.
// The 2-norms in w are bounded above by the largest absolute row sums (exact bounds for
// Hermitian matrices, so w is never underestimated); ||H'||_2 is max_i |l_i| (the
// spectral radius of H' up to the error of the l_i, far below w).
#include "dense.h"

namespace gks {

__device__ __forceinline__ double absv(double a) { return fabs(a); }
__device__ __forceinline__ double absv(zc a) { return sqrt(a.x * a.x + a.y * a.y); }

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// One warp per row i of item z: G = X^H X becomes R = I - G (full storage), l_i from the
// diagonals, and the row sums of |T - diag(l)| and |R| (maxima per item into nrm[z][0..1]);
// nrm[z][2] collects max |l_i|.
template <typename T>
__global__ void __launch_bounds__(256) oa_prepare_kernel(const T* Tm, T* G, long long sMM, int M, double* lam,
                                                         double* nrm) {
  const int z = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= M) return;
  Tm += z * sMM;
  G += z * sMM;
  const T* trow = Tm + (size_t)i * M;
  T* grow = G + (size_t)i * M;
  const double tii = re(trow[i]), gii = re(grow[i]);
  const double li = tii / gii;  // t_ii / (1 - r_ii), 1 - r_ii = (X^H X)_ii
  double st = 0.0, sr = 0.0;
  for (int j = lane; j < M; j += 32) {
    T g = grow[j];
    T r = (j == i) ? from_real<T>(1.0 - re(g)) : zero<T>() - g;
    grow[j] = r;
    sr += absv(r);
    st += (j == i) ? fabs(re(trow[j]) - li) : absv(trow[j]);
  }
  st = warp_sum(st);
  sr = warp_sum(sr);
  if (lane == 0) {
    lam[(size_t)z * M + i] = li;
    atomic_max_nonneg(nrm + 3 * z, st);
    atomic_max_nonneg(nrm + 3 * z + 1, sr);
    atomic_max_nonneg(nrm + 3 * z + 2, fabs(li));
  }
}

// E overwrites T (full storage, item z): the correction matrix of the sweep.
template <typename T>
__global__ void __launch_bounds__(256) oa_correction_kernel(T* Tm, const T* R, long long sMM, int M,
                                                            const double* lam, const double* nrm) {
  const int z = blockIdx.z;
  Tm += z * sMM;
  R += z * sMM;
  lam += (size_t)z * M;
  const double w = 2.0 * (nrm[3 * z] + nrm[3 * z + 2] * nrm[3 * z + 1]);
  for (int i = blockIdx.y; i < M; i += gridDim.y) {
    const double li = lam[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
      const size_t o = (size_t)i * M + j;
      const T r = R[o];
      T e;
      if (j == i) {
        e = from_real<T>(0.5 * re(r));
      } else {
        const double lj = lam[j], d = lj - li;
        if (fabs(d) > w) e = (Tm[o] + lj * r) * (1.0 / d);
        else e = 0.5 * r;
      }
      Tm[o] = e;
    }
  }
}

// Ascending order after refinement (near-degenerate eigenvalues may swap): one CTA per item
// checks the order and, if needed, sorts (eigenvalue, column) pairs stably by odd-even
// transposition in shared memory; perm[z][j] = source column of column j, flag[z] = 1.
__global__ void oa_order_kernel(double* lam, int M, int* perm, int* flag) {
  extern __shared__ unsigned char smem[];
  double* key = reinterpret_cast<double*>(smem);
  int* idx = reinterpret_cast<int*>(key + M);
  __shared__ int unsorted;
  const int z = blockIdx.x, tid = threadIdx.x;
  lam += (size_t)z * M;
  perm += (size_t)z * M;
  if (tid == 0) unsorted = 0;
  __syncthreads();
  for (int i = tid; i + 1 < M; i += blockDim.x)
    if (lam[i] > lam[i + 1]) unsorted = 1;
  __syncthreads();
  if (!unsorted) {
    if (tid == 0) flag[z] = 0;
    return;
  }
  for (int i = tid; i < M; i += blockDim.x) {
    key[i] = lam[i];
    idx[i] = i;
  }
  __syncthreads();
  for (int ph = 0; ph < M; ph++) {
    for (int i = 2 * tid + (ph & 1); i + 1 < M; i += 2 * blockDim.x) {
      if (key[i] > key[i + 1]) {
        double tk = key[i];
        key[i] = key[i + 1];
        key[i + 1] = tk;
        int ti = idx[i];
        idx[i] = idx[i + 1];
        idx[i + 1] = ti;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < M; i += blockDim.x) {
    lam[i] = key[i];
    perm[i] = idx[i];
  }
  if (tid == 0) flag[z] = 1;
}

// Y[z][i][j] = X[z][i][perm[z][j]] for the items whose order changed.
template <typename T>
__global__ void oa_permute_kernel(const T* X, T* Y, long long sMM, int M, const int* perm, const int* flag) {
  const int z = blockIdx.z;
  if (!flag[z]) return;
  X += z * sMM;
  Y += z * sMM;
  perm += (size_t)z * M;
  for (int i = blockIdx.y; i < M; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
      Y[(size_t)i * M + j] = X[(size_t)i * M + perm[j]];
}

template <typename T>
__global__ void oa_copy_back_kernel(const T* Y, T* X, long long sMM, int M, const int* flag) {
  const int z = blockIdx.z;
  if (!flag[z]) return;
  X += z * sMM;
  Y += z * sMM;
  for (int i = blockIdx.y; i < M; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
      X[(size_t)i * M + j] = Y[(size_t)i * M + j];
}

static dim3 grid_rows(int rows, int cols, int count) {
  int gx = (cols + 255) / 256;
  gx = gx > 16 ? 16 : (gx < 1 ? 1 : gx);
  return dim3(gx, rows < 2048 ? (rows > 0 ? rows : 1) : 2048, count);
}

template <typename T>
void oa_prepare(const T* Tm, T* G, long long sMM, int M, double* lam, double* nrm, int count, cudaStream_t s) {
  cudaMemsetAsync(nrm, 0, sizeof(double) * 3 * count, s);
  count_launch();
  oa_prepare_kernel<T><<<dim3((M + 7) / 8, count), 256, 0, s>>>(Tm, G, sMM, M, lam, nrm);
}

template <typename T>
void oa_correction(T* Tm, const T* R, long long sMM, int M, const double* lam, const double* nrm, int count,
                   cudaStream_t s) {
  count_launch();
  oa_correction_kernel<T><<<grid_rows(M, M, count), 256, 0, s>>>(Tm, R, sMM, M, lam, nrm);
}

template <typename T>
void oa_order(double* lam, T* X, T* Y, long long sMM, int M, int* perm, int* flag, int count, cudaStream_t s) {
  const size_t sm = (size_t)M * (sizeof(double) + sizeof(int));
  if (sm > 48 * 1024) cudaFuncSetAttribute(oa_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch(3);
  oa_order_kernel<<<count, 1024, sm, s>>>(lam, M, perm, flag);
  oa_permute_kernel<T><<<grid_rows(M, M, count), 256, 0, s>>>(X, Y, sMM, M, perm, flag);
  oa_copy_back_kernel<T><<<grid_rows(M, M, count), 256, 0, s>>>(Y, X, sMM, M, flag);
}

#define INST(T)                                                                                          \
  template void oa_prepare<T>(const T*, T*, long long, int, double*, double*, int, cudaStream_t);        \
  template void oa_correction<T>(T*, const T*, long long, int, const double*, const double*, int,        \
                                 cudaStream_t);                                                          \
  template void oa_order<T>(double*, T*, T*, long long, int, int*, int*, int, cudaStream_t);
INST(double)
INST(zc)

}  // namespace gks
