// Small dense kernels around the GEMM core: diagonal-block Cholesky, triangular solves
// against a diagonal block, the two-sided reduction of a diagonal block, the compact-WY
// T factor, and elementwise helpers (phase application, Hermitian mirror, eigenvector
// phase, spinor overlap).
#include "dense.h"

namespace gks {

// One CTA per batch item: factor the nb x nb diagonal block of A at (k0, k0) in place
// (lower, A = L L^H).  A non-positive or non-finite pivot records GKS_ENOTSPD with the
// global column and leaves the block untouched.
template <typename T>
__global__ void potf2_kernel(T* A, int lda, long long sA, int k0, int nb, DevStatus* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* a = reinterpret_cast<T*>(smem_raw);
  __shared__ int fail;
  const int z = blockIdx.x, ld = nb + 1, tid = threadIdx.x, nt = blockDim.x;
  A += z * sA;
  for (int e = tid; e < nb * nb; e += nt) {
    int i = e / nb, j = e % nb;
    a[i * ld + j] = (j <= i) ? A[(size_t)(k0 + i) * lda + k0 + j] : zero<T>();
  }
  if (tid == 0) fail = -1;
  __syncthreads();
  for (int j = 0; j < nb; j++) {
    if (tid == 0) {
      double piv = re(a[j * ld + j]);
      if (!(piv > 0.0) || !isfinite(piv)) fail = j;
      else a[j * ld + j] = from_real<T>(sqrt(piv));
    }
    __syncthreads();
    if (fail >= 0) break;
    const double ljj = re(a[j * ld + j]);
    for (int i = j + 1 + tid; i < nb; i += nt) a[i * ld + j] = a[i * ld + j] * (1.0 / ljj);
    __syncthreads();
    const int m = nb - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      int r = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= r) a[r * ld + c] -= a[r * ld + j] * conjg(a[c * ld + j]);
    }
    __syncthreads();
  }
  if (fail >= 0) {
    if (tid == 0) set_status(st ? st + z : nullptr, ST_ENOTSPD, k0 + fail);
    return;
  }
  for (int e = tid; e < nb * nb; e += nt) {
    int i = e / nb, j = e % nb;
    if (j <= i) A[(size_t)(k0 + i) * lda + k0 + j] = a[i * ld + j];
  }
}

// Triangular solves against one nb x nb lower-triangular block L (ldl), by substitution
// (no explicit inverse: the diagonal blocks of the Cholesky factor of an overcomplete
// basis have condition numbers near 1e5).  Each CTA takes 64 right-hand sides into
// shared memory, one thread per right-hand side.
//   TRSM_RIGHT_CONJ : B (nrhs x nb rows)  <- B L^-H
//   TRSM_LEFT       : B (nb x nrhs cols)  <- L^-1 B
//   TRSM_LEFT_CONJ  : B (nb x nrhs cols)  <- L^-H B
template <typename T, int MODE>
__global__ void __launch_bounds__(64) trsm_block_kernel(const T* L, int ldl, long long sL, T* B, int ldb, long long sB,
                                                        int nb, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* x = reinterpret_cast<T*>(smem_raw);  // MODE 0: [64][nb+1] (row per rhs); else [nb][65]
  const int z = blockIdx.y, tid = threadIdx.x, r0 = blockIdx.x * 64;
  L += z * sL;
  B += z * sB;
  const int nr = min(64, nrhs - r0);
  if (MODE == TRSM_RIGHT_CONJ) {
    const int ld = nb + 1;
    for (int e = tid; e < nr * nb; e += 64) {
      int r = e / nb, c = e % nb;
      x[r * ld + c] = B[(size_t)(r0 + r) * ldb + c];
    }
    __syncthreads();
    if (tid < nr) {
      T* xr = x + tid * ld;
      for (int j = 0; j < nb; j++) {  // x L^H = b  <=>  x_j = (b_j - sum_{k<j} x_k conj(L_jk)) / L_jj
        const T* lj = L + (size_t)j * ldl;
        T s0 = xr[j], s1 = zero<T>(), s2 = zero<T>(), s3 = zero<T>();  // four chains (latency)
        int k = 0;
        for (; k + 3 < j; k += 4) {
          s0 -= xr[k] * conjg(lj[k]);
          s1 -= xr[k + 1] * conjg(lj[k + 1]);
          s2 -= xr[k + 2] * conjg(lj[k + 2]);
          s3 -= xr[k + 3] * conjg(lj[k + 3]);
        }
        for (; k < j; k++) s0 -= xr[k] * conjg(lj[k]);
        xr[j] = ((s0 + s1) + (s2 + s3)) * (1.0 / re(lj[j]));
      }
    }
    __syncthreads();
    for (int e = tid; e < nr * nb; e += 64) {
      int r = e / nb, c = e % nb;
      B[(size_t)(r0 + r) * ldb + c] = x[r * ld + c];
    }
  } else {
    const int ld = 65;
    for (int e = tid; e < nb * 64; e += 64) {
      int i = e / 64, c = e % 64;
      if (c < nr) x[i * ld + c] = B[(size_t)i * ldb + r0 + c];
    }
    __syncthreads();
    if (tid < nr) {
      T* xc = x + tid;
      if (MODE == TRSM_LEFT) {
        for (int i = 0; i < nb; i++) {  // x_i = (b_i - sum_{k<i} L_ik x_k) / L_ii
          const T* li = L + (size_t)i * ldl;
          T s0 = xc[i * ld], s1 = zero<T>(), s2 = zero<T>(), s3 = zero<T>();
          int k = 0;
          for (; k + 3 < i; k += 4) {
            s0 -= li[k] * xc[k * ld];
            s1 -= li[k + 1] * xc[(k + 1) * ld];
            s2 -= li[k + 2] * xc[(k + 2) * ld];
            s3 -= li[k + 3] * xc[(k + 3) * ld];
          }
          for (; k < i; k++) s0 -= li[k] * xc[k * ld];
          xc[i * ld] = ((s0 + s1) + (s2 + s3)) * (1.0 / re(li[i]));
        }
      } else {
        for (int i = nb - 1; i >= 0; i--) {  // x_i = (b_i - sum_{k>i} conj(L_ki) x_k) / L_ii
          T s0 = xc[i * ld], s1 = zero<T>(), s2 = zero<T>(), s3 = zero<T>();
          int k = i + 1;
          for (; k + 3 < nb; k += 4) {
            s0 -= conjg(L[(size_t)k * ldl + i]) * xc[k * ld];
            s1 -= conjg(L[(size_t)(k + 1) * ldl + i]) * xc[(k + 1) * ld];
            s2 -= conjg(L[(size_t)(k + 2) * ldl + i]) * xc[(k + 2) * ld];
            s3 -= conjg(L[(size_t)(k + 3) * ldl + i]) * xc[(k + 3) * ld];
          }
          for (; k < nb; k++) s0 -= conjg(L[(size_t)k * ldl + i]) * xc[k * ld];
          xc[i * ld] = ((s0 + s1) + (s2 + s3)) * (1.0 / re(L[(size_t)i * ldl + i]));
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < nb * 64; e += 64) {
      int i = e / 64, c = e % 64;
      if (c < nr) B[(size_t)i * ldb + r0 + c] = x[i * ld + c];
    }
  }
}

// One CTA per batch item: the diagonal block A11 <- L11^-1 A11 L11^-H (A11 read from its
// lower triangle) by the two-sided column recurrence
//   alpha_k = a_kk / l_kk^2,  v = a(k+1:, k)/l_kk - (alpha_k/2) l(k+1:, k),
//   A(k+1:, k+1:) -= l v^H + v l^H,  r_k = v - (alpha_k/2) l(k+1:, k),
// followed by the deferred in-block solve X = L11^-1 [r_0 r_1 ...] (strictly lower part).
// Writes the lower triangle back into A and the full Hermitian block into F (ldF).
template <typename T>
__global__ void hegst_diag_kernel(T* A, int lda, long long sA, const T* L, int ldl, long long sL, int k0, int nb,
                                  T* F, int ldF, long long sF) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* a = reinterpret_cast<T*>(smem_raw);
  T* l = a + nb * (nb + 1);
  const int z = blockIdx.x, ld = nb + 1, tid = threadIdx.x, nt = blockDim.x;
  A += z * sA;
  L += z * sL;
  F += z * sF;
  for (int e = tid; e < nb * nb; e += nt) {
    int i = e / nb, j = e % nb;
    a[i * ld + j] = (j <= i) ? A[(size_t)(k0 + i) * lda + k0 + j] : zero<T>();
    l[i * ld + j] = (j <= i) ? L[(size_t)(k0 + i) * ldl + k0 + j] : zero<T>();
  }
  __syncthreads();
  for (int k = 0; k < nb; k++) {
    const double lkk = re(l[k * ld + k]);
    const double alpha = re(a[k * ld + k]) / (lkk * lkk);
    for (int i = k + 1 + tid; i < nb; i += nt) a[i * ld + k] = a[i * ld + k] * (1.0 / lkk) - (0.5 * alpha) * l[i * ld + k];
    __syncthreads();
    const int m = nb - k - 1;
    for (int e = tid; e < m * m; e += nt) {
      int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) a[i * ld + j] -= l[i * ld + k] * conjg(a[j * ld + k]) + a[i * ld + k] * conjg(l[j * ld + k]);
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < nb; i += nt) a[i * ld + k] = a[i * ld + k] - (0.5 * alpha) * l[i * ld + k];
    if (tid == 0) a[k * ld + k] = from_real<T>(alpha);
    __syncthreads();
  }
  for (int c = tid; c < nb; c += nt) {  // column c: rows i > c, forward substitution with L11
    for (int i = c + 1; i < nb; i++) {
      T s = a[i * ld + c];
      for (int k = c + 1; k < i; k++) s -= l[i * ld + k] * a[k * ld + c];
      a[i * ld + c] = s * (1.0 / re(l[i * ld + i]));
    }
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += nt) {
    int i = e / nb, j = e % nb;
    T v = (j <= i) ? a[i * ld + j] : conjg(a[j * ld + i]);
    if (i == j) v = from_real<T>(re(v));
    F[(size_t)i * ldF + j] = v;
    if (j <= i) A[(size_t)(k0 + i) * lda + k0 + j] = v;
  }
}

// Compact WY T factor for H_1 H_2 ... H_k = I - V T V^H with H_i = I - tau_i v_i v_i^H:
// T upper triangular, T_ii = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i] (V^H V)[0:i, i].
// G = V^H V (k x k, ldG) precomputed; one CTA per batch item.
template <typename T>
__global__ void larft_kernel(const T* G, int ldG, long long sG, const double* tau, long long stau, int k,
                             T* Tm, int ldT, long long sT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* t = reinterpret_cast<T*>(smem_raw);
  T* tmp = t + k * k;
  const int z = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  G += z * sG;
  tau += z * stau;
  Tm += z * sT;
  for (int e = tid; e < k * k; e += nt) t[e] = zero<T>();
  __syncthreads();
  for (int i = 0; i < k; i++) {
    const double ti = tau[i];
    for (int r = tid; r < i; r += nt) {
      T s = zero<T>();
      for (int c = r; c < i; c++) mac(s, t[r * k + c], G[(size_t)c * ldG + i]);
      tmp[r] = s;
    }
    __syncthreads();
    for (int r = tid; r < i; r += nt) t[r * k + i] = (-ti) * tmp[r];
    if (tid == 0) t[i * k + i] = from_real<T>(ti);
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += nt) Tm[(size_t)(e / k) * ldT + (e % k)] = t[e];
}

// X[b][i][c] = ph[b][i] * Z[b][i][c] for the leading `cols` columns (Z real, X of type T)
template <typename T>
__global__ void apply_phase_kernel(T* X, int ldx, long long sX, const double* Z, int ldz, long long sZ,
                                   const T* ph, long long sph, int n, int cols) {
  const int z = blockIdx.z;
  X += z * sX;
  Z += z * sZ;
  ph += z * sph;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    T p = ph[i];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x)
      X[(size_t)i * ldx + c] = p * Z[(size_t)i * ldz + c];
  }
}

// Upper triangle <- conj(lower triangle); diagonal made real.
template <typename T>
__global__ void mirror_lower_kernel(T* A, int lda, long long sA, int n) {
  const int z = blockIdx.z;
  A += z * sA;
  for (int i = blockIdx.y; i < n; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += gridDim.x * blockDim.x) {
      T v = A[(size_t)i * lda + j];
      if (j == i) A[(size_t)i * lda + i] = from_real<T>(re(v));
      else A[(size_t)j * lda + i] = conjg(v);
    }
}

// Column phase convention: the entry of largest modulus (lowest row on ties) becomes
// real and positive.  One warp per column.
template <typename T>
__global__ void column_phase_kernel(T* C, int ldc, long long sC, int rows, int cols) {
  const int z = blockIdx.y;
  C += z * sC;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= cols) return;
  double best = -1.0;
  int bi = 0;
  for (int i = lane; i < rows; i += 32) {
    double a = abs2(C[(size_t)i * ldc + col]);
    if (a > best) { best = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  T p = C[(size_t)bi * ldc + col];
  double mag = sqrt(abs2(p));
  if (!(mag > 0.0)) return;
  T f = conjg(p) * (1.0 / mag);
  for (int i = lane; i < rows; i += 32) C[(size_t)i * ldc + col] = C[(size_t)i * ldc + col] * f;
}

// Fill dst (2n x 2n) with diag(S, S) from the n x n S (lower triangle valid).
template <typename T>
__global__ void spinor_overlap_kernel(T* dst, long long sd, const T* S, int lds, long long ss, int n) {
  const int z = blockIdx.z;
  dst += z * sd;
  S += z * ss;
  const int m = 2 * n;
  for (int i = blockIdx.y; i < m; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
      T v = zero<T>();
      if ((i < n) == (j < n)) {
        int a = i % n, b = j % n;
        v = (b <= a) ? S[(size_t)a * lds + b] : conjg(S[(size_t)b * lds + a]);
      }
      dst[(size_t)i * m + j] = v;
    }
}

// Loewdin factor V = U diag(s)^-1/2 (paper Sec. 3.1 Part 2-2) from the eigenvectors U
// (ldu, sU) and eigenvalues s (ss per item) of S; a non-positive eigenvalue reports
// GKS_ENOTSPD with its index and zeroes the column.
template <typename T>
__global__ void lowdin_factor_kernel(const T* U, int ldu, long long sU, const double* sv, long long ss, T* V, int ldv,
                                     long long sV, int n, DevStatus* st) {
  const int z = blockIdx.z;
  U += z * sU;
  V += z * sV;
  sv += z * ss;
  for (int i = blockIdx.y; i < n; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      const double sj = sv[j];
      if (!(sj > 0.0)) {
        if (i == 0) set_status(st ? st + z : nullptr, ST_ENOTSPD, j);
        V[(size_t)i * ldv + j] = zero<T>();
      } else {
        V[(size_t)i * ldv + j] = U[(size_t)i * ldu + j] * (1.0 / sqrt(sj));
      }
    }
}

// ------------------------------------------------------------------ launchers

static dim3 grid2d(int rows, int cols, int count) {
  int gx = (cols + 255) / 256;
  if (gx > 16) gx = 16;
  if (gx < 1) gx = 1;
  int gy = rows < 2048 ? (rows > 0 ? rows : 1) : 2048;
  return dim3(gx, gy, count);
}

template <typename T>
void potf2(T* A, int lda, long long sA, int k0, int nb, DevStatus* st, int count, cudaStream_t s) {
  size_t sm = sizeof(T) * nb * (nb + 1);
  cudaFuncSetAttribute(potf2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch();
  potf2_kernel<T><<<count, 256, sm, s>>>(A, lda, sA, k0, nb, st);
}

template <typename T>
void trsm_block(int mode, const T* L, int ldl, long long sL, T* B, int ldb, long long sB, int nb, int nrhs,
                int count, cudaStream_t s) {
  if (nrhs <= 0 || nb <= 0 || count <= 0) return;
  dim3 grid((nrhs + 63) / 64, count);
  if (mode == TRSM_RIGHT_CONJ) {
    size_t sm = sizeof(T) * 64 * (nb + 1);
    cudaFuncSetAttribute(trsm_block_kernel<T, TRSM_RIGHT_CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    count_launch();
    trsm_block_kernel<T, TRSM_RIGHT_CONJ><<<grid, 64, sm, s>>>(L, ldl, sL, B, ldb, sB, nb, nrhs);
  } else if (mode == TRSM_LEFT) {
    size_t sm = sizeof(T) * nb * 65;
    cudaFuncSetAttribute(trsm_block_kernel<T, TRSM_LEFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    count_launch();
    trsm_block_kernel<T, TRSM_LEFT><<<grid, 64, sm, s>>>(L, ldl, sL, B, ldb, sB, nb, nrhs);
  } else {
    size_t sm = sizeof(T) * nb * 65;
    cudaFuncSetAttribute(trsm_block_kernel<T, TRSM_LEFT_CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    count_launch();
    trsm_block_kernel<T, TRSM_LEFT_CONJ><<<grid, 64, sm, s>>>(L, ldl, sL, B, ldb, sB, nb, nrhs);
  }
}

template <typename T>
void hegst_diag(T* A, int lda, long long sA, const T* L, int ldl, long long sL, int k0, int nb, T* F, int ldF,
                long long sF, int count, cudaStream_t s) {
  size_t sm = 2 * sizeof(T) * nb * (nb + 1);
  cudaFuncSetAttribute(hegst_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch();
  hegst_diag_kernel<T><<<count, 256, sm, s>>>(A, lda, sA, L, ldl, sL, k0, nb, F, ldF, sF);
}

template <typename T>
void larft(const T* G, int ldG, long long sG, const double* tau, long long stau, int k, T* Tm, int ldT,
           long long sT, int count, cudaStream_t s) {
  size_t sm = sizeof(T) * (k * k + k);
  cudaFuncSetAttribute(larft_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch();
  larft_kernel<T><<<count, 128, sm, s>>>(G, ldG, sG, tau, stau, k, Tm, ldT, sT);
}

template <typename T>
void apply_phase(T* X, int ldx, long long sX, const double* Z, int ldz, long long sZ, const T* ph, long long sph,
                 int n, int cols, int count, cudaStream_t s) {
  count_launch();
  apply_phase_kernel<T><<<grid2d(n, cols, count), 256, 0, s>>>(X, ldx, sX, Z, ldz, sZ, ph, sph, n, cols);
}

template <typename T>
void lowdin_factor(const T* U, int ldu, long long sU, const double* sv, long long ss, T* V, int ldv, long long sV,
                   int n, DevStatus* st, int count, cudaStream_t s) {
  count_launch();
  lowdin_factor_kernel<T><<<grid2d(n, n, count), 256, 0, s>>>(U, ldu, sU, sv, ss, V, ldv, sV, n, st);
}

template <typename T>
void mirror_lower(T* A, int lda, long long sA, int n, int count, cudaStream_t s) {
  count_launch();
  mirror_lower_kernel<T><<<grid2d(n, n, count), 256, 0, s>>>(A, lda, sA, n);
}

template <typename T>
void column_phase(T* C, int ldc, long long sC, int rows, int cols, int count, cudaStream_t s) {
  dim3 grid((cols + 7) / 8, count);
  count_launch();
  column_phase_kernel<T><<<grid, 256, 0, s>>>(C, ldc, sC, rows, cols);
}

template <typename T>
void spinor_overlap(T* dst, long long sd, const T* S, int lds, long long ss, int n, int count, cudaStream_t s) {
  count_launch();
  spinor_overlap_kernel<T><<<grid2d(2 * n, 2 * n, count), 256, 0, s>>>(dst, sd, S, lds, ss, n);
}

// Seeded test pencils for the width tuner (no input data needed): splitmix64 of the
// element index gives uniform numbers.  hermitian = 1: entries in [-1, 1] (both parts);
// hermitian = 0: S = I + entries in [-0.5, 0.5]/m off the diagonal (diagonally dominant).
__device__ __forceinline__ double tune_uniform(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * 0x1.0p-53;
}

template <typename T>
__global__ void tune_pencil_kernel(T* A, int m, int hermitian) {
  const int z = blockIdx.z;
  A += (size_t)z * m * m;
  for (int i = blockIdx.y; i < m; i += gridDim.y)
    for (int jj = blockIdx.x * blockDim.x + threadIdx.x; jj <= i; jj += gridDim.x * blockDim.x) {
      const unsigned long long id = (((unsigned long long)z * m + i) * m + jj) * 2ull;
      const double a = 2.0 * tune_uniform(id) - 1.0, b = 2.0 * tune_uniform(id + 1) - 1.0;
      T v;
      if constexpr (sizeof(T) == 16) v = zc{a, i == jj ? 0.0 : b};
      else v = a;
      if (!hermitian) v = (i == jj) ? from_real<T>(1.0) : (0.5 / m) * v;
      A[(size_t)i * m + jj] = v;
    }
}

template <typename T>
void tune_pencil(T* A, int m, int count, int hermitian, cudaStream_t s) {
  count_launch();
  tune_pencil_kernel<T><<<grid2d(m, m, count), 256, 0, s>>>(A, m, hermitian);
}

#define INST(T)                                                                                         \
  template void potf2<T>(T*, int, long long, int, int, DevStatus*, int, cudaStream_t);                   \
  template void trsm_block<T>(int, const T*, int, long long, T*, int, long long, int, int, int,         \
                              cudaStream_t);                                                            \
  template void hegst_diag<T>(T*, int, long long, const T*, int, long long, int, int, T*, int, long long, \
                              int, cudaStream_t);                                                       \
  template void larft<T>(const T*, int, long long, const double*, long long, int, T*, int, long long,    \
                         int, cudaStream_t);                                                            \
  template void apply_phase<T>(T*, int, long long, const double*, int, long long, const T*, long long,   \
                               int, int, int, cudaStream_t);                                            \
  template void mirror_lower<T>(T*, int, long long, int, int, cudaStream_t);                            \
  template void lowdin_factor<T>(const T*, int, long long, const double*, long long, T*, int, long long, int, \
                                 DevStatus*, int, cudaStream_t);                                           \
  template void column_phase<T>(T*, int, long long, int, int, int, cudaStream_t);                      \
  template void spinor_overlap<T>(T*, long long, const T*, int, long long, int, int, cudaStream_t);         \
  template void tune_pencil<T>(T*, int, int, int, cudaStream_t);
INST(double)
INST(zc)

}  // namespace gks
