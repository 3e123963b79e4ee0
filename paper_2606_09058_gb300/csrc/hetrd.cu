// One-stage Householder reduction of a Hermitian matrix to real-phased tridiagonal form
// (the dense -> tridiagonal half of the standard eigensolve of H', paper Sec. 3.1 Part
// 2-4 / Sec. 3.2 Part 3-5).
//
// Storage: lower triangle, row-major.  The reduction runs upward: step j (j = m-1 .. 2)
// annihilates column j above its super-diagonal, i.e. row j left of its sub-diagonal,
// which is one contiguous row segment in this storage.  With a = A[0:j, j],
//   u = a + ph |a| e_{j-1},  ph = a_{j-1}/|a_{j-1}|,  P_j = I - tau u' u'^H,  u' = u/u_{j-1},
// and the leading j x j block becomes P_j A P_j = A - u q^H - q u^H with
//   p = tau A u,  q = p - (tau/2)(u^H p) u.
// u' (without its unit entry) is stored in row j left of the sub-diagonal.
//
// On GB300 the Hermitian matrix-vector product that dominates each step is bound by the
// FP64 pipe, not by HBM: a complex element read once feeds two complex multiply-adds
// (16 flops per 16 bytes), above the DFMA pipe's balance point of ~0.15 flop/byte.
#include "dense.h"

namespace gks {

// Reflector for step j (one CTA): reads row j left of the diagonal (through L2: in the
// fused form other CTAs have just written it), writes u', tau[j] and the sub-diagonal.
template <typename T>
__device__ void reflector_body(T* A, int lda, int j, T* u, double* tau) {
  __shared__ double redd[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  T* row = A + (size_t)j * lda;
  double s2 = 0.0;
  for (int i = tid; i < j; i += nt) s2 += abs2(ldcg(row + i));
  const double xnorm2 = block_sum(s2, redd);
  const T alpha = conjg(ldcg(row + j - 1));
  const double tail = xnorm2 - abs2(alpha);
  if (!(tail > 0.0)) {  // nothing to annihilate: P_j = I
    for (int i = tid; i < j; i += nt) u[i] = (i == j - 1) ? from_real<T>(1.0) : zero<T>();
    if (tid == 0) tau[j] = 0.0;
    return;
  }
  const double xn = sqrt(xnorm2);
  const double aa = sqrt(abs2(alpha));
  const T ph = aa > 0.0 ? alpha * (1.0 / aa) : from_real<T>(1.0);
  const T upiv = ph * (aa + xn);                       // alpha + ph * xn
  const double beta = 2.0 / (tail + abs2(upiv));
  const T inv = conjg(upiv) * (1.0 / abs2(upiv));       // 1 / upiv
  __syncthreads();
  for (int i = tid; i < j - 1; i += nt) {
    T v = conjg(ldcg(row + i)) * inv;                 // u'_i = a_i / u_{j-1}
    u[i] = v;
    row[i] = v;
  }
  if (tid == 0) {
    u[j - 1] = from_real<T>(1.0);
    tau[j] = beta * abs2(upiv);
    row[j - 1] = conjg(ph) * (-xn);                     // lower-storage sub-diagonal
  }
}

template <typename T>
__global__ void hetrd_reflector_kernel(T* A, int lda, long long sA, int j, T* u, long long sv, double* tau,
                                       long long stau) {
  const int z = blockIdx.x;
  reflector_body<T>(A + z * sA, lda, j, u + z * sv, tau + z * stau);
}

// p = tau * A[0:j,0:j] u  (Hermitian, lower storage).  CTA b owns rows/columns
// [64b, 64b+64): its own row panel left of the diagonal plus its column panel below,
// so every CTA reads the same number of elements and no cross-CTA reduction is needed.
// The last CTA to finish (atomic ticket after a fence; nothing waits) then forms
// q = p - (tau/2)(u^H p) u in place of p.
template <typename T>
__global__ void __launch_bounds__(256) hetrd_hemv_kernel(const T* A, int lda, long long sA, int j, const T* u,
                                                         T* p, long long sv, const double* tau, long long stau,
                                                         int* ticket) {
  __shared__ T part[4][64];
  __shared__ T rowacc[64];
  __shared__ T red[32];
  __shared__ int last;
  const int z = blockIdx.y, tid = threadIdx.x;
  A += z * sA;
  u += z * sv;
  p += z * sv;
  const double t = tau[z * stau + j];
  const int c0 = blockIdx.x * 64;
  const int cend = min(c0 + 64, j);
  // row part: rows r in [c0, cend), columns 0..r ; one warp per row
  const int warp = tid >> 5, lane = tid & 31;
  for (int r = c0 + warp; r < cend; r += 8) {
    const T* ar = A + (size_t)r * lda;
    T s = zero<T>();
    for (int c = lane; c <= r; c += 32) mac(s, ar[c], u[c]);
    s = warp_sum(s);
    if (lane == 0) rowacc[r - c0] = s;
  }
  // column part: columns c in [c0, cend), rows r > c
  const int cc = tid & 63, g = tid >> 6;
  const int c = c0 + cc;
  T s = zero<T>();
  if (c < cend) {
    for (int r = c0 + g; r < j; r += 4)
      if (r > c) macc(s, A[(size_t)r * lda + c], u[r]);
  }
  part[g][cc] = s;
  __syncthreads();
  if (tid < 64 && c0 + tid < cend) {
    T y = rowacc[tid] + part[0][tid] + part[1][tid] + part[2][tid] + part[3][tid];
    p[c0 + tid] = t * y;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(ticket + z, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  if (tid == 0) ticket[z] = 0;
  T d = zero<T>();
  for (int i = tid; i < j; i += blockDim.x) macc(d, u[i], ldcg(p + i));
  d = block_sum(d, red);
  const T K = (0.5 * t) * d;
  for (int i = tid; i < j; i += blockDim.x) p[i] = ldcg(p + i) - K * u[i];
}

// A[0:j,0:j] (lower) -= u q^H + q u^H, one CTA per row; the last CTA of each batch item
// then computes the reflector of step j-1 from the freshly updated row j-1.
template <typename T>
__global__ void hetrd_rank2_kernel(T* A, int lda, long long sA, int j, T* u, const T* q, long long sv,
                                   double* tau, long long stau, int* ticket) {
  __shared__ int last;
  const int z = blockIdx.y, r = blockIdx.x;
  A += z * sA;
  u += z * sv;
  q += z * sv;
  tau += z * stau;
  if (tau[j] != 0.0) {
    const T ur = u[r], qr = q[r];
    T* ar = A + (size_t)r * lda;
    for (int c = threadIdx.x; c <= r; c += blockDim.x) {
      T v = ar[c];
      v -= ur * conjg(q[c]) + qr * conjg(u[c]);
      ar[c] = v;
    }
  }
  if (j - 1 < 2) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket + z, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  if (threadIdx.x == 0) ticket[z] = 0;
  __syncthreads();
  reflector_body<T>(A, lda, j - 1, u, tau);
}

// d_i = Re A_ii, e_i = |A_{i+1,i}|, ph_0 = 1, ph_{i+1} = ph_i A_{i+1,i}/|A_{i+1,i}|.
template <typename T>
__global__ void hetrd_finish_kernel(const T* A, int lda, long long sA, int m, double* d, double* e, long long sde,
                                    T* ph, long long sph) {
  const int z = blockIdx.x;
  A += z * sA;
  d += z * sde;
  e += z * sde;
  ph += z * sph;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    d[i] = re(A[(size_t)i * lda + i]);
    if (i + 1 < m) e[i] = sqrt(abs2(A[(size_t)(i + 1) * lda + i]));
  }
  if (threadIdx.x == 0) {
    T cur = from_real<T>(1.0);
    ph[0] = cur;
    for (int i = 0; i + 1 < m; i++) {
      T s = A[(size_t)(i + 1) * lda + i];
      double a = sqrt(abs2(s));
      if (a > 0.0) cur = cur * (s * (1.0 / a));
      ph[i + 1] = cur;
    }
  }
}

// V[:, c] = u'_{j1-c} (rows 0..j1-1), tb[c] = tau[j1-c].
template <typename T>
__global__ void gather_reflectors_kernel(const T* A, int lda, long long sA, const double* tau, long long stau,
                                         int j0, int j1, T* V, int ldv, long long sV, double* tb, long long stb) {
  const int z = blockIdx.z;
  A += z * sA;
  tau += z * stau;
  V += z * sV;
  tb += z * stb;
  const int nbb = j1 - j0 + 1;
  for (int i = blockIdx.y; i < j1; i += gridDim.y)
    for (int c = threadIdx.x; c < nbb; c += blockDim.x) {
      int jj = j1 - c;
      T v = zero<T>();
      if (i < jj - 1) v = A[(size_t)jj * lda + i];
      else if (i == jj - 1) v = from_real<T>(1.0);
      V[(size_t)i * ldv + c] = v;
      if (i == 0) tb[c] = tau[jj];
    }
}

template <typename T>
void hetrd_reflector(T* A, int lda, long long sA, int j, T* u, long long sv, double* tau, long long stau, int count,
                     cudaStream_t s) {
  count_launch();
  hetrd_reflector_kernel<T><<<count, 256, 0, s>>>(A, lda, sA, j, u, sv, tau, stau);
}

template <typename T>
void hetrd_hemv(const T* A, int lda, long long sA, int j, const T* u, T* p, long long sv, const double* tau,
                long long stau, int* ticket, int count, cudaStream_t s) {
  count_launch();
  hetrd_hemv_kernel<T><<<dim3((j + 63) / 64, count), 256, 0, s>>>(A, lda, sA, j, u, p, sv, tau, stau, ticket);
}

template <typename T>
void hetrd_rank2(T* A, int lda, long long sA, int j, T* u, const T* q, long long sv, double* tau, long long stau,
                 int* ticket, int count, cudaStream_t s) {
  count_launch();
  hetrd_rank2_kernel<T><<<dim3(j, count), 256, 0, s>>>(A, lda, sA, j, u, q, sv, tau, stau, ticket);
}

template <typename T>
void hetrd_finish(const T* A, int lda, long long sA, int m, double* d, double* e, long long sde, T* ph,
                  long long sph, int count, cudaStream_t s) {
  count_launch();
  hetrd_finish_kernel<T><<<count, 256, 0, s>>>(A, lda, sA, m, d, e, sde, ph, sph);
}

template <typename T>
void gather_reflectors(const T* A, int lda, long long sA, const double* tau, long long stau, int j0, int j1,
                       T* V, int ldv, long long sV, double* tb, long long stb, int count, cudaStream_t s) {
  dim3 grid(1, j1 < 2048 ? j1 : 2048, count);
  count_launch();
  gather_reflectors_kernel<T><<<grid, 64, 0, s>>>(A, lda, sA, tau, stau, j0, j1, V, ldv, sV, tb, stb);
}

#define INST(T)                                                                                            \
  template void hetrd_reflector<T>(T*, int, long long, int, T*, long long, double*, long long, int,         \
                                   cudaStream_t);                                                          \
  template void hetrd_hemv<T>(const T*, int, long long, int, const T*, T*, long long, const double*,         \
                              long long, int*, int, cudaStream_t);                                         \
  template void hetrd_rank2<T>(T*, int, long long, int, T*, const T*, long long, double*, long long, int*,   \
                               int, cudaStream_t);                                                         \
  template void hetrd_finish<T>(const T*, int, long long, int, double*, double*, long long, T*, long long,   \
                                int, cudaStream_t);                                                        \
  template void gather_reflectors<T>(const T*, int, long long, const double*, long long, int, int, T*, int, \
                                     long long, double*, long long, int, cudaStream_t);
INST(double)
INST(zc)

}  // namespace gks
