// Shared device-side definitions for the generalized Kohn-Sham eigensolver kernels.
// Scalar types: double (real symmetric pencils) and zc (double complex, Hermitian).
// All matrices are row-major; element (i, j) of a matrix with leading dimension ld sits
// at p[i * ld + j].  Hermitian inputs are read from the lower triangle (i >= j).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gks {

struct zc {
  double x, y;
};

__host__ __device__ __forceinline__ zc mkz(double a, double b) { return zc{a, b}; }

// ---- uniform scalar helpers (double and zc) ----
__host__ __device__ __forceinline__ double conjg(double a) { return a; }
__host__ __device__ __forceinline__ zc conjg(zc a) { return zc{a.x, -a.y}; }
__host__ __device__ __forceinline__ double re(double a) { return a; }
__host__ __device__ __forceinline__ double re(zc a) { return a.x; }
__host__ __device__ __forceinline__ double im(double) { return 0.0; }
__host__ __device__ __forceinline__ double im(zc a) { return a.y; }
__host__ __device__ __forceinline__ double abs2(double a) { return a * a; }
__host__ __device__ __forceinline__ double abs2(zc a) { return a.x * a.x + a.y * a.y; }

template <typename T> __host__ __device__ __forceinline__ T from_real(double a);
template <> __host__ __device__ __forceinline__ double from_real<double>(double a) { return a; }
template <> __host__ __device__ __forceinline__ zc from_real<zc>(double a) { return zc{a, 0.0}; }
template <typename T> __host__ __device__ __forceinline__ T zero() { return from_real<T>(0.0); }

__host__ __device__ __forceinline__ zc operator+(zc a, zc b) { return zc{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ zc operator-(zc a, zc b) { return zc{a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ zc operator-(zc a) { return zc{-a.x, -a.y}; }
__host__ __device__ __forceinline__ zc operator*(zc a, zc b) {
  return zc{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
__host__ __device__ __forceinline__ zc operator*(double s, zc a) { return zc{s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ zc operator*(zc a, double s) { return zc{s * a.x, s * a.y}; }
__host__ __device__ __forceinline__ zc operator/(zc a, double s) { return zc{a.x / s, a.y / s}; }
__host__ __device__ __forceinline__ zc& operator+=(zc& a, zc b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ __forceinline__ zc& operator-=(zc& a, zc b) { a.x -= b.x; a.y -= b.y; return a; }
__host__ __device__ __forceinline__ zc operator/(zc a, zc b) {
  double d = b.x * b.x + b.y * b.y;
  return zc{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// Load through L2 only (bypassing L1): used to read data other CTAs of the same grid
// wrote before a fence.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ zc ldcg(const zc* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return zc{v.x, v.y};
}

// acc += a * b (fused where the type allows)
__device__ __forceinline__ void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void mac(zc& acc, zc a, zc b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void macc(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void macc(zc& acc, zc a, zc b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// ---- single precision (the FP32 tridiagonalization of the mixed-precision path) ----
// float for real problems, cf (complex float, interleaved) for complex ones; scalars that
// come in double (tau, alpha, beta of a product) are applied in double and rounded once.
struct cf {
  float x, y;
};
__host__ __device__ __forceinline__ float conjg(float a) { return a; }
__host__ __device__ __forceinline__ cf conjg(cf a) { return cf{a.x, -a.y}; }
__host__ __device__ __forceinline__ float re(float a) { return a; }
__host__ __device__ __forceinline__ float re(cf a) { return a.x; }
__host__ __device__ __forceinline__ float im(float) { return 0.0f; }
__host__ __device__ __forceinline__ float im(cf a) { return a.y; }
__host__ __device__ __forceinline__ float abs2(float a) { return a * a; }
__host__ __device__ __forceinline__ float abs2(cf a) { return a.x * a.x + a.y * a.y; }
template <> __host__ __device__ __forceinline__ float from_real<float>(double a) { return (float)a; }
template <> __host__ __device__ __forceinline__ cf from_real<cf>(double a) { return cf{(float)a, 0.0f}; }
__host__ __device__ __forceinline__ cf operator+(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ cf operator-(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ cf operator-(cf a) { return cf{-a.x, -a.y}; }
__host__ __device__ __forceinline__ cf operator*(cf a, cf b) {
  return cf{fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}
__host__ __device__ __forceinline__ cf operator*(double s, cf a) { return cf{(float)(s * a.x), (float)(s * a.y)}; }
__host__ __device__ __forceinline__ cf operator*(cf a, double s) { return cf{(float)(s * a.x), (float)(s * a.y)}; }
__host__ __device__ __forceinline__ cf& operator+=(cf& a, cf b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ __forceinline__ cf& operator-=(cf& a, cf b) { a.x -= b.x; a.y -= b.y; return a; }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ cf ldcg(const cf* p) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cf{v.x, v.y};
}
__device__ __forceinline__ void mac(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void mac(cf& acc, cf a, cf b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void macc(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void macc(cf& acc, cf a, cf b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// The single-precision partner of each FP64 element type.
template <typename T> struct Low;
template <> struct Low<double> { using type = float; };
template <> struct Low<zc> { using type = cf; };

// ---- warp / block reductions ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ zc warp_sum(zc v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ cf warp_sum(cf v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

// Sum over the block; every thread receives the result.  `scratch` needs 32 entries.
template <typename T>
__device__ T block_sum(T v, T* scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T r = zero<T>();
  if (wid == 0) {
    r = (lane < nw) ? scratch[lane] : zero<T>();
    r = warp_sum(r);
    if (lane == 0) scratch[0] = r;
  }
  __syncthreads();
  r = scratch[0];
  __syncthreads();
  return r;
}

// Offset of batch item z: z s1, or for a two-level batch (nb2 > 0 items per outer group)
// (z / nb2) s1 + (z % nb2) s2.
__host__ __device__ __forceinline__ long long item_off(int z, long long s1, long long s2, int nb2) {
  return nb2 > 0 ? (long long)(z / nb2) * s1 + (long long)(z % nb2) * s2 : (long long)z * s1;
}

// ---- device status word (one per batch item) ----
// Codes follow gks_status in the public header; info carries a column or iteration.
struct DevStatus {
  int code;
  int info;
};

enum : int { ST_OK = 0, ST_EINVAL = 1, ST_ENOTSPD = 2, ST_ENOCONV = 3, ST_ETIMEOUT = 6 };

__device__ __forceinline__ void set_status(DevStatus* st, int code, int info) {
  if (st == nullptr) return;
  if (atomicCAS(&st->code, 0, code) == 0) st->info = info;
}

}  // namespace gks
