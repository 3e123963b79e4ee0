// Two-stage reduction of a Hermitian matrix to real tridiagonal form (the alternative to
// the one-stage panel Householder of hetrd.cu; paper Sec. 6 names the one-stage
// reduction's matrix-vector half as the limit of the GPU eigensolver):
//
//   stage 1 (dense -> band, bandwidth b): for the panel of columns [k, k+b), QR of the block
//     below the band by Householder reflectors H_c = I - tau_c v_c v_c^H (v_c(0) = 1, complex
//     tau, real beta: H_c^H x = beta e_1), then the two-sided update of the trailing block
//     with Q = H_0 ... H_{kb-1} = I - V T V^H:  X = A22 V T,  W = X - V (T^H V^H X)/2,
//     A22 <- A22 - V W^H - W V^H  (products on the tensor cores);
//   stage 2 (band -> tridiagonal, bulge chasing): sweep i annihilates column i below the
//     subdiagonal with a reflector on rows i+1 .. i+b, and chases the fill it creates down
//     the band window by window (window j: rows q0 = i+1+j b .. q0+b-1, annihilating the
//     previous window's first column below q0).  Each window is a similarity H^H T H on its
//     rows/columns; sweeps run concurrently, sweep i trailing sweep i-1 by a fixed lag.
//
// The reflectors follow the oracle's convention (LAPACK zlarfg: complex tau, real beta), so
// the band matrix and the tridiagonal match the oracle's stage references entry by entry.
#include <algorithm>

#include "dense.h"

namespace gks {

__device__ __forceinline__ double absq(double a) { return a * a; }
__device__ __forceinline__ double absq(zc a) { return a.x * a.x + a.y * a.y; }

// Householder vector of x (length L, x0 = alpha, ||x[1:]||^2 = tail): tau and the scale of
// v[1:] = x[1:] / (alpha - beta); beta real.  tail == 0 and Im alpha == 0: tau = 0, v = e_1.
template <typename T>
__device__ __forceinline__ void householder_coef(T alpha, double tail, T* tau, T* scale, double* beta) {
  if (tail == 0.0 && im(alpha) == 0.0) {
    *tau = zero<T>();
    *scale = zero<T>();
    *beta = re(alpha);
    return;
  }
  const double a2 = absq(alpha) + tail;
  const double bt = -copysign(sqrt(a2), re(alpha));
  *beta = bt;
  *tau = (from_real<T>(bt) - alpha) * (1.0 / bt);  // (beta - alpha) / beta
  const T den = alpha - from_real<T>(bt);
  *scale = conjg(den) * (1.0 / absq(den));          // 1 / (alpha - beta)
}

// ------------------------------------------------------------------ stage 1: panel QR
//
// One CTA per item.  P = A[r0:r0+m, k:k+b] (leading dimension lda) is factored in place:
// reflector c from P[c:, c] (c < kb), P[c, c] = beta, v_c stored below the diagonal
// (unit entry implied), H_c^H applied to the columns right of c (all b columns of the
// panel).  taus (kb, type T) out.  Rows are read in 1 KB segments: warp w walks rows
// r = w, w + 32, ..., lane l covers columns l and l + 32.
template <typename T>
__global__ void __launch_bounds__(1024) panel_qr_kernel(T* A, int lda, long long sA, int r0, int k, int m, int b,
                                                        int kb, T* taus, long long stau) {
  __shared__ T wpart[32][65];
  __shared__ T wsum[64];
  __shared__ double red[32];
  __shared__ T coef[2];  // tau, scale
  const int z = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  T* P = A + z * sA + (size_t)r0 * lda + k;
  taus += z * stau;
  for (int c = 0; c < kb; c++) {
    // norm of P[c+1:, c]
    double s2 = 0.0;
    for (int r = c + 1 + tid; r < m; r += blockDim.x) s2 += absq(P[(size_t)r * lda + c]);
    s2 = warp_sum(s2);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    if (warp == 0) {
      double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) {
        T tau, scale;
        double beta;
        householder_coef<T>(P[(size_t)c * lda + c], t, &tau, &scale, &beta);
        coef[0] = tau;
        coef[1] = scale;
        taus[c] = tau;
        P[(size_t)c * lda + c] = from_real<T>(beta);
      }
    }
    __syncthreads();
    const T tau = coef[0], scale = coef[1];
    // v[1:] = x[1:] * scale, stored in place
    for (int r = c + 1 + tid; r < m; r += blockDim.x) P[(size_t)r * lda + c] = P[(size_t)r * lda + c] * scale;
    __syncthreads();
    // w_j = sum_r conj(v_r) P[r][j] for columns j in (c, b): rows by warp, columns by lane
    const int ncol = b - c - 1;
    if (ncol > 0) {
      T acc0 = zero<T>(), acc1 = zero<T>();
      for (int r = c + warp; r < m; r += 32) {
        const T v = (r == c) ? from_real<T>(1.0) : P[(size_t)r * lda + c];
        const T* row = P + (size_t)r * lda + c + 1;
        if (lane < ncol) macc(acc0, v, row[lane]);
        if (lane + 32 < ncol) macc(acc1, v, row[lane + 32]);
      }
      wpart[warp][lane] = acc0;
      wpart[warp][lane + 32] = acc1;
      __syncthreads();
      if (tid < ncol) {
        T s = zero<T>();
        for (int w = 0; w < 32; w++) s += wpart[w][tid];
        wsum[tid] = conjg(tau) * s;  // the factor of H^H = I - conj(tau) v v^H
      }
      __syncthreads();
      for (int r = c + warp; r < m; r += 32) {
        const T v = (r == c) ? from_real<T>(1.0) : P[(size_t)r * lda + c];
        T* row = P + (size_t)r * lda + c + 1;
        if (lane < ncol) row[lane] = row[lane] - v * wsum[lane];
        if (lane + 32 < ncol) row[lane + 32] = row[lane + 32] - v * wsum[lane + 32];
      }
      __syncthreads();
    }
  }
}

// V (m x kb, ldv, item stride sV): unit lower trapezoidal copy of the panel's reflectors.
template <typename T>
__global__ void panel_v_kernel(const T* A, int lda, long long sA, int r0, int k, int m, int kb, T* V, int ldv,
                               long long sV) {
  const int z = blockIdx.z;
  A += z * sA + (size_t)r0 * lda + k;
  V += z * sV;
  for (int r = blockIdx.y * blockDim.y + threadIdx.y; r < m; r += gridDim.y * blockDim.y)
    for (int c = threadIdx.x; c < kb; c += blockDim.x) {
      T v = zero<T>();
      if (r == c) v = from_real<T>(1.0);
      else if (r > c) v = A[(size_t)r * lda + c];
      V[(size_t)r * ldv + c] = v;
    }
}

// T factor of H_0 ... H_{k-1} = I - V T V^H with complex taus: T upper triangular,
// T_ii = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i] with G = V^H V (k x k).
template <typename T>
__global__ void larft_tau_kernel(const T* G, int ldG, long long sG, const T* tau, long long stau, int k, T* Tm,
                                 int ldT, long long sT) {
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
    const T ti = tau[i];
    for (int r = tid; r < i; r += nt) {
      T s = zero<T>();
      for (int c = r; c < i; c++) mac(s, t[r * k + c], G[(size_t)c * ldG + i]);
      tmp[r] = s;
    }
    __syncthreads();
    for (int r = tid; r < i; r += nt) t[r * k + i] = zero<T>() - ti * tmp[r];
    if (tid == 0) t[i * k + i] = ti;
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += nt) Tm[(size_t)(e / k) * ldT + (e % k)] = t[e];
}

// Zero the panel's column entries below the band (rows r0+c+1.. of column k+c, c < kb) in
// the dense matrix after its reflectors have been copied out.
template <typename T>
__global__ void panel_clear_kernel(T* A, int lda, long long sA, int r0, int k, int m, int kb) {
  const int z = blockIdx.z;
  A += z * sA + (size_t)r0 * lda + k;
  for (int r = blockIdx.y * blockDim.y + threadIdx.y; r < m; r += gridDim.y * blockDim.y)
    for (int c = threadIdx.x; c < kb && c < r; c += blockDim.x) A[(size_t)r * lda + c] = zero<T>();
}

// ------------------------------------------------------------------ band storage
//
// Lower band of the Hermitian band matrix with room for the bulges of stage 2:
// Bd[j * W + d] = T[j + d][j] for 0 <= d < W (W = 2b + 1), zero where j + d >= m.
template <typename T>
__global__ void band_pack_kernel(const T* A, int lda, long long sA, T* Bd, int W, long long sB, int m, int b) {
  const int z = blockIdx.z;
  A += z * sA;
  Bd += z * sB;
  for (int j = blockIdx.y; j < m; j += gridDim.y)
    for (int d = threadIdx.x; d < W; d += blockDim.x) {
      T v = zero<T>();
      if (d <= b && j + d < m) v = A[(size_t)(j + d) * lda + j];
      Bd[(size_t)j * W + d] = v;
    }
}

// Dense full Hermitian matrix from the band storage (stage tests): lower band entries and
// their mirror, zero elsewhere.
template <typename T>
__global__ void band_unpack_kernel(const T* Bd, int W, long long sB, T* A, int lda, long long sA, int m) {
  const int z = blockIdx.z;
  Bd += z * sB;
  A += z * sA;
  for (int i = blockIdx.y; i < m; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
      const int lo = i >= j ? j : i, hi = i >= j ? i : j;
      T v = zero<T>();
      if (hi - lo < W) v = Bd[(size_t)lo * W + (hi - lo)];
      A[(size_t)i * lda + j] = (i >= j) ? v : conjg(v);
    }
}

// ------------------------------------------------------------------ stage 2: bulge chasing
//
// Tasks: sweep i (0 <= i < m-1), window j: rows K = [q0, q0+L) with q0 = i + 1 + j b and
// L = min(b, m - q0); the reflector comes from column cc (cc = i for j = 0, the previous
// window's first row q0 - b otherwise) on rows K.  The similarity H^H T H touches, in the
// lower band: the left block rows K x columns [cc, q0) (column cc becomes beta e_1), the
// diagonal block K x K, and the block below, rows [q0+L, min(m, q0+2b)) x columns K (the
// next bulge).  The last sweep (i = m-2) only makes T[m-1][m-2] real.
//
// Scheduling: persistent workers (grid.x per item, all resident: cooperative launch);
// worker p takes sweeps p, p + P, ...; task j of sweep i starts once sweep i-1 has finished
// task j+3 (or all of its tasks), which keeps their regions disjoint.  prog[i] counts the
// finished tasks of sweep i.  Every wait is bounded: past wait_limit cycles the worker sets
// err and the status (GKS_ETIMEOUT) and all workers stop.
__device__ __forceinline__ double ldcg_s(const double* p) { return __ldcg(p); }
__device__ __forceinline__ zc ldcg_s(const zc* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return zc{v.x, v.y};
}
__device__ __forceinline__ void stcg_s(double* p, double v) { __stcg(p, v); }
__device__ __forceinline__ void stcg_s(zc* p, zc v) { __stcg(reinterpret_cast<double2*>(p), make_double2(v.x, v.y)); }

__device__ __forceinline__ int chase_ntasks(int i, int m, int b) { return (m - 2 - i) / b + 1; }

template <typename T>
__global__ void __launch_bounds__(256) chase_kernel(T* Bd, int W, long long sB, int m, int b, T* V2, long long sV2,
                                                    T* tau2, int ldt, long long sT2, int* prog, long long sprog,
                                                    int* err, DevStatus* st, long long wait_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Lb = reinterpret_cast<T*>(smem_raw);  // b x b: rows K, columns [cc, q0)
  T* Db = Lb + b * b;                       // b x b: K x K (full Hermitian)
  T* Bb = Db + b * b;                       // b x b: rows below K, columns K
  T* vs = Bb + b * b;                       // b
  T* ys = vs + b;                           // b: D v, later w
  T* ws = ys + b;                           // b: left / below products
  __shared__ T coef[2];
  __shared__ double bsh, ash;
  __shared__ int stop;
  const int z = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
  Bd += z * sB;
  V2 += z * sV2;
  tau2 += z * sT2;
  prog += z * sprog;
  const int P = gridDim.x, nsweep = m - 1;
  for (int i = blockIdx.x; i < nsweep; i += P) {
    const int ntask = chase_ntasks(i, m, b);
    for (int j = 0; j < ntask; j++) {
      // ---- wait for sweep i-1 to be 4 tasks ahead (bounded)
      if (tid == 0) {
        stop = 0;
        if (i > 0) {
          const int need = min(j + 4, chase_ntasks(i - 1, m, b));
          const volatile int* pv = prog + (i - 1);
          const long long t0 = clock64();
          while (*pv < need) {
            if (*reinterpret_cast<volatile int*>(err)) { stop = 1; break; }
            if (clock64() - t0 > wait_limit) {
              atomicExch(err, 1);
              set_status(st ? st + z : nullptr, ST_ETIMEOUT, i);
              stop = 1;
              break;
            }
          }
          __threadfence();
        }
      }
      __syncthreads();
      if (stop) return;
      const int q0 = i + 1 + j * b;
      const int L = min(b, m - q0);
      const int cc = j == 0 ? i : q0 - b;
      const int wl = q0 - cc;                    // left block width (1 or b)
      const int hb = max(0, min(m, q0 + 2 * b) - (q0 + L));
      // ---- reflector from column cc, rows K
      if (tid < 32) {
        T x = zero<T>();
        if (tid < L) x = ldcg_s(Bd + (size_t)cc * W + (q0 - cc + tid));
        double t2 = (tid >= 1 && tid < L) ? absq(x) : 0.0;
        t2 = warp_sum(t2);
        T al;  // alpha = x_0, held by lane 0
        if constexpr (sizeof(T) == 16) {
          al = T{__shfl_sync(0xffffffffu, re(x), 0), __shfl_sync(0xffffffffu, im(x), 0)};
        } else {
          al = from_real<T>(__shfl_sync(0xffffffffu, re(x), 0));
        }
        T tau, scale;
        double beta;
        householder_coef<T>(al, t2, &tau, &scale, &beta);
        if (tid < L) vs[tid] = (tid == 0) ? from_real<T>(1.0) : x * scale;
        if (tid == 0) {
          coef[0] = tau;
          bsh = beta;
        }
      }
      // ---- load the blocks
      for (int e = tid; e < L * wl; e += nt) {
        const int t = e / wl, c = e % wl;
        Lb[t * b + c] = ldcg_s(Bd + (size_t)(cc + c) * W + (q0 + t - cc - c));
      }
      for (int e = tid; e < L * L; e += nt) {
        const int t = e / L, u = e % L;
        if (t >= u) {
          const T v = ldcg_s(Bd + (size_t)(q0 + u) * W + (t - u));
          Db[t * b + u] = v;
          if (t > u) Db[u * b + t] = conjg(v);
        }
      }
      for (int e = tid; e < hb * L; e += nt) {
        const int r = e / L, u = e % L;
        Bb[r * b + u] = ldcg_s(Bd + (size_t)(q0 + u) * W + (L + r - u));
      }
      __syncthreads();
      const T tau = coef[0];
      const T ctau = conjg(tau);
      // ---- left block: H^H Lb (column 0 is x -> beta e_1)
      for (int c = 1 + tid; c < wl; c += nt) {
        T s = zero<T>();
        for (int t = 0; t < L; t++) macc(s, vs[t], Lb[t * b + c]);
        ws[c] = ctau * s;
      }
      // ---- diagonal block: y = D v
      for (int t = tid; t < L; t += nt) {
        T s = zero<T>();
        for (int u = 0; u < L; u++) mac(s, Db[t * b + u], vs[u]);
        ys[t] = s;
      }
      __syncthreads();
      if (tid == 0) {
        double a = 0.0;
        for (int t = 0; t < L; t++) {
          T p = zero<T>();
          macc(p, vs[t], ys[t]);
          a += re(p);
        }
        ash = a;
      }
      for (int e = tid; e < L * wl; e += nt) {
        const int t = e / wl, c = e % wl;
        if (c == 0) Lb[t * b] = (t == 0) ? from_real<T>(bsh) : zero<T>();
        else Lb[t * b + c] = Lb[t * b + c] - vs[t] * ws[c];
      }
      __syncthreads();
      // w = tau y - |tau|^2 (v^H D v) v / 2
      for (int t = tid; t < L; t += nt) ys[t] = tau * ys[t] - (0.5 * absq(tau) * ash) * vs[t];
      __syncthreads();
      for (int e = tid; e < L * L; e += nt) {
        const int t = e / L, u = e % L;
        Db[t * b + u] = Db[t * b + u] - ys[t] * conjg(vs[u]) - vs[t] * conjg(ys[u]);
      }
      // ---- below block: Bb H = Bb - tau (Bb v) v^H
      for (int r = tid; r < hb; r += nt) {
        T s = zero<T>();
        for (int u = 0; u < L; u++) mac(s, Bb[r * b + u], vs[u]);
        ws[r] = tau * s;
      }
      __syncthreads();
      for (int e = tid; e < hb * L; e += nt) {
        const int r = e / L, u = e % L;
        Bb[r * b + u] = Bb[r * b + u] - ws[r] * conjg(vs[u]);
      }
      __syncthreads();
      // ---- store the blocks and the reflector
      for (int e = tid; e < L * wl; e += nt) {
        const int t = e / wl, c = e % wl;
        stcg_s(Bd + (size_t)(cc + c) * W + (q0 + t - cc - c), Lb[t * b + c]);
      }
      for (int e = tid; e < L * L; e += nt) {
        const int t = e / L, u = e % L;
        if (t >= u) {
          T v = Db[t * b + u];
          if (t == u) v = from_real<T>(re(v));
          stcg_s(Bd + (size_t)(q0 + u) * W + (t - u), v);
        }
      }
      for (int e = tid; e < hb * L; e += nt) {
        const int r = e / L, u = e % L;
        stcg_s(Bd + (size_t)(q0 + u) * W + (L + r - u), Bb[r * b + u]);
      }
      for (int t = tid; t < L; t += nt) V2[(size_t)i * m + j * b + t] = vs[t];
      if (tid == 0) tau2[(size_t)i * ldt + j] = tau;
      __threadfence();  // every thread's band stores reach L2 before the progress flag
      __syncthreads();
      if (tid == 0) atomicExch(prog + i, j + 1);
    }
  }
}

// d_i = Re T_ii, e_i = T_{i+1,i} (real after the chase) from the band storage.
template <typename T>
__global__ void band_tridiag_kernel(const T* Bd, int W, long long sB, int m, double* d, double* e, long long sde) {
  const int z = blockIdx.y;
  Bd += z * sB;
  d += z * sde;
  e += z * sde;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    d[i] = re(Bd[(size_t)i * W]);
    e[i] = i + 1 < m ? re(Bd[(size_t)i * W + 1]) : 0.0;
  }
}

// ------------------------------------------------------------------ Q2 blocks
//
// Block (g, j) of the chase's reflectors: sweeps s = g nbs + c (c < nbs), window j, as the
// compact-WY factor H_{s0,j} H_{s0+1,j} ... = I - V T V^H on rows [top, top + hp) with
// top = g nbs + 1 + j b: V[c + t][c] = v_{s,j}[t] (reflector rows shift by one per sweep),
// zero elsewhere; a missing reflector (past the last sweep or window) is the identity
// (tau = 0).  Wavefront blocks g = g0 .. g0 + nblk - 1 with j = j0 + 2 (g - g0) are gathered
// for every item: Vw[z][blk] (hp x nbs), tw[z][blk] (nbs).
template <typename T>
__global__ void q2_gather_kernel(const T* V2, long long sV2, const T* tau2, int ldt, long long sT2, int m, int b,
                                 int nbs, int hp, int g0, int j0, int nblk, T* Vw, T* tw) {
  const int z = blockIdx.z, blk = blockIdx.y;
  const int g = g0 + blk, j = j0 + 2 * blk;
  V2 += z * sV2;
  tau2 += z * sT2;
  T* V = Vw + ((size_t)z * nblk + blk) * hp * nbs;
  T* tv = tw + ((size_t)z * nblk + blk) * nbs;
  const int nsweep = m - 1;
  for (int e = threadIdx.x; e < hp * nbs; e += blockDim.x) {
    const int r = e / nbs, c = e % nbs;
    const int s = g * nbs + c;
    T v = zero<T>();
    if (s < nsweep && j < chase_ntasks(s, m, b)) {
      const int q0 = s + 1 + j * b, L = min(b, m - q0), t = r - c;
      if (t >= 0 && t < L) v = V2[(size_t)s * m + j * b + t];
    }
    V[(size_t)r * nbs + c] = v;
  }
  for (int c = threadIdx.x; c < nbs; c += blockDim.x) {
    const int s = g * nbs + c;
    tv[c] = (s < nsweep && j < chase_ntasks(s, m, b)) ? tau2[(size_t)s * ldt + j] : zero<T>();
  }
}

// Real Z into the element type, rows [0, m) of the padded X (ldx), padding rows zeroed.
template <typename T>
__global__ void widen_pad_kernel(const double* Z, int ldz, long long sZ, T* X, int ldx, long long sX, int m,
                                 int rows, int cols) {
  const int zi = blockIdx.z;
  Z += zi * sZ;
  X += zi * sX;
  for (int i = blockIdx.y; i < rows; i += gridDim.y)
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x)
      X[(size_t)i * ldx + c] = i < m ? from_real<T>(Z[(size_t)i * ldz + c]) : zero<T>();
}

// Multi-CTA form of the panel QR: the panel's rows are split over G CTAs per item (rows
// [g R, g R + R)), each keeping its rows in shared memory for the whole panel.  Per column,
// two grid barriers: after the partial sums of the column's squared norm (and the pivot
// entry, published by its owner), every CTA forms the same reflector from the G partials
// summed in a fixed order; after the partial sums of v^H P for the columns to the right,
// every CTA forms w and updates its rows.  The same arithmetic as panel_qr_kernel up to
// the order of the sums.  The barrier is a global arrival counter (grid of G x count CTAs,
// all resident: cooperative launch); every wait is bounded by wait_limit cycles, after
// which the CTA sets err and the status (ETIMEOUT) and all CTAs leave.
struct QrScratch {
  double* pn;      // [count][G] partial squared norms
  void* pw;        // [count][G][32] partial v^H P (type T)
  void* palpha;    // [count] pivot entries (type T)
  unsigned* bar;   // arrival counter
  int* err;
};

__device__ __forceinline__ bool grid_wait(unsigned* bar, unsigned target, int* err, DevStatus* st, int info,
                                          long long limit, int* stop) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const volatile unsigned* pb = bar;
    const long long t0 = clock64();
    int s = 0;
    while (*pb < target) {
      if (*reinterpret_cast<volatile int*>(err)) {
        s = 1;
        break;
      }
      if (clock64() - t0 > limit) {
        atomicExch(err, 1);
        set_status(st, ST_ETIMEOUT, info);
        s = 1;
        break;
      }
    }
    __threadfence();
    *stop = s;
  }
  __syncthreads();
  return *stop == 0;
}

template <typename T>
__global__ void __launch_bounds__(256) panel_qr_coop_kernel(T* A, int lda, long long sA, int r0, int k, int m, int b,
                                                            int kb, T* taus, long long stau, int G, int R,
                                                            QrScratch q, DevStatus* st, long long limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);  // R x (b + 1)
  const int ld = b + 1;
  __shared__ double red[8];
  __shared__ T wpart[8][32];
  __shared__ T wsum[32];
  __shared__ T coef[2];
  __shared__ int stop;
  const int g = blockIdx.x, z = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q0 = g * R, q1 = min(m, q0 + R), nr = max(0, q1 - q0);
  const unsigned ncta = gridDim.x * gridDim.y;
  unsigned inst = 0;
  T* Ag = A + z * sA + (size_t)r0 * lda + k;
  taus += z * stau;
  double* pn = q.pn + (size_t)z * G;
  T* pw = static_cast<T*>(q.pw) + (size_t)z * G * 32;
  T* pal = static_cast<T*>(q.palpha) + z;
  for (int e = tid; e < nr * b; e += blockDim.x) {
    const int r = e / b, cc = e % b;
    P[r * ld + cc] = Ag[(size_t)(q0 + r) * lda + cc];
  }
  __syncthreads();
  for (int c = 0; c < kb; c++) {
    // partial squared norm of column c below row c, and the pivot entry from its owner
    double s2 = 0.0;
    for (int r = max(c + 1 - q0, 0) + tid; r < nr; r += blockDim.x) s2 += absq(P[r * ld + c]);
    s2 = warp_sum(s2);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; w++) t += red[w];
      __stcg(pn + g, t);
      if (c >= q0 && c < q1) stcg_s(pal, P[(c - q0) * ld + c]);
    }
    if (!grid_wait(q.bar, ++inst * ncta, q.err, st ? st + z : nullptr, c, limit, &stop)) return;
    if (tid == 0) {
      double t = 0.0;
      for (int h = 0; h < G; h++) t += __ldcg(pn + h);
      T tau, scale;
      double beta;
      householder_coef<T>(ldcg_s(pal), t, &tau, &scale, &beta);
      coef[0] = tau;
      coef[1] = scale;
      if (g == 0) taus[c] = tau;
      if (c >= q0 && c < q1) P[(c - q0) * ld + c] = from_real<T>(beta);
    }
    __syncthreads();
    const T tau = coef[0], scale = coef[1];
    for (int r = max(c + 1 - q0, 0) + tid; r < nr; r += blockDim.x) P[r * ld + c] = P[r * ld + c] * scale;
    __syncthreads();
    // partial sums of conj(v_r) P[r][j] for the columns j > c (v_c = 1)
    const int ncol = b - c - 1;
    const int rs = max(c - q0, 0);
    T acc = zero<T>();
    if (lane < ncol)
      for (int r = rs + warp; r < nr; r += 8) {
        const T v = (q0 + r == c) ? from_real<T>(1.0) : P[r * ld + c];
        macc(acc, v, P[r * ld + c + 1 + lane]);
      }
    wpart[warp][lane] = acc;
    __syncthreads();
    if (tid < ncol) {
      T t = zero<T>();
      for (int w = 0; w < 8; w++) t += wpart[w][tid];
      stcg_s(pw + (size_t)g * 32 + tid, t);
    }
    if (!grid_wait(q.bar, ++inst * ncta, q.err, st ? st + z : nullptr, c, limit, &stop)) return;
    if (tid < ncol) {
      T t = zero<T>();
      for (int h = 0; h < G; h++) t += ldcg_s(pw + (size_t)h * 32 + tid);
      wsum[tid] = conjg(tau) * t;
    }
    __syncthreads();
    for (int e = tid; e < (nr - rs) * ncol; e += blockDim.x) {
      const int r = rs + e / ncol, j = c + 1 + e % ncol;
      const T v = (q0 + r == c) ? from_real<T>(1.0) : P[r * ld + c];
      P[r * ld + j] = P[r * ld + j] - v * wsum[j - c - 1];
    }
    __syncthreads();
  }
  for (int e = tid; e < nr * b; e += blockDim.x) {
    const int r = e / b, cc = e % b;
    Ag[(size_t)(q0 + r) * lda + cc] = P[r * ld + cc];
  }
}

// ------------------------------------------------------------------ launchers

// Panel QR: the multi-CTA form when its grid fits the GPU at once (cooperative launch),
// else one CTA per item.  scratch: qr_scratch_bytes(count, sizeof(T)) bytes.
size_t qr_scratch_bytes(int count, int es) {
  return 256 + (size_t)count * kQrMaxG * (8 + 32 * (size_t)es) + (size_t)count * es;
}

template <typename T>
void panel_qr(T* A, int lda, long long sA, int r0, int k, int m, int b, int kb, T* taus, long long stau, int count,
              void* scratch, DevStatus* st, long long wait_limit, cudaStream_t s) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  // rows per CTA: the most CTAs that fit at once (each CTA's rows within 200 KB of shared
  // memory, at least 16 rows per CTA, at most kQrMaxG CTAs per item)
  const size_t row_bytes = (size_t)(b + 1) * sizeof(T);
  const int rmax = (int)((200 * 1024) / row_bytes);
  const int gmin = (m + rmax - 1) / rmax;
  int G = std::max(gmin, std::min({kQrMaxG, (m + 15) / 16, std::max(1, sms * 2 / std::max(1, count))}));
  int R = (m + G - 1) / G;
  size_t sm = (size_t)R * row_bytes;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(panel_qr_coop_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_qr_coop_kernel<T>, 256, sm);
  int items = per_sm > 0 ? (per_sm * sms) / G : 0;
  if (G > kQrMaxG || items < 1) {
    count_launch();
    panel_qr_kernel<T><<<count, 1024, 0, s>>>(A, lda, sA, r0, k, m, b, kb, taus, stau);
    return;
  }
  items = std::min(items, count);
  char* base = static_cast<char*>(scratch);
  QrScratch q;
  q.bar = reinterpret_cast<unsigned*>(base);
  q.err = reinterpret_cast<int*>(base + 64);
  q.pn = reinterpret_cast<double*>(base + 256);
  q.pw = base + 256 + (size_t)count * kQrMaxG * 8;
  q.palpha = base + 256 + (size_t)count * kQrMaxG * (8 + 32 * sizeof(T));
  for (int z0 = 0; z0 < count; z0 += items) {
    const int cnt = std::min(items, count - z0);
    T* Az = A + z0 * sA;
    T* tz = taus + z0 * stau;
    DevStatus* sz = st ? st + z0 : nullptr;
    cudaMemsetAsync(base, 0, 128, s);
    void* args[] = {&Az, &lda, &sA, &r0, &k, &m, &b, &kb, &tz, &stau, &G, &R, &q, &sz, &wait_limit};
    count_launch();
    if (cudaLaunchCooperativeKernel((const void*)panel_qr_coop_kernel<T>, dim3(G, cnt), dim3(256), args, sm, s) !=
        cudaSuccess) {
      cudaGetLastError();
      panel_qr_kernel<T><<<cnt, 1024, 0, s>>>(Az, lda, sA, r0, k, m, b, kb, tz, stau);
    }
  }
}

template <typename T>
void panel_v(const T* A, int lda, long long sA, int r0, int k, int m, int kb, T* V, int ldv, long long sV, int count,
             cudaStream_t s) {
  count_launch();
  panel_v_kernel<T><<<dim3(1, (m + 7) / 8 < 1024 ? (m + 7) / 8 : 1024, count), dim3(32, 8), 0, s>>>(A, lda, sA, r0, k,
                                                                                                   m, kb, V, ldv, sV);
}

template <typename T>
void panel_clear(T* A, int lda, long long sA, int r0, int k, int m, int kb, int count, cudaStream_t s) {
  count_launch();
  panel_clear_kernel<T><<<dim3(1, (m + 7) / 8 < 1024 ? (m + 7) / 8 : 1024, count), dim3(32, 8), 0, s>>>(A, lda, sA,
                                                                                                       r0, k, m, kb);
}

template <typename T>
void larft_tau(const T* G, int ldG, long long sG, const T* tau, long long stau, int k, T* Tm, int ldT, long long sT,
               int count, cudaStream_t s) {
  const size_t sm = sizeof(T) * ((size_t)k * k + k);
  if (sm > 48 * 1024) cudaFuncSetAttribute(larft_tau_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch();
  larft_tau_kernel<T><<<count, 128, sm, s>>>(G, ldG, sG, tau, stau, k, Tm, ldT, sT);
}

template <typename T>
void band_pack(const T* A, int lda, long long sA, T* Bd, int W, long long sB, int m, int b, int count, cudaStream_t s) {
  count_launch();
  band_pack_kernel<T><<<dim3(1, m < 4096 ? m : 4096, count), 128, 0, s>>>(A, lda, sA, Bd, W, sB, m, b);
}

template <typename T>
void band_unpack(const T* Bd, int W, long long sB, T* A, int lda, long long sA, int m, int count, cudaStream_t s) {
  count_launch();
  dim3 grid((m + 255) / 256 < 16 ? (m + 255) / 256 : 16, m < 2048 ? m : 2048, count);
  band_unpack_kernel<T><<<grid, 256, 0, s>>>(Bd, W, sB, A, lda, sA, m);
}

template <typename T>
size_t chase_smem(int b) { return sizeof(T) * ((size_t)3 * b * b + 3 * b); }

// Workers per item for the bulge chase: all resident (cooperative launch), at most `cap`.
template <typename T>
int chase_workers(int b, int items, int cap) {
  const size_t sm = chase_smem<T>(b);
  if (sm > 48 * 1024) cudaFuncSetAttribute(chase_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chase_kernel<T>, 256, sm);
  const int total = per_sm * sms;
  return std::max(0, std::min(cap, total / std::max(1, items)));
}

template <typename T>
bool chase(T* Bd, int W, long long sB, int m, int b, T* V2, long long sV2, T* tau2, int ldt, long long sT2, int* prog,
           long long sprog, int* err, DevStatus* st, long long wait_limit, int items, int workers, cudaStream_t s) {
  if (workers < 1) return false;
  const size_t sm = chase_smem<T>(b);
  cudaMemsetAsync(err, 0, sizeof(int), s);
  for (int z = 0; z < items; z++) cudaMemsetAsync(prog + z * sprog, 0, sizeof(int) * (size_t)m, s);
  void* args[] = {&Bd, &W, &sB, &m, &b, &V2, &sV2, &tau2, &ldt, &sT2, &prog, &sprog, &err, &st, &wait_limit};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)chase_kernel<T>, dim3(workers, items), dim3(256), args, sm, s) ==
         cudaSuccess;
}

template <typename T>
void band_tridiag(const T* Bd, int W, long long sB, int m, double* d, double* e, long long sde, int count,
                  cudaStream_t s) {
  count_launch();
  band_tridiag_kernel<T><<<dim3((m + 255) / 256, count), 256, 0, s>>>(Bd, W, sB, m, d, e, sde);
}

template <typename T>
void q2_gather(const T* V2, long long sV2, const T* tau2, int ldt, long long sT2, int m, int b, int nbs, int hp, int g0,
               int j0, int nblk, T* Vw, T* tw, int items, cudaStream_t s) {
  count_launch();
  q2_gather_kernel<T><<<dim3(1, nblk, items), 256, 0, s>>>(V2, sV2, tau2, ldt, sT2, m, b, nbs, hp, g0, j0, nblk, Vw,
                                                           tw);
}

template <typename T>
void widen_pad(const double* Z, int ldz, long long sZ, T* X, int ldx, long long sX, int m, int rows, int cols,
               int count, cudaStream_t s) {
  count_launch();
  dim3 grid((cols + 255) / 256 < 16 ? (cols + 255) / 256 : 16, rows < 2048 ? rows : 2048, count);
  widen_pad_kernel<T><<<grid, 256, 0, s>>>(Z, ldz, sZ, X, ldx, sX, m, rows, cols);
}

#define INST(T)                                                                                           \
  template void q2_gather<T>(const T*, long long, const T*, int, long long, int, int, int, int, int, int,   \
                             int, T*, T*, int, cudaStream_t);                                             \
  template void widen_pad<T>(const double*, int, long long, T*, int, long long, int, int, int, int,        \
                             cudaStream_t);                                                               \
  template int chase_workers<T>(int, int, int);                                                           \
  template bool chase<T>(T*, int, long long, int, int, T*, long long, T*, int, long long, int*, long long,  \
                         int*, DevStatus*, long long, int, int, cudaStream_t);                            \
  template void band_tridiag<T>(const T*, int, long long, int, double*, double*, long long, int,           \
                                cudaStream_t);                                                            \
  template void panel_qr<T>(T*, int, long long, int, int, int, int, int, T*, long long, int, void*,      \
                           DevStatus*, long long, cudaStream_t);                                        \
  template void panel_v<T>(const T*, int, long long, int, int, int, int, T*, int, long long, int,          \
                           cudaStream_t);                                                                 \
  template void panel_clear<T>(T*, int, long long, int, int, int, int, int, cudaStream_t);                 \
  template void larft_tau<T>(const T*, int, long long, const T*, long long, int, T*, int, long long, int,  \
                             cudaStream_t);                                                               \
  template void band_pack<T>(const T*, int, long long, T*, int, long long, int, int, int, cudaStream_t);   \
  template void band_unpack<T>(const T*, int, long long, T*, int, long long, int, int, cudaStream_t);
INST(double)
INST(zc)

}  // namespace gks
