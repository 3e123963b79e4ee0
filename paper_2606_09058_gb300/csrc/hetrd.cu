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
// (16 flops per 16 bytes), above the DFMA pipe's balance point of ~0.15 flop/byte.  The
// rank-2 updates are therefore deferred over panels of steps and applied as GEMMs (the
// panel form below), which the product dispatcher can send to the tensor cores.
#include <type_traits>

#include "dense.h"

namespace gks {

// Reflector for step j (one CTA): reads row j left of the diagonal (through L2: in the
// fused form other CTAs have just written it), writes u', tau[j] and the sub-diagonal.
// uw (complex only, nullable): per element (Re u, Im u - Re u, Re u + Im u), the vector form
// of the three-multiplication complex products of the panel matrix-vector step.
__device__ __forceinline__ void put_uw(double* uw, int i, double ur, double ui) {
  if (uw) {
    uw[3 * i] = ur;
    uw[3 * i + 1] = ui - ur;
    uw[3 * i + 2] = ur + ui;
  }
}

// Scale exponent from the bits of a non-negative double (0 for zero): the e with the value
// below 2^e, i.e. ilogb + 1 (subnormals are counted at the smallest normal exponent).
__device__ __forceinline__ int bscale(unsigned long long bits) {
  return bits ? (int)((bits >> 52) & 0x7ff) - 1022 : 0;
}
// Equilibration exponent d_i = ceil(g_i / 2) of a row whose maximum (bits) lies below 2^{g_i}.
__device__ __forceinline__ int deq(unsigned long long bits) { return (bscale(bits) + 1) >> 1; }

// Digit format of the matrix-vector step: kDig balanced base-256 digits (signed 8-bit,
// in [-128, 127]) of the integer round(|x| 2^{54 - e}) with the sign of x, for |x| < 2^e:
// x = sum_s d_s 2^{e - 6 - 8s} up to 2^{e - 55}.
constexpr int kDig = 7;
constexpr int kMaxLevel = 7;  // digit pairs s + t <= kMaxLevel

// The digits of x below 2^e into d[0..kDig), most significant first.  Integer operations on
// the bits of x only (the FP64 pipe is slow on this GPU): |x| = m 2^{x_e - 1075} with the
// 53-bit significand m, so trunc(|x| 2^{55 - e}) = m shifted by x_e - 1020 - e, and
// rounding halves it with a carry.  Balanced digits from the least significant up keep the
// leading one within [-65, 65].
__device__ __forceinline__ void digits8(double x, int e, int (&d)[kDig]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int xe = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xfffffffffffffull) | (xe ? (1ull << 52) : 0ull);
  const int sh = (xe ? xe : 1) - 1020 - e;
  const unsigned long long q2 = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
  const long long q = (long long)((q2 + 1) >> 1);
  long long v = (b >> 63) ? -q : q;
#pragma unroll
  for (int s = kDig - 1; s >= 1; s--) {
    int t = (int)(v & 255);
    t = t >= 128 ? t - 256 : t;
    d[s] = t;
    v = (v - t) >> 8;
  }
  d[0] = (int)v;
}

// |Re|, |Im| maximum of a value as the bits of a non-negative double (bits of non-negative
// doubles order like the values).
__device__ __forceinline__ unsigned long long absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
template <typename T>
__device__ __forceinline__ unsigned long long maxbits(T a) {
  if constexpr (std::is_same<T, double>::value || std::is_same<T, float>::value) return absbits((double)a);
  else return max(absbits((double)re(a)), absbits((double)im(a)));
}

// Digits of 16 consecutive entries packed as the layout's block: NPL planes of 16 bytes (the
// kDig Re planes, then the Im planes for complex), stored with 16-byte writes.  Entry el is
// cut below 2^{e[el]} (the scale and the equilibration folded into one exponent).
template <typename T, int NPL>
__device__ __forceinline__ void store_digit_block(const T (&vals)[16], const int (&e)[16], signed char* dst) {
  uint4 o[NPL];
#pragma unroll
  for (int q = 0; q < NPL; q++) o[q] = make_uint4(0u, 0u, 0u, 0u);
  auto put = [&](int plane, int el, int dv) {
    const uint32_t bb = (uint32_t)(dv & 0xff) << (8 * (el & 3));
    if ((el >> 2) == 0) o[plane].x |= bb;
    else if ((el >> 2) == 1) o[plane].y |= bb;
    else if ((el >> 2) == 2) o[plane].z |= bb;
    else o[plane].w |= bb;
  };
#pragma unroll
  for (int el = 0; el < 16; el++) {
    int d[kDig];
    digits8((double)re(vals[el]), e[el], d);
#pragma unroll
    for (int sp = 0; sp < kDig; sp++) put(sp, el, d[sp]);
    if constexpr (NPL == 2 * kDig) {
      digits8((double)im(vals[el]), e[el], d);
#pragma unroll
      for (int sp = 0; sp < kDig; sp++) put(kDig + sp, el, d[sp]);
    }
  }
  uint4* out = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int q = 0; q < NPL; q++) out[q] = o[q];
}

// Digits of u (length j) into ud (blocks of 16 entries, each the planes' 16 bytes: Re
// 0..7, Im 8..15; zeros from j up to the next multiple of 16) and its scale exponent fu;
// every thread of the block takes part.
template <typename T>
__device__ void u_digits(const T* u, int j, signed char* ud, int* fu, const unsigned long long* rmax) {
  constexpr bool CPX = !std::is_same<T, double>::value && !std::is_same<T, float>::value;
  constexpr int NPL = CPX ? 2 * kDig : kDig;
  __shared__ int mred[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  __syncthreads();
  // fu: the scale exponent of ũ = D u, the largest bscale(|u_i|) + d_i
  int m = -100000;
  for (int i0 = tid; i0 < j; i0 += 8 * nt) {  // eight independent loads in flight per thread
    unsigned long long mb[8], rb[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int i = i0 + q * nt;
      mb[q] = i < j ? maxbits(u[i]) : 0ull;
      rb[q] = i < j ? rmax[i] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < 8; q++)
      if (mb[q]) m = max(m, bscale(mb[q]) + deq(rb[q]));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) mred[tid >> 5] = m;
  __syncthreads();
  if (tid < 32) {
    int v = tid < (nt >> 5) ? mred[tid] : -100000;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (tid == 0) mred[0] = v;
  }
  __syncthreads();
  const int e = mred[0] == -100000 ? 0 : mred[0];
  if (tid == 0) *fu = e;
  const int nblk = (j + 15) >> 4;
  for (int b = tid; b < nblk; b += nt) {
    T vals[16];
    int ex[16];
#pragma unroll
    for (int el = 0; el < 16; el++) {
      const int i = 16 * b + el;
      vals[el] = i < j ? u[i] : zero<T>();
      ex[el] = i < j ? e - deq(rmax[i]) : 0;  // ũ_i 2^{-fu} = u_i 2^{d_i - fu}
    }
    store_digit_block<T, NPL>(vals, ex, ud + (size_t)b * (NPL * 16));
  }
}

template <typename T>
__device__ void reflector_body(T* A, int lda, int j, T* u, double* tau, double* uw, signed char* ud = nullptr,
                               int* fu = nullptr, const unsigned long long* rmax = nullptr) {
  __shared__ double redd[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  T* row = A + (size_t)j * lda;
  double s2 = 0.0;
  for (int i0 = tid; i0 < j; i0 += 8 * nt) {  // eight independent loads in flight per thread
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = i0 + q * nt < j ? ldcg(row + i0 + q * nt) : zero<T>();
#pragma unroll
    for (int q = 0; q < 8; q++) s2 += abs2(v[q]);
  }
  const double xnorm2 = block_sum(s2, redd);
  const T alpha = conjg(ldcg(row + j - 1));
  const double tail = xnorm2 - abs2(alpha);
  if (!(tail > 0.0)) {  // nothing to annihilate: P_j = I
    for (int i = tid; i < j; i += nt) {
      u[i] = (i == j - 1) ? from_real<T>(1.0) : zero<T>();
      put_uw(uw, i, i == j - 1 ? 1.0 : 0.0, 0.0);
    }
    if (tid == 0) tau[j] = 0.0;
    if (ud) u_digits<T>(u, j, ud, fu, rmax);
    return;
  }
  const double xn = sqrt(xnorm2);
  const double aa = sqrt(abs2(alpha));
  const T ph = aa > 0.0 ? alpha * (1.0 / aa) : from_real<T>(1.0);
  const T upiv = ph * (aa + xn);                       // alpha + ph * xn
  const double beta = 2.0 / (tail + abs2(upiv));
  const T inv = conjg(upiv) * (1.0 / abs2(upiv));       // 1 / upiv
  __syncthreads();
  for (int i0 = tid; i0 < j - 1; i0 += 8 * nt) {
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = i0 + q * nt < j - 1 ? ldcg(row + i0 + q * nt) : zero<T>();
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int i = i0 + q * nt;
      if (i < j - 1) {
        const T w = conjg(v[q]) * inv;  // u'_i = a_i / u_{j-1}
        u[i] = w;
        row[i] = w;
        put_uw(uw, i, re(w), im(w));
      }
    }
  }
  if (tid == 0) {
    u[j - 1] = from_real<T>(1.0);
    put_uw(uw, j - 1, 1.0, 0.0);
    tau[j] = beta * abs2(upiv);
    row[j - 1] = conjg(ph) * (-xn);                     // lower-storage sub-diagonal
  }
  if (ud) u_digits<T>(u, j, ud, fu, rmax);
}

template <typename T>
__global__ void hetrd_reflector_kernel(T* A, int lda, long long sA, int j, T* u, long long sv, double* tau,
                                       long long stau, double* uw, signed char* ud, long long sud, int* fu,
                                       const unsigned long long* rmax, int ldr) {
  const int z = blockIdx.x;
  reflector_body<T>(A + z * sA, lda, j, u + z * sv, tau + z * stau, uw ? uw + z * 3 * sv : nullptr,
                    ud ? ud + z * sud : nullptr, fu ? fu + z : nullptr, rmax ? rmax + (size_t)z * ldr : nullptr);
}

// Sg[r][c] = Re A[r][c] + Im A[r][c] over the lower triangle of the leading n x n block
// (the stale block of a panel), for the three-multiplication products.
__global__ void hetrd_sums_kernel(const zc* A, int lda, long long sA, int n, double* Sg) {
  const int z = blockIdx.z;
  A += z * sA;
  Sg += z * sA;
  for (int r = blockIdx.y; r < n; r += gridDim.y)
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= r; c += gridDim.x * blockDim.x) {
      const zc a = A[(size_t)r * lda + c];
      Sg[(size_t)r * lda + c] = a.x + a.y;
    }
}

// The step's second part once this CTA's p_raw rows [c0, cend) are in prow (shared, one
// per row): p, the CTA's shares of Q^H u, U^H u and u^H p_raw, and in the last CTA (atomic
// ticket after a fence) their sums y1, y2, u^H p and kq.  Pointers are the item's.
template <typename T>
__device__ void phemv_tail(const T* prow, int c0, int cend, const T* u, T* p, double t, const T* U, const T* Q,
                           int ldu, int k, T* part, T* y, int* ticket) {
  __shared__ T red[32];
  __shared__ T gsum[256];
  __shared__ int last;
  const int tid = threadIdx.x;
  const int pst = 2 * ldu + 2;
  T d0 = zero<T>();
  if (tid < cend - c0) {
    const T pr = prow[tid];
    p[c0 + tid] = pr;
    macc(d0, u[c0 + tid], pr);
  }
  d0 = block_sum(d0, red);
  T* mine = part + (size_t)blockIdx.x * pst;
  if (tid == 0) mine[2 * ldu] = d0;
  for (int s = tid; s < k; s += blockDim.x) {
    T a1 = zero<T>(), a2 = zero<T>();
    for (int r0 = c0; r0 < cend; r0 += 8) {  // eight rows' loads in flight
      T qv[8], uv[8], ur[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int r = min(r0 + q, cend - 1);
        qv[q] = Q[(size_t)r * ldu + s];
        uv[q] = U[(size_t)r * ldu + s];
        ur[q] = r0 + q < cend ? u[r] : zero<T>();
      }
#pragma unroll
      for (int q = 0; q < 8; q++) {
        macc(a1, qv[q], ur[q]);
        macc(a2, uv[q], ur[q]);
      }
    }
    mine[s] = a1;
    mine[ldu + s] = a2;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  if (tid == 0) *ticket = 0;
  // Sums over the CTAs' shares of the E = 2k + 1 entries (Q^H u, U^H u, u^H p_raw): G groups
  // of threads per entry take every G-th CTA with eight loads in flight, then one thread per
  // entry adds the groups in order.
  const int nb = gridDim.x, nt = blockDim.x, E = 2 * k + 1;
  const int G = E <= nt ? nt / E : 1;
  for (int t0 = tid; t0 < G * E; t0 += nt) {
    const int e = t0 % E, g = t0 / E;
    const size_t off = e < k ? e : (e < 2 * k ? ldu + (e - k) : 2 * ldu);
    T a = zero<T>();
    for (int b0 = g; b0 < nb; b0 += 8 * G) {
      T v[8];
#pragma unroll
      for (int q = 0; q < 8; q++) v[q] = b0 + q * G < nb ? ldcg(part + (size_t)(b0 + q * G) * pst + off) : zero<T>();
#pragma unroll
      for (int q = 0; q < 8; q++) a += v[q];
    }
    if (G > 1) gsum[t0] = a;
    else if (e < k) y[e] = a;
    else if (e < 2 * k) y[ldu + e - k] = a;
    else red[0] = a;
  }
  __syncthreads();
  if (G > 1 && tid < E) {
    T a = gsum[tid];
    for (int g = 1; g < G; g++) a += gsum[g * E + tid];
    if (tid < k) y[tid] = a;
    else if (tid < 2 * k) y[ldu + tid - k] = a;
    else red[0] = a;
  }
  __syncthreads();
  const T tot = red[0];
  __syncthreads();
  T w = zero<T>();
  for (int e = tid; e < k; e += blockDim.x) {
    macc(w, y[ldu + e], y[e]);
    macc(w, y[e], y[ldu + e]);
  }
  w = block_sum(w, red);
  if (tid == 0) {
    const T uhp = t * (tot - w);
    y[2 * ldu] = tot;
    y[2 * ldu + 1] = (0.5 * t) * uhp;
  }
}

// Panel (blocked) form.  A panel of steps keeps the trailing block A[0:j,0:j] as it was
// at the panel's start; the panel buffers U and Q (M x ldu per item, row r holds u_s[r]
// and q_s[r] for the panel's earlier steps s < k) carry what it has not seen yet:
//   A_true = A - U Q^H - Q U^H   on [0:j, 0:j].
// The panel ends with that rank-2k update as two GEMMs.
//
// Step j, first half: p_raw = A[0:j,0:j] u over the stale block.  CTA b owns rows/columns
// [RB b, RB b + RB): its row panel left of the diagonal plus its column panel below, so every
// CTA reads the same number of elements.  It adds its rows' shares of Q^H u, U^H u and
// u^H p_raw.  The last CTA (atomic ticket after a fence; nothing waits) sums the shares:
//   y1 = Q^H u,  y2 = U^H u,  u^H p = tau (u^H p_raw - y2^H y1 - y1^H y2),
//   kq = (tau/2) u^H p,
// since p = tau A_true u = tau (p_raw - U y1 - Q y2).
// y layout per item: y1 at [0, k), y2 at [ldu, ldu + k), u^H p_raw at 2 ldu, kq at 2 ldu + 1;
// the shares use the same layout per CTA with stride 2 ldu + 2.
template <typename T, int RB>
__global__ void __launch_bounds__(256) hetrd_phemv_kernel(const T* A, int lda, long long sA, int j, const T* u,
                                                          T* p, long long sv, const double* tau, long long stau,
                                                          const T* U, const T* Q, int ldu, long long sU, int k,
                                                          T* part, long long spart, T* y, long long sy,
                                                          int* ticket, const double* Sg, const double* uw) {
  // RB rows/columns per CTA (64, or 16 when the grid would not fill the GPU)
  constexpr int NG = 256 / RB;
  __shared__ T colpart[NG][RB];
  __shared__ T rowacc[RB];
  const int z = blockIdx.y, tid = threadIdx.x;
  A += z * sA;
  u += z * sv;
  p += z * sv;
  U += z * sU;
  Q += z * sU;
  part += z * spart;
  y += z * sy;
  const double t = tau[z * stau + j];
  const int c0 = blockIdx.x * RB;
  const int cend = min(c0 + RB, j);
  const int warp = tid >> 5, lane = tid & 31;
  bool done = false;
  if constexpr (sizeof(T) == 16) {
    if (Sg) {
      // Three real multiply-adds per complex product (Gauss): with s = Re a + Im a (Sg) and
      // the vector form (c, d - c, c + d) of u_c = c + i d (uw),
      //   a u    = (c s - Im a (c + d)) + i (c s + Re a (d - c)),
      //   a* u   = (c s + Im a (d - c)) + i (Re a (c + d) - c s).
      Sg += z * sA;
      uw += z * 3 * sv;
      for (int r = c0 + warp; r < cend; r += 8) {
        const zc* ar = reinterpret_cast<const zc*>(A) + (size_t)r * lda;
        const double* sr = Sg + (size_t)r * lda;
        double k1 = 0.0, k2 = 0.0, k3 = 0.0;
        for (int c = lane; c <= r; c += 32) {
          const zc a = ar[c];
          k1 = fma(uw[3 * c], sr[c], k1);
          k2 = fma(a.x, uw[3 * c + 1], k2);
          k3 = fma(a.y, uw[3 * c + 2], k3);
        }
        k1 = warp_sum(k1);
        k2 = warp_sum(k2);
        k3 = warp_sum(k3);
        if (lane == 0) rowacc[r - c0] = T{k1 - k3, k1 + k2};
      }
      const int cc = tid % RB, g = tid / RB;
      const int c = c0 + cc;
      double l1 = 0.0, l3 = 0.0, l4 = 0.0;
      if (c < cend) {
        for (int r = c0 + g; r < j; r += NG)
          if (r > c) {
            const zc a = reinterpret_cast<const zc*>(A)[(size_t)r * lda + c];
            l1 = fma(uw[3 * r], Sg[(size_t)r * lda + c], l1);
            l3 = fma(a.y, uw[3 * r + 1], l3);
            l4 = fma(a.x, uw[3 * r + 2], l4);
          }
      }
      colpart[g][cc] = T{l1 + l3, l4 - l1};
      done = true;
    }
  }
  if (!done) {
    // row part: rows r in [c0, cend), columns 0..r; one warp per row
    for (int r = c0 + warp; r < cend; r += 8) {
      const T* ar = A + (size_t)r * lda;
      T s = zero<T>();
      for (int c = lane; c <= r; c += 32) mac(s, ar[c], u[c]);
      s = warp_sum(s);
      if (lane == 0) rowacc[r - c0] = s;
    }
    // column part: columns c in [c0, cend), rows r > c
    const int cc = tid % RB, g = tid / RB;
    const int c = c0 + cc;
    T s = zero<T>();
    if (c < cend) {
      for (int r = c0 + g; r < j; r += NG)
        if (r > c) macc(s, A[(size_t)r * lda + c], u[r]);
    }
    colpart[g][cc] = s;
  }
  __syncthreads();
  if (tid < RB && c0 + tid < cend) {
    T pr = rowacc[tid];
#pragma unroll
    for (int g = 0; g < NG; g++) pr += colpart[g][tid];
    rowacc[tid] = pr;
  }
  phemv_tail<T>(rowacc, c0, cend, u, p, t, U, Q, ldu, k, part, y, ticket + z);
}

// ------------------------------------------------------------------ digit form of the step
//
// hetrd_dmax_kernel: row maxima of |Re|, |Im| over the full Hermitian rows of the stale
// block from its lower triangle, where element (r, c) counts for rows r and c.  One CTA per
// chunk of 64 rows: a warp per row for the rows' own maxima (c <= r), then a thread per
// column for the column maxima below the diagonal (c < r), one global atomic max per row,
// and per column and chunk (on the bits of non-negative doubles, which order like the
// values).
template <typename T>
__global__ void __launch_bounds__(256) hetrd_dmax_kernel(const T* A, int lda, long long sA, int n,
                                                         unsigned long long* rmax, int ldr) {
  const int z = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = blockIdx.x * 64, r1 = min(n, r0 + 64);
  A += z * sA;
  rmax += (size_t)z * ldr;
  for (int r = r0 + warp; r < r1; r += 8) {
    unsigned long long m = 0ull;
    for (int c = lane; c <= r; c += 32) m = max(m, maxbits(A[(size_t)r * lda + c]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m) atomicMax(rmax + r, m);
  }
  for (int c = tid; c < r1 - 1; c += blockDim.x) {
    unsigned long long mc = 0ull;
    for (int r = max(r0, c + 1); r < r1; r++) mc = max(mc, maxbits(A[(size_t)r * lda + c]));
    if (mc) atomicMax(rmax + c, mc);
  }
}

// hetrd_digits_kernel: 32 x 32 tiles of the full Hermitian [0:n16, 0:n16] (zero outside
// [0:n, 0:n]); tiles above the diagonal come from the transposed lower tile through shared
// memory, conjugated.  64 threads: thread t packs row t / 2, columns 16 (t % 2) .. + 15.
template <typename T>
__global__ void __launch_bounds__(64) hetrd_digits_kernel(const T* A, int lda, long long sA, int n, HemvDigits hd) {
  constexpr int NPL = sizeof(T) == 16 ? 2 * kDig : kDig;
  __shared__ T tile[32][33];
  const int z = blockIdx.z, tid = threadIdx.x;
  const int R0 = blockIdx.y * 32, C0 = blockIdx.x * 32;
  const int n16 = (n + 15) & ~15;
  if (R0 >= n16 || C0 >= n16) return;
  A += z * sA;
  const bool upper = C0 > R0;
  // source tile: (R0, C0) itself, or (C0, R0) for tiles above the diagonal
  const int sr0 = upper ? C0 : R0, sc0 = upper ? R0 : C0;
  for (int e = tid; e < 32 * 32; e += 64) {
    const int yy = e >> 5, xx = e & 31;
    const int r = sr0 + yy, c = sc0 + xx;
    tile[yy][xx] = (r < n && c < n && c <= r) ? A[(size_t)r * lda + c] : zero<T>();
  }
  __syncthreads();
  const unsigned long long* rm = hd.rmax + (size_t)z * hd.ldd;
  const int rr = tid >> 1, cbk = tid & 1;
  const int r = R0 + rr;
  if (r < n16 && C0 + 16 * cbk < n16) {
    const int dr = r < n ? deq(rm[r]) : 0;
    T vals[16];
    int ex[16];
#pragma unroll
    for (int el = 0; el < 16; el++) {
      const int cc = 16 * cbk + el, c = C0 + cc;
      T v;
      if (upper) v = conjg(tile[cc][rr]);
      else if (c <= r) v = tile[rr][cc];
      else v = (r < n && c < n) ? conjg(tile[cc][rr]) : zero<T>();  // diagonal tile, upper part
      vals[el] = v;
      ex[el] = dr + (c < n ? deq(rm[c]) : 0);  // ã = a 2^{-d_r - d_c}, cut below 1
    }
    const size_t tile = (size_t)(r >> 5) * (hd.ldd >> 4) + (C0 >> 4) + cbk;
    store_digit_block<T, NPL>(vals, ex, hd.D + z * hd.sD + tile * (32 * NPL * 16) + (size_t)(r & 31) * (NPL * 16));
  }
}

__device__ __forceinline__ int dp4(unsigned a, unsigned b, int c) { return __dp4a((int)a, (int)b, c); }
__device__ __forceinline__ int dp4x4(uint4 a, uint4 b, int c) {
  return dp4(a.w, b.w, dp4(a.z, b.z, dp4(a.y, b.y, dp4(a.x, b.x, c))));
}

// 16-byte asynchronous global -> shared copies (L2 only), their groups and waits.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory ring of the digit matrix-vector kernel: per warp STG stages, each the
// digit planes of 32 rows x 16 columns (row stride RS 16-byte words: an odd count puts a
// warp's 16-byte reads of 32 rows on distinct bank groups) followed by u's digits of the
// same 16 columns.
template <typename T>
struct DigRing {
  static constexpr int NPL = sizeof(T) == 16 ? 2 * kDig : kDig;
  static constexpr int RS = NPL % 2 ? NPL : NPL + 1;
  static constexpr int STG = 3;
  static constexpr int SU4 = 32 * RS + NPL;
  static constexpr int SMEM = 8 * STG * SU4 * 16;
};

// p_raw = A_stale[0:j, 0:j] u from the digits, 32 rows per CTA (lane = row), the columns in
// eight ranges (warp w), exact int32 level sums per (row, product, level), summed over the
// warps in shared memory, then weighted in FP64; then the common tail.  Each warp streams its
// 16-column blocks through its own ring of STG stages (asynchronous copies, STG - 1 blocks
// ahead of the one it multiplies; a stage is one contiguous tile, consecutive lanes copying
// consecutive 16-byte words), and the loads in flight hold no registers.
// Digit pairs (digits numbered from 0, most significant first) up to level s + t = 7: the
// dropped pairs lie below 2^-59 of the scales (stopping one level earlier would leave a
// one-signed error near the FP64 unit per term).
// Complex: the four real products Re a Re u, Im a Im u, Re a Im u, Im a Re u
// (Re p = first - second, Im p = third + fourth); real: the first only.
template <typename T>
__global__ void __launch_bounds__(256, 1) hetrd_phemv_dig_kernel(int j, const T* u, T* p, long long sv,
                                                                 const double* tau, long long stau, const T* U,
                                                                 const T* Q, int ldu, long long sU, int k, T* part,
                                                                 long long spart, T* y, long long sy, int* ticket,
                                                                 HemvDigits hd) {
  constexpr bool CPX = sizeof(T) == 16;
  constexpr int NP = CPX ? 4 : 1;  // real products
  constexpr int NPL = DigRing<T>::NPL, RS = DigRing<T>::RS, STG = DigRing<T>::STG, SU4 = DigRing<T>::SU4;
  constexpr int NL = kMaxLevel + 1;  // levels
  static_assert(NP * NL * 33 * 8 * 4 <= DigRing<T>::SMEM, "level sums alias the ring");
  extern __shared__ uint4 ring_all[];
  __shared__ T prow[32];
  const int z = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = blockIdx.x * 32, cend = min(c0 + 32, j);
  const int j16 = (j + 15) & ~15;
  const int chunk = (((j16 + 7) / 8) + 15) & ~15;
  const int cb = min(j16, warp * chunk), ce = min(j16, cb + chunk);
  const int nit = (ce - cb) >> 4;
  // the CTA's row tile: 16-column tiles of 32 rows, each 32 * NPL 16-byte words
  const uint4* Dt = reinterpret_cast<const uint4*>(hd.D + z * hd.sD) + (size_t)blockIdx.x * (hd.ldd >> 4) * (32 * NPL);
  const signed char* ud = hd.ud + z * hd.sud;
  uint4* ring = ring_all + warp * (STG * SU4);
  // stage it % STG <- the contiguous tile of the CTA's 32 rows (rows past j - 1 hold stale
  // digits; their results are unused) and u's digits, columns cb + 16 it .. + 15; an empty
  // group past the range keeps the group count uniform
  auto issue = [&](int it) {
    if (it < nit) {
      const int cbk = (cb >> 4) + it;
      const uint4* src = Dt + (size_t)cbk * (32 * NPL);
      uint4* st = ring + (it % STG) * SU4;
#pragma unroll
      for (int w = lane; w < 32 * NPL; w += 32) {
        const int rr = w / NPL, q = w - rr * NPL;
        cp_async16(st + rr * RS + q, src + w);
      }
      if (lane < NPL)
        cp_async16(st + 32 * RS + lane, reinterpret_cast<const uint4*>(ud + (size_t)cbk * (NPL * 16)) + lane);
    }
    cp_async_commit();
  };
  int acc[NP][NL];
#pragma unroll
  for (int q = 0; q < NP; q++)
#pragma unroll
    for (int L = 0; L < NL; L++) acc[q][L] = 0;
#pragma unroll
  for (int it = 0; it < STG - 1; it++) issue(it);
  for (int it = 0; it < nit; it++) {
    __syncwarp();  // every lane is done with the stage refilled next
    issue(it + STG - 1);
    cp_async_wait<STG - 1>();
    __syncwarp();  // stage it is complete for every lane (each row comes from several lanes)
    const uint4* st = ring + (it % STG) * SU4;
    uint4 av[NPL];
#pragma unroll
    for (int q = 0; q < NPL; q++) av[q] = st[lane * RS + q];
#pragma unroll
    for (int t = 0; t < kDig; t++) {
      const uint4 ur = st[32 * RS + t];
      uint4 ui;
      if constexpr (CPX) ui = st[32 * RS + kDig + t];
#pragma unroll
      for (int s = 0; s < kDig && s + t <= kMaxLevel; s++) {
        acc[0][s + t] = dp4x4(av[s], ur, acc[0][s + t]);
        if constexpr (CPX) {
          acc[1][s + t] = dp4x4(av[kDig + s], ui, acc[1][s + t]);
          acc[2][s + t] = dp4x4(av[s], ui, acc[2][s + t]);
          acc[3][s + t] = dp4x4(av[kDig + s], ur, acc[3][s + t]);
        }
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();  // every ring is idle: the level sums reuse its space
  auto accs = reinterpret_cast<int(*)[33][8]>(ring_all);
#pragma unroll
  for (int q = 0; q < NP; q++)
#pragma unroll
    for (int L = 0; L < NL; L++) accs[q * NL + L][lane][warp] = acc[q][L];
  __syncthreads();
  if (tid < 32 && c0 + tid < cend) {
    // exact sums over the warps, then 2^{d_i + fu - 12 - 8L} per level
    const int E = deq(hd.rmax[(size_t)z * hd.ldd + c0 + tid]) + hd.fu[z] - 12;
    double pre = 0.0, pim = 0.0;
#pragma unroll
    for (int L = NL - 1; L >= 0; L--) {
      long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
      for (int w = 0; w < 8; w++) {
        s0 += accs[L][tid][w];
        if constexpr (CPX) {
          s1 += accs[NL + L][tid][w];
          s2 += accs[2 * NL + L][tid][w];
          s3 += accs[3 * NL + L][tid][w];
        }
      }
      pre += ldexp((double)(s0 - s1), E - 8 * L);
      if constexpr (CPX) pim += ldexp((double)(s2 + s3), E - 8 * L);
    }
    if constexpr (CPX) prow[tid] = T{pre, pim};
    else prow[tid] = pre;
  }
  __syncthreads();
  const double t = tau[z * stau + j];
  phemv_tail<T>(prow, c0, cend, u + z * sv, p + z * sv, t, U + z * sU, Q + z * sU, ldu, k, part + z * spart,
                y + z * sy, ticket + z);
}

// Sum over aligned groups of 8 lanes (every lane of the warp takes part).
__device__ __forceinline__ double group8_sum(double v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ zc group8_sum(zc v) { return zc{group8_sum(v.x), group8_sum(v.y)}; }
__device__ __forceinline__ float group8_sum(float v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ cf group8_sum(cf v) { return cf{group8_sum(v.x), group8_sum(v.y)}; }

// Step j, second half: q = tau (p_raw - U y1 - Q y2) - kq u for the rows of this CTA (64
// per CTA), stored with u as column k of Q and U.  With rowupd, row j-1 of A (columns
// 0..j-1) receives the panel's updates so far,
//   A[j-1][c] -= sum_{s<=k} U[j-1][s] conj(Q[c][s]) + Q[j-1][s] conj(U[c][s]),
// (each CTA computes the single q_k[j-1] it needs itself), and the last CTA forms the
// reflector of step j-1 from that row.  Dynamic shared memory: 4 (ldu + 1) elements.
template <typename T>
__global__ void __launch_bounds__(256) hetrd_pupdate_kernel(T* A, int lda, long long sA, int j, T* u,
                                                            const T* p, long long sv, double* tau, long long stau,
                                                            T* U, T* Q, int ldu, long long sU, int k, const T* y,
                                                            long long sy, int rowupd, int* ticket, double* uw,
                                                            signed char* ud, long long sud, int* fu,
                                                            const unsigned long long* rmax, int ldr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* y1s = reinterpret_cast<T*>(smem_raw);
  T* y2s = y1s + (ldu + 1);
  T* ujs = y2s + (ldu + 1);
  T* qjs = ujs + (ldu + 1);
  __shared__ int last;
  const int z = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  A += z * sA;
  u += z * sv;
  p += z * sv;
  U += z * sU;
  Q += z * sU;
  y += z * sy;
  tau += z * stau;
  if (uw) uw += z * 3 * sv;
  const double t = tau[j];
  const T kq = y[2 * ldu + 1];
  for (int s = tid; s < k; s += blockDim.x) {
    y1s[s] = y[s];
    y2s[s] = y[ldu + s];
    if (rowupd) {
      ujs[s] = U[(size_t)(j - 1) * ldu + s];
      qjs[s] = Q[(size_t)(j - 1) * ldu + s];
    }
  }
  __syncthreads();
  if (rowupd && warp == 0) {
    T corr = zero<T>();
    for (int s = lane; s < k; s += 32) {
      mac(corr, ujs[s], y1s[s]);
      mac(corr, qjs[s], y2s[s]);
    }
    corr = warp_sum(corr);
    if (lane == 0) {
      const T uj = u[j - 1];
      ujs[k] = uj;
      qjs[k] = t * (p[j - 1] - corr) - kq * uj;
    }
  }
  __syncthreads();
  // 32 groups of 8 lanes, two columns per group (more columns in flight, short reductions)
  const int c0 = blockIdx.x * 64, cend = min(c0 + 64, j);
  const int grp = tid >> 3, gl = tid & 7;
  for (int it = 0; it < 2; it++) {
    const int c = c0 + grp + 32 * it;
    const bool ok = c < cend;
    T corr = zero<T>(), rs = zero<T>();
    if (ok) {
      const T* Uc = U + (size_t)c * ldu;
      const T* Qc = Q + (size_t)c * ldu;
      for (int s0 = gl; s0 < k; s0 += 32) {  // four steps' loads in flight
        T ucv[4], qcv[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int sq = min(s0 + 8 * q, k - 1);
          ucv[q] = Uc[sq];
          qcv[q] = Qc[sq];
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int sq = s0 + 8 * q;
          if (sq < k) {
            mac(corr, ucv[q], y1s[sq]);
            mac(corr, qcv[q], y2s[sq]);
            if (rowupd) {
              mac(rs, ujs[sq], conjg(qcv[q]));
              mac(rs, qjs[sq], conjg(ucv[q]));
            }
          }
        }
      }
    }
    corr = group8_sum(corr);
    if (rowupd) rs = group8_sum(rs);
    if (ok && gl == 0) {
      const T uc = u[c];
      const T qc = t * (p[c] - corr) - kq * uc;
      U[(size_t)c * ldu + k] = uc;
      Q[(size_t)c * ldu + k] = qc;
      if (rowupd) {
        mac(rs, ujs[k], conjg(qc));
        mac(rs, qjs[k], conjg(uc));
        T* a = A + (size_t)(j - 1) * lda + c;
        *a = *a - rs;
      }
    }
  }
  if (!rowupd) return;
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(ticket + z, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  if (tid == 0) ticket[z] = 0;
  __syncthreads();
  reflector_body<T>(A, lda, j - 1, u, tau, uw, ud ? ud + z * sud : nullptr, fu ? fu + z : nullptr,
                    rmax ? rmax + (size_t)z * ldr : nullptr);
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

__device__ __forceinline__ double widen(double a) { return a; }
__device__ __forceinline__ double widen(float a) { return (double)a; }
__device__ __forceinline__ zc widen(zc a) { return a; }
__device__ __forceinline__ zc widen(cf a) { return zc{(double)a.x, (double)a.y}; }

// V[:, c] = u'_{j1-c} (rows 0..j1-1), tb[c] = tau[j1-c].  Reflectors stored in single
// precision (the mixed-precision path) are widened exactly to FP64.
template <typename T, typename TV>
__global__ void gather_reflectors_kernel(const T* A, int lda, long long sA, const double* tau, long long stau,
                                         int j0, int j1, TV* V, int ldv, long long sV, double* tb, long long stb) {
  const int z = blockIdx.z;
  A += z * sA;
  tau += z * stau;
  V += z * sV;
  tb += z * stb;
  const int nbb = j1 - j0 + 1;
  for (int i = blockIdx.y; i < j1; i += gridDim.y)
    for (int c = threadIdx.x; c < nbb; c += blockDim.x) {
      int jj = j1 - c;
      TV v = zero<TV>();
      if (i < jj - 1) v = widen(A[(size_t)jj * lda + i]);
      else if (i == jj - 1) v = from_real<TV>(1.0);
      V[(size_t)i * ldv + c] = v;
      if (i == 0) tb[c] = tau[jj];
    }
}

template <typename T>
void hetrd_reflector(T* A, int lda, long long sA, int j, T* u, long long sv, double* tau, long long stau, int count,
                     cudaStream_t s, double* uw, const HemvDigits* hd) {
  count_launch();
  hetrd_reflector_kernel<T><<<count, 256, 0, s>>>(A, lda, sA, j, u, sv, tau, stau, uw, hd ? hd->ud : nullptr,
                                                  hd ? hd->sud : 0, hd ? hd->fu : nullptr, hd ? hd->rmax : nullptr,
                                                  hd ? hd->ldd : 0);
}

template <typename T>
void hetrd_digits(const T* A, int lda, long long sA, int n, const HemvDigits& hd, int count, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(hd.rmax, 0, sizeof(unsigned long long) * hd.ldd * count, s);
  count_launch(2);
  hetrd_dmax_kernel<T><<<dim3((n + 63) / 64, count), 256, 0, s>>>(A, lda, sA, n, hd.rmax, hd.ldd);
  const int nt = ((n + 15) / 16 * 16 + 31) / 32;
  hetrd_digits_kernel<T><<<dim3(nt, nt, count), 64, 0, s>>>(A, lda, sA, n, hd);
}

void hetrd_sums(const zc* A, int lda, long long sA, int n, double* Sg, int count, cudaStream_t s) {
  if (n <= 0) return;
  dim3 grid((n + 255) / 256 < 16 ? (n + 255) / 256 : 16, n < 4096 ? n : 4096, count);
  count_launch();
  hetrd_sums_kernel<<<grid, 256, 0, s>>>(A, lda, sA, n, Sg);
}

template <typename T>
void hetrd_phemv(const T* A, int lda, long long sA, int j, const T* u, T* p, long long sv, const double* tau,
                 long long stau, const T* U, const T* Q, int ldu, long long sU, int k, T* part, long long spart,
                 T* y, long long sy, int* ticket, int count, cudaStream_t s, const double* Sg, const double* uw,
                 const HemvDigits* hd) {
  count_launch();
  if constexpr (std::is_same<T, double>::value || std::is_same<T, zc>::value) {
    if (hd) {
      constexpr int sm = DigRing<T>::SMEM;
      cudaFuncSetAttribute(hetrd_phemv_dig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
      hetrd_phemv_dig_kernel<T><<<dim3((j + 31) / 32, count), 256, sm, s>>>(j, u, p, sv, tau, stau, U, Q, ldu, sU,
                                                                            k, part, spart, y, sy, ticket, *hd);
      return;
    }
  }
  if ((long long)((j + 63) / 64) * count >= 4 * 152)
    hetrd_phemv_kernel<T, 64><<<dim3((j + 63) / 64, count), 256, 0, s>>>(A, lda, sA, j, u, p, sv, tau, stau, U, Q,
                                                                         ldu, sU, k, part, spart, y, sy, ticket, Sg,
                                                                         uw);
  else
    hetrd_phemv_kernel<T, 16><<<dim3((j + 15) / 16, count), 256, 0, s>>>(A, lda, sA, j, u, p, sv, tau, stau, U, Q,
                                                                         ldu, sU, k, part, spart, y, sy, ticket, Sg,
                                                                         uw);
}

template <typename T>
void hetrd_pupdate(T* A, int lda, long long sA, int j, T* u, const T* p, long long sv, double* tau, long long stau,
                   T* U, T* Q, int ldu, long long sU, int k, const T* y, long long sy, int rowupd, int* ticket,
                   int count, cudaStream_t s, double* uw, const HemvDigits* hd) {
  const int sm = (int)(4 * sizeof(T) * (ldu + 1));
  if (sm > 48 * 1024) cudaFuncSetAttribute(hetrd_pupdate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  count_launch();
  hetrd_pupdate_kernel<T><<<dim3((j + 63) / 64, count), 256, sm, s>>>(A, lda, sA, j, u, p, sv, tau, stau, U, Q, ldu,
                                                                      sU, k, y, sy, rowupd, ticket, uw,
                                                                      hd ? hd->ud : nullptr, hd ? hd->sud : 0,
                                                                      hd ? hd->fu : nullptr, hd ? hd->rmax : nullptr,
                                                                      hd ? hd->ldd : 0);
}

template <typename T>
void hetrd_finish(const T* A, int lda, long long sA, int m, double* d, double* e, long long sde, T* ph,
                  long long sph, int count, cudaStream_t s) {
  count_launch();
  hetrd_finish_kernel<T><<<count, 256, 0, s>>>(A, lda, sA, m, d, e, sde, ph, sph);
}

template <typename T, typename TV>
void gather_reflectors(const T* A, int lda, long long sA, const double* tau, long long stau, int j0, int j1,
                       TV* V, int ldv, long long sV, double* tb, long long stb, int count, cudaStream_t s) {
  dim3 grid(1, j1 < 2048 ? j1 : 2048, count);
  count_launch();
  gather_reflectors_kernel<T, TV><<<grid, 64, 0, s>>>(A, lda, sA, tau, stau, j0, j1, V, ldv, sV, tb, stb);
}

// ph (FP64 type) from the single-precision phases of the mixed-precision path.
template <typename T, typename TV>
__global__ void widen_kernel(const T* src, TV* dst, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    dst[t] = widen(src[t]);
}

template <typename T, typename TV>
void widen_copy(const T* src, TV* dst, long long n, cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  const long long b = (n + 255) / 256;
  widen_kernel<T, TV><<<(int)(b < 4096 ? b : 4096), 256, 0, s>>>(src, dst, n);
}

// Lower triangle of the FP64 A (lda, sA) rounded into the single-precision B (ldb, sB).
template <typename T, typename TL>
__global__ void narrow_lower_kernel(const T* A, int lda, long long sA, TL* B, int ldb, long long sB, int n) {
  const int z = blockIdx.z;
  A += z * sA;
  B += z * sB;
  for (int i = blockIdx.y; i < n; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += gridDim.x * blockDim.x) {
      const T a = A[(size_t)i * lda + j];
      TL b;
      if constexpr (sizeof(T) == 16) b = TL{(float)re(a), (float)im(a)};
      else b = (TL)re(a);
      B[(size_t)i * ldb + j] = b;
    }
}

template <typename T, typename TL>
void narrow_lower(const T* A, int lda, long long sA, TL* B, int ldb, long long sB, int n, int count, cudaStream_t s) {
  if (n <= 0) return;
  dim3 grid((n + 255) / 256 < 16 ? (n + 255) / 256 : 16, n < 2048 ? n : 2048, count);
  count_launch();
  narrow_lower_kernel<T, TL><<<grid, 256, 0, s>>>(A, lda, sA, B, ldb, sB, n);
}

#define INST(T)                                                                                            \
  template void hetrd_reflector<T>(T*, int, long long, int, T*, long long, double*, long long, int,         \
                                   cudaStream_t, double*, const HemvDigits*);                              \
  template void hetrd_phemv<T>(const T*, int, long long, int, const T*, T*, long long, const double*,        \
                               long long, const T*, const T*, int, long long, int, T*, long long, T*, long long, \
                               int*, int, cudaStream_t, const double*, const double*, const HemvDigits*);  \
  template void hetrd_pupdate<T>(T*, int, long long, int, T*, const T*, long long, double*, long long, T*,  \
                                 T*, int, long long, int, const T*, long long, int, int*, int, cudaStream_t, \
                                 double*, const HemvDigits*);                                              \
  template void hetrd_finish<T>(const T*, int, long long, int, double*, double*, long long, T*, long long,   \
                                int, cudaStream_t);                                                        \
  template void gather_reflectors<T, T>(const T*, int, long long, const double*, long long, int, int, T*,    \
                                        int, long long, double*, long long, int, cudaStream_t);               \
  template void hetrd_digits<T>(const T*, int, long long, int, const HemvDigits&, int, cudaStream_t);
INST(double)
INST(zc)
#undef INST
#define INST(T)                                                                                            \
  template void hetrd_reflector<T>(T*, int, long long, int, T*, long long, double*, long long, int,         \
                                   cudaStream_t, double*, const HemvDigits*);                              \
  template void hetrd_phemv<T>(const T*, int, long long, int, const T*, T*, long long, const double*,        \
                               long long, const T*, const T*, int, long long, int, T*, long long, T*, long long, \
                               int*, int, cudaStream_t, const double*, const double*, const HemvDigits*);  \
  template void hetrd_pupdate<T>(T*, int, long long, int, T*, const T*, long long, double*, long long, T*,  \
                                 T*, int, long long, int, const T*, long long, int, int*, int, cudaStream_t, \
                                 double*, const HemvDigits*);                                              \
  template void hetrd_finish<T>(const T*, int, long long, int, double*, double*, long long, T*, long long,   \
                                int, cudaStream_t);
INST(float)
INST(cf)
template void gather_reflectors<float, double>(const float*, int, long long, const double*, long long, int, int,
                                               double*, int, long long, double*, long long, int, cudaStream_t);
template void gather_reflectors<cf, zc>(const cf*, int, long long, const double*, long long, int, int, zc*, int,
                                        long long, double*, long long, int, cudaStream_t);
template void widen_copy<float, double>(const float*, double*, long long, cudaStream_t);
template void widen_copy<cf, zc>(const cf*, zc*, long long, cudaStream_t);
template void narrow_lower<double, float>(const double*, int, long long, float*, int, long long, int, int,
                                          cudaStream_t);
template void narrow_lower<zc, cf>(const zc*, int, long long, cf*, int, long long, int, int, cudaStream_t);

}  // namespace gks
