// FP64-accurate GEMM from exact bf16 tensor-core products (split-integer products in the
// manner of Ozaki, Ogita, Oishi and Rump's error-free splitting).
//
// Each row i of op(A) is scaled by 2^-e_i (e_i = 1 + floor(log2 max_k |a_ik|), so every
// entry is below 1 in magnitude) and cut into S digits of 6 bits, truncating toward zero:
//   a_ik = 2^e_i * sum_{s=1..S} d_s(i,k) 2^{-6s} + r,  |d_s| <= 63,  |r| < 2^{e_i - 6S}.
// Columns of op(B) are cut the same way.  Every digit is an integer of at most 6 bits, so
// it is exact in bf16 and every digit product (< 2^12) and every sum of up to 4096 of them
// is exact in the FP32 accumulator of the bf16 mma.  The kernel multiplies the digit pairs
// with s + t <= S + 1 (the dropped pairs are below 2^{-6(S+1)}), drains each exact chunk
// into an FP64 accumulator scaled by 2^{-6(s+t)}, and applies 2^{e_i + f_j} at the end.
// With S = 9 the digits carry 54 bits below each row's largest entry.  (S <= 10 keeps the
// digit integer within 60 bits.)
//
// Complex products use a real embedding that keeps (Re, Im) of one output next to each
// other: A' = [Re a, Im a] interleaved along k, B' column 2j = (Re b, -Im b) interleaved,
// column 2j+1 = (Im b, Re b); then (A' B')[i][2j] = Re c_ij and [i][2j+1] = Im c_ij.
//
// On GB300 the bf16 tensor cores (tcgen05) run the 45 digit products of S = 9 at an
// FP64-equivalent rate of 13-18 TFLOP/s on large products, against 1.2 TFLOP/s for the
// FP64 pipe.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "dense.h"
#include "tcgen05.cuh"

namespace gks {

static constexpr int OZ_BITS = 6;
static constexpr int OZ_KSTEP = 64;   // k per pipeline step
static constexpr int OZ_CHUNK = 4096; // exact FP32 accumulation length (63*63*4096 < 2^24)

// ------------------------------------------------------------------ splitting

// ------------------------------------------------------------------ residue moduli
// Pairwise coprime moduli up to 256 (2^8, 3*5*17, 11*23, 251, 13*19, 241, 239, 233, 229,
// 227, 223, 7*31, 211, 199, 197, 193), largest first: a residue in symmetric form has
// |r| <= 128, an integer exact in bf16, and a product of two is at most 2^14.
static constexpr int CRT_MAXMOD = 16;
__host__ __device__ constexpr uint32_t crt_mod(int l) {
  return l == 0 ? 256u : l == 1 ? 255u : l == 2 ? 253u : l == 3 ? 251u : l == 4 ? 247u : l == 5 ? 241u
       : l == 6 ? 239u : l == 7 ? 233u : l == 8 ? 229u : l == 9 ? 227u : l == 10 ? 223u : l == 11 ? 217u
       : l == 12 ? 211u : l == 13 ? 199u : l == 14 ? 197u : 193u;
}

// The split values of one element x of a vector whose entries are below 2^e in magnitude,
// into o[0..S); sh = 6S - e (digits) or p - e (residues).
// Digits (RES false): the first S base-64 digits of |x| 2^-e truncated toward zero (the
// base-64 digits of the integer trunc(|x| 2^sh), 6S <= 60 bits), with the sign of x.
// Residues (RES true): q = trunc(x 2^sh), |q| < 2^p <= 2^62, modulo each of the first S
// moduli in symmetric form (|q| mod m from its two 32-bit halves, then q's sign).
template <bool RES>
__device__ __forceinline__ void split_vals(double x, int sh, int S, float (&o)[16]) {
  if constexpr (RES) {
    const long long q = __double2ll_rz(ldexp(x, sh));
    const unsigned long long u = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const float sg = q < 0 ? -1.0f : 1.0f;
#pragma unroll
    for (int l = 0; l < CRT_MAXMOD; l++) {
      const uint32_t m = crt_mod(l), w = (uint32_t)((1ull << 32) % m);
      const uint32_t r = l < S ? ((hi % m) * w + lo % m) % m : 0u;
      o[l] = sg * (float)(2u * r > m ? (int)r - (int)m : (int)r);
    }
  } else {
    const long long q = __double2ll_rz(ldexp(fabs(x), sh));
    const float sg = x < 0.0 ? -1.0f : 1.0f;
#pragma unroll
    for (int s = 0; s < 16; s++)
      o[s] = s < S ? sg * (float)((q >> (OZ_BITS * max(S - 1 - s, 0))) & 63) : 0.0f;
  }
}

__device__ __forceinline__ void store_vals(const float (&o)[16], float sg, __nv_bfloat16* dst, long long sstride,
                                           int S) {
#pragma unroll
  for (int s = 0; s < 16; s++)
    if (s < S) dst[s * sstride] = __float2bfloat16_rn(sg * o[s]);
}

__device__ __forceinline__ int scale_exp(double mx) {
  return mx > 0.0 ? ilogb(mx) + 1 : 0;
}

// Element k of vector v of the split operand.
// role 0 (A): vector v = row v of op(A);  role 1 (B): vector v = column v of op(B).
// op N/T/C on the stored matrix X (row-major, ld): op(A)_{v,k} = X[v][k] (N), X[k][v] (T),
// conj X[k][v] (C);  op(B)_{k,v} = X[k][v] (N), X[v][k] (T), conj X[v][k] (C).
template <typename T>
__device__ __forceinline__ T split_elem(const T* X, int ld, int role, int op, int v, int k) {
  const bool contig = (role == 0) == (op == OP_N);
  T x = contig ? X[(size_t)v * ld + k] : X[(size_t)k * ld + v];
  return op == OP_C ? conjg(x) : x;
}

__device__ __forceinline__ double amax(double x) { return fabs(x); }
__device__ __forceinline__ double amax(zc x) { return fmax(fabs(x.x), fabs(x.y)); }

// Write the split values of element k of vector v (scaled by 2^-e) into the embedded
// layout (complex B: column 2v = (Re, -Im), column 2v + 1 = (Im, Re) along k).
template <bool RES>
__device__ __forceinline__ void emit(double x, int e, int, int v, int k, __nv_bfloat16* D, int Kp, long long sstride,
                                     int S, int p) {
  float o[16];
  split_vals<RES>(x, (RES ? p : OZ_BITS * S) - e, S, o);
  store_vals(o, 1.0f, D + (size_t)v * Kp + k, sstride, S);
}
template <bool RES>
__device__ __forceinline__ void emit(zc x, int e, int role, int v, int k, __nv_bfloat16* D, int Kp, long long sstride,
                                     int S, int p) {
  float o[16];
  __nv_bfloat16* r0 = role == 0 ? D + (size_t)v * Kp + 2 * k : D + (size_t)(2 * v) * Kp + 2 * k;
  __nv_bfloat16* r1 = D + (size_t)(2 * v + 1) * Kp + 2 * k;
  const int sh = (RES ? p : OZ_BITS * S) - e;
  split_vals<RES>(x.x, sh, S, o);
  store_vals(o, 1.0f, r0, sstride, S);
  if (role != 0) store_vals(o, 1.0f, r1 + 1, sstride, S);
  split_vals<RES>(x.y, sh, S, o);
  if (role == 0) {
    store_vals(o, 1.0f, r0 + 1, sstride, S);
  } else {
    store_vals(o, -1.0f, r0 + 1, sstride, S);
    store_vals(o, 1.0f, r1, sstride, S);
  }
}

// Item z of the split operand with the optional per-item K (device) and k scaling.
template <typename T>
struct SplitSrc {
  const T* X;
  int ld, role, op;
  const double* ksc;
  __device__ T operator()(int v, int k) const {
    T x = split_elem(X, ld, role, op, v, k);
    return ksc ? x * ksc[k] : x;
  }
};

// Pass 1, one CTA (256 threads) per 32 vectors: the per-vector scale exponents (thread per
// vector when the vector index is the contiguous direction, else a warp sweeps each vector
// along k, four loads in flight per lane).  blockIdx.y runs over the batch items (strides
// sX, sE); kdev (device, per item) cuts K, ksc scales element k by ksc[k] first.
template <typename T>
__global__ void __launch_bounds__(256) oz_scale_kernel(const T* X, int ld, long long sX, int role, int op, int nvec,
                                                       int K, int* ex, long long sE, const double* ksc,
                                                       long long sks, const int* kdev, long long sX2, int nb2) {
  __shared__ double smax[32];
  __shared__ double pm[8][32];
  const int v0 = blockIdx.x * 32, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (kdev) K = min(K, max(0, kdev[blockIdx.y]));
  const SplitSrc<T> elem{X + item_off(blockIdx.y, sX, sX2, nb2), ld, role, op, ksc ? ksc + blockIdx.y * sks : nullptr};
  ex += blockIdx.y * sE;
  const bool contig = (role == 0) == (op == OP_N);  // k contiguous in memory
  if (contig) {
    for (int vv = warp; vv < 32; vv += 8) {
      const int v = v0 + vv;
      double m = 0.0;
      if (v < nvec)
        for (int k0 = lane; k0 < K; k0 += 128) {
          T x[4];
#pragma unroll
          for (int q = 0; q < 4; q++) x[q] = k0 + 32 * q < K ? elem(v, k0 + 32 * q) : zero<T>();
#pragma unroll
          for (int q = 0; q < 4; q++) m = fmax(m, amax(x[q]));
        }
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) smax[vv] = m;
    }
  } else {
    // 8 warps sweep k in parallel, lanes run over the 32 vectors (coalesced), then reduce
    double m = 0.0;
    const int v = v0 + lane;
    if (v < nvec)
      for (int k0 = warp; k0 < K; k0 += 32) {
        T x[4];
#pragma unroll
        for (int q = 0; q < 4; q++) x[q] = k0 + 8 * q < K ? elem(v, k0 + 8 * q) : zero<T>();
#pragma unroll
        for (int q = 0; q < 4; q++) m = fmax(m, amax(x[q]));
      }
    pm[warp][lane] = m;
    __syncthreads();
    if (tid < 32) {
      double mm = 0.0;
      for (int w = 0; w < 8; w++) mm = fmax(mm, pm[w][tid]);
      smax[tid] = mm;
    }
  }
  __syncthreads();
  if (tid < 32 && v0 + tid < nvec) ex[v0 + tid] = scale_exp(smax[tid]);
}

// Pass 2, one CTA (256 threads) per tile of 32 vectors x 32 k (grid x: vectors, y: k,
// z: items) over the padded plane: nvp vectors (padding rows included; complex B: half the
// embedded rows) and kpl k (complex: half the padded K').  The tile is staged through shared
// memory (read along the contiguous direction), then its S digits or residues (RES; residues
// of trunc(x 2^{p - e})) are written with lanes along k; padding vectors and k beyond K
// (the item's, after kdev) get the split values of zero, so the planes need no clearing.
template <typename T, bool RES>
__global__ void __launch_bounds__(256) oz_split_kernel(const T* X, int ld, long long sX, int role, int op, int nvec,
                                                       int K, __nv_bfloat16* D, int Kp, long long sstride,
                                                       long long sD, int S, int p, const int* ex, long long sE,
                                                       const double* ksc, long long sks, const int* kdev,
                                                       long long sX2, int nb2, int nvp, int kpl) {
  __shared__ T tile[32][33];
  __shared__ int sexp[32];
  const int v0 = blockIdx.x * 32, k0 = blockIdx.y * 32, z = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (kdev) K = min(K, max(0, kdev[z]));
  const SplitSrc<T> elem{X + item_off(z, sX, sX2, nb2), ld, role, op, ksc ? ksc + z * sks : nullptr};
  D += z * sD;
  ex += z * sE;
  if (tid < 32) sexp[tid] = v0 + tid < nvec ? ex[v0 + tid] : 0;
  if ((role == 0) == (op == OP_N)) {  // k contiguous: lanes along k
    for (int vv = warp; vv < 32; vv += 8) {
      const int v = v0 + vv, k = k0 + lane;
      tile[lane][vv] = (v < nvec && k < K) ? elem(v, k) : zero<T>();
    }
  } else {  // vectors contiguous: lanes along the vectors
    for (int kk = warp; kk < 32; kk += 8) {
      const int k = k0 + kk, v = v0 + lane;
      tile[kk][lane] = (k < K && v < nvec) ? elem(v, k) : zero<T>();
    }
  }
  __syncthreads();
  for (int vv = warp; vv < 32; vv += 8) {
    const int v = v0 + vv, k = k0 + lane;
    if (v < nvp && k < kpl) emit<RES>(tile[lane][vv], sexp[vv], role, v, k, D, Kp, sstride, S, p);
  }
}

// ------------------------------------------------------------------ product kernel

static constexpr int OZ_BM = 128, OZ_BN = 128;  // output tile of the product kernel

struct OzArgs {
  const __nv_bfloat16* Ad;  // [S][Mp][Kp]
  const __nv_bfloat16* Bd;  // [S][Np][Kp]   (embedded columns, K-major)
  const int* ea;            // exponents of the M rows
  const int* eb;            // exponents of the logical N columns
  void* C;
  int ldc;
  int M, N;                 // logical output (N complex columns when cplx)
  int Mp, Np, Kp;           // padded digit shapes (Np = embedded columns)
  int S;
  int cplx, lower;
  double alpha, beta;
  long long sAd, sBd;       // slice strides (elements)
  long long zAd, zBd, zEa, zEb, zC;  // batch item strides of the digits, exponents and C
  long long zC2;            // two-level batch (nb2 > 0): C of item z at (z / nb2) zC + (z % nb2) zC2
  int nb2;
  const int* kdev;          // optional per-item K read on the device (logical, <= K)
  long long wait;           // bound of every mbarrier wait, in SM clock cycles
  long long skip_copy;      // test hook: the producer leaves out this copy (-1 = none)
};

// ------------------------------------------------------------------ tcgen05 product kernel
//
// The same digit products on the 5th-generation tensor cores.  One CTA owns a 128 x 128
// output tile (of the embedded product) and walks the units in level order: a unit is a
// level L = s + t and a K chunk short enough that the sum over all pairs of the level,
// (L - 1) 63^2 chunk, stays within 2^24, so one FP32 accumulation holds every pair of the
// level exactly and a single drain (scale 2^{-6L}) serves them all.  Warp 0 streams
// 128 x 64 digit tiles of A slice s and B slice t into a
// ring of shared-memory stages with TMA (128-byte swizzle), one thread of warp 1 issues
// tcgen05.mma (M = N = 128, K = 16) into one of two FP32 accumulators in tensor memory,
// and eight epilogue warps read the finished accumulator with tcgen05.ld, scale it by
// 2^{-6L} and add it into FP64 registers (thread = one tile row x 64 columns), while
// the tensor cores fill the other accumulator.  Every wait is bounded: past the limit
// the CTA raises an abort flag and a timeout status, lets its copies and products land,
// frees its tensor memory and exits.
namespace tcg {
// k blocks per unit of level L: (L - 1) pairs, digit products up to 63^2.
__device__ __forceinline__ int level_blocks(int L) {
  const int cb = (int)((1u << 24) / ((unsigned)(L - 1) * 3969u * (unsigned)BK));
  return min(cb, OZ_CHUNK / BK);
}

// x 2^-s as a double, for x an integer-valued float (the exact unit sums): built from the
// float's bits with integer operations (sign, exponent shifted by 896 - s, mantissa moved
// up by 29 bits), so the drain spends one FP64 add per element and no FP64 conversion.
__device__ __forceinline__ double exact_scaled(uint32_t b, uint32_t s) {
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u - s) << 20) | ((b & 0x7fffffu) >> 3);
  const uint32_t lo = b << 29;
  return e ? __hiloint2double((int)hi, (int)lo) : 0.0;
}
}  // namespace tcg

__global__ void __launch_bounds__(tcg::THREADS, 1)
    oz_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs a,
                 DevStatus* status) {
  using namespace tcg;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // grouped tile order: consecutive CTAs walk 8 row tiles of one column tile, then the next
  // column tile, so the CTAs resident together share both operands' digit tiles in L2
  int m0, n0;
  {
    constexpr int G = 8;
    const int ntn = gridDim.x, ntm = gridDim.y;
    const int bid = blockIdx.y * ntn + blockIdx.x, per = G * ntn;
    const int fm = (bid / per) * G, gs = min(ntm - fm, G), r = bid % per;
    m0 = (fm + r % gs) * BM;
    n0 = (r / gs) * BN;
  }
  const int z = blockIdx.z;
  const int ncol0 = a.cplx ? n0 / 2 : n0;
  if (a.lower && m0 + BM - 1 < ncol0) return;  // whole tile above the diagonal (uniform)

  const int S = a.S;
  int kblocks = a.Kp / BK;
  if (a.kdev) {
    const int ke = min(a.Kp, max(0, a.kdev[z]) * (a.cplx ? 2 : 1));
    kblocks = (ke + BK - 1) / BK;
  }

  if (tid == 0) {
    for (int i = 0; i < STAGES; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  volatile int* abort = &abort_flag;

  double acc[64];
#pragma unroll
  for (int i = 0; i < 64; i++) acc[i] = 0.0;

  if (warp == 0) {
    if (lane == 0) {
      // producer: digit tiles of A slice s and B slice t, k block kb, in unit order
      long long q = 0;
      for (int L = 2; L <= S + 1 && !*abort; L++) {
        const int cb = level_blocks(L);
        for (int c0 = 0; c0 < kblocks && !*abort; c0 += cb) {
          const int c1 = min(kblocks, c0 + cb);
          for (int si = 1; si < L && !*abort; si++) {
            const int ya = (z * S + si - 1) * a.Mp + m0, yb = (z * S + (L - si) - 1) * a.Np + n0;
            for (int kb = c0; kb < c1; kb++, q++) {
              const int stg = (int)(q % STAGES);
              const uint32_t ph = (uint32_t)((q / STAGES) & 1);
              if (!mbar_wait(&empty[stg], ph ^ 1u, abort, a.wait)) break;
              if (q == a.skip_copy) continue;  // test hook: this stage never fills
              unsigned char* sa = ring + (size_t)stg * STAGE_BYTES;
              mbar_expect_tx(&full[stg], STAGE_BYTES);
              tma_load_2d(sa, &mapA, &full[stg], kb * BK, ya);
              tma_load_2d(sa + TILE_BYTES, &mapB, &full[stg], kb * BK, yb);
            }
          }
        }
      }
      // let every issued copy land before the CTA can leave
      for (long long r = (q > STAGES ? q - STAGES : 0); r < q; r++)
        if (r != a.skip_copy) mbar_drain(&full[r % STAGES], (uint32_t)((r / STAGES) & 1), a.wait);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      long long q = 0;
      int u = 0;
      bool ok = true;
      for (int L = 2; L <= S + 1 && ok; L++) {
        const int cb = level_blocks(L);
        for (int c0 = 0; c0 < kblocks && ok; c0 += cb, u++) {
          const int c1 = min(kblocks, c0 + cb);
          const int b = u & 1;
          const uint32_t uph = (uint32_t)((u >> 1) & 1);
          if (!mbar_wait(&tempty[b], uph ^ 1u, abort, a.wait)) {
            ok = false;
            break;
          }
          tc_fence_after();
          uint32_t accum = 0;
          for (int si = 1; si < L && ok; si++) {
            for (int kb = c0; kb < c1; kb++, q++) {
              const int stg = (int)(q % STAGES);
              const uint32_t ph = (uint32_t)((q / STAGES) & 1);
              if (!mbar_wait(&full[stg], ph, abort, a.wait)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t sa = smem_u32(ring + (size_t)stg * STAGE_BYTES);
              const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + TILE_BYTES);
#pragma unroll
              for (int kk = 0; kk < BK / 16; kk++) {
                umma(tmem + (uint32_t)(b * BN), da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), accum);
                accum = 1u;
              }
              umma_commit(&empty[stg]);
            }
          }
          if (!ok) break;
          umma_commit(&tfull[b]);
        }
      }
      // all issued products complete before tensor memory is released
      umma_commit(&done);
      mbar_drain(&done, 0, a.wait);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, column half (w - 2) / 4
    const int lq = warp & 3, ch = (warp - 2) >> 2;
    int u = 0;
    bool ok = true;
    for (int L = 2; L <= S + 1 && ok; L++) {
      const int cb = level_blocks(L);
      const uint32_t sh = (uint32_t)(OZ_BITS * L);
      for (int c0 = 0; c0 < kblocks; c0 += cb, u++) {
        const int b = u & 1;
        const uint32_t uph = (uint32_t)((u >> 1) & 1);
        if (!mbar_wait(&tfull[b], uph, abort, a.wait)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(b * BN + ch * 64);
        uint32_t v[32];
        tmem_ld32(taddr, v);
#pragma unroll
        for (int i = 0; i < 32; i++) acc[i] += exact_scaled(v[i], sh);
        tmem_ld32(taddr + 32, v);
#pragma unroll
        for (int i = 0; i < 32; i++) acc[32 + i] += exact_scaled(v[i], sh);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
  }
  if (*abort) {
    if (tid == 0) set_status(status, ST_ETIMEOUT, -2);
    return;
  }
  if (warp < 2) return;
  // C = alpha 2^{e_i + f_j} acc + beta C for this thread's row and 64 embedded columns
  const int lq = warp & 3, ch = (warp - 2) >> 2;
  const int i = m0 + lq * 32 + lane;
  if (i >= a.M) return;
  const long long zz = z;
  const int* ea = a.ea + zz * a.zEa;
  const int* eb = a.eb + zz * a.zEb;
  if (a.cplx) {
    zc* C = static_cast<zc*>(a.C) + item_off(z, a.zC, a.zC2, a.nb2);
    const int j0 = n0 / 2 + ch * 32;
#pragma unroll
    for (int jj = 0; jj < 32; jj++) {
      const int j = j0 + jj;
      if (j >= a.N || (a.lower && j > i)) continue;
      const int ee = ea[i] + eb[j];
      zc v{ldexp(acc[2 * jj], ee) * a.alpha, ldexp(acc[2 * jj + 1], ee) * a.alpha};
      zc* cp = C + (size_t)i * a.ldc + j;
      if (a.beta != 0.0) v = v + a.beta * (*cp);
      *cp = v;
    }
  } else {
    double* C = static_cast<double*>(a.C) + item_off(z, a.zC, a.zC2, a.nb2);
    const int j0 = n0 + ch * 64;
#pragma unroll
    for (int jj = 0; jj < 64; jj++) {
      const int j = j0 + jj;
      if (j >= a.N || (a.lower && j > i)) continue;
      double v = ldexp(acc[jj], ea[i] + eb[j]) * a.alpha;
      double* cp = C + (size_t)i * a.ldc + j;
      if (a.beta != 0.0) v += a.beta * (*cp);
      *cp = v;
    }
  }
}

// ------------------------------------------------------------------ residue products
//
// The modular form of the split product (the integer-modular scheme of Ozaki, Uchino and
// Imamura, here on the bf16 tensor cores).  Row i of op(A) is scaled by 2^{p - e_i} and
// truncated to integers A'_ik (|A'_ik| < 2^p), column j of op(B) the same, and the integer
// product X = A'B' is recovered from its residues modulo n pairwise coprime m_l by the
// Chinese remainder theorem, since |X| < Kp 2^{2p} <= M / 2 with M = m_1 ... m_n.  For each
// modulus the kernel multiplies the residue planes of A' and B' over K: symmetric residues
// are bf16-exact integers of magnitude <= 128, so a k chunk of 1024 sums exactly in the
// FP32 accumulator (<= 2^24).  Eight epilogue warps fold each chunk into a residue kept
// in FP32 registers (x - m round(x / m), exact on integers) while the tensor cores fill the
// other accumulator, and write t_l = (X mod m_l) y_l mod m_l of every element (the
// weight of the reconstruction, y_l = (M / m_l)^-1 mod m_l) as one byte when the modulus
// ends.  One product per modulus: 16 moduli keep p = 55 bits for K up to 16384, where nine
// 6-bit digits keep 54 bits with 45 digit-pair products.  crt_recon_kernel rebuilds X
// from its residues in 32-bit limbs and scales it back by 2^{e_i + f_j - 2p}.
constexpr int CRT_CHUNK_BLOCKS = 16;  // k blocks per exact chunk: 16 * 64 * 128^2 = 2^24

struct CrtArgs {
  const __nv_bfloat16* Ad;  // [count][n][Mp][Kp] residue planes of A'
  const __nv_bfloat16* Bd;  // [count][n][Np][Kp] residue planes of B' (embedded columns, K-major)
  uint8_t* R;               // [count][n][Mp][Np] residues of X
  int Mp, Np, Kp, n, cplx, lower;
  long long zR;             // item stride of R (bytes)
  float y[CRT_MAXMOD];      // (M / m_l)^-1 mod m_l: R holds t_l = (X mod m_l) y_l mod m_l
  const int* kdev;          // optional per-item K read on the device (logical, <= K)
  long long wait;           // bound of every mbarrier wait, in SM clock cycles
  long long skip_copy;      // test hook: the producer leaves out this copy (-1 = none)
};

// Tile of the residue kernel: 128 x 256 outputs per CTA (the B operand tile twice as wide as
// the digit-pair kernel's, so each A tile fetched into shared memory serves twice the MMA
// work), four stages of 48 KB, and two 256-column FP32 accumulators filling the 512 columns
// of tensor memory.
namespace crtc {
constexpr int BN = 256;
constexpr int STAGES = 4;
constexpr int B_BYTES = BN * tcg::BK * 2;
constexpr int STAGE_BYTES = tcg::TILE_BYTES + B_BYTES;
constexpr int TMEM_COLS = 2 * BN;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(tcg::BM >> 4) << 24);
static_assert(SMEM <= 227 * 1024, "shared memory of the residue kernel");
}  // namespace crtc

// x - m round(x / m) for an integer-valued float |x| <= 2^24: the quotient is rounded with
// the 1.5 * 2^23 shift (|x / m| < 2^22), and the fused multiply-add is exact because the
// result is a small integer.
__device__ __forceinline__ float crt_fold(float x, float m, float inv) {
  const float q = __fsub_rn(__fmaf_rn(x, inv, 12582912.0f), 12582912.0f);
  return __fmaf_rn(-q, m, x);
}

__global__ void __launch_bounds__(tcg::THREADS, 1)
    crt_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, CrtArgs a,
                  DevStatus* status) {
  using namespace tcg;
  using crtc::BN;
  using crtc::STAGE_BYTES;
  using crtc::STAGES;
  using crtc::TMEM_COLS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int m0, n0;  // grouped tile order, as in oz_tc_kernel
  {
    constexpr int G = 8;
    const int ntn = gridDim.x, ntm = gridDim.y;
    const int bid = blockIdx.y * ntn + blockIdx.x, per = G * ntn;
    const int fm = (bid / per) * G, gs = min(ntm - fm, G), r = bid % per;
    m0 = (fm + r % gs) * BM;
    n0 = (r / gs) * BN;
  }
  const int z = blockIdx.z;
  const int ncol0 = a.cplx ? n0 / 2 : n0;
  if (a.lower && m0 + BM - 1 < ncol0) return;  // whole tile above the diagonal (uniform)

  const int n = a.n;
  int kblocks = a.Kp / BK;
  if (a.kdev) {
    const int ke = min(a.Kp, max(0, a.kdev[z]) * (a.cplx ? 2 : 1));
    kblocks = (ke + BK - 1) / BK;
  }
  const int nchunk = (kblocks + CRT_CHUNK_BLOCKS - 1) / CRT_CHUNK_BLOCKS;

  if (tid == 0) {
    for (int i = 0; i < STAGES; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  volatile int* abort = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // producer: residue tiles of A' and B' for modulus l, k block kb
      long long q = 0;
      for (int l = 0; l < n && !*abort; l++) {
        const int ya = (z * n + l) * a.Mp + m0, yb = (z * n + l) * a.Np + n0;
        for (int kb = 0; kb < kblocks; kb++, q++) {
          const int stg = (int)(q % STAGES);
          const uint32_t ph = (uint32_t)((q / STAGES) & 1);
          if (!mbar_wait(&empty[stg], ph ^ 1u, abort, a.wait)) break;
          if (q == a.skip_copy) continue;  // test hook: this stage never fills
          unsigned char* sa = ring + (size_t)stg * STAGE_BYTES;
          mbar_expect_tx(&full[stg], STAGE_BYTES);
          tma_load_2d(sa, &mapA, &full[stg], kb * BK, ya);
          tma_load_2d(sa + TILE_BYTES, &mapB, &full[stg], kb * BK, yb);
        }
      }
      for (long long r = (q > STAGES ? q - STAGES : 0); r < q; r++)
        if (r != a.skip_copy) mbar_drain(&full[r % STAGES], (uint32_t)((r / STAGES) & 1), a.wait);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: one accumulator per (modulus, k chunk)
      long long q = 0;
      int u = 0;
      bool ok = true;
      for (int l = 0; l < n && ok; l++) {
        for (int c = 0; c < nchunk && ok; c++, u++) {
          const int b = u & 1;
          const uint32_t uph = (uint32_t)((u >> 1) & 1);
          if (!mbar_wait(&tempty[b], uph ^ 1u, abort, a.wait)) {
            ok = false;
            break;
          }
          tc_fence_after();
          uint32_t accum = 0;
          const int kb1 = min(kblocks, (c + 1) * CRT_CHUNK_BLOCKS);
          for (int kb = c * CRT_CHUNK_BLOCKS; kb < kb1; kb++, q++) {
            const int stg = (int)(q % STAGES);
            const uint32_t ph = (uint32_t)((q / STAGES) & 1);
            if (!mbar_wait(&full[stg], ph, abort, a.wait)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(ring + (size_t)stg * STAGE_BYTES);
            const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + TILE_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; kk++) {
              tcg::umma<crtc::IDESC>(tmem + (uint32_t)(b * BN), da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2),
                                     accum);
              accum = 1u;
            }
            umma_commit(&empty[stg]);
          }
          if (!ok) break;
          umma_commit(&tfull[b]);
        }
      }
      umma_commit(&done);
      mbar_drain(&done, 0, a.wait);
    }
  } else {
    // epilogue: warp w owns TMEM lanes 32 (w % 4) .. +31 (tile rows) and column half
    // (w - 2) / 4 (128 columns)
    const int lq = warp & 3, ch = (warp - 2) >> 2;
    const int i = m0 + lq * 32 + lane;
    int u = 0;
    bool ok = true;
    for (int l = 0; l < n && ok; l++) {
      const float mf = (float)crt_mod(l), inv = __frcp_rn(mf);
      float acc[128];
#pragma unroll
      for (int t = 0; t < 128; t++) acc[t] = 0.0f;
      for (int c = 0; c < nchunk; c++, u++) {
        const int b = u & 1;
        const uint32_t uph = (uint32_t)((u >> 1) & 1);
        if (!mbar_wait(&tfull[b], uph, abort, a.wait)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(b * BN + ch * 128);
#pragma unroll
        for (int g = 0; g < 4; g++) {
          uint32_t v[32];
          tmem_ld32(taddr + 32 * g, v);
#pragma unroll
          for (int t = 0; t < 32; t++) acc[32 * g + t] += crt_fold(__uint_as_float(v[t]), mf, inv);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      if (!ok) break;
      // t_l = (X mod m_l) y_l mod m_l in [0, m_l) for this thread's row and 128 embedded
      // columns, one byte each (both folds exact: |acc| < 2^24, r y_l < 2^16)
      const float yl = a.y[l];
      uint4* dst = reinterpret_cast<uint4*>(a.R + z * a.zR + ((size_t)l * a.Mp + i) * a.Np + n0 + ch * 128);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        uint32_t w[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
          uint32_t word = 0;
#pragma unroll
          for (int s4 = 0; s4 < 4; s4++) {
            float r = crt_fold(acc[16 * q + 4 * t + s4], mf, inv);
            r = r < 0.0f ? r + mf : r;
            r = crt_fold(r * yl, mf, inv);
            r = r < 0.0f ? r + mf : r;
            r = r >= mf ? r - mf : r;
            word |= (uint32_t)r << (8 * s4);
          }
          w[t] = word;
        }
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
  }
  if (*abort && tid == 0) set_status(status, ST_ETIMEOUT, -2);
}

// Constants of the reconstruction for n moduli: X = sum_l t_l (M / m_l) mod M with
// t_l = r_l y_l mod m_l, y_l = (M / m_l)^-1 mod m_l (t_l is what the product kernel stores).
struct CrtRecon {
  uint32_t y[CRT_MAXMOD];
  uint32_t Nl[CRT_MAXMOD][4];  // M / m_l, 32-bit limbs, least significant first
  uint32_t Mv[4], Mh[4];       // M and M / 2
  float inv_mf;                // 2^{32 b} / M
  int b;                       // limb at which the quotient estimate starts: max(0, top limb of M - 1)
  int n;
};

// 128-bit magnitude (hi, lo) to the nearest double (ties to even), from its bits.
__device__ __forceinline__ double u128_to_double(unsigned long long hi, unsigned long long lo) {
  if (hi == 0ull && lo == 0ull) return 0.0;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  unsigned long long h, l;
  if (lz == 0) {
    h = hi;
    l = lo;
  } else if (lz < 64) {
    h = (hi << lz) | (lo >> (64 - lz));
    l = lo << lz;
  } else {
    h = lo << (lz - 64);
    l = 0ull;
  }
  unsigned long long mant = h >> 11;  // 53 significant bits
  const unsigned long long rest = h & 0x7ffull;
  if (rest > 0x400ull || (rest == 0x400ull && (l != 0ull || (mant & 1ull)))) mant++;
  int ex = 127 - lz;  // position of the leading bit
  if (mant >> 53) {
    mant >>= 1;
    ex++;
  }
  return __longlong_as_double((long long)(((unsigned long long)(ex + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

__device__ __forceinline__ bool ge4(const uint32_t (&x)[4], const uint32_t (&y)[4]) {
  for (int t = 3; t >= 0; t--)
    if (x[t] != y[t]) return x[t] > y[t];
  return true;
}

// The signed integer X with X y_l = t_l (mod m_l) for the weighted residues t_l (byte el of
// the 16 loaded for modulus l), |X| < M / 2, as a double times 2^e.
__device__ __forceinline__ double crt_value(const uint32_t (&w)[CRT_MAXMOD][4], int el, const CrtRecon& cr, int e) {
  uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;  // S = sum_l t_l M / m_l < 16 M
#pragma unroll
  for (int l = 0; l < CRT_MAXMOD; l++) {
    if (l < cr.n) {
      const uint32_t t = (w[l][el >> 2] >> (8 * (el & 3))) & 0xffu;
      unsigned long long c = (unsigned long long)t * cr.Nl[l][0] + s0;
      s0 = (uint32_t)c;
      c = (c >> 32) + (unsigned long long)t * cr.Nl[l][1] + s1;
      s1 = (uint32_t)c;
      c = (c >> 32) + (unsigned long long)t * cr.Nl[l][2] + s2;
      s2 = (uint32_t)c;
      c = (c >> 32) + (unsigned long long)t * cr.Nl[l][3] + s3;
      s3 = (uint32_t)c;
      s4 += (uint32_t)(c >> 32);
    }
  }
  // q = floor(S / M) within one: S / M < 16 estimated from the three limbs of S from limb b
  // up (M 2^{-32 b} >= 2^32 unless M < 2^32, so the limbs below b do not matter)
  const uint32_t a2 = cr.b == 0 ? s2 : cr.b == 1 ? s3 : s4;
  const uint32_t a1 = cr.b == 0 ? s1 : cr.b == 1 ? s2 : s3;
  const uint32_t a0 = cr.b == 0 ? s0 : cr.b == 1 ? s1 : s2;
  const float sf = __fmaf_rn((float)a2, 18446744073709551616.0f, __fmaf_rn((float)a1, 4294967296.0f, (float)a0));
  const unsigned q = (unsigned)(sf * cr.inv_mf);
  uint32_t x[4];
  long long d = 0;
  unsigned long long pm = 0;
  const uint32_t sl[4] = {s0, s1, s2, s3};
#pragma unroll
  for (int t = 0; t < 4; t++) {
    pm += (unsigned long long)q * cr.Mv[t];
    d += (long long)sl[t] - (long long)(uint32_t)pm;
    x[t] = (uint32_t)d;
    d >>= 32;
    pm >>= 32;
  }
  d += (long long)s4 - (long long)pm;  // the top limb: -1, 0 or 1 after one of the corrections below
  if (d < 0) {  // q one too large: X += M
    unsigned long long c = 0;
#pragma unroll
    for (int t = 0; t < 4; t++) {
      c += (unsigned long long)x[t] + cr.Mv[t];
      x[t] = (uint32_t)c;
      c >>= 32;
    }
  } else if (d > 0 || ge4(x, cr.Mv)) {  // q one too small: X -= M
    long long b = 0;
#pragma unroll
    for (int t = 0; t < 4; t++) {
      b += (long long)x[t] - (long long)cr.Mv[t];
      x[t] = (uint32_t)b;
      b >>= 32;
    }
  }
  // symmetric representative: X > M / 2 stands for X - M
  bool neg = false;
  if (!ge4(cr.Mh, x)) {
    neg = true;
    long long b = 0;
#pragma unroll
    for (int t = 0; t < 4; t++) {
      b += (long long)cr.Mv[t] - (long long)x[t];
      x[t] = (uint32_t)b;
      b >>= 32;
    }
  }
  const double v = u128_to_double(((unsigned long long)x[3] << 32) | x[2], ((unsigned long long)x[1] << 32) | x[0]);
  return ldexp(neg ? -v : v, e);
}

// C = alpha 2^{e_i + f_j - 2p} X + beta C for the logical outputs (lower: j <= i only).
// A thread takes 16 consecutive embedded columns of a row: one 16-byte load per modulus (the
// residue planes are Np bytes per row, Np a multiple of 256), then the 16 values (8 complex).
template <typename T>
__global__ void __launch_bounds__(128) crt_recon_kernel(const uint8_t* R, long long zR, int Mp, int Np, int M, int N,
                                                        const int* ea, const int* eb, long long zEa, long long zEb,
                                                        int sc, const CrtRecon cr, T* C, int ldc, long long zC,
                                                        long long zC2, int nb2, double alpha, double beta,
                                                        int lower) {
  constexpr bool CPX = sizeof(T) == 16;
  constexpr int PER = CPX ? 8 : 16;  // logical columns per thread
  const int z = blockIdx.z, j0 = (blockIdx.x * 128 + threadIdx.x) * PER;
  if (j0 >= N) return;
  const long long plane = (long long)Mp * Np;
  for (int i = blockIdx.y; i < M; i += gridDim.y) {
    if (lower && j0 > i) continue;
    const uint8_t* Rz = R + z * zR + (size_t)i * Np + (CPX ? 2 * j0 : j0);
    uint32_t w[CRT_MAXMOD][4];
#pragma unroll
    for (int l = 0; l < CRT_MAXMOD; l++) {
      if (l < cr.n) {
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(Rz + l * plane));
        w[l][0] = v.x;
        w[l][1] = v.y;
        w[l][2] = v.z;
        w[l][3] = v.w;
      } else {
        w[l][0] = w[l][1] = w[l][2] = w[l][3] = 0u;
      }
    }
    const int ei = ea[z * zEa + i] + sc;
    T* cp = C + item_off(z, zC, zC2, nb2) + (size_t)i * ldc;
#pragma unroll
    for (int q = 0; q < PER; q++) {
      const int j = j0 + q;
      if (j >= N || (lower && j > i)) break;
      const int e = ei + eb[z * zEb + j];
      if constexpr (CPX) {
        zc v{alpha * crt_value(w, 2 * q, cr, e), alpha * crt_value(w, 2 * q + 1, cr, e)};
        if (beta != 0.0) v = v + beta * cp[j];
        cp[j] = v;
      } else {
        double v = alpha * crt_value(w, q, cr, e);
        if (beta != 0.0) v += beta * cp[j];
        cp[j] = v;
      }
    }
  }
}

// ---- tensor maps (driver entry point looked up once through the runtime)
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
  });
  return fn;
}

// 2-D bf16 map over rows x Kp (row stride Kp), box 64 (k) x 128 (rows), 128-byte swizzle.
static bool digit_map(CUtensorMap* m, const void* base, long long rows, int Kp, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)tcg::BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ------------------------------------------------------------------ host

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Digit planes of an item: the same padded shapes ozaki_gemm uses (K = 0 still takes one
// 64-wide k block of zero digits, so that the product kernel computes C = beta C).
static int padded_k(int K, bool cplx) {
  const int Ke = cplx ? 2 * K : K;
  return round_up(Ke > 0 ? Ke : 1, OZ_KSTEP);
}

// Residue plan for padded length Kp and at least `bits` bits per operand: the fewest
// moduli n whose product M satisfies 2 Kp 2^{2p} <= M with p >= bits (p as large as M
// allows, at most 62), and the reconstruction constants.  False if 16 moduli fall short.
struct CrtPlan {
  int n, p;
  CrtRecon cr;
};
static bool crt_plan(int Kp, int bits, CrtPlan* pl) {
  typedef unsigned __int128 u128;
  u128 M = 1;
  for (int n = 1; n <= CRT_MAXMOD; n++) {
    M *= crt_mod(n - 1);
    const u128 room = M / ((u128)2 * (u128)Kp);  // 2^{2p} <= room
    int lg = -1;
    for (u128 t = room; t; t >>= 1) lg++;
    const int p = lg < 0 ? -1 : std::min(lg / 2, 62);
    if (p < bits) continue;
    pl->n = n;
    pl->p = p;
    CrtRecon& c = pl->cr;
    c = CrtRecon{};
    c.n = n;
    int top = 0;
    for (int t = 0; t < 4; t++) {
      c.Mv[t] = (uint32_t)(M >> (32 * t));
      c.Mh[t] = (uint32_t)((M >> 1) >> (32 * t));
      if (c.Mv[t]) top = t;
    }
    c.b = std::max(0, top - 1);
    c.inv_mf = (float)(std::ldexp(1.0, 32 * c.b) / (double)M);
    for (int l = 0; l < n; l++) {
      const uint32_t m = crt_mod(l);
      const u128 Nl = M / m;
      for (int t = 0; t < 4; t++) c.Nl[l][t] = (uint32_t)(Nl >> (32 * t));
      const uint32_t r = (uint32_t)(Nl % m);
      uint32_t y = 1;
      while ((r * y) % m != 1u) y++;  // r is coprime to m
      c.y[l] = y;
    }
    return true;
  }
  return false;
}

// S > 0: S digits of 6 bits (digit-pair products); S < 0: residues carrying at least 6|S|
// bits (digit pairs again when 16 moduli cannot).
static bool residue_form(int S, int Kp, CrtPlan* pl) { return S < 0 && crt_plan(Kp, OZ_BITS * -S, pl); }

// Embedded output columns padded to the product kernel's tile width.
static int padded_n(int N, bool cplx, bool res) { return round_up(cplx ? 2 * N : N, res ? crtc::BN : OZ_BN); }

size_t ozaki_workspace_bytes(int M, int N, int K, bool cplx, int S) {
  const int Kp = padded_k(K, cplx);
  CrtPlan pl;
  const bool res = residue_form(S, Kp, &pl);
  const int Mp = round_up(M, OZ_BM), Np = padded_n(N, cplx, res);
  size_t b;
  if (res)
    b = (size_t)pl.n * (((size_t)Mp + Np) * Kp * 2 + (size_t)Mp * Np);
  else
    b = (size_t)std::abs(S) * ((size_t)Mp + Np) * Kp * 2;
  b += sizeof(int) * ((size_t)Mp + Np) + 1024;
  return (b + 255) & ~size_t(255);
}

int ozaki_tiles(int M, int N, bool cplx) {
  return (round_up(M, OZ_BM) / OZ_BM) * (round_up(cplx ? 2 * N : N, OZ_BN) / OZ_BN);
}

// count items, item z at A + z sA, B + z sB, C + z sC.  work holds, for all items, the A
// planes [count][P][Mp][Kp], then the B planes [count][P][Np][Kp] (P = S digits or n
// residues), then (residues) the residues of the product [count][n][Mp][Np] as bytes, then
// the exponents [count][Mp] and [count][Np] (within count * ozaki_workspace_bytes).
template <typename T>
bool ozaki_gemm(int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda, long long sA, const T* B,
                int ldb, long long sB, double beta, T* C, int ldc, long long sC, int count, int lower, int S,
                void* work, DevStatus* status, cudaStream_t s, const double* kscale, long long sks,
                const int* kdev, long long wait_cycles, long long skip_copy, long long sA2, long long sB2,
                long long sC2, int nb2) {
  if (M <= 0 || N <= 0 || count <= 0) return true;
  const bool cplx = sizeof(T) == 16;
  const int Kp = padded_k(K, cplx);
  CrtPlan pl;
  const bool res = residue_form(S, Kp, &pl);
  const int Mp = round_up(M, OZ_BM), Np = padded_n(N, cplx, res);
  const int P = res ? pl.n : std::abs(S);  // planes per operand
  const long long zA = (long long)P * Mp * Kp, zB = (long long)P * Np * Kp;
  const long long zR = res ? (long long)P * Mp * Np : 0;
  __nv_bfloat16* Ad = static_cast<__nv_bfloat16*>(work);
  __nv_bfloat16* Bd = Ad + zA * count;
  uint8_t* R = reinterpret_cast<uint8_t*>(Bd + zB * count);
  int* ea = reinterpret_cast<int*>(R + zR * count);
  int* eb = ea + (size_t)Mp * count;
  // exponents zero for the padding rows and columns; the planes are written whole by the
  // split kernels (zeros in the padding), also for K = 0
  cudaMemsetAsync(ea, 0, sizeof(int) * ((size_t)Mp + Np) * count, s);
  {
    // padded extents in the split kernels' terms: vectors (complex B: embedded rows 2v, 2v + 1)
    // and logical k (complex: positions 2k, 2k + 1 of the padded K')
    const int nva = Mp, nvb = cplx ? Np / 2 : Np, kpl = cplx ? Kp / 2 : Kp;
    const dim3 ga((M + 31) / 32, count), gb((N + 31) / 32, count);
    const dim3 ta((nva + 31) / 32, (kpl + 31) / 32, count), tb((nvb + 31) / 32, (kpl + 31) / 32, count);
    count_launch(4);
    oz_scale_kernel<T><<<ga, 256, 0, s>>>(A, lda, sA, 0, opA, M, K, ea, Mp, kscale, sks, kdev, sA2, nb2);
    oz_scale_kernel<T><<<gb, 256, 0, s>>>(B, ldb, sB, 1, opB, N, K, eb, Np, nullptr, 0, kdev, sB2, nb2);
    if (res) {
      oz_split_kernel<T, true><<<ta, 256, 0, s>>>(A, lda, sA, 0, opA, M, K, Ad, Kp, (long long)Mp * Kp, zA, P, pl.p,
                                                  ea, Mp, kscale, sks, kdev, sA2, nb2, nva, kpl);
      oz_split_kernel<T, true><<<tb, 256, 0, s>>>(B, ldb, sB, 1, opB, N, K, Bd, Kp, (long long)Np * Kp, zB, P, pl.p,
                                                  eb, Np, nullptr, 0, kdev, sB2, nb2, nvb, kpl);
    } else {
      oz_split_kernel<T, false><<<ta, 256, 0, s>>>(A, lda, sA, 0, opA, M, K, Ad, Kp, (long long)Mp * Kp, zA, P, 0,
                                                   ea, Mp, kscale, sks, kdev, sA2, nb2, nva, kpl);
      oz_split_kernel<T, false><<<tb, 256, 0, s>>>(B, ldb, sB, 1, opB, N, K, Bd, Kp, (long long)Np * Kp, zB, P, 0,
                                                   eb, Np, nullptr, 0, kdev, sB2, nb2, nvb, kpl);
    }
  }
  const long long wait = wait_cycles > 0 ? wait_cycles : (1ll << 32);
  dim3 grid(Np / (res ? crtc::BN : OZ_BN), Mp / OZ_BM, count);
  CUtensorMap ma, mb;
  if (!digit_map(&ma, Ad, (long long)count * P * Mp, Kp, tcg::BM) ||
      !digit_map(&mb, Bd, (long long)count * P * Np, Kp, res ? crtc::BN : tcg::BN))
    return false;
  if (res) {
    CrtArgs ca;
    ca.Ad = Ad;
    ca.Bd = Bd;
    ca.R = R;
    ca.Mp = Mp;
    ca.Np = Np;
    ca.Kp = Kp;
    ca.n = P;
    ca.cplx = cplx ? 1 : 0;
    ca.lower = lower;
    ca.zR = zR;
    ca.kdev = kdev;
    ca.wait = wait;
    ca.skip_copy = skip_copy;
    for (int l = 0; l < CRT_MAXMOD; l++) ca.y[l] = l < P ? (float)pl.cr.y[l] : 0.0f;
    cudaFuncSetAttribute(crt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, crtc::SMEM);
    count_launch(2);
    crt_tc_kernel<<<grid, tcg::THREADS, crtc::SMEM, s>>>(ma, mb, ca, status);
    const int per = cplx ? 8 : 16;
    crt_recon_kernel<T><<<dim3((N + 128 * per - 1) / (128 * per), std::min(M, 65535), count), 128, 0, s>>>(
        R, zR, Mp, Np, M, N, ea, eb, Mp, Np, -2 * pl.p, pl.cr, C, ldc, sC, sC2, nb2, alpha, beta, lower);
    return true;
  }
  OzArgs oa;
  oa.Ad = Ad;
  oa.Bd = Bd;
  oa.ea = ea;
  oa.eb = eb;
  oa.C = C;
  oa.ldc = ldc;
  oa.M = M;
  oa.N = N;
  oa.Mp = Mp;
  oa.Np = Np;
  oa.Kp = Kp;
  oa.S = P;
  oa.cplx = cplx ? 1 : 0;
  oa.lower = lower;
  oa.alpha = alpha;
  oa.beta = beta;
  oa.sAd = (long long)Mp * Kp;
  oa.sBd = (long long)Np * Kp;
  oa.zAd = zA;
  oa.zBd = zB;
  oa.zEa = Mp;
  oa.zEb = Np;
  oa.zC = sC;
  oa.zC2 = sC2;
  oa.nb2 = nb2;
  oa.kdev = kdev;
  oa.wait = wait;
  oa.skip_copy = skip_copy;
  cudaFuncSetAttribute(oz_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tcg::SMEM);
  count_launch();
  oz_tc_kernel<<<grid, tcg::THREADS, tcg::SMEM, s>>>(ma, mb, oa, status);
  return true;
}

template bool ozaki_gemm<double>(int, int, int, int, int, double, const double*, int, long long, const double*, int,
                                 long long, double, double*, int, long long, int, int, int, void*, DevStatus*,
                                 cudaStream_t, const double*, long long, const int*, long long, long long,
                                 long long, long long, long long, int);
template bool ozaki_gemm<zc>(int, int, int, int, int, double, const zc*, int, long long, const zc*, int, long long,
                             double, zc*, int, long long, int, int, int, void*, DevStatus*, cudaStream_t,
                             const double*, long long, const int*, long long, long long, long long, long long,
                             long long, int);

}  // namespace gks
