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

#include <mutex>

#include "dense.h"

namespace gks {

static constexpr int OZ_BITS = 6;
static constexpr int OZ_KSTEP = 64;   // k per pipeline step
static constexpr int OZ_CHUNK = 4096; // exact FP32 accumulation length (63*63*4096 < 2^24)

// ------------------------------------------------------------------ splitting

// Digits of one value already scaled below 1 in magnitude.  The first S base-64 digits
// of |r| truncated toward zero are the base-64 digits of the integer trunc(|r| 2^{6S})
// (6S <= 60 bits): one conversion, then integer shifts.
__device__ __forceinline__ void put_digits(double r, __nv_bfloat16* dst, long long sstride, int S) {
  const long long q = __double2ll_rz(ldexp(fabs(r), OZ_BITS * S));
  const float sg = r < 0.0 ? -1.0f : 1.0f;
  for (int s = 0; s < S; s++) {
    const int d = (int)((q >> (OZ_BITS * (S - 1 - s))) & 63);
    dst[s * sstride] = __float2bfloat16_rn(sg * (float)d);
  }
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

// Write the digits of element k of vector v (scaled by 2^-e) into the embedded layout.
template <typename T>
__device__ __forceinline__ void emit(T x, int e, int role, int v, int k, __nv_bfloat16* D, int Kp, long long sstride,
                                     int S);
template <>
__device__ __forceinline__ void emit<double>(double x, int e, int, int v, int k, __nv_bfloat16* D, int Kp,
                                             long long sstride, int S) {
  put_digits(ldexp(x, -e), D + (size_t)v * Kp + k, sstride, S);
}
template <>
__device__ __forceinline__ void emit<zc>(zc x, int e, int role, int v, int k, __nv_bfloat16* D, int Kp,
                                         long long sstride, int S) {
  const double re = ldexp(x.x, -e), im = ldexp(x.y, -e);
  if (role == 0) {
    put_digits(re, D + (size_t)v * Kp + 2 * k, sstride, S);
    put_digits(im, D + (size_t)v * Kp + 2 * k + 1, sstride, S);
  } else {
    __nv_bfloat16* r0 = D + (size_t)(2 * v) * Kp + 2 * k;
    __nv_bfloat16* r1 = D + (size_t)(2 * v + 1) * Kp + 2 * k;
    put_digits(re, r0, sstride, S);
    put_digits(-im, r0 + 1, sstride, S);
    put_digits(im, r1, sstride, S);
    put_digits(re, r1 + 1, sstride, S);
  }
}

// One CTA (256 threads) per 32 vectors.  Pass 1: per-vector max (thread per vector when the
// vector index is the contiguous direction, else a warp sweeps each vector along k).
// Pass 2: digits.  Padding vectors and k beyond K are written as zero digits elsewhere.
// blockIdx.y runs over the batch items (strides sX, sD, sE).  Optional per item: kdev
// (device) cuts K to its value, ksc scales element k by ksc[k] before splitting.
template <typename T>
__global__ void __launch_bounds__(256) oz_split_kernel(const T* X, int ld, long long sX, int role, int op, int nvec,
                                                       int K, __nv_bfloat16* D, int Kp, long long sstride,
                                                       long long sD, int S, int* ex, long long sE,
                                                       const double* ksc, long long sks, const int* kdev,
                                                       long long sX2, int nb2) {
  __shared__ double smax[32];
  __shared__ int sexp[32];
  const int v0 = blockIdx.x * 32, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  X += item_off(blockIdx.y, sX, sX2, nb2);
  D += blockIdx.y * sD;
  ex += blockIdx.y * sE;
  if (kdev) K = min(K, max(0, kdev[blockIdx.y]));
  if (ksc) ksc += blockIdx.y * sks;
  auto elem = [&](int v, int k) -> T {
    T x = split_elem(X, ld, role, op, v, k);
    return ksc ? x * ksc[k] : x;
  };
  const bool contig = (role == 0) == (op == OP_N);  // k contiguous in memory
  if (contig) {
    for (int vv = warp; vv < 32; vv += 8) {
      const int v = v0 + vv;
      double m = 0.0;
      if (v < nvec)
        for (int k = lane; k < K; k += 32) m = fmax(m, amax(elem(v, k)));
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) smax[vv] = m;
    }
  } else {
    // 8 warps sweep k in parallel, lanes run over the 32 vectors (coalesced), then reduce
    __shared__ double pm[8][32];
    double m = 0.0;
    const int v = v0 + lane;
    if (v < nvec)
      for (int k = warp; k < K; k += 8) m = fmax(m, amax(elem(v, k)));
    pm[warp][lane] = m;
    __syncthreads();
    if (tid < 32) {
      double mm = 0.0;
      for (int w = 0; w < 8; w++) mm = fmax(mm, pm[w][tid]);
      smax[tid] = mm;
    }
  }
  __syncthreads();
  if (tid < 32) {
    sexp[tid] = scale_exp(smax[tid]);
    if (v0 + tid < nvec) ex[v0 + tid] = sexp[tid];
  }
  __syncthreads();
  if (contig) {
    for (int vv = warp; vv < 32; vv += 8) {
      const int v = v0 + vv;
      if (v >= nvec) continue;
      for (int k = lane; k < K; k += 32) emit<T>(elem(v, k), sexp[vv], role, v, k, D, Kp, sstride, S);
    }
  } else {
    // k strided in memory: stage 32 (k) x 32 (vectors) tiles through shared memory so that
    // the reads run along the vectors and the digit writes along k
    __shared__ T tile[32][33];
    for (int k0 = 0; k0 < K; k0 += 32) {
      for (int kk = warp; kk < 32; kk += 8) {
        const int k = k0 + kk, v = v0 + lane;
        tile[kk][lane] = (k < K && v < nvec) ? elem(v, k) : zero<T>();
      }
      __syncthreads();
      for (int vv = warp; vv < 32; vv += 8) {
        const int v = v0 + vv, k = k0 + lane;
        if (v < nvec && k < K) emit<T>(tile[lane][vv], sexp[vv], role, v, k, D, Kp, sstride, S);
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ product kernel

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

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
constexpr int BM = 128, BN = 128, BK = 64;           // BK bf16 = 128 bytes = one swizzle row
constexpr int STAGES = 6;
constexpr int TILE_BYTES = BM * BK * 2;              // 16 KB per operand tile
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr int TMEM_COLS = 2 * BN;                    // two FP32 accumulators
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024;    // + alignment slack

// kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, both K-major, M x N.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

// k blocks per unit of level L: (L - 1) pairs, digit products up to 63^2.
__device__ __forceinline__ int level_blocks(int L) {
  const int cb = (int)((1u << 24) / ((unsigned)(L - 1) * 3969u * (unsigned)BK));
  return min(cb, OZ_CHUNK / BK);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false on abort or timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      *abort = 1;
      return false;
    }
  }
  return true;
}
// Wait without watching the abort flag (draining after an abort), still bounded.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile of 8-row groups 1024 bytes apart,
// 128-byte swizzle, descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// x 2^-s as a double, for x an integer-valued float (the exact unit sums): built from the
// float's bits with integer operations (sign, exponent shifted by 896 - s, mantissa moved
// up by 29 bits), so the drain spends one FP64 add per element and no FP64 conversion.
__device__ __forceinline__ double exact_scaled(uint32_t b, uint32_t s) {
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u - s) << 20) | ((b & 0x7fffffu) >> 3);
  const uint32_t lo = b << 29;
  return e ? __hiloint2double((int)hi, (int)lo) : 0.0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
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
static bool digit_map(CUtensorMap* m, const void* base, long long rows, int Kp) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)tcg::BK, (cuuint32_t)tcg::BM};
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

size_t ozaki_workspace_bytes(int M, int N, int K, bool cplx, int S) {
  const int Kp = padded_k(K, cplx);
  const int Mp = round_up(M, OZ_BM), Np = round_up(cplx ? 2 * N : N, OZ_BN);
  const size_t b = (size_t)S * ((size_t)Mp + Np) * Kp * 2 + sizeof(int) * ((size_t)Mp + Np) + 1024;
  return (b + 255) & ~size_t(255);
}

int ozaki_tiles(int M, int N, bool cplx) {
  return (round_up(M, OZ_BM) / OZ_BM) * (round_up(cplx ? 2 * N : N, OZ_BN) / OZ_BN);
}

// count items, item z at A + z sA, B + z sB, C + z sC.  work holds, for all items, the A
// digits [count][S][Mp][Kp], then the B digits [count][S][Np][Kp], then the exponents
// [count][Mp] and [count][Np] (within count * ozaki_workspace_bytes).
template <typename T>
bool ozaki_gemm(int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda, long long sA, const T* B,
                int ldb, long long sB, double beta, T* C, int ldc, long long sC, int count, int lower, int S,
                void* work, DevStatus* status, cudaStream_t s, const double* kscale, long long sks,
                const int* kdev, long long wait_cycles, long long skip_copy, long long sA2, long long sB2,
                long long sC2, int nb2) {
  if (M <= 0 || N <= 0 || count <= 0) return true;
  const bool cplx = sizeof(T) == 16;
  const int Kp = padded_k(K, cplx);
  const int Mp = round_up(M, OZ_BM), Np = round_up(cplx ? 2 * N : N, OZ_BN);
  const long long zA = (long long)S * Mp * Kp, zB = (long long)S * Np * Kp;
  __nv_bfloat16* Ad = static_cast<__nv_bfloat16*>(work);
  __nv_bfloat16* Bd = Ad + zA * count;
  int* ea = reinterpret_cast<int*>(Bd + zB * count);
  int* eb = ea + (size_t)Mp * count;
  // zero digits and exponents (padding rows/columns and k beyond K stay zero)
  cudaMemsetAsync(work, 0, ((size_t)(zA + zB) * 2 + sizeof(int) * ((size_t)Mp + Np)) * count, s);
  if (K > 0) {
    count_launch();
    oz_split_kernel<T><<<dim3((M + 31) / 32, count), 256, 0, s>>>(A, lda, sA, 0, opA, M, K, Ad, Kp,
                                                                   (long long)Mp * Kp, zA, S, ea, Mp, kscale, sks,
                                                                   kdev, sA2, nb2);
    count_launch();
    oz_split_kernel<T><<<dim3((N + 31) / 32, count), 256, 0, s>>>(B, ldb, sB, 1, opB, N, K, Bd, Kp,
                                                                   (long long)Np * Kp, zB, S, eb, Np, nullptr, 0,
                                                                   kdev, sB2, nb2);
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
  oa.S = S;
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
  oa.wait = wait_cycles > 0 ? wait_cycles : (1ll << 32);
  oa.skip_copy = skip_copy;
  dim3 grid(Np / OZ_BN, Mp / OZ_BM, count);
  CUtensorMap ma, mb;
  if (!digit_map(&ma, Ad, (long long)count * S * Mp, Kp) || !digit_map(&mb, Bd, (long long)count * S * Np, Kp))
    return false;
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
