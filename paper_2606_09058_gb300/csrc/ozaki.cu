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
// On GB300 the legacy bf16 mma.sync path runs at about 606 TFLOP/s (measured), so the 45
// digit products of S = 9 still deliver roughly ten times the DFMA rate of an FP64 GEMM.
#include <cuda_bf16.h>

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
// blockIdx.y runs over the batch items (strides sX, sD, sE).
template <typename T>
__global__ void __launch_bounds__(256) oz_split_kernel(const T* X, int ld, long long sX, int role, int op, int nvec,
                                                       int K, __nv_bfloat16* D, int Kp, long long sstride,
                                                       long long sD, int S, int* ex, long long sE) {
  __shared__ double smax[32];
  __shared__ int sexp[32];
  const int v0 = blockIdx.x * 32, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  X += blockIdx.y * sX;
  D += blockIdx.y * sD;
  ex += blockIdx.y * sE;
  const bool contig = (role == 0) == (op == OP_N);  // k contiguous in memory
  if (contig) {
    for (int vv = warp; vv < 32; vv += 8) {
      const int v = v0 + vv;
      double m = 0.0;
      if (v < nvec)
        for (int k = lane; k < K; k += 32) m = fmax(m, amax(split_elem(X, ld, role, op, v, k)));
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) smax[vv] = m;
    }
  } else {
    // 8 warps sweep k in parallel, lanes run over the 32 vectors (coalesced), then reduce
    __shared__ double pm[8][32];
    double m = 0.0;
    const int v = v0 + lane;
    if (v < nvec)
      for (int k = warp; k < K; k += 8) m = fmax(m, amax(split_elem(X, ld, role, op, v, k)));
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
      for (int k = lane; k < K; k += 32) emit<T>(split_elem(X, ld, role, op, v, k), sexp[vv], role, v, k, D, Kp, sstride, S);
    }
  } else {
    // k strided in memory: stage 32 (k) x 32 (vectors) tiles through shared memory so that
    // the reads run along the vectors and the digit writes along k
    __shared__ T tile[32][33];
    for (int k0 = 0; k0 < K; k0 += 32) {
      for (int kk = warp; kk < 32; kk += 8) {
        const int k = k0 + kk, v = v0 + lane;
        tile[kk][lane] = (k < K && v < nvec) ? split_elem(X, ld, role, op, v, k) : zero<T>();
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

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(sdst)), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

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
  long long zAd, zBd, zE, zC;  // batch item strides of the digits, exponents and C
};

static constexpr int OZ_BM = 128, OZ_BN = 128, OZ_LDS = OZ_KSTEP + 8, OZ_STAGES = 2;
static constexpr int OZ_ACC_LD = OZ_BN + 2;  // padded FP64 accumulator rows (drain bank spread)
static constexpr int OZ_SMEM = OZ_BM * OZ_ACC_LD * 8 + OZ_STAGES * (OZ_BM + OZ_BN) * OZ_LDS * 2;

__global__ void __launch_bounds__(256, 1) oz_gemm_kernel(OzArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* acc64 = reinterpret_cast<double*>(smem_raw);  // [128][OZ_ACC_LD]
  __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(smem_raw + OZ_BM * OZ_ACC_LD * 8);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, warp tile 64 x 32
  const int m0 = blockIdx.y * OZ_BM, n0 = blockIdx.x * OZ_BN;
  {
    const long long z = blockIdx.z;
    a.Ad += z * a.zAd;
    a.Bd += z * a.zBd;
    a.ea += z * a.zE;
    a.eb += z * a.zE;
    a.C = static_cast<char*>(a.C) + z * a.zC * (a.cplx ? 16 : 8);
  }
  // lower triangle of the logical output: skip tiles strictly above the diagonal
  const int ncol0 = a.cplx ? n0 / 2 : n0;
  if (a.lower && m0 + OZ_BM - 1 < ncol0) return;
  for (int e = tid; e < OZ_BM * OZ_ACC_LD; e += 256) acc64[e] = 0.0;

  // pairs (s, t), s + t <= S + 1, s,t >= 1
  const int S = a.S;
  const int ksteps = a.Kp / OZ_KSTEP;
  int npairs = 0;
  for (int s = 1; s <= S; s++) npairs += (S + 1 - s);
  const long long total = (long long)npairs * ksteps;
  const int chunk_steps = OZ_CHUNK / OZ_KSTEP;

  auto pair_of = [&](int p, int& s, int& t) {
    int q = p;
    for (s = 1; s <= S; s++) {
      int cnt = S + 1 - s;
      if (q < cnt) { t = 1 + q; return; }
      q -= cnt;
    }
  };
  auto stage_ptr = [&](int stg) { return st + (size_t)stg * (OZ_BM + OZ_BN) * OZ_LDS; };
  auto load_step = [&](long long q, int stg) {
    const int p = (int)(q / ksteps), kk = (int)(q % ksteps);
    int s, t;
    pair_of(p, s, t);
    const __nv_bfloat16* ga = a.Ad + (size_t)(s - 1) * a.sAd + (size_t)m0 * a.Kp + (size_t)kk * OZ_KSTEP;
    const __nv_bfloat16* gb = a.Bd + (size_t)(t - 1) * a.sBd + (size_t)n0 * a.Kp + (size_t)kk * OZ_KSTEP;
    __nv_bfloat16* sa = stage_ptr(stg);
    __nv_bfloat16* sb = sa + OZ_BM * OZ_LDS;
    // 128 rows x OZ_KSTEP bf16 = 128 x (OZ_KSTEP/8) chunks of 16 B for each operand
    constexpr int CPR = OZ_KSTEP / 8;
    for (int c = tid; c < OZ_BM * CPR; c += 256) {
      int r = c / CPR, cc = (c % CPR) * 8;
      cp_async16(sa + r * OZ_LDS + cc, ga + (size_t)r * a.Kp + cc);
      cp_async16(sb + r * OZ_LDS + cc, gb + (size_t)r * a.Kp + cc);
    }
  };

  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) acc[i][j][r] = 0.f;

  // prologue
  for (int stg = 0; stg < OZ_STAGES - 1; stg++) {
    if (stg < total) load_step(stg, stg);
    cp_commit();
  }
  __syncthreads();
  for (long long q = 0; q < total; q++) {
    cp_wait<OZ_STAGES - 2>();
    __syncthreads();
    {
      long long nq = q + OZ_STAGES - 1;
      if (nq < total) load_step(nq, (int)(nq % OZ_STAGES));
      cp_commit();
    }
    const __nv_bfloat16* sa = stage_ptr((int)(q % OZ_STAGES));
    const __nv_bfloat16* sb = sa + OZ_BM * OZ_LDS;
    uint32_t af[2][4][4], bf[2][4][2];
    auto load_frags = [&](int k16, int buf) {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int row = wm * 64 + i * 16 + (lane & 15);
        const int col = k16 + (lane >> 4) * 8;
        ldsm_x4(af[buf][i][0], af[buf][i][1], af[buf][i][2], af[buf][i][3], sa + row * OZ_LDS + col);
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        // two n8 blocks x two k halves: matrices (n 0-7,k0), (n 0-7,k8), (n 8-15,k0), (n 8-15,k8)
        const int nrow = wn * 32 + j * 8 + (lane & 7) + ((lane >> 4) << 3);
        const int col = k16 + ((lane >> 3) & 1) * 8;
        uint32_t r0, r1, r2, r3;
        ldsm_x4(r0, r1, r2, r3, sb + nrow * OZ_LDS + col);
        bf[buf][j][0] = r0;
        bf[buf][j][1] = r1;
        bf[buf][j + 1][0] = r2;
        bf[buf][j + 1][1] = r3;
      }
    };
    load_frags(0, 0);
#pragma unroll
    for (int ks = 0; ks < OZ_KSTEP / 16; ks++) {
      const int cur = ks & 1;
      if (ks + 1 < OZ_KSTEP / 16) load_frags((ks + 1) * 16, cur ^ 1);
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], af[cur][i], bf[cur][j][0], bf[cur][j][1]);
    }
    // drain at the end of each exact chunk and of each pair
    const int kk = (int)(q % ksteps);
    if (kk == ksteps - 1 || (kk + 1) % chunk_steps == 0) {
      int s, t;
      pair_of((int)(q / ksteps), s, t);
      const double sc = ldexp(1.0, -OZ_BITS * (s + t));
      const int g = lane >> 2, tq = lane & 3;
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int r = wm * 64 + i * 16 + g, c = wn * 32 + j * 8 + tq * 2;
          acc64[r * OZ_ACC_LD + c] += sc * (double)acc[i][j][0];
          acc64[r * OZ_ACC_LD + c + 1] += sc * (double)acc[i][j][1];
          acc64[(r + 8) * OZ_ACC_LD + c] += sc * (double)acc[i][j][2];
          acc64[(r + 8) * OZ_ACC_LD + c + 1] += sc * (double)acc[i][j][3];
#pragma unroll
          for (int rr = 0; rr < 4; rr++) acc[i][j][rr] = 0.f;
        }
    }
  }
  cp_wait<0>();
  __syncthreads();
  // epilogue: C = alpha 2^{e_i + f_j} acc + beta C
  if (a.cplx) {
    zc* C = static_cast<zc*>(a.C);
    for (int e = tid; e < OZ_BM * (OZ_BN / 2); e += 256) {
      const int r = e / (OZ_BN / 2), cj = e % (OZ_BN / 2);
      const int i = m0 + r, j = n0 / 2 + cj;
      if (i >= a.M || j >= a.N || (a.lower && j > i)) continue;
      const int ee = a.ea[i] + a.eb[j];
      zc v{ldexp(acc64[r * OZ_ACC_LD + 2 * cj], ee) * a.alpha, ldexp(acc64[r * OZ_ACC_LD + 2 * cj + 1], ee) * a.alpha};
      zc* cp = C + (size_t)i * a.ldc + j;
      if (a.beta != 0.0) v = v + a.beta * (*cp);
      *cp = v;
    }
  } else {
    double* C = static_cast<double*>(a.C);
    for (int e = tid; e < OZ_BM * OZ_BN; e += 256) {
      const int r = e / OZ_BN, c = e % OZ_BN;
      const int i = m0 + r, j = n0 + c;
      if (i >= a.M || j >= a.N || (a.lower && j > i)) continue;
      double v = ldexp(acc64[r * OZ_ACC_LD + c], a.ea[i] + a.eb[j]) * a.alpha;
      double* cp = C + (size_t)i * a.ldc + j;
      if (a.beta != 0.0) v += a.beta * (*cp);
      *cp = v;
    }
  }
}

// ------------------------------------------------------------------ host

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

size_t ozaki_workspace_bytes(int M, int N, int K, bool cplx, int S) {
  const int Kp = round_up(cplx ? 2 * K : K, OZ_KSTEP);
  const int Mp = round_up(M, OZ_BM), Np = round_up(cplx ? 2 * N : N, OZ_BN);
  const size_t b = (size_t)S * ((size_t)Mp + Np) * Kp * 2 + sizeof(int) * ((size_t)Mp + Np) + 1024;
  return (b + 255) & ~size_t(255);
}

int ozaki_tiles(int M, int N, bool cplx) {
  return (round_up(M, OZ_BM) / OZ_BM) * (round_up(cplx ? 2 * N : N, OZ_BN) / OZ_BN);
}

// count items, item z at A + z sA, B + z sB, C + z sC; work holds count workspaces of
// ozaki_workspace_bytes each.
template <typename T>
void ozaki_gemm(int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda, long long sA, const T* B,
                int ldb, long long sB, double beta, T* C, int ldc, long long sC, int count, int lower, int S,
                void* work, cudaStream_t s) {
  if (M <= 0 || N <= 0 || count <= 0) return;
  const bool cplx = sizeof(T) == 16;
  const int Ke = cplx ? 2 * K : K;
  const int Kp = round_up(Ke > 0 ? Ke : 1, OZ_KSTEP);
  const int Mp = round_up(M, OZ_BM), Np = round_up(cplx ? 2 * N : N, OZ_BN);
  const size_t item = ozaki_workspace_bytes(M, N, K, cplx, S);
  // per item: A digits [S][Mp][Kp], B digits [S][Np][Kp], then Mp + Np exponents
  __nv_bfloat16* Ad = static_cast<__nv_bfloat16*>(work);
  __nv_bfloat16* Bd = Ad + (size_t)S * Mp * Kp;
  int* ea = reinterpret_cast<int*>(Bd + (size_t)S * Np * Kp);
  int* eb = ea + Mp;
  const long long zD = (long long)(item / 2), zE = (long long)(item / sizeof(int));
  // zero digits and exponents (padding rows/columns and k beyond K stay zero)
  cudaMemsetAsync(work, 0, item * count, s);
  if (K > 0) {
    count_launch();
    oz_split_kernel<T><<<dim3((M + 31) / 32, count), 256, 0, s>>>(A, lda, sA, 0, opA, M, K, Ad, Kp,
                                                                   (long long)Mp * Kp, zD, S, ea, zE);
    count_launch();
    oz_split_kernel<T><<<dim3((N + 31) / 32, count), 256, 0, s>>>(B, ldb, sB, 1, opB, N, K, Bd, Kp,
                                                                   (long long)Np * Kp, zD, S, eb, zE);
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
  oa.zAd = zD;
  oa.zBd = zD;
  oa.zE = zE;
  oa.zC = sC;
  cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  dim3 grid(Np / OZ_BN, Mp / OZ_BM, count);
  count_launch();
  oz_gemm_kernel<<<grid, 256, OZ_SMEM, s>>>(oa);
}

template void ozaki_gemm<double>(int, int, int, int, int, double, const double*, int, long long, const double*, int,
                                 long long, double, double*, int, long long, int, int, int, void*, cudaStream_t);
template void ozaki_gemm<zc>(int, int, int, int, int, double, const zc*, int, long long, const zc*, int, long long,
                             double, zc*, int, long long, int, int, int, void*, cudaStream_t);

}  // namespace gks
