// Adjoint (vector-Jacobian product) of eps, rho and E_band with respect to H and S.
//
// First-order perturbation of H C = S C eps with C^H S C = I gives, for M = C^H dH C and
// N = C^H dS C: d eps_i = M_ii - eps_i N_ii and, at fixed mu,
//   d rho = g_s C [G o M - G' o N] C^H,
//   G_ij = (f_i - f_j)/(eps_i - eps_j),  G'_ij = (f_i eps_i - f_j eps_j)/(eps_i - eps_j).
// The fixed electron count moves mu by sum w f' d eps / sum w f'.  The VJP collects into
//   H_bar = C [g_s G o W + diag(e)] C^H,   S_bar = -C [g_s G' o W + diag(eps e)] C^H,
// with W = C^H rho_bar C and the effective eigenvalue weights e (see adj_weights_kernel).
//
// G is evaluated without cancellation: with a = x_i/2, b = x_j/2, x = (eps - mu)/kT and
// d = a - b, f_i - f_j = -sinh(d) sech(a) sech(b)/2 and eps_i - eps_j = 2 kT d, so
//   G_ij = -sinhc(d) sech(a) sech(b) / (4 kT),
// computed from exponentials of non-positive arguments (no overflow); d -> 0 gives f'.
#include "dense.h"

namespace gks {

__device__ __forceinline__ double fermi_of(double x) {
  if (x > 0.0) {
    double t = exp(-x);
    return t / (1.0 + t);
  }
  return 1.0 / (1.0 + exp(x));
}

__device__ __forceinline__ double gamma_fd(double xi, double xj, double kT) {
  const double a = 0.5 * xi, b = 0.5 * xj, d = a - b;
  const double fa = fabs(a), fb = fabs(b);
  const double ea = exp(-2.0 * fa), eb = exp(-2.0 * fb);
  const double den = (1.0 + ea) * (1.0 + eb);
  if (fabs(d) < 1e-3) {
    const double d2 = d * d;
    const double sinhc = 1.0 + d2 / 6.0 * (1.0 + d2 / 20.0);
    return -sinhc * 4.0 * exp(-fa - fb) / den / (4.0 * kT);
  }
  const double sh = 2.0 * (exp(d - fa - fb) - exp(-d - fa - fb)) / den;  // sinh(d) sech(a) sech(b)
  return -sh / (d * 4.0 * kT);
}

// f, f' per (k, i); one grid over nk * M.
__global__ void adj_occ_kernel(const double* eps, const double* mu, double kT, long long tot, double* f,
                               double* fp) {
  const double m = *mu;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    double x = (eps[t] - m) / kT;
    double fv = fermi_of(x);
    f[t] = fv;
    fp[t] = -fv * (1.0 - fv) / kT;
  }
}

// Effective eigenvalue weights (one CTA):
//   e_ki = eps_bar_ki + E_bar g_s w_k (f + eps f') + A w_k f'_ki / sum w f',
//   A = -g_s sum_k sum_i f'_ki Re W_k,ii - E_bar g_s sum_k w_k sum_i f'_ki eps_ki.
template <typename T>
__global__ void __launch_bounds__(1024) adj_weights_kernel(const double* eps, const double* f, const double* fp,
                                                           const double* w, const T* W, long long sW, int M, int nk,
                                                           double gs, const double* eps_bar, double e_band_bar,
                                                           int have_w, double* e) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long tot = (long long)nk * M;
  double s_wfp = 0.0, s_a = 0.0;
  for (long long t = tid; t < tot; t += nt) {
    const int k = (int)(t / M), i = (int)(t % M);
    s_wfp += w[k] * fp[t];
    double aw = 0.0;
    if (have_w) aw = re(W[k * sW + (size_t)i * M + i]);
    s_a += -gs * fp[t] * aw - e_band_bar * gs * w[k] * fp[t] * eps[t];
  }
  const double wfp = block_sum(s_wfp, red);
  const double A = block_sum(s_a, red);
  for (long long t = tid; t < tot; t += nt) {
    const int k = (int)(t / M);
    double v = eps_bar ? eps_bar[t] : 0.0;
    v += e_band_bar * gs * w[k] * (f[t] + eps[t] * fp[t]);
    if (wfp != 0.0) v += A * w[k] * fp[t] / wfp;
    e[t] = v;
  }
}

// BH = g_s G o W + diag(e), BS = -(g_s G' o W + diag(eps e)); W is overwritten by BS.
template <typename T>
__global__ void adj_build_kernel(T* W, T* BH, long long sW, int M, const double* eps, const double* f,
                                 const double* e, const double* mu, double kT, double gs, int have_w) {
  const int z = blockIdx.z;
  W += z * sW;
  BH += z * sW;
  eps += (long long)z * M;
  f += (long long)z * M;
  e += (long long)z * M;
  const double m = *mu;
  for (int i = blockIdx.y; i < M; i += gridDim.y) {
    const double ei = eps[i], xi = (ei - m) / kT, fi = f[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
      const double ej = eps[j];
      const double g = gamma_fd(xi, (ej - m) / kT, kT);
      const double gp = 0.5 * (fi + f[j]) + 0.5 * (ei + ej) * g;
      T wv = have_w ? W[(size_t)i * M + j] : zero<T>();
      T bh = (gs * g) * wv;
      T bs = (-gs * gp) * wv;
      if (i == j) {
        bh = bh + from_real<T>(e[i]);
        bs = bs - from_real<T>(ei * e[i]);
      }
      BH[(size_t)i * M + j] = bh;
      W[(size_t)i * M + j] = bs;
    }
  }
}

// dst = (src + src^H)/2 (in place allowed: each thread owns the pair (i, j), (j, i), i >= j).
template <typename T>
__global__ void herm_part_kernel(T* dst, const T* src, long long sd, long long ss, int M) {
  const int z = blockIdx.z;
  dst += z * sd;
  src += z * ss;
  for (int i = blockIdx.y; i < M; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += gridDim.x * blockDim.x) {
      T a = src[(size_t)i * M + j], b = src[(size_t)j * M + i];
      T v = 0.5 * (a + conjg(b));
      dst[(size_t)i * M + j] = v;
      dst[(size_t)j * M + i] = conjg(v);
    }
}

// S_bar (n x n) = Hermitian part of the sum of the two diagonal spin blocks of the 2n x 2n
// gradient (S_NC = diag(S, S)).
template <typename T>
__global__ void spin_block_sum_kernel(T* dst, long long sd, const T* src, long long ss, int n) {
  const int z = blockIdx.z;
  dst += z * sd;
  src += z * ss;
  const int m = 2 * n;
  for (int i = blockIdx.y; i < n; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      T a = src[(size_t)i * m + j] + src[(size_t)(i + n) * m + j + n];
      T b = src[(size_t)j * m + i] + src[(size_t)(j + n) * m + i + n];
      dst[(size_t)i * n + j] = 0.5 * (a + conjg(b));
    }
}

// Spin-polarized runs: S_bar_k (n x n) = Hermitian part of the sum of the gradients of the
// two spin channels (items 2k and 2k+1), which share S_k.
template <typename T>
__global__ void spin_pair_sum_kernel(T* dst, long long sd, const T* src, long long ss, int n) {
  const int z = blockIdx.z;
  dst += z * sd;
  const T* s0 = src + (2 * (long long)z) * ss;
  const T* s1 = s0 + ss;
  for (int i = blockIdx.y; i < n; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
      T a = s0[(size_t)i * n + j] + s1[(size_t)i * n + j];
      T b = s0[(size_t)j * n + i] + s1[(size_t)j * n + i];
      dst[(size_t)i * n + j] = 0.5 * (a + conjg(b));
    }
}

static dim3 g2(int rows, int cols, int count) {
  int gx = (cols + 255) / 256;
  if (gx > 16) gx = 16;
  if (gx < 1) gx = 1;
  return dim3(gx, rows < 2048 ? (rows > 0 ? rows : 1) : 2048, count);
}

void adj_occ(const double* eps, const double* mu, double kT, long long tot, double* f, double* fp, cudaStream_t s) {
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  count_launch();
  adj_occ_kernel<<<blocks, 256, 0, s>>>(eps, mu, kT, tot, f, fp);
}

template <typename T>
void adj_weights(const double* eps, const double* f, const double* fp, const double* w, const T* W, long long sW,
                 int M, int nk, double gs, const double* eps_bar, double e_band_bar, int have_w, double* e,
                 cudaStream_t s) {
  count_launch();
  adj_weights_kernel<T><<<1, 1024, 0, s>>>(eps, f, fp, w, W, sW, M, nk, gs, eps_bar, e_band_bar, have_w, e);
}

template <typename T>
void adj_build(T* W, T* BH, long long sW, int M, const double* eps, const double* f, const double* e,
               const double* mu, double kT, double gs, int have_w, int nk, cudaStream_t s) {
  count_launch();
  adj_build_kernel<T><<<g2(M, M, nk), 256, 0, s>>>(W, BH, sW, M, eps, f, e, mu, kT, gs, have_w);
}

template <typename T>
void herm_part(T* dst, const T* src, long long sd, long long ss, int M, int nk, cudaStream_t s) {
  count_launch();
  herm_part_kernel<T><<<g2(M, M, nk), 256, 0, s>>>(dst, src, sd, ss, M);
}

template <typename T>
void spin_block_sum(T* dst, long long sd, const T* src, long long ss, int n, int nk, cudaStream_t s) {
  count_launch();
  spin_block_sum_kernel<T><<<g2(n, n, nk), 256, 0, s>>>(dst, sd, src, ss, n);
}

template <typename T>
void spin_pair_sum(T* dst, long long sd, const T* src, long long ss, int n, int nk, cudaStream_t s) {
  count_launch();
  spin_pair_sum_kernel<T><<<g2(n, n, nk), 256, 0, s>>>(dst, sd, src, ss, n);
}

#define INST(T)                                                                                            \
  template void adj_weights<T>(const double*, const double*, const double*, const double*, const T*,        \
                               long long, int, int, double, const double*, double, int, double*,            \
                               cudaStream_t);                                                              \
  template void adj_build<T>(T*, T*, long long, int, const double*, const double*, const double*,           \
                             const double*, double, double, int, int, cudaStream_t);                       \
  template void herm_part<T>(T*, const T*, long long, long long, int, int, cudaStream_t);                   \
  template void spin_block_sum<T>(T*, long long, const T*, long long, int, int, cudaStream_t);              \
  template void spin_pair_sum<T>(T*, long long, const T*, long long, int, int, cudaStream_t);
INST(double)
INST(zc)

}  // namespace gks
