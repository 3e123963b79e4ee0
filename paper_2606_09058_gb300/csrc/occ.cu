// Fermi-Dirac occupations, chemical potential and band energy (paper Sec. 3.1 Part 3,
// Sec. 3.2 Part 4; occupation f_i of Sec. 2).
//
//   f(x) = 1 / (1 + e^x),  x = (eps - mu) / kT, evaluated as e^-x/(1+e^-x) for x > 0;
//   N(mu) = sum_k w_k g_s sum_i f((eps_ki - mu)/kT) is increasing in mu, and mu solves
//   N(mu) = n_elec by bisection on [min eps - 1, max eps + 1] (stop when the bracket is
//   below 4u max(1, |mu|), at most 200 halvings);
//   E_band = sum_k w_k g_s sum_i f_ki eps_ki.
// Also writes kscale = g_s f (zero where f < f_cut) and n_rho(k) = #{i : f_ki >= f_cut},
// the leading columns kept in rho (eps ascending, so f is non-increasing in i).
#include <algorithm>

#include "dense.h"

namespace gks {

__device__ __forceinline__ double fermi_fn(double x) {
  if (x > 0.0) {
    double t = exp(-x);
    return t / (1.0 + t);
  }
  return 1.0 / (1.0 + exp(x));
}

// One CTA per system; system q owns k-points [q*nk, (q+1)*nk).
__global__ void __launch_bounds__(1024) fermi_mu_kernel(const double* eps, int m, int nk, const double* w, double gs,
                                                        double kT, double n_elec, double f_cut, double* occ,
                                                        double* kscale, double* mu_out, double* e_band,
                                                        int* nrho, DevStatus* st) {
  __shared__ double red[32];
  const int q = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const long long base = (long long)q * nk * m;
  eps += base;
  occ += base;
  kscale += base;
  const long long tot = (long long)nk * m;
  double lo, hi;
  {
    // min / max reductions
    double vmin = 1e300, vmax = -1e300;
    for (long long t = tid; t < tot; t += nt) { vmin = fmin(vmin, eps[t]); vmax = fmax(vmax, eps[t]); }
    for (int o = 16; o > 0; o >>= 1) {
      vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
      vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    __shared__ double smin[32], smax[32];
    if ((tid & 31) == 0) { smin[tid >> 5] = vmin; smax[tid >> 5] = vmax; }
    __syncthreads();
    if (tid < 32) {
      int nw = (nt + 31) >> 5;
      vmin = tid < nw ? smin[tid] : 1e300;
      vmax = tid < nw ? smax[tid] : -1e300;
      for (int o = 16; o > 0; o >>= 1) {
        vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      }
      if (tid == 0) { smin[0] = vmin; smax[0] = vmax; }
    }
    __syncthreads();
    lo = smin[0] - 1.0;
    hi = smax[0] + 1.0;
    __syncthreads();
  }
  double wsum = 0.0;
  for (int k = 0; k < nk; k++) wsum += w[k];
  const bool bad = !(kT > 0.0) || !(n_elec > 0.0) || !(n_elec < gs * m * wsum) || !isfinite(lo) || !isfinite(hi);
  if (bad) {
    if (tid == 0) set_status(st, ST_EINVAL, 0);
    return;
  }
  const double u = 1.1102230246251565e-16;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (hi - lo <= 4.0 * u * fmax(1.0, fabs(mid))) break;
    double s = 0.0;
    for (long long t = tid; t < tot; t += nt) s += w[t / m] * fermi_fn((eps[t] - mid) / kT);
    s = gs * block_sum(s, red);
    if (s < n_elec) lo = mid;
    else hi = mid;
  }
  const double mu = 0.5 * (lo + hi);
  double eb = 0.0;
  for (long long t = tid; t < tot; t += nt) {
    double f = fermi_fn((eps[t] - mu) / kT);
    occ[t] = f;
    kscale[t] = (f >= f_cut) ? gs * f : 0.0;
    eb += w[t / m] * gs * f * eps[t];
  }
  eb = block_sum(eb, red);
  if (tid == 0) {
    mu_out[q] = mu;
    e_band[q] = eb;
  }
  __syncthreads();
  for (int k = tid; k < nk; k += nt) {
    // f non-increasing along the ascending eigenvalues: binary search for the last kept
    const double* fk = occ + (long long)k * m;
    int lo_i = 0, hi_i = m;
    while (lo_i < hi_i) {
      int mid = (lo_i + hi_i) >> 1;
      if (fk[mid] >= f_cut) lo_i = mid + 1;
      else hi_i = mid;
    }
    nrho[(long long)q * nk + k] = lo_i;
  }
}

void fermi_mu(const double* eps, int m, int nk, const double* w, double gs, double kT, double n_elec, double f_cut,
              double* occ, double* kscale, double* mu, double* e_band, int* nrho, DevStatus* st, int nsys,
              cudaStream_t s) {
  count_launch();
  fermi_mu_kernel<<<nsys, 1024, 0, s>>>(eps, m, nk, w, gs, kT, n_elec, f_cut, occ, kscale, mu, e_band, nrho, st);
}

__global__ void expand_weights_kernel(const double* w, int nk, int rep, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nk * rep) return;
  const int k = t / rep;
  out[t] = w ? w[k] : 1.0 / nk;
}

void expand_weights(const double* w, int nk, int rep, double* out, cudaStream_t s) {
  count_launch();
  expand_weights_kernel<<<(nk * rep + 255) / 256, 256, 0, s>>>(w, nk, rep, out);
}

__global__ void clamp_nrho_kernel(int* nrho, int nk, int cols, DevStatus* st, int st_stride) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  if (nrho[k] > cols) {
    set_status(st ? st + (long long)k * st_stride : nullptr, ST_EINVAL, nrho[k]);
    nrho[k] = cols;
  }
}

void clamp_nrho(int* nrho, int nk, int cols, DevStatus* st, int st_stride, cudaStream_t s) {
  count_launch();
  clamp_nrho_kernel<<<(nk + 255) / 256, 256, 0, s>>>(nrho, nk, cols, st, st_stride);
}

__global__ void mul_elem_kernel(const double* a, const double* b, double* out, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = a[t] * b[t];
}

void mul_elem(const double* a, const double* b, double* out, long long n, cudaStream_t s) {
  count_launch();
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  mul_elem_kernel<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(a, b, out, n);
}

}  // namespace gks
