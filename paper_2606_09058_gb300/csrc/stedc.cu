// Divide-and-conquer eigensolver for the real symmetric tridiagonal T (paper Sec. 6:
// the GEMM-rich second half of the dense eigensolve; written here from Cuppen's method
// with Gu-Eisenstat vector recomputation).
//
//  * Tear: T = diag(T1, T2) + rho v v^T at every split s (rho = |e_{s-1}|,
//    v = (e_last; sign e_first)), i.e. d_{s-1} -= rho and d_s -= rho before the leaves.
//  * Leaves (<= 32 rows): one warp each runs implicit QL redundantly on every lane, lane
//    i accumulating row i of the leaf's eigenvector block.
//  * Merge of (lam1, Z1), (lam2, Z2): z = (last row of Z1; sign * first row of Z2)/sqrt2,
//    rho' = 2 rho; poles merged in ascending order; deflation of negligible z_i and of
//    close pole pairs (Givens rotation); the K remaining roots of
//    1 + rho' sum z_i^2/(d_i - lam) = 0 are found by bisection in tau = lam - d_origin
//    (origin the nearer pole) so that every difference d_i - lam = (d_i - d_origin) - tau is
//    accurate; z_hat is recomputed from the roots (Gu-Eisenstat) so the vectors
//    z_hat_i/(d_i - lam_j) are numerically orthogonal.
//  * The merged eigenvector matrix is diag(Z1, Z2) W, W = G^T [unit vectors | secular
//    vectors] in ascending eigenvalue order: two GEMMs per merge (Z1 W_top, Z2 W_bottom),
//    grouped over all merges of a level and all batch items in one launch.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dense.h"

namespace gks {

static constexpr int DC_LEAF = 32;
static constexpr double DC_U = 1.1102230246251565e-16;

struct DcNode {
  int off, n1, n2;
};

struct DcLevel {
  std::vector<DcNode> nodes;
  DcNode* d_nodes = nullptr;
  GemmDesc* d_gemm = nullptr;
  int maxn = 0, maxhalf = 0;
};

struct DcPlan {
  int m = 0, count = 0, depth = 0;
  std::vector<DcLevel> levels;  // levels[t]: t = 0 merges leaves, t = depth-1 is the root
  std::vector<int> leaves;      // (off, n) pairs
  std::vector<int> splits;      // split positions s (tear between s-1 and s)
  int* d_leaves = nullptr;
  int* d_splits = nullptr;
  const double* zbound = nullptr;  // Z pointer the GEMM lists were built for
  void* wbound = nullptr;
  long long sZbound = 0;
};

// per-item workspace layout (all arrays of length m)
struct DcWs {
  double *Zb, *W, *lamA, *lamB, *ds, *zs, *dK, *zK, *lamK, *tauK, *zhat, *dD, *rc, *rs;
  int *src, *idxK, *orig, *idxD, *ra, *rb, *colsrc, *cnt;
};

__host__ __device__ inline size_t dc_item_bytes(int m) {
  size_t mm = (size_t)m * m;
  return sizeof(double) * (2 * mm + 14 * (size_t)m) + sizeof(int) * (10 * (size_t)m) + 256;
}

__host__ __device__ inline DcWs dc_ws(void* base, int m) {
  DcWs w;
  double* pd = static_cast<double*>(base);
  const size_t mm = (size_t)m * m;
  w.Zb = pd; pd += mm;
  w.W = pd; pd += mm;
  double** dl[14] = {&w.lamA, &w.lamB, &w.ds, &w.zs, &w.dK, &w.zK, &w.lamK, &w.tauK, &w.zhat, &w.dD, &w.rc, &w.rs,
                     nullptr, nullptr};
  for (int k = 0; k < 12; k++) { *dl[k] = pd; pd += m; }
  int* pi = reinterpret_cast<int*>(pd);
  int** il[8] = {&w.src, &w.idxK, &w.orig, &w.idxD, &w.ra, &w.rb, &w.colsrc, &w.cnt};
  for (int k = 0; k < 7; k++) { *il[k] = pi; pi += m; }
  w.cnt = pi;
  return w;
}

// ------------------------------------------------------------------ kernels

__global__ void dc_tear_kernel(double* d, const double* e, long long sde, const int* splits, int nsplit) {
  const int z = blockIdx.x;
  if (threadIdx.x != 0) return;
  d += z * sde;
  e += z * sde;
  for (int k = 0; k < nsplit; k++) {
    int s = splits[k];
    double rho = fabs(e[s - 1]);
    d[s - 1] -= rho;
    d[s] -= rho;
  }
}

// One warp per leaf. Every lane runs the same QL iteration on private copies of (d, e);
// lane i applies the rotations to row i of the leaf's eigenvector block.
__global__ void dc_leaf_kernel(const double* d, const double* e, long long sde, double* lam, long long slam,
                               double* Z, long long sZ, int m, const int* leaves, int nleaves, DevStatus* st) {
  const int z = blockIdx.y;
  const int leaf = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (leaf >= nleaves) return;
  const int off = leaves[2 * leaf], n = leaves[2 * leaf + 1];
  d += z * sde;
  e += z * sde;
  lam += z * slam;
  Z += z * sZ;
  double dd[DC_LEAF], ee[DC_LEAF], zr[DC_LEAF];
  for (int i = 0; i < n; i++) {
    dd[i] = d[off + i];
    ee[i] = (i + 1 < n) ? e[off + i] : 0.0;
    zr[i] = (i == lane) ? 1.0 : 0.0;
  }
  bool ok = true;
  for (int l = 0; l < n && ok; l++) {
    for (int sweep = 0;; sweep++) {
      int q = l;
      while (q < n - 1) {
        if (fabs(ee[q]) <= DC_U * (fabs(dd[q]) + fabs(dd[q + 1]))) { ee[q] = 0.0; break; }
        q++;
      }
      if (q == l) break;
      if (sweep >= 60) { ok = false; break; }
      // shift: eigenvalue of [[d_l, e_l], [e_l, d_{l+1}]] nearer to d_l
      double h = 0.5 * (dd[l + 1] - dd[l]);
      double r = hypot(h, ee[l]);
      double mu = dd[l] - ee[l] * ee[l] / (h + copysign(r, h));
      double x = dd[q] - mu, y = ee[q - 1];
      for (int k = q; k > l; k--) {
        double rr = hypot(x, y);
        double c = rr > 0.0 ? x / rr : 1.0, s = rr > 0.0 ? y / rr : 0.0;
        if (k < q) ee[k] = rr;
        double a = dd[k - 1], b = ee[k - 1], g = dd[k];
        double cs = c * s;
        dd[k - 1] = c * c * a - 2.0 * cs * b + s * s * g;
        dd[k] = s * s * a + 2.0 * cs * b + c * c * g;
        ee[k - 1] = cs * (a - g) + (c * c - s * s) * b;
        double z0 = zr[k - 1], z1 = zr[k];
        zr[k - 1] = c * z0 - s * z1;
        zr[k] = s * z0 + c * z1;
        if (k - 1 > l) {
          x = ee[k - 1];
          y = s * ee[k - 2];
          ee[k - 2] = c * ee[k - 2];
        }
      }
    }
  }
  if (!ok) {
    if (lane == 0) set_status(st ? st + z : nullptr, ST_ENOCONV, off);
  }
  // ascending order by selection (ties keep the lower index)
  int perm[DC_LEAF];
  for (int i = 0; i < n; i++) perm[i] = i;
  for (int i = 0; i < n; i++) {
    int b = i;
    for (int k = i + 1; k < n; k++)
      if (dd[perm[k]] < dd[perm[b]]) b = k;
    int t = perm[i]; perm[i] = perm[b]; perm[b] = t;
  }
  for (int c = 0; c < n; c++) {
    if (lane == 0) lam[off + c] = dd[perm[c]];
    if (lane < n) Z[(size_t)(off + lane) * m + off + c] = zr[perm[c]];
  }
}

__device__ __forceinline__ int lower_bound_d(const double* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (a[mid] < v) lo = mid + 1; else hi = mid; }
  return lo;
}
__device__ __forceinline__ int upper_bound_d(const double* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) { int mid = (lo + hi) >> 1; if (a[mid] <= v) lo = mid + 1; else hi = mid; }
  return lo;
}

struct DcArgs {
  int m;
  long long sitem;      // bytes between batch items' workspaces
  char* ws;             // workspace base (item 0)
  const double* e;      // off-diagonal (untouched by the tear)
  long long sde;
  const double* lam;    // current eigenvalues (children)
  double* lamNew;
  long long slam;
  const double* Zc;     // current eigenvector blocks
  long long sZ;
};

__device__ __forceinline__ DcWs item_ws(const DcArgs& a, int z) { return dc_ws(a.ws + z * a.sitem, a.m); }

// Merge setup, one CTA per (node, item): z vector, merged poles, deflation.
__global__ void dc_merge_prep_kernel(DcArgs a, const DcNode* nodes) {
  __shared__ double red[32];
  const DcNode nd = nodes[blockIdx.x];
  const int z = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
  DcWs w = item_ws(a, z);
  const int m = a.m, off = nd.off, n1 = nd.n1, n2 = nd.n2, n = n1 + n2, s = off + n1;
  const double* lam = a.lam + z * a.slam;
  const double* Zc = a.Zc + z * a.sZ;
  const double beta = a.e[z * a.sde + s - 1];
  const double rho2 = 2.0 * fabs(beta);
  const double sg = beta < 0.0 ? -1.0 : 1.0;
  const double isq2 = 0.70710678118654752440;
  double dmax = 0.0;
  for (int i = tid; i < n; i += nt) {
    int pos;
    double zv, dv;
    if (i < n1) {
      dv = lam[off + i];
      zv = Zc[(size_t)(s - 1) * m + off + i] * isq2;
      pos = i + lower_bound_d(lam + s, n2, dv);
    } else {
      int k = i - n1;
      dv = lam[s + k];
      zv = sg * Zc[(size_t)s * m + s + k] * isq2;
      pos = k + upper_bound_d(lam + off, n1, dv);
    }
    w.ds[off + pos] = dv;
    w.zs[off + pos] = zv;
    w.src[off + pos] = i;
    dmax = fmax(dmax, fabs(dv));
  }
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((tid & 31) == 0) red[tid >> 5] = dmax;
  __syncthreads();
  if (tid != 0) return;
  for (int k = 1; k < (nt + 31) / 32; k++) dmax = fmax(dmax, red[k]);
  dmax = fmax(dmax, red[0]);
  const double tol = 8.0 * DC_U * fmax(dmax, rho2);
  int K = 0, nD = 0, nrot = 0;
  bool have = false;
  double pd = 0, pz = 0;
  int ps = 0;
  for (int p = 0; p < n; p++) {
    double dp = w.ds[off + p], zp = w.zs[off + p];
    int sp = w.src[off + p];
    if (rho2 * fabs(zp) <= tol) {
      w.dD[off + nD] = dp; w.idxD[off + nD] = sp; nD++;
      continue;
    }
    if (!have) { pd = dp; pz = zp; ps = sp; have = true; continue; }
    double r = hypot(pz, zp);
    double c = zp / r, sn = pz / r;
    if (fabs(c * sn * (dp - pd)) <= tol) {
      w.ra[off + nrot] = ps; w.rb[off + nrot] = sp; w.rc[off + nrot] = c; w.rs[off + nrot] = sn; nrot++;
      w.dD[off + nD] = c * c * pd + sn * sn * dp; w.idxD[off + nD] = ps; nD++;
      pd = sn * sn * pd + c * c * dp; pz = r; ps = sp;
    } else {
      w.dK[off + K] = pd; w.zK[off + K] = pz; w.idxK[off + K] = ps; K++;
      pd = dp; pz = zp; ps = sp;
    }
  }
  if (have) { w.dK[off + K] = pd; w.zK[off + K] = pz; w.idxK[off + K] = ps; K++; }
  // rotations can perturb the order slightly: insertion sorts on nearly sorted data
  for (int i = 1; i < K; i++) {
    double dv = w.dK[off + i], zv = w.zK[off + i];
    int iv = w.idxK[off + i], j = i - 1;
    while (j >= 0 && w.dK[off + j] > dv) {
      w.dK[off + j + 1] = w.dK[off + j]; w.zK[off + j + 1] = w.zK[off + j]; w.idxK[off + j + 1] = w.idxK[off + j]; j--;
    }
    w.dK[off + j + 1] = dv; w.zK[off + j + 1] = zv; w.idxK[off + j + 1] = iv;
  }
  for (int i = 1; i < nD; i++) {
    double dv = w.dD[off + i];
    int iv = w.idxD[off + i], j = i - 1;
    while (j >= 0 && w.dD[off + j] > dv) { w.dD[off + j + 1] = w.dD[off + j]; w.idxD[off + j + 1] = w.idxD[off + j]; j--; }
    w.dD[off + j + 1] = dv; w.idxD[off + j + 1] = iv;
  }
  w.cnt[3 * off + 0] = K;
  w.cnt[3 * off + 1] = nD;
  w.cnt[3 * off + 2] = nrot;
}

// Secular roots, one warp per root.  With origin pole d_o and tau = lam - d_o the function
//   f(tau) = 1 + rho' sum_i z_i^2 / (delta_i - tau),  delta_i = d_i - d_o,
// is increasing between its poles.  Each iteration evaluates psi (poles left of the root),
// phi (poles right of it) and their derivatives (lanes split the K terms), models each
// part by one pole plus a constant matched in value and slope,
//   psi ~ p + q/(delta_j - tau),  phi ~ s + t/(delta_{j+1} - tau),
// and takes the root of the model (a quadratic in u = delta_j - tau) when it falls inside
// the current sign bracket; otherwise it bisects, and it also bisects whenever two steps
// failed to halve the bracket.  Stops when f is below its rounding level or the bracket
// is at the working precision of tau.
__global__ void dc_secular_kernel(DcArgs a, const DcNode* nodes, DevStatus* st) {
  const DcNode nd = nodes[blockIdx.y];
  const int z = blockIdx.z;
  DcWs w = item_ws(a, z);
  const int off = nd.off, s = off + nd.n1;
  const int K = w.cnt[3 * off];
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= K) return;
  const double rho2 = 2.0 * fabs(a.e[z * a.sde + s - 1]);
  const double* dK = w.dK + off;
  const double* zK = w.zK + off;
  int o;
  double lo, hi;
  if (j < K - 1) {
    const double gap = dK[j + 1] - dK[j];
    const double mid = 0.5 * gap;
    double f = 0.0;
    for (int i = lane; i < K; i += 32) f += zK[i] * zK[i] / ((dK[i] - dK[j]) - mid);
    f = 1.0 + rho2 * warp_sum(f);
    if (f >= 0.0) { o = j; lo = 0.0; hi = mid; }
    else { o = j + 1; lo = -mid; hi = 0.0; }
  } else {
    double zz = 0.0;
    for (int i = lane; i < K; i += 32) zz += zK[i] * zK[i];
    zz = warp_sum(zz);
    o = j; lo = 0.0; hi = rho2 * zz * (1.0 + 4.0 * DC_U) + 4.0 * DC_U * fabs(dK[j]);
  }
  const double d0 = dK[o];
  // poles bracketing the root, relative to the origin: left = delta_j, right = delta_{j+1}
  const double dl = dK[j] - d0;
  const bool last = (j == K - 1);
  const double dr = last ? 0.0 : dK[j + 1] - d0;
  double tau = 0.5 * (lo + hi);
  double wref = hi - lo;  // bracket width two iterations ago: a step must halve it
  int it = 0;
  for (; it < 200; it++) {
    double ps = 0.0, psd = 0.0, fs = 0.0, fsd = 0.0, absum = 0.0;
    for (int i = lane; i < K; i += 32) {
      double den = (dK[i] - d0) - tau;
      double t = zK[i] / den;
      double term = zK[i] * t;          // z_i^2 / den
      double dterm = t * t;             // z_i^2 / den^2
      if (i <= j) { ps += term; psd += dterm; }
      else { fs += term; fsd += dterm; }
      absum += fabs(term);
    }
    ps = warp_sum(ps); psd = warp_sum(psd); fs = warp_sum(fs); fsd = warp_sum(fsd); absum = warp_sum(absum);
    const double f = 1.0 + rho2 * (ps + fs);
    if (f < 0.0) lo = tau; else hi = tau;
    if (fabs(f) <= 8.0 * DC_U * (1.0 + rho2 * absum)) break;
    if (!(hi - lo > 2.0 * DC_U * fmax(fabs(lo), fabs(hi)))) break;
    // two-pole model
    const double ul = dl - tau;                        // delta_j - tau
    const double qa = rho2 * psd * ul * ul;            // rho' q
    const double c0 = 1.0 + rho2 * (ps - psd * ul);    // 1 + rho' p
    double cand;
    if (last) {
      double c = c0 + rho2 * fs;                       // no pole on the right
      cand = (c > 0.0) ? dl + qa / c : 0.5 * (lo + hi);   // c + qa/(dl - x) = 0
    } else {
      const double ur = dr - tau;
      const double ta = rho2 * fsd * ur * ur;            // rho' t
      const double c = c0 + rho2 * (fs - fsd * ur);      // 1 + rho'(p + s)
      const double D = dr - dl;
      // c u^2 + (c D + qa + ta) u + qa D = 0, u = dl - x in (-D, 0)
      const double B = c * D + qa + ta, C = qa * D;
      double u;
      if (c == 0.0) {
        u = -C / B;
      } else {
        double disc = B * B - 4.0 * c * C;
        disc = disc > 0.0 ? sqrt(disc) : 0.0;
        // roots: (-B -+ disc)/(2c); stable form picks the root in (-D, 0)
        double r1 = (B > 0.0) ? (-B - disc) / (2.0 * c) : (2.0 * C) / (-B + disc);
        double r2 = (B > 0.0) ? (2.0 * C) / (-B - disc) : (-B + disc) / (2.0 * c);
        u = (r1 < 0.0 && r1 > -D) ? r1 : r2;
      }
      cand = dl - u;
    }
    if ((it & 1) == 1) {
      if (hi - lo > 0.5 * wref) cand = 0.5 * (lo + hi);  // slow one-sided progress: bisect
      wref = hi - lo;
    }
    if (!(cand > lo && cand < hi)) cand = 0.5 * (lo + hi);
    if (cand == tau) break;
    tau = cand;
  }
  if (it >= 200 && lane == 0) set_status(st ? st + z : nullptr, ST_ENOCONV, off + j);
  if (lane == 0) {
    w.orig[off + j] = o;
    w.tauK[off + j] = tau;
    w.lamK[off + j] = d0 + tau;
  }
}

// Gu-Eisenstat: z_hat_i^2 = (lam_i - d_i)/rho' * prod_{j != i} (lam_j - d_i)/(d_j - d_i).
__global__ void dc_zhat_kernel(DcArgs a, const DcNode* nodes) {
  const DcNode nd = nodes[blockIdx.y];
  const int z = blockIdx.z;
  DcWs w = item_ws(a, z);
  const int off = nd.off, s = off + nd.n1;
  const int K = w.cnt[3 * off];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  const double rho2 = 2.0 * fabs(a.e[z * a.sde + s - 1]);
  const double* dK = w.dK + off;
  const double di = dK[i];
  double prod = ((dK[w.orig[off + i]] - di) + w.tauK[off + i]) / rho2;
  for (int j = 0; j < K; j++) {
    if (j == i) continue;
    double lj = (dK[w.orig[off + j]] - di) + w.tauK[off + j];
    prod *= lj / (dK[j] - di);
  }
  double zh = sqrt(fabs(prod));
  w.zhat[off + i] = w.zK[off + i] < 0.0 ? -zh : zh;
}

// Output column positions: roots and deflated values merged in ascending order.
__global__ void dc_colmap_kernel(DcArgs a, const DcNode* nodes) {
  const DcNode nd = nodes[blockIdx.y];
  const int z = blockIdx.z;
  DcWs w = item_ws(a, z);
  const int off = nd.off;
  const int K = w.cnt[3 * off], nD = w.cnt[3 * off + 1];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double* lamNew = a.lamNew + z * a.slam;
  if (t < K) {
    double v = w.lamK[off + t];
    int pos = t + lower_bound_d(w.dD + off, nD, v);
    w.colsrc[off + pos] = t;
    lamNew[off + pos] = v;
  } else if (t < K + nD) {
    int i = t - K;
    double v = w.dD[off + i];
    int pos = i + upper_bound_d(w.lamK + off, K, v);
    w.colsrc[off + pos] = -1 - i;
    lamNew[off + pos] = v;
  }
}

// W^T columns (children-basis vectors), one warp per output column, then the deflation
// rotations G^T applied last-to-first.
__global__ void dc_buildw_kernel(DcArgs a, const DcNode* nodes) {
  const DcNode nd = nodes[blockIdx.y];
  const int z = blockIdx.z;
  DcWs w = item_ws(a, z);
  const int m = a.m, off = nd.off, n = nd.n1 + nd.n2;
  const int K = w.cnt[3 * off], nrot = w.cnt[3 * off + 2];
  const int lane = threadIdx.x & 31;
  const int pos = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (pos >= n) return;
  double* col = w.W + (size_t)(off + pos) * m + off;
  for (int r = lane; r < n; r += 32) col[r] = 0.0;
  __syncwarp();
  const int nD = w.cnt[3 * off + 1];
  const int src = w.colsrc[off + pos];
  if (src >= K || src < -nD) return;  // only reachable on non-finite input: leave the column zero
  if (src >= 0) {
    const int j = src;
    const double* dK = w.dK + off;
    const double dj = dK[w.orig[off + j]], tj = w.tauK[off + j];
    double s2 = 0.0;
    for (int i = lane; i < K; i += 32) {
      double v = w.zhat[off + i] / ((dK[i] - dj) - tj);
      s2 += v * v;
    }
    s2 = warp_sum(s2);
    const double inv = 1.0 / sqrt(s2);
    for (int i = lane; i < K; i += 32) col[w.idxK[off + i]] = w.zhat[off + i] / ((dK[i] - dj) - tj) * inv;
  } else {
    if (lane == 0) col[w.idxD[off + (-1 - src)]] = 1.0;
  }
  __syncwarp();
  if (lane == 0) {
    for (int r = nrot - 1; r >= 0; r--) {
      const int ia = w.ra[off + r], ib = w.rb[off + r];
      const double c = w.rc[off + r], sn = w.rs[off + r];
      const double xa = col[ia], xb = col[ib];
      col[ia] = c * xa + sn * xb;
      col[ib] = -sn * xa + c * xb;
    }
  }
}

// ------------------------------------------------------------------ host side

static void build_tree(DcPlan* p) {
  int m = p->m, depth = 0;
  while (((m + (1 << depth) - 1) >> depth) > DC_LEAF) depth++;
  p->depth = depth;
  // nodes per depth from the root down
  std::vector<std::vector<std::pair<int, int>>> seg(depth + 1);
  seg[0].push_back({0, m});
  for (int l = 0; l < depth; l++)
    for (auto& sg : seg[l]) {
      int n1 = sg.second / 2;
      seg[l + 1].push_back({sg.first, n1});
      seg[l + 1].push_back({sg.first + n1, sg.second - n1});
      p->splits.push_back(sg.first + n1);
    }
  for (auto& sg : seg[depth]) { p->leaves.push_back(sg.first); p->leaves.push_back(sg.second); }
  p->levels.resize(depth);
  for (int t = 0; t < depth; t++) {
    int l = depth - 1 - t;  // depth of the parents merged at step t
    DcLevel& L = p->levels[t];
    for (auto& sg : seg[l]) {
      int n1 = sg.second / 2;
      L.nodes.push_back({sg.first, n1, sg.second - n1});
      L.maxn = std::max(L.maxn, sg.second);
      L.maxhalf = std::max(L.maxhalf, sg.second - n1);
    }
  }
  std::sort(p->splits.begin(), p->splits.end());
}

DcPlan* dc_plan_create(int m, int count) {
  DcPlan* p = new DcPlan();
  p->m = m;
  p->count = count;
  build_tree(p);
  cudaMalloc(&p->d_leaves, sizeof(int) * std::max<size_t>(1, p->leaves.size()));
  cudaMemcpy(p->d_leaves, p->leaves.data(), sizeof(int) * p->leaves.size(), cudaMemcpyHostToDevice);
  cudaMalloc(&p->d_splits, sizeof(int) * std::max<size_t>(1, p->splits.size()));
  if (!p->splits.empty())
    cudaMemcpy(p->d_splits, p->splits.data(), sizeof(int) * p->splits.size(), cudaMemcpyHostToDevice);
  for (auto& L : p->levels) {
    cudaMalloc(&L.d_nodes, sizeof(DcNode) * L.nodes.size());
    cudaMemcpy(L.d_nodes, L.nodes.data(), sizeof(DcNode) * L.nodes.size(), cudaMemcpyHostToDevice);
    cudaMalloc(&L.d_gemm, sizeof(GemmDesc) * 2 * L.nodes.size() * count);
  }
  return p;
}

void dc_plan_destroy(DcPlan* p) {
  if (!p) return;
  cudaFree(p->d_leaves);
  cudaFree(p->d_splits);
  for (auto& L : p->levels) { cudaFree(L.d_nodes); cudaFree(L.d_gemm); }
  delete p;
}

size_t dc_workspace_bytes(const DcPlan* p) { return dc_item_bytes(p->m) * p->count; }

// Z buffer used at merge step t (input) is buf[t % 2]; leaves write buf[0]; the root
// writes buf[depth % 2], chosen to be the caller's Z.
static void build_gemm_lists(DcPlan* p, double* Z, long long sZ, void* work) {
  const int m = p->m;
  const size_t item = dc_item_bytes(m);
  for (int t = 0; t < p->depth; t++) {
    DcLevel& L = p->levels[t];
    std::vector<GemmDesc> h;
    for (int z = 0; z < p->count; z++) {
      DcWs w = dc_ws(static_cast<char*>(work) + z * item, m);
      double* buf[2];
      buf[p->depth % 2] = Z + z * sZ;
      buf[(p->depth + 1) % 2] = w.Zb;
      const double* in = buf[t % 2];
      double* out = buf[(t + 1) % 2];
      for (auto& nd : L.nodes) {
        const int off = nd.off, n = nd.n1 + nd.n2, s = off + nd.n1;
        GemmDesc g1{in + (size_t)off * m + off, w.W + (size_t)off * m + off, out + (size_t)off * m + off, nullptr,
                    nd.n1, n, nd.n1, m, m, m};
        GemmDesc g2{in + (size_t)s * m + s, w.W + (size_t)off * m + s, out + (size_t)s * m + off, nullptr, nd.n2, n,
                    nd.n2, m, m, m};
        h.push_back(g1);
        h.push_back(g2);
      }
    }
    cudaMemcpy(L.d_gemm, h.data(), sizeof(GemmDesc) * h.size(), cudaMemcpyHostToDevice);
  }
  p->zbound = Z;
  p->wbound = work;
  p->sZbound = sZ;
}

size_t dc_split_item_bytes(const DcPlan* p, int min_half, int S) {
  size_t b = 0;
  for (auto& L : p->levels)
    if (L.maxhalf >= min_half)
      for (auto& nd : L.nodes) {
        const int n = nd.n1 + nd.n2;
        b = std::max(b, ozaki_workspace_bytes(nd.n1, n, nd.n1, false, S));
        b = std::max(b, ozaki_workspace_bytes(nd.n2, n, nd.n2, false, S));
      }
  return b;
}

void dc_solve(DcPlan* p, double* d, double* e, long long sde, double* lam, double* Z, long long sZ, void* work,
              DevStatus* st, cudaStream_t s, Prof* prof, const DcSplit* sp) {
  const int m = p->m, cnt = p->count;
  if (p->zbound != Z || p->wbound != work || p->sZbound != sZ) build_gemm_lists(p, Z, sZ, work);
  const size_t item = dc_item_bytes(m);
  DcWs w0 = dc_ws(work, m);
  // lam ping-pong: leaves write lamA (item stride = item bytes / 8 doubles)
  const long long slam = (long long)(item / sizeof(double));
  double* lamBuf[2] = {w0.lamA, w0.lamB};
  double* zbuf0 = (p->depth % 2 == 0) ? Z : w0.Zb;
  const long long sZ0 = (p->depth % 2 == 0) ? sZ : slam;
  int tok = prof->begin();
  count_launch();
  dc_tear_kernel<<<cnt, 32, 0, s>>>(d, e, sde, p->d_splits, (int)p->splits.size());
  const int nleaves = (int)p->leaves.size() / 2;
  count_launch();
  dc_leaf_kernel<<<dim3((nleaves + 3) / 4, cnt), 128, 0, s>>>(d, e, sde, lamBuf[0], slam, zbuf0, sZ0, m,
                                                              p->d_leaves, nleaves, st);
  prof->end(tok, PC_DC_LEAF, 0.0, 0.0);
  for (int t = 0; t < p->depth; t++) {
    DcLevel& L = p->levels[t];
    const int nn = (int)L.nodes.size();
    DcArgs a;
    a.m = m;
    a.sitem = (long long)item;
    a.ws = static_cast<char*>(work);
    a.e = e;
    a.sde = sde;
    a.lam = lamBuf[t % 2];
    a.lamNew = lamBuf[(t + 1) % 2];
    a.slam = slam;
    const bool in_is_Z = ((t % 2) == (p->depth % 2));
    a.Zc = in_is_Z ? Z : w0.Zb;
    a.sZ = in_is_Z ? sZ : slam;
    tok = prof->begin();
    count_launch();
    dc_merge_prep_kernel<<<dim3(nn, cnt), 256, 0, s>>>(a, L.d_nodes);
    dim3 g1((L.maxn + 127) / 128, nn, cnt);
    count_launch();
    dc_secular_kernel<<<dim3((L.maxn + 7) / 8, nn, cnt), 256, 0, s>>>(a, L.d_nodes, st);
    count_launch();
    dc_zhat_kernel<<<g1, 128, 0, s>>>(a, L.d_nodes);
    count_launch();
    dc_colmap_kernel<<<g1, 128, 0, s>>>(a, L.d_nodes);
    count_launch();
    dc_buildw_kernel<<<dim3((L.maxn + 7) / 8, nn, cnt), 256, 0, s>>>(a, L.d_nodes);
    prof->end(tok, PC_DC_SECULAR, 0.0, 0.0);
    double gfl = 0.0, gby = 0.0;
    for (auto& nd : L.nodes) {
      const double nn1 = nd.n1, nn2 = nd.n2, n = nn1 + nn2;
      gfl += 2.0 * (nn1 * nn1 + nn2 * nn2) * n;
      gby += 8.0 * (nn1 * nn1 + nn2 * nn2 + 2.0 * n * n);
    }
    if (sp && sp->per > 0 && L.maxhalf >= sp->min_half) {
      // large merges: per node, exact split-bf16 products batched over the items
      tok = prof->begin();
      const long long sin = in_is_Z ? sZ : slam, sout = in_is_Z ? slam : sZ;
      double* in0 = in_is_Z ? Z : w0.Zb;
      double* out0 = in_is_Z ? w0.Zb : Z;
      bool ok = true;
      for (auto& nd : L.nodes) {
        const int off = nd.off, n = nd.n1 + nd.n2, sft = off + nd.n1;
        for (int z0 = 0; z0 < cnt && ok; z0 += sp->per) {
          const int c = std::min(sp->per, cnt - z0);
          const DcWs wz = dc_ws(static_cast<char*>(work) + (size_t)z0 * item, m);
          const long long iz = (long long)z0 * sin, oz = (long long)z0 * sout;
          ok = ozaki_gemm<double>(OP_N, OP_T, nd.n1, n, nd.n1, 1.0, in0 + iz + (size_t)off * m + off, m, sin,
                                  wz.W + (size_t)off * m + off, m, slam, 0.0, out0 + oz + (size_t)off * m + off, m,
                                  sout, c, 0, sp->S, sp->work, st, s, nullptr, 0, nullptr, sp->wait) &&
               ozaki_gemm<double>(OP_N, OP_T, nd.n2, n, nd.n2, 1.0, in0 + iz + (size_t)sft * m + sft, m, sin,
                                  wz.W + (size_t)off * m + sft, m, slam, 0.0, out0 + oz + (size_t)sft * m + off, m,
                                  sout, c, 0, sp->S, sp->work, st, s, nullptr, 0, nullptr, sp->wait);
        }
      }
      prof->end(tok, PC_OZAKI, gfl * cnt, gby * cnt);
      if (ok) continue;
    }
    tok = prof->begin();
    GemmBatch gb{};
    gb.list = L.d_gemm;
    gb.count = 2 * nn * cnt;
    gb.opA = OP_N;
    gb.opB = OP_T;
    gb.alpha = 1.0;
    gb.beta = 0.0;
    gemm<double>(gb, L.maxhalf, L.maxn, s);
    prof->end(tok, PC_DC_GEMM, gfl * cnt, gby * cnt);
  }
  // final eigenvalues
  double* lamFinal = lamBuf[p->depth % 2];
  copy2d<double>(lam, m, sde, lamFinal, m, slam, 1, m, cnt, s);
}

}  // namespace gks
