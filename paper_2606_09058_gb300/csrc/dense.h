// Launchers for the small dense kernels (dense.cu), the Householder reduction
// (hetrd.cu), the divide-and-conquer tridiagonal solver (stedc.cu) and occupations
// (occ.cu).
#pragma once
#include "launch.h"

namespace gks {

enum { TRSM_RIGHT_CONJ = 0, TRSM_LEFT = 1, TRSM_LEFT_CONJ = 2 };
template <typename T>
void potf2(T* A, int lda, long long sA, int k0, int nb, DevStatus* st, int count, cudaStream_t s);
template <typename T>
void trsm_block(int mode, const T* L, int ldl, long long sL, T* B, int ldb, long long sB, int nb, int nrhs,
                int count, cudaStream_t s);
template <typename T>
void hegst_diag(T* A, int lda, long long sA, const T* L, int ldl, long long sL, int k0, int nb, T* F, int ldF,
                long long sF, int count, cudaStream_t s);
template <typename T>
void larft(const T* G, int ldG, long long sG, const double* tau, long long stau, int k, T* Tm, int ldT,
           long long sT, int count, cudaStream_t s);
template <typename T>
void apply_phase(T* X, int ldx, long long sX, const double* Z, int ldz, long long sZ, const T* ph, long long sph,
                 int n, int cols, int count, cudaStream_t s);
template <typename T>
void mirror_lower(T* A, int lda, long long sA, int n, int count, cudaStream_t s);
// V = U diag(s)^-1/2 (Loewdin factor); non-positive s_j: GKS_ENOTSPD with index j.
template <typename T>
void lowdin_factor(const T* U, int ldu, long long sU, const double* sv, long long ss, T* V, int ldv, long long sV,
                   int n, DevStatus* st, int count, cudaStream_t s);
template <typename T>
void column_phase(T* C, int ldc, long long sC, int rows, int cols, int count, cudaStream_t s);
template <typename T>
void spinor_overlap(T* dst, long long sd, const T* S, int lds, long long ss, int n, int count, cudaStream_t s);
// Seeded lower-triangle test pencils for the width tuner (hermitian 1: H, 0: SPD S).
template <typename T>
void tune_pencil(T* A, int m, int count, int hermitian, cudaStream_t s);

// ---- Householder tridiagonalization (hetrd.cu) ----
// Workspace per batch item: u (m), p (m) vectors, tau (m), two zeroed tickets, and for the
// panel form U, Q (m x ldu), per-CTA shares (ceil(m/16) x (2 ldu + 2)) and y (2 ldu + 2).
// hetrd_reflector starts a panel at step j; step j is hetrd_phemv then hetrd_pupdate (which
// with rowupd also forms the reflector of step j-1).
// Digit form of the panel matrix-vector step.  The stale block A = [0:n, 0:n] is
// equilibrated symmetrically by powers of two, A = D Ã D with D = diag(2^{d_i}),
// d_i = ceil(g_i / 2) for row maxima below 2^{g_i} (largest |Re|, |Im| over the full
// row), so every |Re ã|, |Im ã| < 1; the full Hermitian Ã (upper triangle mirrored,
// conjugated) is stored as 7 balanced base-256 digits (signed 8-bit) of round(2^54 Re ã)
// (planes 0..6, most significant first) and of Im ã (planes 7..13, complex only):
// ã = sum_s d_s 2^{-6 - 8s} up to 2^{-55}.  ũ = D u gets the same digits below its own
// scale 2^{fu}.  Then (A u)_i = 2^{d_i} sum over digit pairs s + t <= 7 of exact integer
// dot products (dp4a, int32 sums) weighted by 2^{fu - 12 - 8(s + t)}.
// Layout: tiles of 32 rows x 16 columns, row-tile-major, each tile contiguous (3584 or
// 7168 bytes: the 32 rows one after the other, a row's 16 columns as the planes' 16 bytes
// one after the other); ũ per 16 columns the same way.  Rows are padded to a multiple of 32.
struct HemvDigits {
  signed char* D;            // [item][ldd32 / 32][ldd / 16][32][planes][16], ldd32 = ldd rounded up to 32
  long long sD;              // item stride (bytes)
  int ldd;                   // columns per row, multiple of 16
  signed char* ud;           // [item][ldd / 16][planes][16] digits of ũ (zero beyond the step's length)
  long long sud;             // item stride (bytes)
  int* fu;                   // [item] scale exponent of ũ
  unsigned long long* rmax;  // [item][ldd] row maxima of the stale block (bits of doubles)
};
template <typename T>
void hetrd_reflector(T* A, int lda, long long sA, int j, T* u, long long sv, double* tau, long long stau, int count,
                     cudaStream_t s, double* uw = nullptr, const HemvDigits* hd = nullptr);
// Digits of the stale block [0:n, 0:n] (FP64 forms only).
template <typename T>
void hetrd_digits(const T* A, int lda, long long sA, int n, const HemvDigits& hd, int count, cudaStream_t s);
// Complex panel form only: Sg = Re + Im of the stale block (lower, leading n x n, stride sA
// per item, same indexing as A) and uw = (Re u, Im u - Re u, Re u + Im u) per element (3 sv
// doubles per item); with both, the matrix-vector step uses three real products per
// complex product.
void hetrd_sums(const zc* A, int lda, long long sA, int n, double* Sg, int count, cudaStream_t s);
template <typename T>
void hetrd_phemv(const T* A, int lda, long long sA, int j, const T* u, T* p, long long sv, const double* tau,
                 long long stau, const T* U, const T* Q, int ldu, long long sU, int k, T* part, long long spart,
                 T* y, long long sy, int* ticket, int count, cudaStream_t s, const double* Sg = nullptr,
                 const double* uw = nullptr, const HemvDigits* hd = nullptr);
template <typename T>
void hetrd_pupdate(T* A, int lda, long long sA, int j, T* u, const T* p, long long sv, double* tau, long long stau,
                   T* U, T* Q, int ldu, long long sU, int k, const T* y, long long sy, int rowupd, int* ticket,
                   int count, cudaStream_t s, double* uw = nullptr, const HemvDigits* hd = nullptr);
template <typename T>
void hetrd_finish(const T* A, int lda, long long sA, int m, double* d, double* e, long long sde, T* ph,
                  long long sph, int count, cudaStream_t s);
// Gather reflectors j0..j1 (descending) into Vblk (rows x (j1-j0+1)) and their taus; TV may
// be the FP64 partner of a single-precision T.
template <typename T, typename TV>
void gather_reflectors(const T* A, int lda, long long sA, const double* tau, long long stau, int j0, int j1,
                       TV* V, int ldv, long long sV, double* tb, long long stb, int count, cudaStream_t s);
// dst[t] = src[t] widened to FP64 (single-precision phases of the mixed-precision path).
template <typename T, typename TV>
void widen_copy(const T* src, TV* dst, long long n, cudaStream_t s);
// Lower triangle of the order-n FP64 A rounded to single precision in B.
template <typename T, typename TL>
void narrow_lower(const T* A, int lda, long long sA, TL* B, int ldb, long long sB, int n, int count, cudaStream_t s);

// ---- divide and conquer (stedc.cu) ----
struct DcPlan;
DcPlan* dc_plan_create(int m, int count);
void dc_plan_destroy(DcPlan* p);
size_t dc_workspace_bytes(const DcPlan* p);
// Merges whose halves reach min_half rows run as split products on `work` (per items per
// launch, S digits); the rest use the grouped FP64 kernel.
struct DcSplit {
  void* work;
  int per, S, min_half;
  long long wait;  // bound of the product kernels' device-side waits (SM cycles, 0 = default)
};
size_t dc_split_item_bytes(const DcPlan* p, int min_half, int S);
// d (m), e (m-1) per item (stride sde); Z out (m x m, ld m, stride sZ); lam out (stride sde).
void dc_solve(DcPlan* p, double* d, double* e, long long sde, double* lam, double* Z, long long sZ, void* work,
              DevStatus* st, cudaStream_t s, Prof* prof, const DcSplit* sp = nullptr);

// ---- adjoint (adjoint.cu) ----
void adj_occ(const double* eps, const double* mu, double kT, long long tot, double* f, double* fp, cudaStream_t s);
template <typename T>
void adj_weights(const double* eps, const double* f, const double* fp, const double* w, const T* W, long long sW,
                 int M, int nk, double gs, const double* eps_bar, double e_band_bar, int have_w, double* e,
                 cudaStream_t s);
template <typename T>
void adj_build(T* W, T* BH, long long sW, int M, const double* eps, const double* f, const double* e,
               const double* mu, double kT, double gs, int have_w, int nk, cudaStream_t s);
template <typename T>
void herm_part(T* dst, const T* src, long long sd, long long ss, int M, int nk, cudaStream_t s);
template <typename T>
void spin_block_sum(T* dst, long long sd, const T* src, long long ss, int n, int nk, cudaStream_t s);
template <typename T>
void spin_pair_sum(T* dst, long long sd, const T* src, long long ss, int n, int nk, cudaStream_t s);

// ---- FP64-accurate GEMM from exact bf16 digit products (ozaki.cu) ----
// Workspace bytes per batch item (a multiple of 256), and output tiles per item.
size_t ozaki_workspace_bytes(int M, int N, int K, bool cplx, int S);
int ozaki_tiles(int M, int N, bool cplx);
// Returns false (nothing enqueued) when the TMA tensor maps cannot be encoded.  Optional:
// kscale (per item, stride sks) scales column k of op(A) before the product; kdev (per
// item, device) cuts K to its value; wait_cycles bounds every device-side wait (0 = 2^32
// SM cycles); skip_copy >= 0 makes every CTA leave out that operand copy (a test hook
// that lets the bounded waits expire).
template <typename T>
bool ozaki_gemm(int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda, long long sA, const T* B,
                int ldb, long long sB, double beta, T* C, int ldc, long long sC, int count, int lower, int S,
                void* work, DevStatus* status, cudaStream_t s, const double* kscale = nullptr, long long sks = 0,
                const int* kdev = nullptr, long long wait_cycles = 0, long long skip_copy = -1, long long sA2 = 0,
                long long sB2 = 0, long long sC2 = 0, int nb2 = 0);

// ---- FP64 unit throughput probes (peaks.cu) ----
// which 0: DFMA, 1: DMMA (mma.sync f64).  Enqueues one probe on sms x 4 CTAs and returns
// the flops it executes; `out` needs sms * 1024 doubles.
double peak_probe(int which, int sms, long long iters, double* out, cudaStream_t s);

// ---- two-stage tridiagonalization (sbr.cu) ----
// Stage 1: in-place QR of the panel A[r0:r0+m, k:k+b] (kb reflectors, complex tau, real
// beta; v below the diagonal), its unit lower trapezoidal V (m x kb), and the T factor of
// H_0 .. H_{k-1} = I - V T V^H from G = V^H V.
// The multi-CTA panel QR splits the rows over up to kQrMaxG CTAs per item (all resident,
// bounded grid barriers: a wait past wait_limit cycles sets GKS_ETIMEOUT in st[item]);
// scratch holds qr_scratch_bytes(count, sizeof(T)) bytes.
constexpr int kQrMaxG = 64;
size_t qr_scratch_bytes(int count, int es);
template <typename T>
void panel_qr(T* A, int lda, long long sA, int r0, int k, int m, int b, int kb, T* taus, long long stau, int count,
              void* scratch, DevStatus* st, long long wait_limit, cudaStream_t s);
template <typename T>
void panel_v(const T* A, int lda, long long sA, int r0, int k, int m, int kb, T* V, int ldv, long long sV, int count,
             cudaStream_t s);
template <typename T>
void panel_clear(T* A, int lda, long long sA, int r0, int k, int m, int kb, int count, cudaStream_t s);
template <typename T>
void larft_tau(const T* G, int ldG, long long sG, const T* tau, long long stau, int k, T* Tm, int ldT, long long sT,
               int count, cudaStream_t s);
// Band storage Bd[j W + d] = T[j+d][j] (W = 2b + 1, room for the bulges of stage 2).
template <typename T>
void band_pack(const T* A, int lda, long long sA, T* Bd, int W, long long sB, int m, int b, int count, cudaStream_t s);
template <typename T>
void band_unpack(const T* Bd, int W, long long sB, T* A, int lda, long long sA, int m, int count, cudaStream_t s);
// Stage 2: persistent bulge chasing (cooperative launch of `workers` CTAs per item, see
// chase_workers); reflector (sweep i, window j) in V2[i m + j b ..], tau2[i ldt + j].
// Returns false if the launch was refused (then nothing ran).
template <typename T>
int chase_workers(int b, int items, int cap);
template <typename T>
bool chase(T* Bd, int W, long long sB, int m, int b, T* V2, long long sV2, T* tau2, int ldt, long long sT2, int* prog,
           long long sprog, int* err, DevStatus* st, long long wait_limit, int items, int workers, cudaStream_t s);
template <typename T>
void band_tridiag(const T* Bd, int W, long long sB, int m, double* d, double* e, long long sde, int count,
                  cudaStream_t s);
// Q2 compact-WY blocks of one wavefront (see sbr.cu) into Vw (items x nblk x hp x nbs), tw.
template <typename T>
void q2_gather(const T* V2, long long sV2, const T* tau2, int ldt, long long sT2, int m, int b, int nbs, int hp, int g0,
               int j0, int nblk, T* Vw, T* tw, int items, cudaStream_t s);
template <typename T>
void widen_pad(const double* Z, int ldz, long long sZ, T* X, int ldx, long long sX, int m, int rows, int cols,
               int count, cudaStream_t s);

// ---- Ogita-Aishima refinement (refine.cu) ----
// Per item (stride sMM, order M, full storage): G = X^H X becomes R = I - X^H X, lam = the
// refined Rayleigh quotients t_ii/(1 - r_ii) of T = X^H H' X, nrm[3 z + 0..2] = row-sum bounds
// of ||T - diag(lam)||_2 and ||R||_2 and max |lam|.
template <typename T>
void oa_prepare(const T* Tm, T* G, long long sMM, int M, double* lam, double* nrm, int count, cudaStream_t s);
// T <- E, the sweep's correction (cluster threshold from nrm).
template <typename T>
void oa_correction(T* Tm, const T* R, long long sMM, int M, const double* lam, const double* nrm, int count,
                   cudaStream_t s);
// Restore ascending lam (and the columns of X with it, through Y) where refinement swapped
// near-degenerate eigenvalues; M * 12 bytes of shared memory per item.
template <typename T>
void oa_order(double* lam, T* X, T* Y, long long sMM, int M, int* perm, int* flag, int count, cudaStream_t s);

// ---- occupations (occ.cu) ----
void fermi_mu(const double* eps, int m, int nk, const double* w, double gs, double kT, double n_elec,
              double f_cut, double* occ, double* kscale, double* mu, double* e_band, int* nrho, DevStatus* st,
              int nsys, cudaStream_t s);
// out[k * rep + r] = w[k] (w == nullptr: 1/nk) for r < rep: per-item k weights when rep
// items (spin channels) share one k-point.
void expand_weights(const double* w, int nk, int rep, double* out, cudaStream_t s);
// n_rho(k) = min(n_rho(k), cols); a count above `cols` (the eigenvectors computed) sets the
// status word st[k * st_stride] to GKS_EINVAL with the count.
void clamp_nrho(int* nrho, int nk, int cols, DevStatus* st, int st_stride, cudaStream_t s);
// out[t] = a[t] * b[t] for t < n.
void mul_elem(const double* a, const double* b, double* out, long long n, cudaStream_t s);

}  // namespace gks
