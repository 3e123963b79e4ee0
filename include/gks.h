/* gks.h -- C ABI of the GB300 generalized Kohn-Sham eigensolver and density matrix.
 *
 * Problem (arXiv 2606.09058, Sec. 2, generalized eigenvalue problem H C = S C eps; its
 * Bloch form per k-point, Eq. eigenval_problem; the noncollinear spinor form of Sec. 2
 * and Sec. 3.2 with S_NC = diag(S, S)); occupations and chemical potential (Sec. 3.1
 * Part 3, Sec. 3.2 Part 4); density matrix (Sec. 2 n_lm, Sec. 3.1 Part 4).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers allocated and owned by the caller, contiguous
 *    and row-major.  Complex data is interleaved (re, im) double pairs.
 *  - Hermitian inputs are read from their LOWER triangle only (row >= column).
 *  - M is the matrix order: M = n (collinear, spin-polarized) or 2n (noncollinear).
 *  - All work is enqueued on the stream given at context creation.  gks_solve returns
 *    host-side validation status; device-side failures (S not positive definite, no
 *    convergence, invalid occupation parameters) are returned by gks_sync.
 *  - Errors never cross the ABI as exceptions and never trap on the device.  The text
 *    of the last error (with the failing column / batch item) is in gks_last_error.
 *  - One context per host thread.  A context owns its workspace (device memory sized
 *    for the last problem shape) until gks_destroy.
 */
#ifndef GKS_H
#define GKS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gks_ctx gks_ctx;

typedef enum {
  GKS_OK = 0,
  GKS_EINVAL = 1,    /* bad argument (shape, pointer, kT <= 0, n_elec out of range, NaN) */
  GKS_ENOTSPD = 2,   /* S is not positive definite (column in gks_last_error) */
  GKS_ENOCONV = 3,   /* an iteration did not converge */
  GKS_ENOMEM = 4,    /* device allocation failed */
  GKS_ECUDA = 5,     /* CUDA runtime error */
  GKS_ETIMEOUT = 6,  /* a bounded device-side wait expired */
  GKS_ENOTIMPL = 7   /* option not implemented */
} gks_status;

typedef enum { GKS_R64 = 0, GKS_C128 = 1 } gks_dtype;        /* real symmetric / complex Hermitian */

/* Spin treatment (paper Sec. 2): collinear spin-degenerate runs carry g_s = 2 electrons per
 * state; noncollinear runs solve the 2n x 2n spinor problem with g_s = 1; spin-polarized
 * collinear runs (paper Sec. 1/2: the extension to spin-polarized cases) solve one n x n
 * pencil per spin channel, both channels sharing S_k and one chemical potential, g_s = 1.
 * Spin-polarized arrays carry the channel right after the k index: H, C, rho (nk, 2, n, n),
 * eps (nk, 2, n); S stays (nk, n, n). */
typedef enum { GKS_COLLINEAR = 0, GKS_NONCOLLINEAR = 1, GKS_SPIN_POLARIZED = 2 } gks_spin;

/* Arithmetic of the eigensolve.  GKS_FP64: every stage FP64-accurate (products as exact
 * split-bf16 tensor-core products with FP64 accumulation).  GKS_MIXED_SPLITBF16: H' is
 * rounded to single precision and tridiagonalized on the FP32 pipe, the divide and
 * conquer stays FP64, the back-transform products take 5 digits (about FP32 accuracy),
 * then opts.refine_sweeps Ogita-Aishima sweeps refine every eigenpair of H' with
 * FP64-accurate products (Ogita & Aishima 2018); the Cholesky of S, the reduction to H',
 * the secular roots, the refinement residuals and C = L^-H X stay FP64.  Mixed precision
 * needs opts.n_ev = 0 and M <= 18000.  GKS_MIXED_TF32 is not implemented (gks_create
 * returns GKS_ENOTIMPL). */
typedef enum { GKS_FP64 = 0, GKS_MIXED_TF32 = 1, GKS_MIXED_SPLITBF16 = 2 } gks_prec;

/* Reduction to the standard problem.  GKS_REDUCE_CHOLESKY: S = L L^H, H' = L^-1 H L^-H,
 * C = L^-H X.  GKS_REDUCE_LOWDIN (the paper's own route, Sec. 3.1 Parts 2-1 .. 2-5):
 * S = U diag(s) U^H by this library's standard eigensolve, V = U diag(s)^-1/2,
 * H' = V^H H V, C = V X; V is what GKS_REUSE_S_FACTOR keeps.  On an ill-conditioned S the
 * Loewdin factor carries s_min^-1/2 into every product, so its results are less accurate
 * than Cholesky's (compare them with the tests); collinear and spin-polarized runs with
 * n_ev = 0 only (noncollinear: GKS_ENOTIMPL). */
typedef enum { GKS_REDUCE_CHOLESKY = 0, GKS_REDUCE_LOWDIN = 1 } gks_reduction;

/* Reduction of H' to real tridiagonal form.  GKS_TRIDIAG_ONE_STAGE: Householder steps whose
 * rank-2 updates are deferred over panels and applied as tensor-core products (the
 * matrix-vector half runs on the FP64 pipe).  GKS_TRIDIAG_TWO_STAGE (paper Sec. 6: the
 * one-stage reduction is matrix-vector bound): dense -> band of width opts.band by panel QR
 * with two-sided updates as tensor-core products, band -> tridiagonal by a persistent
 * bulge-chasing kernel (bounded waits), and the back-transform applies the chase's
 * reflectors (Q2, compact-WY blocks in wavefronts) and the panels' (Q1) as products.  Its
 * back-transforms cost more than the one-stage one, so it pays when only the lowest n_ev
 * eigenvectors are needed.  Not combined with GKS_MIXED_SPLITBF16 (which keeps the
 * one-stage single-precision reduction). */
typedef enum { GKS_TRIDIAG_ONE_STAGE = 0, GKS_TRIDIAG_TWO_STAGE = 1 } gks_tridiag;

/* Form of the FP64-accurate tensor-core products (opts.split).  Both scale each row of the
 * left operand and each column of the right one by a power of two and multiply exact bf16
 * integers with FP32 accumulation (the error-free splittings of Ozaki, Ogita, Oishi and
 * Rump, and of Ozaki, Uchino and Imamura).  GKS_SPLIT_RESIDUES: operands truncated to
 * integers of p >= 6 * opts.slices bits, the integer product recovered from its residues
 * modulo n pairwise coprime moduli <= 256 by the Chinese remainder theorem (one product per
 * modulus; 16 moduli give p = 55 for inner dimensions up to 16384).  GKS_SPLIT_DIGITS:
 * opts.slices digits of 6 bits per operand, products of digit pairs up to slices + 1 levels
 * (45 products for 9 digits). */
typedef enum { GKS_SPLIT_RESIDUES = 0, GKS_SPLIT_DIGITS = 1 } gks_split;

/* The Hermitian matrix-vector step of the one-stage reduction (opts.hemv), about half of
 * the reduction's work and bound by the arithmetic unit that runs it (paper Sec. 6).
 * GKS_HEMV_DIGITS: the stale block of each panel as 8 signed 7-bit digits of Re and Im of
 * every entry (scaled by a power of two of the block's largest entry, 56 bits below it),
 * the vector the same, products of digit pairs up to the 56-bit level as exact 8-bit
 * integer dot products with 32-bit sums, weighted and summed in FP64: the error is that of
 * the 56-bit truncation, relative to the largest entries (normwise).  GKS_HEMV_FP64: FP64
 * multiply-adds (three real products per complex product).  Mixed precision keeps its
 * single-precision step. */
typedef enum { GKS_HEMV_DIGITS = 0, GKS_HEMV_FP64 = 1 } gks_hemv;

/* gks_solve flags. */
enum {
  /* Skip the copy and Cholesky of S: reuse the factor kept from the last solve on this
   * context with the same S array, n, nk, dtype and spin mode (the analogue of the paper's
   * reuse of its S factorization across SCF cycles, Sec. 5.1).  The caller guarantees that
   * S has not changed.  Without a matching kept factor the flag has no effect. */
  GKS_REUSE_S_FACTOR = 1u,
  /* Keep device copies of C, eps and mu of this solve in the context, so that a later
   * gks_adjoint may pass NULL for C, eps and mu (the caller may overwrite its outputs). */
  GKS_SAVE_FOR_BACKWARD = 2u,
  /* Eigenpairs only: eps and C are written; occupations, mu, rho and e_band are not (mu,
   * rho and e_band may be NULL; kT and n_elec are not checked).  For runs whose k-points
   * are spread over several solves or processes: gks_occupy then finds the shared mu. */
  GKS_EIGEN_ONLY = 4u
};

/* Test hooks (opts.debug). */
enum {
  /* The next split product on this context leaves out one operand copy in every CTA, so
   * that its bounded waits expire and gks_sync reports GKS_ETIMEOUT; no fault, no trap. */
  GKS_DEBUG_SKIP_COPY = 1
};

typedef struct {
  int device;          /* CUDA device ordinal */
  void* cuda_stream;   /* cudaStream_t to enqueue on (NULL = legacy default stream) */
  int precision;       /* gks_prec */
  double f_cut;        /* occupations below f_cut are left out of rho (default 1e-16) */
  int profile;         /* 1: record CUDA events around every launch group (see gks_profile) */
  int graph;           /* 1: capture each solve (and each batch) into a CUDA graph and replay it
                          while the arguments are unchanged; needs a non-default stream */
  int gemm;            /* FP64 products: 0 = large ones as exact split-bf16 tensor-core products
                          with FP64 accumulation, small ones on the FP64 pipe (default);
                          1 = FP64 pipe only; 2 = split products for every product */
  int slices;          /* precision of split products in 6-bit units (4..10, 0 = 9): digits per
                          operand (GKS_SPLIT_DIGITS) or at least 6 slices bits (residues) */
  int block;           /* outer block width of the two-level blocked Cholesky, reduction and
                          back-transforms: a multiple of 64 in 64..1024; 0 = 512 for orders
                          from 4096 up and 256 below (gks_tune overrides per shape class) */
  int refine_sweeps;   /* GKS_MIXED_SPLITBF16: refinement sweeps, 1..8 (0 = 6).  From the
                          single-precision start the eigenvector error is about
                          u32 ||H'|| / gap, up to 1e-2 on the Si Gaussian basis; pairs closer
                          than the sweep's cluster threshold are only orthonormalized and get
                          resolved in a later sweep, so the defect can rise once before it
                          falls to the FP64 floor (six sweeps on the 512-atom k-batch) */
  int n_ev;            /* eigenvectors computed per item: the lowest n_ev (0 = all M).  With
                          0 < n_ev < M, C is (nk, M, n_ev) and the back-transforms and the
                          density matrix touch only those columns (paper Sec. 6: a quarter to
                          a half of the spectrum is needed); eps still holds all M eigenvalues.
                          More occupied states (f >= f_cut) than n_ev is a device-side
                          GKS_EINVAL. */
  long long wait_limit;/* bound of every device-side wait, in SM clock cycles (0 = 2^32,
                          about two seconds); past it the waiting kernel stops, frees its
                          resources and gks_sync returns GKS_ETIMEOUT */
  const char* autotune_cache; /* file of tuned widths: read at gks_create if it exists, rewritten
                          by gks_tune and gks_tune_set; NULL = none.  The string is copied. */
  int debug;           /* test hooks, GKS_DEBUG_* (0 = none) */
  int reduction;       /* gks_reduction: how H C = S C eps becomes a standard problem */
  int tridiag;         /* gks_tridiag */
  int band;            /* two-stage bandwidth, 2..32 (0 = 32) */
  int split;           /* gks_split: form of the split products (0 = residues) */
  int hemv;            /* gks_hemv: form of the one-stage matrix-vector step (0 = digits) */
} gks_opts;

/* One problem of gks_solve_batched: the arguments of gks_solve. */
typedef struct {
  const void* H;
  const void* S;
  int64_t n, nk;
  int dtype, spin_mode;
  double kT, n_elec;
  const double* kweights;
  double* eps;
  void* C;
  double* mu;
  void* rho;
  double* e_band;
} gks_problem;

/* One row of the event profile: a kernel class ("gemm", "hetrd_hemv", ...) or a stage
 * ("stage:potrf", ...), with its algorithmic FP64 flops and bytes (inputs read plus
 * outputs written once) summed over the recorded launch groups. */
typedef struct {
  char name[32];
  int groups;          /* recorded launch groups */
  double ms;           /* summed device time (CUDA events on the context's stream) */
  double flops;        /* algorithmic flops (complex multiply-add = 8) */
  double bytes;        /* algorithmic bytes */
} gks_prof_entry;

/* Create a context bound to opts->device and opts->cuda_stream.  opts may be NULL
 * (device 0, default stream).  On success *ctx is set; release with gks_destroy. */
gks_status gks_create(gks_ctx** ctx, const gks_opts* opts);

/* Release the context and its workspace.  NULL is accepted. */
gks_status gks_destroy(gks_ctx* ctx);

/* Message describing the last error on this context ("" if none).  Valid until the next
 * call on the same context. */
const char* gks_last_error(const gks_ctx* ctx);

/* Full hot path for nk pencils that share one chemical potential (paper Sec. 3.1 Parts
 * 2-4; Sec. 3.2 Parts 3-5):
 *   Cholesky S_k = L_k L_k^H; H'_k = L_k^-1 H_k L_k^-H; Householder tridiagonalization;
 *   divide-and-conquer tridiagonal eigensolve; C_k = L_k^-H Q_k D_k Z_k;
 *   mu from sum_k w_k g_s sum_i f((eps_ki - mu)/kT) = n_elec, f(x) = 1/(1+e^x);
 *   rho_k = C_k diag(g_s f_k) C_k^H over the columns with f >= f_cut;
 *   E_band = sum_k w_k g_s sum_i f_ki eps_ki.
 * Arguments:
 *   H       (nk, M, M) dtype, Hermitian, lower triangle read.  Noncollinear: spin-major
 *           2 x 2 blocks [[H_aa, H_ab], [H_ba, H_bb]] (paper Sec. 3.2 H_NC).
 *           Spin-polarized: (nk, 2, n, n), the up and down channels of each k-point.
 *   S       (nk, n, n) dtype, Hermitian positive definite, lower triangle read.
 *           Noncollinear: the n x n S; S_NC = I_2 (x) S is implied and only S is factored
 *           (paper Sec. 3.2 Parts 3-1..3-4: the spin blocks are reduced with the one
 *           factor).  Spin-polarized: shared by both channels, factored once per k.
 *   n, nk   basis size per spin and number of k-points (n >= 1, nk >= 1).
 *   dtype   GKS_R64 (collinear or spin-polarized Gamma) or GKS_C128.  Noncollinear
 *           requires C128.
 *   kT      Fermi smearing (Hartree), > 0.  n_elec in (0, g_s M) (spin-polarized:
 *           (0, 2 M)).
 *   kweights device (nk) doubles summing to 1, or NULL for 1/nk (spin-polarized: the
 *           weight of a k-point applies to both channels).
 *   flags   0 or GKS_REUSE_S_FACTOR | GKS_SAVE_FOR_BACKWARD | GKS_EIGEN_ONLY.
 * Outputs (device, caller-allocated):
 *   eps (nk, M) ascending per k; C (nk, M, M) dtype ((nk, M, n_ev) with opts.n_ev), column
 *   i = eigenvector i with C^H S C = I and its largest-modulus entry real positive (lowest
 *   row on ties); mu (1); rho (nk, M, M) full Hermitian storage; e_band (1) or NULL.
 *   Spin-polarized: eps (nk, 2, n), C and rho (nk, 2, n, n).
 *   rho follows C diag(g_s f) C^H; the paper's n_lm = sum_i f_i c*_li c_mi equals
 *   conj(rho)/g_s (its transpose for Hermitian rho).
 * The inputs are not modified.  Returns GKS_OK or a host validation error; device
 * status comes from gks_sync. */
gks_status gks_solve(gks_ctx* ctx, const void* H, const void* S, int64_t n, int64_t nk, int dtype, int spin_mode,
                     double kT, double n_elec, const double* kweights, unsigned flags, double* eps, void* C,
                     double* mu, void* rho, double* e_band);

/* Independent problems of uneven order in one launch sequence: problem b is enqueued on
 * worker stream b mod nstreams (nstreams <= 0: 8), the workers forked from and joined back
 * into the context's stream, so small systems run concurrently.  With opts->graph the
 * whole batch is captured into one CUDA graph (first call eager, second call captures,
 * later calls replay).  Each problem keeps its own workspace.  Same conventions and
 * outputs as gks_solve; gks_sync reports the first failing problem. */
gks_status gks_solve_batched(gks_ctx* ctx, int64_t count, const gks_problem* probs, int nstreams);

/* Vector-Jacobian product of a real loss L(rho, eps, E_band) through gks_solve, with
 * n_elec fixed (mu moves with H and S).  First-order perturbation of H C = S C eps,
 * C^H S C = I gives d eps_i = c_i^H (dH - eps_i dS) c_i and, at fixed mu,
 * d rho = g_s C [G o (C^H dH C) - G' o (C^H dS C)] C^H with
 * G_ij = (f_i - f_j)/(eps_i - eps_j), G'_ij = (f_i eps_i - f_j eps_j)/(eps_i - eps_j)
 * (limits f'_i and f_i + eps_i f'_i on equal eigenvalues); the returned gradients satisfy
 * dL = Re tr(H_bar^H dH) + Re tr(S_bar^H dS) for Hermitian dH, dS.
 * Inputs: C, eps, mu as returned by gks_solve for the same (n, nk, dtype, spin, kT,
 * kweights), or C = eps = NULL to use the copies kept by the last solve of that shape
 * with GKS_SAVE_FOR_BACKWARD (mu = NULL: the kept mu too); rho_bar (nk, M, M) = dL/d rho
 * (its Hermitian part is used; NULL = 0); eps_bar (nk, M) = explicit dL/d eps (NULL = 0);
 * e_band_bar = dL/dE_band.  Needs every eigenvector (opts.n_ev = 0).
 * Outputs: H_bar (nk, M, M) and S_bar (nk, n, n), full Hermitian storage (noncollinear:
 * S_bar is the sum of the two diagonal spin blocks, since S_NC = diag(S, S);
 * spin-polarized: H_bar (nk, 2, n, n), S_bar the sum over the two channels).
 * The context keeps a separate workspace (3 M^2 elements per item) for this call. */
gks_status gks_adjoint(gks_ctx* ctx, const void* C, const double* eps, const double* mu, int64_t n, int64_t nk,
                       int dtype, int spin_mode, double kT, const double* kweights, const void* rho_bar,
                       const double* eps_bar, double e_band_bar, void* H_bar, void* S_bar);

/* Occupations, shared chemical potential, density matrix and energy-density matrix for
 * k-points whose eigenpairs come from separate solves (paper Sec. 3.1 Parts 3 and 4; the
 * k-points of one run may be spread over solves or processes, each with GKS_EIGEN_ONLY):
 *   mu from sum_k w_k g_s sum_i f((eps_ki - mu)/kT) = n_elec over ALL nk_all k-points,
 *   rho_k = C_k diag(g_s f_k) C_k^H and E_k = C_k diag(g_s f_k eps_k) C_k^H (the
 *   energy-density matrix of paper Sec. 3.1 Part 4) for the local k-points k0 .. k0+nk-1,
 *   E_band = sum_k w_k g_s sum_i f_ki eps_ki over all k-points.
 * The same bisection as gks_solve: with eps_all equal to a solve's eps, mu and rho equal
 * that solve's bit for bit.  Arguments:
 *   eps_all (nk_all, M) device, ascending per k (spin-polarized: (nk_all, 2, n));
 *   kweights_all (nk_all) device or NULL (1/nk_all);
 *   C (nk, M, ncols) the eigenvectors of the local k-points (ncols = opts.n_ev or M);
 *   mu (1) out; rho, edm (nk, M, M) out or NULL (full Hermitian storage); e_band out or
 *   NULL.  n, dtype, spin_mode, kT, n_elec as in gks_solve.
 * Device-side failures (invalid parameters, more occupied states than n_ev) are reported
 * by gks_sync. */
gks_status gks_occupy(gks_ctx* ctx, const double* eps_all, int64_t nk_all, int64_t k0, const void* C, int64_t n,
                      int64_t nk, int dtype, int spin_mode, double kT, double n_elec, const double* kweights_all,
                      double* mu, void* rho, double* e_band, void* edm);

/* Wait for the context's stream and report the first device-side failure of the work
 * enqueued since the previous gks_sync (GKS_ENOTSPD with the failing column and
 * k-point, GKS_ENOCONV, GKS_EINVAL for occupation parameters found invalid, GKS_ETIMEOUT
 * when a bounded wait expired in a product of a solve, gks_gemm or
 * gks_gemm_split_noalloc). */
gks_status gks_sync(gks_ctx* ctx);

/* Wait for the stream and return the event profile of everything enqueued since the
 * previous gks_profile call (requires opts->profile = 1): up to `max` entries are written
 * to `out`; the return value is the number of entries (0 when profiling is off). */
int gks_profile(gks_ctx* ctx, gks_prof_entry* out, int max);

/* Refinement statistics of the last GKS_MIXED_SPLITBF16 solve on this context (the
 * contraction of the Ogita-Aishima sweeps): out[2 (s items + b) + 0] = the bound on
 * ||I - X^H X||_2 and out[... + 1] = the bound on ||X^H H' X - diag(l)||_2 measured at the
 * start of sweep s for item b (largest absolute row sums).  Waits for the stream; returns
 * the number of values written (at most max), 0 without a mixed-precision solve. */
int gks_refine_stats(gks_ctx* ctx, double* out, int max);

/* Number of kernel launches this library has issued in the calling process. */
long long gks_launch_count(void);

/* Measured throughput of an FP64 unit of the context's device, the denominator of the
 * FP64 rooflines (the paper quotes the H100's FP64 peaks, Sec. 6; this GPU's are
 * measured, not taken from a datasheet): which = 0 DFMA (fma.rn.f64, the FP64 pipe the
 * matrix-vector steps and the FP64 product kernel use), 1 DMMA (mma.sync m8n8k4 f64).
 * Runs about 0.3 s of probes on the context's stream (every SM, independent register
 * chains) and writes the best rate in TFLOP/s to *tflops (host).  Synchronizes. */
gks_status gks_measure_peak(gks_ctx* ctx, int which, double* tflops);

/* C = alpha op(A) op(B) + beta C for one product (row-major, op 0 = N, 1 = T, 2 = conjugate
 * transpose; op(A) is M x K, op(B) K x N).  mode 1: the FP64 pipe; mode 2: split-bf16
 * tensor-core products in the context's opts.split form (the path large products of
 * gks_solve take).  Exposed to check the product kernels on their own. */
gks_status gks_gemm(gks_ctx* ctx, int dtype, int opA, int opB, int64_t M, int64_t N, int64_t K, double alpha,
                    const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                    int mode);

/* Width tuner (the outer block of the two-level blocked Cholesky, reduction and
 * back-transforms, which is also the Householder panel length).  Solves seeded synthetic
 * pencils of order n (2n noncollinear), nk items, dtype and spin as gks_solve would, twice
 * per candidate width (multiples of 64 in 64..1024, host array `widths`), and keeps the
 * fastest for every later solve on this context whose matrix order falls in the same
 * power-of-two bucket, element type and spin mode.  Host outputs: ms[i] the device time of
 * the second solve with widths[i]; *best the chosen width.  Allocates and frees its own
 * test pencils (≈ 3·nk·M² elements); GKS_EINVAL for invalid arguments or pencils above
 * 64 GB.  Graph capture is off for the tuning solves. */
gks_status gks_tune(gks_ctx* ctx, int64_t n, int64_t nk, int dtype, int spin_mode, const int* widths, int count,
                    double* ms, int* best);

/* Set (width > 0) or forget (width = 0) the tuned width of a shape class, e.g. from a
 * cache the caller keeps between runs; gks_tune_get returns the width solves of order n
 * would use now (the tuned one, else opts->block, else the size default). */
gks_status gks_tune_set(gks_ctx* ctx, int64_t n, int dtype, int spin_mode, int width);
int gks_tune_get(const gks_ctx* ctx, int64_t n, int dtype, int spin_mode);

/* Size in bytes of the fixed device scratch behind gks_gemm_split_noalloc. */
#define GKS_NOALLOC_SCRATCH_BYTES 16777216

/* The split-bf16 product of gks_gemm (mode 2) without any device allocation: the digit
 * scratch is a fixed region of GKS_NOALLOC_SCRATCH_BYTES (16 MiB) compiled into this
 * library, one per device, instead of memory the context obtains with cudaMalloc.  For
 * callers that must not allocate device memory at the point of the call: a process whose
 * device memory is already handed out to another allocator or capped, or a loop that
 * cannot afford the device-wide synchronization an allocation implies.  The paper has no
 * counterpart; this is a library service around the same product kernels.
 *
 * Arguments as in gks_gemm; always the digit-pair form (GKS_SPLIT_DIGITS, whatever
 * opts.split says) with the context's opts->slices digits (S, default 9).
 * The scratch needed is S * (Mp + Np) * Kp * 2 + 4 * (Mp + Np) + 1024 bytes with
 * Mp = M rounded up to 128, Np = N' rounded up to 128, Kp = K' rounded up to 64, where
 * N' = N, K' = K for GKS_R64 and N' = 2N, K' = 2K for GKS_C128 (e.g. real 512 x 512 x 512
 * at S = 9 needs 9.4 MB).  A larger product returns GKS_EINVAL before any work is
 * enqueued, with the sizes in gks_last_error.
 *
 * The first call on a device looks up the scratch address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture on the device.
 * A bounded wait that expires in the product (opts.wait_limit) leaves C incomplete and is
 * reported by the next gks_sync on this context as GKS_ETIMEOUT; the call itself returns
 * GKS_OK once the work is enqueued.
 * The work is enqueued on the context's stream and the call returns without waiting.
 * All calls on one device share the one scratch region: two calls whose work overlaps in
 * time (other streams, other contexts, other host threads) corrupt each other's results.
 * Order them on one stream or synchronize between them. */
gks_status gks_gemm_split_noalloc(gks_ctx* ctx, int dtype, int opA, int opB, int64_t M, int64_t N, int64_t K,
                                  double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                                  double beta, void* C, int64_t ldc);

/* Stage entry points (same conventions; `count` independent matrices of order m,
 * stride m*m elements).  Used to check each stage on its own. */

/* In place: A_b = L_b L_b^H, L in the lower triangle (upper triangle untouched). */
gks_status gks_potrf(gks_ctx* ctx, void* A, int64_t m, int64_t count, int dtype);

/* In place: H_b <- L_b^-1 H_b L_b^-H (lower triangle written; upper untouched), with L_b
 * the Cholesky factor of S_b.  S_b is overwritten by L_b. */
gks_status gks_reduce(gks_ctx* ctx, void* H, void* S, int64_t m, int64_t count, int dtype);

/* Stage 1 of the two-stage reduction (dense -> band of width `band`, 2..32): A (count, m, m),
 * Hermitian, lower triangle read, is replaced by the band matrix B = Q1^H A Q1 in full
 * Hermitian storage (zero outside the band); Q (count, m, m) receives Q1 (NULL: not formed).
 * Reflectors follow LAPACK's zlarfg convention (complex tau, real beta). */
gks_status gks_he2hb(gks_ctx* ctx, void* A, int64_t m, int64_t count, int dtype, int band, void* Q);

/* Stage 2 of the two-stage reduction (band -> tridiagonal by bulge chasing): B (count, m, m)
 * Hermitian band of width `band` (lower band read), d (count, m) and e (count, m) receive
 * the real tridiagonal T = Q2^H B Q2 (e[b][i] = T_{i+1,i}, last entry 0); X (count, m, ncols)
 * is replaced by Q2 X (NULL or ncols = 0: not applied).  The chase is a persistent kernel
 * whose waits are bounded by opts.wait_limit (GKS_ETIMEOUT from gks_sync). */
gks_status gks_hb2st(gks_ctx* ctx, const void* B, int64_t m, int64_t count, int dtype, int band, double* d, double* e,
                     void* X, int64_t ncols);

/* Real symmetric tridiagonal eigensolve by divide and conquer: d (count, m) diagonal,
 * e (count, m) with e[b][i] = T_{i+1,i} (last entry ignored); lam (count, m) ascending,
 * Z (count, m, m) real, column j = eigenvector j.  d and e are not modified. */
gks_status gks_stedc(gks_ctx* ctx, const double* d, const double* e, int64_t m, int64_t count, double* lam,
                     double* Z);

#ifdef __cplusplus
}
#endif
#endif /* GKS_H */
