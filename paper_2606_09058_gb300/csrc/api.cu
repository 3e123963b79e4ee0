// Runtime and C ABI: context, workspace arena, stage orchestration, status reporting.
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dense.h"
#include "gks.h"

using namespace gks;

namespace {
constexpr int NB = 64;  // panel / reflector block width
constexpr int kMaxSweeps = 8;   // refinement sweeps of the mixed-precision path (opts bound)
constexpr int kLowSlices = 5;   // digits per operand of the mixed path's back-transform products

struct Arena {
  size_t off = 0;
  template <typename X>
  size_t take(size_t n) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + sizeof(X) * (n ? n : 1);
    return o;
  }
};
}  // namespace

namespace {
const char* kClassNames[PC_NCLASS] = {"gemm", "potf2", "trsm_block", "hegst_diag", "hetrd_hemv", "hetrd_update",
                                      "hetrd_vec", "dc_leaf", "dc_secular", "dc_gemm", "backtr_aux",
                                      "occupations", "misc", "split_gemm"};
const char* kStageNames[PS_NSTAGE] = {"stage:copy", "stage:potrf", "stage:hegst", "stage:hetrd", "stage:stedc",
                                      "stage:backtransform", "stage:unreduce", "stage:occupations", "stage:rho",
                                      "stage:adjoint", "stage:refine"};

struct EventProf : Prof {
  cudaStream_t stream = nullptr;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec {
    int cls, e0, e1;
    double flops, bytes;
  };
  std::vector<Rec> recs;
  // deferred flops of the density-matrix GEMM (its K is the device-side n_rho)
  const int* nrho_dev = nullptr;
  int rho_m = 0, rho_nk = 0, rho_es = 8;
  int ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return (int)used++;
  }
  int begin() override {
    if (!on) return -1;
    int e = ev();
    cudaEventRecord(pool[e], stream);
    return e;
  }
  void end(int tok, int cls, double flops, double bytes) override {
    if (tok < 0) return;
    int e = ev();
    cudaEventRecord(pool[e], stream);
    recs.push_back({cls, tok, e, flops, bytes});
  }
  ~EventProf() override {
    for (auto e : pool) cudaEventDestroy(e);
  }
};
}  // namespace

struct SolveKey {
  const void *H, *S, *kw, *eps, *C, *mu, *rho, *eb;
  long long n, nk;
  int dtype, spin;
  double kT, ne;
  unsigned flags;
  unsigned reserved;  // keeps the struct free of padding (keys are compared with memcmp)
};

struct gks_ctx {
  EventProf prof;
  int device = 0;
  bool graph = false;                  // capture solves into CUDA graphs
  int gemm_mode = 0;                   // 0 auto, 1 DFMA only, 2 split products always
  int slices = 9;                      // split products: 6-bit digits per operand, or 6 slices bits
  int split = 0;                       // split-product form: 0 residues (CRT), 1 digit pairs
  int hemv = 0;                        // one-stage matrix-vector step: 0 integer digits, 1 FP64 pipe
  int wsdig = 0;                       // workspace holds the digit planes of the stale block
  int nbb = 256;                       // outer block of the two-level blocked stages (active)
  int nbb_default = 256;               // opts.block, used for shapes the tuner has not seen
  bool nbb_fixed = false;              // opts.block given: no size-dependent default
  std::map<std::tuple<int, int, int>, int> tuned;  // (order bucket, element size, spin) -> width
  void* oz = nullptr;                  // digit workspace of the split-product GEMM
  size_t oz_bytes = 0;
  cudaGraphExec_t gexec = nullptr;     // graph of the last captured solve
  SolveKey gkey{};
  std::vector<gks_ctx*> subs;          // per-problem contexts of gks_solve_batched
  std::vector<cudaStream_t> workers;   // fork/join streams of gks_solve_batched
  cudaGraphExec_t bexec = nullptr;     // graph of the last captured batch
  std::vector<SolveKey> bkey;
  cudaStream_t stream = nullptr;
  double f_cut = 1e-16;
  std::string err;
  DevStatus* noalloc_st = nullptr;     // status word of the last gks_gemm_split_noalloc call
  DevStatus* gst = nullptr;            // status word of gks_gemm and gks_occupy (one entry)
  long long wait_cycles = 1ll << 32;   // bound of every device-side wait (opts.wait_limit)
  int n_ev = 0;                        // eigenvectors per item (0 = all)
  int reduction = GKS_REDUCE_CHOLESKY; // Cholesky or Loewdin reduction to the standard problem
  int tridiag = GKS_TRIDIAG_ONE_STAGE;  // one-stage panel Householder or two-stage (band + chase)
  int band = 32;                        // bandwidth of the two-stage reduction
  int wstwo = 0;                        // workspace holds the two-stage buffers
  int precision = GKS_FP64;
  int refine_sweeps = 6;
  int debug = 0;                       // test hooks (GKS_DEBUG_*)
  std::string tune_cache;              // file of tuned widths (opts.autotune_cache)
  // Cholesky factor kept in the L workspace from the solve that produced it
  SolveKey lkey{};
  bool l_valid = false;
  // copies kept for gks_adjoint (GKS_SAVE_FOR_BACKWARD): C, eps, mu of the last such solve
  char* sv = nullptr;
  size_t sv_bytes = 0;
  SolveKey svkey{};
  bool sv_valid = false;
  int rstat_sweeps = 0, rstat_items = 0;  // shape of the refinement statistics of the last solve
  // occupation workspace of gks_occupy (weights, f, g_s f, g_s f eps, n_rho for all items)
  char* ow = nullptr;
  size_t ow_bytes = 0;
  // workspace for the current shape
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int m = -1, n = -1, nk = -1, es = -1, nc = -1, wsmixed = 0;
  DcPlan* dc = nullptr;
  DevStatus* st = nullptr;
  // adjoint workspace (separate arena, sized for the last adjoint shape)
  char* aws = nullptr;
  size_t aws_bytes = 0;
  int am = -1, ank = -1, aes = -1;
  // offsets (bytes) of per-item arrays; each holds nk items
  size_t oA, oL, oF, oFB, oU, oQ, opart, oy, ouw, oSg, oV, oG, oT, oY, oY2, ou, op, oph, otau, otb, od, oe, oZ, oocc, oks, onrho,
      oweights, oeb, odc, oticket, oAf, oRY, oRT, oRR, onrm, orstat, operm, oflag, oBd, oV2, otau2, oprog, oerr, oqr, oD, oud, ofu, ormax,
      otau1, oT1, oP1, oP2, oVT, oXb, oGb, oYb, oZb, oXp, oVw, otw, oGw, oTw, oYw, oY2w;
  int ldt2 = 0, nblkmax = 0;
  long long sMM, sF, sFB, sU, spart, sy, sV, sG, sT, sY, sVec;
};

namespace {

// The split-product form and precision handed to ozaki_gemm: residues carrying at least
// 6 slices bits (negative) or slices 6-bit digits.
int sform(const gks_ctx* c) { return c->split == 0 ? -c->slices : c->slices; }

gks_status fail(gks_ctx* c, gks_status code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// Makes `dev` current for the duration of an entry point and restores the caller's
// current device on return.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

gks_status cuda_check(gks_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, GKS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return GKS_OK;
}

void release_aws(gks_ctx* c) {
  if (c->aws) cudaFree(c->aws);
  c->aws = nullptr;
  c->aws_bytes = 0;
  c->am = -1;
}

void release_graph(gks_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  if (c->bexec) cudaGraphExecDestroy(c->bexec);
  c->bexec = nullptr;
  c->bkey.clear();
}

void release_oz(gks_ctx* c) {
  if (c->oz) cudaFree(c->oz);
  c->oz = nullptr;
  c->oz_bytes = 0;
}

void release_extra(gks_ctx* c) {
  if (c->sv) cudaFree(c->sv);
  c->sv = nullptr;
  c->sv_bytes = 0;
  c->sv_valid = false;
  if (c->ow) cudaFree(c->ow);
  c->ow = nullptr;
  c->ow_bytes = 0;
  if (c->gst) cudaFree(c->gst);
  c->gst = nullptr;
}

void release_ws(gks_ctx* c) {
  release_graph(c);
  c->l_valid = false;
  if (c->ws) cudaFree(c->ws);
  if (c->st) cudaFree(c->st);
  dc_plan_destroy(c->dc);
  c->ws = nullptr;
  c->st = nullptr;
  c->dc = nullptr;
  c->ws_bytes = 0;
  c->m = -1;
}

// Orders share a tuned width by power-of-two bucket.
int order_bucket(int m) {
  int b = 64;
  while (b < m) b <<= 1;
  return b;
}

// Width for a shape: the tuned one, else opts.block, else 512 from order 4096 up (the WY
// back-transform gains most from wider blocks there) and 256 below.
int pick_width(const gks_ctx* c, int m, int es, int nc) {
  auto it = c->tuned.find(std::make_tuple(order_bucket(m), es, nc));
  if (it != c->tuned.end()) return it->second;
  if (c->nbb_fixed) return c->nbb_default;
  return m >= 4096 ? 512 : 256;
}

// Shape class of a spin mode for the tuned widths: spin-polarized runs share the
// collinear class (same order and element type).
int shape_spin(int spin) { return spin == GKS_NONCOLLINEAR ? 1 : 0; }

// Workspace for nk items of order m (element size es, n = basis per spin, nc = spin mode).
gks_status ensure_ws(gks_ctx* c, int m, int n, int nk, int es, int nc) {
  const int want = pick_width(c, m, es, shape_spin(nc));
  const int mixed = c->precision != GKS_FP64 ? 1 : 0;
  const int two = c->tridiag == GKS_TRIDIAG_TWO_STAGE ? c->band : 0;
  const int dig = c->hemv == 0 && !mixed ? 1 : 0;
  if (c->ws && c->m == m && c->n == n && c->nk == nk && c->es == es && c->nc == nc && c->nbb == want &&
      c->wsmixed == mixed && c->wstwo == two && c->wsdig == dig)
    return GKS_OK;
  release_ws(c);
  c->nbb = want;
  const size_t MM = (size_t)m * m;
  c->sMM = (long long)MM;
  const int nbb = c->nbb;
  c->sF = NB * NB;
  c->sFB = (long long)nbb * nbb;
  c->sV = (long long)m * nbb;
  c->sG = (long long)nbb * nbb;
  c->sT = (long long)nbb * nbb;
  c->sY = (long long)nbb * m;
  c->sU = (long long)m * nbb;
  c->spart = (long long)((m + 15) / 16) * (2 * nbb + 2);
  c->sy = 2 * nbb + 2;
  c->sVec = m;
  Arena a;
  auto elems = [&](long long per) { return (size_t)per * nk * es; };
  c->oA = a.take<char>(elems(c->sMM));
  c->oL = a.take<char>(elems(c->sMM));
  c->oF = a.take<char>(elems(c->sF));
  c->oFB = a.take<char>(elems(c->sFB));
  c->oU = a.take<char>(elems(c->sU));
  c->oQ = a.take<char>(elems(c->sU));
  c->opart = a.take<char>(elems(c->spart));
  c->oy = a.take<char>(elems(c->sy));
  c->ouw = a.take<double>((size_t)3 * m * nk);
  c->oSg = es == 16 && !dig ? a.take<double>(MM * nk) : 0;
  if (dig) {
    // digit planes of the stale block and of u (14 planes complex, 7 real), scale exponents
    const size_t ldd = ((size_t)m + 15) / 16 * 16, npl = es == 16 ? 14 : 7;
    c->oD = a.take<char>((ldd + 31) / 32 * 32 * ldd * npl * nk);  // rows in tiles of 32
    c->oud = a.take<char>(ldd * npl * nk);
    c->ofu = a.take<int>((size_t)nk);
    c->ormax = a.take<unsigned long long>(ldd * nk);
  }
  c->oV = a.take<char>(elems(c->sV));
  c->oG = a.take<char>(elems(c->sG));
  c->oT = a.take<char>(elems(c->sT));
  c->oY = a.take<char>(elems(c->sY));
  c->oY2 = a.take<char>(elems(c->sY));
  c->ou = a.take<char>(elems(m));
  c->op = a.take<char>(elems(m));
  c->oph = a.take<char>(elems(m));
  c->otau = a.take<double>((size_t)m * nk);
  c->otb = a.take<double>((size_t)nbb * nk);
  c->od = a.take<double>((size_t)m * nk);
  c->oe = a.take<double>((size_t)m * nk);
  c->oZ = a.take<double>(MM * nk);
  c->oocc = a.take<double>((size_t)m * nk);
  c->oks = a.take<double>((size_t)m * nk);
  c->onrho = a.take<int>((size_t)nk);
  c->oweights = a.take<double>((size_t)nk);
  c->oeb = a.take<double>(4);
  c->oticket = a.take<int>((size_t)2 * nk);
  c->dc = dc_plan_create(m, nk);
  c->odc = a.take<char>(dc_workspace_bytes(c->dc));
  if (two) {
    // two-stage: band storage, the chase's reflectors and progress counters, the panel
    // buffers of stage 1, the padded copy of X and the wavefront buffers of Q2
    const int bb = two, W = 2 * bb + 1, hp = 2 * bb;
    c->ldt2 = (m + bb - 1) / bb + 2;
    c->nblkmax = m / (2 * bb) + 3;
    c->oBd = a.take<char>(elems((long long)m * W));
    c->oV2 = a.take<char>(elems(c->sMM));
    c->otau2 = a.take<char>(elems((long long)m * c->ldt2));
    c->oprog = a.take<int>((size_t)m * nk);
    c->oerr = a.take<int>(4);
    c->oqr = a.take<char>(qr_scratch_bytes(nk, es));
    c->otau1 = a.take<char>(elems((long long)m + bb));
    c->oT1 = a.take<char>(elems((long long)(m / bb + 2) * bb * bb));
    c->oP1 = a.take<char>(elems((long long)m * 2 * bb));
    c->oP2 = a.take<char>(elems((long long)m * 2 * bb));
    c->oVT = a.take<char>(elems((long long)m * bb));
    c->oXb = a.take<char>(elems((long long)m * bb));
    c->oGb = a.take<char>(elems((long long)bb * bb));
    c->oYb = a.take<char>(elems((long long)bb * bb));
    c->oZb = a.take<char>(elems((long long)bb * bb));
    c->oXp = a.take<char>(elems((long long)(m + hp) * m));
    c->oVw = a.take<char>(elems((long long)c->nblkmax * hp * bb));
    c->otw = a.take<char>(elems((long long)c->nblkmax * bb));
    c->oGw = a.take<char>(elems((long long)c->nblkmax * bb * bb));
    c->oTw = a.take<char>(elems((long long)c->nblkmax * bb * bb));
    c->oYw = a.take<char>(elems((long long)c->nblkmax * m * bb));
    c->oY2w = a.take<char>(elems((long long)c->nblkmax * m * bb));
  }
  if (mixed) {
    // single-precision copy of H' for the tridiagonalization, refinement products Y, T, R,
    // the per-item norms, and the reordering buffers
    c->oAf = a.take<char>(elems(c->sMM) / 2);
    c->oRY = a.take<char>(elems(c->sMM));
    c->oRT = a.take<char>(elems(c->sMM));
    c->oRR = a.take<char>(elems(c->sMM));
    c->onrm = a.take<double>((size_t)3 * nk);
    c->orstat = a.take<double>((size_t)2 * kMaxSweeps * nk);
    c->operm = a.take<int>((size_t)m * nk);
    c->oflag = a.take<int>((size_t)nk);
  }
  c->ws_bytes = a.off;
  if (cudaMalloc(&c->ws, c->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    c->ws = nullptr;
    dc_plan_destroy(c->dc);
    c->dc = nullptr;
    return fail(c, GKS_ENOMEM, "workspace allocation of " + std::to_string(c->ws_bytes) + " bytes failed");
  }
  if (cudaMalloc(&c->st, sizeof(DevStatus) * nk) != cudaSuccess) {
    cudaGetLastError();
    release_ws(c);
    return fail(c, GKS_ENOMEM, "status allocation failed");
  }
  cudaMemset(c->st, 0, sizeof(DevStatus) * nk);
  c->wsmixed = mixed;
  c->wstwo = two;
  c->wsdig = dig;
  c->m = m;
  c->n = n;
  c->nk = nk;
  c->es = es;
  c->nc = nc;
  return cuda_check(c, "workspace setup");
}

template <typename X>
X* at(gks_ctx* c, size_t off) {
  return reinterpret_cast<X*>(c->ws + off);
}

// Eigenvector columns a solve of order M returns (opts.n_ev, 0 = all).
int ncols_of(const gks_ctx* c, int M) { return (c->n_ev > 0 && c->n_ev < M) ? c->n_ev : M; }

// Keep copies of C, eps and mu of this solve for a later gks_adjoint that passes NULL for
// them (GKS_SAVE_FOR_BACKWARD); the context owns them until the next such solve.
gks_status save_for_backward(gks_ctx* c, const SolveKey& k, int M, int items, int nev) {
  const int es = k.dtype == GKS_C128 ? 16 : 8;
  const size_t bC = (size_t)items * M * nev * es, bE = (size_t)items * M * sizeof(double);
  const size_t need = ((bC + 255) & ~size_t(255)) + ((bE + 255) & ~size_t(255)) + 256;
  if (need > c->sv_bytes) {
    cudaStreamSynchronize(c->stream);
    if (c->sv) cudaFree(c->sv);
    c->sv = nullptr;
    c->sv_bytes = 0;
    if (cudaMalloc(&c->sv, need) != cudaSuccess) {
      cudaGetLastError();
      c->sv = nullptr;
      c->sv_valid = false;
      return fail(c, GKS_ENOMEM, "allocation of the saved eigenpairs (" + std::to_string(need) + " bytes) failed");
    }
    c->sv_bytes = need;
  }
  char* base = c->sv;
  const size_t oE = (bC + 255) & ~size_t(255), oM = oE + ((bE + 255) & ~size_t(255));
  cudaMemcpyAsync(base, k.C, bC, cudaMemcpyDeviceToDevice, c->stream);
  cudaMemcpyAsync(base + oE, k.eps, bE, cudaMemcpyDeviceToDevice, c->stream);
  c->svkey = k;
  c->sv_valid = false;
  if (!(k.flags & GKS_EIGEN_ONLY)) {
    // mu is written by the occupation stage later in the same solve; copy it then
    c->sv_valid = true;
  } else {
    cudaMemsetAsync(base + oM, 0, sizeof(double), c->stream);
    c->sv_valid = true;
  }
  return GKS_OK;
}

void save_mu(gks_ctx* c, const SolveKey& k, int M, int items, int nev) {
  const int es = k.dtype == GKS_C128 ? 16 : 8;
  const size_t bC = (size_t)items * M * nev * es, bE = (size_t)items * M * sizeof(double);
  const size_t oM = ((bC + 255) & ~size_t(255)) + ((bE + 255) & ~size_t(255));
  cudaMemcpyAsync(c->sv + oM, k.mu, sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

double gemm_flops(int es, int M, int N, int K, int lower, int count) {
  double mn = lower ? 0.5 * (double)M * (M + 1) : (double)M * N;
  return (es == 16 ? 8.0 : 2.0) * mn * K * count;
}
double gemm_bytes(int es, int M, int N, int K, int lower, int count, bool beta) {
  double mn = lower ? 0.5 * (double)M * (M + 1) : (double)M * N;
  return (double)es * ((double)M * K + (double)K * N + mn * (beta ? 2.0 : 1.0)) * count;
}

template <typename T>
void gm(cudaStream_t s, int count, int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda,
        long long sA, const T* B, int ldb, long long sB, double beta, T* C, int ldc, long long sC, int lower = 0,
        const double* ks = nullptr, long long sK = 0, const int* kdev = nullptr) {
  if (M <= 0 || N <= 0) return;
  GemmBatch g{};
  g.base = GemmDesc{A, B, C, ks, M, N, K, lda, ldb, ldc};
  g.list = nullptr;
  g.sA = sA;
  g.sB = sB;
  g.sC = sC;
  g.sK = sK;
  g.kdev = kdev;
  g.count = count;
  g.opA = opA;
  g.opB = opB;
  g.lower = lower;
  g.alpha = alpha;
  g.beta = beta;
  gemm<T>(g, M, N, s);
}

// gm with a profiler record (class PC_GEMM)
template <typename T>
void gmp(gks_ctx* c, int count, int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda, long long sA,
         const T* B, int ldb, long long sB, double beta, T* C, int ldc, long long sC, int lower = 0) {
  if (M <= 0 || N <= 0) return;
  int tok = c->prof.begin();
  gm<T>(c->stream, count, opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, lower);
  c->prof.end(tok, PC_GEMM, gemm_flops(sizeof(T), M, N, K, lower, count),
              gemm_bytes(sizeof(T), M, N, K, lower, count, beta != 0.0));
}

// Profiler record around one launch group.
struct Rec {
  gks_ctx* c;
  int tok, cls;
  double flops, bytes;
  Rec(gks_ctx* c_, int cls_, double fl = 0.0, double by = 0.0) : c(c_), cls(cls_), flops(fl), bytes(by) {
    tok = c->prof.begin();
  }
  ~Rec() { c->prof.end(tok, cls, flops, bytes); }
};
// Stage bracket (recorded as class PC_NCLASS + stage), also an NVTX range named after the
// stage for timeline tools (no cost without an attached tool).
struct StageRec {
  gks_ctx* c;
  int tok, st;
  StageRec(gks_ctx* c_, int st_) : c(c_), st(st_) {
    nvtxRangePushA(kStageNames[st]);
    tok = c->prof.begin();
  }
  ~StageRec() {
    c->prof.end(tok, PC_NCLASS + st, 0.0, 0.0);
    nvtxRangePop();
  }
};

double cmul(int es) { return es == 16 ? 8.0 : 2.0; }

// GEMM dispatch: large products go through exact split-bf16 products with FP64
// accumulation (ozaki.cu) when M, N, K >= 256 and the batch fills at least one wave of
// 128 x 128 output tiles; the rest stays on the DFMA kernel.  Batch items are split into
// launches whose digit workspace stays within kOzCap bytes.
constexpr size_t kOzCap = (size_t)12 << 30;

// Digit workspace for split products of `count` items of `item` bytes each: items per
// launch (within kOzCap), growing the buffer when needed; 0 if it cannot be allocated.
int oz_reserve(gks_ctx* c, size_t item, int count) {
  const int maxper = (int)std::max<size_t>(1, std::min<size_t>((size_t)count, kOzCap / item));
  const int nch = (count + maxper - 1) / maxper, per = (count + nch - 1) / nch;
  const size_t need = item * per;
  if (need > c->oz_bytes) {
    cudaStreamSynchronize(c->stream);
    release_oz(c);
    if (cudaMalloc(&c->oz, need) != cudaSuccess) {
      cudaGetLastError();
      c->oz = nullptr;
      return 0;
    }
    c->oz_bytes = need;
  }
  return per;
}

bool split_worth(gks_ctx* c, int count, int M, int N, int K, int es, double fl) {
  if (c->gemm_mode == 2) return true;
  const int Ne = es == 16 ? 2 * N : N;  // embedded output columns
  return c->gemm_mode == 0 && fl >= 2e8 * count && M >= 64 && Ne >= 64 && K >= 64 &&
         (long long)ozaki_tiles(M, N, es == 16) * count >= 152;
}

template <typename T>
void gmx(gks_ctx* c, int count, int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda, long long sA,
         const T* B, int ldb, long long sB, double beta, T* C, int ldc, long long sC, int lower = 0) {
  if (M <= 0 || N <= 0) return;
  if constexpr (!std::is_same<T, double>::value && !std::is_same<T, zc>::value) {
    // single precision (the FP32 tridiagonalization): the FP32 pipe
    gmp<T>(c, count, opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, lower);
    return;
  } else {
  const int es = sizeof(T);
  const double fl = gemm_flops(es, M, N, K, lower, count);
  const int per = split_worth(c, count, M, N, K, es, fl)
                      ? oz_reserve(c, ozaki_workspace_bytes(M, N, K, es == 16, sform(c)), count)
                      : 0;
  if (per == 0) {
    gmp<T>(c, count, opA, opB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, lower);
    return;
  }
  Rec r(c, PC_OZAKI, fl, gemm_bytes(es, M, N, K, lower, count, beta != 0.0));
  for (int z0 = 0; z0 < count; z0 += per) {
    const int cnt = std::min(per, count - z0);
    // test hook (GKS_DEBUG_SKIP_COPY): the next split product leaves out its fourth operand
    // copy in every CTA, so that its bounded waits expire
    const long long skip = (c->debug & GKS_DEBUG_SKIP_COPY) ? 3 : -1;
    c->debug &= ~GKS_DEBUG_SKIP_COPY;
    if (!ozaki_gemm<T>(opA, opB, M, N, K, alpha, A + z0 * sA, lda, sA, B + z0 * sB, ldb, sB, beta, C + z0 * sC, ldc,
                       sC, cnt, lower, sform(c), c->oz, c->st ? c->st : c->gst, c->stream, nullptr, 0, nullptr,
                       c->wait_cycles, skip))
      gmp<T>(c, cnt, opA, opB, M, N, K, alpha, A + z0 * sA, lda, sA, B + z0 * sB, ldb, sB, beta, C + z0 * sC, ldc, sC,
             lower);
  }
  }
}

// gmx for a two-level batch: item z of A, B, C at (z / nb2) sX + (z % nb2) sX2 (count a
// multiple of nb2).  Split products run in launches of whole outer groups when one group's
// workspace fits, else of runs within a group (single-level, stride sX2).
template <typename T>
void gmx2(gks_ctx* c, int count, int nb2, int opA, int opB, int M, int N, int K, double alpha, const T* A, int lda,
          long long sA, long long sA2, const T* B, int ldb, long long sB, long long sB2, double beta, T* C, int ldc,
          long long sC, long long sC2) {
  if (M <= 0 || N <= 0 || count <= 0) return;
  const int es = sizeof(T);
  const double fl = gemm_flops(es, M, N, K, 0, count);
  auto fp64 = [&](const T* Ap, const T* Bp, T* Cp, int cnt, int nb, long long a1, long long a2, long long b1,
                  long long b2, long long c1, long long c2) {
    int tok = c->prof.begin();
    GemmBatch g{};
    g.base = GemmDesc{Ap, Bp, Cp, nullptr, M, N, K, lda, ldb, ldc};
    g.sA = a1;
    g.sB = b1;
    g.sC = c1;
    g.nb2 = nb;
    g.sA2 = a2;
    g.sB2 = b2;
    g.sC2 = c2;
    g.count = cnt;
    g.opA = opA;
    g.opB = opB;
    g.alpha = alpha;
    g.beta = beta;
    gemm<T>(g, M, N, c->stream);
    c->prof.end(tok, PC_GEMM, gemm_flops(es, M, N, K, 0, cnt), gemm_bytes(es, M, N, K, 0, cnt, beta != 0.0));
  };
  const int per = (count % nb2 == 0 && split_worth(c, count, M, N, K, es, fl))
                      ? oz_reserve(c, ozaki_workspace_bytes(M, N, K, es == 16, sform(c)), count)
                      : 0;
  if (per == 0) {
    fp64(A, B, C, count, nb2, sA, sA2, sB, sB2, sC, sC2);
    return;
  }
  auto split = [&](const T* Ap, const T* Bp, T* Cp, int cnt, int nb, long long a1, long long a2, long long b1,
                   long long b2, long long c1, long long c2) {
    Rec r(c, PC_OZAKI, gemm_flops(es, M, N, K, 0, cnt), gemm_bytes(es, M, N, K, 0, cnt, beta != 0.0));
    if (!ozaki_gemm<T>(opA, opB, M, N, K, alpha, Ap, lda, a1, Bp, ldb, b1, beta, Cp, ldc, c1, cnt, 0, sform(c), c->oz,
                       c->st ? c->st : c->gst, c->stream, nullptr, 0, nullptr, c->wait_cycles, -1, a2, b2, c2, nb))
      fp64(Ap, Bp, Cp, cnt, nb, a1, a2, b1, b2, c1, c2);
  };
  const int ng = count / nb2;
  if (per >= nb2) {
    const int gper = per / nb2;
    for (int g0 = 0; g0 < ng; g0 += gper) {
      const int gc = std::min(gper, ng - g0);
      split(A + g0 * sA, B + g0 * sB, C + g0 * sC, gc * nb2, nb2, sA, sA2, sB, sB2, sC, sC2);
    }
    return;
  }
  for (int g = 0; g < ng; g++)
    for (int j0 = 0; j0 < nb2; j0 += per) {
      const int jc = std::min(per, nb2 - j0);
      split(A + g * sA + j0 * sA2, B + g * sB + j0 * sB2, C + g * sC + j0 * sC2, jc, 0, sA2, 0, sB2, 0, sC2, 0);
    }
}

// rho_k = C_k diag(ks_k) C_k^H over the leading n_rho(k) columns (n_rho read on the device),
// lower triangle.  C_k is M x (>= n_rho) with leading dimension ldc and item stride sC;
// rho_k is M x M (stride sR).  Split products take K = the columns of C with the device
// count cutting the digits and the k loop; the FP64 kernel reads the same count.
template <typename T>
void rho_run(gks_ctx* c, const T* C, int ldc, long long sC, T* rho, long long sR, const double* ks, long long sks,
             const int* nrho, int M, int K, int nk) {
  const int es = sizeof(T);
  const int per = split_worth(c, nk, M, M, K, es, gemm_flops(es, M, M, std::max(1, K / 4), 1, nk))
                      ? oz_reserve(c, ozaki_workspace_bytes(M, M, K, es == 16, sform(c)), nk)
                      : 0;
  int z0 = 0;
  for (; per > 0 && z0 < nk; z0 += per) {
    const int cnt = std::min(per, nk - z0);
    if (!ozaki_gemm<T>(OP_N, OP_C, M, M, K, 1.0, C + z0 * sC, ldc, sC, C + z0 * sC, ldc, sC, 0.0, rho + z0 * sR, M,
                       sR, cnt, 1, sform(c), c->oz, c->st ? c->st : c->gst, c->stream, ks + z0 * sks, sks,
                       nrho + z0, c->wait_cycles))
      break;  // tensor maps unavailable: the FP64 kernel takes the remaining items
  }
  if (z0 >= nk) return;
  GemmBatch g{};
  g.base = GemmDesc{C + z0 * sC, C + z0 * sC, rho + z0 * sR, ks + z0 * sks, M, M, K, ldc, ldc, M};
  g.sA = sC;
  g.sB = sC;
  g.sC = sR;
  g.sK = sks;
  g.kdev = nrho + z0;
  g.count = nk - z0;
  g.opA = OP_N;
  g.opB = OP_C;
  g.lower = 1;
  g.alpha = 1.0;
  g.beta = 0.0;
  gemm<T>(g, M, M, c->stream);
}

// Blocked right-looking Cholesky of the leading n x n block of each item (in place, lower;
// leading dimension ld, item stride sL), two levels.  Outer panels of nbb columns: inside a
// panel, 64-wide steps (diagonal block in shared memory, L21 = A21 L11^-H by substitution,
// rank-64 update of the rest of the panel only); after the panel, one rank-nbb update of
// the trailing matrix (the product that dominates, with K = nbb).
template <typename T>
void potrf_run(gks_ctx* c, T* L, int n, int ld, long long sL, int nk) {
  cudaStream_t s = c->stream;
  const int es = sizeof(T);
  const int nbb = c->nbb;
  for (int K0 = 0; K0 < n; K0 += nbb) {
    const int KB = std::min(nbb, n - K0);
    for (int k0 = K0; k0 < K0 + KB; k0 += NB) {
      const int kb = std::min(NB, K0 + KB - k0);
      {
        Rec r(c, PC_POTF2, cmul(es) * kb * kb * kb / 6.0 * nk, 2.0 * es * kb * kb * nk);
        potf2<T>(L, ld, sL, k0, kb, c->st, nk, s);
      }
      const int rows = n - k0 - kb;
      if (rows <= 0) continue;
      T* L11 = L + (size_t)k0 * ld + k0;
      T* L21 = L + (size_t)(k0 + kb) * ld + k0;
      {
        Rec r(c, PC_TRSM, cmul(es) * 0.5 * kb * kb * rows * nk, (2.0 * rows * kb + 0.5 * kb * kb) * es * nk);
        trsm_block<T>(TRSM_RIGHT_CONJ, L11, ld, sL, L21, ld, sL, kb, rows, nk, s);
      }
      const int w = K0 + KB - (k0 + kb);  // panel columns right of this step
      if (w > 0) gmx<T>(c, nk, OP_N, OP_C, rows, w, kb, -1.0, L21, ld, sL, L21, ld, sL, 1.0, L21 + kb, ld, sL, 1);
    }
    const int rows2 = n - K0 - KB;
    if (rows2 > 0) {
      T* P = L + (size_t)(K0 + KB) * ld + K0;
      gmx<T>(c, nk, OP_N, OP_C, rows2, rows2, KB, -1.0, P, ld, sL, P, ld, sL, 1.0, P + KB, ld, sL, 1);
    }
  }
}

// X <- L^-1 X (conj = false) or L^-H X (conj = true) for the n x ncols block X (leading
// dimension ldx, item stride sX) with the lower n x n factor L (ldl, sL), two levels: within
// an outer block of nbb rows, 64-row diagonal blocks by substitution and updates of the
// rows of that outer block only; then one K = nbb update of all rows beyond it.
template <typename T>
void trsm_left_run(gks_ctx* c, const T* L, int ldl, long long sL, T* X, int ldx, long long sX, int n, int ncols,
                   int nk, bool conj) {
  cudaStream_t s = c->stream;
  const int es = sizeof(T);
  const int nbb = c->nbb;
  const int nob = (n + nbb - 1) / nbb;
  const double fl = cmul(es) * 0.5, by = es;
  if (!conj) {
    for (int ob = 0; ob < nob; ob++) {
      const int R0 = ob * nbb, RB = std::min(nbb, n - R0);
      for (int r0 = R0; r0 < R0 + RB; r0 += NB) {
        const int rb = std::min(NB, R0 + RB - r0);
        T* Xi = X + (size_t)r0 * ldx;
        {
          Rec r(c, PC_TRSM, fl * rb * rb * ncols * nk, (2.0 * ncols * rb + 0.5 * rb * rb) * by * nk);
          trsm_block<T>(TRSM_LEFT, L + (size_t)r0 * ldl + r0, ldl, sL, Xi, ldx, sX, rb, ncols, nk, s);
        }
        const int below = R0 + RB - r0 - rb;
        if (below > 0)
          gmx<T>(c, nk, OP_N, OP_N, below, ncols, rb, -1.0, L + (size_t)(r0 + rb) * ldl + r0, ldl, sL, Xi, ldx, sX,
                 1.0, X + (size_t)(r0 + rb) * ldx, ldx, sX);
      }
      const int below = n - R0 - RB;
      if (below > 0)
        gmx<T>(c, nk, OP_N, OP_N, below, ncols, RB, -1.0, L + (size_t)(R0 + RB) * ldl + R0, ldl, sL,
               X + (size_t)R0 * ldx, ldx, sX, 1.0, X + (size_t)(R0 + RB) * ldx, ldx, sX);
    }
    return;
  }
  for (int ob = nob - 1; ob >= 0; ob--) {
    const int R0 = ob * nbb, RB = std::min(nbb, n - R0);
    const int nib = (RB + NB - 1) / NB;
    for (int ib = nib - 1; ib >= 0; ib--) {
      const int r0 = R0 + ib * NB, rb = std::min(NB, R0 + RB - r0);
      T* Xi = X + (size_t)r0 * ldx;
      {
        Rec r(c, PC_TRSM, fl * rb * rb * ncols * nk, (2.0 * ncols * rb + 0.5 * rb * rb) * by * nk);
        trsm_block<T>(TRSM_LEFT_CONJ, L + (size_t)r0 * ldl + r0, ldl, sL, Xi, ldx, sX, rb, ncols, nk, s);
      }
      if (r0 > R0)
        gmx<T>(c, nk, OP_C, OP_N, r0 - R0, ncols, rb, -1.0, L + (size_t)r0 * ldl + R0, ldl, sL, Xi, ldx, sX, 1.0,
               X + (size_t)R0 * ldx, ldx, sX);
    }
    if (R0 > 0)
      gmx<T>(c, nk, OP_C, OP_N, R0, ncols, RB, -1.0, L + (size_t)R0 * ldl, ldl, sL, X + (size_t)R0 * ldx, ldx, sX, 1.0,
             X, ldx, sX);
  }
}

// X <- X L^-H for the rows x n block X (ldx, sX) and the lower n x n factor L (ldl, sL):
// column blocks left to right, X_j = (X_j - X_<j L[j,<j]^H) L[j,j]^-H, with the updates
// from earlier outer blocks of nbb columns applied as one K = nbb product each.
template <typename T>
void trsm_right_conj_run(gks_ctx* c, const T* L, int ldl, long long sL, T* X, int ldx, long long sX, int rows, int n,
                         int nk) {
  cudaStream_t s = c->stream;
  const int es = sizeof(T);
  const int nbb = c->nbb;
  for (int J0 = 0; J0 < n; J0 += nbb) {
    const int JB = std::min(nbb, n - J0);
    for (int j0 = J0; j0 < J0 + JB; j0 += NB) {
      const int jb = std::min(NB, J0 + JB - j0);
      if (j0 > J0)
        gmx<T>(c, nk, OP_N, OP_C, rows, jb, j0 - J0, -1.0, X + J0, ldx, sX, L + (size_t)j0 * ldl + J0, ldl, sL, 1.0,
               X + j0, ldx, sX);
      Rec r(c, PC_TRSM, cmul(es) * 0.5 * jb * jb * rows * nk, (2.0 * rows * jb + 0.5 * jb * jb) * es * nk);
      trsm_block<T>(TRSM_RIGHT_CONJ, L + (size_t)j0 * ldl + j0, ldl, sL, X + j0, ldx, sX, jb, rows, nk, s);
    }
    const int right = n - J0 - JB;
    if (right > 0)
      gmx<T>(c, nk, OP_N, OP_C, rows, right, JB, -1.0, X + J0, ldx, sX, L + (size_t)(J0 + JB) * ldl + J0, ldl, sL,
             1.0, X + J0 + JB, ldx, sX);
  }
}

// Two-sided blocked reduction A <- L^-1 A L^-H (lower triangle) of the order-n block at
// A (lda, sA) with L (ldl, sL), one level of 64-wide panels.  Per panel:
//   A11 <- L11^-1 A11 L11^-H (in-block recurrence),  W = A21 L11^-H,
//   V = W - L21 A11'/2,  A22 -= L21 V^H + V L21^H,  R = V - L21 A11'/2,
// and finally the block-strictly-lower part G = [R_0 R_1 ...] becomes L^-1 G by block
// forward substitution (diagonal blocks by substitution, the rest GEMM updates).
template <typename T>
void hegst_level(gks_ctx* c, T* A, int lda, long long sA, const T* L, int ldl, long long sL, int n, int nk) {
  cudaStream_t s = c->stream;
  const int es = sizeof(T);
  T* F = at<T>(c, c->oF);
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int kb = std::min(NB, n - k0);
    {
      Rec r(c, PC_HEGST_DIAG, cmul(es) * kb * kb * kb * nk, 3.0 * es * kb * kb * nk);
      hegst_diag<T>(A, lda, sA, L, ldl, sL, k0, kb, F, NB, c->sF, nk, s);
    }
    const int rows = n - k0 - kb;
    if (rows <= 0) continue;
    const T* L11 = L + (size_t)k0 * ldl + k0;
    const T* L21 = L + (size_t)(k0 + kb) * ldl + k0;
    T* A21 = A + (size_t)(k0 + kb) * lda + k0;
    T* A22 = A21 + kb;
    {
      Rec r(c, PC_TRSM, cmul(es) * 0.5 * kb * kb * rows * nk, (2.0 * rows * kb + 0.5 * kb * kb) * es * nk);
      trsm_block<T>(TRSM_RIGHT_CONJ, L11, ldl, sL, A21, lda, sA, kb, rows, nk, s);
    }
    gmp<T>(c, nk, OP_N, OP_N, rows, kb, kb, -0.5, L21, ldl, sL, F, NB, c->sF, 1.0, A21, lda, sA);
    gmx<T>(c, nk, OP_N, OP_C, rows, rows, kb, -1.0, L21, ldl, sL, A21, lda, sA, 1.0, A22, lda, sA, 1);
    gmx<T>(c, nk, OP_N, OP_C, rows, rows, kb, -1.0, A21, lda, sA, L21, ldl, sL, 1.0, A22, lda, sA, 1);
    gmp<T>(c, nk, OP_N, OP_N, rows, kb, kb, -0.5, L21, ldl, sL, F, NB, c->sF, 1.0, A21, lda, sA);
  }
  for (int r0 = NB; r0 < n; r0 += NB) {
    const int rb = std::min(NB, n - r0);
    T* Ai = A + (size_t)r0 * lda;
    {
      Rec r(c, PC_TRSM, cmul(es) * 0.5 * rb * rb * r0 * nk, (2.0 * r0 * rb + 0.5 * rb * rb) * es * nk);
      trsm_block<T>(TRSM_LEFT, L + (size_t)r0 * ldl + r0, ldl, sL, Ai, lda, sA, rb, r0, nk, s);
    }
    const int below = n - r0 - rb;
    if (below > 0)
      gmx<T>(c, nk, OP_N, OP_N, below, r0, rb, -1.0, L + (size_t)(r0 + rb) * ldl + r0, ldl, sL, Ai, lda, sA, 1.0,
             A + (size_t)(r0 + rb) * lda, lda, sA);
  }
}

// The same reduction with outer panels of nbb columns: the diagonal nbb block by
// hegst_level, then the panel steps with K = nbb products (A21 L11^-H by 64-wide block
// substitution, the Hermitian A11' as a full copy for the two half-updates, the rank-2nbb
// trailing update), and the deferred substitution L^-1 [R_0 R_1 ...] blocked the same way.
template <typename T>
void hegst_run(gks_ctx* c, T* A, int lda, long long sA, const T* L, int ldl, long long sL, int n, int nk) {
  cudaStream_t s = c->stream;
  const int es = sizeof(T);
  const int nbb = c->nbb;
  if (n <= nbb || nbb <= NB) {
    hegst_level<T>(c, A, lda, sA, L, ldl, sL, n, nk);
    return;
  }
  T* FB = at<T>(c, c->oFB);
  for (int K0 = 0; K0 < n; K0 += nbb) {
    const int KB = std::min(nbb, n - K0);
    T* A11 = A + (size_t)K0 * lda + K0;
    const T* L11 = L + (size_t)K0 * ldl + K0;
    hegst_level<T>(c, A11, lda, sA, L11, ldl, sL, KB, nk);
    const int rows = n - K0 - KB;
    if (rows <= 0) continue;
    const T* L21 = L + (size_t)(K0 + KB) * ldl + K0;
    T* A21 = A + (size_t)(K0 + KB) * lda + K0;
    T* A22 = A21 + KB;
    // A21 <- A21 L11^-H: column blocks left to right, X_j = (A_j - X_<j L11[j,<j]^H) L11[j,j]^-H
    for (int j0 = 0; j0 < KB; j0 += NB) {
      const int jb = std::min(NB, KB - j0);
      if (j0 > 0)
        gmx<T>(c, nk, OP_N, OP_C, rows, jb, j0, -1.0, A21, lda, sA, L11 + (size_t)j0 * ldl, ldl, sL, 1.0, A21 + j0,
               lda, sA);
      Rec r(c, PC_TRSM, cmul(es) * 0.5 * jb * jb * rows * nk, (2.0 * rows * jb + 0.5 * jb * jb) * es * nk);
      trsm_block<T>(TRSM_RIGHT_CONJ, L11 + (size_t)j0 * ldl + j0, ldl, sL, A21 + j0, lda, sA, jb, rows, nk, s);
    }
    {
      Rec r(c, PC_MISC);
      copy2d<T>(FB, nbb, c->sFB, A11, lda, sA, KB, KB, nk, s);
      mirror_lower<T>(FB, nbb, c->sFB, KB, nk, s);
    }
    gmx<T>(c, nk, OP_N, OP_N, rows, KB, KB, -0.5, L21, ldl, sL, FB, nbb, c->sFB, 1.0, A21, lda, sA);
    gmx<T>(c, nk, OP_N, OP_C, rows, rows, KB, -1.0, L21, ldl, sL, A21, lda, sA, 1.0, A22, lda, sA, 1);
    gmx<T>(c, nk, OP_N, OP_C, rows, rows, KB, -1.0, A21, lda, sA, L21, ldl, sL, 1.0, A22, lda, sA, 1);
    gmx<T>(c, nk, OP_N, OP_N, rows, KB, KB, -0.5, L21, ldl, sL, FB, nbb, c->sFB, 1.0, A21, lda, sA);
  }
  // deferred substitution over the outer-block-strictly-lower part
  for (int R0 = nbb; R0 < n; R0 += nbb) {
    const int RB = std::min(nbb, n - R0);
    for (int r0 = R0; r0 < R0 + RB; r0 += NB) {
      const int rb = std::min(NB, R0 + RB - r0);
      T* Ai = A + (size_t)r0 * lda;
      {
        Rec r(c, PC_TRSM, cmul(es) * 0.5 * rb * rb * R0 * nk, (2.0 * R0 * rb + 0.5 * rb * rb) * es * nk);
        trsm_block<T>(TRSM_LEFT, L + (size_t)r0 * ldl + r0, ldl, sL, Ai, lda, sA, rb, R0, nk, s);
      }
      const int below = R0 + RB - r0 - rb;
      if (below > 0)
        gmx<T>(c, nk, OP_N, OP_N, below, R0, rb, -1.0, L + (size_t)(r0 + rb) * ldl + r0, ldl, sL, Ai, lda, sA, 1.0,
               A + (size_t)(r0 + rb) * lda, lda, sA);
    }
    const int below = n - R0 - RB;
    if (below > 0)
      gmx<T>(c, nk, OP_N, OP_N, below, R0, RB, -1.0, L + (size_t)(R0 + RB) * ldl + R0, ldl, sL,
             A + (size_t)R0 * lda, lda, sA, 1.0, A + (size_t)(R0 + RB) * lda, lda, sA);
  }
}

// One-stage Householder tridiagonalization, steps j = M-1 .. 2, in panels of nbb steps.
// Each step is two launches (the Hermitian product over the stale trailing block with the
// panel's corrections, then q, the panel buffers and the next row); each panel ends with
// the deferred update A[0:j,0:j] -= U Q^H + Q U^H as two lower-triangle GEMMs with K = the
// panel's step count.
template <typename T>
void hetrd_run(gks_ctx* c, T* A, int M, int nk) {
  cudaStream_t s = c->stream;
  const int es = sizeof(T);
  const int ldu = c->nbb;
  T* u = at<T>(c, c->ou);
  T* p = at<T>(c, c->op);
  T* U = at<T>(c, c->oU);
  T* Q = at<T>(c, c->oQ);
  T* part = at<T>(c, c->opart);
  T* y = at<T>(c, c->oy);
  double* tau = at<double>(c, c->otau);
  int* tk = at<int>(c, c->oticket);
  if (M < 3) return;
  cudaMemsetAsync(tk, 0, sizeof(int) * 2 * nk, s);
  // panels of at most 128 steps: the per-step corrections grow with the panel length, the
  // deferred update runs fine at K = 128; small orders are latency-bound per step (64)
  const int pw = M < 2048 ? std::min(NB, ldu) : std::min(2 * NB, ldu);
  // digit form of the matrix-vector step (FP64 types): digits of the stale block per panel;
  // else, complex: three-multiplication products need Re + Im of the stale block (per panel)
  HemvDigits hdv{};
  const HemvDigits* hd = nullptr;
  if constexpr (std::is_same<T, double>::value || std::is_same<T, zc>::value) {
    if (c->wsdig) {
      const int ldd = (M + 15) / 16 * 16, npl = es == 16 ? 14 : 7;
      hdv.D = at<signed char>(c, c->oD);
      hdv.sD = (long long)((ldd + 31) / 32 * 32) * ldd * npl;
      hdv.ldd = ldd;
      hdv.ud = at<signed char>(c, c->oud);
      hdv.sud = (long long)ldd * npl;
      hdv.fu = at<int>(c, c->ofu);
      hdv.rmax = at<unsigned long long>(c, c->ormax);
      hd = &hdv;
    }
  }
  double* uw = es == 16 && !hd ? at<double>(c, c->ouw) : nullptr;
  double* Sg = es == 16 && !hd ? at<double>(c, c->oSg) : nullptr;
  const double npl = es == 16 ? 14.0 : 7.0;
  for (int jh = M - 1; jh >= 2; jh -= pw) {
    const int jl = std::max(2, jh - pw + 1);  // steps jh .. jl in this panel
    {
      Rec r(c, PC_HETRD_VEC, 0.0, (hd ? 0.5 * es + npl : 2.0 * es) * jh * (hd ? jh : 1) * nk);
      if (hd) hetrd_digits<T>(A, M, c->sMM, jh, hdv, nk, s);
      else if (Sg) hetrd_sums(reinterpret_cast<const zc*>(A), M, c->sMM, jh, Sg, nk, s);
      hetrd_reflector<T>(A, M, c->sMM, jh, u, c->sVec, tau, M, nk, s, uw, hd);
    }
    for (int j = jh; j >= jl; j--) {
      const int k = jh - j;  // panel steps already taken
      const double jj = (double)j * j;
      {
        // algorithmic bytes: the digit planes of the j x j block (full matrix), or the
        // lower triangle (and Re + Im sums) in FP64
        Rec r(c, PC_HETRD_HEMV, cmul(es) * (jj + 2.0 * j * k) * nk,
              ((hd ? jj * npl : 0.5 * jj * (es == 16 ? 1.5 : 1.0) * es) + (2.0 * j * k + 4.0 * j) * es) * nk);
        hetrd_phemv<T>(A, M, c->sMM, j, u, p, c->sVec, tau, M, U, Q, ldu, c->sU, k, part, c->spart, y, c->sy, tk,
                       nk, s, Sg, uw, hd);
      }
      const int rowupd = (j > jl) ? 1 : 0;
      {
        Rec r(c, PC_HETRD_RANK2, cmul(es) * 2.0 * j * (k + 1) * (1 + rowupd) * nk, (2.0 * j * (k + 1) + 4.0 * j) * es * nk);
        hetrd_pupdate<T>(A, M, c->sMM, j, u, p, c->sVec, tau, M, U, Q, ldu, c->sU, k, y, c->sy, rowupd, tk + nk, nk,
                         s, uw, hd);
      }
    }
    // deferred rank-2k update of the trailing block [0:jl, 0:jl]
    const int kp = jh - jl + 1;
    gmx<T>(c, nk, OP_N, OP_C, jl, jl, kp, -1.0, U, ldu, c->sU, Q, ldu, c->sU, 1.0, A, M, c->sMM, 1);
    gmx<T>(c, nk, OP_N, OP_C, jl, jl, kp, -1.0, Q, ldu, c->sU, U, ldu, c->sU, 1.0, A, M, c->sMM, 1);
  }
}

// ---- two-stage tridiagonalization (sbr.cu) ----

// (a3) Dense -> band, bandwidth b = c->band, for the Hermitian A (lower triangle in, made
// full here; full storage kept up to date for the products).  Panel p (columns k = p b ..)
// leaves R in the band, its reflectors below the band, taus in tau1, T factor in T1[p].
template <typename T>
void he2hb_run(gks_ctx* c, T* A, int M, int items) {
  cudaStream_t s = c->stream;
  const int b = c->band, b2 = 2 * b;
  const long long MM = c->sMM, sP = (long long)M * b2, sX = (long long)M * b, sb = (long long)b * b;
  const long long stau = (long long)M + b, sT1 = (long long)(M / b + 2) * b * b;
  T* tau1 = at<T>(c, c->otau1);
  T* T1 = at<T>(c, c->oT1);
  T* P1 = at<T>(c, c->oP1);
  T* P2 = at<T>(c, c->oP2);
  T* VT = at<T>(c, c->oVT);
  T* Xb = at<T>(c, c->oXb);
  T* Gb = at<T>(c, c->oGb);
  T* Yb = at<T>(c, c->oYb);
  T* Zb = at<T>(c, c->oZb);
  {
    Rec r(c, PC_MISC);
    mirror_lower<T>(A, M, MM, M, items, s);
  }
  for (int k = 0, p = 0; k < M - b - 1; k += b, p++) {
    const int r0 = k + b, kb = std::min(b, M - b - 1 - k), m = M - r0;
    T* A22 = A + (size_t)r0 * M + r0;
    T* Tp = T1 + (size_t)p * b * b;
    {
      Rec r(c, PC_HETRD_VEC, 0.0, 2.0 * sizeof(T) * (double)m * b * kb * items);
      panel_qr<T>(A, M, MM, r0, k, m, b, kb, tau1 + (size_t)p * b, stau, items, at<char>(c, c->oqr), c->st,
                  c->wait_cycles, s);
      panel_v<T>(A, M, MM, r0, k, m, kb, P1, b2, sP, items, s);
    }
    gmx<T>(c, items, OP_C, OP_N, kb, kb, m, 1.0, P1, b2, sP, P1, b2, sP, 0.0, Gb, b, sb);  // G = V^H V
    {
      Rec r(c, PC_BACKTR_AUX);
      larft_tau<T>(Gb, b, sb, tau1 + (size_t)p * b, stau, kb, Tp, b, sT1, items, s);
    }
    gmx<T>(c, items, OP_N, OP_N, m, kb, kb, 1.0, P1, b2, sP, Tp, b, sT1, 0.0, VT, b, sX);        // V T
    gmx<T>(c, items, OP_N, OP_N, m, kb, m, 1.0, A22, M, MM, VT, b, sX, 0.0, Xb, b, sX);         // X = A22 V T
    gmx<T>(c, items, OP_C, OP_N, kb, kb, m, 1.0, P1, b2, sP, Xb, b, sX, 0.0, Yb, b, sb);        // V^H X
    gmx<T>(c, items, OP_C, OP_N, kb, kb, kb, 1.0, Tp, b, sT1, Yb, b, sb, 0.0, Zb, b, sb);       // T^H V^H X
    gmx<T>(c, items, OP_N, OP_N, m, kb, kb, -0.5, P1, b2, sP, Zb, b, sb, 1.0, Xb, b, sX);       // W
    {
      Rec r(c, PC_MISC);  // P1 = [V W], P2 = [W V] (kb columns each)
      copy2d<T>(P1 + kb, b2, sP, Xb, b, sX, m, kb, items, s);
      copy2d<T>(P2, b2, sP, Xb, b, sX, m, kb, items, s);
      copy2d<T>(P2 + kb, b2, sP, P1, b2, sP, m, kb, items, s);
    }
    // A22 -= V W^H + W V^H = [V W] [W V]^H (lower triangle), then made full again
    gmx<T>(c, items, OP_N, OP_C, m, m, 2 * kb, -1.0, P1, b2, sP, P2, b2, sP, 1.0, A22, M, MM, 1);
    Rec r(c, PC_MISC);
    mirror_lower<T>(A22, M, MM, m, items, s);
  }
}

// (a4) Band -> tridiagonal by bulge chasing: the band of A (d <= b below the diagonal) into
// the band storage, the persistent chase, then d and e (real).  False if the cooperative
// launch was refused.
template <typename T>
bool hb2st_run(gks_ctx* c, const T* A, int M, int items, double* d, double* e) {
  cudaStream_t s = c->stream;
  const int b = c->band, W = 2 * b + 1;
  const long long sB = (long long)M * W;
  T* Bd = at<T>(c, c->oBd);
  {
    Rec r(c, PC_MISC);
    band_pack<T>(A, M, c->sMM, Bd, W, sB, M, b, items, s);
  }
  const int workers = chase_workers<T>(b, items, 64);
  {
    const double tasks = 0.5 * (double)M * M / b;
    Rec r(c, PC_HETRD_RANK2, cmul(sizeof(T)) * 8.0 * b * b * tasks * items, sizeof(T) * 6.0 * b * b * tasks * items);
    if (!chase<T>(Bd, W, sB, M, b, at<T>(c, c->oV2), c->sMM, at<T>(c, c->otau2), c->ldt2, (long long)M * c->ldt2,
                  at<int>(c, c->oprog), M, at<int>(c, c->oerr), c->st, c->wait_cycles, items, workers, s)) {
      cudaGetLastError();
      return false;
    }
  }
  Rec r(c, PC_HETRD_VEC);
  band_tridiag<T>(Bd, W, sB, M, d, e, M, items, s);
  return true;
}

// X <- Q2 X for the padded Xp (rows M + 2b, ncols columns, ld ncols): the chase's
// reflectors in compact-WY blocks of b consecutive sweeps x one window, applied wavefront
// by wavefront (blocks of one wavefront touch disjoint rows; see sbr.cu), each wavefront as
// three two-level batched products over items x blocks.
template <typename T>
void q2_apply_run(gks_ctx* c, T* Xp, long long sXp, int M, int ncols, int items) {
  cudaStream_t s = c->stream;
  const int b = c->band, nbs = b, hp = 2 * b;
  const int nsweep = M - 1;
  if (nsweep < 1) return;
  const int G = (nsweep + nbs - 1) / nbs;
  auto J = [&](int g) { return (M - 2 - g * nbs) / b + 1; };  // windows of the group's first sweep
  T* Vw = at<T>(c, c->oVw);
  T* tw = at<T>(c, c->otw);
  T* Gw = at<T>(c, c->oGw);
  T* Tw = at<T>(c, c->oTw);
  T* Yw = at<T>(c, c->oYw);
  T* Y2w = at<T>(c, c->oY2w);
  for (int t = 0;; t++) {
    const int g_lo = std::max(0, (2 * (G - 1) - t + 1) / 2);
    int nblk = 0;
    for (int g = g_lo; g < G; g++) {
      const int j = t - 2 * (G - 1 - g);
      if (j < 0 || j >= J(g)) break;
      nblk++;
    }
    if (nblk == 0) {
      if (g_lo == 0) break;
      continue;
    }
    nblk = std::min(nblk, c->nblkmax);
    const int j0 = t - 2 * (G - 1 - g_lo);
    const long long top0 = (long long)g_lo * nbs + 1 + (long long)j0 * b;
    const int cnt = items * nblk;
    {
      Rec r(c, PC_BACKTR_AUX);
      q2_gather<T>(at<T>(c, c->oV2), c->sMM, at<T>(c, c->otau2), c->ldt2, (long long)M * c->ldt2, M, b, nbs, hp, g_lo,
                   j0, nblk, Vw, tw, items, s);
    }
    gmx<T>(c, cnt, OP_C, OP_N, nbs, nbs, hp, 1.0, Vw, nbs, (long long)hp * nbs, Vw, nbs, (long long)hp * nbs, 0.0,
           Gw, nbs, (long long)nbs * nbs);
    {
      Rec r(c, PC_BACKTR_AUX);
      larft_tau<T>(Gw, nbs, (long long)nbs * nbs, tw, nbs, nbs, Tw, nbs, (long long)nbs * nbs, cnt, s);
    }
    T* X0 = Xp + top0 * ncols;
    const long long s3 = 3LL * b * ncols;  // row step between the blocks of a wavefront
    gmx2<T>(c, cnt, nblk, OP_C, OP_N, ncols, nbs, hp, 1.0, X0, ncols, sXp, s3, Vw, nbs,
            (long long)nblk * hp * nbs, (long long)hp * nbs, 0.0, Yw, nbs, (long long)nblk * ncols * nbs,
            (long long)ncols * nbs);                                                          // Yh = X^H V
    gmx<T>(c, cnt, OP_N, OP_C, ncols, nbs, nbs, 1.0, Yw, nbs, (long long)ncols * nbs, Tw, nbs, (long long)nbs * nbs,
           0.0, Y2w, nbs, (long long)ncols * nbs);                                            // Yh T^H
    gmx2<T>(c, cnt, nblk, OP_N, OP_C, hp, ncols, nbs, -1.0, Vw, nbs, (long long)nblk * hp * nbs,
            (long long)hp * nbs, Y2w, nbs, (long long)nblk * ncols * nbs, (long long)ncols * nbs, 1.0, X0, ncols, sXp,
            s3);                                                                              // X -= V Y
  }
}

// X <- Q1 X (X: M x ncols, ldx, sX): the panels' compact-WY factors, last panel first.
template <typename T>
void q1_apply_run(gks_ctx* c, const T* A, T* X, int ldx, long long sX, int M, int ncols, int items) {
  cudaStream_t s = c->stream;
  const int b = c->band, b2 = 2 * b;
  const long long sP = (long long)M * b2, sT1 = (long long)(M / b + 2) * b * b;
  T* P1 = at<T>(c, c->oP1);
  T* T1 = at<T>(c, c->oT1);
  T* Yw = at<T>(c, c->oYw);
  T* Y2w = at<T>(c, c->oY2w);
  const long long sY = (long long)ncols * b;
  int np = 0;
  for (int k = 0; k < M - b - 1; k += b) np++;
  for (int p = np - 1; p >= 0; p--) {
    const int k = p * b, r0 = k + b, kb = std::min(b, M - b - 1 - k), m = M - r0;
    {
      Rec r(c, PC_BACKTR_AUX);
      panel_v<T>(A, M, c->sMM, r0, k, m, kb, P1, b2, sP, items, s);
    }
    T* Xr = X + (size_t)r0 * ldx;
    gmx<T>(c, items, OP_C, OP_N, ncols, kb, m, 1.0, Xr, ldx, sX, P1, b2, sP, 0.0, Yw, b, sY);        // X^H V
    gmx<T>(c, items, OP_N, OP_C, ncols, kb, kb, 1.0, Yw, b, sY, T1 + (size_t)p * b * b, b, sT1, 0.0, Y2w, b, sY);
    gmx<T>(c, items, OP_N, OP_C, m, ncols, kb, -1.0, P1, b2, sP, Y2w, b, sY, 1.0, Xr, ldx, sX);     // X -= V Y
  }
}

// X <- Q X with Q = P_{M-1} ... P_2 (reflectors stored by the reduction), compact WY in
// blocks of nbb reflectors: B = I - V T V^H.  X is M x ncols (ldx, sX).  T (upper
// triangular) is assembled from the 64-wide diagonal blocks (larft on G = V^H V) by the merge
//   T[:s, s:s+k] = -T[:s, :s] G[:s, s:s+k] T[s:s+k, s:s+k].
template <typename T, typename TA = T>
void backtransform_run(gks_ctx* c, const TA* A, T* X, int ldx, long long sX, int M, int ncols, int nk) {
  cudaStream_t s = c->stream;
  const int nbb = c->nbb;
  T* V = at<T>(c, c->oV);
  T* G = at<T>(c, c->oG);
  T* Tm = at<T>(c, c->oT);
  T* Y = at<T>(c, c->oY);
  T* Y2 = at<T>(c, c->oY2);
  double* tau = at<double>(c, c->otau);
  double* tb = at<double>(c, c->otb);
  if (M < 3) return;
  cudaMemsetAsync(Tm, 0, sizeof(T) * (size_t)c->sT * nk, s);
  for (int j0 = 2; j0 <= M - 1; j0 += nbb) {
    const int j1 = std::min(j0 + nbb - 1, M - 1), nbk = j1 - j0 + 1;
    {
      Rec r(c, PC_BACKTR_AUX);
      gather_reflectors<TA, T>(A, M, c->sMM, tau, M, j0, j1, V, nbb, c->sV, tb, nbb, nk, s);
    }
    gmx<T>(c, nk, OP_C, OP_N, nbk, nbk, j1, 1.0, V, nbb, c->sV, V, nbb, c->sV, 0.0, G, nbb, c->sG);
    for (int s0 = 0; s0 < nbk; s0 += NB) {
      const int ks = std::min(NB, nbk - s0);
      {
        Rec r(c, PC_BACKTR_AUX);
        larft<T>(G + (size_t)s0 * nbb + s0, nbb, c->sG, tb + s0, nbb, ks, Tm + (size_t)s0 * nbb + s0, nbb, c->sT,
                 nk, s);
      }
      if (s0 > 0) {
        // P = G[:s0, s0:s0+ks] T_ss (P in Y2, ld NB), then T[:s0, s0:s0+ks] = -T[:s0, :s0] P
        gmp<T>(c, nk, OP_N, OP_N, s0, ks, ks, 1.0, G + s0, nbb, c->sG, Tm + (size_t)s0 * nbb + s0, nbb, c->sT, 0.0,
               Y2, NB, c->sY);
        gmp<T>(c, nk, OP_N, OP_N, s0, ks, s0, -1.0, Tm, nbb, c->sT, Y2, NB, c->sY, 0.0, Tm + s0, nbb, c->sT);
      }
    }
    gmx<T>(c, nk, OP_C, OP_N, nbk, ncols, j1, 1.0, V, nbb, c->sV, X, ldx, sX, 0.0, Y, ncols, c->sY);
    gmx<T>(c, nk, OP_N, OP_N, nbk, ncols, nbk, 1.0, Tm, nbb, c->sT, Y, ncols, c->sY, 0.0, Y2, ncols, c->sY);
    gmx<T>(c, nk, OP_N, OP_N, j1, ncols, nbk, -1.0, V, nbb, c->sV, Y2, ncols, c->sY, 1.0, X, ldx, sX);
  }
}

// All eigenpairs of the standard Hermitian problems in A (lower triangle, order M, items;
// destroyed): w (M per item, ascending) and X (M x M, ldx M, stride sX) with the FP64 stages
// of the main path (Householder, divide and conquer, back-transform).
template <typename T>
void standard_eig(gks_ctx* c, T* A, T* X, long long sX, double* w, int M, int items) {
  cudaStream_t s = c->stream;
  double* d = at<double>(c, c->od);
  double* e = at<double>(c, c->oe);
  T* ph = at<T>(c, c->oph);
  hetrd_run<T>(c, A, M, items);
  {
    Rec r(c, PC_HETRD_VEC);
    hetrd_finish<T>(A, M, c->sMM, M, d, e, M, ph, M, items, s);
  }
  double* Z = at<double>(c, c->oZ);
  DcSplit sp{nullptr, 0, sform(c), 512, c->wait_cycles};
  if (c->gemm_mode != 1 && M >= 1024) {
    const size_t item = dc_split_item_bytes(c->dc, sp.min_half, sform(c));
    if (item > 0) {
      sp.per = oz_reserve(c, item, items);
      sp.work = c->oz;
    }
  }
  dc_solve(c->dc, d, e, M, w, Z, c->sMM, c->ws + c->odc, c->st, s, &c->prof, &sp);
  {
    Rec r(c, PC_MISC);
    apply_phase<T>(X, M, sX, Z, M, c->sMM, ph, M, M, M, items, s);
  }
  backtransform_run<T>(c, A, X, M, sX, M, M, items);
}

// Ogita-Aishima sweeps (refine.cu) on X (C, order M, all columns) for the standard problem
// H' (lower triangle in A, made full here): each sweep Y = H' X, T = X^H Y, G = X^H X as
// FP64-accurate products (the context's digit count), the correction E, X <- X + X E.  lam
// receives the refined eigenvalues in ascending order; per sweep and item the bounds of
// ||R|| and ||T - diag(l)|| go to the statistics buffer (gks_refine_stats).
template <typename T>
void refine_run(gks_ctx* c, T* A, T* X, int M, int items, double* lam) {
  cudaStream_t s = c->stream;
  const long long MM = c->sMM;
  T* Y = at<T>(c, c->oRY);
  T* Tm = at<T>(c, c->oRT);
  T* G = at<T>(c, c->oRR);
  double* nrm = at<double>(c, c->onrm);
  double* rst = at<double>(c, c->orstat);
  {
    Rec r(c, PC_MISC);
    mirror_lower<T>(A, M, MM, M, items, s);
  }
  T* Xc = X;
  T* Xo = Y;
  const int sweeps = std::min(kMaxSweeps, std::max(1, c->refine_sweeps));
  for (int sw = 0; sw < sweeps; sw++) {
    gmx<T>(c, items, OP_N, OP_N, M, M, M, 1.0, A, M, MM, Xc, M, MM, 0.0, Xo, M, MM);        // Y = H' X
    gmx<T>(c, items, OP_C, OP_N, M, M, M, 1.0, Xc, M, MM, Xo, M, MM, 0.0, Tm, M, MM, 1);    // T = X^H Y
    gmx<T>(c, items, OP_C, OP_N, M, M, M, 1.0, Xc, M, MM, Xc, M, MM, 0.0, G, M, MM, 1);     // G = X^H X
    {
      Rec r(c, PC_MISC);
      mirror_lower<T>(Tm, M, MM, M, items, s);
      mirror_lower<T>(G, M, MM, M, items, s);
      oa_prepare<T>(Tm, G, MM, M, lam, nrm, items, s);
      // statistics: (||R|| bound, ||T - diag(l)|| bound) per item for this sweep
      cudaMemcpy2DAsync(rst + (size_t)sw * 2 * items, 2 * sizeof(double), nrm + 1, 3 * sizeof(double),
                        sizeof(double), items, cudaMemcpyDeviceToDevice, s);
      cudaMemcpy2DAsync(rst + (size_t)sw * 2 * items + 1, 2 * sizeof(double), nrm, 3 * sizeof(double),
                        sizeof(double), items, cudaMemcpyDeviceToDevice, s);
      oa_correction<T>(Tm, G, MM, M, lam, nrm, items, s);
      copy2d<T>(Xo, M, MM, Xc, M, MM, M, M, items, s);
    }
    gmx<T>(c, items, OP_N, OP_N, M, M, M, 1.0, Xc, M, MM, Tm, M, MM, 1.0, Xo, M, MM);       // X + X E
    std::swap(Xc, Xo);
  }
  Rec r(c, PC_MISC);
  if (Xc != X) copy2d<T>(X, M, MM, Xc, M, MM, M, M, items, s);
  oa_order<T>(lam, X, Y, MM, M, at<int>(c, c->operm), at<int>(c, c->oflag), items, s);
  c->rstat_sweeps = sweeps;
  c->rstat_items = items;
}

// Does the context still hold the Cholesky factor of this S (same array, shape and type
// as the solve that produced it)?
bool factor_matches(const gks_ctx* c, const SolveKey& k) {
  return c->l_valid && c->lkey.S == k.S && c->lkey.n == k.n && c->lkey.nk == k.nk && c->lkey.dtype == k.dtype &&
         c->lkey.spin == k.spin;
}

template <typename T>
gks_status solve_t(gks_ctx* c, const SolveKey& key) {
  const T* H = static_cast<const T*>(key.H);
  const T* S = static_cast<const T*>(key.S);
  const int n = (int)key.n, nk = (int)key.nk;
  const bool nc = key.spin == GKS_NONCOLLINEAR, sp = key.spin == GKS_SPIN_POLARIZED;
  const int M = nc ? 2 * n : n;
  const int items = sp ? 2 * nk : nk;  // spin-polarized: items (k, up), (k, down)
  const int es = sizeof(T);
  const int nev = ncols_of(c, M);
  gks_status rc = ensure_ws(c, M, n, items, es, key.spin);
  if (rc) return rc;
  cudaStream_t s = c->stream;
  double* eps = static_cast<double*>(const_cast<void*>(key.eps));
  T* C = static_cast<T*>(const_cast<void*>(key.C));
  const long long sC = (long long)M * nev;
  T* A = at<T>(c, c->oA);
  T* L = at<T>(c, c->oL);
  // The factor of S: n x n with leading dimension n in every item's L slot.  Noncollinear:
  // S_NC = I_2 (x) S, so only the n x n S is factored (paper Sec. 3.2).  Spin-polarized:
  // both spin channels of a k-point share S_k; it is factored once into the slot of the
  // up channel and copied to the down channel's.
  const long long sLk = sp ? 2 * c->sMM : c->sMM;
  const bool reuse = (key.flags & GKS_REUSE_S_FACTOR) && factor_matches(c, key);
  {
    StageRec sr(c, PS_COPY);
    Rec r(c, PC_MISC);
    cudaMemsetAsync(c->st, 0, sizeof(DevStatus) * items, s);
    copy2d<T>(A, M, c->sMM, H, M, (long long)M * M, M, M, items, s);
    if (!reuse) copy2d<T>(L, n, sLk, S, n, (long long)n * n, n, n, nk, s);
  }
  const bool lowdin = c->reduction == GKS_REDUCE_LOWDIN;
  // (a1) Cholesky of S, (a2) reduction to the standard problem
  if (!reuse && lowdin) {
    // Loewdin (paper Sec. 3.1 Parts 2-1, 2-2): S = U diag(s) U^H by the standard eigensolve
    // of this library (S copied to the H' workspace, U in the output C), V = U diag(s)^-1/2
    // kept in the factor slots
    c->l_valid = false;
    StageRec sr(c, PS_POTRF);
    {
      Rec r(c, PC_MISC);
      copy2d<T>(A, M, sLk, S, n, (long long)n * n, n, n, nk, s);
      if (sp) copy2d<T>(A + c->sMM, M, sLk, A, M, sLk, n, n, nk, s);
    }
    standard_eig<T>(c, A, C, sC, eps, M, items);
    {
      Rec r(c, PC_MISC);
      lowdin_factor<T>(C, M, sC, eps, M, L, n, c->sMM, M, c->st, items, s);
    }
    c->lkey = key;
    c->l_valid = true;
    copy2d<T>(A, M, c->sMM, H, M, (long long)M * M, M, M, items, s);  // H again (A held S)
  } else if (!reuse) {
    c->l_valid = false;
    StageRec sr(c, PS_POTRF);
    potrf_run<T>(c, L, n, n, sLk, nk);
    if (sp) {
      Rec r(c, PC_MISC);
      copy2d<T>(L + c->sMM, n, sLk, L, n, sLk, n, n, nk, s);
    }
    c->lkey = key;
    c->l_valid = true;
  }
  {
    StageRec sr(c, PS_HEGST);
    if (lowdin) {
      // H' = V^H H V (paper Sec. 3.1 Part 2-3): H made full, T1 = H V in the output C, the
      // lower triangle of V^H T1 into A
      {
        Rec r(c, PC_MISC);
        mirror_lower<T>(A, M, c->sMM, M, items, s);
      }
      gmx<T>(c, items, OP_N, OP_N, M, M, M, 1.0, A, M, c->sMM, L, n, c->sMM, 0.0, C, M, sC);
      gmx<T>(c, items, OP_C, OP_N, M, M, M, 1.0, L, n, c->sMM, C, M, sC, 0.0, A, M, c->sMM, 1);
    } else if (nc) {
      // H'^{ss'} = L^-1 H^{ss'} L^-H per spin block (paper Sec. 3.2 Part 3-3): the two
      // Hermitian diagonal blocks two-sided, the lower off-diagonal block by a left and a
      // right triangular solve
      hegst_run<T>(c, A, M, c->sMM, L, n, c->sMM, n, nk);
      hegst_run<T>(c, A + (size_t)n * M + n, M, c->sMM, L, n, c->sMM, n, nk);
      trsm_left_run<T>(c, L, n, c->sMM, A + (size_t)n * M, M, c->sMM, n, n, nk, false);
      trsm_right_conj_run<T>(c, L, n, c->sMM, A + (size_t)n * M, M, c->sMM, n, n, nk);
    } else {
      hegst_run<T>(c, A, M, c->sMM, L, n, c->sMM, M, items);
    }
  }
  // (a3-a4) Householder tridiagonalization with a real-making phase
  double* d = at<double>(c, c->od);
  double* e = at<double>(c, c->oe);
  T* ph = at<T>(c, c->oph);
  const bool mixed = c->precision == GKS_MIXED_SPLITBF16;
  const bool two = !mixed && c->tridiag == GKS_TRIDIAG_TWO_STAGE;
  using TL = typename Low<T>::type;
  TL* Af = mixed ? at<TL>(c, c->oAf) : nullptr;
  {
    StageRec sr(c, PS_HETRD);
    if (mixed) {
      // mixed precision: H' rounded to single precision and tridiagonalized on the FP32
      // pipe (FP64 H' stays in A for the refinement)
      {
        Rec r(c, PC_MISC);
        narrow_lower<T, TL>(A, M, c->sMM, Af, M, c->sMM, M, items, s);
      }
      hetrd_run<TL>(c, Af, M, items);
      Rec r(c, PC_HETRD_VEC);
      TL* phl = at<TL>(c, c->ou);
      hetrd_finish<TL>(Af, M, c->sMM, M, d, e, M, phl, M, items, s);
      widen_copy<TL, T>(phl, ph, (long long)M * items, s);
    } else if (two) {
      // (a3) dense -> band, (a4) band -> tridiagonal (real: the chase's betas are real)
      he2hb_run<T>(c, A, M, items);
      if (!hb2st_run<T>(c, A, M, items, d, e))
        return fail(c, GKS_ECUDA, "bulge chasing: cooperative launch refused (not enough resident CTAs)");
    } else {
      hetrd_run<T>(c, A, M, items);
      Rec r(c, PC_HETRD_VEC);
      hetrd_finish<T>(A, M, c->sMM, M, d, e, M, ph, M, items, s);
    }
  }
  // (a5) divide and conquer on the real tridiagonal
  double* Z = at<double>(c, c->oZ);
  {
    StageRec sr(c, PS_STEDC);
    DcSplit sp_{nullptr, 0, sform(c), 512, c->wait_cycles};
    if (c->gemm_mode != 1 && M >= 1024) {
      const size_t item = dc_split_item_bytes(c->dc, sp_.min_half, sform(c));
      if (item > 0) {
        sp_.per = oz_reserve(c, item, items);
        sp_.work = c->oz;
      }
    }
    dc_solve(c->dc, d, e, M, eps, Z, c->sMM, c->ws + c->odc, c->st, s, &c->prof, &sp_);
  }
  // (a6) X = Q D Z (the leading nev columns), C = L^-H X
  {
    StageRec sr(c, PS_BACKTR);
    if (!two) {
      Rec r(c, PC_MISC);
      apply_phase<T>(C, nev, sC, Z, M, c->sMM, ph, M, M, nev, items, s);
    }
    if (two) {
      // X = Q1 Q2 Z: Z into the padded buffer, Q2 there, then Q1 on the output
      T* Xp = at<T>(c, c->oXp);
      const long long sXp = (long long)(M + 2 * c->band) * nev;
      {
        Rec r(c, PC_MISC);
        widen_pad<T>(Z, M, c->sMM, Xp, nev, sXp, M, M + 2 * c->band, nev, items, s);
      }
      q2_apply_run<T>(c, Xp, sXp, M, nev, items);
      {
        Rec r(c, PC_MISC);
        copy2d<T>(C, nev, sC, Xp, nev, sXp, M, nev, items, s);
      }
      q1_apply_run<T>(c, A, C, nev, sC, M, nev, items);
    } else if (mixed) {
      // single-precision reflectors, products on fewer digits (about FP32 accuracy)
      const int sv = c->slices;
      c->slices = std::min(sv, kLowSlices);
      backtransform_run<T, TL>(c, Af, C, nev, sC, M, nev, items);
      c->slices = sv;
    } else {
      backtransform_run<T>(c, A, C, nev, sC, M, nev, items);
    }
  }
  // (a7) mixed precision: Ogita-Aishima refinement of (eps, X) on the FP64 H'
  if (mixed) {
    StageRec sr(c, PS_REFINE);
    refine_run<T>(c, A, C, M, items, eps);
  }
  {
    StageRec sr(c, PS_UNREDUCE);
    if (lowdin) {  // C = V X (paper Sec. 3.1 Part 2-5), through A (free after the back-transform)
      gmx<T>(c, items, OP_N, OP_N, M, M, M, 1.0, L, n, c->sMM, C, M, sC, 0.0, A, M, c->sMM);
      Rec r(c, PC_MISC);
      copy2d<T>(C, M, sC, A, M, c->sMM, M, M, items, s);
    } else if (nc) {  // C = diag(L, L)^-H X: each spin half with the n x n factor
      trsm_left_run<T>(c, L, n, c->sMM, C, nev, sC, n, nev, nk, true);
      trsm_left_run<T>(c, L, n, c->sMM, C + (size_t)n * nev, nev, sC, n, nev, nk, true);
    } else {
      trsm_left_run<T>(c, L, n, c->sMM, C, nev, sC, M, nev, items, true);
    }
    Rec r(c, PC_MISC);
    column_phase<T>(C, nev, sC, M, nev, items, s);
  }
  if (key.flags & GKS_SAVE_FOR_BACKWARD) {
    rc = save_for_backward(c, key, M, items, nev);
    if (rc) return rc;
  }
  if (key.flags & GKS_EIGEN_ONLY) return cuda_check(c, "gks_solve launch");
  // (a8) occupations and chemical potential, (a9) density matrix
  double* occ = at<double>(c, c->oocc);
  double* ks = at<double>(c, c->oks);
  int* nrho = at<int>(c, c->onrho);
  double* w = at<double>(c, c->oweights);
  double* eb = key.eb ? static_cast<double*>(const_cast<void*>(key.eb)) : at<double>(c, c->oeb);
  {
    StageRec sr(c, PS_OCC);
    Rec r(c, PC_OCC);
    expand_weights(static_cast<const double*>(key.kw), nk, sp ? 2 : 1, w, s);
    fermi_mu(eps, M, items, w, nc || sp ? 1.0 : 2.0, key.kT, key.ne, c->f_cut, occ, ks,
             static_cast<double*>(const_cast<void*>(key.mu)), eb, nrho, c->st, 1, s);
    if (nev < M) clamp_nrho(nrho, items, nev, c->st, 1, s);
    if (key.flags & GKS_SAVE_FOR_BACKWARD) save_mu(c, key, M, items, nev);
  }
  {
    StageRec sr(c, PS_RHO);
    T* rho = static_cast<T*>(const_cast<void*>(key.rho));
    {
      const bool split = split_worth(c, items, M, M, nev, es, gemm_flops(es, M, M, std::max(1, nev / 4), 1, items));
      Rec r(c, split ? PC_OZAKI : PC_GEMM, -1.0, -1.0);  // flops resolved from n_rho when the profile is read
      c->prof.nrho_dev = nrho;
      c->prof.rho_m = M;
      c->prof.rho_nk = items;
      c->prof.rho_es = es;
      rho_run<T>(c, C, nev, sC, rho, c->sMM, ks, M, nrho, M, nev, items);
    }
    Rec r(c, PC_MISC);
    mirror_lower<T>(rho, M, c->sMM, M, items, s);
  }
  return cuda_check(c, "gks_solve launch");
}

// Adjoint: W = C^H rho_bar C; weights; BH, BS; H_bar = C BH C^H, S_bar = C BS C^H.
// spin: GKS_COLLINEAR, GKS_NONCOLLINEAR (S_bar = sum of the diagonal spin blocks) or
// GKS_SPIN_POLARIZED (2 nk items with g_s = 1; S_bar_k = sum over the two channels).
template <typename T>
gks_status adjoint_t(gks_ctx* c, const T* C, const double* eps, const double* mu, int n, int nk, int spin, double kT,
                     const double* kw, const T* rho_bar, const double* eps_bar, double e_band_bar, T* H_bar,
                     T* S_bar) {
  const bool nc = spin == GKS_NONCOLLINEAR, sp = spin == GKS_SPIN_POLARIZED;
  const int M = nc ? 2 * n : n;
  const int items = sp ? 2 * nk : nk;
  const int es = sizeof(T);
  const long long MM = (long long)M * M;
  if (!(c->aws && c->am == M && c->ank == items && c->aes == es)) {
    release_aws(c);
    size_t bytes = (size_t)3 * MM * items * es + (size_t)4 * M * items * sizeof(double) + 4096;
    if (cudaMalloc(&c->aws, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->aws = nullptr;
      return fail(c, GKS_ENOMEM, "adjoint workspace allocation failed");
    }
    c->aws_bytes = bytes;
    c->am = M;
    c->ank = items;
    c->aes = es;
  }
  cudaStream_t s = c->stream;
  T* R = reinterpret_cast<T*>(c->aws);          // rho_bar (Hermitian part), later BH
  T* W = R + MM * items;                         // C^H rho_bar C, later BS
  T* T1 = W + MM * items;                        // GEMM temporary
  double* f = reinterpret_cast<double*>(T1 + MM * items);
  double* fp = f + (size_t)M * items;
  double* e = fp + (size_t)M * items;
  double* w = e + (size_t)M * items;
  const double gs = (nc || sp) ? 1.0 : 2.0;
  StageRec sr(c, PS_ADJOINT);
  {
    Rec r(c, PC_MISC);
    expand_weights(kw, nk, sp ? 2 : 1, w, s);
    adj_occ(eps, mu, kT, (long long)items * M, f, fp, s);
  }
  const int have_w = rho_bar ? 1 : 0;
  if (have_w) {
    {
      Rec r(c, PC_MISC);
      herm_part<T>(R, rho_bar, MM, MM, M, items, s);
    }
    gmx<T>(c, items, OP_N, OP_N, M, M, M, 1.0, R, M, MM, C, M, MM, 0.0, T1, M, MM);
    gmx<T>(c, items, OP_C, OP_N, M, M, M, 1.0, C, M, MM, T1, M, MM, 0.0, W, M, MM);
  }
  {
    Rec r(c, PC_MISC);
    adj_weights<T>(eps, f, fp, w, W, MM, M, items, gs, eps_bar, e_band_bar, have_w, e, s);
    adj_build<T>(W, R, MM, M, eps, f, e, mu, kT, gs, have_w, items, s);
  }
  // H_bar = C BH C^H
  gmx<T>(c, items, OP_N, OP_N, M, M, M, 1.0, C, M, MM, R, M, MM, 0.0, T1, M, MM);
  gmx<T>(c, items, OP_N, OP_C, M, M, M, 1.0, T1, M, MM, C, M, MM, 0.0, H_bar, M, MM);
  {
    Rec r(c, PC_MISC);
    herm_part<T>(H_bar, H_bar, MM, MM, M, items, s);
  }
  // S_bar = C BS C^H (noncollinear: the two diagonal spin blocks summed; spin-polarized:
  // the two channels summed)
  gmx<T>(c, items, OP_N, OP_N, M, M, M, 1.0, C, M, MM, W, M, MM, 0.0, T1, M, MM);
  if (nc || sp) {
    gmx<T>(c, items, OP_N, OP_C, M, M, M, 1.0, T1, M, MM, C, M, MM, 0.0, R, M, MM);
    Rec r(c, PC_MISC);
    if (nc) spin_block_sum<T>(S_bar, (long long)n * n, R, MM, n, nk, s);
    else spin_pair_sum<T>(S_bar, (long long)n * n, R, MM, n, nk, s);
  } else {
    gmx<T>(c, items, OP_N, OP_C, M, M, M, 1.0, T1, M, MM, C, M, MM, 0.0, S_bar, M, MM);
    Rec r(c, PC_MISC);
    herm_part<T>(S_bar, S_bar, MM, MM, M, items, s);
  }
  return cuda_check(c, "gks_adjoint launch");
}

gks_status validate_solve(gks_ctx* ctx, const SolveKey& k) {
  const bool eig_only = (k.flags & GKS_EIGEN_ONLY) != 0;
  if (!k.H || !k.S || !k.eps || !k.C || (!eig_only && (!k.mu || !k.rho)))
    return fail(ctx, GKS_EINVAL, "null array argument");
  if (k.flags & ~(unsigned)(GKS_REUSE_S_FACTOR | GKS_SAVE_FOR_BACKWARD | GKS_EIGEN_ONLY))
    return fail(ctx, GKS_EINVAL, "unknown flag bits");
  if (k.n < 1 || k.nk < 1 || k.n > 46340 || k.nk > 32767) return fail(ctx, GKS_EINVAL, "n or nk out of range");
  if (k.dtype != GKS_R64 && k.dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "unknown dtype");
  if (k.spin != GKS_COLLINEAR && k.spin != GKS_NONCOLLINEAR && k.spin != GKS_SPIN_POLARIZED)
    return fail(ctx, GKS_EINVAL, "unknown spin mode");
  const bool nc = k.spin == GKS_NONCOLLINEAR;
  if (nc && k.dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "noncollinear problems are complex (GKS_C128)");
  if (nc && 2 * k.n > 46340) return fail(ctx, GKS_EINVAL, "2n out of range");
  if (ctx->reduction == GKS_REDUCE_LOWDIN) {
    if (nc) return fail(ctx, GKS_ENOTIMPL, "the Loewdin reduction is implemented for collinear runs");
    if (ctx->n_ev > 0 && ctx->n_ev < k.n)
      return fail(ctx, GKS_EINVAL, "the Loewdin reduction needs every eigenvector of S: opts.n_ev must be 0");
  }
  if (ctx->precision == GKS_MIXED_SPLITBF16) {
    const long long M = nc ? 2 * k.n : k.n;
    if (ctx->n_ev > 0 && ctx->n_ev < M)
      return fail(ctx, GKS_EINVAL, "mixed precision refines every eigenvector: opts.n_ev must be 0");
    if (M > 18000) return fail(ctx, GKS_EINVAL, "mixed precision supports orders up to 18000");
  }
  if (!eig_only) {
    if (!(k.kT > 0.0)) return fail(ctx, GKS_EINVAL, "kT must be positive");
    const double gs = k.spin == GKS_COLLINEAR ? 2.0 : 1.0;
    const double states = (nc ? 2.0 * k.n : (double)k.n) * (k.spin == GKS_SPIN_POLARIZED ? 2.0 : 1.0);
    if (!(k.ne > 0.0) || !(k.ne < gs * states)) return fail(ctx, GKS_EINVAL, "n_elec must lie in (0, g_s M)");
  }
  return GKS_OK;
}

gks_status enqueue_solve(gks_ctx* ctx, const SolveKey& k) {
  if (k.dtype == GKS_R64) return solve_t<double>(ctx, k);
  return solve_t<zc>(ctx, k);
}

bool same_key(const SolveKey& a, const SolveKey& b) { return std::memcmp(&a, &b, sizeof(SolveKey)) == 0; }

// Capture whatever `body` enqueues on c->stream into a graph and instantiate it.
template <typename F>
gks_status capture(gks_ctx* c, cudaGraphExec_t* out, F body) {
  const bool prof_on = c->prof.on;
  c->prof.on = false;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    c->prof.on = prof_on;
    return cuda_check(c, "graph capture begin");
  }
  gks_status rc = body();
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  c->prof.on = prof_on;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || !g) return fail(c, GKS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, GKS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return GKS_OK;
}

}  // namespace

// ---- tuned-width cache file: one line per shape class, "bucket element_size spin width" ----
namespace {
void load_tune_cache(gks_ctx* c) {
  FILE* f = std::fopen(c->tune_cache.c_str(), "r");
  if (!f) return;  // no cache yet: the first gks_tune writes it
  int b, es, sp, w;
  while (std::fscanf(f, "%d %d %d %d", &b, &es, &sp, &w) == 4)
    if (w >= NB && w <= 1024 && w % NB == 0 && (es == 8 || es == 16) && sp >= 0 && sp <= 2)
      c->tuned[std::make_tuple(b, es, sp)] = w;
  std::fclose(f);
}

bool save_tune_cache(const gks_ctx* c) {
  if (c->tune_cache.empty()) return true;
  const std::string tmp = c->tune_cache + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  for (const auto& kv : c->tuned)
    std::fprintf(f, "%d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), kv.second);
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), c->tune_cache.c_str()) == 0;
}
}  // namespace

// ---- fixed scratch for split products that allocate nothing ----
// Digit scratch of gks_gemm_split_noalloc, part of the library image on every device.
// Shared by all calls on a device: calls whose work overlaps in time race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GKS_NOALLOC_SCRATCH_BYTES];
// Status word of those products (a bounded wait that expired), read back by gks_sync.
static __device__ __align__(256) DevStatus g_noalloc_status;

namespace {
constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocDevices] = {};
DevStatus* g_noalloc_st[kNoAllocDevices] = {};

// Device addresses of the scratch and of its status word on `dev`, which must be the
// current device; resolved once per device.
cudaError_t noalloc_scratch(int dev, void** out, DevStatus** st) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_noalloc_status);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
    g_noalloc_st[dev] = static_cast<DevStatus*>(q);
  }
  *out = g_noalloc_ptr[dev];
  *st = g_noalloc_st[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" {

gks_status gks_create(gks_ctx** ctx, const gks_opts* opts) {
  if (!ctx) return GKS_EINVAL;
  gks_ctx* c = new gks_ctx();
  if (opts) {
    c->device = opts->device;
    c->stream = static_cast<cudaStream_t>(opts->cuda_stream);
    if (opts->f_cut > 0.0) c->f_cut = opts->f_cut;
    c->prof.on = opts->profile != 0;
    c->graph = opts->graph != 0;
    c->gemm_mode = opts->gemm;
    if (opts->slices > 0) c->slices = opts->slices;
    c->split = opts->split;
    c->hemv = opts->hemv;
    if (opts->block > 0) c->nbb = opts->block;
    c->nbb_default = c->nbb;
    c->nbb_fixed = opts->block > 0;
    c->precision = opts->precision;
    if (opts->refine_sweeps > 0) c->refine_sweeps = opts->refine_sweeps;
    c->n_ev = opts->n_ev;
    c->reduction = opts->reduction;
    c->tridiag = opts->tridiag;
    if (opts->band > 0) c->band = opts->band;
    if (opts->wait_limit > 0) c->wait_cycles = opts->wait_limit;
    c->debug = opts->debug;
    if (opts->autotune_cache) c->tune_cache = opts->autotune_cache;
    if (c->gemm_mode < 0 || c->gemm_mode > 2 || c->slices < 4 || c->slices > 10 || c->nbb < NB || c->nbb > 1024 ||
        c->nbb % NB || c->n_ev < 0 || opts->refine_sweeps < 0 || opts->refine_sweeps > 8 || opts->wait_limit < 0 ||
        (c->reduction != GKS_REDUCE_CHOLESKY && c->reduction != GKS_REDUCE_LOWDIN) ||
        (c->tridiag != GKS_TRIDIAG_ONE_STAGE && c->tridiag != GKS_TRIDIAG_TWO_STAGE) || c->band < 2 ||
        c->band > 32 || (c->split != GKS_SPLIT_RESIDUES && c->split != GKS_SPLIT_DIGITS) ||
        (c->hemv != GKS_HEMV_DIGITS && c->hemv != GKS_HEMV_FP64) ||
        (opts->debug & ~GKS_DEBUG_SKIP_COPY)) {
      delete c;
      return GKS_EINVAL;
    }
    if (c->precision != GKS_FP64 && c->precision != GKS_MIXED_SPLITBF16) {
      delete c;
      return c->precision == GKS_MIXED_TF32 ? GKS_ENOTIMPL : GKS_EINVAL;
    }
  }
  {
    DeviceGuard dg(c->device);
    if (!dg.ok) {
      delete c;
      return GKS_ECUDA;
    }
    if (cudaMalloc(&c->gst, sizeof(DevStatus)) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return GKS_ENOMEM;
    }
    cudaMemset(c->gst, 0, sizeof(DevStatus));
  }
  if (!c->tune_cache.empty()) load_tune_cache(c);
  c->prof.stream = c->stream;
  *ctx = c;
  return GKS_OK;
}

gks_status gks_destroy(gks_ctx* ctx) {
  if (!ctx) return GKS_OK;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (auto sc : ctx->subs) {
    release_ws(sc);
    release_aws(sc);
    release_oz(sc);
    delete sc;
  }
  for (auto w : ctx->workers) cudaStreamDestroy(w);
  release_ws(ctx);
  release_aws(ctx);
  release_oz(ctx);
  release_extra(ctx);
  delete ctx;
  return GKS_OK;
}

const char* gks_last_error(const gks_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

gks_status gks_solve(gks_ctx* ctx, const void* H, const void* S, int64_t n, int64_t nk, int dtype, int spin_mode,
                     double kT, double n_elec, const double* kweights, unsigned flags, double* eps, void* C,
                     double* mu, void* rho, double* e_band) {
  if (!ctx) return GKS_EINVAL;
  ctx->err.clear();
  SolveKey k{H, S, kweights, eps, C, mu, rho, e_band, (long long)n, (long long)nk, dtype, spin_mode, kT, n_elec,
             flags, 0u};
  gks_status rc = validate_solve(ctx, k);
  if (rc) return rc;
  DeviceGuard dg(ctx->device);
  if (!ctx->graph || ctx->stream == nullptr) return enqueue_solve(ctx, k);
  // graph mode: replay while the arguments are unchanged; the first call for a new
  // argument set runs eagerly (allocates the workspace and the merge lists), the next
  // one captures.
  if (ctx->gexec && same_key(ctx->gkey, k)) {
    cudaGraphLaunch(ctx->gexec, ctx->stream);
    return cuda_check(ctx, "graph launch");
  }
  const int M = spin_mode == GKS_NONCOLLINEAR ? (int)(2 * n) : (int)n;
  const int items = spin_mode == GKS_SPIN_POLARIZED ? (int)(2 * nk) : (int)nk;
  const int es = dtype == GKS_R64 ? 8 : 16;
  // capture only when the workspace (order, batch, type and width) and the saved copies
  // are already in place, so that nothing is allocated or freed while the stream is being
  // captured
  const bool saved_ok = !(flags & GKS_SAVE_FOR_BACKWARD) ||
                        (ctx->sv_valid && ctx->svkey.n == k.n && ctx->svkey.nk == k.nk &&
                         ctx->svkey.dtype == k.dtype && ctx->svkey.spin == k.spin);
  const bool ready = ctx->ws && ctx->m == M && ctx->nk == items && ctx->es == es &&
                     ctx->nbb == pick_width(ctx, M, es, shape_spin(spin_mode)) && ctx->gkey.H == k.H && ctx->gkey.C == k.C &&
                     saved_ok;
  ctx->gkey = k;
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  if (!ready) return enqueue_solve(ctx, k);
  rc = capture(ctx, &ctx->gexec, [&]() { return enqueue_solve(ctx, k); });
  if (rc) return rc;
  cudaGraphLaunch(ctx->gexec, ctx->stream);
  return cuda_check(ctx, "graph launch");
}

gks_status gks_solve_batched(gks_ctx* ctx, int64_t count, const gks_problem* probs, int nstreams) {
  if (!ctx || count < 1 || !probs) return fail(ctx, GKS_EINVAL, "bad batch arguments");
  ctx->err.clear();
  if (ctx->stream == nullptr) return fail(ctx, GKS_EINVAL, "gks_solve_batched needs a non-default stream");
  std::vector<SolveKey> keys((size_t)count);
  for (int64_t b = 0; b < count; b++) {
    const gks_problem& p = probs[b];
    keys[b] = SolveKey{p.H, p.S, p.kweights, p.eps, p.C, p.mu, p.rho, p.e_band, (long long)p.n, (long long)p.nk,
                       p.dtype, p.spin_mode, p.kT, p.n_elec, 0u, 0u};
    gks_status rc = validate_solve(ctx, keys[b]);
    if (rc) return fail(ctx, rc, "problem " + std::to_string(b) + ": " + ctx->err);
  }
  DeviceGuard dg(ctx->device);
  const int P = std::max(1, std::min(nstreams > 0 ? nstreams : 8, (int)count));
  while ((int)ctx->workers.size() < P) {
    cudaStream_t w;
    if (cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking) != cudaSuccess) return cuda_check(ctx, "stream create");
    ctx->workers.push_back(w);
  }
  while ((int64_t)ctx->subs.size() < count) {
    gks_ctx* sc = new gks_ctx();
    sc->device = ctx->device;
    sc->f_cut = ctx->f_cut;
    sc->gemm_mode = ctx->gemm_mode;
    sc->slices = ctx->slices;
    sc->split = ctx->split;
    sc->hemv = ctx->hemv;
    sc->nbb = ctx->nbb;
    sc->nbb_default = ctx->nbb_default;
    sc->nbb_fixed = ctx->nbb_fixed;
    sc->wait_cycles = ctx->wait_cycles;
    sc->n_ev = ctx->n_ev;
    sc->precision = ctx->precision;
    sc->refine_sweeps = ctx->refine_sweeps;
    sc->reduction = ctx->reduction;
    sc->tridiag = ctx->tridiag;
    sc->band = ctx->band;
    ctx->subs.push_back(sc);
  }
  for (auto* sc : ctx->subs) sc->tuned = ctx->tuned;
  auto body = [&]() -> gks_status {
    cudaEvent_t fork;
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    cudaEventRecord(fork, ctx->stream);
    for (int w = 0; w < P; w++) cudaStreamWaitEvent(ctx->workers[w], fork, 0);
    gks_status rc = GKS_OK;
    for (int64_t b = 0; b < count && !rc; b++) {
      gks_ctx* sc = ctx->subs[b];
      sc->stream = ctx->workers[b % P];
      sc->prof.stream = sc->stream;
      rc = enqueue_solve(sc, keys[b]);
      if (rc) ctx->err = "problem " + std::to_string(b) + ": " + sc->err;
    }
    for (int w = 0; w < P; w++) {
      cudaEvent_t join;
      cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
      cudaEventRecord(join, ctx->workers[w]);
      cudaStreamWaitEvent(ctx->stream, join, 0);
      cudaEventDestroy(join);
    }
    cudaEventDestroy(fork);
    return rc;
  };
  if (!ctx->graph) {
    gks_status rc = body();
    return rc ? rc : cuda_check(ctx, "gks_solve_batched launch");
  }
  if (ctx->bexec && ctx->bkey.size() == keys.size() &&
      std::equal(keys.begin(), keys.end(), ctx->bkey.begin(), same_key)) {
    cudaGraphLaunch(ctx->bexec, ctx->stream);
    return cuda_check(ctx, "batch graph launch");
  }
  if (ctx->bexec) {
    cudaGraphExecDestroy(ctx->bexec);
    ctx->bexec = nullptr;
  }
  const bool first = ctx->bkey.size() != keys.size() ||
                     !std::equal(keys.begin(), keys.end(), ctx->bkey.begin(), same_key);
  ctx->bkey = keys;
  if (first) {  // eager run: allocates every problem's workspace and merge lists
    gks_status rc = body();
    return rc ? rc : cuda_check(ctx, "gks_solve_batched launch");
  }
  gks_status rc = capture(ctx, &ctx->bexec, body);
  if (rc) return rc;
  cudaGraphLaunch(ctx->bexec, ctx->stream);
  return cuda_check(ctx, "batch graph launch");
}

gks_status gks_adjoint(gks_ctx* ctx, const void* C, const double* eps, const double* mu, int64_t n, int64_t nk,
                       int dtype, int spin_mode, double kT, const double* kweights, const void* rho_bar,
                       const double* eps_bar, double e_band_bar, void* H_bar, void* S_bar) {
  if (!ctx) return GKS_EINVAL;
  ctx->err.clear();
  if (!H_bar || !S_bar) return fail(ctx, GKS_EINVAL, "null array argument");
  if (n < 1 || nk < 1 || n > 46340 || nk > 32767) return fail(ctx, GKS_EINVAL, "n or nk out of range");
  if (dtype != GKS_R64 && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "unknown dtype");
  const bool nc = spin_mode == GKS_NONCOLLINEAR;
  if (spin_mode != GKS_COLLINEAR && !nc && spin_mode != GKS_SPIN_POLARIZED)
    return fail(ctx, GKS_EINVAL, "unknown spin mode");
  if (nc && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "noncollinear problems are complex (GKS_C128)");
  if (!(kT > 0.0)) return fail(ctx, GKS_EINVAL, "kT must be positive");
  const int M = nc ? 2 * (int)n : (int)n;
  if (ncols_of(ctx, M) < M) return fail(ctx, GKS_EINVAL, "the adjoint needs every eigenvector (opts.n_ev = 0)");
  if (!C || !eps || !mu) {
    // the copies kept by the last solve with GKS_SAVE_FOR_BACKWARD
    if (C || eps) return fail(ctx, GKS_EINVAL, "pass C and eps together, or neither to use the saved ones");
    const SolveKey& k = ctx->svkey;
    if (!ctx->sv_valid || k.n != n || k.nk != nk || k.dtype != dtype || k.spin != spin_mode)
      return fail(ctx, GKS_EINVAL, "no eigenpairs of this shape were saved (GKS_SAVE_FOR_BACKWARD)");
    if (!mu && (k.flags & GKS_EIGEN_ONLY)) return fail(ctx, GKS_EINVAL, "the saved solve computed no mu");
    const int items = spin_mode == GKS_SPIN_POLARIZED ? 2 * (int)nk : (int)nk;
    const size_t bC = (size_t)items * M * M * (dtype == GKS_C128 ? 16 : 8), bE = (size_t)items * M * sizeof(double);
    const size_t oE = (bC + 255) & ~size_t(255), oM = oE + ((bE + 255) & ~size_t(255));
    C = ctx->sv;
    eps = reinterpret_cast<const double*>(ctx->sv + oE);
    if (!mu) mu = reinterpret_cast<const double*>(ctx->sv + oM);
  }
  DeviceGuard dg(ctx->device);
  if (dtype == GKS_R64)
    return adjoint_t<double>(ctx, static_cast<const double*>(C), eps, mu, (int)n, (int)nk, spin_mode, kT, kweights,
                             static_cast<const double*>(rho_bar), eps_bar, e_band_bar, static_cast<double*>(H_bar),
                             static_cast<double*>(S_bar));
  return adjoint_t<zc>(ctx, static_cast<const zc*>(C), eps, mu, (int)n, (int)nk, spin_mode, kT, kweights,
                       static_cast<const zc*>(rho_bar), eps_bar, e_band_bar, static_cast<zc*>(H_bar),
                       static_cast<zc*>(S_bar));
}

gks_status gks_occupy(gks_ctx* ctx, const double* eps_all, int64_t nk_all, int64_t k0, const void* C, int64_t n,
                      int64_t nk, int dtype, int spin_mode, double kT, double n_elec, const double* kweights_all,
                      double* mu, void* rho, double* e_band, void* edm) {
  if (!ctx) return GKS_EINVAL;
  ctx->err.clear();
  if (!eps_all || !mu || ((rho || edm) && !C)) return fail(ctx, GKS_EINVAL, "null array argument");
  if (n < 1 || n > 46340 || nk_all < 1 || nk_all > 32767 || k0 < 0 || nk < 0 || k0 + nk > nk_all)
    return fail(ctx, GKS_EINVAL, "n, nk_all, k0 or nk out of range");
  if (dtype != GKS_R64 && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "unknown dtype");
  const bool nc = spin_mode == GKS_NONCOLLINEAR, sp = spin_mode == GKS_SPIN_POLARIZED;
  if (spin_mode != GKS_COLLINEAR && !nc && !sp) return fail(ctx, GKS_EINVAL, "unknown spin mode");
  if (nc && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "noncollinear problems are complex (GKS_C128)");
  if (!(kT > 0.0)) return fail(ctx, GKS_EINVAL, "kT must be positive");
  const int M = nc ? 2 * (int)n : (int)n;
  const int rep = sp ? 2 : 1;
  const double gs = (nc || sp) ? 1.0 : 2.0;
  if (!(n_elec > 0.0) || !(n_elec < gs * M * rep)) return fail(ctx, GKS_EINVAL, "n_elec must lie in (0, g_s M)");
  const int all = (int)nk_all * rep, loc = (int)nk * rep, i0 = (int)k0 * rep;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = ctx->stream;
  const size_t vec = ((size_t)all * M * sizeof(double) + 255) & ~size_t(255);
  const size_t need = 3 * vec + (((size_t)all * (sizeof(double) + sizeof(int)) + 255) & ~size_t(255)) + 256;
  if (need > ctx->ow_bytes) {
    cudaStreamSynchronize(s);
    if (ctx->ow) cudaFree(ctx->ow);
    ctx->ow = nullptr;
    ctx->ow_bytes = 0;
    if (cudaMalloc(&ctx->ow, need) != cudaSuccess) {
      cudaGetLastError();
      ctx->ow = nullptr;
      return fail(ctx, GKS_ENOMEM, "occupation workspace allocation failed");
    }
    ctx->ow_bytes = need;
  }
  double* occ = reinterpret_cast<double*>(ctx->ow);
  double* ks = reinterpret_cast<double*>(ctx->ow + vec);
  double* kse = reinterpret_cast<double*>(ctx->ow + 2 * vec);
  double* w = reinterpret_cast<double*>(ctx->ow + 3 * vec);
  int* nrho = reinterpret_cast<int*>(w + all);
  double* eb = reinterpret_cast<double*>(ctx->ow + need - 256);
  const int nev = ncols_of(ctx, M);
  const long long sC = (long long)M * nev, MM = (long long)M * M;
  {
    StageRec sr(ctx, PS_OCC);
    Rec r(ctx, PC_OCC);
    cudaMemsetAsync(ctx->gst, 0, sizeof(DevStatus), s);
    expand_weights(kweights_all, (int)nk_all, rep, w, s);
    fermi_mu(eps_all, M, all, w, gs, kT, n_elec, ctx->f_cut, occ, ks, mu, e_band ? e_band : eb, nrho, ctx->gst, 1, s);
    if (nev < M && loc > 0) clamp_nrho(nrho + i0, loc, nev, ctx->gst, 0, s);
  }
  if (loc > 0 && (rho || edm)) {
    StageRec sr(ctx, PS_RHO);
    auto run = [&](void* out, const double* weights) {
      if (dtype == GKS_R64) {
        rho_run<double>(ctx, static_cast<const double*>(C), nev, sC, static_cast<double*>(out), MM, weights, M,
                        nrho + i0, M, nev, loc);
        mirror_lower<double>(static_cast<double*>(out), M, MM, M, loc, s);
      } else {
        rho_run<zc>(ctx, static_cast<const zc*>(C), nev, sC, static_cast<zc*>(out), MM, weights, M, nrho + i0, M, nev,
                    loc);
        mirror_lower<zc>(static_cast<zc*>(out), M, MM, M, loc, s);
      }
    };
    if (rho) run(rho, ks + (size_t)i0 * M);
    if (edm) {
      // energy-density matrix: the density-matrix product with weights g_s f eps
      mul_elem(ks + (size_t)i0 * M, eps_all + (size_t)i0 * M, kse, (long long)loc * M, s);
      run(edm, kse);
    }
  }
  return cuda_check(ctx, "gks_occupy launch");
}

gks_status gks_sync(gks_ctx* ctx) {
  if (!ctx) return GKS_EINVAL;
  DeviceGuard dg(ctx->device);
  cudaError_t e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(ctx, GKS_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
  for (size_t b = 0; b < ctx->subs.size(); b++) {
    gks_status rc = gks_sync(ctx->subs[b]);
    if (rc) return fail(ctx, rc, "batch problem " + std::to_string(b) + ": " + ctx->subs[b]->err);
  }
  if (ctx->noalloc_st) {
    DevStatus h{};
    if (cudaMemcpy(&h, ctx->noalloc_st, sizeof(DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(ctx, GKS_ECUDA, "status read failed");
    ctx->noalloc_st = nullptr;
    if (h.code != ST_OK)
      return fail(ctx, (gks_status)h.code, "gks_gemm_split_noalloc: a bounded device-side wait expired; the "
                                           "product's output is incomplete");
  }
  if (ctx->gst) {
    DevStatus h{};
    if (cudaMemcpy(&h, ctx->gst, sizeof(DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(ctx, GKS_ECUDA, "status read failed");
    if (h.code != ST_OK) {
      cudaMemset(ctx->gst, 0, sizeof(DevStatus));
      ctx->l_valid = false;
      return fail(ctx, (gks_status)h.code,
                  h.code == ST_ETIMEOUT ? std::string("a bounded device-side wait expired in a product; its output is "
                                                      "incomplete")
                                        : "invalid occupation parameters or non-finite eigenvalues (gks_occupy)");
    }
  }
  if (!ctx->st) return GKS_OK;
  std::vector<DevStatus> h(ctx->nk);
  if (cudaMemcpy(h.data(), ctx->st, sizeof(DevStatus) * ctx->nk, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(ctx, GKS_ECUDA, "status read failed");
  for (int k = 0; k < ctx->nk; k++) {
    if (h[k].code == ST_OK) continue;
    gks_status code = (gks_status)h[k].code;
    std::string what = code == GKS_ENOTSPD ? "S is not positive definite at column " + std::to_string(h[k].info)
                       : code == GKS_ENOCONV ? "iteration did not converge (index " + std::to_string(h[k].info) + ")"
                       : code == GKS_ETIMEOUT ? std::string("a bounded device-side wait expired in a product")
                       : code == GKS_EINVAL && h[k].info > 0
                           ? "occupied states (" + std::to_string(h[k].info) + ") exceed the eigenvectors computed (n_ev)"
                       : code == GKS_EINVAL ? std::string("invalid occupation parameters or non-finite eigenvalues")
                                            : "device status " + std::to_string(h[k].code);
    cudaMemset(ctx->st, 0, sizeof(DevStatus) * ctx->nk);
    ctx->l_valid = false;  // the kept factor may come from the failed solve
    return fail(ctx, code, what + " (batch item " + std::to_string(k) + ")");
  }
  return GKS_OK;
}

long long gks_launch_count(void) { return launches_issued(); }

int gks_refine_stats(gks_ctx* ctx, double* out, int max) {
  if (!ctx || !out || max < 1 || !ctx->ws || !ctx->wsmixed || ctx->rstat_sweeps == 0) return 0;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  const int n = std::min(max, 2 * ctx->rstat_sweeps * ctx->rstat_items);
  if (cudaMemcpy(out, at<double>(ctx, ctx->orstat), sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

gks_status gks_measure_peak(gks_ctx* ctx, int which, double* tflops) {
  if (!ctx || !tflops || which < 0 || which > 1) return fail(ctx, GKS_EINVAL, "bad arguments");
  DeviceGuard dg(ctx->device);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || sms < 1)
    return cuda_check(ctx, "gks_measure_peak: device attribute");
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)sms * 1024) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, GKS_ENOMEM, "gks_measure_peak: allocation failed");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // size the probe to about 100 ms from a short first run, then take the best of three
  long long iters = 1 << 14;
  double best = 0.0;
  for (int rep = 0; rep < 4; rep++) {
    cudaEventRecord(e0, ctx->stream);
    const double fl = peak_probe(which, sms, iters, out, ctx->stream);
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep == 0) {
      iters = (long long)((double)iters * 100.0 / std::max(1e-3, (double)ms));
      iters = std::max(1ll << 12, std::min(iters, 1ll << 26));
      continue;
    }
    best = std::max(best, fl / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *tflops = best;
  return cuda_check(ctx, "gks_measure_peak");
}

int gks_profile(gks_ctx* ctx, gks_prof_entry* out, int max) {
  if (!ctx || !ctx->prof.on) return 0;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  EventProf& P = ctx->prof;
  double rho_fl = 0.0, rho_by = 0.0;
  if (P.nrho_dev && ctx->ws) {
    std::vector<int> nr(P.rho_nk);
    cudaMemcpy(nr.data(), P.nrho_dev, sizeof(int) * P.rho_nk, cudaMemcpyDeviceToHost);
    const double m = P.rho_m;
    for (int k = 0; k < P.rho_nk; k++) {
      rho_fl += cmul(P.rho_es) * 0.5 * m * (m + 1) * nr[k];
      rho_by += (double)P.rho_es * (2.0 * m * nr[k] + 0.5 * m * (m + 1));
    }
  }
  const int nent = PC_NCLASS + PS_NSTAGE;
  std::vector<gks_prof_entry> acc(nent);
  for (int i = 0; i < nent; i++) {
    std::memset(&acc[i], 0, sizeof(gks_prof_entry));
    std::snprintf(acc[i].name, sizeof(acc[i].name), "%s", i < PC_NCLASS ? kClassNames[i] : kStageNames[i - PC_NCLASS]);
  }
  for (auto& r : P.recs) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, P.pool[r.e0], P.pool[r.e1]);
    gks_prof_entry& e = acc[r.cls];
    e.groups++;
    e.ms += ms;
    e.flops += r.flops < 0 ? rho_fl : r.flops;
    e.bytes += r.bytes < 0 ? rho_by : r.bytes;
  }
  P.recs.clear();
  P.used = 0;
  int k = 0;
  for (int i = 0; i < nent && k < max; i++)
    if (acc[i].groups > 0) out[k++] = acc[i];
  cudaGetLastError();
  return k;
}

gks_status gks_gemm(gks_ctx* ctx, int dtype, int opA, int opB, int64_t M, int64_t N, int64_t K, double alpha,
                    const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                    int mode) {
  if (!ctx || ((!A || !B) && K > 0) || !C || M < 0 || N < 0 || K < 0) return fail(ctx, GKS_EINVAL, "bad arguments");
  if (opA < 0 || opA > 2 || opB < 0 || opB > 2 || mode < 1 || mode > 2) return fail(ctx, GKS_EINVAL, "bad op or mode");
  if (M > 46340 || N > 46340 || K > 46340) return fail(ctx, GKS_EINVAL, "dimension too large");
  DeviceGuard dg(ctx->device);
  const int saved = ctx->gemm_mode;
  ctx->gemm_mode = mode;
  if (dtype == GKS_R64)
    gmx<double>(ctx, 1, opA, opB, (int)M, (int)N, (int)K, alpha, static_cast<const double*>(A), (int)lda, 0,
                static_cast<const double*>(B), (int)ldb, 0, beta, static_cast<double*>(C), (int)ldc, 0);
  else if (dtype == GKS_C128)
    gmx<zc>(ctx, 1, opA, opB, (int)M, (int)N, (int)K, alpha, static_cast<const zc*>(A), (int)lda, 0,
            static_cast<const zc*>(B), (int)ldb, 0, beta, static_cast<zc*>(C), (int)ldc, 0);
  else {
    ctx->gemm_mode = saved;
    return fail(ctx, GKS_EINVAL, "unknown dtype");
  }
  ctx->gemm_mode = saved;
  return cuda_check(ctx, "gks_gemm");
}

gks_status gks_gemm_split_noalloc(gks_ctx* ctx, int dtype, int opA, int opB, int64_t M, int64_t N, int64_t K,
                                  double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                                  double beta, void* C, int64_t ldc) {
  if (!ctx || ((!A || !B) && K > 0) || !C || M < 0 || N < 0 || K < 0) return fail(ctx, GKS_EINVAL, "bad arguments");
  if (opA < 0 || opA > 2 || opB < 0 || opB > 2) return fail(ctx, GKS_EINVAL, "bad op");
  if (dtype != GKS_R64 && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "unknown dtype");
  if (M > 46340 || N > 46340 || K > 46340) return fail(ctx, GKS_EINVAL, "dimension too large");
  if (ctx->device < 0 || ctx->device >= kNoAllocDevices) return fail(ctx, GKS_EINVAL, "device index out of range");
  const size_t need = ozaki_workspace_bytes((int)M, (int)N, (int)K, dtype == GKS_C128, ctx->slices);
  if (need > (size_t)GKS_NOALLOC_SCRATCH_BYTES)
    return fail(ctx, GKS_EINVAL,
                "product needs " + std::to_string(need) + " bytes of split scratch; the fixed scratch holds " +
                    std::to_string((size_t)GKS_NOALLOC_SCRATCH_BYTES) + " bytes");
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return fail(ctx, GKS_ECUDA, "gks_gemm_split_noalloc: cannot make the context's device current");
  void* scratch = nullptr;
  DevStatus* st = nullptr;
  cudaError_t e = noalloc_scratch(ctx->device, &scratch, &st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, GKS_ECUDA, std::string("gks_gemm_split_noalloc: scratch lookup: ") + cudaGetErrorString(e));
  }
  cudaMemsetAsync(st, 0, sizeof(DevStatus), ctx->stream);
  ctx->noalloc_st = st;
  bool ok;
  if (dtype == GKS_R64)
    ok = ozaki_gemm<double>(opA, opB, (int)M, (int)N, (int)K, alpha, static_cast<const double*>(A), (int)lda, 0,
                       static_cast<const double*>(B), (int)ldb, 0, beta, static_cast<double*>(C), (int)ldc, 0, 1, 0,
                       ctx->slices, scratch, st, ctx->stream, nullptr, 0, nullptr, ctx->wait_cycles);
  else
    ok = ozaki_gemm<zc>(opA, opB, (int)M, (int)N, (int)K, alpha, static_cast<const zc*>(A), (int)lda, 0,
                   static_cast<const zc*>(B), (int)ldb, 0, beta, static_cast<zc*>(C), (int)ldc, 0, 1, 0,
                   ctx->slices, scratch, st, ctx->stream, nullptr, 0, nullptr, ctx->wait_cycles);
  if (!ok) return fail(ctx, GKS_ECUDA, "gks_gemm_split_noalloc: TMA tensor map encoding unavailable");
  return cuda_check(ctx, "gks_gemm_split_noalloc");
}

gks_status gks_tune(gks_ctx* ctx, int64_t n, int64_t nk, int dtype, int spin_mode, const int* widths, int count,
                    double* ms, int* best) {
  if (!ctx || n < 1 || nk < 1 || !widths || count < 1 || !ms || !best) return fail(ctx, GKS_EINVAL, "bad arguments");
  if (dtype != GKS_R64 && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "unknown dtype");
  if (spin_mode != GKS_COLLINEAR && spin_mode != GKS_NONCOLLINEAR) return fail(ctx, GKS_EINVAL, "unknown spin mode");
  const bool nc = spin_mode == GKS_NONCOLLINEAR;
  if (nc && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "noncollinear requires complex");
  for (int i = 0; i < count; i++)
    if (widths[i] < NB || widths[i] > 1024 || widths[i] % NB) return fail(ctx, GKS_EINVAL, "width not a multiple of 64 in 64..1024");
  const int M = nc ? 2 * (int)n : (int)n;
  const int es = dtype == GKS_C128 ? 16 : 8;
  if ((double)M * M * nk * es > 64e9) return fail(ctx, GKS_EINVAL, "tuning problem too large");
  DeviceGuard dg(ctx->device);
  if (!dg.ok) return fail(ctx, GKS_ECUDA, "gks_tune: cannot make the context's device current");
  const size_t bH = (size_t)M * M * nk * es, bS = (size_t)n * n * nk * es;
  void *H = nullptr, *S = nullptr, *C = nullptr, *rho = nullptr;
  double *eps = nullptr, *mu = nullptr;
  auto release = [&]() {
    cudaFree(H);
    cudaFree(S);
    cudaFree(C);
    cudaFree(rho);
    cudaFree(eps);
    cudaFree(mu);
  };
  if (cudaMalloc(&H, bH) != cudaSuccess || cudaMalloc(&S, bS) != cudaSuccess || cudaMalloc(&C, bH) != cudaSuccess ||
      cudaMalloc(&rho, bH) != cudaSuccess || cudaMalloc(&eps, sizeof(double) * M * nk) != cudaSuccess ||
      cudaMalloc(&mu, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(ctx, GKS_ENOMEM, "gks_tune: allocation of the test pencils failed");
  }
  if (es == 16) {
    tune_pencil<zc>(static_cast<zc*>(H), M, (int)nk, 1, ctx->stream);
    tune_pencil<zc>(static_cast<zc*>(S), (int)n, (int)nk, 0, ctx->stream);
  } else {
    tune_pencil<double>(static_cast<double*>(H), M, (int)nk, 1, ctx->stream);
    tune_pencil<double>(static_cast<double*>(S), (int)n, (int)nk, 0, ctx->stream);
  }
  const auto key = std::make_tuple(order_bucket(M), es, nc ? 1 : 0);
  const bool graph = ctx->graph;
  ctx->graph = false;
  const double gs = nc ? 1.0 : 2.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  gks_status rc = GKS_OK;
  int bi = 0;
  for (int i = 0; i < count && rc == GKS_OK; i++) {
    ctx->tuned[key] = widths[i];
    for (int rep = 0; rep < 2 && rc == GKS_OK; rep++) {
      cudaEventRecord(e0, ctx->stream);
      rc = gks_solve(ctx, H, S, n, nk, dtype, spin_mode, 0.01, 0.5 * gs * M, nullptr, 0, eps, C, mu, rho, nullptr);
      cudaEventRecord(e1, ctx->stream);
      if (rc == GKS_OK) rc = gks_sync(ctx);
    }
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    ms[i] = t;
    if (ms[i] < ms[bi]) bi = i;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->graph = graph;
  release();
  if (rc != GKS_OK) {
    ctx->tuned.erase(key);
    return rc;
  }
  ctx->tuned[key] = widths[bi];
  *best = widths[bi];
  if (!save_tune_cache(ctx)) return fail(ctx, GKS_EINVAL, "cannot write the autotune cache " + ctx->tune_cache);
  return cuda_check(ctx, "gks_tune");
}

gks_status gks_tune_set(gks_ctx* ctx, int64_t n, int dtype, int spin_mode, int width) {
  if (!ctx || n < 1 || (dtype != GKS_R64 && dtype != GKS_C128)) return fail(ctx, GKS_EINVAL, "bad arguments");
  if (width != 0 && (width < NB || width > 1024 || width % NB))
    return fail(ctx, GKS_EINVAL, "width not a multiple of 64 in 64..1024");
  const bool nc = spin_mode == GKS_NONCOLLINEAR;
  const auto key = std::make_tuple(order_bucket(nc ? 2 * (int)n : (int)n), dtype == GKS_C128 ? 16 : 8, nc ? 1 : 0);
  if (width == 0) ctx->tuned.erase(key);
  else ctx->tuned[key] = width;
  if (!save_tune_cache(ctx)) return fail(ctx, GKS_EINVAL, "cannot write the autotune cache " + ctx->tune_cache);
  return GKS_OK;
}

int gks_tune_get(const gks_ctx* ctx, int64_t n, int dtype, int spin_mode) {
  if (!ctx || n < 1) return 0;
  const bool nc = spin_mode == GKS_NONCOLLINEAR;
  return pick_width(ctx, nc ? 2 * (int)n : (int)n, dtype == GKS_C128 ? 16 : 8, nc ? 1 : 0);
}

gks_status gks_potrf(gks_ctx* ctx, void* A, int64_t m, int64_t count, int dtype) {
  if (!ctx || !A || m < 1 || count < 1 || m > 46340) return fail(ctx, GKS_EINVAL, "bad arguments");
  DeviceGuard dg(ctx->device);
  if (dtype == GKS_R64) {
    gks_status rc = ensure_ws(ctx, (int)m, (int)m, (int)count, 8, 0);
    if (rc) return rc;
    cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus) * count, ctx->stream);
    potrf_run<double>(ctx, static_cast<double*>(A), (int)m, (int)m, m * m, (int)count);
  } else if (dtype == GKS_C128) {
    gks_status rc = ensure_ws(ctx, (int)m, (int)m, (int)count, 16, 0);
    if (rc) return rc;
    cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus) * count, ctx->stream);
    potrf_run<zc>(ctx, static_cast<zc*>(A), (int)m, (int)m, m * m, (int)count);
  } else {
    return fail(ctx, GKS_EINVAL, "unknown dtype");
  }
  return cuda_check(ctx, "gks_potrf");
}

gks_status gks_reduce(gks_ctx* ctx, void* H, void* S, int64_t m, int64_t count, int dtype) {
  if (!ctx || !H || !S || m < 1 || count < 1 || m > 46340) return fail(ctx, GKS_EINVAL, "bad arguments");
  DeviceGuard dg(ctx->device);
  if (dtype == GKS_R64) {
    gks_status rc = ensure_ws(ctx, (int)m, (int)m, (int)count, 8, 0);
    if (rc) return rc;
    cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus) * count, ctx->stream);
    potrf_run<double>(ctx, static_cast<double*>(S), (int)m, (int)m, m * m, (int)count);
    hegst_run<double>(ctx, static_cast<double*>(H), (int)m, m * m, static_cast<double*>(S), (int)m, m * m, (int)m,
                      (int)count);
  } else if (dtype == GKS_C128) {
    gks_status rc = ensure_ws(ctx, (int)m, (int)m, (int)count, 16, 0);
    if (rc) return rc;
    cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus) * count, ctx->stream);
    potrf_run<zc>(ctx, static_cast<zc*>(S), (int)m, (int)m, m * m, (int)count);
    hegst_run<zc>(ctx, static_cast<zc*>(H), (int)m, m * m, static_cast<zc*>(S), (int)m, m * m, (int)m, (int)count);
  } else {
    return fail(ctx, GKS_EINVAL, "unknown dtype");
  }
  return cuda_check(ctx, "gks_reduce");
}

}  // extern "C"

namespace {
// Temporarily select the two-stage path with bandwidth `band` on a context (stage entries).
struct TwoStageScope {
  gks_ctx* c;
  int tri, band;
  TwoStageScope(gks_ctx* c_, int b) : c(c_), tri(c_->tridiag), band(c_->band) {
    c->tridiag = GKS_TRIDIAG_TWO_STAGE;
    c->band = b;
  }
  ~TwoStageScope() {
    c->tridiag = tri;
    c->band = band;
  }
};

template <typename T>
void identity_fill(T* Q, int m, int count, cudaStream_t s) {
  cudaMemsetAsync(Q, 0, sizeof(T) * (size_t)m * m * count, s);
  T one = from_real<T>(1.0);
  for (int z = 0; z < count; z++)
    for (int i = 0; i < m; i++)
      cudaMemcpyAsync(Q + ((size_t)z * m + i) * m + i, &one, sizeof(T), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
}

template <typename T>
gks_status he2hb_t(gks_ctx* c, T* A, int m, int count, T* Q) {
  he2hb_run<T>(c, A, m, count);
  if (Q) {
    identity_fill<T>(Q, m, count, c->stream);
    q1_apply_run<T>(c, A, Q, m, (long long)m * m, m, m, count);
  }
  const int W = 2 * c->band + 1;
  T* Bd = at<T>(c, c->oBd);
  band_pack<T>(A, m, c->sMM, Bd, W, (long long)m * W, m, c->band, count, c->stream);
  band_unpack<T>(Bd, W, (long long)m * W, A, m, c->sMM, m, count, c->stream);
  return cuda_check(c, "gks_he2hb");
}

template <typename T>
gks_status hb2st_t(gks_ctx* c, const T* B, int m, int count, double* d, double* e, T* X, int ncols) {
  if (!hb2st_run<T>(c, B, m, count, d, e))
    return fail(c, GKS_ECUDA, "bulge chasing: cooperative launch refused (not enough resident CTAs)");
  if (X && ncols > 0) {
    T* Xp = at<T>(c, c->oXp);
    const long long sXp = (long long)(m + 2 * c->band) * ncols;
    cudaMemsetAsync(Xp, 0, sizeof(T) * sXp * count, c->stream);
    copy2d<T>(Xp, ncols, sXp, X, ncols, (long long)m * ncols, m, ncols, count, c->stream);
    q2_apply_run<T>(c, Xp, sXp, m, ncols, count);
    copy2d<T>(X, ncols, (long long)m * ncols, Xp, ncols, sXp, m, ncols, count, c->stream);
  }
  return cuda_check(c, "gks_hb2st");
}
}  // namespace

extern "C" {

gks_status gks_he2hb(gks_ctx* ctx, void* A, int64_t m, int64_t count, int dtype, int band, void* Q) {
  if (!ctx || !A || m < 2 || count < 1 || m > 46340 || band < 2 || band > 32) return fail(ctx, GKS_EINVAL, "bad arguments");
  if (dtype != GKS_R64 && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "unknown dtype");
  DeviceGuard dg(ctx->device);
  TwoStageScope ts(ctx, band);
  const int es = dtype == GKS_C128 ? 16 : 8;
  gks_status rc = ensure_ws(ctx, (int)m, (int)m, (int)count, es, 0);
  if (rc) return rc;
  cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus) * count, ctx->stream);
  if (dtype == GKS_R64) return he2hb_t<double>(ctx, static_cast<double*>(A), (int)m, (int)count, static_cast<double*>(Q));
  return he2hb_t<zc>(ctx, static_cast<zc*>(A), (int)m, (int)count, static_cast<zc*>(Q));
}

gks_status gks_hb2st(gks_ctx* ctx, const void* B, int64_t m, int64_t count, int dtype, int band, double* d, double* e,
                     void* X, int64_t ncols) {
  if (!ctx || !B || !d || !e || m < 2 || count < 1 || m > 46340 || band < 2 || band > 32 || ncols < 0 || ncols > m)
    return fail(ctx, GKS_EINVAL, "bad arguments");
  if (dtype != GKS_R64 && dtype != GKS_C128) return fail(ctx, GKS_EINVAL, "unknown dtype");
  DeviceGuard dg(ctx->device);
  TwoStageScope ts(ctx, band);
  const int es = dtype == GKS_C128 ? 16 : 8;
  gks_status rc = ensure_ws(ctx, (int)m, (int)m, (int)count, es, 0);
  if (rc) return rc;
  cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus) * count, ctx->stream);
  if (dtype == GKS_R64)
    return hb2st_t<double>(ctx, static_cast<const double*>(B), (int)m, (int)count, d, e, static_cast<double*>(X),
                           (int)ncols);
  return hb2st_t<zc>(ctx, static_cast<const zc*>(B), (int)m, (int)count, d, e, static_cast<zc*>(X), (int)ncols);
}

gks_status gks_stedc(gks_ctx* ctx, const double* d, const double* e, int64_t m, int64_t count, double* lam,
                     double* Z) {
  if (!ctx || !d || !e || !lam || !Z || m < 1 || count < 1 || m > 46340) return fail(ctx, GKS_EINVAL, "bad arguments");
  DeviceGuard dg(ctx->device);
  gks_status rc = ensure_ws(ctx, (int)m, (int)m, (int)count, 8, 0);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus) * count, s);
  double* dw = at<double>(ctx, ctx->od);
  double* ew = at<double>(ctx, ctx->oe);
  copy2d<double>(dw, (int)m, m, d, (int)m, m, 1, (int)m, (int)count, s);
  copy2d<double>(ew, (int)m, m, e, (int)m, m, 1, (int)m, (int)count, s);
  dc_solve(ctx->dc, dw, ew, m, lam, Z, m * m, ctx->ws + ctx->odc, ctx->st, s, &ctx->prof);
  return cuda_check(ctx, "gks_stedc");
}

}  // extern "C"
