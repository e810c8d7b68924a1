// Internal declarations shared by the translation units of libridc.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/ridc.h"

namespace ridc {

constexpr int kMaxOrder = 12;
constexpr int kMaxSpecies = 2;
constexpr int kMaxPasses = 5;       // solve passes of the mixed forms: 1 + up to 4 refinements
constexpr int kMaxPlanes = kMaxOrder * kMaxSpecies;
constexpr int kMaxStages = 8;       // stages of an ARK predictor (the fourth-order one has 7)
constexpr int kMaxCoefs = 4;        // distinct solve operators (I - a dt D): a = 1 and the
                                    // ARK diagonals (the third-order one adds 1/2, 2/3, 2)
constexpr int kMaxTerms = kMaxOrder;   // terms of an ARK stage right-hand side

// One implicit stage i >= 1 of an ARK predictor (Section II) in delta form. With K^S_j = F_j -
// KN_j (F = f^N + D Y and KN = f^N(Y) of stage j; stage 0 is y_n itself):
//   (I - dt a_ii D) delta_i = dt sum_t w[t] X[src[t]],   Y_i = y_n + delta_i,
// X[2j] = F_j, X[2j+1] = KN_j, and w from a^S_ij (+ a_ii for j = 0) on F_j and
// a^N_ij - a^S_ij (- a_ii for j = 0) on KN_j, in exact rationals (zero terms dropped).
struct ArkStage {
  int coef;                  // index of a_ii in Ctx::coef
  int nterms;
  int src[kMaxTerms];
  double w[kMaxTerms];       // units of dt
};
// Fill the stages of predictor `pred` (RIDC_PRED_ARK3/4): returns the stage count s (the
// last stage is the new solution: both tableaux are stiffly accurate), or 0 for FBE / an
// unknown value. coef[0] = 1 is the correctors' operator; new diagonals are appended.
int ark_plan(int pred, ArkStage* st, double* coef, int* ncoef);
// order p0 of a predictor (0 for an unknown value)
int predictor_order(int pred);
// FP16 form: an operand plane is scaled by 2^k with max|v| 2^k in [2^(K0-1), 2^K0),
// K0 = 15 - ceil(log2 N), so every intermediate of the transform, at most N 2^K0 <= 2^15,
// stays finite in FP16 while small values keep clear of its subnormals
inline int f16_k0(int n) {
  int l = 0;
  while ((1L << l) < (long)n) ++l;
  return 15 - l;
}

inline bool is_mixed(int prec) { return prec == RIDC_MIXED_BF16X3 || prec == RIDC_MIXED_FP16X3; }

// exponent k of the power-of-two scale of an FP16-form plane from the FP32 bits of its
// maximum magnitude: max 2^k in [2^(K0-1), 2^K0). A zero, subnormal or non-finite maximum
// gives k = 0 (zeros stay zeros; Inf and NaN pass through to the non-finite checks); k is
// clamped to [-100, 100] so that 2^k and 2^-(k + table exponent) stay normal FP32 numbers.
__host__ __device__ inline int f16_plane_exp(unsigned maxbits, int k0) {
  const int e = (int)((maxbits >> 23) & 0xFF);
  if (e == 0 || e == 255) return 0;
  int k = k0 - 1 - (e - 127);
  if (k > 100) k = 100;
  if (k < -100) k = -100;
  return k;
}
// 2^k as an FP32 number, |k| <= 126
__host__ __device__ inline float pow2f(int k) {
  union { unsigned u; float f; } v;
  v.u = (unsigned)(127 + k) << 23;
  return v.f;
}

// ---- launch descriptors ---------------------------------------------------------------

// Right-hand side of one advancing level in delta form (the Dy of the base cancels):
//   FBE predictor: r = dt * F^0_n                                      (eq. (pred))
//   ARK stage i:   r = sum_t w_t X_t  (w_t in units of dt already; see ArkStage)
//   corrector:     r = (eta^j_n - eta^{j-1}_{n+1}) + dt (f^N(eta^j_n) - f^N(eta^{j-1}_n))
//                      + dt sum_i w_i F^{j-1}_{b+i}                     (eq. (corr))
// ARK stages (RhsArgs::combo) take the sum of the nnodes terms w_i Fn_i as the whole
// right-hand side; the FBE predictor (eta_j == nullptr) takes w_0 Fn_0.
struct RhsLevel {
  const double* eta_j;    // eta^j_n          [S][N][N]  (nullptr: predictor / ARK stage)
  const double* fN_j;     // f^N(eta^j_n)
  const double* eta_pn;   // eta^{j-1}_{n+1}
  const double* fN_p;     // f^N(eta^{j-1}_n)
  const double* Fn[kMaxOrder];   // F = f^N + D eta at the quadrature nodes
  double w[kMaxOrder];           // dt * quadrature weight per node
  int nnodes;
};

struct RhsArgs {
  RhsLevel lv[kMaxOrder];
  int nlev;
  long plane;             // S * N * N values per level
  double dt;
  double* r;              // [nlev*S][N][N]
  __nv_bfloat16* r_hi;    // split of r along both axes for the tensor-core solve (nullptr:
  __nv_bfloat16* r_lo;    //   FP64 and FP16 forms), layout [plane][gx][gy][N/2][N/2]
  float* r_stage;         // FP16 form: the split values in FP32, same layout (else nullptr)
  unsigned* pmax;         // FP16 form: per-plane max |staged value| (FP32 bits), pass 0
  int n;
  int combo;              // every level is an ARK stage: r = sum_k w_k Fn_k (own kernel)
};

// New state of one advancing level: eta = base + d64 + d32, then f^N(eta) and
// F = f^N + D eta. The solve's increment arrives as an FP64 part and/or an FP32 part (the
// last tensor-core pass); nullptr parts are absent (both absent: eta = base).
struct FinLevel {
  const double* base;     // [S][N][N]
  const double* d64;      // [S][N][N] or nullptr
  const float* d32;       // [S][N][N] or nullptr
  double* eta;            // outputs, [S][N][N]
  double* fN;
  double* F;              // nullptr when no consumer needs f of this level
};

// Where a batched solve left delta: delta = d64 + d32 (either may be nullptr).
struct DeltaParts {
  const double* d64;
  const float* d32;
};

struct FinArgs {
  FinLevel lv[kMaxOrder];
  int nlev;
  int n;
  int kind;
  double c_lap[kMaxSpecies];   // nu_s / h^2
  double c_lap4[kMaxSpecies];  // -4 nu_s / h^2
  double a2h, b2h;             // a / (2h), b / (2h)
  double gsF, gsk;             // Gray-Scott rates
  double gsFk;                 // -(F + k)
};

// ---- the handle -----------------------------------------------------------------------------

struct Ctx {
  // problem
  int kind = 0, dim = 1, n = 0, S = 1, P = 1, prec = RIDC_FP64, n_refine = 0;
  double a = 0, b = 0, gsF = 0, gsk = 0, dt = 0, h = 0;
  double nu[kMaxSpecies] = {0, 0};
  cudaStream_t stream = nullptr;
  int device = 0;

  // schedule state: steps taken by each level since the current start (set_initial or the
  // latest restart), and the top-level steps completed before that start
  long p[kMaxOrder] = {0};
  bool initialised = false;
  long restart_every = 0;    // restart interval in top-level steps (0: none), Section III-E
  long seg_base = 0;

  // quadrature weights w[d][m][i] (units of dt) of the (d+1)-node stencils, exact rationals
  // rounded to FP64; corrector j uses d = p0 + j - 1
  std::vector<double> wq;   // [W][W][W]
  int W = 1;                // p0 + P - 1: the widest stencil's node count

  // predictor (Section II / Theorem 2): FBE or an ARK method of order p0 with nstages stages
  int pred = RIDC_PRED_FBE, p0 = 1, nstages = 1;
  ArkStage stage[kMaxStages];        // stages 1..nstages-1
  double coef[kMaxCoefs] = {1.0};    // diagonal coefficients a of the solve operators
  int ncoef = 1;
  int plane_coef[kMaxPlanes] = {0};  // operator of each plane of the next solve (index in coef)
  double* stF[kMaxStages] = {nullptr};    // stage fields F_i, KN_i (stages 1..nstages-2), and
  double* stKN[kMaxStages] = {nullptr};   // the stage value Y_i that the finalize kernel writes
  double* stY = nullptr;

  // level rings: ring j has cap[j] slots of [S][N][N] values; slot of index t is t % cap[j]
  int cap[kMaxOrder] = {0};
  double* eta[kMaxOrder] = {nullptr};
  double* fN[kMaxOrder] = {nullptr};
  double* Fq[kMaxOrder] = {nullptr};   // F = f^N + D eta (levels with a consumer)

  // work buffers
  long plane = 0;            // S * N^dim
  double* r = nullptr;       // [P*S][N][N]
  double* delta = nullptr;   // [P*S][N][N]  FP64 solution increment (ping)
  double* delta2 = nullptr;  // [P*S][N][N]  (pong, refinement passes)
  float* dinc = nullptr;     // [P*S][N][N]  FP32 increment of the latest tensor-core pass
  double* t1 = nullptr;      // FP64 GEMM intermediates
  double* t2 = nullptr;
  // split operands, ping (xh/xl) and pong (yh/yl); 16-bit words holding BF16 values, or
  // FP16 values in the FP16 form (the tensor maps only move 2-byte elements)
  __nv_bfloat16* xh = nullptr;
  __nv_bfloat16* xl = nullptr;
  __nv_bfloat16* yh = nullptr;
  __nv_bfloat16* yl = nullptr;
  // FP16 form: FP32 staging of the first operand ([P*S][gx][gy][N/2][N/2]), the per-plane
  // maxima of every solve pass ([kMaxPasses][kMaxPlanes], FP32 bits, zeroed per solve) and
  // the exponent of the eigenvector tables' scale 2^qexp
  float* xs = nullptr;
  unsigned* pmax = nullptr;
  int qexp = 0;
  int k0 = 0;                // f16_k0(n)

  // fast-diagonalisation tables (2D): Q[x][k] orthonormal eigenvectors of the 1D Laplacian
  double* Q = nullptr;       // [N][N]   Q, its columns in split order when N is even
  double* Qt = nullptr;      // [N][N]   Q^T, its rows in split order when N is even
  double* inv_den = nullptr; // [ncoef][S][N][N] 1 / (1 - a dt nu_s (lam_ky + lam_kx)), FP64 path
                             //           (split order for ky and kx when N is even)
  float* lam_f = nullptr;    // [N] eigenvalues in split order (even modes, then odd), FP32
  // parity-split eigenvector tables, BF16 (or scaled FP16) hi/lo, each [N][N/2]:
  //   Bf = [Qe^T; Qo^T] (forward products), Bb = [Qe; Qo] (inverse products)
  __nv_bfloat16 *Bfh = nullptr, *Bfl = nullptr, *Bbh = nullptr, *Bbl = nullptr;
  long grows = 0;            // P*S*N: rows of an inverse operand (half those of a forward one)
  // A operands: X = [plane][gx][gy][N/2][N/2] (right-hand side split along both axes),
  // Y = [plane][gy][N][N/2] (first transform, rows kx), W, Z = [plane][N][N] (inverse);
  // X/W share xh/xl and Y/Z share yh/yl, each plane at the same addresses in every layout
  CUtensorMap tm_Xh, tm_Xl, tm_Yh, tm_Yl, tm_Wh, tm_Wl, tm_Zh, tm_Zl, tm_Bfh, tm_Bfl, tm_Bbh, tm_Bbl;

  // 1D: constants of the tridiagonal solves and the quadrature weights, one table: for each
  // operator (I - coef[k] dt D), k < ncoef, a block of oned_table_doubles(n, npad) values
  //   [0, npad]            rho^k
  //   npad+1               periodic: 1 / (1 - rho^n);  Dirichlet: kappa (Sherman-Morrison)
  //   npad+2               rho / mu
  //   [npad+3, npad+3+n)   Dirichlet: g = M^-1 e_{n-1}  (zeros when periodic)
  // then the quadrature weights [W][W][W]
  double* tri = nullptr;
  double* st1d = nullptr;    // 1D ARK stages: F_i and f^N_i of stages 1..s-2, and Y ([2s+1][n])
  int npad = 0;              // n rounded up to a multiple of the 1D block size
  unsigned* sched_dev = nullptr;   // step masks of one 1D advance
  size_t sched_cap = 0;
  long* p_dev = nullptr;

  // staging for host <-> device copies
  double* pinned = nullptr;
  size_t pinned_count = 0;
  int* err_dev = nullptr;    // device-side error flag (timeouts)
  int stall_next_gemm = 0;   // test hook: the next tensor-core GEMM leaves one stage unloaded

  // instrumentation
  int profiling = 0;         // 0 off; 1 every launch; k > 1 the launches of every k-th 2D step
  bool prof_now = false;     // record the launches being issued now
  long prof_steps = 0;       // 2D pipeline steps since ridc_set_initial
  long launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int kind; cudaEvent_t e0, e1; };
  std::vector<Rec> recs;
  size_t ev_next = 0;
  long k_launch[RIDC_KERNEL_COUNT] = {0};
  double k_ms[RIDC_KERNEL_COUNT] = {0};
};

// ---- host helpers -------------------------------------------------------------------------------
int cuda_status(cudaError_t e);
// return the RIDC_* code of a failed call / CUDA call from the enclosing int function
#define RIDC_TRY(expr)                 \
  do {                                 \
    const int rc__ = (expr);           \
    if (rc__ != RIDC_OK) return rc__;  \
  } while (0)
#define RIDC_CUDA(expr) RIDC_TRY(cuda_status(expr))
// device allocation behind the allocation-failure hook of ridc_debug_fail_alloc: cudaMalloc,
// or the caller's allocator (ridc_set_allocator)
cudaError_t dev_malloc(void** p, size_t bytes);
// gives back a dev_malloc pointer (nullptr: nothing). With the caller's allocator the stream
// that used it (nullptr: the device) is synchronised first; cudaFree synchronises by itself.
void dev_free(void* p, cudaStream_t used_on);
// live handles and batches (ridc_set_allocator refuses to switch while any exists)
void live_handles_add(int d);

// The calls of a handle run on the device it was created on: the guard makes that device
// current for the call and gives the caller's current device back on return.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess)
      prev = cur;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Kernel attributes are per device: raise a kernel's dynamic shared-memory limit once on
// each device that launches it (bit d of *done: device d is set up).
template <class Kernel>
inline int raise_smem_limit_once(Kernel kernel, int bytes, std::atomic<unsigned long long>* done) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done->load() & bit) return RIDC_OK;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return cuda_status(e);
  done->fetch_or(bit);
  return RIDC_OK;
}

// SM count of the current device (queried once per device)
inline int current_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  cudaGetDevice(&dev);
  int s = cache[dev & 63].load();
  if (s <= 0) {
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    if (s <= 0) s = 1;
    cache[dev & 63].store(s);
  }
  return s;
}
void prof_begin(Ctx* c, int kind, cudaEvent_t* e0);
void prof_end(Ctx* c, int kind, cudaEvent_t e0);

// lock-step rule (Section III-E): which levels advance in one pipeline step, for a predictor
// of order p0 (corrector j reads a p0+j-node stencil)
unsigned plan_step(int P, const long* p, long target_top, int p0);

// ---- kernel launchers (each returns RIDC_OK or an error code) -------------------------------------
int launch_rhs(Ctx* c, const RhsArgs& a);
int launch_finalize(Ctx* c, const FinArgs& a);
// r' = r - (I - dt nu_s L)(dprev + inc), split to BF16 hi/lo into xh/xl (FP16 form: staged
// in FP32 with the per-plane maxima of solve pass `pass`); the new total dprev + inc is
// written to dout. dprev, inc may be nullptr (absent); with both absent the kernel only
// splits r.
int launch_residual(Ctx* c, int plane0, int nplanes, const double* dprev, const float* inc,
                    double* dout, int pass);
// FP16 form: zero the per-plane maxima of every pass (before a solve's first producer)
int reset_plane_max(Ctx* c);
// FP16 form: scale the staged operand planes [plane0, plane0 + nplanes) by their powers of
// two and split them to FP16 hi/lo into xh/xl (maxima of solve pass `pass`)
int launch_split_f16(Ctx* c, int plane0, int nplanes, int pass);
// out = d64 + d32 elementwise over count values (either part may be nullptr)
int launch_combine(Ctx* c, const double* d64, const float* d32, double* out, long count);
// one transform of the FP64 fast diagonalisation: forward (contract with Q, B = Q^T rows) or
// inverse (B = Q); for even n parity-split (tables in split order), otherwise plain
int launch_gemm_f64(Ctx* c, const double* A, const double* B, double* out, int nplanes, int epi,
                    bool forward);
// pass: the solve pass whose per-plane scales the FP16 form undoes in the last transform
int launch_gemm_sym(Ctx* c, const CUtensorMap* ah, const CUtensorMap* al, const CUtensorMap* bh,
                    const CUtensorMap* bl, int plane0, int nplanes, int mode, __nv_bfloat16* oh,
                    __nv_bfloat16* ol, float* o32, int pass);
// fwd: operands of the forward products (32-value K slices, 64B swizzle); else 64-value
// slices with 128B swizzle
int make_tensor_map(CUtensorMap* tm, const void* base, long rows, long cols, int box_rows,
                    bool fwd);
// column-tile width of the forward parity-split products for side n (the B box height)
int gemm_sym_fwd_bn(int n);
int launch_1d(Ctx* c, long nsteps_pipe, int init_only);
// 1D launch shape: a cluster of min(order, 8) CTAs of ONED_THREADS threads, levels dealt
// round-robin; rows padded to a multiple of ONED_THREADS
constexpr int ONED_THREADS = 256;
constexpr long kOneDMaxSmemDoubles = 28000;   // 224 KB of the 227 KB a CTA may use
inline int oned_cluster(int P) { return P < 8 ? P : 8; }
inline int oned_npad(int n) { return (n + ONED_THREADS - 1) / ONED_THREADS * ONED_THREADS; }
// ark: an ARK predictor also keeps the powers of its stage operator's rho (npad + 1 more)
inline long oned_smem_doubles(int P, int n, int npad, bool ark = false) {
  const long L = (P + oned_cluster(P) - 1) / oned_cluster(P);
  return L * npad + L * n + (ark ? 2L : 1L) * (npad + 1);
}
// 1D solver table of one operator (I - a dt D): rho^k (k <= npad), wrap or kappa, rho/mu, g[n]
inline long oned_table_doubles(int n, int npad) { return (long)npad + 3 + n; }
int launch_check_finite(Ctx* c, const double* x, long count, int* flag_dev);

// epilogue kinds of the FP64 fast-diagonalisation GEMM
enum { EPI_STORE = 0, EPI_SCALE_DEN = 1 };
// modes of the parity-split tensor-core GEMM
enum { SYM_FWD_SPLIT = 0, SYM_FWD_DEN = 1, SYM_BWD_SPLIT = 2, SYM_BWD_F32 = 3 };

}  // namespace ridc
