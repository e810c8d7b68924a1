// C ABI of libridc.so: handle lifetime, the lock-step level scheduler, level-history rings in
// HBM, solver tables, and the per-step driver that chains the device kernels.
//
// Paper: Ong, Melfi & Christlieb, "Parallel Semi-Implicit Time Integrators", arXiv:1209.4297.
//   Section II   eq. (imex_diffusion): FBE step = one solve with (I - dt D).
//   Section III-B eq. (pred), III-C eq. (corr): predictor / corrector; quadrature weights.
//   Section III-E: staggered start-up (level j waits j(j+1)/2 steps), idle tail.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <new>
#include <unordered_map>

#include "ridc_internal.h"

using namespace ridc;

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
extern "C" const char* ridc_error_string(int code) {
  switch (code) {
    case RIDC_OK: return "ok";
    case RIDC_ERR_ARG: return "invalid argument";
    case RIDC_ERR_OOM: return "out of memory";
    case RIDC_ERR_CUDA: return "CUDA error";
    case RIDC_ERR_NONFINITE: return "solution is not finite";
    case RIDC_ERR_TIMEOUT: return "device wait timed out";
    case RIDC_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
  }
}

namespace ridc {

// ---- host-side fault injection (tests): the k-th device allocation from now on fails -------
static std::atomic<long> g_fail_alloc{0};

// ---- the caller's allocator (ridc_set_allocator); sizes are kept for its free ------------
static ridc_alloc_fn g_alloc = nullptr;
static ridc_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::mutex g_alloc_mu;
static std::unordered_map<void*, size_t> g_alloc_sizes;
static std::atomic<long> g_live{0};

void live_handles_add(int d) { g_live.fetch_add(d); }

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1) return cudaErrorMemoryAllocation;
  if (!g_alloc) return cudaMalloc(p, bytes);
  int dev = 0;
  cudaGetDevice(&dev);
  void* q = g_alloc(bytes, dev, g_alloc_ctx);
  if (!q) return cudaErrorMemoryAllocation;
  if (reinterpret_cast<uintptr_t>(q) & 255u) {   // TMA and vector accesses need the alignment
    g_free(q, bytes, dev, g_alloc_ctx);
    return cudaErrorInvalidValue;
  }
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc_sizes[q] = bytes;
  }
  *p = q;
  return cudaSuccess;
}

void dev_free(void* p, cudaStream_t used_on) {
  if (!p) return;
  if (!g_free) {
    cudaFree(p);
    return;
  }
  if (used_on) cudaStreamSynchronize(used_on);
  else cudaDeviceSynchronize();
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = g_alloc_sizes.find(p);
    if (it != g_alloc_sizes.end()) {
      bytes = it->second;
      g_alloc_sizes.erase(it);
    }
  }
  int dev = 0;
  cudaGetDevice(&dev);
  g_free(p, bytes, dev, g_alloc_ctx);
}

extern "C" int ridc_set_allocator(ridc_alloc_fn alloc, ridc_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return RIDC_ERR_ARG;
  if (g_live.load() != 0) return RIDC_ERR_ARG;
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = alloc ? ctx : nullptr;
  return RIDC_OK;
}

extern "C" int ridc_debug_fail_alloc(int k) {
  if (k < 0) return RIDC_ERR_ARG;
  g_fail_alloc.store(k);
  return RIDC_OK;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RIDC_OK;
  if (e == cudaErrorMemoryAllocation) return RIDC_ERR_OOM;
  if (getenv("RIDC_DEBUG")) fprintf(stderr, "[ridc] CUDA error: %s\n", cudaGetErrorString(e));
  return RIDC_ERR_CUDA;
}


// ------------------------------------------------------------------------------------------
// lock-step schedule (Section III-E)
// ------------------------------------------------------------------------------------------
// Corrector j reads a K_j = p0 + j node stencil of level j-1 (Section III-C with p0 = 1 for
// the FBE predictor; a p0-th order predictor needs one node per order gained, Theorem 2).
// Level j may take its step n -> n+1 (n = p[j]) when
//   (a) it has not reached its target: the top level stops at target_top, the lower levels
//       at max(target_top, K_{P-1} - 1), the last index a start-up stencil of the top level
//       reads;
//   (b) its inputs exist: level j-1 holds index max(n+1, K_j - 1) (the stencil ends at
//       t_{n+1}, or at t_{K_j - 1} during start-up);
//   (c) (lower levels only) writing index n+1 into its ring of K_{j+1} + 1 slots does not
//       evict a value level j+1 still reads: level j+1's next stencil starts at
//       b = max(0, p[j+1] + 2 - K_{j+1}), so n - b <= K_{j+1} - 1.
// All tests use the values from before the step, so the levels of one step are independent.
// Rule (b) alone gives the paper's start-up waits j(j+1)/2 (p0 = 1); rule (c) holds lower
// levels back so that memory stays at K_{j+1} + 1 fields per level, after which every level
// lags the one below by exactly one step.
unsigned plan_step(int P, const long* p, long target_top, int p0) {
  if (p[P - 1] >= target_top) return 0;   // the run is complete once the top level arrives
  const long target_low = std::max(target_top, (long)(p0 + P - 2));
  unsigned mask = 0;
  for (int j = 0; j < P; ++j) {
    const long tgt = (j == P - 1) ? target_top : target_low;
    bool ok = p[j] < tgt;
    if (ok && j > 0) ok = p[j - 1] >= std::max(p[j] + 1, (long)(p0 + j - 1));
    if (ok && j < P - 1) ok = p[j] - std::max(0L, p[j + 1] + 1 - p0 - j) <= p0 + j;
    if (ok) mask |= 1u << j;
  }
  return mask;
}

static int ring_cap(int P, int j, int p0) { return j < P - 1 ? p0 + j + 2 : 2; }

// ------------------------------------------------------------------------------------------
// ARK predictors (Section II): the third- and fourth-order IMEX additive Runge-Kutta methods,
// as exact rationals. Row i of A^S holds a^S_i0..a^S_ii, row i of A^N a^N_i0..a^N_i,i-1. The
// third-order tableau is garbled in the paper's source; it is read stage by stage (five
// stages, diagonals 0, 1/2, 2/3, 2, 1), which satisfies every additive-RK order condition to
// order 3. Both methods are stiffly accurate: the last stage is the new solution.
// ------------------------------------------------------------------------------------------
struct Rat {
  long long p, q;   // p / q, q > 0
};
static long long gcdll(long long a, long long b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { const long long t = a % b; a = b; b = t; }
  return a ? a : 1;
}
static Rat rat(long long p, long long q) {
  if (q < 0) { p = -p; q = -q; }
  const long long g = gcdll(p, q);
  return {p / g, q / g};
}
static Rat radd(Rat a, Rat b) { return rat(a.p * b.q + b.p * a.q, a.q * b.q); }
static Rat rneg(Rat a) { return {-a.p, a.q}; }
static double rdbl(Rat a) { return (double)a.p / (double)a.q; }   // both exact: one rounding

struct Tableau {
  int s;
  Rat AS[kMaxStages][kMaxStages];
  Rat AN[kMaxStages][kMaxStages];
};

static void tab_row(Rat* row, std::initializer_list<Rat> v) {
  int k = 0;
  for (const Rat& x : v) row[k++] = x;
}

static bool get_tableau(int pred, Tableau* t) {
  *t = Tableau{};
  for (auto& r : t->AS) for (auto& x : r) x = {0, 1};
  for (auto& r : t->AN) for (auto& x : r) x = {0, 1};
  const Rat z = {0, 1};
  if (pred == RIDC_PRED_ARK3) {
    t->s = 5;
    tab_row(t->AS[1], {z, rat(1, 2)});
    tab_row(t->AS[2], {rat(1, 4), rat(-5, 12), rat(2, 3)});
    tab_row(t->AS[3], {rat(2, 1), rat(-7, 2), rat(1, 2), rat(2, 1)});
    tab_row(t->AS[4], {rat(1, 6), z, rat(2, 3), rat(-5, 6), rat(1, 1)});
    tab_row(t->AN[1], {rat(1, 2)});
    tab_row(t->AN[2], {rat(1, 4), rat(1, 4)});
    tab_row(t->AN[3], {z, rat(1, 1), z});
    tab_row(t->AN[4], {rat(1, 6), z, rat(2, 3), rat(1, 6)});
    return true;
  }
  if (pred == RIDC_PRED_ARK4) {
    t->s = 7;
    tab_row(t->AS[1], {rat(-1, 6), rat(1, 2)});
    tab_row(t->AS[2], {rat(1, 6), rat(-1, 3), rat(1, 2)});
    tab_row(t->AS[3], {rat(3, 8), rat(-3, 8), z, rat(1, 2)});
    tab_row(t->AS[4], {rat(1, 8), z, rat(3, 8), rat(-1, 2), rat(1, 2)});
    tab_row(t->AS[5], {rat(-1, 2), z, rat(3, 1), rat(-3, 1), rat(1, 1), rat(1, 2)});
    tab_row(t->AS[6], {rat(1, 6), z, z, z, rat(2, 3), rat(-1, 2), rat(2, 3)});
    tab_row(t->AN[1], {rat(1, 3)});
    tab_row(t->AN[2], {rat(1, 6), rat(1, 6)});
    tab_row(t->AN[3], {rat(1, 8), z, rat(3, 8)});
    tab_row(t->AN[4], {rat(1, 8), z, rat(3, 8), z});
    tab_row(t->AN[5], {rat(1, 2), z, rat(-3, 2), z, rat(2, 1)});
    tab_row(t->AN[6], {rat(1, 6), z, z, z, rat(2, 3), rat(1, 6)});
    return true;
  }
  return false;
}

int predictor_order(int pred) {
  switch (pred) {
    case RIDC_PRED_FBE: return 1;
    case RIDC_PRED_ARK3: return 3;
    case RIDC_PRED_ARK4: return 4;
    default: return 0;
  }
}

int ark_plan(int pred, ArkStage* st, double* coef, int* ncoef) {
  Tableau t;
  if (!get_tableau(pred, &t)) return 0;
  for (int i = 1; i < t.s; ++i) {
    const Rat aii = t.AS[i][i];
    // operator of this stage: an existing coefficient or a new one
    int k = 0;
    while (k < *ncoef && coef[k] != rdbl(aii)) ++k;
    if (k == *ncoef) {
      if (*ncoef >= kMaxCoefs) return 0;
      coef[(*ncoef)++] = rdbl(aii);
    }
    ArkStage& S = st[i];
    S = ArkStage{};
    S.coef = k;
    for (int j = 0; j < i; ++j) {
      // F_j carries a^S_ij, KN_j carries a^N_ij - a^S_ij; stage 0 adds a_ii K^S_0
      Rat cF = t.AS[i][j], cN = radd(t.AN[i][j], rneg(t.AS[i][j]));
      if (j == 0) {
        cF = radd(cF, aii);
        cN = radd(cN, rneg(aii));
      }
      if (cF.p != 0) { S.src[S.nterms] = 2 * j; S.w[S.nterms++] = rdbl(cF); }
      if (cN.p != 0) { S.src[S.nterms] = 2 * j + 1; S.w[S.nterms++] = rdbl(cN); }
    }
  }
  return t.s;
}

// ------------------------------------------------------------------------------------------
// quadrature weights: exact rationals (Section III-C), rounded once
// ------------------------------------------------------------------------------------------
typedef __int128 i128;

static i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { i128 t = a % b; a = b; b = t; }
  return a;
}

// w = int_m^{m+1} prod_{l != i} (s - l) / (i - l) ds on nodes s = 0..j
static double lagrange_weight(int j, int m, int i) {
  i128 coef[kMaxOrder + 1] = {0};   // coefficients of prod_{l != i} (s - l), ascending powers
  coef[0] = 1;
  int deg = 0;
  i128 denom = 1;
  for (int l = 0; l <= j; ++l) {
    if (l == i) continue;
    for (int q = deg + 1; q >= 1; --q) coef[q] = coef[q - 1] - coef[q] * l;
    coef[0] = -coef[0] * l;
    ++deg;
    denom *= (i - l);
  }
  i128 L = 1;   // lcm(1..deg+1)
  for (int q = 1; q <= deg + 1; ++q) L = L / gcd128(L, q) * q;
  i128 num = 0;
  for (int q = 0; q <= deg; ++q) {
    i128 hi = 1, lo = 1;
    for (int e = 0; e < q + 1; ++e) { hi *= (m + 1); lo *= m; }
    num += coef[q] * (hi - lo) * (L / (q + 1));
  }
  i128 den = L * denom;
  if (den < 0) { den = -den; num = -num; }
  const i128 g = gcd128(num, den);
  if (g > 1) { num /= g; den /= g; }
  // integer part plus a correctly rounded fraction (|rem| < den < 2^53 for order <= 12)
  const i128 ip = num / den, rem = num % den;
  return (double)(long long)ip + (double)(long long)rem / (double)(long long)den;
}

static void fill_weights(int P, double* out) {
  for (int x = 0; x < P * P * P; ++x) out[x] = 0.0;
  for (int j = 1; j < P; ++j)
    for (int m = 0; m < j; ++m)
      for (int i = 0; i <= j; ++i) out[(j * P + m) * P + i] = lagrange_weight(j, m, i);
}

// ------------------------------------------------------------------------------------------
// instrumentation
// ------------------------------------------------------------------------------------------
static cudaEvent_t ev_get(Ctx* c) {
  if (c->ev_next >= c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_next++];
}

void prof_begin(Ctx* c, int kind, cudaEvent_t* e0) {
  (void)kind;
  c->launches++;
  *e0 = nullptr;
  if (!c->prof_now) return;
  *e0 = ev_get(c);
  if (*e0) cudaEventRecord(*e0, c->stream);
}

void prof_end(Ctx* c, int kind, cudaEvent_t e0) {
  if (!c->prof_now || !e0) return;
  cudaEvent_t e1 = ev_get(c);
  if (!e1) return;
  cudaEventRecord(e1, c->stream);
  c->recs.push_back({kind, e0, e1});
}

static void prof_collect(Ctx* c) {
  cudaStreamSynchronize(c->stream);
  for (auto& r : c->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
      c->k_launch[r.kind]++;
      c->k_ms[r.kind] += ms;
    }
  }
  c->recs.clear();
  c->ev_next = 0;
}

}  // namespace ridc

// ------------------------------------------------------------------------------------------
// tables
// ------------------------------------------------------------------------------------------
// Eigenvectors of the 1D cell-centred Laplacian with reflecting ghosts: cosines for the even
// (Neumann) ghost, k = 0..N-1; sines for the odd (Dirichlet) ghost, frequencies K = 1..N.
// Orthonormal columns: Q[x][k]. Eigenvalues lam_K = -(4/h^2) sin^2(pi K / 2N).
static void build_eigen(int n, bool odd, std::vector<double>& Q, std::vector<double>& lam) {
  Q.assign((size_t)n * n, 0.0);
  lam.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const long K = odd ? k + 1 : k;
    const double c = (odd ? (K == n) : (K == 0)) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    const double s = std::sin(pi * (double)K / (2.0 * n));
    lam[k] = -4.0 * (double)n * (double)n * s * s;
    for (int x = 0; x < n; ++x) {
      const long t = (K * (2L * x + 1)) % (4L * n);   // angle = pi t / (2N), reduced exactly
      const double ang = pi * (double)t / (2.0 * n);
      Q[(size_t)x * n + k] = c * (odd ? std::sin(ang) : std::cos(ang));
    }
  }
}

// hi + lo ~= src * 2^e, as BF16 or FP16 pairs (16-bit words of the split operand tables)
static void split_table(const std::vector<double>& src, bool f16, int e,
                        std::vector<__nv_bfloat16>& hi, std::vector<__nv_bfloat16>& lo) {
  hi.resize(src.size());
  lo.resize(src.size());
  const double sc = std::ldexp(1.0, e);
  for (size_t i = 0; i < src.size(); ++i) {
    const double v = src[i] * sc;
    if (f16) {
      const __half h = __float2half_rn((float)v);
      const __half l = __float2half_rn((float)(v - (double)__half2float(h)));
      std::memcpy(&hi[i], &h, 2);
      std::memcpy(&lo[i], &l, 2);
    } else {
      hi[i] = __float2bfloat16_rn((float)v);
      lo[i] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi[i])));
    }
  }
}

template <class T>
static int upload(Ctx* c, T** dst, const std::vector<T>& src) {
  RIDC_CUDA(dev_malloc((void**)dst, src.size() * sizeof(T)));
  return cuda_status(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
}

static int build_tables_2d(Ctx* c) {
  const int n = c->n;
  std::vector<double> Q, lam;
  build_eigen(n, c->kind == RIDC_ADV_DIFF_2D_DIRICHLET, Q, lam);
  std::vector<double> Qt((size_t)n * n);
  for (int x = 0; x < n; ++x)
    for (int k = 0; k < n; ++k) Qt[(size_t)k * n + x] = Q[(size_t)x * n + k];
  if (c->prec == RIDC_FP64) {
    // even n: the parity-split transforms take Q^T with its rows and Q with its columns in
    // split order c = (k % 2) n/2 + k/2 (even modes, then odd), and 1/den in split order too;
    // odd n: plain Q^T and Q, natural order
    const bool split = n % 2 == 0;
    const int H = n / 2;
    auto ord = [&](int k) { return split ? (k % 2) * H + k / 2 : k; };
    std::vector<double> Qa((size_t)n * n), Qb((size_t)n * n), ls(n);
    for (int k = 0; k < n; ++k) {
      ls[ord(k)] = lam[k];
      for (int x = 0; x < n; ++x) {
        Qa[(size_t)x * n + ord(k)] = Q[(size_t)x * n + k];    // Q, columns reordered
        Qb[(size_t)ord(k) * n + x] = Q[(size_t)x * n + k];    // Q^T, rows reordered
      }
    }
    RIDC_TRY(upload(c, &c->Q, Qa));
    RIDC_TRY(upload(c, &c->Qt, Qb));
    // one table per solve operator (I - a dt nu_s L): a = 1, then the ARK diagonals;
    // (a dt) nu_s with a = 1 is exactly dt nu_s
    std::vector<double> inv((size_t)c->ncoef * c->S * n * n);
    for (int k = 0; k < c->ncoef; ++k)
      for (int s = 0; s < c->S; ++s) {
        const double adtnu = (c->coef[k] * c->dt) * c->nu[s];
        double* t = inv.data() + ((size_t)k * c->S + s) * n * n;
        for (int ky = 0; ky < n; ++ky)
          for (int kx = 0; kx < n; ++kx)
            t[(size_t)ky * n + kx] = 1.0 / (1.0 - adtnu * (ls[ky] + ls[kx]));
      }
    RIDC_TRY(upload(c, &c->inv_den, inv));
  } else {
    // parity split: Q[n-1-x][k] = (-1)^k Q[x][k]; Qe[x'][k'] = Q[x'][2k'], Qo[x'][k'] = Q[x'][2k'+1]
    const int H = n / 2;
    std::vector<double> bf((size_t)n * H), bb((size_t)n * H);
    for (int g = 0; g < 2; ++g)
      for (int i = 0; i < H; ++i)
        for (int j = 0; j < H; ++j) {
          bf[((size_t)g * H + i) * H + j] = Q[(size_t)j * n + 2 * i + g];   // Qe^T / Qo^T
          bb[((size_t)g * H + i) * H + j] = Q[(size_t)i * n + 2 * j + g];   // Qe / Qo
        }
    // FP16 form: entries are at most sqrt(2/N) in magnitude; 2^qexp, qexp = 13 +
    // floor(log2(N/2)/2), brings the largest to (2^13, 2^14], inside FP16's range, and keeps
    // the low halves of all but the tiniest entries clear of its subnormals (the products
    // accumulate in FP32, where 2^14 times an operand of at most 2^15 is harmless)
    const bool f16 = c->prec == RIDC_MIXED_FP16X3;
    c->qexp = 0;
    c->k0 = f16_k0(n);
    if (f16) {
      while ((2L << (2 * (c->qexp + 1))) <= (long)n) ++c->qexp;   // 4^(qexp+1) <= n/2
      c->qexp += 13;
    }
    std::vector<__nv_bfloat16> h, l;
    split_table(bf, f16, c->qexp, h, l);
    RIDC_TRY(upload(c, &c->Bfh, h));
    RIDC_TRY(upload(c, &c->Bfl, l));
    split_table(bb, f16, c->qexp, h, l);
    RIDC_TRY(upload(c, &c->Bbh, h));
    RIDC_TRY(upload(c, &c->Bbl, l));
    std::vector<float> lf(n);   // eigenvalues in split order: even modes, then odd modes
    for (int k = 0; k < n; ++k) lf[k] = (float)lam[k < H ? 2 * k : 2 * (k - H) + 1];
    RIDC_TRY(upload(c, &c->lam_f, lf));
  }
  return RIDC_OK;
}

static bool is_1d_dirichlet(int kind) { return kind == RIDC_BURGERS_1D_DIRICHLET; }

// (I - dt nu L) with L the second difference: diagonal 1 + 2 mu, off-diagonals -mu,
// mu = nu dt / h^2. With the shift (S x)_j = x_{j+1} and rho the root in (0, 1) of
// mu rho^2 - (1 + 2 mu) rho + mu = 0 (written without cancellation as
// rho = 2 mu / (1 + 2 mu + sqrt(1 + 4 mu))), M = (mu/rho)(1 - rho S)(1 - rho S^T) equals
//   periodic  (cyclic S):        the matrix itself;
//   Dirichlet (S x)_{n-1} = 0:   the matrix minus mu rho e_{n-1} e_{n-1}^T,
// so the Dirichlet solve is M^-1 plus a Sherman-Morrison correction along g = M^-1 e_{n-1}:
//   x = y - kappa y_{n-1} g,  y = M^-1 r,  kappa = mu rho / (1 + mu rho g_{n-1}).
static int build_tables_1d(Ctx* c) {
  const int n = c->n, npad = c->npad;
  const long T = oned_table_doubles(n, npad);
  std::vector<double> tri((size_t)c->ncoef * T + (size_t)c->W * c->W * c->W, 0.0);
  for (int k = 0; k < c->ncoef; ++k) {
    // operator (I - a dt nu L): mu = nu (a dt) / h^2, with a = 1 exactly nu dt / h^2
    double* t = tri.data() + (size_t)k * T;
    const double mu = c->nu[0] * (c->coef[k] * c->dt) / (c->h * c->h);
    const double rho = 2.0 * mu / (1.0 + 2.0 * mu + std::sqrt(1.0 + 4.0 * mu));
    const double s = rho / mu;
    for (int q = 0; q <= npad; ++q) t[q] = std::pow(rho, (double)q);
    t[npad + 2] = s;
    if (is_1d_dirichlet(c->kind)) {
      // g = M^-1 e_{n-1}: z_j = rho^(n-1-j), then g_j = s z_j + rho g_{j-1}
      double* gv = t + npad + 3;
      double prev = 0.0;
      for (int j = 0; j < n; ++j) {
        prev = s * std::pow(rho, (double)(n - 1 - j)) + rho * prev;
        gv[j] = prev;
      }
      t[npad + 1] = mu * rho / (1.0 + mu * rho * gv[n - 1]);
    } else {
      t[npad + 1] = 1.0 / (1.0 - std::pow(rho, (double)n));
    }
  }
  fill_weights(c->W, tri.data() + (size_t)c->ncoef * T);
  return upload(c, &c->tri, tri);
}

// ------------------------------------------------------------------------------------------
// lifetime
// ------------------------------------------------------------------------------------------
static void free_all(Ctx* c) {
  auto f = [c](void* p) { dev_free(p, c->stream); };
  for (int j = 0; j < kMaxOrder; ++j) { f(c->eta[j]); f(c->fN[j]); f(c->Fq[j]); }
  f(c->r); f(c->delta); f(c->delta2); f(c->dinc); f(c->t1); f(c->t2); f(c->xh); f(c->xl); f(c->yh); f(c->yl);
  f(c->Q); f(c->Qt); f(c->inv_den); f(c->lam_f); f(c->Bfh); f(c->Bfl); f(c->Bbh); f(c->Bbl);
  f(c->xs); f(c->pmax);
  f(c->tri); f(c->sched_dev); f(c->p_dev); f(c->err_dev);
  for (int i = 0; i < kMaxStages; ++i) { f(c->stF[i]); f(c->stKN[i]); }
  f(c->stY); f(c->st1d);
  if (c->pinned) cudaFreeHost(c->pinned);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
}

static int create_impl(Ctx* c, const ridc_problem* pr, const ridc_grid* g, const double* nu,
                       double dt, int order, void* stream) {
  c->kind = pr->kind;
  c->a = pr->a; c->b = pr->b; c->gsF = pr->F; c->gsk = pr->k;
  c->prec = pr->precision;
  c->n_refine = pr->n_refine;
  c->restart_every = pr->restart_every;
  c->dim = g->dim;
  c->n = g->n;
  c->P = order;
  c->dt = dt;
  c->stream = (cudaStream_t)stream;
  c->S = (pr->kind == RIDC_GRAY_SCOTT_2D_NEUMANN) ? 2 : 1;
  for (int s = 0; s < c->S; ++s) c->nu[s] = nu[s];
  c->h = is_1d_dirichlet(c->kind) ? 1.0 / (c->n + 1) : 1.0 / c->n;
  c->npad = oned_npad(c->n);
  RIDC_CUDA(cudaGetDevice(&c->device));

  const long n = c->n;
  c->plane = (c->dim == 1) ? n : (long)c->S * n * n;
  c->pred = pr->predictor;
  c->p0 = predictor_order(pr->predictor);
  c->W = c->p0 + order - 1;
  c->ncoef = 1;
  c->coef[0] = 1.0;
  c->nstages = 1;
  if (c->pred != RIDC_PRED_FBE) {
    c->nstages = ark_plan(c->pred, c->stage, c->coef, &c->ncoef);
    if (c->nstages < 2) return RIDC_ERR_ARG;
  }
  std::vector<double> w((size_t)c->W * c->W * c->W);
  fill_weights(c->W, w.data());
  c->wq = w;

  const size_t pb = (size_t)c->plane * sizeof(double);
  // ARK stages 1..s-2 keep F and f^N of their stage value for the later stages; the stage
  // value itself is written to one scratch field
  if (c->dim == 2) {
    for (int i = 1; i + 1 < c->nstages; ++i) {
      RIDC_CUDA(dev_malloc((void**)&c->stF[i], pb));
      RIDC_CUDA(dev_malloc((void**)&c->stKN[i], pb));
    }
    if (c->nstages > 1) RIDC_CUDA(dev_malloc((void**)&c->stY, pb));
  } else if (c->nstages > 1) {
    RIDC_CUDA(dev_malloc((void**)&c->st1d, (size_t)(2 * c->nstages + 1) * pb));
  }
  for (int j = 0; j < order; ++j) {
    c->cap[j] = ring_cap(order, j, c->p0);
    RIDC_CUDA(dev_malloc((void**)&c->eta[j], c->cap[j] * pb));
    RIDC_CUDA(dev_malloc((void**)&c->fN[j], c->cap[j] * pb));
    if (j < order - 1 || j == 0) RIDC_CUDA(dev_malloc((void**)&c->Fq[j], c->cap[j] * pb));
  }
  RIDC_CUDA(dev_malloc((void**)&c->r, (size_t)order * pb));
  RIDC_CUDA(dev_malloc((void**)&c->delta, (size_t)order * pb));
  RIDC_CUDA(dev_malloc((void**)&c->err_dev, sizeof(int)));
  RIDC_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
  if (c->dim == 1) {
    RIDC_TRY(build_tables_1d(c));
    RIDC_CUDA(dev_malloc((void**)&c->p_dev, kMaxOrder * sizeof(long)));
  } else {
    if (c->prec == RIDC_FP64) {
      RIDC_CUDA(dev_malloc((void**)&c->t1, (size_t)order * pb));
      RIDC_CUDA(dev_malloc((void**)&c->t2, (size_t)order * pb));
    } else {
      RIDC_CUDA(dev_malloc((void**)&c->delta2, (size_t)order * pb));
      RIDC_CUDA(dev_malloc((void**)&c->dinc, (size_t)order * c->plane * sizeof(float)));
      const size_t hb = (size_t)order * c->plane * sizeof(__nv_bfloat16);
      RIDC_CUDA(dev_malloc((void**)&c->xh, hb));
      RIDC_CUDA(dev_malloc((void**)&c->xl, hb));
      RIDC_CUDA(dev_malloc((void**)&c->yh, hb));
      RIDC_CUDA(dev_malloc((void**)&c->yl, hb));
      if (c->prec == RIDC_MIXED_FP16X3) {
        RIDC_CUDA(dev_malloc((void**)&c->xs, (size_t)order * c->plane * sizeof(float)));
        RIDC_CUDA(dev_malloc((void**)&c->pmax, (size_t)kMaxPasses * kMaxPlanes * sizeof(unsigned)));
      }
    }
    RIDC_TRY(build_tables_2d(c));
    if (is_mixed(c->prec)) {
      const long rows = (long)order * c->S * n, H = n / 2;
      c->grows = rows;
      // forward operands (X, Y, forward tables) and inverse ones (W, Z, inverse tables)
      RIDC_TRY(make_tensor_map(&c->tm_Xh, c->xh, 2 * rows, H, 128, true));
      RIDC_TRY(make_tensor_map(&c->tm_Xl, c->xl, 2 * rows, H, 128, true));
      RIDC_TRY(make_tensor_map(&c->tm_Yh, c->yh, 2 * rows, H, 128, true));
      RIDC_TRY(make_tensor_map(&c->tm_Yl, c->yl, 2 * rows, H, 128, true));
      RIDC_TRY(make_tensor_map(&c->tm_Wh, c->xh, rows, n, 128, false));
      RIDC_TRY(make_tensor_map(&c->tm_Wl, c->xl, rows, n, 128, false));
      RIDC_TRY(make_tensor_map(&c->tm_Zh, c->yh, rows, n, 128, false));
      RIDC_TRY(make_tensor_map(&c->tm_Zl, c->yl, rows, n, 128, false));
      RIDC_TRY(make_tensor_map(&c->tm_Bfh, c->Bfh, n, H, gemm_sym_fwd_bn(n), true));
      RIDC_TRY(make_tensor_map(&c->tm_Bfl, c->Bfl, n, H, gemm_sym_fwd_bn(n), true));
      RIDC_TRY(make_tensor_map(&c->tm_Bbh, c->Bbh, n, H, 128, false));
      RIDC_TRY(make_tensor_map(&c->tm_Bbl, c->Bbl, n, H, 128, false));
    }
  }
  RIDC_CUDA(cudaDeviceSynchronize());
  return RIDC_OK;
}

extern "C" int ridc_create(const ridc_problem* pr, const ridc_grid* g, const double* nu,
                           double dt, int order, void* stream, ridc_handle* out) {
  if (!pr || !g || !nu || !out) return RIDC_ERR_ARG;
  if (order < 1 || order > kMaxOrder) return RIDC_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return RIDC_ERR_ARG;
  if (pr->restart_every < 0) return RIDC_ERR_ARG;
  if (pr->kind < 0 || pr->kind > 4) return RIDC_ERR_ARG;
  if (pr->precision != RIDC_FP64 && !is_mixed(pr->precision)) return RIDC_ERR_ARG;
  if (pr->n_refine < 0 || pr->n_refine > 4) return RIDC_ERR_ARG;
  if (predictor_order(pr->predictor) == 0) return RIDC_ERR_ARG;
  // the widest quadrature stencil has p0 + order - 1 nodes (at most 12)
  if (predictor_order(pr->predictor) + order - 1 > kMaxOrder) return RIDC_ERR_UNSUPPORTED;
  const int S = (pr->kind == RIDC_GRAY_SCOTT_2D_NEUMANN) ? 2 : 1;
  for (int s = 0; s < S; ++s)
    if (!(nu[s] > 0.0) || !std::isfinite(nu[s])) return RIDC_ERR_ARG;
  if (pr->kind == RIDC_ADV_DIFF_1D_PERIODIC || pr->kind == RIDC_ADV_DIFF_1D_UPWIND_PERIODIC ||
      pr->kind == RIDC_BURGERS_1D_DIRICHLET) {
    if (g->dim != 1 || g->n < 8) return RIDC_ERR_ARG;
    if (pr->precision != RIDC_FP64) return RIDC_ERR_UNSUPPORTED;
    // shared-memory rows of the levels one CTA carries
    if (oned_smem_doubles(order, g->n, oned_npad(g->n), pr->predictor != RIDC_PRED_FBE) >
        kOneDMaxSmemDoubles)
      return RIDC_ERR_UNSUPPORTED;
  } else {
    if (g->dim != 2 || g->n < 4) return RIDC_ERR_ARG;
    if (is_mixed(pr->precision) && ((g->n % 256) != 0 || g->n > 4096))
      return RIDC_ERR_UNSUPPORTED;
    if (g->n > 16384) return RIDC_ERR_UNSUPPORTED;
  }
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return RIDC_ERR_OOM;
  const int rc = create_impl(c, pr, g, nu, dt, order, stream);
  if (rc != RIDC_OK) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = reinterpret_cast<ridc_handle>(c);
  live_handles_add(1);
  return RIDC_OK;
}

extern "C" void ridc_destroy(ridc_handle h) {
  if (!h) return;
  Ctx* c = reinterpret_cast<Ctx*>(h);
  DeviceGuard dg(c->device);
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  live_handles_add(-1);
}

static Ctx* ctx_of(ridc_handle h) { return reinterpret_cast<Ctx*>(h); }

static int ensure_pinned(Ctx* c, size_t count) {
  if (c->pinned_count >= count) return RIDC_OK;
  if (c->pinned) cudaFreeHost(c->pinned);
  c->pinned = nullptr;
  c->pinned_count = 0;
  RIDC_CUDA(cudaMallocHost((void**)&c->pinned, count * sizeof(double)));
  c->pinned_count = count;
  return RIDC_OK;
}

// constants of the finalize kernel, computed once in FP64 on the host
static void fill_fin_consts(Ctx* c, FinArgs* fa) {
  for (int s = 0; s < c->S; ++s) {
    fa->c_lap[s] = c->nu[s] / (c->h * c->h);
    fa->c_lap4[s] = -4.0 * fa->c_lap[s];
  }
  fa->a2h = c->a / (2.0 * c->h);
  fa->b2h = c->b / (2.0 * c->h);
  fa->gsF = c->gsF;
  fa->gsk = c->gsk;
  fa->gsFk = -(c->gsF + c->gsk);
}

// ------------------------------------------------------------------------------------------
// initial state
// ------------------------------------------------------------------------------------------
// Every level's slot 0 := u0 (host or device), with f^N and F of that state; p := 0.
static int start_from(Ctx* c, const double* u0, int on_device) {
  const size_t bytes = (size_t)c->plane * sizeof(double);
  if (on_device) {
    RIDC_CUDA(cudaMemcpyAsync(c->eta[0], u0, bytes, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    RIDC_CUDA(cudaStreamSynchronize(c->stream));   // staging buffer may still be in use
    RIDC_TRY(ensure_pinned(c, (size_t)c->plane));
    memcpy(c->pinned, u0, bytes);
    RIDC_CUDA(cudaMemcpyAsync(c->eta[0], c->pinned, bytes, cudaMemcpyHostToDevice, c->stream));
  }
  // every other ring slot is filled with NaN (all bits set): a read of a slot the schedule
  // has not written yet would show up as NaN in the results instead of passing unnoticed
  const size_t slot_bytes = (size_t)c->plane * sizeof(double);
  for (int j = 0; j < c->P; ++j) {
    double* rings[3] = {c->eta[j], c->fN[j], c->Fq[j]};
    for (double* ring : rings) {
      if (!ring) continue;
      const size_t skip = (ring == c->eta[0]) ? 1 : 0;   // keeps the new initial state
      RIDC_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(ring) + skip * slot_bytes, 0xFF,
                                (c->cap[j] - skip) * slot_bytes, c->stream));
    }
  }
  // f^N and F of the initial state, written into slot 0 of level 0
  if (c->dim == 2) {
    FinArgs fa{};
    fa.nlev = 1;
    fa.n = c->n;
    fa.kind = c->kind;
    fill_fin_consts(c, &fa);
    fa.lv[0] = {c->eta[0], nullptr, nullptr, c->eta[0], c->fN[0], c->Fq[0]};
    RIDC_TRY(launch_finalize(c, fa));
  } else {
    RIDC_CUDA(cudaMemsetAsync(c->p_dev, 0, kMaxOrder * sizeof(long), c->stream));
    RIDC_TRY(launch_1d(c, 0, 1));   // evaluates f^N and F of slot 0 only
  }
  // every level starts from the same data
  for (int j = 1; j < c->P; ++j) {
    RIDC_CUDA(cudaMemcpyAsync(c->eta[j], c->eta[0], bytes, cudaMemcpyDeviceToDevice, c->stream));
    RIDC_CUDA(cudaMemcpyAsync(c->fN[j], c->fN[0], bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (c->Fq[j])
      RIDC_CUDA(cudaMemcpyAsync(c->Fq[j], c->Fq[0], bytes, cudaMemcpyDeviceToDevice, c->stream));
  }
  for (int j = 0; j < kMaxOrder; ++j) c->p[j] = 0;
  c->initialised = true;
  return RIDC_OK;
}

extern "C" int ridc_set_initial(ridc_handle h, const double* u0, size_t count, int on_device) {
  Ctx* c = ctx_of(h);
  if (!c || !u0 || count != (size_t)c->plane) return RIDC_ERR_ARG;
  DeviceGuard dg(c->device);
  c->seg_base = 0;
  c->prof_steps = 0;
  return start_from(c, u0, on_device);
}

// ------------------------------------------------------------------------------------------
// the batched implicit solve (I - dt nu_s L) delta = r on nplanes planes (2D)
// ------------------------------------------------------------------------------------------
// Fast diagonalisation: delta = Q ((Q^T R Q) ./ den) Q^T, den = 1 - dt nu_s (lam_ky + lam_kx).
// Each GEMM contracts the contiguous axis of every plane and stores its result transposed,
// so four "rows x Q" products realise the two-sided transform (the mixed form splits each
// into even and odd eigenvector halves, see gemm_sym.cu).
// Mixed solve of planes [p0, p0 + np) on the handle's stream.
static int solve_group_mixed(Ctx* c, int p0, int np, bool rhs_split_done, const double** total) {
  const double* tot = nullptr;
  for (int pass = 0; pass <= c->n_refine; ++pass) {
    if (pass == 0) {
      if (!rhs_split_done) {
        if (c->prec == RIDC_MIXED_FP16X3) RIDC_TRY(reset_plane_max(c));
        RIDC_TRY(launch_residual(c, p0, np, nullptr, nullptr, nullptr, 0));
      }
    } else {
      double* dst = (tot == c->delta) ? c->delta2 : c->delta;
      RIDC_TRY(launch_residual(c, p0, np, tot, c->dinc, dst, pass));
      tot = dst;
    }
    // x forward of the operand split along both axes (right-hand side or residual kernel)
    // -> Y, rows kx per y parity;  y forward, divided by the denominators -> W
    RIDC_TRY(launch_gemm_sym(c, &c->tm_Xh, &c->tm_Xl, &c->tm_Bfh, &c->tm_Bfl, p0, np,
                             SYM_FWD_SPLIT, c->yh, c->yl, nullptr, pass));
    RIDC_TRY(launch_gemm_sym(c, &c->tm_Yh, &c->tm_Yl, &c->tm_Bfh, &c->tm_Bfl, p0, np,
                             SYM_FWD_DEN, c->xh, c->xl, nullptr, pass));
    // x inverse -> Z;  y inverse -> FP32 increment
    RIDC_TRY(launch_gemm_sym(c, &c->tm_Wh, &c->tm_Wl, &c->tm_Bbh, &c->tm_Bbl, p0, np,
                             SYM_BWD_SPLIT, c->yh, c->yl, nullptr, pass));
    RIDC_TRY(launch_gemm_sym(c, &c->tm_Zh, &c->tm_Zl, &c->tm_Bbh, &c->tm_Bbl, p0, np,
                             SYM_BWD_F32, nullptr, nullptr, c->dinc, pass));
  }
  *total = tot;
  return RIDC_OK;
}

// The mixed form: pass 0 solves from the split right-hand side; every refinement pass forms
// the FP64 residual of the running total (ping-pong buffers, so neighbours read a consistent
// total) and solves for the next FP32 increment. The result stays split as total + increment.
static int solve_planes_dev(Ctx* c, int nplanes, bool rhs_split_done, DeltaParts* out) {
  if (c->prec == RIDC_FP64) {
    // forward products take Q^T (rows in split order for even n), inverse products Q
    RIDC_TRY(launch_gemm_f64(c, c->r, c->Qt, c->t1, nplanes, EPI_STORE, true));
    RIDC_TRY(launch_gemm_f64(c, c->t1, c->Qt, c->t2, nplanes, EPI_SCALE_DEN, true));
    RIDC_TRY(launch_gemm_f64(c, c->t2, c->Q, c->t1, nplanes, EPI_STORE, false));
    RIDC_TRY(launch_gemm_f64(c, c->t1, c->Q, c->delta, nplanes, EPI_STORE, false));
    *out = {c->delta, nullptr};
    return RIDC_OK;
  }
  const double* total = nullptr;
  RIDC_TRY(solve_group_mixed(c, 0, nplanes, rhs_split_done, &total));
  *out = {total, c->dinc};
  return RIDC_OK;
}

extern "C" int ridc_solve_planes(ridc_handle h, const double* r, double* delta, int nplanes,
                                 int on_device) {
  Ctx* c = ctx_of(h);
  if (!c || !r || !delta) return RIDC_ERR_ARG;
  DeviceGuard dg(c->device);
  if (c->dim != 2) return RIDC_ERR_UNSUPPORTED;
  if (nplanes < 1 || nplanes > c->P * c->S) return RIDC_ERR_ARG;
  const long nn = (long)c->n * c->n;
  const size_t bytes = (size_t)nplanes * nn * sizeof(double);
  RIDC_CUDA(cudaMemcpyAsync(c->r, r, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice, c->stream));
  DeltaParts parts;
  RIDC_TRY(solve_planes_dev(c, nplanes, false, &parts));
  const double* src = parts.d64;
  if (parts.d32) {   // fold the FP32 increment into an FP64 buffer the solve no longer needs
    double* dst = (parts.d64 == c->delta) ? c->delta2 : c->delta;
    RIDC_TRY(launch_combine(c, parts.d64, parts.d32, dst, (long)nplanes * nn));
    src = dst;
  }
  RIDC_CUDA(cudaMemcpyAsync(delta, src, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyDeviceToHost, c->stream));
  RIDC_CUDA(cudaStreamSynchronize(c->stream));
  int err = 0;
  RIDC_CUDA(cudaMemcpy(&err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {   // reported once: the flag is cleared for the calls that follow
    RIDC_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
    return RIDC_ERR_TIMEOUT;
  }
  return RIDC_OK;
}

// ------------------------------------------------------------------------------------------
// one pipeline step in 2D
// ------------------------------------------------------------------------------------------
static inline double* slot_ptr(Ctx* c, double* ring, int j, long t) {
  return ring + (size_t)(t % c->cap[j]) * c->plane;
}

static int step_2d_launch(Ctx* c, unsigned mask);

static int step_2d(Ctx* c, unsigned mask) {
  // with a sampling period k > 1 only every k-th step of an integration is timed
  c->prof_now = c->profiling == 1 || (c->profiling > 1 && c->prof_steps % c->profiling == 0);
  c->prof_steps++;
  const int rc = step_2d_launch(c, mask);
  c->prof_now = c->profiling == 1;
  return rc;
}

// Level 0's step n -> n+1 with an ARK predictor (Section II), stage by stage: each implicit
// stage forms its right-hand side from the earlier stages' F and f^N (ArkStage), solves with
// (I - a_ii dt D) on the same batched solver (per-plane operators), and evaluates F and f^N of
// its stage value; the last stage is the new solution and goes into level 0's ring. It runs
// ahead of the correctors' batched step: the levels of one pipeline step are independent.
static int ark_predictor_step(Ctx* c) {
  const long n = c->p[0];
  const double* y = slot_ptr(c, c->eta[0], 0, n);
  const double* X[2 * kMaxStages] = {nullptr};
  X[0] = slot_ptr(c, c->Fq[0], 0, n);
  X[1] = slot_ptr(c, c->fN[0], 0, n);
  for (int i = 1; i + 1 < c->nstages; ++i) {
    X[2 * i] = c->stF[i];
    X[2 * i + 1] = c->stKN[i];
  }
  const bool f16 = c->prec == RIDC_MIXED_FP16X3;
  for (int i = 1; i < c->nstages; ++i) {
    const ArkStage& st = c->stage[i];
    RhsArgs ra{};
    RhsLevel& L = ra.lv[0];
    L.eta_j = nullptr;
    for (int t = 0; t < st.nterms; ++t) {
      L.Fn[t] = X[st.src[t]];
      L.w[t] = c->dt * st.w[t];
    }
    L.nnodes = st.nterms;
    ra.nlev = 1;
    ra.combo = 1;
    ra.plane = c->plane;
    ra.dt = c->dt;
    ra.r = c->r;
    ra.r_hi = (c->prec == RIDC_MIXED_BF16X3) ? c->xh : nullptr;
    ra.r_lo = (c->prec == RIDC_MIXED_BF16X3) ? c->xl : nullptr;
    ra.r_stage = f16 ? c->xs : nullptr;
    ra.pmax = f16 ? c->pmax : nullptr;
    ra.n = c->n;
    if (f16) RIDC_TRY(reset_plane_max(c));
    RIDC_TRY(launch_rhs(c, ra));
    if (f16) RIDC_TRY(launch_split_f16(c, 0, c->S, 0));
    for (int q = 0; q < c->S; ++q) c->plane_coef[q] = st.coef;
    DeltaParts parts;
    const int rc = solve_planes_dev(c, c->S, true, &parts);
    for (int q = 0; q < c->S; ++q) c->plane_coef[q] = 0;
    RIDC_TRY(rc);
    FinArgs fa{};
    fa.n = c->n;
    fa.kind = c->kind;
    fill_fin_consts(c, &fa);
    fa.nlev = 1;
    const bool last = i == c->nstages - 1;
    FinLevel& Fl = fa.lv[0];
    Fl.base = y;
    Fl.d64 = parts.d64;
    Fl.d32 = parts.d32;
    Fl.eta = last ? slot_ptr(c, c->eta[0], 0, n + 1) : c->stY;
    Fl.fN = last ? slot_ptr(c, c->fN[0], 0, n + 1) : c->stKN[i];
    Fl.F = last ? (c->Fq[0] ? slot_ptr(c, c->Fq[0], 0, n + 1) : nullptr) : c->stF[i];
    RIDC_TRY(launch_finalize(c, fa));
  }
  return RIDC_OK;
}

static int levels_step_2d(Ctx* c, unsigned mask);

static int step_2d_launch(Ctx* c, unsigned mask) {
  const bool ark = c->nstages > 1;
  if (ark && (mask & 1u)) RIDC_TRY(ark_predictor_step(c));
  const unsigned rest = ark ? (mask & ~1u) : mask;
  if (rest) RIDC_TRY(levels_step_2d(c, rest));
  for (int j = 0; j < c->P; ++j)
    if (mask & (1u << j)) c->p[j]++;
  return RIDC_OK;
}

// The FBE predictor (if in the mask) and the correctors of one pipeline step: one fused
// right-hand-side launch, one batched solve, one finalize launch. Does not advance c->p.
static int levels_step_2d(Ctx* c, unsigned mask) {
  RhsArgs ra{};
  FinArgs fa{};
  fa.n = c->n;
  fa.kind = c->kind;
  fill_fin_consts(c, &fa);
  const int P = c->P;
  int na = 0;
  for (int j = 0; j < P; ++j) {
    if (!(mask & (1u << j))) continue;
    const long n = c->p[j];
    RhsLevel& L = ra.lv[na];
    const double* base;
    if (j == 0) {
      L.eta_j = nullptr;
      L.Fn[0] = slot_ptr(c, c->Fq[0], 0, n);
      L.w[0] = c->dt;
      L.nnodes = 1;
      base = slot_ptr(c, c->eta[0], 0, n);
    } else {
      L.eta_j = slot_ptr(c, c->eta[j], j, n);
      L.fN_j = slot_ptr(c, c->fN[j], j, n);
      L.eta_pn = slot_ptr(c, c->eta[j - 1], j - 1, n + 1);
      L.fN_p = slot_ptr(c, c->fN[j - 1], j - 1, n);
      // K-node stencil of level j-1 (K = p0 + j): t_b..t_{b+K-1}, interval m = n - b
      const int K = c->p0 + j, d = K - 1, W = c->W;
      const long b = std::max(0L, n + 2 - K);
      const long m = n - b;
      for (int i = 0; i < K; ++i) {
        L.Fn[i] = slot_ptr(c, c->Fq[j - 1], j - 1, b + i);
        L.w[i] = c->dt * c->wq[((size_t)d * W + m) * W + i];
      }
      L.nnodes = K;
      base = L.eta_pn;
    }
    FinLevel& Fl = fa.lv[na];
    Fl.base = base;
    Fl.d64 = nullptr;   // set after the solve, which decides where delta lives
    Fl.d32 = nullptr;
    Fl.eta = slot_ptr(c, c->eta[j], j, n + 1);
    Fl.fN = slot_ptr(c, c->fN[j], j, n + 1);
    Fl.F = c->Fq[j] ? slot_ptr(c, c->Fq[j], j, n + 1) : nullptr;
    ++na;
  }
  if (na == 0) return RIDC_OK;
  ra.nlev = na;
  ra.plane = c->plane;
  ra.dt = c->dt;
  ra.r = c->r;
  ra.r_hi = (c->prec == RIDC_MIXED_BF16X3) ? c->xh : nullptr;
  ra.r_lo = (c->prec == RIDC_MIXED_BF16X3) ? c->xl : nullptr;
  const bool f16 = c->prec == RIDC_MIXED_FP16X3;
  ra.r_stage = f16 ? c->xs : nullptr;
  ra.pmax = f16 ? c->pmax : nullptr;   // pass 0
  ra.n = c->n;
  fa.nlev = na;
  if (f16) RIDC_TRY(reset_plane_max(c));
  RIDC_TRY(launch_rhs(c, ra));
  if (f16) RIDC_TRY(launch_split_f16(c, 0, na * c->S, 0));
  DeltaParts parts;
  RIDC_TRY(solve_planes_dev(c, na * c->S, true, &parts));
  for (int q = 0; q < na; ++q) {
    fa.lv[q].d64 = parts.d64 ? parts.d64 + (size_t)q * c->plane : nullptr;
    fa.lv[q].d32 = parts.d32 ? parts.d32 + (size_t)q * c->plane : nullptr;
  }
  RIDC_TRY(launch_finalize(c, fa));
  return RIDC_OK;
}

// Advance the top level by nsteps within the current start (no restart boundary inside).
static int advance_run(Ctx* c, long nsteps) {
  const long target = c->p[c->P - 1] + nsteps;
  if (c->dim == 1) {
    // plan on the host (the same rule the device replays), then one persistent launch
    std::vector<unsigned> masks;
    long p[kMaxOrder];
    for (int j = 0; j < kMaxOrder; ++j) p[j] = c->p[j];
    for (;;) {
      const unsigned m = plan_step(c->P, p, target, c->p0);
      if (!m) break;
      masks.push_back(m);
      for (int j = 0; j < c->P; ++j)
        if (m & (1u << j)) p[j]++;
    }
    if (p[c->P - 1] != target) return RIDC_ERR_CUDA;   // schedule stalled: cannot happen
    if (masks.size() > c->sched_cap) {
      dev_free(c->sched_dev, c->stream);   // the previous 1D launch may still read it
      c->sched_dev = nullptr;
      c->sched_cap = 0;
      RIDC_CUDA(dev_malloc((void**)&c->sched_dev, masks.size() * sizeof(unsigned)));
      c->sched_cap = masks.size();
    }
    RIDC_CUDA(cudaMemcpyAsync(c->sched_dev, masks.data(), masks.size() * sizeof(unsigned),
                              cudaMemcpyHostToDevice, c->stream));
    RIDC_CUDA(cudaMemcpyAsync(c->p_dev, c->p, kMaxOrder * sizeof(long), cudaMemcpyHostToDevice,
                              c->stream));
    // the pageable sources above are consumed before cudaMemcpyAsync returns
    RIDC_TRY(launch_1d(c, (long)masks.size(), 0));
    for (int j = 0; j < c->P; ++j) c->p[j] = p[j];
    return RIDC_OK;
  }
  for (;;) {
    const unsigned m = plan_step(c->P, c->p, target, c->p0);
    if (!m) break;
    RIDC_TRY(step_2d(c, m));
  }
  return c->p[c->P - 1] == target ? RIDC_OK : RIDC_ERR_CUDA;
}

extern "C" int ridc_advance(ridc_handle h, long nsteps) {
  Ctx* c = ctx_of(h);
  if (!c || nsteps < 0) return RIDC_ERR_ARG;
  DeviceGuard dg(c->device);
  if (!c->initialised) return RIDC_ERR_ARG;
  const long R = c->restart_every;
  while (nsteps > 0) {
    // with restarts, a run never crosses the next restart time (Section III-E): all levels
    // drain to it, and the most corrected solution there starts a fresh computation
    const long k = (R > 0) ? std::min(nsteps, R - c->p[c->P - 1]) : nsteps;
    RIDC_TRY(advance_run(c, k));
    nsteps -= k;
    if (R > 0 && c->p[c->P - 1] == R && c->P > 1) {
      const int top = c->P - 1;
      RIDC_TRY(start_from(c, slot_ptr(c, c->eta[top], top, R), 1));
      c->seg_base += R;
    } else if (R > 0 && c->p[c->P - 1] == R) {
      // one level: restarting from its own newest state changes nothing but the index of
      // the current start; move that state (and its f^N, F) to slot 0
      const long t = c->p[0];
      if (t % c->cap[0] != 0) {
        const size_t bytes = (size_t)c->plane * sizeof(double);
        double* rings[3] = {c->eta[0], c->fN[0], c->Fq[0]};
        for (double* ring : rings)
          if (ring)
            RIDC_CUDA(cudaMemcpyAsync(ring, slot_ptr(c, ring, 0, t), bytes,
                                      cudaMemcpyDeviceToDevice, c->stream));
      }
      c->p[0] = 0;
      c->seg_base += R;
    }
  }
  return RIDC_OK;
}

// ------------------------------------------------------------------------------------------
// results
// ------------------------------------------------------------------------------------------
static int copy_out(Ctx* c, const double* src, double* out, size_t count, int out_on_device) {
  const size_t bytes = count * sizeof(double);
  if (out_on_device) {
    RIDC_CUDA(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    int* flag = c->err_dev;   // reuse: 0 stays 0 unless a non-finite value is found
    int bad = 0;
    RIDC_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
    RIDC_TRY(launch_check_finite(c, out, (long)count, flag));
    RIDC_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    RIDC_CUDA(cudaStreamSynchronize(c->stream));
    return bad ? RIDC_ERR_NONFINITE : RIDC_OK;
  }
  RIDC_CUDA(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, c->stream));
  RIDC_CUDA(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < count; ++i)
    if (!std::isfinite(out[i])) return RIDC_ERR_NONFINITE;
  return RIDC_OK;
}

static int check_device_error(Ctx* c) {
  int err = 0;
  RIDC_CUDA(cudaStreamSynchronize(c->stream));
  RIDC_CUDA(cudaMemcpy(&err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    cudaMemset(c->err_dev, 0, sizeof(int));
    return RIDC_ERR_TIMEOUT;
  }
  return RIDC_OK;
}

extern "C" int ridc_get_level(ridc_handle h, int level, double* out, size_t count,
                              int out_on_device, long* step) {
  Ctx* c = ctx_of(h);
  if (!c || !out || level < 0 || level >= c->P || count != (size_t)c->plane) return RIDC_ERR_ARG;
  DeviceGuard dg(c->device);
  if (!c->initialised) return RIDC_ERR_ARG;
  RIDC_TRY(check_device_error(c));
  if (step) *step = c->seg_base + c->p[level];
  return copy_out(c, slot_ptr(c, c->eta[level], level, c->p[level]), out, count, out_on_device);
}

extern "C" int ridc_get_solution(ridc_handle h, double* out, size_t count, int out_on_device) {
  Ctx* c = ctx_of(h);
  if (!c) return RIDC_ERR_ARG;
  return ridc_get_level(h, c->P - 1, out, count, out_on_device, nullptr);
}

extern "C" int ridc_get_time(ridc_handle h, double* t) {
  Ctx* c = ctx_of(h);
  if (!c || !t) return RIDC_ERR_ARG;
  *t = (double)(c->seg_base + c->p[c->P - 1]) * c->dt;
  return RIDC_OK;
}

extern "C" int ridc_get_progress(ridc_handle h, long* steps, int nlevels) {
  Ctx* c = ctx_of(h);
  if (!c || !steps || nlevels < 1 || nlevels > c->P) return RIDC_ERR_ARG;
  for (int j = 0; j < nlevels; ++j) steps[j] = c->seg_base + c->p[j];
  return RIDC_OK;
}

// ------------------------------------------------------------------------------------------
// checkpoint / resume
// ------------------------------------------------------------------------------------------
// A state is this header followed by the rings of levels 0..P-1, each as eta, f^N and (when
// the level keeps it) f, every slot in slot order: cap[j] * plane FP64 values per field.
struct StateHeader {
  char magic[8];
  int32_t version, kind, dim, n, S, P, predictor, reserved;
  double dt, nu[kMaxSpecies], a, b, F, k;
  int64_t restart_every, seg_base, p[kMaxOrder];
  int32_t cap[kMaxOrder];
  int32_t has_F[kMaxOrder];
  uint64_t payload;
};
static const char kStateMagic[8] = {'R', 'I', 'D', 'C', 'S', 'T', 'A', 'T'};
constexpr int32_t kStateVersion = 2;

static uint64_t state_payload(const Ctx* c) {
  uint64_t vals = 0;
  for (int j = 0; j < c->P; ++j)
    vals += (uint64_t)c->cap[j] * (uint64_t)c->plane * (c->Fq[j] ? 3u : 2u);
  return vals * sizeof(double);
}

static void fill_header(const Ctx* c, StateHeader* hd) {
  memset(hd, 0, sizeof(*hd));
  memcpy(hd->magic, kStateMagic, sizeof(kStateMagic));
  hd->version = kStateVersion;
  hd->kind = c->kind; hd->dim = c->dim; hd->n = c->n; hd->S = c->S; hd->P = c->P;
  hd->predictor = c->pred;
  hd->dt = c->dt;
  for (int s = 0; s < kMaxSpecies; ++s) hd->nu[s] = (s < c->S) ? c->nu[s] : 0.0;
  hd->a = c->a; hd->b = c->b; hd->F = c->gsF; hd->k = c->gsk;
  hd->restart_every = c->restart_every;
  hd->seg_base = c->seg_base;
  for (int j = 0; j < kMaxOrder; ++j) {
    hd->p[j] = (j < c->P) ? c->p[j] : 0;
    hd->cap[j] = (j < c->P) ? c->cap[j] : 0;
    hd->has_F[j] = (j < c->P && c->Fq[j]) ? 1 : 0;
  }
  hd->payload = state_payload(c);
}

extern "C" int ridc_save_state(ridc_handle h, void* buf, size_t* len) {
  Ctx* c = ctx_of(h);
  if (!c || !len) return RIDC_ERR_ARG;
  DeviceGuard dg(c->device);
  if (!c->initialised) return RIDC_ERR_ARG;
  const size_t need = sizeof(StateHeader) + state_payload(c);
  if (!buf) {
    *len = need;
    return RIDC_OK;
  }
  if (*len < need) {
    *len = need;
    return RIDC_ERR_ARG;
  }
  RIDC_TRY(check_device_error(c));   // synchronises: the rings hold the finished state
  StateHeader hd;
  fill_header(c, &hd);
  uint8_t* out = static_cast<uint8_t*>(buf);
  memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  const size_t ring_bytes_per_slot = (size_t)c->plane * sizeof(double);
  for (int j = 0; j < c->P; ++j) {
    const double* rings[3] = {c->eta[j], c->fN[j], c->Fq[j]};
    for (const double* ring : rings) {
      if (!ring) continue;
      const size_t bytes = (size_t)c->cap[j] * ring_bytes_per_slot;
      RIDC_CUDA(cudaMemcpy(out + off, ring, bytes, cudaMemcpyDeviceToHost));
      off += bytes;
    }
  }
  *len = need;
  return RIDC_OK;
}

extern "C" int ridc_load_state(ridc_handle h, const void* buf, size_t len) {
  Ctx* c = ctx_of(h);
  if (!c || !buf || len < sizeof(StateHeader)) return RIDC_ERR_ARG;
  DeviceGuard dg(c->device);
  StateHeader hd, mine;
  memcpy(&hd, buf, sizeof(hd));
  fill_header(c, &mine);
  if (memcmp(hd.magic, kStateMagic, sizeof(kStateMagic)) != 0 || hd.version != kStateVersion)
    return RIDC_ERR_ARG;
  // same problem: every parameter the stored f^N and f depend on, bit for bit
  if (hd.kind != mine.kind || hd.dim != mine.dim || hd.n != mine.n || hd.S != mine.S ||
      hd.P != mine.P || hd.predictor != mine.predictor || memcmp(&hd.dt, &mine.dt, sizeof(double)) != 0 ||
      memcmp(hd.nu, mine.nu, sizeof(hd.nu)) != 0 || memcmp(&hd.a, &mine.a, sizeof(double)) != 0 ||
      memcmp(&hd.b, &mine.b, sizeof(double)) != 0 || memcmp(&hd.F, &mine.F, sizeof(double)) != 0 ||
      memcmp(&hd.k, &mine.k, sizeof(double)) != 0 || hd.restart_every != mine.restart_every ||
      memcmp(hd.cap, mine.cap, sizeof(hd.cap)) != 0 ||
      memcmp(hd.has_F, mine.has_F, sizeof(hd.has_F)) != 0 || hd.payload != mine.payload)
    return RIDC_ERR_ARG;
  if (len < sizeof(StateHeader) + hd.payload) return RIDC_ERR_ARG;
  for (int j = 0; j < c->P; ++j)
    if (hd.p[j] < 0 || (j > 0 && hd.p[j] > hd.p[j - 1])) return RIDC_ERR_ARG;
  if (hd.seg_base < 0 || (hd.restart_every > 0 && hd.p[c->P - 1] >= hd.restart_every))
    return RIDC_ERR_ARG;
  const uint8_t* in = static_cast<const uint8_t*>(buf);
  size_t off = sizeof(hd);
  const size_t ring_bytes_per_slot = (size_t)c->plane * sizeof(double);
  for (int j = 0; j < c->P; ++j) {
    double* rings[3] = {c->eta[j], c->fN[j], c->Fq[j]};
    for (double* ring : rings) {
      if (!ring) continue;
      const size_t bytes = (size_t)c->cap[j] * ring_bytes_per_slot;
      RIDC_CUDA(cudaMemcpyAsync(ring, in + off, bytes, cudaMemcpyHostToDevice, c->stream));
      off += bytes;
    }
  }
  // a pinned source is read asynchronously: finish before the caller may reuse buf
  RIDC_CUDA(cudaStreamSynchronize(c->stream));
  for (int j = 0; j < kMaxOrder; ++j) c->p[j] = (j < c->P) ? (long)hd.p[j] : 0;
  c->seg_base = (long)hd.seg_base;
  c->initialised = true;
  return RIDC_OK;
}

// ------------------------------------------------------------------------------------------
// host-only helpers
// ------------------------------------------------------------------------------------------
extern "C" int ridc_schedule_plan(int order, long nsteps, unsigned* active, size_t cap,
                                  size_t* count) {
  const long zero[kMaxOrder] = {0};
  return ridc_schedule_plan_from(order, zero, nsteps, active, cap, count);
}

extern "C" int ridc_schedule_plan_from(int order, const long* start, long nsteps,
                                       unsigned* active, size_t cap, size_t* count) {
  if (!start) return RIDC_ERR_ARG;
  return ridc_schedule_plan_predictor(order, RIDC_PRED_FBE, start, nsteps, active, cap, count);
}

extern "C" int ridc_schedule_plan_predictor(int order, int predictor, const long* start,
                                            long nsteps, unsigned* active, size_t cap,
                                            size_t* count) {
  const int p0 = predictor_order(predictor);
  if (p0 == 0 || order < 1 || order > kMaxOrder || p0 + order - 1 > kMaxOrder || nsteps < 0 ||
      !count || (cap && !active))
    return RIDC_ERR_ARG;
  const long zero[kMaxOrder] = {0};
  if (!start) start = zero;
  long p[kMaxOrder] = {0};
  for (int j = 0; j < order; ++j) {
    p[j] = start[j];
    if (p[j] < 0 || (j > 0 && p[j] > p[j - 1])) return RIDC_ERR_ARG;
  }
  if (p[order - 1] > nsteps) return RIDC_ERR_ARG;
  size_t s = 0;
  for (;;) {
    const unsigned m = plan_step(order, p, nsteps, p0);
    if (!m) break;
    if (s < cap) active[s] = m;
    ++s;
    for (int j = 0; j < order; ++j)
      if (m & (1u << j)) p[j]++;
  }
  *count = s;
  if (p[order - 1] != nsteps) return RIDC_ERR_CUDA;
  return s > cap ? RIDC_ERR_ARG : RIDC_OK;
}

extern "C" int ridc_quadrature_weights(int order, double* out, size_t cap) {
  if (order < 1 || order > kMaxOrder || !out || cap < (size_t)order * order * order)
    return RIDC_ERR_ARG;
  fill_weights(order, out);
  return RIDC_OK;
}

// ------------------------------------------------------------------------------------------
// instrumentation
// ------------------------------------------------------------------------------------------
extern "C" int ridc_debug_stall_next_gemm(ridc_handle h) {
  Ctx* c = ctx_of(h);
  if (!c) return RIDC_ERR_ARG;
  if (c->dim != 2 || !is_mixed(c->prec)) return RIDC_ERR_UNSUPPORTED;
  c->stall_next_gemm = 1;
  return RIDC_OK;
}

extern "C" int ridc_set_profiling(ridc_handle h, int enable) {
  Ctx* c = ctx_of(h);
  if (!c) return RIDC_ERR_ARG;
  DeviceGuard dg(c->device);
  prof_collect(c);
  for (int k = 0; k < RIDC_KERNEL_COUNT; ++k) { c->k_launch[k] = 0; c->k_ms[k] = 0.0; }
  if (enable < 0) return RIDC_ERR_ARG;
  c->profiling = enable;
  c->prof_now = enable == 1;
  return RIDC_OK;
}

extern "C" int ridc_get_kernel_stats(ridc_handle h, int kernel, long* launches, double* total_ms) {
  Ctx* c = ctx_of(h);
  if (!c || kernel < 0 || kernel >= RIDC_KERNEL_COUNT || !launches || !total_ms)
    return RIDC_ERR_ARG;
  prof_collect(c);
  *launches = c->k_launch[kernel];
  *total_ms = c->k_ms[kernel];
  return RIDC_OK;
}

extern "C" long ridc_launch_count(ridc_handle h) {
  Ctx* c = ctx_of(h);
  return c ? c->launches : -1;
}
