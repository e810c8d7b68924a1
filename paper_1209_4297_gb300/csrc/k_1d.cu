// Persistent kernel for the 1D problems (periodic advection-diffusion with central or
// upwind advection, viscous Burgers with Dirichlet walls): one launch runs every pipeline
// step of an advance call. The paper gives every correction level its own processor
// (Section III-E); here every level gets its own SM: a thread-block cluster of
// min(order, 8) CTAs, CTA r taking levels r, r + 8, ... The level rings stay in global
// memory (L2 resident); right-hand sides, the tridiagonal solves and the new states live
// in shared memory. Within a pipeline step the levels are independent (the lock-step rule
// never writes a ring slot that any level reads in the same step), so one cluster barrier
// per step orders the whole exchange. Per step, for every advancing level j (n -> n+1):
//   r   = dt F^0_n                                                    (j = 0, eq. (pred))
//   r   = (eta^j_n - eta^{j-1}_{n+1}) + dt (f^N(eta^j_n) - f^N(eta^{j-1}_n))
//         + dt sum_i w[j][m][i] F^{j-1}_{b+i}                          (j >= 1, eq. (corr))
//   solve (I - dt nu L) delta = r   (two warp-parallel first-order recurrences)
//   eta^j_{n+1} = base + delta, base = eta^0_n (j = 0) or eta^{j-1}_{n+1}
//   f^N(eta) (Section IV's operators) and F = f^N + nu (eta_{i+1} - 2 eta_i + eta_{i-1}) / h^2
// The step masks come from the host's plan of the same lock-step rule.
// With an ARK predictor (Section II, Theorem 2) level 0 takes its step stage by stage on its
// CTA: each implicit stage sums dt w X over the earlier stages' F and f^N (ArkStage), solves
// with its own operator (I - a_ii dt D: its rho powers are loaded into a second shared table)
// and evaluates F and f^N of the stage value into global scratch, which only this CTA reads;
// the last stage is the new solution. Correctors read p0 + j-node stencils.
#include "ridc_internal.h"

namespace ridc {

struct OneDStage {
  int coef;                  // operator table index
  int nterms;
  int src[kMaxTerms];        // 2 j: F_j, 2 j + 1: f^N_j (stage 0: level 0's ring slot n)
  double w[kMaxTerms];       // dt * weight
};

struct OneDArgs {
  double* eta[kMaxOrder];
  double* fN[kMaxOrder];
  double* F[kMaxOrder];
  int cap[kMaxOrder];
  const double* wq;        // [W][W][W]
  const double* tri;       // per operator: rho^k (k = 0..npad), wrap or kappa, rho/mu, g
  const unsigned* sched;   // step masks
  long nsteps_pipe;
  long* p_dev;             // steps taken per level (read at start, written at the end)
  int P, n, npad, init_only, kind;
  int p0, W;               // predictor order, weight-table side p0 + P - 1
  double dt, c_lap;
  double cadv;             // central: a/(2h); upwind: a/h; Burgers: 1/(4h)
  bool upwind_left;        // upwind with a >= 0: backward difference
  // ARK predictor (nstages > 1): stages 1..nstages-1; scratch [2 nstages + 1][n]: F_i at
  // row 2 i, f^N_i at row 2 i + 1, the stage value Y at row 2 nstages
  int nstages;
  OneDStage st[kMaxStages];
  double* scratch;
};

// f^N and F of one state; periodic wrap or zero Dirichlet ghosts
__device__ __forceinline__ void eval_state(const OneDArgs& a, const double* e, double* fN,
                                           double* F) {
  const int n = a.n;
  const bool dir = a.kind == RIDC_BURGERS_1D_DIRICHLET;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double em, ep;
    if (dir) {
      em = i > 0 ? e[i - 1] : 0.0;
      ep = i < n - 1 ? e[i + 1] : 0.0;
    } else {
      em = e[i == 0 ? n - 1 : i - 1];
      ep = e[i == n - 1 ? 0 : i + 1];
    }
    const double ei = e[i];
    double fn;
    if (a.kind == RIDC_ADV_DIFF_1D_PERIODIC) fn = -a.cadv * (ep - em);
    else if (a.kind == RIDC_ADV_DIFF_1D_UPWIND_PERIODIC)
      fn = a.upwind_left ? -a.cadv * (ei - em) : -a.cadv * (ep - ei);
    else fn = -a.cadv * fma(ep, ep, -(em * em));
    fN[i] = fn;
    if (F) F[i] = fma(a.c_lap, (ep + em) - 2.0 * ei, fn);
  }
}

// Solve of (I - dt nu L) x = r for one level by the whole block, in place on r[0, npad); the
// result is x / s with s = rho / mu (the caller applies s in the FMA that consumes x).
// With the shift S and rho = 2mu / (1 + 2mu + sqrt(1 + 4mu)) < 1,
// M = (mu/rho)(1 - rho S)(1 - rho S^T):
//   z = (1 - rho S)^-1 r      : z_j = r_j + rho z_{j+1},  z_n = 0           (backward)
//   y = (rho/mu)(1 - rho S^T)^-1 z = s y' : y'_j = z_j + rho y'_{j-1},  y'_{-1} = 0  (forward)
// Each first-order recurrence is a scan over the block: every thread runs its chunk of
// m = npad / blockDim values, a 5-step shuffle scan combines the chunk carries of a warp with
// weights rho^(m 2^k), and the warps' totals are chained through shared memory. Entries
// past n are zero on entry, so the backward scan ends with z_n = 0 and the forward scan only
// leaves values past n, which nothing reads. Then
//   periodic  (cyclic S, M is the matrix): exact wrap terms make both recurrences cyclic,
//             z_j += rho^(n-j) z_0 / (1 - rho^n),  y'_j += rho^(j+1) y'_{n-1} / (1 - rho^n);
//   Dirichlet (the matrix is M + mu rho e_{n-1} e_{n-1}^T): Sherman-Morrison,
//             x'_j = y'_j - kappa y'_{n-1} g_j with the tabulated g = M^-1 e_{n-1}.
// The solve runs on one SM's FP64 pipe, so its operations per cell set its time. A chunk's
// carry terms share a factor: rho^(n-j) = rho^(m-i) rho^(n-j0-m) and rho^(j+1) =
// rho^(i+1) rho^j0 for cell j = j0 + i. So each wrap term is folded into the thread's carry
// (one FMA per thread instead of one per cell). The forward wrap needs y'_{n-1}, which the
// thread holding it forms first, so carry and wrap are applied in one sweep.
// Spreading the chunks over all warps uses the FP64 pipes of all four SM partitions.
__device__ void tri_solve_block(double* r, int n, int npad, const double* rp, double corr,
                                const double* gvec, bool cyclic, double* scratch) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, NW = blockDim.x >> 5;
  const int m = npad / blockDim.x;
  const int j0 = tid * m;
  const double rho = rp[1], rho_w = rp[32 * m];   // rho^m per lane, rho^(32 m) per warp
  for (int i = 0; i < m; ++i)
    if (j0 + i >= n) r[j0 + i] = 0.0;
  // ---- backward recurrence, local part: t_j = r_j + rho t_{j+1}, t_{j0+m} = 0
  double t = 0.0;
  for (int i = m - 1; i >= 0; --i) {
    t = fma(rho, t, r[j0 + i]);
    r[j0 + i] = t;
  }
  // carries within the warp: C_l = t_{l m} + rho^m C_{l+1} (reverse inclusive scan)
  double C = t;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double up = __shfl_down_sync(0xffffffffu, C, d);
    if (lane + d < 32) C = fma(rp[m * d], up, C);
  }
  if (lane == 0) scratch[w] = C;   // the warp's chunk of z, without what lies above it
  __syncthreads();
  // z at the first index of warp w+1: Z = C_{w+1} + rho^(32m) Z_{w+2}
  double Z = 0.0;
  for (int v = NW - 1; v > w; --v) Z = fma(rho_w, Z, scratch[v]);
  C = fma(rp[m * (32 - lane)], Z, C);           // full carry: z at this thread's first index
  if (tid == 0) scratch[NW] = C;                // non-cyclic z_0
  double Cnext = __shfl_down_sync(0xffffffffu, C, 1);
  if (lane == 31) Cnext = Z;
  __syncthreads();
  // periodic wrap, folded into the carry for chunks that lie inside [0, n)
  const bool inside = j0 + m <= n;
  double z0 = 0.0;
  if (cyclic) {
    z0 = scratch[NW] * corr;
    if (inside) Cnext = fma(rp[n - j0 - m], z0, Cnext);
  }
  for (int i = 0; i < m; ++i) {
    const int j = j0 + i;
    double v = fma(rp[m - i], Cnext, r[j]);
    if (cyclic && !inside && j < n) v = fma(rp[n - j], z0, v);
    r[j] = v;
  }
  // ---- forward recurrence, local part: t_j = z_j + rho t_{j-1}, t_{j0-1} = 0
  t = 0.0;
  for (int i = 0; i < m; ++i) {
    t = fma(rho, t, r[j0 + i]);
    r[j0 + i] = t;
  }
  // carries within the warp: D_l = t_{(l+1)m-1} + rho^m D_{l-1} (inclusive scan)
  double D = t;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double dn = __shfl_up_sync(0xffffffffu, D, d);
    if (lane >= d) D = fma(rp[m * d], dn, D);
  }
  if (lane == 31) scratch[w] = D;
  __syncthreads();
  // y' at the last index of warp w-1: Y = D_{w-1} + rho^(32m) Y_{w-2}
  double Y = 0.0;
  for (int v = 0; v < w; ++v) Y = fma(rho_w, Y, scratch[v]);
  D = fma(rp[m * (lane + 1)], Y, D);            // full carry: y' at this thread's last index
  double Dprev = __shfl_up_sync(0xffffffffu, D, 1);
  if (lane == 0) Dprev = Y;
  // y'_{n-1} without its wrap or Sherman-Morrison term, from the thread that holds it
  if (j0 <= n - 1 && n - 1 < j0 + m) scratch[NW + 1] = fma(rp[n - j0], Dprev, r[n - 1]);
  __syncthreads();
  const double yl = scratch[NW + 1];
  if (cyclic) {
    // y'_j += rho^(i+1) (Dprev + rho^j0 y'_{n-1} corr); cells past n get a finite value that
    // nothing reads
    const double Dw = fma(rp[j0], yl * corr, Dprev);
    for (int i = 0; i < m; ++i) r[j0 + i] = fma(rp[i + 1], Dw, r[j0 + i]);
  } else {
    const double wv = -corr * yl;
    for (int i = 0; i < m; ++i) {
      const int j = j0 + i;
      double v = fma(rp[i + 1], Dprev, r[j]);
      if (j < n) v = fma(wv, gvec[j], v);
      r[j] = v;
    }
  }
  __syncthreads();
}

// Corrector right-hand side of one level over this CTA's cells, with the K quadrature nodes
// of the level below: every thread issues the loads of U of its cells (4 + K ring values each,
// read past L1 because other SMs wrote them) before any arithmetic, so their L2 round trips
// overlap instead of following one another; the arithmetic per cell is that of eq. (corr) in
// delta form, in a fixed order.
template <int K>
__device__ __forceinline__ void rhs_corrector_1d(int n, double dt, const double* ej,
                                                 const double* fj, const double* ep,
                                                 const double* fp, const double* Fring, long b,
                                                 int cap, const double* wq, double* r, double* e) {
  constexpr int U = 2;
  const double* F[K];
  double w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    F[k] = Fring + ((b + k) % cap) * n;
    w[k] = dt * wq[k];
  }
  for (int i0 = threadIdx.x; i0 < n; i0 += U * blockDim.x) {
    double vb[U], vfj[U], vfp[U], vej[U], vF[K][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n) {
        vb[u] = __ldcg(ep + i);
        vfj[u] = __ldcg(fj + i);
        vfp[u] = __ldcg(fp + i);
        vej[u] = __ldcg(ej + i);
#pragma unroll
        for (int k = 0; k < K; ++k) vF[k][u] = __ldcg(F[k] + i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n) {
        double acc = fma(dt, vfj[u] - vfp[u], vej[u] - vb[u]);
#pragma unroll
        for (int k = 0; k < K; ++k) acc = fma(w[k], vF[k][u], acc);
        r[i] = acc;
        e[i] = vb[u];
      }
    }
  }
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// every thread of every CTA of the cluster; release/acquire orders the ring writes in
// global memory (and shared memory) before the other CTAs' reads in the next step
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ARK: level 0 is an ARK predictor (a separate instantiation keeps the FBE kernel's code)
template <bool ARK>
__global__ void __launch_bounds__(ONED_THREADS) ridc1d_kernel(const __grid_constant__ OneDArgs a) {
  extern __shared__ double sm[];
  const int n = a.n, P = a.P, npad = a.npad;
  const int rank = (int)cluster_rank(), CL = (int)cluster_size();
  const int L = (P + CL - 1) / CL;      // levels of this CTA at most
  double* R = sm;                       // [L][npad] right-hand sides, then solutions
  double* E = sm + (size_t)L * npad;    // [L][n] new states
  double* rp = E + (size_t)L * n;       // [npad+1] powers rho^k
  double* rq = rp + npad + 1;           // ARK: [npad+1] powers of the stage operator's rho
  __shared__ long p[kMaxOrder];
  __shared__ int lev[kMaxOrder];
  __shared__ int na;
  __shared__ double scratch[ONED_THREADS / 32 + 2];
  __shared__ double s_last;             // ARK predictor: s of its last stage's operator

  if (a.init_only) {
    if (rank == 0) eval_state(a, a.eta[0], a.fN[0], a.F[0]);
    return;
  }
  for (int i = threadIdx.x; i <= npad; i += blockDim.x) rp[i] = a.tri[i];
  if (threadIdx.x < kMaxOrder) p[threadIdx.x] = a.p_dev[threadIdx.x];
  const double corr = a.tri[npad + 1], sfac = a.tri[npad + 2];
  const double* gvec = a.tri + npad + 3;
  const bool cyclic = a.kind != RIDC_BURGERS_1D_DIRICHLET;
  const long T = (long)npad + 3 + n;    // one operator's table
  constexpr bool ark = ARK;
  int rq_coef = -1;                     // operator whose powers rq holds
  __syncthreads();

  for (long s = 0; s < a.nsteps_pipe; ++s) {
    const unsigned mask = a.sched[s];
    if (threadIdx.x == 0) {
      int k = 0;
      for (int j = rank; j < P; j += CL)
        if (mask & (1u << j)) lev[k++] = j;
      na = k;
    }
    __syncthreads();
    // right-hand sides of this CTA's advancing levels; the base of each new state
    // (eta^0_n, or eta^{j-1}_{n+1}, which the right-hand side reads anyway) is kept in E
    for (int q = 0; q < na; ++q) {
      const int j = lev[q];
      const long nj = p[j];
      double* r = R + (size_t)q * npad;
      double* e = E + (size_t)q * n;
      // ring reads bypass L1 (__ldcg): other SMs of the cluster wrote them
      if (j == 0 && ark) {
        // ARK predictor: stages 1..s-1; the last one leaves its solved delta in r and y_n
        // in e, and the shared solve below skips it
        const double* F0 = a.F[0] + (nj % a.cap[0]) * n;
        const double* f0 = a.fN[0] + (nj % a.cap[0]) * n;
        const double* e0 = a.eta[0] + (nj % a.cap[0]) * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) e[i] = __ldcg(e0 + i);
        double* Y = a.scratch + (size_t)2 * a.nstages * n;
        for (int si = 1; si < a.nstages; ++si) {
          const OneDStage& S = a.st[si];
          for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double acc = 0.0;
            for (int t = 0; t < S.nterms; ++t) {
              const int src = S.src[t];
              const double* X = src == 0 ? F0 : src == 1 ? f0 : a.scratch + (size_t)src * n;
              const double x = src < 2 ? __ldcg(X + i) : X[i];
              acc = t == 0 ? S.w[0] * x : fma(S.w[t], x, acc);
            }
            r[i] = acc;
          }
          if (S.coef != rq_coef) {      // powers of this stage's rho into shared memory
            for (int i = threadIdx.x; i <= npad; i += blockDim.x) rq[i] = a.tri[S.coef * T + i];
            rq_coef = S.coef;
          }
          __syncthreads();
          tri_solve_block(r, n, npad, rq, a.tri[S.coef * T + npad + 1],
                          a.tri + S.coef * T + npad + 3, cyclic, scratch);
          const double ss = a.tri[S.coef * T + npad + 2];   // the solve leaves delta / s
          if (si == a.nstages - 1) {
            if (threadIdx.x == 0) s_last = ss;
            break;
          }
          // stage value Y = y_n + delta, then F and f^N of it (read back by this CTA only)
          for (int i = threadIdx.x; i < n; i += blockDim.x) Y[i] = fma(ss, r[i], e[i]);
          __syncthreads();
          eval_state(a, Y, a.scratch + (size_t)(2 * si + 1) * n, a.scratch + (size_t)2 * si * n);
          __syncthreads();
        }
      } else if (j == 0) {
        const double* F0 = a.F[0] + (nj % a.cap[0]) * n;
        const double* e0 = a.eta[0] + (nj % a.cap[0]) * n;
        // when a thread has several cells, the loads of up to four are issued together
        if (n <= 2 * (int)blockDim.x) {
          for (int i = threadIdx.x; i < n; i += blockDim.x) {
            r[i] = a.dt * __ldcg(F0 + i);
            e[i] = __ldcg(e0 + i);
          }
        } else for (int i0 = threadIdx.x; i0 < n; i0 += 4 * blockDim.x) {
          double vF[4], ve[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) {
              vF[u] = __ldcg(F0 + i);
              ve[u] = __ldcg(e0 + i);
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n) {
              r[i] = a.dt * vF[u];
              e[i] = ve[u];
            }
          }
        }
      } else {
        const double* ej = a.eta[j] + (nj % a.cap[j]) * n;
        const double* fj = a.fN[j] + (nj % a.cap[j]) * n;
        const double* ep = a.eta[j - 1] + ((nj + 1) % a.cap[j - 1]) * n;
        const double* fp = a.fN[j - 1] + (nj % a.cap[j - 1]) * n;
        // K-node stencil of level j-1 (K = p0 + j): t_b..t_{b+K-1}, interval m = nj - b
        const int K = a.p0 + j;
        const long b = nj + 2 - K > 0 ? nj + 2 - K : 0;
        const int m = (int)(nj - b);
        const double* w = a.wq + ((size_t)(K - 1) * a.W + m) * a.W;
        const double* Fr = a.F[j - 1];
        const int cp = a.cap[j - 1];
        switch (K) {
          case 2: rhs_corrector_1d<2>(n, a.dt, ej, fj, ep, fp, Fr, b, cp, w, r, e); break;
          case 3: rhs_corrector_1d<3>(n, a.dt, ej, fj, ep, fp, Fr, b, cp, w, r, e); break;
          case 4: rhs_corrector_1d<4>(n, a.dt, ej, fj, ep, fp, Fr, b, cp, w, r, e); break;
          case 5: rhs_corrector_1d<5>(n, a.dt, ej, fj, ep, fp, Fr, b, cp, w, r, e); break;
          default:   // wider stencils (orders above 6): one cell at a time
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
              const double base = __ldcg(ep + i);
              double acc = fma(a.dt, __ldcg(fj + i) - __ldcg(fp + i), __ldcg(ej + i) - base);
              for (int k = 0; k < K; ++k)
                acc = fma(a.dt * w[k], __ldcg(Fr + ((b + k) % cp) * n + i), acc);
              r[i] = acc;
              e[i] = base;
            }
        }
      }
    }
    __syncthreads();
    for (int q = 0; q < na; ++q)
      if (!(ark && lev[q] == 0))   // an ARK predictor's last stage is solved already
        tri_solve_block(R + (size_t)q * npad, n, npad, rp, corr, gvec, cyclic, scratch);
    // new states: base + s (delta / s) (each thread updates the entries it stored the base
    // of; s_last was set before the barrier that ends the ARK stages' last solve)
    for (int q = 0; q < na; ++q) {
      const double sq = (ark && lev[q] == 0) ? s_last : sfac;
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        E[(size_t)q * n + i] = fma(sq, R[(size_t)q * npad + i], E[(size_t)q * n + i]);
    }
    __syncthreads();
    for (int q = 0; q < na; ++q) {
      const int j = lev[q];
      const long slot = ((p[j] + 1) % a.cap[j]) * n;
      const double* e = E + (size_t)q * n;
      for (int i = threadIdx.x; i < n; i += blockDim.x) a.eta[j][slot + i] = e[i];
      eval_state(a, e, a.fN[j] + slot, a.F[j] ? a.F[j] + slot : nullptr);
    }
    __syncthreads();
    if (threadIdx.x == 0)   // every CTA follows every level's progress
      for (int j = 0; j < P; ++j)
        if (mask & (1u << j)) p[j]++;
    cluster_sync_all();     // also orders this CTA's shared memory (p) for the next step
  }
  if (rank == 0 && threadIdx.x < kMaxOrder) a.p_dev[threadIdx.x] = p[threadIdx.x];
}

int launch_1d(Ctx* c, long nsteps_pipe, int init_only) {
  OneDArgs a{};
  for (int j = 0; j < c->P; ++j) {
    a.eta[j] = c->eta[j];
    a.fN[j] = c->fN[j];
    a.F[j] = c->Fq[j];
    a.cap[j] = c->cap[j];
  }
  a.tri = c->tri;
  a.p0 = c->p0;
  a.W = c->W;
  a.nstages = c->nstages;
  a.scratch = c->st1d;
  for (int i = 1; i < c->nstages; ++i) {
    const ArkStage& S = c->stage[i];
    a.st[i].coef = S.coef;
    a.st[i].nterms = S.nterms;
    for (int t = 0; t < S.nterms; ++t) {
      a.st[i].src[t] = S.src[t];
      a.st[i].w[t] = c->dt * S.w[t];
    }
  }
  a.sched = c->sched_dev;
  a.nsteps_pipe = nsteps_pipe;
  a.p_dev = c->p_dev;
  a.P = c->P;
  a.n = c->n;
  a.npad = c->npad;
  a.init_only = init_only;
  a.kind = c->kind;
  a.dt = c->dt;
  a.c_lap = c->nu[0] / (c->h * c->h);
  if (c->kind == RIDC_ADV_DIFF_1D_PERIODIC) a.cadv = c->a / (2.0 * c->h);
  else if (c->kind == RIDC_ADV_DIFF_1D_UPWIND_PERIODIC) a.cadv = c->a / c->h;
  else a.cadv = 1.0 / (4.0 * c->h);
  a.upwind_left = c->a >= 0.0;
  // the quadrature weights follow the solver tables: uploaded once per handle
  a.wq = c->tri + (size_t)c->ncoef * oned_table_doubles(c->n, c->npad);
  const int CL = init_only ? 1 : oned_cluster(c->P);
  const size_t smem = oned_smem_doubles(c->P, c->n, c->npad, c->nstages > 1) * sizeof(double);
  static std::atomic<unsigned long long> attr_done{0}, attr_done_ark{0};
  const bool ark = c->nstages > 1;
  if (ark)
    RIDC_TRY(raise_smem_limit_once(ridc1d_kernel<true>,
                                   (int)(kOneDMaxSmemDoubles * sizeof(double)), &attr_done_ark));
  else
    RIDC_TRY(raise_smem_limit_once(ridc1d_kernel<false>,
                                   (int)(kOneDMaxSmemDoubles * sizeof(double)), &attr_done));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(ONED_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_1D, &e0);
  const cudaError_t e = ark ? cudaLaunchKernelEx(&cfg, ridc1d_kernel<true>, a)
                            : cudaLaunchKernelEx(&cfg, ridc1d_kernel<false>, a);
  prof_end(c, RIDC_KERNEL_1D, e0);
  return cuda_status(e);
}

}  // namespace ridc
