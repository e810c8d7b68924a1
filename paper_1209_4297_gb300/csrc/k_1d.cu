// Persistent single-CTA kernel for 1D periodic advection-diffusion: one launch runs every
// pipeline step of an advance call. The level rings stay in global memory (a few KB, L1/L2
// resident); right-hand sides, the tridiagonal sweeps and the new states live in shared
// memory. Per pipeline step, for every advancing level j (step n -> n+1):
//   r   = dt F^0_n                                                    (j = 0, eq. (pred))
//   r   = (eta^j_n - eta^{j-1}_{n+1}) + dt (f^N(eta^j_n) - f^N(eta^{j-1}_n))
//         + dt sum_i w[j][m][i] F^{j-1}_{b+i}                          (j >= 1, eq. (corr))
//   solve (I - dt nu L) delta = r   (cyclic tridiagonal: two warp-parallel recurrences)
//   eta^j_{n+1} = base + delta, base = eta^0_n (j = 0) or eta^{j-1}_{n+1}
//   f^N = -a (eta_{i+1} - eta_{i-1}) / 2h,  F = f^N + nu (eta_{i+1} - 2 eta_i + eta_{i-1}) / h^2
// The step masks come from the host's plan of the same lock-step rule.
#include "ridc_internal.h"

namespace ridc {

struct OneDArgs {
  double* eta[kMaxOrder];
  double* fN[kMaxOrder];
  double* F[kMaxOrder];
  int cap[kMaxOrder];
  const double* wq;        // [P][P][P]
  const double* tri;       // rho^k (k = 0..n), 1/(1 - rho^n), rho/mu, then the weights
  const unsigned* sched;   // step masks
  long nsteps_pipe;
  long* p_dev;             // steps taken per level (read at start, written at the end)
  int P, n, init_only;
  double dt, a2h, c_lap;
};

__device__ __forceinline__ void eval_state(const double* e, double* fN, double* F, int n,
                                           double a2h, double c_lap) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double em = e[i == 0 ? n - 1 : i - 1], ep = e[i == n - 1 ? 0 : i + 1], ei = e[i];
    const double fn = -a2h * (ep - em);
    fN[i] = fn;
    if (F) F[i] = fma(c_lap, (ep + em) - 2.0 * ei, fn);
  }
}

// Cyclic solve of (I - dt nu L) x = r for one level by one warp. The periodic tridiagonal
// matrix (diagonal 1 + 2mu, off-diagonals -mu) factors as (mu/rho)(1 - rho E)(1 - rho E^-1)
// with the cyclic shift (E x)_j = x_{j+1} and rho = 2mu / (1 + 2mu + sqrt(1 + 4mu)) < 1, so
//   z = (1 - rho E)^-1 r      : z_j = r_j + rho z_{j+1}          (backward, cyclic)
//   x = (rho/mu)(1 - rho E^-1)^-1 z : x_j = (rho/mu) z_j + rho x_{j-1}   (forward, cyclic)
// Each first-order recurrence is a scan: every lane runs its chunk of N/32 values, a 5-step
// shuffle scan combines the chunk carries with weights rho^(chunk * 2^k), and the cyclic wrap
// is exact: z_cyc_j = z_j + rho^(N-j) z_0 / (1 - rho^N), x_cyc_j = x_j + rho^(j+1) x_{N-1} / (1 - rho^N).
// The dependent FP64 chain is about 30 operations instead of the 2N of a Thomas sweep.
__device__ void cyclic_solve_warp(double* r, int n, const double* rp, double inv_wrap, double s) {
  const int lane = threadIdx.x & 31;
  const int m = n >> 5;
  const int j0 = lane * m;
  const double rho = rp[1];
  // backward recurrence, local part: t_j = r_j + rho t_{j+1}, t_{j0+m} = 0
  double t = 0.0;
  for (int i = m - 1; i >= 0; --i) {
    t = fma(rho, t, r[j0 + i]);
    r[j0 + i] = t;
  }
  // carry C_l = z_{l m} = t_{l m} + rho^m C_{l+1}: reverse inclusive scan over the lanes
  double C = t;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double up = __shfl_down_sync(0xffffffffu, C, d);
    if (lane + d < 32) C = fma(rp[m * d], up, C);
  }
  const double z0 = __shfl_sync(0xffffffffu, C, 0) * inv_wrap;   // cyclic z_0
  double Cnext = __shfl_down_sync(0xffffffffu, C, 1);
  if (lane == 31) Cnext = 0.0;
  __syncwarp();
  for (int i = 0; i < m; ++i) {
    const int j = j0 + i;
    r[j] = fma(rp[n - j], z0, fma(rp[m - i], Cnext, r[j]));
  }
  __syncwarp();
  // forward recurrence, local part: t_j = s z_j + rho t_{j-1}, t_{j0-1} = 0
  t = 0.0;
  for (int i = 0; i < m; ++i) {
    t = fma(rho, t, s * r[j0 + i]);
    r[j0 + i] = t;
  }
  // carry D_l = x_{(l+1)m-1} = t_{(l+1)m-1} + rho^m D_{l-1}: inclusive scan over the lanes
  double D = t;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double dn = __shfl_up_sync(0xffffffffu, D, d);
    if (lane >= d) D = fma(rp[m * d], dn, D);
  }
  const double xl = __shfl_sync(0xffffffffu, D, 31) * inv_wrap;  // cyclic x_{N-1}
  double Dprev = __shfl_up_sync(0xffffffffu, D, 1);
  if (lane == 0) Dprev = 0.0;
  __syncwarp();
  for (int i = 0; i < m; ++i) {
    const int j = j0 + i;
    r[j] = fma(rp[j + 1], xl, fma(rp[i + 1], Dprev, r[j]));
  }
  __syncwarp();
}

__global__ void __launch_bounds__(256) ridc1d_kernel(const __grid_constant__ OneDArgs a) {
  extern __shared__ double sm[];
  const int n = a.n, P = a.P;
  double* R = sm;                    // [P][n] right-hand sides, then solutions
  double* E = sm + (size_t)P * n;    // [P][n] new states
  double* rp = E + (size_t)P * n;    // [n+1] powers rho^k
  __shared__ long p[kMaxOrder];
  __shared__ int lev[kMaxOrder];
  __shared__ int na;

  if (a.init_only) {
    eval_state(a.eta[0], a.fN[0], a.F[0], n, a.a2h, a.c_lap);
    return;
  }
  for (int i = threadIdx.x; i <= n; i += blockDim.x) rp[i] = a.tri[i];
  if (threadIdx.x < kMaxOrder) p[threadIdx.x] = a.p_dev[threadIdx.x];
  const double inv_wrap = a.tri[n + 1], sfac = a.tri[n + 2];
  __syncthreads();
  const int warp = threadIdx.x >> 5;

  for (long s = 0; s < a.nsteps_pipe; ++s) {
    const unsigned mask = a.sched[s];
    if (threadIdx.x == 0) {
      int k = 0;
      for (int j = 0; j < P; ++j)
        if (mask & (1u << j)) lev[k++] = j;
      na = k;
    }
    __syncthreads();
    // right-hand sides
    for (int q = 0; q < na; ++q) {
      const int j = lev[q];
      const long nj = p[j];
      double* r = R + (size_t)q * n;
      if (j == 0) {
        const double* F0 = a.F[0] + (nj % a.cap[0]) * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = a.dt * F0[i];
      } else {
        const double* ej = a.eta[j] + (nj % a.cap[j]) * n;
        const double* fj = a.fN[j] + (nj % a.cap[j]) * n;
        const double* ep = a.eta[j - 1] + ((nj + 1) % a.cap[j - 1]) * n;
        const double* fp = a.fN[j - 1] + (nj % a.cap[j - 1]) * n;
        const long b = nj + 1 - j > 0 ? nj + 1 - j : 0;
        const int m = (int)(nj - b);
        const double* w = a.wq + ((size_t)j * P + m) * P;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          double acc = fma(a.dt, fj[i] - fp[i], ej[i] - ep[i]);
          for (int k = 0; k <= j; ++k)
            acc = fma(a.dt * w[k], a.F[j - 1][((b + k) % a.cap[j - 1]) * n + i], acc);
          r[i] = acc;
        }
      }
    }
    __syncthreads();
    // cyclic solves, one warp per level
    for (int q = warp; q < na; q += (int)(blockDim.x >> 5))
      cyclic_solve_warp(R + (size_t)q * n, n, rp, inv_wrap, sfac);
    __syncthreads();
    // new states
    for (int q = 0; q < na; ++q) {
      const int j = lev[q];
      const long nj = p[j];
      const double* base = (j == 0) ? a.eta[0] + (nj % a.cap[0]) * n
                                    : a.eta[j - 1] + ((nj + 1) % a.cap[j - 1]) * n;
      for (int i = threadIdx.x; i < n; i += blockDim.x) E[(size_t)q * n + i] = base[i] + R[(size_t)q * n + i];
    }
    __syncthreads();
    for (int q = 0; q < na; ++q) {
      const int j = lev[q];
      const long slot = ((p[j] + 1) % a.cap[j]) * n;
      const double* e = E + (size_t)q * n;
      for (int i = threadIdx.x; i < n; i += blockDim.x) a.eta[j][slot + i] = e[i];
      eval_state(e, a.fN[j] + slot, a.F[j] ? a.F[j] + slot : nullptr, n, a.a2h, a.c_lap);
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int q = 0; q < na; ++q) p[lev[q]]++;
    __syncthreads();
  }
  if (threadIdx.x < kMaxOrder) a.p_dev[threadIdx.x] = p[threadIdx.x];
}

int launch_1d(Ctx* c, long nsteps_pipe, int init_only) {
  OneDArgs a{};
  for (int j = 0; j < c->P; ++j) {
    a.eta[j] = c->eta[j];
    a.fN[j] = c->fN[j];
    a.F[j] = c->Fq[j];
    a.cap[j] = c->cap[j];
  }
  a.wq = nullptr;
  a.tri = c->tri;
  a.sched = c->sched_dev;
  a.nsteps_pipe = nsteps_pipe;
  a.p_dev = c->p_dev;
  a.P = c->P;
  a.n = c->n;
  a.init_only = init_only;
  a.dt = c->dt;
  a.a2h = c->a / (2.0 * c->h);
  a.c_lap = c->nu[0] / (c->h * c->h);
  // the quadrature weights follow the solver constants: uploaded once per handle
  a.wq = c->tri + c->n + 3;
  const size_t smem = ((size_t)2 * c->P * c->n + (size_t)c->n + 1) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(ridc1d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
  }
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_1D, &e0);
  ridc1d_kernel<<<1, 256, smem, c->stream>>>(a);
  prof_end(c, RIDC_KERNEL_1D, e0);
  return cuda_status(cudaGetLastError());
}

}  // namespace ridc
