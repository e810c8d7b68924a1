// ridc_solve_planes_fixed: the FP64 batched implicit solve of ridc_solve_planes, for callers
// that cannot let a library allocate device memory. Examples are a host code that reserves
// all device memory for its own pool up front, so a cudaMalloc here would fail or break its
// budget, and a time-critical loop that must not pay for cudaMalloc/cudaFree, which may
// synchronise the device.
//
// Everything the solve needs besides the caller's input and output lives in one fixed
// device array compiled into the library: the eigenvector tables, the 1/den table and two
// intermediate plane stacks. Each GPU that loads libridc.so holds the array (2.5 MiB) until
// the process exits. Sizes beyond its capacity (n > 128 or more than 8 planes) are rejected
// with RIDC_ERR_UNSUPPORTED.
//
// In host code the array's name stands for a host-side shadow, not a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress (with that device
// current) and every kernel receives it as a pointer. The address is kept per device together
// with the identity of the device's CUDA context; when that context has been replaced (the
// caller ran cudaDeviceReset), the next call looks the address up again.
#include <cuda.h>
#include <mutex>

#include "ridc_internal.h"

namespace {

constexpr int kFixMaxN = 128;
constexpr int kFixMaxPlanes = 8;
constexpr size_t kFixNN = (size_t)kFixMaxN * kFixMaxN;
// Q | Q^T | 1/den for two species | two intermediate stacks of kFixMaxPlanes planes
constexpr size_t kFixQ = 0, kFixQt = kFixNN, kFixInv = 2 * kFixNN, kFixT1 = 4 * kFixNN,
                 kFixT2 = kFixT1 + kFixMaxPlanes * kFixNN,
                 kFixDoubles = kFixT2 + kFixMaxPlanes * kFixNN;   // 2.5 MiB

constexpr int kFixMaxDevices = 64;
// per device: the array's device address and the id of the context it was looked up in
struct FixAddr {
  double* base = nullptr;
  unsigned long long ctx_id = 0;
};
FixAddr g_fix_addr[kFixMaxDevices];
std::mutex g_fix_mu;

}  // namespace

static __device__ __align__(256) double g_fix_scratch[kFixDoubles];

namespace {

// Eigenvectors Q[x][k] of the 1D cell-centred Laplacian (cosines for the even ghost, sines at
// frequencies k+1 for the odd ghost), their transpose, and 1/(1 - dt nu_s (lam_ky + lam_kx)).
// One thread per (x, k); the angle pi t / 2n is reduced exactly in integers first.
__global__ void fix_tables_kernel(double* base, int n, int odd, double dt, double nu0,
                                  double nu1) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int x = blockIdx.y;
  if (k >= n) return;
  const long K = odd ? k + 1 : k;
  const double c = (odd ? (K == n) : (K == 0)) ? sqrt(1.0 / n) : sqrt(2.0 / n);
  const long t = (K * (2L * x + 1)) % (4L * n);
  double s, co;
  sincospi((double)t / (2.0 * n), &s, &co);
  const double q = c * (odd ? s : co);
  base[kFixQ + (size_t)x * n + k] = q;
  base[kFixQt + (size_t)k * n + x] = q;
  // x doubles as ky and k as kx for the denominator table [s][ky][kx]
  const long Ky = odd ? x + 1 : x;
  const double sx = sinpi((double)K / (2.0 * n)), sy = sinpi((double)Ky / (2.0 * n));
  const double lam = -4.0 * (double)n * (double)n * (sx * sx + sy * sy);
  base[kFixInv + (size_t)x * n + k] = 1.0 / (1.0 - dt * nu0 * lam);
  base[kFixInv + kFixNN + (size_t)x * n + k] = 1.0 / (1.0 - dt * nu1 * lam);
}

// C[row][m] = sum_k A[row][k] B[m][k] (rows = planes * n), stored as out[plane][m][row % n],
// optionally times inv_den[plane % S][m][row % n]. 64 x 64 tile, 4 x 4 per thread, FP64 DFMA.
template <bool SCALE>
__global__ void __launch_bounds__(256) fix_gemm_kernel(const double* __restrict__ A,
                                                       const double* __restrict__ B,
                                                       double* __restrict__ out,
                                                       const double* __restrict__ inv, int n,
                                                       int rows, int S) {
  __shared__ double As[16][66];
  __shared__ double Bs[16][66];
  const int t = threadIdx.x, tr = t & 15, tc = t >> 4;
  const int row0 = blockIdx.x * 64, col0 = blockIdx.y * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 16) {
    const int lr = t >> 2, lk = (t & 3) * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + lk + q;
      As[lk + q][lr] = (row0 + lr < rows && k < n) ? A[(long)(row0 + lr) * n + k] : 0.0;
      Bs[lk + q][lr] = (col0 + lr < n && k < n) ? B[(long)(col0 + lr) * n + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(As[kk][tr * 4 + i], Bs[kk][tc * 4 + j], acc[i][j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + tr * 4 + i;
    if (gr >= rows) continue;
    const int plane = gr / n, rl = gr - plane * n;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = col0 + tc * 4 + j;
      if (m >= n) continue;
      double v = acc[i][j];
      if (SCALE) v *= inv[(size_t)(plane % S) * kFixNN + (size_t)m * n + rl];
      out[((long)plane * n + m) * n + rl] = v;
    }
  }
}

// Unique id of the current device's CUDA context (cuCtxGetCurrent + cuCtxGetId through the
// runtime's driver entry points; ids are never reused within a process).
int fix_current_context_id(int dev, unsigned long long* id) {
  using namespace ridc;
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(f);
  });
  if (!get_current || !get_id) return RIDC_ERR_CUDA;
  // cudaSetDevice initialises the device's primary context and makes it current (it
  // allocates nothing; the device is the current one already)
  const cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return cuda_status(e);
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return RIDC_ERR_CUDA;
  if (get_id(ctx, id) != CUDA_SUCCESS) return RIDC_ERR_CUDA;
  return RIDC_OK;
}

}  // namespace

extern "C" int ridc_solve_planes_fixed(int kind, int n, const double* nu, double dt,
                                       const double* r, double* delta, int nplanes,
                                       void* stream) {
  using namespace ridc;
  if (!nu || !r || !delta) return RIDC_ERR_ARG;
  if (kind != RIDC_GRAY_SCOTT_2D_NEUMANN && kind != RIDC_ADV_DIFF_2D_DIRICHLET) return RIDC_ERR_ARG;
  if (n < 4 || nplanes < 1 || !(dt > 0.0) || !isfinite(dt)) return RIDC_ERR_ARG;
  const int S = (kind == RIDC_GRAY_SCOTT_2D_NEUMANN) ? 2 : 1;
  for (int s = 0; s < S; ++s)
    if (!(nu[s] > 0.0) || !isfinite(nu[s])) return RIDC_ERR_ARG;
  if (n > kFixMaxN || nplanes > kFixMaxPlanes) return RIDC_ERR_UNSUPPORTED;

  // an error left pending by an earlier, unrelated call is the caller's: report it and
  // leave it in place instead of clearing it here
  if (cudaPeekAtLastError() != cudaSuccess) return RIDC_ERR_CUDA;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= kFixMaxDevices) return RIDC_ERR_UNSUPPORTED;
  unsigned long long ctx_id = 0;
  RIDC_TRY(fix_current_context_id(dev, &ctx_id));
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_fix_mu);
    FixAddr& fa = g_fix_addr[dev];
    if (!fa.base || fa.ctx_id != ctx_id) {
      // set-up, once per device context, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_fix_scratch);
      if (e != cudaSuccess) return cuda_status(e);
      fa.base = static_cast<double*>(p);
      fa.ctx_id = ctx_id;
    }
    base = fa.base;
  }

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int rows = nplanes * n;
  fix_tables_kernel<<<dim3((n + 127) / 128, n), 128, 0, st>>>(
      base, n, kind == RIDC_ADV_DIFF_2D_DIRICHLET, dt, nu[0], nu[S - 1]);
  const dim3 grid((rows + 63) / 64, (n + 63) / 64);
  const double* Q = base + kFixQ;
  const double* Qt = base + kFixQt;
  const double* inv = base + kFixInv;
  double* t1 = base + kFixT1;
  double* t2 = base + kFixT2;
  fix_gemm_kernel<false><<<grid, 256, 0, st>>>(r, Qt, t1, inv, n, rows, S);
  fix_gemm_kernel<true><<<grid, 256, 0, st>>>(t1, Qt, t2, inv, n, rows, S);
  fix_gemm_kernel<false><<<grid, 256, 0, st>>>(t2, Q, t1, inv, n, rows, S);
  fix_gemm_kernel<false><<<grid, 256, 0, st>>>(t1, Q, delta, inv, n, rows, S);
  // nothing was pending on entry, so an error now comes from these launches
  return cuda_status(cudaPeekAtLastError());
}
