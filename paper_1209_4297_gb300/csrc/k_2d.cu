// 2D device kernels of one pipeline step, all FP64 except the BF16 split outputs:
//   rhs_kernel       right-hand side of every advancing level in delta form (eq. (pred),
//                    eq. (corr)), with the Lagrange quadrature of Section III-C; elementwise.
//   finalize_kernel  eta_{n+1} = base + delta, then f^N(eta) and f = f^N + D eta of the new
//                    state (5-point stencil from a shared-memory tile with ghost cells).
//   residual_kernel  refinement residual r - (I - dt nu L) delta of the mixed solve, split
//                    into BF16 hi/lo for the next tensor-core pass.
//   gemm_f64_kernel  FP64 fast-diagonalisation GEMM (DFMA; GB300's DMMA is slower than DFMA).
#include "ridc_internal.h"

namespace ridc {

// BF16 hi/lo split of an FP64 value: x ~= hi + lo with |x - hi - lo| <= 2^-17 |x| (about).
__device__ __forceinline__ void split2(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  const float f = (float)x;
  hi = __float2bfloat16_rn(f);
  lo = __float2bfloat16_rn(f - __bfloat162float(hi));
}

// ---------------------------------------------------------------------------------------------
// right-hand side: one level per blockIdx.y, S*N*N values, two per thread per iteration
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) rhs_kernel(const __grid_constant__ RhsArgs a) {
  const RhsLevel& L = a.lv[blockIdx.y];
  const long half = a.plane >> 1;
  const long out_off = (long)blockIdx.y * a.plane;
  const double2* Fn[kMaxOrder];
  const int nn = L.nnodes;
#pragma unroll
  for (int k = 0; k < kMaxOrder; ++k) Fn[k] = (k < nn) ? (const double2*)L.Fn[k] : nullptr;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < half;
       i += (long)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    if (L.eta_j) {
      const double2 e = ((const double2*)L.eta_j)[i], ep = ((const double2*)L.eta_pn)[i];
      const double2 f = ((const double2*)L.fN_j)[i], fp = ((const double2*)L.fN_p)[i];
      acc.x = fma(a.dt, f.x - fp.x, e.x - ep.x);
      acc.y = fma(a.dt, f.y - fp.y, e.y - ep.y);
    }
#pragma unroll
    for (int k = 0; k < kMaxOrder; ++k) {
      if (k < nn) {
        const double2 F = __ldg(Fn[k] + i);
        acc.x = fma(L.w[k], F.x, acc.x);
        acc.y = fma(L.w[k], F.y, acc.y);
      }
    }
    ((double2*)(a.r + out_off))[i] = acc;
    if (a.r_hi) {
      __nv_bfloat16 h0, l0, h1, l1;
      split2(acc.x, h0, l0);
      split2(acc.y, h1, l1);
      __nv_bfloat162 hv, lv;
      hv.x = h0; hv.y = h1;
      lv.x = l0; lv.y = l1;
      ((__nv_bfloat162*)(a.r_hi + out_off))[i] = hv;
      ((__nv_bfloat162*)(a.r_lo + out_off))[i] = lv;
    }
  }
}

int launch_rhs(Ctx* c, const RhsArgs& a) {
  const long half = a.plane / 2;
  long bx = (half + 255) / 256;
  const long cap = 148L * 16 / (a.nlev > 0 ? a.nlev : 1) + 1;
  if (bx > cap * 8) bx = cap * 8;
  dim3 grid((unsigned)bx, a.nlev);
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_RHS, &e0);
  rhs_kernel<<<grid, 256, 0, c->stream>>>(a);
  prof_end(c, RIDC_KERNEL_RHS, e0);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// tile loader with reflecting ghosts: even (Neumann) or odd (Dirichlet) continuation
// ---------------------------------------------------------------------------------------------
constexpr int TX = 32, TY = 8;

// Fills tile[TY+2][TX+2] with (x + d) around (x0, y0), ghosts by reflection with `sign`.
__device__ __forceinline__ void load_tile(double (*tile)[TX + 2], const double* __restrict__ x,
                                          const double* __restrict__ d, int n, int x0, int y0,
                                          double sign) {
  for (int idx = threadIdx.y * TX + threadIdx.x; idx < (TY + 2) * (TX + 2); idx += TX * TY) {
    const int ly = idx / (TX + 2), lx = idx % (TX + 2);
    int gy = y0 + ly - 1, gx = x0 + lx - 1;
    double sg = 1.0;
    if (gy < 0) { gy = 0; sg *= sign; }
    if (gy >= n) { gy = n - 1; sg *= sign; }
    if (gx < 0) { gx = 0; sg *= sign; }
    if (gx >= n) { gx = n - 1; sg *= sign; }
    const long o = (long)gy * n + gx;
    double v = x[o];
    if (d) v += d[o];
    tile[ly][lx] = sg * v;
  }
}

// ---------------------------------------------------------------------------------------------
// new state of every advancing level: eta = base + delta, f^N(eta), f = f^N + nu L eta
// ---------------------------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(TX * TY) finalize_kernel(const __grid_constant__ FinArgs a) {
  constexpr int S = (KIND == RIDC_GRAY_SCOTT_2D_NEUMANN) ? 2 : 1;
  constexpr double sign = (KIND == RIDC_ADV_DIFF_2D_DIRICHLET) ? -1.0 : 1.0;
  __shared__ double tile[S][TY + 2][TX + 2];
  const FinLevel& L = a.lv[blockIdx.z];
  const int n = a.n;
  const long nn = (long)n * n;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
#pragma unroll
  for (int s = 0; s < S; ++s)
    load_tile(tile[s], L.base + s * nn, L.delta ? L.delta + s * nn : nullptr, n, x0, y0, sign);
  __syncthreads();
  const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
  const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
  if (gx >= n || gy >= n) return;
  const long o = (long)gy * n + gx;
  double u[S], lap[S], fn[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    u[s] = tile[s][ty][tx];
    lap[s] = ((tile[s][ty - 1][tx] + tile[s][ty + 1][tx]) + (tile[s][ty][tx - 1] + tile[s][ty][tx + 1]))
             - 4.0 * u[s];
  }
  if (KIND == RIDC_GRAY_SCOTT_2D_NEUMANN) {
    const double uvv = u[0] * u[S - 1] * u[S - 1];
    fn[0] = fma(a.gsF, 1.0 - u[0], -uvv);
    fn[S - 1] = fma(-(a.gsF + a.gsk), u[S - 1], uvv);
  } else {
    fn[0] = -a.a2h * (tile[0][ty][tx + 1] - tile[0][ty][tx - 1])
            - a.b2h * (tile[0][ty + 1][tx] - tile[0][ty - 1][tx]);
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if (L.delta) L.eta[s * nn + o] = u[s];
    L.fN[s * nn + o] = fn[s];
    if (L.F) L.F[s * nn + o] = fma(a.c_lap[s], lap[s], fn[s]);
  }
}

int launch_finalize(Ctx* c, const FinArgs& a) {
  dim3 grid((a.n + TX - 1) / TX, (a.n + TY - 1) / TY, a.nlev);
  dim3 block(TX, TY);
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_FINALIZE, &e0);
  if (a.kind == RIDC_GRAY_SCOTT_2D_NEUMANN)
    finalize_kernel<RIDC_GRAY_SCOTT_2D_NEUMANN><<<grid, block, 0, c->stream>>>(a);
  else
    finalize_kernel<RIDC_ADV_DIFF_2D_DIRICHLET><<<grid, block, 0, c->stream>>>(a);
  prof_end(c, RIDC_KERNEL_FINALIZE, e0);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// refinement residual of the mixed solve: r' = r - delta + dt nu_s L delta, split to BF16
// ---------------------------------------------------------------------------------------------
struct ResArgs {
  const double* r;
  const double* delta;      // nullptr on the first pass: r' = r
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  int n, S;
  double c[kMaxSpecies];    // dt nu_s / h^2
  double sign;
};

__global__ void __launch_bounds__(TX * TY) residual_kernel(const __grid_constant__ ResArgs a) {
  __shared__ double tile[TY + 2][TX + 2];
  const int n = a.n;
  const long nn = (long)n * n;
  const int p = blockIdx.z;
  const long off = (long)p * nn;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
  double v;
  if (a.delta) {
    load_tile(tile, a.delta + off, nullptr, n, x0, y0, a.sign);
    __syncthreads();
    if (gx >= n || gy >= n) return;
    const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
    const double d = tile[ty][tx];
    const double lap = ((tile[ty - 1][tx] + tile[ty + 1][tx]) + (tile[ty][tx - 1] + tile[ty][tx + 1]))
                       - 4.0 * d;
    v = fma(a.c[p % a.S], lap, a.r[off + (long)gy * n + gx] - d);
  } else {
    if (gx >= n || gy >= n) return;
    v = a.r[off + (long)gy * n + gx];
  }
  __nv_bfloat16 h, l;
  split2(v, h, l);
  a.hi[off + (long)gy * n + gx] = h;
  a.lo[off + (long)gy * n + gx] = l;
}

int launch_residual(Ctx* c, int nplanes, int first) {
  ResArgs a{};
  a.r = c->r;
  a.delta = first ? nullptr : c->delta;
  a.hi = c->xh;
  a.lo = c->xl;
  a.n = c->n;
  a.S = c->S;
  for (int s = 0; s < c->S; ++s) a.c[s] = c->dt * c->nu[s] / (c->h * c->h);
  a.sign = (c->kind == RIDC_ADV_DIFF_2D_DIRICHLET) ? -1.0 : 1.0;
  dim3 grid((c->n + TX - 1) / TX, (c->n + TY - 1) / TY, nplanes);
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_RESIDUAL, &e0);
  residual_kernel<<<grid, dim3(TX, TY), 0, c->stream>>>(a);
  prof_end(c, RIDC_KERNEL_RESIDUAL, e0);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// finite check (sets *flag = 1 if any value is NaN or Inf)
// ---------------------------------------------------------------------------------------------
__global__ void check_finite_kernel(const double* x, long count, int* flag) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
       i += (long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) { *flag = 1; return; }
}

int launch_check_finite(Ctx* c, const double* x, long count, int* flag_dev) {
  long blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  check_finite_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(x, count, flag_dev);
  c->launches++;
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// FP64 fast-diagonalisation GEMM:
//   C[row][m] = sum_k A[row][k] B[m][k],  rows = nplanes * N (planes stacked), m, k < N,
//   stored transposed per plane: out[plane][m][row % N] (times 1/den for EPI_SCALE_DEN).
// 64x64 output tile per 256-thread block, 16-deep K slices staged transposed in shared memory,
// 4x4 register tile per thread; consecutive threads own consecutive rows so the transposed
// store writes 512 contiguous bytes per column.
// ---------------------------------------------------------------------------------------------
constexpr int GB = 64, GK = 16;

template <int EPI>
__global__ void __launch_bounds__(256) gemm_f64_kernel(const double* __restrict__ A,
                                                       const double* __restrict__ B,
                                                       double* __restrict__ out,
                                                       const double* __restrict__ inv_den, int n,
                                                       int rows, int S) {
  __shared__ __align__(16) double As[GK][GB + 2];
  __shared__ __align__(16) double Bs[GK][GB + 2];
  const int t = threadIdx.x;
  const int tr = t & 15, tc = t >> 4;
  const int row0 = blockIdx.x * GB, col0 = blockIdx.y * GB;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += GK) {
    // 64 x 16 slices of A and B: thread t loads 4 consecutive k of one row
#pragma unroll
    for (int h = 0; h < 1; ++h) {
      const int lr = t >> 2, lk = (t & 3) * 4;
      const int gr = row0 + lr, gc = col0 + lr;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + lk + q;
        As[lk + q][lr] = (gr < rows && k < n) ? A[(long)gr * n + k] : 0.0;
        Bs[lk + q][lr] = (gc < n && k < n) ? B[(long)gc * n + k] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][tr * 4 + i]; b[i] = Bs[kk][tc * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
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
      if (EPI == EPI_SCALE_DEN) v *= inv_den[((long)(plane % S) * n + m) * n + rl];
      out[((long)plane * n + m) * n + rl] = v;
    }
  }
}

int launch_gemm_f64(Ctx* c, const double* A, const double* B, double* out, int nplanes, int epi) {
  const int n = c->n, rows = nplanes * n;
  dim3 grid((rows + GB - 1) / GB, (n + GB - 1) / GB);
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_GEMM_F64, &e0);
  if (epi == EPI_SCALE_DEN)
    gemm_f64_kernel<EPI_SCALE_DEN><<<grid, 256, 0, c->stream>>>(A, B, out, c->inv_den, n, rows, c->S);
  else
    gemm_f64_kernel<EPI_STORE><<<grid, 256, 0, c->stream>>>(A, B, out, c->inv_den, n, rows, c->S);
  prof_end(c, RIDC_KERNEL_GEMM_F64, e0);
  return cuda_status(cudaGetLastError());
}

}  // namespace ridc
