// 2D device kernels of one pipeline step, all FP64 except the split outputs:
//   rhs_kernel       right-hand side of every advancing level in delta form (eq. (pred),
//                    eq. (corr)), with the Lagrange quadrature of Section III-C; elementwise.
//   finalize_kernel  eta_{n+1} = base + delta, then f^N(eta) and f = f^N + D eta of the new
//                    state (5-point stencil from a shared-memory tile with ghost cells).
//   residual_kernel  refinement residual r - (I - dt nu L) delta of the mixed solve, parity-
//                    split along both axes and split into BF16 hi/lo for the next
//                    tensor-core pass (FP16 form: staged in FP32 with the plane maxima).
//   split_f16_kernel FP16 form: scales each staged plane by its power of two and splits it
//                    into FP16 hi/lo.
//   gemm_f64_kernel  FP64 fast-diagonalisation GEMM (DFMA; GB300's DMMA is slower than DFMA),
//                    parity-split for even n (gemm_f64_split_kernel).
#include "ridc_internal.h"

namespace ridc {

// GB300 executes FP64 arithmetic and FP64<->FP32 conversions on its narrow FP64 pipe (about
// 2 operations per clock per SM), so the kernels below do format conversions and ghost-cell
// sign flips with integer bit operations, which run on the full-rate integer pipes.

// FP64 -> FP32, round to nearest even, from the IEEE-754 formats: keep the top 23 of the 52
// mantissa bits; a carry out of the mantissa bumps the exponent. Magnitudes below the FP32
// normal range become signed zero (they are below 1.2e-38, far under every tolerance here);
// magnitudes above it become infinity and NaN stays NaN, so a blow-up stays visible.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ef = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7F800000u | ((ef == 1151 && m) ? 0x400000u : 0u));
  const unsigned long long mr = m + 0xFFFFFFFull + ((m >> 29) & 1ull);
  return __uint_as_float(sign | (unsigned)(((unsigned long long)ef << 23) + (mr >> 29)));
}

// FP32 -> FP64, exact for normal values; FP32 subnormals (below 1.2e-38) become signed zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFF;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ed = (e == 255) ? 2047ull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

__device__ __forceinline__ double flip_sign(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}

// ---------------------------------------------------------------------------------------------
// right-hand side: one level per blockIdx.y, S*N*N values, two per thread per iteration.
// The quadrature has exactly NODES terms per level (a switch picks the instantiation): on
// GB300 a predicated-off FP64 instruction still occupies the FP64 pipe, so no FP64 work may
// be issued for absent nodes.
// ---------------------------------------------------------------------------------------------
// COMBO: the right-hand side of an ARK stage, sum_k w_k Fn_k (a separate instantiation, so
// that the corrector kernels keep their registers)
template <int NODES, bool COMBO>
__device__ __forceinline__ double2 rhs_at(const RhsArgs& a, const RhsLevel& L,
                                          const double2* const (&Fn)[NODES],
                                          const double (&w)[NODES], long i) {
  double2 acc;
  if (COMBO) {
    const double2 F = __ldg(Fn[0] + i);
    acc.x = w[0] * F.x;
    acc.y = w[0] * F.y;
#pragma unroll
    for (int k = 1; k < NODES; ++k) {
      const double2 G = __ldg(Fn[k] + i);
      acc.x = fma(w[k], G.x, acc.x);
      acc.y = fma(w[k], G.y, acc.y);
    }
  } else if (L.eta_j) {
    const double2 e = ((const double2*)L.eta_j)[i], ep = ((const double2*)L.eta_pn)[i];
    const double2 f = ((const double2*)L.fN_j)[i], fp = ((const double2*)L.fN_p)[i];
    acc.x = fma(a.dt, f.x - fp.x, e.x - ep.x);
    acc.y = fma(a.dt, f.y - fp.y, e.y - ep.y);
#pragma unroll
    for (int k = 0; k < NODES; ++k) {
      const double2 F = __ldg(Fn[k] + i);
      acc.x = fma(w[k], F.x, acc.x);
      acc.y = fma(w[k], F.y, acc.y);
    }
  } else {
    const double2 F = __ldg(Fn[0] + i);
    acc.x = w[0] * F.x;
    acc.y = w[0] * F.y;
  }
  return acc;
}

__device__ __forceinline__ void store_split2(__nv_bfloat16* hi, __nv_bfloat16* lo, long idx,
                                             float v0, float v1) {
  __nv_bfloat162 hv, lv;
  hv.x = __float2bfloat16_rn(v0);
  hv.y = __float2bfloat16_rn(v1);
  lv.x = __float2bfloat16_rn(v0 - __bfloat162float(hv.x));
  lv.y = __float2bfloat16_rn(v1 - __bfloat162float(hv.y));
  *reinterpret_cast<__nv_bfloat162*>(hi + idx) = hv;
  *reinterpret_cast<__nv_bfloat162*>(lo + idx) = lv;
}

// one value, in the same operation order as rhs_at (the FP64 path of odd planes: one species
// and odd n make n^2 odd, so ring slots are only 8-byte aligned and double2 cannot be used)
template <int NODES, bool COMBO>
__device__ __forceinline__ double rhs_at1(const RhsArgs& a, const RhsLevel& L, long i) {
  if (COMBO) {
    double acc = L.w[0] * __ldg(L.Fn[0] + i);
#pragma unroll
    for (int k = 1; k < NODES; ++k) acc = fma(L.w[k], __ldg(L.Fn[k] + i), acc);
    return acc;
  }
  if (L.eta_j) {
    double acc = fma(a.dt, L.fN_j[i] - L.fN_p[i], L.eta_j[i] - L.eta_pn[i]);
#pragma unroll
    for (int k = 0; k < NODES; ++k) acc = fma(L.w[k], __ldg(L.Fn[k] + i), acc);
    return acc;
  }
  return L.w[0] * __ldg(L.Fn[0] + i);
}

// FP16 form: v0, v1 staged in FP32 (8-byte aligned: idx is even)
__device__ __forceinline__ void store_stage2(float* st, long idx, float v0, float v1) {
  *reinterpret_cast<float2*>(st + idx) = make_float2(v0, v1);
}

// running maximum of |v| as FP32 bits (non-negative floats order like their bit patterns;
// a NaN's bits exceed every finite value's, so a NaN plane keeps a non-finite maximum)
__device__ __forceinline__ unsigned abs_bits_max(unsigned m, float v) {
  const unsigned b = __float_as_uint(v) & 0x7FFFFFFFu;
  return b > m ? b : m;
}

// warp-wide maximum, then one atomic per warp (every lane of the warp active)
__device__ __forceinline__ void flush_plane_max(unsigned* pmax, unsigned m) {
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(pmax, m);
}

// STAGE: the FP16 form (FP32 staging and plane maxima); a separate instantiation keeps the
// FP64 and BF16 code free of its branches and registers
template <int NODES, bool STAGE, bool COMBO>
__device__ __forceinline__ void rhs_level(const RhsArgs& a, const RhsLevel& L, long out_off) {
  const double2* Fn[NODES];
  double w[NODES];
#pragma unroll
  for (int k = 0; k < NODES; ++k) {
    Fn[k] = (const double2*)L.Fn[k];
    w[k] = L.w[k];
  }
  double2* r2 = (double2*)(a.r + out_off);
  if (!STAGE && !a.r_hi) {
    const long half = a.plane >> 1;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < half;
         i += (long)gridDim.x * blockDim.x)
      r2[i] = rhs_at<NODES, COMBO>(a, L, Fn, w, i);
    return;
  }
  // mixed form: each thread takes cells (2q, 2q+1) of rows y and n-1-y (y < n/2) and their
  // mirrors (n-2-2q, n-1-2q), and also writes the parity split along both axes of the FP32
  // values, v[gx][gy] = (v[y][x'] +- v[y][n-1-x']) +- (v[n-1-y][x'] +- v[n-1-y][n-1-x']),
  // as BF16 hi/lo (layout [plane][gx][gy][y'][x'], x', y' < n/2)
  const int n = a.n, q4 = n / 4, H = n / 2;
  const long nn = (long)n * n, cells = a.plane / 8;
  const long plane0 = out_off / nn;   // first plane of this level in the stacked operand
  // FP16 form: running max of the staged values of plane `mp` (cells per plane, n^2 / 8, and
  // the grid stride are multiples of 32, so a warp's lanes always share one plane)
  unsigned mx = 0;
  long mp = -1;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < cells;
       e += (long)gridDim.x * blockDim.x) {
    const long sp = e / ((long)H * q4), rem = e - sp * (long)H * q4;
    const int y = (int)(rem / q4), q = (int)(rem - (long)y * q4);
    float v[2][4];   // [row: y, n-1-y][x: 2q, 2q+1, n-1-2q, n-2-2q]
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const long rowoff = sp * nn + (long)(side ? n - 1 - y : y) * n;
      const long iL = (rowoff + 2 * q) >> 1, iR = (rowoff + n - 2 - 2 * q) >> 1;
      const double2 vL = rhs_at<NODES, COMBO>(a, L, Fn, w, iL);
      const double2 vR = rhs_at<NODES, COMBO>(a, L, Fn, w, iR);
      r2[iL] = vL;
      r2[iR] = vR;
      v[side][0] = f64_to_f32(vL.x);
      v[side][1] = f64_to_f32(vL.y);
      v[side][2] = f64_to_f32(vR.y);   // mirror of 2q
      v[side][3] = f64_to_f32(vR.x);   // mirror of 2q+1
    }
    const long p = plane0 + sp;
    if (STAGE && p != mp) {
      if (mp >= 0) flush_plane_max(a.pmax + mp, mx);
      mp = p;
      mx = 0;
    }
#pragma unroll
    for (int gx = 0; gx < 2; ++gx) {
      // x butterfly of each row, then y butterfly
      const float s = gx ? -1.f : 1.f;
      const float a0 = v[0][0] + s * v[0][2], a1 = v[0][1] + s * v[0][3];
      const float b0 = v[1][0] + s * v[1][2], b1 = v[1][1] + s * v[1][3];
      const long base = ((p * 2 + gx) * n + y) * H + 2 * q;   // gy = 0 block; gy = 1 is H rows on
      if (STAGE) {
        store_stage2(a.r_stage, base, a0 + b0, a1 + b1);
        store_stage2(a.r_stage, base + (long)H * H, a0 - b0, a1 - b1);
        mx = abs_bits_max(abs_bits_max(mx, a0 + b0), a1 + b1);
        mx = abs_bits_max(abs_bits_max(mx, a0 - b0), a1 - b1);
      } else {
        store_split2(a.r_hi, a.r_lo, base, a0 + b0, a1 + b1);
        store_split2(a.r_hi, a.r_lo, base + (long)H * H, a0 - b0, a1 - b1);
      }
    }
  }
  if (STAGE && mp >= 0) flush_plane_max(a.pmax + mp, mx);
}

// FP64 right-hand side of odd planes (one species, odd n), one value per thread and step
template <int NODES, bool COMBO>
__device__ __forceinline__ void rhs_level_scalar(const RhsArgs& a, const RhsLevel& L,
                                                 long out_off) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < a.plane;
       i += (long)gridDim.x * blockDim.x)
    a.r[out_off + i] = rhs_at1<NODES, COMBO>(a, L, i);
}

template <bool COMBO>
__global__ void __launch_bounds__(256) rhs_scalar_kernel(const __grid_constant__ RhsArgs a) {
  const RhsLevel& L = a.lv[blockIdx.y];
  const long out_off = (long)blockIdx.y * a.plane;
  switch (L.nnodes) {
    case 1: rhs_level_scalar<1, COMBO>(a, L, out_off); break;
    case 2: rhs_level_scalar<2, COMBO>(a, L, out_off); break;
    case 3: rhs_level_scalar<3, COMBO>(a, L, out_off); break;
    case 4: rhs_level_scalar<4, COMBO>(a, L, out_off); break;
    case 5: rhs_level_scalar<5, COMBO>(a, L, out_off); break;
    case 6: rhs_level_scalar<6, COMBO>(a, L, out_off); break;
    case 7: rhs_level_scalar<7, COMBO>(a, L, out_off); break;
    case 8: rhs_level_scalar<8, COMBO>(a, L, out_off); break;
    case 9: rhs_level_scalar<9, COMBO>(a, L, out_off); break;
    case 10: rhs_level_scalar<10, COMBO>(a, L, out_off); break;
    case 11: rhs_level_scalar<11, COMBO>(a, L, out_off); break;
    default: rhs_level_scalar<12, COMBO>(a, L, out_off); break;
  }
}

// the corrector kernels are capped at 64 registers (32 warps per SM); the ARK-stage sums,
// with up to 12 terms held for two cells of four rows, keep 128
template <bool STAGE, bool COMBO>
__global__ void __launch_bounds__(256, COMBO ? 2 : 4) rhs_kernel(const __grid_constant__ RhsArgs a) {
  const RhsLevel& L = a.lv[blockIdx.y];
  const long out_off = (long)blockIdx.y * a.plane;
  switch (L.nnodes) {
    case 1: rhs_level<1, STAGE, COMBO>(a, L, out_off); break;
    case 2: rhs_level<2, STAGE, COMBO>(a, L, out_off); break;
    case 3: rhs_level<3, STAGE, COMBO>(a, L, out_off); break;
    case 4: rhs_level<4, STAGE, COMBO>(a, L, out_off); break;
    case 5: rhs_level<5, STAGE, COMBO>(a, L, out_off); break;
    case 6: rhs_level<6, STAGE, COMBO>(a, L, out_off); break;
    case 7: rhs_level<7, STAGE, COMBO>(a, L, out_off); break;
    case 8: rhs_level<8, STAGE, COMBO>(a, L, out_off); break;
    case 9: rhs_level<9, STAGE, COMBO>(a, L, out_off); break;
    case 10: rhs_level<10, STAGE, COMBO>(a, L, out_off); break;
    case 11: rhs_level<11, STAGE, COMBO>(a, L, out_off); break;
    default: rhs_level<12, STAGE, COMBO>(a, L, out_off); break;
  }
}

template <bool COMBO>
static void launch_rhs_kind(Ctx* c, const RhsArgs& a, dim3 grid) {
  if (a.r_stage)
    rhs_kernel<true, COMBO><<<grid, 256, 0, c->stream>>>(a);
  else if (!a.r_hi && (a.plane & 1))   // FP64, odd plane: fields only 8-byte aligned
    rhs_scalar_kernel<COMBO><<<grid, 256, 0, c->stream>>>(a);
  else
    rhs_kernel<false, COMBO><<<grid, 256, 0, c->stream>>>(a);
}

int launch_rhs(Ctx* c, const RhsArgs& a) {
  const long half = (a.r_hi || a.r_stage) ? a.plane / 8 : a.plane / 2;
  long bx = (half + 255) / 256;
  const long cap = 148L * 16 / (a.nlev > 0 ? a.nlev : 1) + 1;
  if (bx > cap * 8) bx = cap * 8;
  dim3 grid((unsigned)bx, a.nlev);
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_RHS, &e0);
  if (a.combo) launch_rhs_kind<true>(c, a, grid);
  else launch_rhs_kind<false>(c, a, grid);
  prof_end(c, RIDC_KERNEL_RHS, e0);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// tile loader with reflecting ghosts: even (Neumann) or odd (Dirichlet) continuation
// ---------------------------------------------------------------------------------------------
// A 256-thread block (32 x 8) covers a 32 x 32 tile, four rows per thread; the one-cell halo
// costs 34*34/(32*32) = 1.13 loads per cell.
constexpr int TX = 32, TY = 32, BY = 8, RPT = TY / BY;

// tile[TY+2][TX+2] = (x + d64 + d32) around (x0, y0); ghost cells take the mirrored value,
// negated for the odd continuation (ODD). Absent addends are nullptr.
template <bool ODD>
__device__ __forceinline__ void load_tile(double (*tile)[TX + 2], const double* __restrict__ x,
                                          const double* __restrict__ d64,
                                          const float* __restrict__ d32, int n, int x0, int y0) {
  for (int idx = threadIdx.y * TX + threadIdx.x; idx < (TY + 2) * (TX + 2); idx += TX * BY) {
    const int ly = idx / (TX + 2), lx = idx - ly * (TX + 2);
    int gy = y0 + ly - 1, gx = x0 + lx - 1;
    bool neg = false;
    if (gy < 0) { gy = 0; neg = !neg; }
    if (gy >= n) { gy = n - 1; neg = !neg; }
    if (gx < 0) { gx = 0; neg = !neg; }
    if (gx >= n) { gx = n - 1; neg = !neg; }
    const long o = (long)gy * n + gx;
    double v = x ? x[o] : 0.0;
    if (d64) v = x ? v + d64[o] : d64[o];
    if (d32) v = (x || d64) ? v + f32_to_f64(d32[o]) : f32_to_f64(d32[o]);
    tile[ly][lx] = ODD ? flip_sign(v, neg) : v;
  }
}

// ---------------------------------------------------------------------------------------------
// new state of every advancing level: eta = base + delta, f^N(eta), f = f^N + nu L eta
// ---------------------------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(TX * BY) finalize_kernel(const __grid_constant__ FinArgs a) {
  constexpr int S = (KIND == RIDC_GRAY_SCOTT_2D_NEUMANN) ? 2 : 1;
  constexpr bool ODD = (KIND == RIDC_ADV_DIFF_2D_DIRICHLET);
  __shared__ double tile[S][TY + 2][TX + 2];
  const FinLevel& L = a.lv[blockIdx.z];
  const int n = a.n;
  const long nn = (long)n * n;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
#pragma unroll
  for (int s = 0; s < S; ++s)
    load_tile<ODD>(tile[s], L.base + s * nn, L.d64 ? L.d64 + s * nn : nullptr,
                   L.d32 ? L.d32 + s * nn : nullptr, n, x0, y0);
  __syncthreads();
  const int tx = threadIdx.x + 1;
  const int gx = x0 + threadIdx.x;
  if (gx >= n) return;
  const bool new_state = L.d64 || L.d32;
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int ty = threadIdx.y + rr * BY + 1, gy = y0 + ty - 1;
    if (gy >= n) break;
    const long o = (long)gy * n + gx;
    double u[S], fn[S];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = tile[s][ty][tx];
    if (KIND == RIDC_GRAY_SCOTT_2D_NEUMANN) {
      const double uvv = u[0] * u[S - 1] * u[S - 1];
      fn[0] = fma(a.gsF, 1.0 - u[0], -uvv);
      fn[S - 1] = fma(a.gsFk, u[S - 1], uvv);
    } else {
      fn[0] = -a.a2h * (tile[0][ty][tx + 1] - tile[0][ty][tx - 1])
              - a.b2h * (tile[0][ty + 1][tx] - tile[0][ty - 1][tx]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (new_state) L.eta[s * nn + o] = u[s];
      L.fN[s * nn + o] = fn[s];
      if (L.F) {
        // f = f^N + c (N + S + W + E) - 4 c u,  c = nu_s / h^2
        const double sum = (tile[s][ty - 1][tx] + tile[s][ty + 1][tx]) +
                           (tile[s][ty][tx - 1] + tile[s][ty][tx + 1]);
        L.F[s * nn + o] = fma(a.c_lap[s], sum, fma(a.c_lap4[s], u[s], fn[s]));
      }
    }
  }
}

int launch_finalize(Ctx* c, const FinArgs& a) {
  dim3 grid((a.n + TX - 1) / TX, (a.n + TY - 1) / TY, a.nlev);
  dim3 block(TX, BY);
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
// refinement residual of the mixed solve:
//   d = dprev + inc  (written to dout),   r' = r - (I - c_s L) d = r - (1 + 4 c_s) d + c_s (N+S+W+E)
// with c_s = dt nu_s / h^2, then r' split to BF16 hi/lo (FP16 form: staged in FP32, with the
// plane maxima). Without dprev and inc: r' = r.
// ---------------------------------------------------------------------------------------------
struct ResArgs {
  const double* r;
  const double* dprev;
  const float* inc;
  double* dout;
  __nv_bfloat16* hi;        // parity-split operand [plane][gx][gy][y'][x'], x', y' < n/2
  __nv_bfloat16* lo;
  float* stage;             // FP16 form: the same values in FP32 (else nullptr)
  unsigned* pmax;           // FP16 form: per-plane maxima of this solve pass
  int n, S, plane0;
  double c[kMaxPlanes];     // c_p = a_p dt nu_s / h^2 of plane p (a_p: its operator's diagonal)
  double c1[kMaxPlanes];    // -(1 + 4 c_p)
};

// One block covers a 32 x 32 tile at (x0, y0), x0, y0 < n/2, and its three mirror tiles
// (n-32-x0 and/or n-32-y0): it forms r' on all four, then the parity split along both axes,
// (r'[y'][x'] +- r'[y'][n-1-x']) +- (r'[n-1-y'][x'] +- r'[n-1-y'][n-1-x']) (FP32), as BF16
// hi/lo in the layout [plane][gx][gy][y'][x'].
template <bool ODD>
__global__ void __launch_bounds__(TX * BY) residual_kernel(const __grid_constant__ ResArgs a) {
  __shared__ double tile[TY + 2][TX + 2];
  __shared__ float rv[4][TY][TX + 1];   // [sy * 2 + sx]
  const int n = a.n;
  const long nn = (long)n * n;
  const int p = a.plane0 + blockIdx.z;
  const long off = (long)p * nn;
  const bool has_d = a.dprev || a.inc;
  const double cs = a.c[p], c1 = a.c1[p];
  for (int side = 0; side < 4; ++side) {
    const int sx = side & 1, sy = side >> 1;
    const int x0 = sx == 0 ? blockIdx.x * TX : n - TX - blockIdx.x * TX;
    const int y0 = sy == 0 ? blockIdx.y * TY : n - TY - blockIdx.y * TY;
    if (has_d) {
      __syncthreads();
      load_tile<ODD>(tile, nullptr, a.dprev ? a.dprev + off : nullptr,
                     a.inc ? a.inc + off : nullptr, n, x0, y0);
      __syncthreads();
    }
    const int gx = x0 + threadIdx.x;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int ty = threadIdx.y + rr * BY + 1, gy = y0 + ty - 1;
      const long o = off + (long)gy * n + gx;
      double v = a.r[o];
      if (has_d) {
        const int tx = threadIdx.x + 1;
        const double d = tile[ty][tx];
        const double sum = (tile[ty - 1][tx] + tile[ty + 1][tx]) + (tile[ty][tx - 1] + tile[ty][tx + 1]);
        v = fma(cs, sum, fma(c1, d, v));
        a.dout[o] = d;
      }
      rv[side][ty - 1][threadIdx.x] = f64_to_f32(v);
    }
  }
  __syncthreads();
  const int H = n / 2;
  const int xp = blockIdx.x * TX + threadIdx.x;   // x' < n/2; its mirror is column 31 - tx
  unsigned vmax = 0;
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const int ly = threadIdx.y + rr * BY, yp = blockIdx.y * TY + ly;   // y' < n/2
    const int mx = TX - 1 - threadIdx.x, my = TY - 1 - ly;
    const float v00 = rv[0][ly][threadIdx.x], v01 = rv[1][ly][mx];
    const float v10 = rv[2][my][threadIdx.x], v11 = rv[3][my][mx];
#pragma unroll
    for (int gxp = 0; gxp < 2; ++gxp) {
      const float s = gxp ? -1.f : 1.f;
      const float top = v00 + s * v01, bot = v10 + s * v11;
      const long i0 = ((long)(p * 2 + gxp) * n + yp) * H + xp;   // gy = 0; gy = 1 is H rows on
      const long i1 = i0 + (long)H * H;
      const float vp = top + bot, vm = top - bot;
      if (a.stage) {
        a.stage[i0] = vp;
        a.stage[i1] = vm;
        vmax = abs_bits_max(abs_bits_max(vmax, vp), vm);
        continue;
      }
      __nv_bfloat16 h = __float2bfloat16_rn(vp);
      a.hi[i0] = h;
      a.lo[i0] = __float2bfloat16_rn(vp - __bfloat162float(h));
      h = __float2bfloat16_rn(vm);
      a.hi[i1] = h;
      a.lo[i1] = __float2bfloat16_rn(vm - __bfloat162float(h));
    }
  }
  if (a.stage) flush_plane_max(a.pmax + p, vmax);   // every thread of the block gets here
}

int launch_residual(Ctx* c, int plane0, int nplanes, const double* dprev, const float* inc,
                    double* dout, int pass) {
  ResArgs a{};
  a.plane0 = plane0;
  a.r = c->r;
  a.dprev = dprev;
  a.inc = inc;
  a.dout = dout;
  a.hi = c->xh;
  a.lo = c->xl;
  if (c->prec == RIDC_MIXED_FP16X3) {
    if (pass < 0 || pass >= kMaxPasses) return RIDC_ERR_ARG;
    a.stage = c->xs;
    a.pmax = c->pmax + (size_t)pass * kMaxPlanes;
  }
  a.n = c->n;
  a.S = c->S;
  if (plane0 < 0 || nplanes < 0 || plane0 + nplanes > kMaxPlanes) return RIDC_ERR_ARG;
  for (int p = plane0; p < plane0 + nplanes; ++p) {
    // (a dt) nu / h^2: with a = 1 exactly the correctors' dt nu / h^2
    a.c[p] = (c->coef[c->plane_coef[p]] * c->dt) * c->nu[p % c->S] / (c->h * c->h);
    a.c1[p] = -(1.0 + 4.0 * a.c[p]);
  }
  if (c->n % (2 * TX) != 0 || c->n % (2 * TY) != 0) return RIDC_ERR_UNSUPPORTED;
  dim3 grid(c->n / (2 * TX), c->n / (2 * TY), nplanes);
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_RESIDUAL, &e0);
  if (c->kind == RIDC_ADV_DIFF_2D_DIRICHLET)
    residual_kernel<true><<<grid, dim3(TX, BY), 0, c->stream>>>(a);
  else
    residual_kernel<false><<<grid, dim3(TX, BY), 0, c->stream>>>(a);
  prof_end(c, RIDC_KERNEL_RESIDUAL, e0);
  RIDC_TRY(cuda_status(cudaGetLastError()));
  return (c->prec == RIDC_MIXED_FP16X3) ? launch_split_f16(c, plane0, nplanes, pass) : RIDC_OK;
}

// ---------------------------------------------------------------------------------------------
// FP16 form: v 2^k -> FP16 hi + lo for every staged value of a plane, k from the plane's
// maximum (max|v| 2^k in [2^(K0-1), 2^K0)); scaling by a power of two is exact.
// blockIdx.y = plane.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) split_f16_kernel(const float* __restrict__ st,
                                                        __half* __restrict__ hi,
                                                        __half* __restrict__ lo,
                                                        const unsigned* __restrict__ pmax,
                                                        int plane0, long per_plane, int k0) {
  const int p = plane0 + blockIdx.y;
  const float sc = pow2f(f16_plane_exp(pmax[p], k0));
  const long off = (long)p * per_plane;
  const float4* s4 = reinterpret_cast<const float4*>(st + off);
  uint2* h4 = reinterpret_cast<uint2*>(hi + off);
  uint2* l4 = reinterpret_cast<uint2*>(lo + off);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < per_plane / 4;
       i += (long)gridDim.x * blockDim.x) {
    const float4 v = s4[i];
    const float f[4] = {v.x * sc, v.y * sc, v.z * sc, v.w * sc};
    __half h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] = __float2half_rn(f[k]);
      l[k] = __float2half_rn(f[k] - __half2float(h[k]));
    }
    uint2 ph, pl;
    ph.x = (unsigned)__half_as_ushort(h[0]) | ((unsigned)__half_as_ushort(h[1]) << 16);
    ph.y = (unsigned)__half_as_ushort(h[2]) | ((unsigned)__half_as_ushort(h[3]) << 16);
    pl.x = (unsigned)__half_as_ushort(l[0]) | ((unsigned)__half_as_ushort(l[1]) << 16);
    pl.y = (unsigned)__half_as_ushort(l[2]) | ((unsigned)__half_as_ushort(l[3]) << 16);
    h4[i] = ph;
    l4[i] = pl;
  }
}

int launch_split_f16(Ctx* c, int plane0, int nplanes, int pass) {
  if (pass < 0 || pass >= kMaxPasses || !c->xs || !c->pmax) return RIDC_ERR_ARG;
  const long per_plane = (long)c->n * c->n;   // n is a multiple of 256: per_plane % 4 == 0
  long bx = (per_plane / 4 + 255) / 256;
  const long cap = 152L * 8 / nplanes + 1;
  if (bx > cap) bx = cap;
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_SPLIT, &e0);
  split_f16_kernel<<<dim3((unsigned)bx, nplanes), 256, 0, c->stream>>>(
      c->xs, reinterpret_cast<__half*>(c->xh), reinterpret_cast<__half*>(c->xl),
      c->pmax + (size_t)pass * kMaxPlanes, plane0, per_plane, c->k0);
  prof_end(c, RIDC_KERNEL_SPLIT, e0);
  return cuda_status(cudaGetLastError());
}

int reset_plane_max(Ctx* c) {
  return cuda_status(
      cudaMemsetAsync(c->pmax, 0, (size_t)kMaxPasses * kMaxPlanes * sizeof(unsigned), c->stream));
}

// out = d64 + d32 (either part may be absent)
__global__ void combine_kernel(const double* __restrict__ d64, const float* __restrict__ d32,
                               double* __restrict__ out, long count) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
       i += (long)gridDim.x * blockDim.x) {
    double v = d64 ? d64[i] : 0.0;
    if (d32) v = d64 ? v + f32_to_f64(d32[i]) : f32_to_f64(d32[i]);
    out[i] = v;
  }
}

int launch_combine(Ctx* c, const double* d64, const float* d32, double* out, long count) {
  long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  combine_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(d64, d32, out, count);
  c->launches++;
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

// 1/den table of each plane of a solve: the table [t][N][N] of inv_den, t = coef * S + species
struct PlaneTabs {
  int t[kMaxPlanes];
};

template <int EPI>
__global__ void __launch_bounds__(256) gemm_f64_kernel(const double* __restrict__ A,
                                                       const double* __restrict__ B,
                                                       double* __restrict__ out,
                                                       const double* __restrict__ inv_den, int n,
                                                       int rows, const PlaneTabs pt) {
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
      if (EPI == EPI_SCALE_DEN) v *= inv_den[((long)pt.t[plane] * n + m) * n + rl];
      out[((long)plane * n + m) * n + rl] = v;
    }
  }
}

// Parity-split form of the same transform for even n (H = n/2; spectral indices in split order
// c = g H + k', k = 2k' + g; Q[n-1-x][k] = (-1)^k Q[x][k]):
//   forward: out[.][g H + k'] = sum_{x'<H} (A[x'] +- A[n-1-x']) Q[x'][2k'+g], B = Q^T with its
//            rows in split order (A is butterflied as it is loaded);
//   inverse: out[.][x'] = E + O, out[.][n-1-x'] = E - O, E = sum_{k'} A[k'] Q[x'][2k'],
//            O = sum_{k'} A[H+k'] Q[x'][2k'+1], B = Q with its columns in split order.
// Half the DFMAs of the plain product. Tile: 64 rows x 32 half-columns, each thread 4 rows x
// (2 + 2) columns, one accumulator set per half.
template <bool FWD, int EPI>
__global__ void __launch_bounds__(256) gemm_f64_split_kernel(const double* __restrict__ A,
                                                             const double* __restrict__ B,
                                                             double* __restrict__ out,
                                                             const double* __restrict__ inv_den,
                                                             int n, int rows, const PlaneTabs pt) {
  constexpr int GH = GB / 2;
  __shared__ __align__(16) double As[2][GK][GB + 2];
  __shared__ __align__(16) double Bs[2][GK][GH + 2];
  const int t = threadIdx.x;
  const int tr = t & 15, tc = t >> 4;
  const int H = n / 2;
  const int row0 = blockIdx.x * GB, col0 = blockIdx.y * GH;
  double acc[2][4][2] = {};
  for (int k0 = 0; k0 < H; k0 += GK) {
    {
      // A: 64 rows x 16 k per half; thread t loads 4 consecutive k of one row (and mirrors)
      const int lr = t >> 2, lk = (t & 3) * 4, gr = row0 + lr;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + lk + q;
        double v0 = 0.0, v1 = 0.0;
        if (gr < rows && k < H) {
          const double* ar = A + (long)gr * n;
          if (FWD) {
            const double x = ar[k], m = ar[n - 1 - k];
            v0 = x + m;
            v1 = x - m;
          } else {
            v0 = ar[k];
            v1 = ar[H + k];
          }
        }
        As[0][lk + q][lr] = v0;
        As[1][lk + q][lr] = v1;
      }
      // B: 32 columns x 16 k per half; thread t loads 2 consecutive k of one column
      const int lc = t >> 3, lk2 = (t & 7) * 2, gc = col0 + lc;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = k0 + lk2 + q;
        double b0 = 0.0, b1 = 0.0;
        if (gc < H && k < H) {
          b0 = FWD ? B[(long)gc * n + k] : B[(long)gc * n + k];
          b1 = FWD ? B[(long)(H + gc) * n + k] : B[(long)gc * n + H + k];
        }
        Bs[0][lk2 + q][lc] = b0;
        Bs[1][lk2 + q][lc] = b1;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        double a[4], b[2];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[h][kk][tr * 4 + i];
#pragma unroll
        for (int j = 0; j < 2; ++j) b[j] = Bs[h][kk][tc * 2 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) acc[h][i][j] = fma(a[i], b[j], acc[h][i][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + tr * 4 + i;
    if (gr >= rows) continue;
    const int plane = gr / n, rl = gr - plane * n;
    double* op = out + (long)plane * n * n;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int cc = col0 + tc * 2 + j;
      if (cc >= H) continue;
      if (FWD) {
        double v0 = acc[0][i][j], v1 = acc[1][i][j];
        if (EPI == EPI_SCALE_DEN) {
          const double* id = inv_den + (long)pt.t[plane] * n * n;
          v0 *= id[(long)cc * n + rl];
          v1 *= id[(long)(H + cc) * n + rl];
        }
        op[(long)cc * n + rl] = v0;
        op[(long)(H + cc) * n + rl] = v1;
      } else {
        const double ev = acc[0][i][j], ov = acc[1][i][j];
        op[(long)cc * n + rl] = ev + ov;
        op[(long)(n - 1 - cc) * n + rl] = ev - ov;
      }
    }
  }
}

int launch_gemm_f64(Ctx* c, const double* A, const double* B, double* out, int nplanes, int epi,
                    bool forward) {
  const int n = c->n, rows = nplanes * n;
  if (nplanes < 1 || nplanes > kMaxPlanes) return RIDC_ERR_ARG;
  PlaneTabs pt{};
  for (int p = 0; p < nplanes; ++p) pt.t[p] = c->plane_coef[p] * c->S + p % c->S;
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_GEMM_F64, &e0);
  if (n % 2 == 0) {
    dim3 grid((rows + GB - 1) / GB, (n / 2 + GB / 2 - 1) / (GB / 2));
    if (forward && epi == EPI_SCALE_DEN)
      gemm_f64_split_kernel<true, EPI_SCALE_DEN><<<grid, 256, 0, c->stream>>>(A, B, out, c->inv_den, n,
                                                                           rows, pt);
    else if (forward)
      gemm_f64_split_kernel<true, EPI_STORE><<<grid, 256, 0, c->stream>>>(A, B, out, c->inv_den, n,
                                                                       rows, pt);
    else
      gemm_f64_split_kernel<false, EPI_STORE><<<grid, 256, 0, c->stream>>>(A, B, out, c->inv_den, n,
                                                                        rows, pt);
  } else {
    dim3 grid((rows + GB - 1) / GB, (n + GB - 1) / GB);
    if (epi == EPI_SCALE_DEN)
      gemm_f64_kernel<EPI_SCALE_DEN><<<grid, 256, 0, c->stream>>>(A, B, out, c->inv_den, n, rows, pt);
    else
      gemm_f64_kernel<EPI_STORE><<<grid, 256, 0, c->stream>>>(A, B, out, c->inv_den, n, rows, pt);
  }
  prof_end(c, RIDC_KERNEL_GEMM_F64, e0);
  return cuda_status(cudaGetLastError());
}

}  // namespace ridc
