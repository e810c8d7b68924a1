// Batched ensemble: many independent RIDC instances (2D Dirichlet advection-diffusion of
// uneven grid sizes, orders and coefficients) advanced by one persistent launch, replayed
// as a CUDA graph.
//
// A cluster of CL CTAs (CL = 1, 2 or 4, chosen by the autotuner) takes instances from a shared
// counter, largest work first (a longest-processing-time order fixed at creation), and
// integrates its instance through every pipeline step of the advance call before taking the
// next. Inside a cluster every phase is split across its CTAs (GEMM tiles, cells) and the
// phases are separated by cluster barriers (release/acquire, so global writes of one CTA are
// visible to the others); different clusters never wait on one another. Per pipeline step of
// an instance, for every advancing level (Section III, eq. (pred) / eq. (corr)):
//   1. right-hand side in delta form, FP64 (defect + Lagrange quadrature, Section III-C);
//   2. (I - dt nu L) delta = r by fast diagonalisation in FP32: four transforms with the sine
//      eigenvectors of the cell-centred Dirichlet Laplacian (tables per grid side), each a
//      parity-split pair of FP32 SIMT products of half size, in 64 x 32 or 128 x 64 tiles of
//      half-columns (the autotuner picks one per side);
//   3. optional refinement: FP64 residual r - (I - dt nu L) delta, FP32 solve, FP64 update;
//   4. eta = base + delta in FP64, then f^N = -a u_x - b u_y and f = f^N + nu L eta (FP64).
// FP64 work uses integer bit operations for conversions and sign flips (GB300's FP64 pipe is
// narrow) and never issues predicated-off FP64 instructions. Workspace is per cluster, sized
// for the largest instance.
#include <algorithm>
#include <cooperative_groups.h>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "ridc_internal.h"

namespace ridc {

namespace {

constexpr int EMaxP = 4;           // orders of the ensemble: 1..4
constexpr int ENS_THREADS = 256;

__device__ __forceinline__ float e_f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int ef = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7F800000u | ((ef == 1151 && m) ? 0x400000u : 0u));
  const unsigned long long mr = m + 0xFFFFFFFull + ((m >> 29) & 1ull);
  return __uint_as_float(sign | (unsigned)(((unsigned long long)ef << 23) + (mr >> 29)));
}

__device__ __forceinline__ double e_f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFF;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ed = (e == 255) ? 2047ull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double(
      (long long)(sign | (ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// value of field x at (gy, gx) with the odd (Dirichlet) reflection for one ghost layer
__device__ __forceinline__ double odd_at(const double* __restrict__ x, int s, int gy, int gx) {
  bool neg = false;
  if (gy < 0) { gy = 0; neg = !neg; }
  if (gy >= s) { gy = s - 1; neg = !neg; }
  if (gx < 0) { gx = 0; neg = !neg; }
  if (gx >= s) { gx = s - 1; neg = !neg; }
  const double v = x[gy * s + gx];
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}

}  // namespace

struct EnsInst {
  double* eta[EMaxP];
  double* fN[EMaxP];
  double* F[EMaxP];
  int cap[EMaxP];
  int s, P, cls;
  double dt, a2h, b2h, c_lap, c_lap4, cres, cres1;
  float dtnu;
  long p[EMaxP];
};

struct EnsClass {
  const float* Qts;  // [s][s]  Qts[c][x] = Q[x][k]: rows of Q^T in split order c = g s/2 + k'
  const float* Qs;   // [s][s]  Qs[x][c] = Q[x][k]: Q with its columns in split order
  const float* lam;  // [s]     eigenvalues in split order
  int s;
  int variant;       // GEMM tile: 0 = 64 rows x 32 half-columns (4 x 2+2 per thread),
                     //            1 = 128 rows x 64 half-columns (8 x 4+4 per thread)
};

struct EnsArgs {
  EnsInst* inst;
  int ntotal;         // instances in the batch (bound of the ids in `order`)
  int ninst;          // length of `order`
  const int* order;
  int* next;
  const EnsClass* cls;
  const unsigned* masks[EMaxP + 1];
  int nmask[EMaxP + 1];
  const double* wq;   // [kMaxOrder][kMaxOrder][kMaxOrder]
  double* r_ws;       // per cluster: [EMaxP][s_max^2] FP64
  double* d_ws;       // per cluster: [EMaxP][s_max^2] FP64 (refinement total)
  float* f_ws;        // per cluster: 3 x [EMaxP][s_max^2] FP32 (operand, two intermediates)
  long ws_plane;
  int nref;
};

// ---- cluster-level FP32 GEMMs of the fast diagonalisation, parity-split ----------------------
// The sine eigenvectors obey Q[s-1-x][k] = (-1)^k Q[x][k]. With H = s/2 and spectral indices
// in split order (even k, then odd k: c = g H + k', k = 2k' + g) every transform is two
// (rows x H) x (H x H) products instead of one (rows x s) x (s x s): half the flops.
//   forward (FWD): out[.][g H + k'] = sum_{x'<H} (A[x'] +- A[s-1-x']) Q[x'][2k'+g]; A is
//                  butterflied as it is loaded, B rows are rows of Qts (Q^T in split order);
//   inverse:       out[.][x'] = E + O, out[.][s-1-x'] = E - O with E = sum_{k'} A[k'] Q[x'][2k'],
//                  O = sum_{k'} A[H+k'] Q[x'][2k'+1]; B rows are rows of Qs (Q, columns in
//                  split order).
// Every thread accumulates both halves (TM rows x TN/2 columns each), so a block tile covers
// 16 TM rows x 8 TN half-columns. Results are stored transposed per plane, out[plane][m][row %
// s], optionally times 1/(1 - dtnu (lam[row % s] + lam[m])) (forward, split order). Tiles are
// dealt round-robin to the CL CTAs of the cluster. 16-deep K slices: the next slice is fetched
// into registers (float4) while the current one is multiplied out of shared memory.
template <int TM, int TN>
struct DualSmem {
  float A[2][2][16][16 * TM + 4];   // [half][buffer][k][row]
  float B[2][2][16][8 * TN + 4];    // [half][buffer][k][column]
};
constexpr size_t ENS_SMEM_BYTES =
    sizeof(DualSmem<8, 8>) > sizeof(DualSmem<4, 4>) ? sizeof(DualSmem<8, 8>) : sizeof(DualSmem<4, 4>);

__device__ __forceinline__ float4 f4_add(float4 a, float4 b, float sg) {
  return make_float4(a.x + sg * b.x, a.y + sg * b.y, a.z + sg * b.z, a.w + sg * b.w);
}

template <int TM, int TN, bool FWD>
__device__ void dual_sgemm(const float* __restrict__ A, const float* __restrict__ B,
                           float* __restrict__ out, int s, int rows, const float* lam,
                           float dtnu, bool scale, DualSmem<TM, TN>& sm, int rank, int CL) {
  constexpr int BM = 16 * TM, BH = 8 * TN, TH = TN / 2;
  constexpr int AV = BM * 4 / ENS_THREADS;            // float4 of A per thread and half
  constexpr int BV = (BH * 4 + ENS_THREADS - 1) / ENS_THREADS;
  const int t = threadIdx.x;
  const int tr = t & 15, tc = t >> 4;
  const int H = s / 2;
  const int nrt = (rows + BM - 1) / BM, nct = (H + BH - 1) / BH;
  const int KT = H / 16;
  for (int tile = rank; tile < nrt * nct; tile += CL) {
    const int row0 = (tile / nct) * BM, col0 = (tile % nct) * BH;
    float acc[2][TM][TH];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TH; ++j) acc[h][i][j] = 0.f;
    float4 ra[2][AV], rb[2][BV];
    auto fetch = [&](int kt) {
#pragma unroll
      for (int v = 0; v < AV; ++v) {
        const int e = t + v * ENS_THREADS, lr = e >> 2, q = e & 3, gr = row0 + lr;
        const int k0 = kt * 16 + q * 4;
        if (gr < rows) {
          const float* ar = A + (long)gr * s;
          if (FWD) {
            // x' = k0..k0+3 and their mirrors s-1-x' (a reversed float4)
            const float4 x = *reinterpret_cast<const float4*>(ar + k0);
            const float4 m4 = *reinterpret_cast<const float4*>(ar + s - 4 - k0);
            const float4 m = make_float4(m4.w, m4.z, m4.y, m4.x);
            ra[0][v] = f4_add(x, m, 1.f);
            ra[1][v] = f4_add(x, m, -1.f);
          } else {
            ra[0][v] = *reinterpret_cast<const float4*>(ar + k0);
            ra[1][v] = *reinterpret_cast<const float4*>(ar + H + k0);
          }
        } else {
          ra[0][v] = ra[1][v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int v = 0; v < BV; ++v) {
        const int e = t + v * ENS_THREADS, lr = e >> 2, q = e & 3, gc = col0 + lr;
        const int k0 = kt * 16 + q * 4;
        if (e < BH * 4 && gc < H) {
          // forward: rows k' and H + k' of Qts; inverse: row x' of Qs, columns k' and H + k'
          const float* b0 = FWD ? B + (long)gc * s + k0 : B + (long)gc * s + k0;
          const float* b1 = FWD ? B + (long)(H + gc) * s + k0 : B + (long)gc * s + H + k0;
          rb[0][v] = *reinterpret_cast<const float4*>(b0);
          rb[1][v] = *reinterpret_cast<const float4*>(b1);
        } else {
          rb[0][v] = rb[1][v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int v = 0; v < AV; ++v) {
          const int e = t + v * ENS_THREADS, lr = e >> 2, q = e & 3;
          sm.A[h][buf][q * 4 + 0][lr] = ra[h][v].x;
          sm.A[h][buf][q * 4 + 1][lr] = ra[h][v].y;
          sm.A[h][buf][q * 4 + 2][lr] = ra[h][v].z;
          sm.A[h][buf][q * 4 + 3][lr] = ra[h][v].w;
        }
#pragma unroll
        for (int v = 0; v < BV; ++v) {
          const int e = t + v * ENS_THREADS, lr = e >> 2, q = e & 3;
          if (e < BH * 4) {
            sm.B[h][buf][q * 4 + 0][lr] = rb[h][v].x;
            sm.B[h][buf][q * 4 + 1][lr] = rb[h][v].y;
            sm.B[h][buf][q * 4 + 2][lr] = rb[h][v].z;
            sm.B[h][buf][q * 4 + 3][lr] = rb[h][v].w;
          }
        }
      }
    };
    __syncthreads();
    fetch(0);
    stash(0);
    __syncthreads();
    for (int kt = 0; kt < KT; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < KT) fetch(kt + 1);
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float av[TM], bv[TH];
#pragma unroll
          for (int i = 0; i < TM; ++i) av[i] = sm.A[h][buf][kk][tr * TM + i];
#pragma unroll
          for (int j = 0; j < TH; ++j) bv[j] = sm.B[h][buf][kk][tc * TH + j];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TH; ++j) acc[h][i][j] = fmaf(av[i], bv[j], acc[h][i][j]);
        }
      }
      if (kt + 1 < KT) stash(buf ^ 1);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gr = row0 + tr * TM + i;
      if (gr >= rows) continue;
      const int plane = gr / s, rl = gr - plane * s;
      float* op = out + (long)plane * s * s;
#pragma unroll
      for (int j = 0; j < TH; ++j) {
        const int c = col0 + tc * TH + j;   // k' (forward) or x' (inverse), < H
        if (c >= H) continue;
        if (FWD) {
          float v0 = acc[0][i][j], v1 = acc[1][i][j];
          if (scale) {
            v0 = __fdividef(v0, 1.0f - dtnu * (lam[rl] + lam[c]));
            v1 = __fdividef(v1, 1.0f - dtnu * (lam[rl] + lam[H + c]));
          }
          op[(long)c * s + rl] = v0;
          op[(long)(H + c) * s + rl] = v1;
        } else {
          const float ev = acc[0][i][j], ov = acc[1][i][j];
          op[(long)c * s + rl] = ev + ov;
          op[(long)(s - 1 - c) * s + rl] = ev - ov;
        }
      }
    }
  }
}

// The FP64 phases below are latency-bound (16 warps per SM): each thread takes two elements
// per iteration, i and i + gs, and issues all their loads before any arithmetic or store, so
// twice as many loads are in flight. Every element's arithmetic is unchanged. When i + gs is
// past the end the second element repeats the first and is not stored.

// right-hand side with NJ quadrature terms (eq. (corr) in delta form) and its FP32 copy
template <int NJ>
__device__ __forceinline__ void ens_rhs(const double* ej, const double* fj, const double* ep,
                                        const double* fp, const double* const (&Fb)[EMaxP],
                                        const double (&wd)[EMaxP], double dt, double* rq,
                                        float* fq, long ss, long g0, long gs) {
  for (long i = g0; i < ss; i += 2 * gs) {
    const bool two = i + gs < ss;
    const long i1 = two ? i + gs : i;
    const double e0 = ej[i], e1 = ej[i1], p0 = ep[i], p1 = ep[i1];
    const double f0 = fj[i], f1 = fj[i1], q0 = fp[i], q1 = fp[i1];
    double F0[NJ], F1[NJ];
#pragma unroll
    for (int k = 0; k < NJ; ++k) {
      F0[k] = Fb[k][i];
      F1[k] = Fb[k][i1];
    }
    double a0 = fma(dt, f0 - q0, e0 - p0), a1 = fma(dt, f1 - q1, e1 - p1);
#pragma unroll
    for (int k = 0; k < NJ; ++k) {
      a0 = fma(wd[k], F0[k], a0);
      a1 = fma(wd[k], F1[k], a1);
    }
    rq[i] = a0;
    fq[i] = e_f64_to_f32(a0);
    if (two) {
      rq[i1] = a1;
      fq[i1] = e_f64_to_f32(a1);
    }
  }
}

template <int CL>
__device__ __forceinline__ void csync() {
  if (CL > 1) cooperative_groups::this_cluster().sync();
  else __syncthreads();
}

// FP32 fast-diagonalisation solve of np planes: df = Q ((Q^T rf Q) ./ den) Q^T, each transform
// as a parity-split pair of half-size products (spectral indices in split order throughout)
template <int CL, int TM, int TN>
__device__ void cl_solve(const EnsClass& C, const EnsInst& I, int np, const float* rf, float* t1,
                         float* t2, float* df, DualSmem<TM, TN>& sm, int rank) {
  const int s = C.s, rows = np * s;
  dual_sgemm<TM, TN, true>(rf, C.Qts, t1, s, rows, C.lam, I.dtnu, false, sm, rank, CL);
  csync<CL>();
  dual_sgemm<TM, TN, true>(t1, C.Qts, t2, s, rows, C.lam, I.dtnu, true, sm, rank, CL);
  csync<CL>();
  dual_sgemm<TM, TN, false>(t2, C.Qs, t1, s, rows, C.lam, I.dtnu, false, sm, rank, CL);
  csync<CL>();
  dual_sgemm<TM, TN, false>(t1, C.Qs, df, s, rows, C.lam, I.dtnu, false, sm, rank, CL);
  csync<CL>();
}

template <int CL>
__device__ __forceinline__ void solve_any(const EnsClass& C, const EnsInst& I, int np,
                                          const float* rf, float* t1, float* t2, float* df,
                                          unsigned char* smem, int rank) {
  if (C.variant == 1)
    cl_solve<CL, 8, 8>(C, I, np, rf, t1, t2, df, *reinterpret_cast<DualSmem<8, 8>*>(smem), rank);
  else
    cl_solve<CL, 4, 4>(C, I, np, rf, t1, t2, df, *reinterpret_cast<DualSmem<4, 4>*>(smem), rank);
}

template <int CL>
__global__ void __launch_bounds__(ENS_THREADS, 2) ensemble_kernel(const __grid_constant__ EnsArgs a) {
  extern __shared__ __align__(16) unsigned char ens_smem[];   // ENS_SMEM_BYTES: GEMM tiles
  __shared__ int item;
  const int rank = (CL > 1) ? (int)cooperative_groups::this_cluster().block_rank() : 0;
  const long cid = blockIdx.x / CL;
  const long wp = a.ws_plane;
  double* r = a.r_ws + cid * EMaxP * wp;
  double* dt_tot = a.d_ws + cid * EMaxP * wp;
  float* rf = a.f_ws + cid * 3 * EMaxP * wp;
  float* t1 = rf + EMaxP * wp;
  float* t2 = t1 + EMaxP * wp;
  const long g0 = (long)rank * ENS_THREADS + threadIdx.x, gs = (long)CL * ENS_THREADS;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) item = atomicAdd(a.next, 1);
    csync<CL>();
    int w;
    if (CL > 1) w = *cooperative_groups::this_cluster().map_shared_rank(&item, 0);
    else w = item;
    // every CTA must have read rank 0's `item` before any CTA of the cluster may exit (its
    // shared memory goes away) or take the next instance
    csync<CL>();
    if (w >= a.ninst) break;
    const int id = a.order[w];
    if (id < 0 || id >= a.ntotal) continue;   // cannot happen: host-built list; never index past it
    EnsInst& Ig = a.inst[id];
    const EnsInst I = Ig;
    const EnsClass C = a.cls[I.cls];
    const int s = I.s, P = I.P;
    const long ss = (long)s * s;
    long p[EMaxP];
#pragma unroll
    for (int j = 0; j < EMaxP; ++j) p[j] = I.p[j];
    const unsigned* masks = a.masks[P];
    const int nm = a.nmask[P];
    for (int st = 0; st < nm; ++st) {
      const unsigned mask = masks[st];
      int lev[EMaxP], na = 0;
#pragma unroll
      for (int j = 0; j < EMaxP; ++j)
        if (j < P && (mask & (1u << j))) lev[na++] = j;
      // 1. right-hand sides (FP64) and their FP32 copies
      for (int q = 0; q < na; ++q) {
        const int j = lev[q];
        const long n = p[j];
        double* rq = r + q * ss;
        float* fq = rf + q * ss;
        if (j == 0) {
          const double* F0 = I.F[0] + (n % I.cap[0]) * ss;
          for (long i = g0; i < ss; i += gs) {
            const double v = I.dt * F0[i];
            rq[i] = v;
            fq[i] = e_f64_to_f32(v);
          }
        } else {
          const double* ej = I.eta[j] + (n % I.cap[j]) * ss;
          const double* fj = I.fN[j] + (n % I.cap[j]) * ss;
          const double* ep = I.eta[j - 1] + ((n + 1) % I.cap[j - 1]) * ss;
          const double* fp = I.fN[j - 1] + (n % I.cap[j - 1]) * ss;
          const long b = (n + 1 - j > 0) ? n + 1 - j : 0;
          const int m = (int)(n - b);
          const double* w = a.wq + ((long)j * kMaxOrder + m) * kMaxOrder;
          const double* Fb[EMaxP];
          double wd[EMaxP];
#pragma unroll
          for (int k = 0; k < EMaxP; ++k) {
            Fb[k] = (k <= j) ? I.F[j - 1] + ((b + k) % I.cap[j - 1]) * ss : nullptr;
            wd[k] = (k <= j) ? I.dt * w[k] : 0.0;
          }
          // exactly j+1 quadrature terms: no predicated-off FP64 work (it still costs pipe time)
          if (j == 1) ens_rhs<2>(ej, fj, ep, fp, Fb, wd, I.dt, rq, fq, ss, g0, gs);
          else if (j == 2) ens_rhs<3>(ej, fj, ep, fp, Fb, wd, I.dt, rq, fq, ss, g0, gs);
          else ens_rhs<4>(ej, fj, ep, fp, Fb, wd, I.dt, rq, fq, ss, g0, gs);
        }
      }
      csync<CL>();
      // 2./3. FP32 solve (the increment overwrites rf, free after the first GEMM), then
      // refinement passes against the FP64 residual
      const float* df = rf;
      solve_any<CL>(C, I, na, rf, t1, t2, rf, ens_smem, rank);
      for (int pass = 1; pass <= a.nref; ++pass) {
        for (long e = g0; e < na * ss; e += gs)
          dt_tot[e] = (pass == 1) ? e_f32_to_f64(df[e]) : dt_tot[e] + e_f32_to_f64(df[e]);
        csync<CL>();
        const long tot = na * ss;
        for (long e = g0; e < tot; e += 2 * gs) {
          const bool two = e + gs < tot;
          const long e1 = two ? e + gs : e;
          double nb[2][4], dc[2], rr[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const long ee = u ? e1 : e;
            const long q = ee / ss, i = ee - q * ss;
            const int gy = (int)(i / s), gx = (int)(i - (long)gy * s);
            const double* d = dt_tot + q * ss;
            nb[u][0] = odd_at(d, s, gy - 1, gx);
            nb[u][1] = odd_at(d, s, gy + 1, gx);
            nb[u][2] = odd_at(d, s, gy, gx - 1);
            nb[u][3] = odd_at(d, s, gy, gx + 1);
            dc[u] = d[i];
            rr[u] = r[ee];
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const double sum = (nb[u][0] + nb[u][1]) + (nb[u][2] + nb[u][3]);
            const double v = fma(I.cres, sum, fma(I.cres1, dc[u], rr[u]));
            if (u == 0 || two) rf[u ? e1 : e] = e_f64_to_f32(v);   // df is folded into dt_tot
          }
        }
        csync<CL>();
        solve_any<CL>(C, I, na, rf, t1, t2, rf, ens_smem, rank);
      }
      // 4a. new states eta = base + delta (FP64)
      for (int q = 0; q < na; ++q) {
        const int j = lev[q];
        const long n = p[j];
        const double* base = (j == 0) ? I.eta[0] + (n % I.cap[0]) * ss
                                      : I.eta[j - 1] + ((n + 1) % I.cap[j - 1]) * ss;
        double* out = I.eta[j] + ((n + 1) % I.cap[j]) * ss;
        const float* dq = df + q * ss;
        const double* tq = dt_tot + q * ss;
        for (long i = g0; i < ss; i += 2 * gs) {
          const bool two = i + gs < ss;
          const long i1 = two ? i + gs : i;
          const double b0 = base[i], b1 = base[i1];
          const float d0 = dq[i], d1 = dq[i1];
          double o0, o1;
          if (a.nref > 0) {
            const double t0 = tq[i], t1 = tq[i1];
            o0 = b0 + (e_f32_to_f64(d0) + t0);
            o1 = b1 + (e_f32_to_f64(d1) + t1);
          } else {
            o0 = b0 + e_f32_to_f64(d0);
            o1 = b1 + e_f32_to_f64(d1);
          }
          out[i] = o0;
          if (two) out[i1] = o1;
        }
      }
      csync<CL>();
      // 4b. f^N and f of the new states
      for (int q = 0; q < na; ++q) {
        const int j = lev[q];
        const long slot = ((p[j] + 1) % I.cap[j]) * ss;
        const double* e = I.eta[j] + slot;
        double* fN = I.fN[j] + slot;
        double* F = I.F[j] ? I.F[j] + slot : nullptr;
        for (long i = g0; i < ss; i += 2 * gs) {
          const bool two = i + gs < ss;
          const long i1 = two ? i + gs : i;
          double xe[2], xw[2], yn[2], ys[2], ec[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const long ii = u ? i1 : i;
            const int gy = (int)(ii / s), gx = (int)(ii - (long)gy * s);
            xe[u] = odd_at(e, s, gy, gx + 1);
            xw[u] = odd_at(e, s, gy, gx - 1);
            yn[u] = odd_at(e, s, gy + 1, gx);
            ys[u] = odd_at(e, s, gy - 1, gx);
            ec[u] = e[ii];
          }
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (u == 1 && !two) break;
            const long ii = u ? i1 : i;
            const double fn = -I.a2h * (xe[u] - xw[u]) - I.b2h * (yn[u] - ys[u]);
            fN[ii] = fn;
            if (F) F[ii] = fma(I.c_lap, (xe[u] + xw[u]) + (yn[u] + ys[u]), fma(I.c_lap4, ec[u], fn));
          }
        }
      }
      csync<CL>();
      for (int q = 0; q < na; ++q) p[lev[q]]++;
    }
    if (rank == 0 && threadIdx.x == 0)
      for (int j = 0; j < EMaxP; ++j) Ig.p[j] = p[j];
  }
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
struct BatchCtx {
  int n = 0;
  int device = 0;                      // the device the batch lives on
  cudaStream_t stream = nullptr;
  // every advance is one CUDA graph (counter reset + the persistent cluster launch), captured
  // on a private stream (the caller's may be the legacy default stream, which cannot be
  // captured), updated in place while its shape holds and launched on the caller's stream
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long graph_launches = 0;
  int nref = 0;
  std::vector<EnsInst> inst;           // host mirror (progress kept in sync on the host)
  std::vector<EnsClass> cls;
  std::vector<void*> allocs;
  EnsInst* inst_dev = nullptr;
  EnsClass* cls_dev = nullptr;
  int* order_dev = nullptr;
  int* sub_dev = nullptr;              // scratch instance list of the autotuner
  int* next_dev = nullptr;
  double* wq_dev = nullptr;
  unsigned* masks_dev[EMaxP + 1] = {nullptr};
  size_t masks_cap[EMaxP + 1] = {0};
  double *r_ws = nullptr, *d_ws = nullptr;
  float* f_ws = nullptr;
  long ws_plane = 0;
  int cl = 1;                          // autotuned cluster size (CTAs per instance)
  int per_sm = 1;                      // autotuned CTAs per SM
  int sms = 0;
  bool initialised = false;
  long cells_per_step = 0;
};

static int b_alloc(BatchCtx* b, void** p, size_t bytes) {
  cudaError_t e = dev_malloc(p, bytes);
  if (e != cudaSuccess) return cuda_status(e);
  b->allocs.push_back(*p);
  return RIDC_OK;
}

static void b_free(BatchCtx* b) {
  for (void* p : b->allocs) dev_free(p, b->stream);
  b->allocs.clear();
}

template <int CL>
static int launch_cl(cudaStream_t stream, const EnsArgs& a, int grid) {
  static std::atomic<unsigned long long> attr_done{0};
  RIDC_TRY(raise_smem_limit_once(ensemble_kernel<CL>, (int)ENS_SMEM_BYTES, &attr_done));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(ENS_THREADS);
  cfg.dynamicSmemBytes = ENS_SMEM_BYTES;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cuda_status(cudaLaunchKernelEx(&cfg, ensemble_kernel<CL>, a));
}

// grid for cluster size cl and `per_sm` CTAs per SM (workspace holds 2 * sms clusters)
static int grid_for(const BatchCtx* b, int cl, int per_sm, int count) {
  const int clusters = std::max(1, std::min(count, per_sm * b->sms / cl));
  return clusters * cl;
}

// Advance the instances listed in `order` (count of them) by nsteps top-level steps.
static int batch_run(BatchCtx* b, long nsteps, int cl, int per_sm, const int* order, int count) {
  EnsArgs a{};
  a.inst = b->inst_dev;
  a.ntotal = b->n;
  a.ninst = count;
  a.order = order;
  a.next = b->next_dev;
  a.cls = b->cls_dev;
  a.wq = b->wq_dev;
  a.r_ws = b->r_ws;
  a.d_ws = b->d_ws;
  a.f_ws = b->f_ws;
  a.ws_plane = b->ws_plane;
  a.nref = b->nref;
  long newp[EMaxP + 1][EMaxP] = {{0}};
  bool have[EMaxP + 1] = {false};
  for (const EnsInst& I : b->inst) {
    if (have[I.P]) continue;
    have[I.P] = true;
    long p[kMaxOrder] = {0};
    for (int j = 0; j < I.P; ++j) p[j] = I.p[j];
    const long target = p[I.P - 1] + nsteps;
    std::vector<unsigned> masks;
    for (;;) {
      const unsigned m = plan_step(I.P, p, target, 1);
      if (!m) break;
      masks.push_back(m);
      for (int j = 0; j < I.P; ++j)
        if (m & (1u << j)) p[j]++;
    }
    if (masks.size() > b->masks_cap[I.P]) {
      dev_free(b->masks_dev[I.P], b->stream);   // an earlier replay may still read it
      b->masks_dev[I.P] = nullptr;
      b->masks_cap[I.P] = 0;
      cudaError_t e = dev_malloc((void**)&b->masks_dev[I.P], (masks.size() + 1) * sizeof(unsigned));
      if (e != cudaSuccess) return cuda_status(e);
      b->masks_cap[I.P] = masks.size();
    }
    if (!masks.empty()) {
      cudaError_t e = cudaMemcpyAsync(b->masks_dev[I.P], masks.data(), masks.size() * sizeof(unsigned),
                                      cudaMemcpyHostToDevice, b->stream);
      if (e != cudaSuccess) return cuda_status(e);
    }
    a.masks[I.P] = b->masks_dev[I.P];
    a.nmask[I.P] = (int)masks.size();
    for (int j = 0; j < I.P; ++j) newp[I.P][j] = p[j];
  }
  const int grid = grid_for(b, cl, per_sm, count);
  // capture: work-counter reset + the persistent launch
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  int rc = cuda_status(cudaMemsetAsync(b->next_dev, 0, sizeof(int), b->cap_stream));
  if (rc == RIDC_OK) {
    if (cl == 4) rc = launch_cl<4>(b->cap_stream, a, grid);
    else if (cl == 2) rc = launch_cl<2>(b->cap_stream, a, grid);
    else rc = launch_cl<1>(b->cap_stream, a, grid);
  }
  e = cudaStreamEndCapture(b->cap_stream, &graph);
  if (rc != RIDC_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return rc != RIDC_OK ? rc : cuda_status(e);
  }
  if (b->gexec) {   // same shape (same kernel instance): update the parameters in place
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(b->gexec, graph, &info) != cudaSuccess) {
      cudaGetLastError();   // the update is refused when the shape changed: rebuild
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
  }
  if (!b->gexec) {
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    if (e != cudaSuccess) {
      b->gexec = nullptr;
      cudaGraphDestroy(graph);
      return cuda_status(e);
    }
  }
  cudaGraphDestroy(graph);
  rc = cuda_status(cudaGraphLaunch(b->gexec, b->stream));
  if (rc != RIDC_OK) return rc;
  b->graph_launches++;
  for (EnsInst& I : b->inst)
    for (int j = 0; j < I.P; ++j) I.p[j] = newp[I.P][j];
  return RIDC_OK;
}

}  // namespace ridc

using namespace ridc;

extern "C" int ridc_batch_create(int count, const ridc_problem* problems, const ridc_grid* grids,
                                 const double* nu, const double* dt, const int* order, void* stream,
                                 ridc_batch* out) {
  if (count < 1 || !problems || !grids || !nu || !dt || !order || !out) return RIDC_ERR_ARG;
  int nref = -1;
  for (int i = 0; i < count; ++i) {
    const ridc_problem& pr = problems[i];
    if (pr.kind != RIDC_ADV_DIFF_2D_DIRICHLET) return RIDC_ERR_UNSUPPORTED;
    if (pr.precision != RIDC_FP32_SOLVE) return RIDC_ERR_UNSUPPORTED;
    if (pr.restart_every != 0) return RIDC_ERR_UNSUPPORTED;
    if (pr.predictor != RIDC_PRED_FBE) return RIDC_ERR_UNSUPPORTED;
    if (pr.n_refine < 0 || pr.n_refine > 4) return RIDC_ERR_ARG;
    if (nref >= 0 && pr.n_refine != nref) return RIDC_ERR_ARG;   // one setting per batch
    nref = pr.n_refine;
    if (grids[i].dim != 2 || grids[i].n < 32 || grids[i].n > 512) return RIDC_ERR_ARG;
    if (grids[i].n % 32 != 0) return RIDC_ERR_UNSUPPORTED;   // 16-deep K slices of n/2
    if (order[i] < 1 || order[i] > EMaxP) return RIDC_ERR_UNSUPPORTED;
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i]) || !(nu[i] > 0.0) || !std::isfinite(nu[i]))
      return RIDC_ERR_ARG;
  }
  BatchCtx* b = new (std::nothrow) BatchCtx();
  if (!b) return RIDC_ERR_OOM;
  b->n = count;
  b->stream = (cudaStream_t)stream;
  b->nref = nref;
  int rc = RIDC_OK;
  auto fail = [&](int code) {
    b_free(b);
    for (int p = 0; p <= EMaxP; ++p) dev_free(b->masks_dev[p], b->stream);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return code;
  };
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(RIDC_ERR_CUDA);
  int dev = 0;
  cudaGetDevice(&dev);
  b->device = dev;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (b->sms <= 0) b->sms = 1;
  // side classes and their FP32 eigenvector tables
  std::vector<int> sides;
  for (int i = 0; i < count; ++i) sides.push_back(grids[i].n);
  std::sort(sides.begin(), sides.end());
  sides.erase(std::unique(sides.begin(), sides.end()), sides.end());
  const double pi = 3.14159265358979323846;
  int smax = 0;
  for (int s : sides) {
    smax = std::max(smax, s);
    // orthonormal sine eigenvectors Q[x][k] (k = 0..s-1 for the modes K = k + 1), stored with
    // the spectral index in split order c = (k % 2) s/2 + k/2
    std::vector<float> Qs((size_t)s * s), Qts((size_t)s * s), lam(s);
    const int H = s / 2;
    for (int k = 0; k < s; ++k) {
      const long K = k + 1;
      const int c = (k % 2) * H + k / 2;
      const double cn = (K == s) ? std::sqrt(1.0 / s) : std::sqrt(2.0 / s);
      const double sk = std::sin(pi * (double)K / (2.0 * s));
      lam[c] = (float)(-4.0 * (double)s * s * sk * sk);
      for (int x = 0; x < s; ++x) {
        const long t = (K * (2L * x + 1)) % (4L * s);
        const double q = cn * std::sin(pi * (double)t / (2.0 * s));
        Qs[(size_t)x * s + c] = (float)q;
        Qts[(size_t)c * s + x] = (float)q;
      }
    }
    EnsClass C{};
    C.s = s;
    C.variant = s >= 128 ? 1 : 0;   // until the autotuner decides
    void* p;
    if ((rc = b_alloc(b, &p, Qs.size() * 4)) != RIDC_OK) return fail(rc);
    cudaMemcpy(p, Qs.data(), Qs.size() * 4, cudaMemcpyHostToDevice);
    C.Qs = (const float*)p;
    if ((rc = b_alloc(b, &p, Qts.size() * 4)) != RIDC_OK) return fail(rc);
    cudaMemcpy(p, Qts.data(), Qts.size() * 4, cudaMemcpyHostToDevice);
    C.Qts = (const float*)p;
    if ((rc = b_alloc(b, &p, lam.size() * 4)) != RIDC_OK) return fail(rc);
    cudaMemcpy(p, lam.data(), lam.size() * 4, cudaMemcpyHostToDevice);
    C.lam = (const float*)p;
    b->cls.push_back(C);
  }
  // instances: rings and constants
  b->inst.resize(count);
  for (int i = 0; i < count; ++i) {
    EnsInst& I = b->inst[i];
    memset(&I, 0, sizeof(I));
    const int s = grids[i].n, P = order[i];
    const double h = 1.0 / s;
    I.s = s;
    I.P = P;
    I.cls = (int)(std::lower_bound(sides.begin(), sides.end(), s) - sides.begin());
    I.dt = dt[i];
    I.a2h = problems[i].a / (2.0 * h);
    I.b2h = problems[i].b / (2.0 * h);
    I.c_lap = nu[i] / (h * h);
    I.c_lap4 = -4.0 * I.c_lap;
    I.cres = dt[i] * nu[i] / (h * h);
    I.cres1 = -(1.0 + 4.0 * I.cres);
    I.dtnu = (float)(dt[i] * nu[i]);
    const size_t pb = (size_t)s * s * sizeof(double);
    for (int j = 0; j < P; ++j) {
      I.cap[j] = (j < P - 1) ? j + 3 : 2;
      void* p;
      if ((rc = b_alloc(b, &p, I.cap[j] * pb)) != RIDC_OK) return fail(rc);
      I.eta[j] = (double*)p;
      if ((rc = b_alloc(b, &p, I.cap[j] * pb)) != RIDC_OK) return fail(rc);
      I.fN[j] = (double*)p;
      if (j < P - 1 || j == 0) {
        if ((rc = b_alloc(b, &p, I.cap[j] * pb)) != RIDC_OK) return fail(rc);
        I.F[j] = (double*)p;
      }
    }
    b->cells_per_step += (long)s * s;
  }
  // work order: largest (order x side^3) first
  std::vector<int> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    const double wx = (double)order[x] * grids[x].n * grids[x].n * (double)grids[x].n;
    const double wy = (double)order[y] * grids[y].n * grids[y].n * (double)grids[y].n;
    return wx > wy;
  });
  void* p;
  if ((rc = b_alloc(b, &p, count * sizeof(int))) != RIDC_OK) return fail(rc);
  b->order_dev = (int*)p;
  cudaMemcpy(b->order_dev, ord.data(), count * sizeof(int), cudaMemcpyHostToDevice);
  if ((rc = b_alloc(b, &p, count * sizeof(int))) != RIDC_OK) return fail(rc);
  b->sub_dev = (int*)p;
  if ((rc = b_alloc(b, &p, sizeof(int))) != RIDC_OK) return fail(rc);
  b->next_dev = (int*)p;
  if ((rc = b_alloc(b, &p, b->cls.size() * sizeof(EnsClass))) != RIDC_OK) return fail(rc);
  b->cls_dev = (EnsClass*)p;
  cudaMemcpy(p, b->cls.data(), b->cls.size() * sizeof(EnsClass), cudaMemcpyHostToDevice);
  if ((rc = b_alloc(b, &p, count * sizeof(EnsInst))) != RIDC_OK) return fail(rc);
  b->inst_dev = (EnsInst*)p;
  std::vector<double> wq((size_t)kMaxOrder * kMaxOrder * kMaxOrder, 0.0);
  {
    std::vector<double> w4((size_t)EMaxP * EMaxP * EMaxP);
    if (ridc_quadrature_weights(EMaxP, w4.data(), w4.size()) != RIDC_OK) return fail(RIDC_ERR_ARG);
    for (int j = 0; j < EMaxP; ++j)
      for (int m = 0; m < EMaxP; ++m)
        for (int i = 0; i < EMaxP; ++i)
          wq[((size_t)j * kMaxOrder + m) * kMaxOrder + i] = w4[((size_t)j * EMaxP + m) * EMaxP + i];
  }
  if ((rc = b_alloc(b, &p, wq.size() * sizeof(double))) != RIDC_OK) return fail(rc);
  b->wq_dev = (double*)p;
  cudaMemcpy(p, wq.data(), wq.size() * sizeof(double), cudaMemcpyHostToDevice);
  // per-cluster workspace, enough for one-CTA clusters, two per SM
  b->ws_plane = (long)smax * smax;
  const long ctas = 2L * b->sms;
  if ((rc = b_alloc(b, &p, (size_t)ctas * EMaxP * b->ws_plane * sizeof(double))) != RIDC_OK) return fail(rc);
  b->r_ws = (double*)p;
  if ((rc = b_alloc(b, &p, (size_t)ctas * EMaxP * b->ws_plane * sizeof(double))) != RIDC_OK) return fail(rc);
  b->d_ws = (double*)p;
  if ((rc = b_alloc(b, &p, (size_t)ctas * 3 * EMaxP * b->ws_plane * sizeof(float))) != RIDC_OK) return fail(rc);
  b->f_ws = (float*)p;
  b->cl = 4;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_status(e));
  *out = reinterpret_cast<ridc_batch>(b);
  live_handles_add(1);
  return RIDC_OK;
}

static BatchCtx* bctx(ridc_batch h) { return reinterpret_cast<BatchCtx*>(h); }

extern "C" void ridc_batch_destroy(ridc_batch h) {
  BatchCtx* b = bctx(h);
  if (!b) return;
  DeviceGuard dg(b->device);
  cudaStreamSynchronize(b->stream);
  b_free(b);
  for (int p = 0; p <= EMaxP; ++p) dev_free(b->masks_dev[p], b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
  live_handles_add(-1);
}

extern "C" long ridc_batch_graph_launches(ridc_batch h) {
  BatchCtx* b = bctx(h);
  return b ? b->graph_launches : -1;
}

// f^N and F of instance i's level-0 slot 0 (initial state), by a 1-step-free launch of the
// same kernel machinery: a small dedicated kernel keeps it simple.
__global__ void ens_init_kernel(EnsInst* inst, int ninst) {
  const int i = blockIdx.y;
  if (i >= ninst) return;
  const EnsInst I = inst[i];
  const int s = I.s;
  const long ss = (long)s * s;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < ss; e += (long)gridDim.x * blockDim.x) {
    const int gy = (int)(e / s), gx = (int)(e - (long)gy * s);
    const double* u = I.eta[0];
    const double xe = odd_at(u, s, gy, gx + 1), xw = odd_at(u, s, gy, gx - 1);
    const double yn = odd_at(u, s, gy + 1, gx), ys = odd_at(u, s, gy - 1, gx);
    const double fn = -I.a2h * (xe - xw) - I.b2h * (yn - ys);
    const double F = fma(I.c_lap, (xe + xw) + (yn + ys), fma(I.c_lap4, u[e], fn));
    for (int j = 0; j < I.P; ++j) {
      if (j > 0) I.eta[j][e] = u[e];
      I.fN[j][e] = fn;
      if (I.F[j]) I.F[j][e] = F;
    }
  }
}

extern "C" int ridc_batch_set_initial(ridc_batch h, const double* const* u0, int on_device) {
  BatchCtx* b = bctx(h);
  if (!b || !u0) return RIDC_ERR_ARG;
  DeviceGuard dg(b->device);
  for (int i = 0; i < b->n; ++i) {
    if (!u0[i]) return RIDC_ERR_ARG;
    EnsInst& I = b->inst[i];
    const size_t bytes = (size_t)I.s * I.s * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(I.eta[0], u0[i], bytes,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (int j = 0; j < EMaxP; ++j) I.p[j] = 0;
  }
  cudaError_t e = cudaMemcpyAsync(b->inst_dev, b->inst.data(), b->n * sizeof(EnsInst),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  ens_init_kernel<<<dim3(64, b->n), 256, 0, b->stream>>>(b->inst_dev, b->n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaStreamSynchronize(b->stream);   // host sources may be reused on return
  if (e != cudaSuccess) return cuda_status(e);
  b->initialised = true;
  return RIDC_OK;
}

extern "C" int ridc_batch_advance(ridc_batch h, long nsteps) {
  BatchCtx* b = bctx(h);
  if (!b || nsteps < 0 || !b->initialised) return RIDC_ERR_ARG;
  DeviceGuard dg(b->device);
  if (nsteps == 0) return RIDC_OK;
  return batch_run(b, nsteps, b->cl, b->per_sm, b->order_dev, b->n);
}

extern "C" int ridc_batch_get_solution(ridc_batch h, int i, double* out, size_t count,
                                       int out_on_device) {
  BatchCtx* b = bctx(h);
  if (!b || !out || i < 0 || i >= b->n || !b->initialised) return RIDC_ERR_ARG;
  DeviceGuard dg(b->device);
  const EnsInst& I = b->inst[i];
  if (count != (size_t)I.s * I.s) return RIDC_ERR_ARG;
  const int top = I.P - 1;
  const double* src = I.eta[top] + (I.p[top] % I.cap[top]) * (long)I.s * I.s;
  cudaError_t e = cudaMemcpyAsync(out, src, count * sizeof(double),
                                  out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (!out_on_device)
    for (size_t k = 0; k < count; ++k)
      if (!std::isfinite(out[k])) return RIDC_ERR_NONFINITE;
  return RIDC_OK;
}

extern "C" long ridc_batch_cells(ridc_batch h) {
  BatchCtx* b = bctx(h);
  return b ? b->cells_per_step : -1;
}

// Autotuner. First, per grid side, the GEMM tile (64 x 32 or 128 x 64) that integrates the
// instances of that side fastest on their own (one-CTA clusters); then the cluster size (1, 2
// or 4 CTAs per instance) and the CTAs per SM (1 or 2) that run the whole batch fastest with
// those tiles. Each trial advances `nsteps` top-level steps from the current state. The
// choice is kept for later advances; *choice = CTAs per SM * 16 + cluster size.
// The state is scrambled: call ridc_batch_set_initial afterwards.
extern "C" int ridc_batch_autotune(ridc_batch h, long nsteps, int* choice, float* best_ms) {
  BatchCtx* b = bctx(h);
  if (!b || nsteps < 1) return RIDC_ERR_ARG;
  DeviceGuard dg(b->device);
  if (!b->initialised) return RIDC_ERR_ARG;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const std::vector<EnsInst> saved = b->inst;
  auto restore = [&]() {
    b->inst = saved;
    return cudaMemcpyAsync(b->inst_dev, b->inst.data(), b->n * sizeof(EnsInst),
                           cudaMemcpyHostToDevice, b->stream);
  };
  auto timed = [&](int cl, int per_sm, const int* ord, int cnt, float* ms) -> int {
    restore();
    int rc = batch_run(b, nsteps, cl, per_sm, ord, cnt);   // warm-up
    if (rc != RIDC_OK) return rc;
    restore();
    cudaEventRecord(e0, b->stream);
    rc = batch_run(b, nsteps, cl, per_sm, ord, cnt);
    if (rc != RIDC_OK) return rc;
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    return RIDC_OK;
  };
  int rc = RIDC_OK;
  int mask = 0;
  for (size_t c = 0; c < b->cls.size() && rc == RIDC_OK; ++c) {
    std::vector<int> sub;
    for (int i = 0; i < b->n; ++i)
      if (b->inst[i].cls == (int)c) sub.push_back(i);
    if (sub.empty()) continue;
    cudaMemcpyAsync(b->sub_dev, sub.data(), sub.size() * sizeof(int), cudaMemcpyHostToDevice,
                    b->stream);
    float best = 1e30f;
    int bv = b->cls[c].variant;
    for (int v = 0; v < 2 && rc == RIDC_OK; ++v) {
      b->cls[c].variant = v;
      cudaMemcpyAsync(b->cls_dev, b->cls.data(), b->cls.size() * sizeof(EnsClass),
                      cudaMemcpyHostToDevice, b->stream);
      float ms = 0.f;
      rc = timed(1, 1, b->sub_dev, (int)sub.size(), &ms);
      if (ms < best) { best = ms; bv = v; }
    }
    b->cls[c].variant = bv;
    if (bv) mask |= 1 << c;
  }
  cudaMemcpyAsync(b->cls_dev, b->cls.data(), b->cls.size() * sizeof(EnsClass),
                  cudaMemcpyHostToDevice, b->stream);
  float best = 1e30f;
  int bcl = b->cl, bps = b->per_sm;
  for (int per_sm = 1; per_sm <= 2 && rc == RIDC_OK; ++per_sm)
    for (int cl = 1; cl <= 4 && rc == RIDC_OK; cl *= 2) {
      float ms = 0.f;
      rc = timed(cl, per_sm, b->order_dev, b->n, &ms);
      if (ms < best) { best = ms; bcl = cl; bps = per_sm; }
    }
  restore();
  cudaStreamSynchronize(b->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RIDC_OK) return rc;
  b->cl = bcl;
  b->per_sm = bps;
  b->initialised = false;
  (void)mask;
  if (choice) *choice = bps * 16 + bcl;
  if (best_ms) *best_ms = best;
  return RIDC_OK;
}

extern "C" int ridc_batch_set_launch(ridc_batch h, int choice) {
  BatchCtx* b = bctx(h);
  if (!b) return RIDC_ERR_ARG;
  const int per_sm = choice / 16, cl = choice % 16;
  if ((per_sm != 1 && per_sm != 2) || (cl != 1 && cl != 2 && cl != 4)) return RIDC_ERR_ARG;
  b->per_sm = per_sm;
  b->cl = cl;
  return RIDC_OK;
}
