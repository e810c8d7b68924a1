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
//   2. (I - dt nu L) delta = r by fast diagonalisation at FP32 accuracy: four transforms with
//      the sine eigenvectors of the cell-centred Dirichlet Laplacian (tables per grid side),
//      each a parity-split pair of half-size products on the tensor cores (TF32 hi/lo split,
//      dual_umma below), in tiles of 128 rows by up to 64 half-columns;
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
#include "tc_util.cuh"

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
  int bn;            // tile width (half-columns) of this size's products, chosen by the
                     // autotuner: a multiple of 16 up to 64 that divides s/2
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
  int* err;           // set when a bounded device wait gives up
  float* f_ws;        // per cluster: 3 x [EMaxP][s_max^2] FP32 (operand, two intermediates)
  long ws_plane;
  int nref;
};

// ---- cluster-level GEMMs of the fast diagonalisation on the tensor cores, parity-split -------
// The sine eigenvectors obey Q[s-1-x][k] = (-1)^k Q[x][k]. With H = s/2 and spectral indices
// in split order (even k, then odd k: c = g H + k', k = 2k' + g) every transform is two
// (rows x H) x (H x H) products instead of one (rows x s) x (s x s): half the flops.
//   forward (FWD): out[.][g H + k'] = sum_{x'<H} (A[x'] +- A[s-1-x']) Q[x'][2k'+g]; A is
//                  butterflied as it is staged, B rows are rows of Qts (Q^T in split order);
//   inverse:       out[.][x'] = E + O, out[.][s-1-x'] = E - O with E = sum_{k'} A[k'] Q[x'][2k'],
//                  O = sum_{k'} A[H+k'] Q[x'][2k'+1]; B rows are rows of Qs (Q, columns in
//                  split order).
// Results are stored transposed per plane, out[plane][m][row % s], optionally times
// 1/(1 - dtnu (lam[row % s] + lam[m])) (forward, split order).
//
// Each product runs on the 5th-generation tensor cores as kind::tf32 with split operands:
// v = hi + lo, hi = v rounded to TF32 (10 fraction bits), lo = v - hi (exact in FP32) rounded
// to TF32 too, and C ~= Ah Bh + Ah Bl + Al Bh, about 22 significant bits per product with FP32
// accumulation in tensor memory: the accuracy of the FP32 solves it replaces. A tile is 128
// rows (M) by BN half-columns (N, a multiple of 16 up to 64 that divides H) per parity half,
// both halves accumulated side by side in 2 BN TMEM columns. K advances in slices of 32 values
// (128-byte rows, 128B swizzle), one parity half at a time through one set of buffers (48 KB,
// so four CTAs fit per SM): all 256 threads load the half-slice's A operand from global memory
// (float4) into registers, then wait (bounded) on the mbarrier of the previous MMAs, which
// still read the buffers, so that the loads and the MMAs overlap; then they butterfly, split
// and write A and B to shared memory, and one thread issues the 12 MMAs (3 products x 4 steps
// of K = 8) and commits them to the mbarrier. The epilogue reads the accumulators
// with tcgen05.ld: warp w covers TMEM lanes (= tile rows) 32 (w % 4).. and every other group
// of 16 columns. Tiles are dealt round-robin to the CL CTAs of the cluster.
constexpr int UM_BM = 128, UM_BK = 32, UM_MAXBN = 64;
constexpr int UM_TILE_A = UM_BM * UM_BK * 4;       // 16 KB: 128 rows x 32 FP32
constexpr int UM_TILE_B = UM_MAXBN * UM_BK * 4;    // 8 KB
constexpr uint32_t UM_TMEM_COLS = 2 * UM_MAXBN;    // two halves of BN <= 64 FP32 columns
struct UmmaSmem {                                  // 1 KB aligned; one parity half at a time
  unsigned char a[2][UM_TILE_A];                   // [hi, lo]
  unsigned char b[2][UM_TILE_B];                   // [hi, lo]
};
constexpr size_t ENS_SMEM_BYTES = sizeof(UmmaSmem) + 1024;   // + alignment slack

// per-CTA state of the tensor-core GEMMs: tensor-memory base, the MMA-completion mbarrier and
// the number of commits so far (every thread counts them alike, so the parity is known)
struct UmmaState {
  uint32_t tmem;
  uint32_t bar;
  uint32_t commits;
  int* err;
};

// default tile column width: the largest multiple of 16 up to 64 that divides H (H = s/2,
// s a multiple of 32); narrower tiles give a cluster more tiles to share on small grids
__host__ __device__ __forceinline__ int um_bn(int H) {
  for (int bn = UM_MAXBN; bn >= 16; bn -= 16)
    if (H % bn == 0) return bn;
  return 16;
}

static bool um_bn_valid(int s, int bn) {
  return bn >= 16 && bn <= UM_MAXBN && bn % 16 == 0 && (s / 2) % bn == 0;
}

// v ~= hi + lo, both TF32 values in FP32 words
__device__ __forceinline__ void um_split(float v, float& hi, float& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
  const float r = v - __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
  hi = __uint_as_float(h);
  lo = __uint_as_float(l);
}

// write the split of 4 consecutive K values (chunk c of row r) into hi and lo tiles with the
// 128B swizzle: the 16-byte chunk index is XORed with r % 8
__device__ __forceinline__ void um_put(unsigned char* hi, unsigned char* lo, int r, int c, float4 v) {
  float4 h, l;
  um_split(v.x, h.x, l.x);
  um_split(v.y, h.y, l.y);
  um_split(v.z, h.z, l.z);
  um_split(v.w, h.w, l.w);
  const int off = r * 128 + ((c ^ (r & 7)) << 4);
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = l;
}

__device__ __forceinline__ float4 f4_add(float4 a, float4 b, float sg) {
  return make_float4(a.x + sg * b.x, a.y + sg * b.y, a.z + sg * b.z, a.w + sg * b.w);
}

// bounded wait for the latest commit; false (and the error flagged) if it never completes
__device__ __forceinline__ bool um_wait(UmmaState& st) {
  return tc::s_wait(st.bar, (st.commits - 1) & 1u, st.err);
}

template <bool FWD>
__device__ void dual_umma(const float* __restrict__ A, const float* __restrict__ B,
                          float* __restrict__ out, int s, int BN, int rows, const float* lam,
                          float dtnu, bool scale, UmmaSmem& sm, UmmaState& st, int rank, int CL) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int H = s / 2;
  const int nrt = (rows + UM_BM - 1) / UM_BM, nct = H / BN;
  const int KS = (H + UM_BK - 1) / UM_BK;
  // instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32 (bits
  // 7-9 and 10-12 = 2), both K-major, N / 8 (bits 17-22), M / 16 (bits 24-28)
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                         ((uint32_t)(UM_BM >> 4) << 24);
  // an earlier wait of this launch gave up: leave at once (decided CTA-wide)
  if (__syncthreads_or(*(volatile int*)st.err != 0)) return;
  for (int tile = rank; tile < nrt * nct; tile += CL) {
    const int row0 = (tile / nct) * UM_BM, col0 = (tile % nct) * BN;
    for (int kb = 0; kb < KS; ++kb) {
      const int k0 = kb * UM_BK;
      for (int h = 0; h < 2; ++h) {   // the parity halves in turn through one set of buffers
        // the half-slice's A operand into registers first, so that its loads overlap the
        // previous MMAs, which still read the slice buffers.
        // A: 128 rows x 8 chunks of 4 K values; 4 chunks per thread
        constexpr int NA = UM_BM * 8 / ENS_THREADS;
        float4 av[NA];
#pragma unroll
        for (int v = 0; v < NA; ++v) {
          const int e = t + v * ENS_THREADS, r = e >> 3, c = e & 7, gr = row0 + r;
          const int k = k0 + c * 4;
          av[v] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (gr < rows && k < H) {
            const float* ar = A + (long)gr * s;
            if (FWD) {
              // x' = k..k+3 and their mirrors s-1-x' (a reversed float4)
              const float4 x = *reinterpret_cast<const float4*>(ar + k);
              const float4 m4 = *reinterpret_cast<const float4*>(ar + s - 4 - k);
              const float4 m = make_float4(m4.w, m4.z, m4.y, m4.x);
              av[v] = f4_add(x, m, h ? -1.f : 1.f);
            } else {
              av[v] = *reinterpret_cast<const float4*>(ar + h * H + k);
            }
          }
        }
        // the decision to give up is made by the whole CTA together, so every thread leaves
        // at the same point
        const bool ok = st.commits == 0 || um_wait(st);
        if (__syncthreads_or(!ok)) return;
#pragma unroll
        for (int v = 0; v < NA; ++v) {
          const int e = t + v * ENS_THREADS;
          um_put(sm.a[0], sm.a[1], e >> 3, e & 7, av[v]);
        }
        // B (tables that stay in L2): BN rows x 8 chunks
        for (int e = t; e < BN * 8; e += ENS_THREADS) {
          const int r = e >> 3, c = e & 7, gc = col0 + r;
          const int k = k0 + c * 4;
          float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (k < H) {
            // forward: rows k' and H + k' of Qts; inverse: row x' of Qs, columns k' and H + k'
            bv = FWD ? *reinterpret_cast<const float4*>(B + (long)(h * H + gc) * s + k)
                     : *reinterpret_cast<const float4*>(B + (long)gc * s + h * H + k);
          }
          um_put(sm.b[0], sm.b[1], r, c, bv);
        }
        tc::s_fence_async_smem();
        __syncthreads();
        if (t == 0) {
          tc::s_fence_after();
          const int kst = min(4, (H - k0) / 8);   // H is a multiple of 16: 2 or 4 steps
          const uint64_t ah = tc::s_desc(tc::s_u32(sm.a[0])), al = tc::s_desc(tc::s_u32(sm.a[1]));
          const uint64_t bh = tc::s_desc(tc::s_u32(sm.b[0])), bl = tc::s_desc(tc::s_u32(sm.b[1]));
          const uint32_t acc = st.tmem + (uint32_t)(h * BN);
          for (int ks = 0; ks < kst; ++ks) {
            const uint64_t adv = (uint64_t)(ks * 32 >> 4);   // 8 FP32 = 32 bytes along K
            tc::s_mma_tf32(acc, ah + adv, bh + adv, idesc, (kb | ks) != 0);
            tc::s_mma_tf32(acc, ah + adv, bl + adv, idesc, 1);
            tc::s_mma_tf32(acc, al + adv, bh + adv, idesc, 1);
          }
          tc::s_commit(st.bar);
        }
        ++st.commits;
      }
    }
    if (__syncthreads_or(!um_wait(st))) return;
    tc::s_fence_after();
    // epilogue: TMEM lane = tile row; warp w reads lanes 32 (w % 4).. and column groups of 16
    const int rl0 = row0 + 32 * (warp & 3) + lane;
    const bool live = rl0 < rows;
    const int plane = live ? rl0 / s : 0, rl = rl0 - plane * s;
    float* op = out + (long)plane * s * s;
    const uint32_t tl = st.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int ch = warp >> 2; ch < BN / 16; ch += 2) {
      uint32_t v0[16], v1[16];
      tc::s_ld16(tl + (uint32_t)(ch * 16), v0);
      tc::s_ld16(tl + (uint32_t)(BN + ch * 16), v1);
      tc::s_ld_wait();
      if (!live) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = col0 + ch * 16 + j;   // k' (forward) or x' (inverse), < H
        float x0 = __uint_as_float(v0[j]), x1 = __uint_as_float(v1[j]);
        if (FWD) {
          if (scale) {   // den = 1 - dtnu (lam_y + lam_x) as one explicit fma
            x0 = __fdividef(x0, __fmaf_rn(-dtnu, lam[rl] + lam[c], 1.0f));
            x1 = __fdividef(x1, __fmaf_rn(-dtnu, lam[rl] + lam[H + c], 1.0f));
          }
          op[(long)c * s + rl] = x0;
          op[(long)(H + c) * s + rl] = x1;
        } else {
          op[(long)c * s + rl] = x0 + x1;
          op[(long)(s - 1 - c) * s + rl] = x0 - x1;
        }
      }
    }
    // the accumulators are free again once every thread has read them (the next tile's MMAs
    // are issued after the barrier of its first slice)
    tc::s_fence_before();
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

// Fast-diagonalisation solve of np planes on the tensor cores: df = Q ((Q^T rf Q) ./ den) Q^T,
// each transform as a parity-split pair of half-size products (spectral indices in split
// order throughout), FP32 in and out
template <int CL>
__device__ void cl_solve(const EnsClass& C, const EnsInst& I, int np, const float* rf, float* t1,
                         float* t2, float* df, UmmaSmem& sm, UmmaState& st, int rank) {
  const int s = C.s, rows = np * s;
  dual_umma<true>(rf, C.Qts, t1, s, C.bn, rows, C.lam, I.dtnu, false, sm, st, rank, CL);
  csync<CL>();
  dual_umma<true>(t1, C.Qts, t2, s, C.bn, rows, C.lam, I.dtnu, true, sm, st, rank, CL);
  csync<CL>();
  dual_umma<false>(t2, C.Qs, t1, s, C.bn, rows, C.lam, I.dtnu, false, sm, st, rank, CL);
  csync<CL>();
  dual_umma<false>(t1, C.Qs, df, s, C.bn, rows, C.lam, I.dtnu, false, sm, st, rank, CL);
  csync<CL>();
}

// 64 registers: four CTAs (32 warps) fit per SM, as shared memory (49 KB) and tensor memory
// (128 columns) allow. The FP64 phases need the warps to hide their load latency, and while
// one CTA waits in a GEMM round the others keep the FP64 pipe busy (measured: 0.98 s against
// 1.08 s with 80 registers and three CTAs, despite some spilling in the cluster versions)
template <int CL>
__global__ void __launch_bounds__(ENS_THREADS, 4) ensemble_kernel(const __grid_constant__ EnsArgs a) {
  extern __shared__ __align__(16) unsigned char ens_smem[];   // ENS_SMEM_BYTES: GEMM slices
  __shared__ int item;
  __shared__ __align__(8) uint64_t um_bar;
  __shared__ uint32_t um_tmem_slot;
  const int rank = (CL > 1) ? (int)cooperative_groups::this_cluster().block_rank() : 0;
  // tensor-core set-up: the slice buffers on a 1 KB boundary (128B swizzle), the MMA-completion
  // barrier, and UM_TMEM_COLS columns of tensor memory for the accumulators
  const uint32_t pad = (1024u - (tc::s_u32(ens_smem) & 1023u)) & 1023u;
  UmmaSmem& usm = *reinterpret_cast<UmmaSmem*>(ens_smem + pad);
  if (threadIdx.x == 0) {
    tc::s_init(tc::s_u32(&um_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) tc::s_tmem_alloc(tc::s_u32(&um_tmem_slot), UM_TMEM_COLS);
  tc::s_fence_before();
  __syncthreads();
  tc::s_fence_after();
  UmmaState ust{um_tmem_slot, tc::s_u32(&um_bar), 0u, a.err};
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
      cl_solve<CL>(C, I, na, rf, t1, t2, rf, usm, ust, rank);
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
        cl_solve<CL>(C, I, na, rf, t1, t2, rf, usm, ust, rank);
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
            // explicit roundings: every instantiation (cluster size) computes the same bits
            const double fn = __dsub_rn(__dmul_rn(-I.a2h, xe[u] - xw[u]),
                                        __dmul_rn(I.b2h, yn[u] - ys[u]));
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
  // every MMA has been waited for (or a wait gave up and flagged the error): free the tensor
  // memory
  tc::s_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc::s_fence_after();
    tc::s_tmem_free(ust.tmem, UM_TMEM_COLS);
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
  int* err_dev = nullptr;              // device-side error flag (bounded waits that gave up)
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

// grid for cluster size cl and `per_sm` CTAs per SM (workspace holds 4 * sms clusters)
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
  a.err = b->err_dev;
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
    C.bn = um_bn(s / 2);
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
  // per-cluster workspace, enough for one-CTA clusters, four per SM
  b->ws_plane = (long)smax * smax;
  const long ctas = 4L * b->sms;
  if ((rc = b_alloc(b, &p, (size_t)ctas * EMaxP * b->ws_plane * sizeof(double))) != RIDC_OK) return fail(rc);
  b->r_ws = (double*)p;
  if ((rc = b_alloc(b, &p, (size_t)ctas * EMaxP * b->ws_plane * sizeof(double))) != RIDC_OK) return fail(rc);
  b->d_ws = (double*)p;
  if ((rc = b_alloc(b, &p, (size_t)ctas * 3 * EMaxP * b->ws_plane * sizeof(float))) != RIDC_OK) return fail(rc);
  b->f_ws = (float*)p;
  if ((rc = b_alloc(b, &p, sizeof(int))) != RIDC_OK) return fail(rc);
  b->err_dev = (int*)p;
  cudaMemset(p, 0, sizeof(int));
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
    const double fn = __dsub_rn(__dmul_rn(-I.a2h, xe - xw), __dmul_rn(I.b2h, yn - ys));
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
  int err = 0;
  e = cudaMemcpy(&err, b->err_dev, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (err) {   // reported once: the flag is cleared for the calls that follow
    cudaMemset(b->err_dev, 0, sizeof(int));
    return RIDC_ERR_TIMEOUT;
  }
  if (!out_on_device)
    for (size_t k = 0; k < count; ++k)
      if (!std::isfinite(out[k])) return RIDC_ERR_NONFINITE;
  return RIDC_OK;
}

extern "C" long ridc_batch_cells(ridc_batch h) {
  BatchCtx* b = bctx(h);
  return b ? b->cells_per_step : -1;
}

// Autotuner: first the cluster size (1, 2 or 4 CTAs per instance) and the CTAs per SM (1 to 4)
// that run the whole batch fastest, then, at that launch shape, the tile width of each grid
// side's tensor-core products (a multiple of 16 up to 64 that divides side/2) one side at a
// time. Each trial advances `nsteps` top-level steps of the whole batch from the current state.
// The choices are kept for later advances; *choice = CTAs per SM * 16 + cluster size.
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
  float best = 1e30f;
  int bcl = b->cl, bps = b->per_sm;
  for (int per_sm = 1; per_sm <= 4 && rc == RIDC_OK; ++per_sm)
    for (int cl = 1; cl <= 4 && rc == RIDC_OK; cl *= 2) {
      float ms = 0.f;
      rc = timed(cl, per_sm, b->order_dev, b->n, &ms);
      if (ms < best) { best = ms; bcl = cl; bps = per_sm; }
    }
  // then, at that launch shape, the tile width of each grid side's products in turn
  auto upload = [&]() {
    return cudaMemcpyAsync(b->cls_dev, b->cls.data(), b->cls.size() * sizeof(EnsClass),
                           cudaMemcpyHostToDevice, b->stream);
  };
  for (size_t c = 0; c < b->cls.size() && rc == RIDC_OK; ++c) {
    const int s = b->cls[c].s, keep = b->cls[c].bn;
    int best_bn = keep;
    for (int bn = 16; bn <= UM_MAXBN && rc == RIDC_OK; bn += 16) {
      if (bn == keep || !um_bn_valid(s, bn)) continue;
      b->cls[c].bn = bn;
      if (upload() != cudaSuccess) { rc = RIDC_ERR_CUDA; break; }
      float ms = 0.f;
      rc = timed(bcl, bps, b->order_dev, b->n, &ms);
      if (rc == RIDC_OK && ms < best) { best = ms; best_bn = bn; }
    }
    b->cls[c].bn = best_bn;
    if (upload() != cudaSuccess && rc == RIDC_OK) rc = RIDC_ERR_CUDA;
  }
  restore();
  cudaStreamSynchronize(b->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RIDC_OK) return rc;
  b->cl = bcl;
  b->per_sm = bps;
  b->initialised = false;
  if (choice) *choice = bps * 16 + bcl;
  if (best_ms) *best_ms = best;
  return RIDC_OK;
}

extern "C" int ridc_batch_tile_width(ridc_batch h, int side) {
  BatchCtx* b = bctx(h);
  if (!b) return RIDC_ERR_ARG;
  for (const EnsClass& C : b->cls)
    if (C.s == side) return C.bn;
  return RIDC_ERR_ARG;
}

extern "C" int ridc_batch_set_tile_width(ridc_batch h, int side, int width) {
  BatchCtx* b = bctx(h);
  if (!b) return RIDC_ERR_ARG;
  DeviceGuard dg(b->device);
  for (EnsClass& C : b->cls) {
    if (C.s != side) continue;
    if (!um_bn_valid(side, width)) return RIDC_ERR_ARG;
    C.bn = width;
    // stream-ordered after every advance already issued
    return cuda_status(cudaMemcpyAsync(b->cls_dev, b->cls.data(), b->cls.size() * sizeof(EnsClass),
                                       cudaMemcpyHostToDevice, b->stream));
  }
  return RIDC_ERR_ARG;
}

extern "C" int ridc_batch_set_launch(ridc_batch h, int choice) {
  BatchCtx* b = bctx(h);
  if (!b) return RIDC_ERR_ARG;
  const int per_sm = choice / 16, cl = choice % 16;
  if (per_sm < 1 || per_sm > 4 || (cl != 1 && cl != 2 && cl != 4)) return RIDC_ERR_ARG;
  b->per_sm = per_sm;
  b->cl = cl;
  return RIDC_OK;
}
