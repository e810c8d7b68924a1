// Split-precision fast-diagonalisation GEMMs on the 5th-generation tensor cores (sm_103a),
// with the parity of the eigenvectors folded in.
//
// The cosine (Neumann) and sine (Dirichlet) eigenvectors of the cell-centred Laplacian obey
// Q[N-1-x][k] = (-1)^k Q[x][k]. With H = N/2, Qe[x'][k'] = Q[x'][2k'], Qo[x'][k'] = Q[x'][2k'+1]:
//   forward   V[2k']   = sum_{x'<H} (v[x'] + v[N-1-x']) Qe[x'][k']
//             V[2k'+1] = sum_{x'<H} (v[x'] - v[N-1-x']) Qo[x'][k']
//   inverse   u[x'] = E[x'] + O[x'],  u[N-1-x'] = E[x'] - O[x'],
//             E = sum_{k'} V[2k'] Qe[x'][k'],  O = sum_{k'} V[2k'+1] Qo[x'][k']
// so each transform is two (rows x H) x (H x H) products instead of one (rows x N) x (N x N):
// half the tensor-core work. Spectral indices are kept in split order (even k, then odd k).
//
// The y parity split is applied to the right-hand side before the first transform (the
// transforms are linear): its operand holds, per plane and x parity gx, the rows gy*N/2 + y'
// of v[gx][gy][y'][x'] = (v[y'][x'] +- v[y'][N-1-x']) +- (v[N-1-y'][x'] +- v[N-1-y'][N-1-x']).
// The first transform then writes each result row straight into the second's operand.
//
// Operands are BF16 hi/lo splits, C ~= Ah Bh + Ah Bl + Al Bh with FP32 accumulation in TMEM,
// or FP16 hi/lo splits of scaled values (the FP16 form): tables times 2^qexp, each plane of the
// first operand times its own 2^k. Every epilogue then multiplies by 2^-qexp, and the last
// also by 2^-k; the intermediates stay in the scaled units, which keeps them inside FP16's
// range (at most N 2^3 <= 2^15) and above its subnormals.
// Every product contracts the contiguous axis of its A rows and stores transposed per plane.
//   SYM_FWD_SPLIT forward, hi/lo store into [plane][gy][kx][y'] (first transform, x)
//   SYM_FWD_DEN   forward, times 1/den, hi/lo store     (second transform, y)
//   SYM_BWD_SPLIT inverse with the E +- O butterfly, hi/lo (third transform, x)
//   SYM_BWD_F32   inverse with the E +- O butterfly, FP32  (fourth transform, y: the increment)
//
// Persistent: one CTA per SM over a static tile list; a TMA producer thread and an MMA thread
// run ahead over a ring of stages (Ah, Al, Bh, Bl tiles, K = 64, 128B swizzle): forward
// products use 128 x 256 tiles in two 96 KB stages, inverse products 128 x 128 tiles with E
// and O accumulators in three 64 KB stages; two TMEM buffers of 256 columns let four epilogue
// warps drain one tile while the next is computed. Every mbarrier wait is bounded
// (2 s of %globaltimer); on expiry the kernel flags the error, drains and frees TMEM.
#include <cudaTypedefs.h>

#include "ridc_internal.h"
#include "tc_util.cuh"

namespace ridc {

namespace {

using namespace tc;

constexpr int SY_BM = 128;
constexpr int SY_MAXN = 4096;

// Tile shapes. Forward products (one accumulator) use 128 x 256 tiles when N/2 allows: the
// tensor cores read both operands from shared memory, and 256 columns per instruction keep
// that traffic under the per-SM bandwidth (128 columns need about 95% of it). Inverse
// products keep two 128-column accumulators (E and O) per tile.
template <bool FWD, int BN>
struct SyCfg {
  // K slice per pipeline stage. Forward products take 32 BF16 values per row (64-byte rows,
  // 64B swizzle): 48 KB stages at 128 x 256, so four fit where two 96 KB stages did, and the
  // tensor cores wait less for TMA (measured: with two stages the MMA thread waited on TMA
  // data 29% of its time in the forward products, 10% in the inverse ones). Inverse products
  // keep 64 values (128-byte rows, 128B swizzle) in three 64 KB stages.
  static constexpr int BK = FWD ? 32 : 64;
  static constexpr int ATILE = SY_BM * BK * 2;
  static constexpr int BTILE = BN * BK * 2;
  static constexpr int STAGE = 2 * ATILE + 2 * BTILE;
  static constexpr int STAGES = FWD ? (BN == 256 ? 4 : 6) : 3;
  static constexpr int NSEG = FWD ? 1 : 2;
  // shared-memory descriptor: swizzle mode (bits 61-63: 2 = 128B, 4 = 64B) and the byte
  // stride between 8-row groups
  static constexpr uint32_t SWZ = FWD ? 4 : 2;
  static constexpr uint32_t SBO = 8 * BK * 2;
  // instruction descriptor of kind::f16: FP32 accumulator (bits 4-5), A and B formats (bits
  // 7-9 and 10-12: 1 = BF16, 0 = FP16; both operands always share one), N / 8, M / 16
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(SY_BM >> 4) << 24);
  static constexpr uint32_t IDESC_F16 = IDESC & ~((7u << 7) | (7u << 10));
};

// K-major operand tile of 8-row groups SBO bytes apart, swizzle mode SWZ; the tile starts on
// a 1 KB boundary
__device__ __forceinline__ uint64_t sy_desc(uint32_t addr, uint32_t sbo, uint32_t swz) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)swz << 61;
  return d;
}
// dynamic shared memory: stages + barriers + alignment slack, plus the eigenvalues in the
// denominator mode only
template <bool FWD, int BN>
constexpr int sy_smem_base() { return SyCfg<FWD, BN>::STAGES * SyCfg<FWD, BN>::STAGE + 1024 + 1024; }
constexpr int SY_SMEM_MAX =
    (SyCfg<true, 256>::STAGES * SyCfg<true, 256>::STAGE > SyCfg<false, 128>::STAGES * SyCfg<false, 128>::STAGE
         ? SyCfg<true, 256>::STAGES * SyCfg<true, 256>::STAGE
         : SyCfg<false, 128>::STAGES * SyCfg<false, 128>::STAGE) +
    2048 + SY_MAXN * 4;
static_assert(SyCfg<true, 128>::STAGES * SyCfg<true, 128>::STAGE <=
                  SyCfg<true, 256>::STAGES * SyCfg<true, 256>::STAGE,
              "stage sets fit the shared-memory limit");
constexpr int SY_THREADS = 192;
constexpr uint32_t SY_ACC_COLS = 256;        // per TMEM buffer: E (128) + O (128)

__device__ __forceinline__ void s_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void s_tma(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int c0,
                                      int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void s_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                      uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// v = hi + lo to about 16 (BF16) or 22 (FP16) significant bits; v - hi is exact in FP32
__device__ __forceinline__ void s_split(float v, __nv_bfloat16* hi, __nv_bfloat16* lo, size_t idx,
                                        bool f16) {
  if (f16) {
    const __half h = __float2half_rn(v);
    reinterpret_cast<__half*>(hi)[idx] = h;
    reinterpret_cast<__half*>(lo)[idx] = __float2half_rn(v - __half2float(h));
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

struct SymArgs {
  int n, H, rows, mode, S, plane0;
  float* o32;
  __nv_bfloat16* oh;
  __nv_bfloat16* ol;
  const float* lam;   // eigenvalues in split order
  float dtnu[kMaxPlanes];   // a_p dt nu_s of plane p (a_p: its operator's diagonal)
  int* err;
  int stall;            // test hook: CTA 0 leaves its first stage unloaded
  int f16;              // FP16 form: FP16 operands and the power-of-two scales below
  float tscale;         // 2^-qexp (1 for BF16)
  const unsigned* pmax; // FP16 form: per-plane maxima of this solve pass (plane scales)
  int k0;               // FP16 form: target exponent of the plane scales
};

// tile -> (A row base, B row base, output plane-row base, column base, group)
struct SymTile {
  int arow, brow, m0, c0, g;
};

__device__ __forceinline__ SymTile sym_tile(const SymArgs& a, int t, bool fwd, int BN) {
  const int rt = a.rows / SY_BM, ct = a.H / BN;
  SymTile T;
  if (fwd) {
    T.g = t / (rt * ct);
    const int r = t - T.g * rt * ct;
    T.m0 = (r / ct) * SY_BM;
    T.c0 = (r % ct) * BN;
    // forward operands are laid out [plane][parity group][row][H]
    const int pl = a.plane0 + T.m0 / a.n;
    T.arow = (pl * 2 + T.g) * a.n + (T.m0 - (T.m0 / a.n) * a.n);
    T.brow = T.g * a.H + T.c0;
  } else {
    T.g = 0;
    T.m0 = (t / ct) * SY_BM;
    T.c0 = (t % ct) * BN;
    T.arow = a.plane0 * a.n + T.m0;
    T.brow = T.c0;
  }
  return T;
}

// F16: the FP16 form (FP16 operands, power-of-two scales in the epilogues), instantiated
// apart so the BF16 code carries none of it
template <bool FWD, int BN, bool F16>
__global__ void __launch_bounds__(SY_THREADS, 1)
    gemm_sym_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                    const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                    const __grid_constant__ SymArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  using Cfg = SyCfg<FWD, BN>;
  constexpr int SY_STAGES = Cfg::STAGES, SY_STAGE = Cfg::STAGE, BTILE = Cfg::BTILE;
  constexpr int BK = Cfg::BK, ATILE = Cfg::ATILE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SY_STAGES * SY_STAGE);
  // full[S], empty[S], acc_full[2], acc_empty[2], mma_done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SY_STAGES + 5);
  float* lam_s = reinterpret_cast<float*>(smem + SY_STAGES * SY_STAGE + 1024);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool fwd = FWD;
  constexpr int nseg = Cfg::NSEG;
  const int KB = a.H / BK;
  const int ntiles = (fwd ? 2 : 1) * (a.rows / SY_BM) * (a.H / BN);
  volatile int* errv = a.err;
  auto full = [&](int s) { return s_u32(bars + s); };
  auto empty = [&](int s) { return s_u32(bars + SY_STAGES + s); };
  auto accf = [&](int b) { return s_u32(bars + 2 * SY_STAGES + b); };
  auto acce = [&](int b) { return s_u32(bars + 2 * SY_STAGES + 2 + b); };
  const uint32_t mma_done = s_u32(bars + 2 * SY_STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < SY_STAGES; ++s) {
      s_init(full(s), 1);
      s_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      s_init(accf(b), 1);
      s_init(acce(b), 4);
    }
    s_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tAh)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tAl)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tBh)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tBl)) : "memory");
  }
  if (a.mode == SYM_FWD_DEN)
    for (int i = threadIdx.x; i < a.n; i += SY_THREADS) lam_s[i] = a.lam[i];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_u32(tmem_slot)),
                 "r"(2 * SY_ACC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    long issued = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok && !*errv; t += gridDim.x) {
      const SymTile T = sym_tile(a, t, fwd, BN);
      for (int seg = 0; seg < nseg && ok; ++seg) {
        const int koff = seg * a.H, brow = T.brow + seg * a.H;
        for (int kb = 0; kb < KB; ++kb, ++issued) {
          const int s = (int)(issued % SY_STAGES);
          const long it = issued / SY_STAGES;
          if (issued >= SY_STAGES && !s_wait(empty(s), (uint32_t)((it - 1) & 1), a.err)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * SY_STAGE;
          // test hook: the stage is never loaded, so its consumer's bounded wait runs out
          if (a.stall && blockIdx.x == 0 && issued == 0) continue;
          s_expect(full(s), SY_STAGE);
          s_tma(s_u32(st), &tAh, full(s), (fwd ? 0 : koff) + kb * BK, T.arow);
          s_tma(s_u32(st + ATILE), &tAl, full(s), (fwd ? 0 : koff) + kb * BK, T.arow);
          s_tma(s_u32(st + 2 * ATILE), &tBh, full(s), kb * BK, brow);
          s_tma(s_u32(st + 2 * ATILE + BTILE), &tBl, full(s), kb * BK, brow);
        }
      }
    }
    for (long q = issued - 1; q >= 0 && q >= issued - SY_STAGES; --q)
      s_wait(full((int)(q % SY_STAGES)), (uint32_t)((q / SY_STAGES) & 1), a.err);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    constexpr uint32_t idesc = F16 ? Cfg::IDESC_F16 : Cfg::IDESC;
    long consumed = 0;
    int local = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok && !*errv; t += gridDim.x, ++local) {
      const int b = local & 1;
      const int use = local >> 1;
      if (use > 0 && !s_wait(acce(b), (uint32_t)((use - 1) & 1), a.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int seg = 0; seg < nseg && ok; ++seg) {
        const uint32_t acc = tmem + (uint32_t)(b * SY_ACC_COLS + seg * BN);
        for (int kb = 0; kb < KB; ++kb, ++consumed) {
          const int s = (int)(consumed % SY_STAGES);
          if (!s_wait(full(s), (uint32_t)((consumed / SY_STAGES) & 1), a.err)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = s_u32(smem + s * SY_STAGE);
          const uint64_t ah = sy_desc(st, Cfg::SBO, Cfg::SWZ);
          const uint64_t al = sy_desc(st + ATILE, Cfg::SBO, Cfg::SWZ);
          const uint64_t bh = sy_desc(st + 2 * ATILE, Cfg::SBO, Cfg::SWZ);
          const uint64_t bl = sy_desc(st + 2 * ATILE + BTILE, Cfg::SBO, Cfg::SWZ);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            s_mma(acc, ah + adv, bh + adv, idesc, (kb | kk) != 0);
            s_mma(acc, ah + adv, bl + adv, idesc, 1);
            s_mma(acc, al + adv, bh + adv, idesc, 1);
          }
          s_commit(empty(s));
        }
      }
      if (!ok) break;
      s_commit(accf(b));
    }
    s_commit(mma_done);
    s_wait(mma_done, 0, a.err);
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int q = warp & 3;
    const int n = a.n;
    int local = 0;
    for (int t = blockIdx.x; t < ntiles && !*errv; t += gridDim.x, ++local) {
      const int b = local & 1;
      if (!s_wait(accf(b), (uint32_t)((local >> 1) & 1), a.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const SymTile T = sym_tile(a, t, fwd, BN);
      const int row = T.m0 + q * 32 + lane;
      const int plane = a.plane0 + row / n, rl = row - (row / n) * n;
      const size_t pbase = (size_t)plane * n;
      const uint32_t acc = tmem + (uint32_t)(b * SY_ACC_COLS) + ((uint32_t)(q * 32) << 16);
      if (fwd) {
        const int cbase = T.g * a.H + T.c0;   // output column position (split order)
        const float dtnu = a.dtnu[plane];
        const float den_r = (a.mode == SYM_FWD_DEN) ? 1.0f - dtnu * lam_s[rl] : 0.f;
        // first transform: row rl = gy N/2 + y' goes to row block gy of the next operand
        const int gy = rl >= a.H ? 1 : 0, yp = rl - gy * a.H;
        const size_t sbase = (size_t)(plane * 2 + gy) * n;
        for (int c = 0; c < BN; c += 16) {
          uint32_t v[16];
          s_ld16(acc + (uint32_t)c, v);
          // eigenvalues of the 16 columns: one shared-memory wavefront (a lane per column),
          // then shuffles; shared-memory bandwidth is what the tensor cores run short of
          const float lam_lane = (a.mode == SYM_FWD_DEN) ? lam_s[cbase + c + (lane & 15)] : 0.f;
          s_ld_wait();
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int m = cbase + c + jj;
            float val = __uint_as_float(v[jj]);
            if (a.mode == SYM_FWD_SPLIT) {
              s_split(F16 ? val * a.tscale : val, a.oh, a.ol, (sbase + m) * a.H + yp, F16);
            } else {
              const float den = fmaf(-dtnu, __shfl_sync(0xffffffffu, lam_lane, jj), den_r);
              // a BF16 split keeps ~16 bits: a 2-ulp fast division is ample; an FP16 split
              // keeps ~22, so it takes the correctly rounded quotient
              val = F16 ? __fdiv_rn(val * a.tscale, den) : __fdividef(val, den);
              s_split(val, a.oh, a.ol, (pbase + m) * n + rl, F16);
            }
          }
        }
      } else {
        // the last transform also removes the plane's own scale
        const float mult = !F16 ? 1.0f
                           : (a.mode == SYM_BWD_F32)
                               ? a.tscale * pow2f(-f16_plane_exp(a.pmax[plane], a.k0)) : a.tscale;
        for (int c = 0; c < BN; c += 16) {
          uint32_t e[16], o[16];
          s_ld16(acc + (uint32_t)c, e);
          s_ld16(acc + (uint32_t)(BN + c), o);
          s_ld_wait();
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int x = T.c0 + c + jj;
            const float ev = __uint_as_float(e[jj]), ov = __uint_as_float(o[jj]);
            const size_t i0 = (pbase + x) * n + rl, i1 = (pbase + (n - 1 - x)) * n + rl;
            const float sum = F16 ? (ev + ov) * mult : ev + ov;
            const float dif = F16 ? (ev - ov) * mult : ev - ov;
            if (a.mode == SYM_BWD_F32) {
              a.o32[i0] = sum;
              a.o32[i1] = dif;
            } else {
              s_split(sum, a.oh, a.ol, i0, F16);
              s_split(dif, a.oh, a.ol, i1, F16);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce(b)) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * SY_ACC_COLS)
                 : "memory");
  }
}

}  // namespace

int make_tensor_map(CUtensorMap* tm, const void* base, long rows, long cols, int box_rows,
                    bool fwd) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return RIDC_ERR_CUDA;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  // forward operands: 32-value rows, 64B swizzle; inverse operands: 64-value rows, 128B
  cuuint32_t box[2] = {(cuuint32_t)(fwd ? SyCfg<true, 256>::BK : SyCfg<false, 128>::BK),
                       (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      fwd ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RIDC_OK : RIDC_ERR_CUDA;
}

int gemm_sym_fwd_bn(int n) { return (n / 2) % 256 == 0 ? 256 : 128; }

template <bool FWD, int BN, bool F16>
static int launch_sym(Ctx* c, const CUtensorMap* ah, const CUtensorMap* al, const CUtensorMap* bh,
                      const CUtensorMap* bl, const SymArgs& a, int sms) {
  static std::atomic<unsigned long long> attr_done{0};
  RIDC_TRY(raise_smem_limit_once(gemm_sym_kernel<FWD, BN, F16>, SY_SMEM_MAX, &attr_done));
  const int ntiles = (FWD ? 2 : 1) * (a.rows / SY_BM) * (a.H / BN);
  dim3 grid(ntiles < sms ? ntiles : sms);
  const int smem = sy_smem_base<FWD, BN>() + (a.mode == SYM_FWD_DEN ? a.n * 4 : 0);
  gemm_sym_kernel<FWD, BN, F16><<<grid, SY_THREADS, smem, c->stream>>>(*ah, *al, *bh, *bl, a);
  return cuda_status(cudaGetLastError());
}

int launch_gemm_sym(Ctx* c, const CUtensorMap* ah, const CUtensorMap* al, const CUtensorMap* bh,
                    const CUtensorMap* bl, int plane0, int nplanes, int mode, __nv_bfloat16* oh,
                    __nv_bfloat16* ol, float* o32, int pass) {
  const int n = c->n;
  if (n % 256 != 0 || n > SY_MAXN) return RIDC_ERR_UNSUPPORTED;
  const int sms = current_sm_count();
  SymArgs a{};
  a.n = n;
  a.H = n / 2;
  a.rows = nplanes * n;
  a.plane0 = plane0;
  a.mode = mode;
  a.S = c->S;
  a.o32 = o32;
  a.oh = oh;
  a.ol = ol;
  a.lam = c->lam_f;
  if (plane0 < 0 || nplanes < 1 || plane0 + nplanes > kMaxPlanes) return RIDC_ERR_ARG;
  // (a dt) nu: with a = 1 exactly the correctors' dt nu
  for (int p = plane0; p < plane0 + nplanes; ++p)
    a.dtnu[p] = (float)((c->coef[c->plane_coef[p]] * c->dt) * c->nu[p % c->S]);
  a.err = c->err_dev;
  a.stall = c->stall_next_gemm;
  c->stall_next_gemm = 0;
  a.f16 = c->prec == RIDC_MIXED_FP16X3;
  a.tscale = a.f16 ? pow2f(-c->qexp) : 1.0f;
  a.pmax = a.f16 ? c->pmax + (size_t)pass * kMaxPlanes : nullptr;
  a.k0 = c->k0;
  const bool fwd = mode == SYM_FWD_SPLIT || mode == SYM_FWD_DEN;
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_GEMM_TC, &e0);
  int rc;
  const bool wide = gemm_sym_fwd_bn(n) == 256;
  if (a.f16) {
    if (!fwd) rc = launch_sym<false, 128, true>(c, ah, al, bh, bl, a, sms);
    else if (wide) rc = launch_sym<true, 256, true>(c, ah, al, bh, bl, a, sms);
    else rc = launch_sym<true, 128, true>(c, ah, al, bh, bl, a, sms);
  } else {
    if (!fwd) rc = launch_sym<false, 128, false>(c, ah, al, bh, bl, a, sms);
    else if (wide) rc = launch_sym<true, 256, false>(c, ah, al, bh, bl, a, sms);
    else rc = launch_sym<true, 128, false>(c, ah, al, bh, bl, a, sms);
  }
  prof_end(c, RIDC_KERNEL_GEMM_TC, e0);
  return rc;
}

}  // namespace ridc
