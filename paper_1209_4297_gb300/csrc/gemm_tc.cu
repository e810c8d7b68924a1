// Split-precision fast-diagonalisation GEMM on the 5th-generation tensor cores (sm_103a).
//
//   C[row][m] = sum_k A[row][k] B[m][k]          rows = nplanes * N, m, k < N
//   A ~= Ah + Al, B ~= Bh + Bl (BF16 hi/lo), C ~= Ah Bh + Ah Bl + Al Bh, FP32 accumulation.
//   The result is stored transposed per plane, out[plane][m][row % N], so the next GEMM again
//   contracts a contiguous axis; four such products give Q ((Q^T R Q) ./ den) Q^T.
//
// Output tiles are 128 x 256, K consumed in 64-wide blocks. A producer thread moves Ah, Al,
// Bh, Bl tiles (128B-swizzled) into a 2-stage shared-memory ring with TMA; one thread issues
// 3 x 4 tcgen05.mma (M=128, N=256, K=16) per block into one of two TMEM accumulators; four
// epilogue warps read TMEM with tcgen05.ld and apply the epilogue:
//   EPI_STORE      re-split to BF16 hi/lo for the next GEMM,
//   EPI_SCALE_DEN  multiply by 1 / (1 - dt nu_s (lam_kx + lam_ky)) first,
//   EPI_DELTA      write the FP32 solution increment of this pass (the refinement residual
//                  kernel folds it into the FP64 total, so the epilogue reads nothing).
// Every mbarrier wait is bounded by a 2 s %globaltimer budget; on expiry the kernel records an
// error flag, lets its copies and MMAs drain, frees its TMEM and returns.
#include <cudaTypedefs.h>

#include "ridc_internal.h"

namespace ridc {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 64, TC_STAGES = 2;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;                  // 16 KB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;                  // 32 KB
constexpr int TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;  // 96 KB
constexpr int TC_MAX_N = 4096;   // eigenvalue staging in shared memory
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024 + 1024 + TC_MAX_N * 4;
constexpr int TC_THREADS = 192;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

struct TcArgs {
  int n, rows, epi, S;
  __nv_bfloat16* oh;
  __nv_bfloat16* ol;
  float* o32;
  const float* lam;
  float dtnu[kMaxSpecies];
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity; false (and *err = 1) after TC_WAIT_NS
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      const unsigned long long t = gtimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > TC_WAIT_NS) {
        atomicExch(err, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile whose 64-element (128 B) rows were
// written by TMA with 128B swizzling; 8-row groups are 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)(16u >> 4) << 16;           // leading byte offset (unused with swizzling)
  d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 D, both K-major, M=128, N=256.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Persistent: one CTA per SM walks the output tiles t = blockIdx.x + i * gridDim.x (n-tile
// fastest, so CTAs running together share A rows in L2). The TMA producer and the MMA issuer
// run ahead across tile boundaries; two TMEM accumulators (256 columns each) let the four
// epilogue warps drain tile i while the tensor cores compute tile i+1.
__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                   const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                   const __grid_constant__ TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TC_STAGES * TC_STAGE_BYTES);
  // full[S], empty[S], acc_full[2], acc_empty[2], mma_done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 5);
  float* lam_s = reinterpret_cast<float*>(smem + TC_STAGES * TC_STAGE_BYTES + 1024);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = a.n / TC_BK;
  const int ntn = a.n / TC_BN;
  const int ntiles = (a.rows / TC_BM) * ntn;
  volatile int* errv = a.err;
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + TC_STAGES + s); };
  auto accf = [&](int b) { return smem_u32(bars + 2 * TC_STAGES + b); };
  auto acce = [&](int b) { return smem_u32(bars + 2 * TC_STAGES + 2 + b); };
  const uint32_t mma_done = smem_u32(bars + 2 * TC_STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf(b), 1);
      mbar_init(acce(b), 4);   // one arrival per epilogue warp
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tAh)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tAl)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tBh)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tBl)) : "memory");
  }
  if (a.epi == EPI_SCALE_DEN)
    for (int i = threadIdx.x; i < a.n; i += TC_THREADS) lam_s[i] = a.lam[i];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    long issued = 0;   // K blocks issued so far (stage ring position)
    for (int t = blockIdx.x; t < ntiles && !*errv; t += gridDim.x) {
      const int m0 = (t / ntn) * TC_BM, n0 = (t % ntn) * TC_BN;
      bool ok = true;
      for (int kb = 0; kb < KB; ++kb, ++issued) {
        const int s = (int)(issued % TC_STAGES);
        const long it = issued / TC_STAGES;
        if (issued >= TC_STAGES && !mbar_wait(empty(s), (uint32_t)((it - 1) & 1), a.err)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * TC_STAGE_BYTES;
        mbar_expect_tx(full(s), TC_STAGE_BYTES);
        tma_load_2d(smem_u32(st), &tAh, full(s), kb * TC_BK, m0);
        tma_load_2d(smem_u32(st + TC_A_BYTES), &tAl, full(s), kb * TC_BK, m0);
        tma_load_2d(smem_u32(st + 2 * TC_A_BYTES), &tBh, full(s), kb * TC_BK, n0);
        tma_load_2d(smem_u32(st + 2 * TC_A_BYTES + TC_B_BYTES), &tBl, full(s), kb * TC_BK, n0);
      }
      if (!ok) break;
    }
    // none of our copies may still be in flight when the CTA retires
    for (long q = issued - 1; q >= 0 && q >= issued - TC_STAGES; --q)
      mbar_wait(full((int)(q % TC_STAGES)), (uint32_t)((q / TC_STAGES) & 1), a.err);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    long consumed = 0;
    int local = 0;
    for (int t = blockIdx.x; t < ntiles && !*errv; t += gridDim.x, ++local) {
      const int b = local & 1;
      const int use = local >> 1;   // how often accumulator b was used before
      if (use > 0 && !mbar_wait(acce(b), (uint32_t)((use - 1) & 1), a.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)(b * TC_TMEM_COLS);
      bool ok = true;
      for (int kb = 0; kb < KB; ++kb, ++consumed) {
        const int s = (int)(consumed % TC_STAGES);
        if (!mbar_wait(full(s), (uint32_t)((consumed / TC_STAGES) & 1), a.err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = smem_u32(smem + s * TC_STAGE_BYTES);
        const uint64_t ah = sdesc(st), al = sdesc(st + TC_A_BYTES);
        const uint64_t bh = sdesc(st + 2 * TC_A_BYTES), bl = sdesc(st + 2 * TC_A_BYTES + TC_B_BYTES);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;   // 16 BF16 = 32 bytes along K
          mma_bf16(acc, ah + adv, bh + adv, (kb | kk) != 0);
          mma_bf16(acc, ah + adv, bl + adv, 1);
          mma_bf16(acc, al + adv, bh + adv, 1);
        }
        mma_commit(empty(s));
      }
      if (!ok) break;
      mma_commit(accf(b));
    }
    // every MMA issued by this CTA completes before TMEM is released
    mma_commit(mma_done);
    mbar_wait(mma_done, 0, a.err);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM -> registers -> global, transposed per plane ----
    const int q = warp & 3;   // TMEM lane quarter this warp may access
    const int n = a.n;
    int local = 0;
    for (int t = blockIdx.x; t < ntiles && !*errv; t += gridDim.x, ++local) {
      const int b = local & 1;
      if (!mbar_wait(accf(b), (uint32_t)((local >> 1) & 1), a.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m0 = (t / ntn) * TC_BM, n0 = (t % ntn) * TC_BN;
      const int row = m0 + q * 32 + lane;
      const int plane = row / n, rl = row - plane * n;
      const int s = plane % a.S;
      // den = 1 - dt nu_s (lam_kx + lam_ky) = den_r + den_m
      const float dtnu = a.dtnu[s];
      const float den_r = (a.epi == EPI_SCALE_DEN) ? 1.0f - dtnu * lam_s[rl] : 0.f;
      const uint32_t acc = tmem + (uint32_t)(b * TC_TMEM_COLS) + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < TC_BN; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(acc + (uint32_t)c0, v);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int m = n0 + c0 + jj;
          float val = __uint_as_float(v[jj]);
          const size_t idx = ((size_t)plane * n + m) * n + rl;
          if (a.epi == EPI_DELTA) {
            a.o32[idx] = val;
          } else {
            if (a.epi == EPI_SCALE_DEN) val *= __frcp_rn(fmaf(-dtnu, lam_s[m], den_r));
            const __nv_bfloat16 h = __float2bfloat16_rn(val);
            a.oh[idx] = h;
            a.ol[idx] = __float2bfloat16_rn(val - __bfloat162float(h));
          }
        }
      }
      // accumulator b may be overwritten once all four warps have read it
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
                 "r"(2 * TC_TMEM_COLS)
                 : "memory");
  }
}

int make_tensor_map(CUtensorMap* tm, const void* base, long rows, long cols, int box_rows) {
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
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RIDC_OK : RIDC_ERR_CUDA;
}

int launch_gemm_tc(Ctx* c, const CUtensorMap* ah, const CUtensorMap* al, const CUtensorMap* bh,
                   const CUtensorMap* bl, int nplanes, int epi, __nv_bfloat16* oh,
                   __nv_bfloat16* ol, float* o32) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TC_SMEM);
    if (e != cudaSuccess) return cuda_status(e);
    attr_done = true;
  }
  const int n = c->n;
  if (n % TC_BN != 0) return RIDC_ERR_UNSUPPORTED;
  TcArgs a{};
  a.n = n;
  a.rows = nplanes * n;
  a.epi = epi;
  a.S = c->S;
  a.oh = oh;
  a.ol = ol;
  a.o32 = o32;
  a.lam = c->lam_f;
  for (int s = 0; s < c->S; ++s) a.dtnu[s] = (float)(c->dt * c->nu[s]);
  a.err = c->err_dev;
  if (n > TC_MAX_N) return RIDC_ERR_UNSUPPORTED;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int ntiles = (a.rows / TC_BM) * (n / TC_BN);
  dim3 grid(ntiles < sms ? ntiles : sms);
  cudaEvent_t e0;
  prof_begin(c, RIDC_KERNEL_GEMM_TC, &e0);
  gemm_tc_kernel<<<grid, TC_THREADS, TC_SMEM, c->stream>>>(*ah, *al, *bh, *bl, a);
  prof_end(c, RIDC_KERNEL_GEMM_TC, e0);
  return cuda_status(cudaGetLastError());
}

}  // namespace ridc
