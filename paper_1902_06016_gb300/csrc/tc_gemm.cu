// tcgen05 GEMM kernel (see tc_gemm.cuh). Hand-written PTX: TMA (cp.async.bulk.tensor) loads into
// 128-byte-swizzled shared memory, mbarrier pipeline, tcgen05.mma with the accumulator in TMEM,
// tcgen05.ld epilogue. Every wait is bounded: on timeout the kernel records an error, skips the
// remaining work, releases its TMEM and returns.
#include "tc_gemm.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace gfcc {
namespace {

constexpr int BM = 128, BN = 256, STAGES = 4;
constexpr int KB_BYTES = 128;                        // one swizzle row of K per operand row
constexpr int A_BYTES = BM * KB_BYTES;               // 16 KB
constexpr int B_BYTES = BN * KB_BYTES;               // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TMEM_COLS = 512;                       // 128 lanes x (2 x 256) FP32 columns
constexpr long long WAIT_CYCLES = 4000000000LL;      // about two seconds at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused with 128-byte swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// instruction descriptor: FP32 accumulate, A/B format (bf16 = 1 for kind::f16, tf32 = 2 for
// kind::tf32), both K-major, N = 256, M = 128
template <TcKind K>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((K == TcKind::BF16 ? 1u : 2u) << 7) | ((K == TcKind::BF16 ? 1u : 2u) << 10) |
         ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <TcKind K>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  if constexpr (K == TcKind::BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc<K>()), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc<K>()), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// work unit u -> (split z, M tile, N tile). Within a split the M tiles are taken in groups of gm:
// a group runs through all N tiles with its gm M tiles fastest, so that the CTAs working at the same
// time share gm A tiles (kept in L2) and about (grid / gm) B tiles, each read from DRAM about once
// per group instead of once per wave.
struct Unit {
  int z, mt, nt;
};
__device__ __forceinline__ Unit decode_unit(int u, int tiles_m, int tiles_n, int gm) {
  const int per_z = tiles_m * tiles_n;
  Unit r;
  r.z = u / per_z;
  const int t = u - r.z * per_z;
  const int g = t / (gm * tiles_n);
  const int m0 = g * gm;
  const int gsz = min(gm, tiles_m - m0);
  const int w = t - m0 * tiles_n;
  r.nt = w / gsz;
  r.mt = m0 + (w - r.nt * gsz);
  return r;
}

// Persistent kernel: CTA b processes the work units b, b + gridDim.x, ... (unit = split z x 128-row
// M tile x 256-column N tile, K range [z nk_split, (z+1) nk_split) in k-blocks). Warp 0 is the TMA
// producer (one k-block per stage), warp 1 issues the MMAs, the remaining warps drain TMEM. The
// accumulator is double-buffered in TMEM (2 x 256 columns): while the epilogue reads buffer b of
// one accumulation, the MMAs of the next run into the other buffer.
//
// EXACT = false: one accumulation per unit; the epilogue writes FP32 C (beta = 1 adds to C).
// EXACT = true (bf16 operands holding small integers, see ozaki.cuh): the unit's K range is cut into
// accumulations of at most CH k-blocks (2048 products, whose FP32 sum is exact), and the epilogue
// adds each one, converted to int32, into per-thread integer registers; the unit writes int32 sums to
// C (as int) + z * split_stride. The caller bounds a unit to 255 accumulations, so |sum| < 2^31.
template <TcKind KIND, bool EXACT>
__global__ void __launch_bounds__(EXACT ? 320 : 192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, void* Cv,
                   long long ldc, long long M, long long N, int tiles_m, int tiles_n, int gm, int zs,
                   int nk_total, int nk_split, long long split_stride, int beta, int* err) {
  constexpr int KB_ELEMS = KIND == TcKind::BF16 ? 64 : 32;
  constexpr int MMA_K_BYTES = 32;                            // K = 16 bf16 or 8 tf32 per instruction
  constexpr int NEPI = EXACT ? 8 : 4;                        // epilogue warps
  constexpr int CH = 32;                                     // k-blocks per exact accumulation
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  // barriers: full[STAGES], empty[STAGES], accumulator full[2] and empty[2], and one that the MMA
  // issuer's final commit arrives on (all of its MMAs complete) before TMEM is released
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  __shared__ volatile int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = zs * tiles_m * tiles_n;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const uint32_t accf0 = smem_u32(bars + 2 * STAGES), acce0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t drain = smem_u32(bars + 2 * STAGES + 4);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int st = 0; st < STAGES; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, NEPI);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {   // TMA producer
      long long g = 0;  // k-blocks issued by this CTA
      for (int u = blockIdx.x; u < total && !s_fail; u += gridDim.x) {
        const Unit w = decode_unit(u, tiles_m, tiles_n, gm);
        const int kb0 = w.z * nk_split;
        const int nk = max(0, min(nk_total, kb0 + nk_split) - kb0);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int st = (int)(g % STAGES);
          const uint32_t ph = (uint32_t)((g / STAGES) & 1);
          if (!mbar_wait(empty0 + 8 * st, ph ^ 1)) { s_fail = 1; break; }
          mbar_expect_tx(full0 + 8 * st, STAGE_BYTES);
          tma_load_2d(smem_u32(sA + st * A_BYTES), &tmA, (kb0 + kb) * KB_ELEMS, w.mt * BM, full0 + 8 * st);
          tma_load_2d(smem_u32(sB + st * B_BYTES), &tmB, (kb0 + kb) * KB_ELEMS, w.nt * BN, full0 + 8 * st);
        }
      }
      // no copy may still be in flight when the CTA exits: wait (bounded) for the last stages issued
      for (long long i = (g > STAGES ? g - STAGES : 0); i < g; ++i)
        if (!mbar_wait(full0 + 8 * (int)(i % STAGES), (uint32_t)((i / STAGES) & 1))) s_fail = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      long long g = 0;  // k-blocks consumed
      int seg = 0;      // accumulations started (TMEM buffer = seg & 1)
      bool ok = true;
      for (int u = blockIdx.x; u < total && ok && !s_fail; u += gridDim.x) {
        const Unit w = decode_unit(u, tiles_m, tiles_n, gm);
        const int kb0 = w.z * nk_split;
        const int nk = max(0, min(nk_total, kb0 + nk_split) - kb0);
        const int nseg = nk == 0 ? 1 : (EXACT ? (nk + CH - 1) / CH : 1);
        for (int sgi = 0; sgi < nseg && ok; ++sgi, ++seg) {
          const int buf = seg & 1;
          if (seg >= 2 && !mbar_wait(acce0 + 8 * buf, (uint32_t)(((seg >> 1) - 1) & 1))) { ok = false; break; }
          tc_fence_after();
          const uint32_t tacc = taddr + (uint32_t)(buf * BN);
          const int k_lo = EXACT ? sgi * CH : 0;
          const int k_hi = EXACT ? min(nk, k_lo + CH) : nk;
          for (int kb = k_lo; kb < k_hi; ++kb, ++g) {
            const int st = (int)(g % STAGES);
            const uint32_t ph = (uint32_t)((g / STAGES) & 1);
            if (!mbar_wait(full0 + 8 * st, ph)) { ok = false; break; }
            tc_fence_after();
            const uint64_t ad = sdesc(smem_u32(sA + st * A_BYTES));
            const uint64_t bd = sdesc(smem_u32(sB + st * B_BYTES));
#pragma unroll
            for (int kk = 0; kk < KB_BYTES / MMA_K_BYTES; ++kk)
              mma<KIND>(tacc, ad + (uint64_t)(kk * MMA_K_BYTES >> 4), bd + (uint64_t)(kk * MMA_K_BYTES >> 4),
                        (kb > k_lo || kk > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * st);   // frees the stage once these MMAs have read it
          }
          if (!ok) break;
          mma_commit(accf0 + 8 * buf);     // accumulation complete (immediately for an empty K range)
        }
      }
      if (!ok) s_fail = 1;
      // When a wait gave up above, MMAs issued before it may still be running; the CTA must not free
      // TMEM under them. The commit arrives once every MMA this thread issued has completed (at once
      // if there are none); the wait for it is bounded like every other.
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) s_fail = 1;
    }
  } else {   // epilogue warps: TMEM lane quarter warp % 4; in EXACT mode two warps per quarter split N
    const int q = warp & 3;
    const int half = EXACT ? (warp - 2) / 4 : 0;
    constexpr int NCOL = EXACT ? BN / 2 : BN;   // columns per thread
    int seg = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
      const Unit w = decode_unit(u, tiles_m, tiles_n, gm);
      const int kb0 = w.z * nk_split;
      const int nk = max(0, min(nk_total, kb0 + nk_split) - kb0);
      const int nseg = nk == 0 ? 1 : (EXACT ? (nk + CH - 1) / CH : 1);
      const long long grow = (long long)w.mt * BM + q * 32 + lane;
      const long long gcol0 = (long long)w.nt * BN + half * NCOL;
      int iacc[EXACT ? NCOL : 1];
      if constexpr (EXACT) {
#pragma unroll
        for (int j = 0; j < NCOL; ++j) iacc[j] = 0;
      }
      for (int sgi = 0; sgi < nseg; ++sgi, ++seg) {
        const int buf = seg & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * buf, (uint32_t)((seg >> 1) & 1)) && !s_fail);
        if (!ok) break;
        tc_fence_after();
        const uint32_t trow = taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + half * NCOL);
        if constexpr (EXACT) {
#pragma unroll
          for (int ch = 0; ch < NCOL / 32; ++ch) {
            uint32_t r[32];
            tmem_ld32(trow + (uint32_t)(ch * 32), r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              // exact integer |v| < 2^23: add 1.5 * 2^23 and read the low mantissa bits
              const float v = nk == 0 ? 0.f : __uint_as_float(r[j]);
              iacc[ch * 32 + j] += __float_as_int(v + 12582912.0f) - 0x4B400000;
            }
          }
        } else {
          float* Cz = reinterpret_cast<float*>(Cv) + (long long)w.z * split_stride;
          const bool vec = (ldc % 4 == 0);
#pragma unroll 1
          for (int ch = 0; ch < NCOL / 32; ++ch) {
            uint32_t r[32];
            tmem_ld32(trow + (uint32_t)(ch * 32), r);
            const long long gcol = gcol0 + ch * 32;
            if (grow < M && gcol < N) {
              float* p = Cz + grow * ldc + gcol;
              if (vec && gcol + 32 <= N) {
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                  float4 v = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                         __uint_as_float(r[j + 3]));
                  if (nk == 0) v = make_float4(0.f, 0.f, 0.f, 0.f);
                  if (beta) {
                    float4 o = *reinterpret_cast<float4*>(p + j);
                    v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
                  }
                  *reinterpret_cast<float4*>(p + j) = v;
                }
              } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                  if (gcol + j < N) {
                    float v = nk == 0 ? 0.f : __uint_as_float(r[j]);
                    if (beta) v += p[j];
                    p[j] = v;
                  }
                }
              }
            }
          }
        }
        // this warp's reads of the buffer are complete (tcgen05.wait::ld in tmem_ld32): release it
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce0 + 8 * buf);
      }
      if constexpr (EXACT) {
        if (ok && grow < M) {
          int* Pz = reinterpret_cast<int*>(Cv) + (long long)w.z * split_stride + grow * ldc;
          if (ldc % 4 == 0 && gcol0 + NCOL <= N) {
#pragma unroll
            for (int j = 0; j < NCOL; j += 4)
              *reinterpret_cast<int4*>(Pz + gcol0 + j) = make_int4(iacc[j], iacc[j + 1], iacc[j + 2], iacc[j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < NCOL; ++j)
              if (gcol0 + j < N) Pz[gcol0 + j] = iacc[j];
          }
        }
      }
    }
    if (!ok && lane == 0) s_fail = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ---- host side ----------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    GFCC_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    GFCC_CHECK(q == cudaDriverEntryPointSuccess && p, GFCC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

CUtensorMap make_map(TcKind kind, const TcOperand& op, int box_rows) {
  CUtensorMap m;
  const int esize = kind == TcKind::BF16 ? 2 : 4;
  GFCC_CHECK(op.k_pad % (KB_BYTES / esize) == 0, GFCC_ERR_ARG, "tc_gemm: K not padded to the k-block");
  GFCC_CHECK((reinterpret_cast<uintptr_t>(op.ptr) & 15) == 0, GFCC_ERR_ARG, "tc_gemm: operand not 16-byte aligned");
  GFCC_CHECK(op.ld >= op.k_pad && op.ld % (KB_BYTES / esize) == 0, GFCC_ERR_ARG, "tc_gemm: bad row stride");
  cuuint64_t dims[2] = {(cuuint64_t)op.k_pad, (cuuint64_t)op.rows};
  cuuint64_t strides[1] = {(cuuint64_t)op.ld * esize};
  cuuint32_t box[2] = {(cuuint32_t)(KB_BYTES / esize), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, kind == TcKind::BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           2, const_cast<void*>(op.ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GFCC_CHECK(r == CUDA_SUCCESS, GFCC_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) GFCC_CUDA(cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev));
  return cached[dev];
}

// ---- autotuner of the M-tile group size ----------------------------------------------------------
// The group size gm (how many 128-row A tiles a group of work units shares while it runs through the N
// tiles) trades DRAM re-reads of B against L2 room; it changes the order of the work units, not their
// arithmetic, so every candidate writes the same result. On the first launch of a shape bucket that
// overwrites its output (beta = 0; not under stream capture) each distinct gm of the L2 budgets below
// is timed twice with CUDA events on the launching stream, and the fastest is kept for the process.
// GFCC_AUTOTUNE=0 keeps the default (40 MB) everywhere.
struct TuneKey {
  int kind, exact, tiles_m, tn_log2, nk_split, zs;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, exact, tiles_m, tn_log2, nk_split, zs) <
           std::tie(o.kind, o.exact, o.tiles_m, o.tn_log2, o.nk_split, o.zs);
  }
};
struct TuneResult {
  int gm = 1, gm_default = 1;
  float ms_best = 0.f, ms_default = 0.f;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune;
std::vector<TuneKey> g_tune_order;   // keys in the order they were tuned (for the report)
constexpr long long kGmBudgetMB[] = {16, 40, 64, 96, 128};
constexpr long long kGmDefaultMB = 40;

bool autotune_enabled() {
  static const int on = [] {
    const char* e = getenv("GFCC_AUTOTUNE");
    return (e && e[0] == '0') ? 0 : 1;
  }();
  return on != 0;
}
int gm_for_budget(long long budget_mb, long long a_tile_bytes, int tiles_m) {
  return (int)std::max<long long>(1, std::min<long long>(tiles_m, (budget_mb << 20) / std::max(a_tile_bytes, 1LL)));
}

template <TcKind K, bool EXACT>
void launch(const CUtensorMap& ma, const CUtensorMap& mb, void* C, long long ldc, long long M, long long N,
            int tiles_m, int tiles_n, int zs, int nk_total, int nk_split, long long split_stride, int beta, int* err,
            cudaStream_t s) {
  static bool attr[64] = {};   // function attributes belong to each device's context: set once per device
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  GFCC_CHECK(dev >= 0 && dev < 64, GFCC_ERR_ARG, "tc_gemm: device ordinal above 63");
  if (!attr[dev]) {
    GFCC_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<K, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr[dev] = true;
  }
  const long long units = (long long)zs * tiles_m * tiles_n;
  const int grid = (int)std::min<long long>(units, sm_count());
  auto run = [&](int gm) {
    tc_gemm_kernel<K, EXACT><<<grid, EXACT ? 320 : 192, SMEM_BYTES, s>>>(ma, mb, C, ldc, M, N, tiles_m, tiles_n, gm,
                                                                         zs, nk_total, nk_split, split_stride, beta,
                                                                         err);
    GFCC_LAUNCH_CHECK();
  };
  // M-tile group: by default the A tiles of one group (128 rows x the split's K) fit in about 40 MB of L2
  const long long a_tile_bytes = (long long)BM * nk_split * KB_BYTES;
  const int gm_default = gm_for_budget(kGmDefaultMB, a_tile_bytes, tiles_m);
  int gm = gm_default;
  std::vector<int> cand;
  for (long long mb : kGmBudgetMB) {
    const int g = gm_for_budget(mb, a_tile_bytes, tiles_m);
    if (std::find(cand.begin(), cand.end(), g) == cand.end()) cand.push_back(g);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (beta == 0 && cand.size() > 1 && autotune_enabled() && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone) {
    int tl = 0;
    while ((1 << tl) < tiles_n) ++tl;
    const TuneKey key{K == TcKind::BF16 ? 0 : 1, EXACT ? 1 : 0, tiles_m, tl, nk_split, zs};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      gm = it->second.gm;
    } else {
      std::vector<cudaEvent_t> ev(2 * cand.size());
      for (auto& e : ev) GFCC_CUDA(cudaEventCreate(&e));
      std::vector<float> best(cand.size(), 1e30f);
      for (int pass = 0; pass < 2; ++pass) {
        for (size_t q = 0; q < cand.size(); ++q) {
          const size_t i = pass == 0 ? q : cand.size() - 1 - q;   // second pass in reverse order
          GFCC_CUDA(cudaEventRecord(ev[2 * i], s));
          run(cand[i]);
          GFCC_CUDA(cudaEventRecord(ev[2 * i + 1], s));
        }
        GFCC_CUDA(cudaStreamSynchronize(s));
        for (size_t i = 0; i < cand.size(); ++i) {
          float ms = 0.f;
          GFCC_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
          best[i] = std::min(best[i], ms);
        }
      }
      for (auto& e : ev) cudaEventDestroy(e);
      size_t ib = 0;
      for (size_t i = 1; i < cand.size(); ++i)
        if (best[i] < best[ib]) ib = i;
      TuneResult r;
      r.gm = cand[ib];
      r.gm_default = gm_default;
      r.ms_best = best[ib];
      for (size_t i = 0; i < cand.size(); ++i)
        if (cand[i] == gm_default) r.ms_default = best[i];
      g_tune[key] = r;
      g_tune_order.push_back(key);
      return;   // the output already holds the product (every candidate computes the same)
    }
  }
  run(gm);
}

}  // namespace

void tc_gemm(TcKind kind, const TcOperand& A, const TcOperand& B, float* C, long long ldc, long long M, long long N,
             int beta, int ksplit, long long split_stride, int* err_dev, cudaStream_t s, int prof_class,
             long long k_alg) {
  if (M <= 0 || N <= 0) return;
  GFCC_CHECK(A.k_pad == B.k_pad, GFCC_ERR_ARG, "tc_gemm: K mismatch");
  GFCC_CHECK(A.rows >= M && B.rows >= N, GFCC_ERR_ARG, "tc_gemm: operand rows");
  GFCC_CHECK(ksplit >= 1 && (ksplit == 1 || beta == 0), GFCC_ERR_ARG, "tc_gemm: split-K needs beta = 0");
  GFCC_CHECK(A.rows < (1LL << 31) && B.rows < (1LL << 31), GFCC_ERR_ARG, "tc_gemm: too many rows");
  const int kb_elems = tc_kblock(kind);
  GFCC_CHECK(A.k_pad / kb_elems < (1LL << 30), GFCC_ERR_ARG, "tc_gemm: K too large");
  const int nk_total = (int)(A.k_pad / kb_elems);
  const int nk_split = (nk_total + ksplit - 1) / ksplit;
  const int zs = std::max(1, (nk_total + nk_split - 1) / nk_split);
  const long long tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  GFCC_CHECK(tiles_m * tiles_n * zs < (1LL << 31), GFCC_ERR_ARG, "tc_gemm: too many tiles");
  CUtensorMap ma = make_map(kind, A, BM);
  CUtensorMap mb = make_map(kind, B, BN);
  ProfScope prof(prof_class, 2.0 * (double)M * (double)N * (double)(k_alg > 0 ? k_alg : A.k_pad), s);
  if (kind == TcKind::BF16)
    launch<TcKind::BF16, false>(ma, mb, C, ldc, M, N, (int)tiles_m, (int)tiles_n, zs, nk_total, nk_split,
                                split_stride, beta, err_dev, s);
  else
    launch<TcKind::TF32, false>(ma, mb, C, ldc, M, N, (int)tiles_m, (int)tiles_n, zs, nk_total, nk_split,
                                split_stride, beta, err_dev, s);
}

int tc_gemm_exact(const TcOperand& A, const TcOperand& B, int* P, long long ldp, long long M, long long N, int zs,
                  long long split_stride, int* err_dev, cudaStream_t s, int prof_class) {
  if (M <= 0 || N <= 0) return 0;
  GFCC_CHECK(zs >= 1, GFCC_ERR_ARG, "tc_gemm_exact: zs < 1");
  GFCC_CHECK(A.k_pad == B.k_pad, GFCC_ERR_ARG, "tc_gemm_exact: K mismatch");
  GFCC_CHECK(A.rows >= M && B.rows >= N, GFCC_ERR_ARG, "tc_gemm_exact: operand rows");
  GFCC_CHECK(A.rows < (1LL << 31) && B.rows < (1LL << 31), GFCC_ERR_ARG, "tc_gemm_exact: too many rows");
  GFCC_CHECK(A.k_pad / 64 < (1LL << 30), GFCC_ERR_ARG, "tc_gemm_exact: K too large");
  const int nk_total = (int)(A.k_pad / 64);
  const int nk_split = std::max(1, (nk_total + zs - 1) / std::max(zs, 1));
  GFCC_CHECK(nk_split <= TC_EXACT_MAX_KB, GFCC_ERR_ARG, "tc_gemm_exact: split too long for exact int32 sums");
  const int z_eff = std::max(1, (nk_total + nk_split - 1) / nk_split);
  const long long tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  GFCC_CHECK(tiles_m * tiles_n * z_eff < (1LL << 31), GFCC_ERR_ARG, "tc_gemm_exact: too many tiles");
  CUtensorMap ma = make_map(TcKind::BF16, A, BM);
  CUtensorMap mb = make_map(TcKind::BF16, B, BN);
  ProfScope prof(prof_class, 2.0 * (double)M * (double)N * (double)A.k_pad, s);
  GFCC_CHECK(z_eff <= zs, GFCC_ERR_ARG, "tc_gemm_exact: split count");
  launch<TcKind::BF16, true>(ma, mb, P, ldp, M, N, (int)tiles_m, (int)tiles_n, z_eff, nk_total, nk_split,
                             split_stride, 0, err_dev, s);
  return z_eff;
}

int tc_exact_splits(long long M, long long N, long long k_pad) {
  const long long nk = k_pad / 64;
  const long long tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  long long zs = std::max<long long>(1, (sm_count() + tiles - 1) / tiles);   // about one wave of units
  zs = std::min<long long>(zs, std::max<long long>(1, nk / 32));              // at least 32 k-blocks per split
  zs = std::max<long long>(zs, (nk + TC_EXACT_MAX_KB - 1) / TC_EXACT_MAX_KB);
  return (int)zs;
}

}  // namespace gfcc

extern "C" int gfcc_autotune_info(int i, int* kind, int* exact, int* tiles_m, int* tiles_n_log2, int* gm, int* gm_default,
                                  double* ms_best, double* ms_default) {
  std::lock_guard<std::mutex> lk(gfcc::g_tune_mu);
  if (i < 0 || i >= (int)gfcc::g_tune_order.size()) return GFCC_ERR_ARG;
  const gfcc::TuneKey& k = gfcc::g_tune_order[i];
  const gfcc::TuneResult& r = gfcc::g_tune[k];
  if (kind) *kind = k.kind == 0 ? GFCC_PREC_BF16 : GFCC_PREC_TF32;
  if (exact) *exact = k.exact;
  if (tiles_m) *tiles_m = k.tiles_m;
  if (tiles_n_log2) *tiles_n_log2 = k.tn_log2;
  if (gm) *gm = r.gm;
  if (gm_default) *gm_default = r.gm_default;
  if (ms_best) *ms_best = r.ms_best;
  if (ms_default) *ms_default = r.ms_default;
  return GFCC_OK;
}
