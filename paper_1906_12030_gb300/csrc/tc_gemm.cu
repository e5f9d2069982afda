// Tensor-core GEMM for sm_103a: TMA -> shared memory (128-byte swizzle,
// K-major) -> tcgen05.mma (FP32 accumulator in tensor memory) -> scattered
// epilogue that writes the next contraction's operand layout directly.
//
// Persistent kernel: each CTA walks output tiles (128 x BN) t = blockIdx.x,
// blockIdx.x + gridDim.x, ...  Tensor memory holds two accumulators, so the
// epilogue of one tile overlaps the MMAs of the next.  Warp roles:
//   warp 0      TMA producer (one elected lane), STAGES-deep ring shared by
//               all of the CTA's tiles
//   warp 1      tensor-memory allocator + MMA issuer (one lane)
//   warps 2..17 epilogue: tcgen05.ld of the accumulator, convert, store; four
//               warps per tensor-memory lane quarter, each taking a quarter of
//               the tile's columns; the accumulator is handed back to the MMA
//               warp after the last load of all sixteen.  At short K the
//               epilogue, not the MMA, sets the pace, so it is written for
//               few instructions per element: paired conversions and 32-bit
//               column offsets when the destination allows them
// Every mbarrier wait is bounded; a wait that gives up records
// MERA_ETIMEOUT in a device status word, raises a CTA-wide abort flag, and
// every role drains its copies in flight and leaves.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "../../include/mera.h"
#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace mera {

__device__ int g_device_status = 0;

namespace {

constexpr int kBM = 128;          // UMMA M (cta_group::1)
constexpr int kStageBudget = 192 * 1024;  // shared memory for the operand ring
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;
constexpr uint64_t kTimeoutNs = 2000000000ull;  // a wait longer than 2 s is a failure
constexpr uint32_t kSpinCap = 1u << 30;            // second bound, independent of the timer

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on the phase with the given parity.  Gives up (false) when
// the CTA's abort flag is raised or after kTimeoutNs; a timeout raises the
// flag and records MERA_ETIMEOUT.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1; i < kSpinCap; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > kTimeoutNs) break;
    }
  }
  atomicOr(&g_device_status, 1 << MERA_ETIMEOUT);
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, both K-major.
template <int PREC>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (PREC == PREC_TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
  }
}

// Shared-memory matrix descriptor: K-major, SLAB-byte swizzle (128 or 64),
// 8-row groups 8 * SLAB bytes apart (start address and offsets in 16-byte
// units).  A K step inside the swizzled row advances the start address.
template <int SLAB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  static_assert(SLAB == 128 || SLAB == 64, "swizzle span");
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t(1) << 16;                  // leading-dimension offset (unused for these layouts)
  d |= uint64_t((8 * SLAB) >> 4) << 32;    // stride-dimension offset
  d |= uint64_t(1) << 46;                  // descriptor version
  d |= uint64_t(SLAB == 128 ? 2 : 4) << 61;  // 128-byte / 64-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M x N.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Operand tensor maps, one per plane (hi, lo / hi, mid, lo for split modes).
constexpr int kMaxPlanes = 4;
struct TMaps {
  CUtensorMap a[kMaxPlanes];
  CUtensorMap b[kMaxPlanes];
};

struct Epilogue {
  int64_t M, N, K;
  void* C;
  int64_t c_plane;  // elements between hi and lo planes (BF16X3 operand)
  LegMap m_dst, n_dst;
  double alpha;
  int accumulate;
  int c_final;      // 1: FP64 output of the caller
  int split;        // K split: work item t covers output tile t % tiles and k-range t / tiles
  int kc;           // k-blocks per split
  float* partial;   // split > 1: raw FP32 partials [split][N][M], summed by splitk_reduce_kernel
  int64_t p_plane;  // fixed-point split modes: floats from the hi to the lo plane of the partials
  int off32;        // every column offset n_dst(n) is below 2^31
  int alpha_exp;    // alpha == 2^alpha_exp exactly (alpha_pow2 set)
  int alpha_pow2;
  int group_m;      // tile order: groups of this many row tiles, every column tile of a group in turn
};

// Output tile (row tile, column tile) of the mn-th tile in the kernels' walk
// order.  Tiles are taken in groups of group_m row tiles; within a group the
// column tile changes slowest, so one column tile of B meets group_m row
// tiles of A while both are in L2, and the group's A rows (sized by the host
// to a fraction of L2) stay resident across the group's column tiles.
__device__ __forceinline__ void tile_of(int64_t mn, int64_t tiles_m, int64_t tiles_n, int group_m, int64_t& tm,
                                        int64_t& tn) {
  const int64_t per_group = int64_t(group_m) * tiles_n;
  const int64_t g = mn / per_group, r = mn - g * per_group;
  const int64_t rows = min(int64_t(group_m), tiles_m - g * group_m);  // row tiles in this group
  tn = r / rows;
  tm = g * group_m + (r - tn * rows);
}

// binary32 -> binary64 times 2^e by integer operations, exact for every
// class of input (zero, subnormal, normal, infinity, NaN; e must keep a
// normal result in range).  The FP64 pipe of this GPU runs at a small
// fraction of its FP32 rate, so a conversion and a multiply per element in
// FP64 made the caller-format epilogue several times slower than its stores.
__device__ __forceinline__ double f32_to_f64_pow2(float f, int e) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xFFu, mant = u & 0x7FFFFFu;
  uint64_t bits = uint64_t(u & 0x80000000u) << 32;  // sign; zero stays a signed zero
  if (ex == 0xFFu) {
    bits |= (uint64_t(0x7FFu) << 52) | (uint64_t(mant) << 29);  // infinity, NaN
  } else if (ex != 0u) {  // normal: rebias the exponent, widen the fraction
    bits |= (uint64_t(ex + (1023u - 127u) + uint32_t(e)) << 52) | (uint64_t(mant) << 29);
  } else if (mant != 0u) {  // subnormal: mant * 2^-149 = 2^(p - 149) * (mant / 2^p), p = msb of mant
    const int p = 31 - __clz(mant);
    bits |= (uint64_t(p - 149 + 1023 + e) << 52) | ((uint64_t(mant) - (uint64_t(1) << p)) << (52 - p));
  }
  return __longlong_as_double(static_cast<long long>(bits));
}

// Stages hold 128-byte slabs (64 BF16 or 32 TF32 along K) of every plane.
// (64-byte slabs, which fit twice as many stages for the split-BF16 modes,
// measured 2-5 % slower on the chi = 16 and chi = 32 contractions.)
template <int PREC, int BN>
struct Cfg {
  static constexpr int kElem = (PREC == PREC_TF32) ? 4 : 2;
  static constexpr int kPlanes = (PREC == PREC_BF16X3) ? 2 : (PREC == PREC_BF16X6 ? 3 : 1);
  static constexpr int kSlab = 128;                         // swizzle span = bytes along K per stage
  static constexpr int kBK = kSlab / kElem;                 // K per stage
  static constexpr int kABytes = kBM * kSlab;               // one plane of A
  static constexpr int kBBytes = BN * kSlab;
  static constexpr int kStageBytes = kPlanes * (kABytes + kBBytes);
  static constexpr int kStages = kStageBudget / kStageBytes > 8 ? 8
                                 : (kStageBudget / kStageBytes < 2 ? 2 : kStageBudget / kStageBytes);
  static constexpr int kAccCols = BN < 32 ? 32 : BN;     // one accumulator
  // column distance of the two (double-buffered) accumulators: a power of
  // two, as the allocation must be (160 and 192 wide tiles use 256)
  static constexpr int kAccStride = kAccCols <= 32 ? 32 : kAccCols <= 64 ? 64 : kAccCols <= 128 ? 128 : 256;
  static constexpr int kTmemCols = 2 * kAccStride;
  static constexpr uint32_t kFmt = (PREC == PREC_TF32) ? 2u : 1u;  // TF32 / BF16
  static constexpr size_t kSmem = 1024 + size_t(kStages) * kStageBytes + 1024 + BN * (sizeof(int64_t) + sizeof(int));
};

// One row's 32 accumulator values -> operand-format stores at row offset
// off_m plus the 32-bit column offsets s_off[j] in shared memory (hi, lo /
// hi, mid, lo planes
// c_plane elements apart).  Conversions run on pairs (cvt.rn.bf16x2.f32);
// each value is rounded exactly as the per-element path rounds it.
template <int PREC>
__device__ __forceinline__ void store_chunk(void* C, int64_t off_m, int64_t c_plane, const int* __restrict__ s_off,
                                            const uint32_t (&v)[32]) {
  if constexpr (PREC == PREC_TF32) {
    float* r = static_cast<float*>(C) + off_m;
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      const int4 q = *reinterpret_cast<const int4*>(s_off + j);
      r[q.x] = round_tf32(__uint_as_float(v[j]));
      r[q.y] = round_tf32(__uint_as_float(v[j + 1]));
      r[q.z] = round_tf32(__uint_as_float(v[j + 2]));
      r[q.w] = round_tf32(__uint_as_float(v[j + 3]));
    }
  } else {
    __nv_bfloat16* __restrict__ r0 = static_cast<__nv_bfloat16*>(C) + off_m;
    __nv_bfloat16* __restrict__ r1 = r0 + c_plane;
    __nv_bfloat16* __restrict__ r2 = r1 + c_plane;
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const int2 q = *reinterpret_cast<const int2*>(s_off + j);
      const int o[2] = {q.x, q.y};
      const float f0 = __uint_as_float(v[j]), f1 = __uint_as_float(v[j + 1]);
      const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
      r0[o[0]] = h.x;
      r0[o[1]] = h.y;
      if constexpr (PREC == PREC_BF16X3 || PREC == PREC_BF16X6) {
        const float2 hf = __bfloat1622float2(h);
        const float e0 = f0 - hf.x, e1 = f1 - hf.y;
        const __nv_bfloat162 l = __floats2bfloat162_rn(e0, e1);
        r1[o[0]] = l.x;
        r1[o[1]] = l.y;
        if constexpr (PREC == PREC_BF16X6) {
          const float2 lf = __bfloat1622float2(l);
          const __nv_bfloat162 q = __floats2bfloat162_rn(e0 - lf.x, e1 - lf.y);
          r2[o[0]] = q.x;
          r2[o[1]] = q.y;
        }
      }
    }
  }
}

template <int PREC, int BN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ TMaps tm, const __grid_constant__ Epilogue ep) {
  using C = Cfg<PREC, BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint8_t* aux = smem + size_t(C::kStages) * C::kStageBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(aux);
  uint64_t* empty = full + C::kStages;
  uint64_t* acc_full = empty + C::kStages;   // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;        // [2] epilogue -> MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* abort_snapshot = abort_flag + 1;
  volatile int* never = abort_flag + 2;  // stays 0: waits that must not be cut short
  int64_t* off_n = reinterpret_cast<int64_t*>(aux + 1024);
  int* off_n32 = reinterpret_cast<int*>(off_n + BN);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t tiles_n = (ep.N + BN - 1) / BN;
  const int64_t tiles_mn = ((ep.M + kBM - 1) / kBM) * tiles_n;
  const int64_t tiles = tiles_mn * ep.split;
  const int num_k = int((ep.K + C::kBK - 1) / C::kBK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);  // one arrive per epilogue warp
    }
    *abort_flag = 0;
    *abort_snapshot = 0;
    *never = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(uint32_t(C::kTmemCols))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer ---------------------------------------------------------
      uint32_t it = 0;
      bool alive = true;
      for (int64_t t = blockIdx.x; t < tiles && alive; t += gridDim.x) {
        int64_t row_t, col_t;
        tile_of(t % tiles_mn, tiles_mn / tiles_n, tiles_n, ep.group_m, row_t, col_t);
        const int m0 = int(row_t * kBM), n0 = int(col_t * BN);
        const int kb0 = int(t / tiles_mn) * ep.kc, kb1 = min(kb0 + ep.kc, num_k);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const uint32_t s = it % C::kStages;
          if (it >= uint32_t(C::kStages) && !mbar_wait(&empty[s], ((it / C::kStages) & 1) ^ 1, abort_flag)) {
            alive = false;
            break;
          }
          uint8_t* st = stage_base + size_t(s) * C::kStageBytes;
          mbar_arrive_expect_tx(&full[s], C::kStageBytes);
          const int x = kb * C::kBK;
#pragma unroll
          for (int pl = 0; pl < C::kPlanes; ++pl) {  // plane pl: A then B
            uint8_t* dst = st + pl * (C::kABytes + C::kBBytes);
            tma_load_2d(dst, &tm.a[pl], x, m0, &full[s]);
            tma_load_2d(dst + C::kABytes, &tm.b[pl], x, n0, &full[s]);
          }
        }
      }
      // drain: every issued stage must have landed before the CTA may exit
      for (uint32_t j = (it > uint32_t(C::kStages) ? it - C::kStages : 0); j < it; ++j)
        mbar_wait(&full[j % C::kStages], (j / C::kStages) & 1, never);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer -------------------------------------------------------
      constexpr uint32_t idesc = make_idesc(C::kFmt, kBM, BN < 16 ? 16 : BN);
      uint32_t it = 0, tc = 0;
      bool alive = true;
      for (int64_t t = blockIdx.x; t < tiles && alive; t += gridDim.x, ++tc) {
        const uint32_t b = tc & 1;
        if (tc >= 2 && !mbar_wait(&acc_empty[b], ((tc >> 1) - 1) & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t d = tmem + b * uint32_t(C::kAccStride);
        const int kb0 = int(t / tiles_mn) * ep.kc, kb1 = min(kb0 + ep.kc, num_k);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const uint32_t s = it % C::kStages;
          if (!mbar_wait(&full[s], (it / C::kStages) & 1, abort_flag)) {
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t s0 = smem_u32(stage_base + size_t(s) * C::kStageBytes);
          constexpr uint32_t kPlaneStride = C::kABytes + C::kBBytes;
#pragma unroll
          for (int k = 0; k < C::kSlab / 32; ++k) {
            const uint32_t koff = uint32_t(k * 32);
            // products of A plane pa and B plane pb with pa + pb < planes:
            // (0,0) | (0,0) (0,1) (1,0) | (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
#pragma unroll
            for (int pa = 0; pa < C::kPlanes; ++pa) {
#pragma unroll
              for (int pb = 0; pb + pa < C::kPlanes; ++pb) {
                const uint32_t a_addr = s0 + pa * kPlaneStride + koff;
                const uint32_t b_addr = s0 + pb * kPlaneStride + C::kABytes + koff;
                const uint32_t acc = (kb > kb0 || k > 0 || pa > 0 || pb > 0) ? 1u : 0u;
                tc_mma<PREC>(d, smem_desc<C::kSlab>(a_addr), smem_desc<C::kSlab>(b_addr), idesc, acc);
              }
            }
          }
          tc_commit(&empty[s]);
        }
        tc_commit(&acc_full[b]);  // also fires after an abort, so nobody waits on it forever
      }
    }
  } else {
    // ---- epilogue (warps 2..17) ------------------------------------------------
    const int et = threadIdx.x - 64;  // 0..kEpiThreads-1
    const int quarter = warp % 4;     // tensor-memory lanes this warp may read
    const int sub = (warp - 2) / 4;   // which quarter of the tile's 32-column chunks
    constexpr int kSub = kEpiWarps / 4;
    const int row = quarter * 32 + lane;
    constexpr int kChunks = BN < 32 ? 1 : BN / 32;
    const int ch_lo = (sub * kChunks) / kSub, ch_hi = ((sub + 1) * kChunks) / kSub;
    const float alpha = float(ep.alpha);
    const bool fast_ok = !ep.c_final && ep.split <= 1 && ep.off32 && ep.alpha == 1.0;
    const bool final_fast = ep.c_final && ep.split <= 1 && ep.off32 && ep.alpha_pow2;
    uint32_t tc = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++tc) {
      const int64_t ks = t / tiles_mn;
      int64_t row_t, col_t;
      tile_of(t % tiles_mn, tiles_mn / tiles_n, tiles_n, ep.group_m, row_t, col_t);
      const int64_t m0 = row_t * kBM, n0 = col_t * BN;
      const uint32_t b = tc & 1;
      // all epilogue threads are done with the previous tile's offsets;
      // decide together whether to go on
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
      if (et == 0) *abort_snapshot = *abort_flag;
      for (int c = et; c < BN; c += kEpiThreads) {
        const int64_t n = n0 + c;
        const int64_t o = n < ep.N ? legmap_offset32(ep.n_dst, uint32_t(n)) : 0;
        off_n[c] = o;
        off_n32[c] = int(o);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
      if (*abort_snapshot) break;
      const int64_t m = m0 + row;
      const bool row_ok = m < ep.M;
      const int64_t off_m = row_ok ? legmap_offset32(ep.m_dst, uint32_t(m)) : 0;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (tc >> 1) & 1, abort_flag) ? 1 : 0);
      tc_fence_after();
      if (!ok) continue;  // the next snapshot sees the abort flag
      const uint32_t taddr = tmem + b * uint32_t(C::kAccStride) + (uint32_t(quarter * 32) << 16);
      if (ch_lo >= ch_hi) {  // no columns for this warp: hand the accumulator back at once
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
        continue;
      }
#pragma unroll 1
      for (int ch = ch_lo; ch < ch_hi; ++ch) {
        const int c0 = ch * 32;
        uint32_t v[32];
        tmem_ld32(taddr + uint32_t(c0), v);
        if (ch + 1 == ch_hi) {  // this warp's last read of the accumulator: hand it back
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        if (!row_ok) continue;
        if (ep.split > 1) {  // raw partial sums, reduced afterwards (splitk_reduce_kernel)
          float* p = ep.partial + (ks * ep.N + n0 + c0) * ep.M + m;
#pragma unroll
          for (int j = 0; j < 32; ++j, p += ep.M)
            if (c0 + j < BN && n0 + c0 + j < ep.N) *p = __uint_as_float(v[j]);
          continue;
        }
        if (fast_ok && c0 + 32 <= BN && n0 + c0 + 32 <= ep.N) {
          // whole chunk, operand-format destination, offsets in 32 bits
          store_chunk<PREC>(ep.C, off_m, ep.c_plane, off_n32 + c0, v);
          continue;
        }
        if (final_fast && c0 + 32 <= BN && n0 + c0 + 32 <= ep.N) {
          // whole chunk into the caller's binary64 output, alpha a power of two
          double* __restrict__ r = static_cast<double*>(ep.C) + off_m;
          const int* __restrict__ so = off_n32 + c0;
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            // four offsets in registers before the four stores
            const int4 q4 = *reinterpret_cast<const int4*>(so + j);
            const int o[4] = {q4.x, q4.y, q4.z, q4.w};
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = f32_to_f64_pow2(__uint_as_float(v[j + q]), ep.alpha_exp);
            if (ep.accumulate) {
              double y[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) y[q] = r[o[q]];
#pragma unroll
              for (int q = 0; q < 4; ++q) r[o[q]] = y[q] + x[q];
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q) r[o[q]] = x[q];
            }
          }
          continue;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = c0 + j;
          if (c >= BN || n0 + c >= ep.N) continue;
          const int64_t off = off_m + off_n[c];
          if (ep.c_final) {
            double* dst = static_cast<double*>(ep.C) + off;
            const double val = ep.alpha * double(__uint_as_float(v[j]));
            *dst = ep.accumulate ? (*dst + val) : val;
          } else {
            const float val = alpha * __uint_as_float(v[j]);
            if constexpr (PREC == PREC_TF32) {
              static_cast<float*>(ep.C)[off] = round_tf32(val);
            } else if constexpr (PREC == PREC_BF16) {
              static_cast<__nv_bfloat16*>(ep.C)[off] = __float2bfloat16_rn(val);
            } else if constexpr (PREC == PREC_BF16X3) {
              const __nv_bfloat16 hi = __float2bfloat16_rn(val);
              const __nv_bfloat16 lo = __float2bfloat16_rn(val - __bfloat162float(hi));
              static_cast<__nv_bfloat16*>(ep.C)[off] = hi;
              static_cast<__nv_bfloat16*>(ep.C)[off + ep.c_plane] = lo;
            } else {
              const __nv_bfloat16 hi = __float2bfloat16_rn(val);
              const float r1 = val - __bfloat162float(hi);
              const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
              const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
              __nv_bfloat16* c = static_cast<__nv_bfloat16*>(ep.C);
              c[off] = hi;
              c[off + ep.c_plane] = mid;
              c[off + 2 * ep.c_plane] = lo;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(uint32_t(C::kTmemCols))
                 : "memory");
  }
}

// Sum of the K-split partials in a fixed order, then the same epilogue as
// the GEMM.  The sum is kept as an unevaluated pair hi + lo of binary32
// values (Knuth's TwoSum per partial), which carries ~48 significant bits
// like a binary64 sum but runs on the FP32 pipe.  One thread per row m,
// looping over a chunk of columns.
template <int PREC>
__global__ void __launch_bounds__(256) splitk_reduce_kernel(const __grid_constant__ Epilogue ep) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= ep.M) return;
  const int64_t off_m = legmap_offset32(ep.m_dst, uint32_t(m));
  const int64_t n_per = (ep.N + gridDim.y - 1) / gridDim.y;
  const int64_t n_lo = int64_t(blockIdx.y) * n_per, n_hi = min(ep.N, n_lo + n_per);
  for (int64_t n = n_lo; n < n_hi; ++n) {
    float hi = 0.0f, lo = 0.0f;
    for (int s = 0; s < ep.split; ++s) {
      const float x = ep.partial[(int64_t(s) * ep.N + n) * ep.M + m];
      const float t = __fadd_rn(hi, x);
      const float xp = __fsub_rn(t, hi);
      lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, xp)), __fsub_rn(x, xp)));
      hi = t;
    }
    const int64_t off = off_m + legmap_offset32(ep.n_dst, uint32_t(n));
    if (ep.c_final) {
      double* dst = static_cast<double*>(ep.C) + off;
      const double val = ep.alpha_pow2 ? f32_to_f64_pow2(hi, ep.alpha_exp) + f32_to_f64_pow2(lo, ep.alpha_exp)
                                       : ep.alpha * (double(hi) + double(lo));
      *dst = ep.accumulate ? (*dst + val) : val;
    } else {
      OperandStore<PREC>::store_f(ep.C, off, ep.c_plane, __fmul_rn(float(ep.alpha), __fadd_rn(hi, lo)));
    }
  }
}

#include "oz_gemm.cuh"

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D K-major operand: rows x K, row pitch ld elements, box (slab, box_rows).
bool encode_operand(CUtensorMap* tm, const void* base, int prec, int64_t rows, int64_t K, int64_t ld, int box_rows,
                    int slab) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int elem = (prec == PREC_TF32) ? 4 : 2;
  const CUtensorMapDataType dt = (prec == PREC_TF32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(ld) * elem};
  cuuint32_t box[2] = {cuuint32_t(slab / elem), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  slab == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Row tiles per group of the tile walk (tile_of): as many as keep the
// group's A rows within 32 MB (a quarter of L2), at least one.
int group_rows(const TcGemmArgs& a, int64_t a_row_bytes) {
  const int64_t tile_bytes = int64_t(kBM) * a_row_bytes;
  const int64_t tiles_m = (a.M + kBM - 1) / kBM;
  const int64_t g = std::max<int64_t>(1, (int64_t(32) << 20) / std::max<int64_t>(1, tile_bytes));
  return int(std::min<int64_t>(g, tiles_m));
}

template <int PREC, int BN>
cudaError_t launch_cfg(const TcGemmArgs& a, cudaStream_t stream) {
  using C = Cfg<PREC, BN>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(tc_gemm_kernel<PREC, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(C::kSmem));
  });
  if (attr_err != cudaSuccess) return attr_err;
  TMaps tm;
  const char* A = static_cast<const char*>(a.A);
  const char* B = static_cast<const char*>(a.B);
  for (int pl = 0; pl < kMaxPlanes; ++pl) {
    const int q = pl < C::kPlanes ? pl : 0;  // unused slots repeat plane 0
    if (!encode_operand(&tm.a[pl], A + q * a.a_plane_bytes, PREC, a.M, a.K, a.lda, kBM, C::kSlab))
      return cudaErrorInvalidValue;
    if (!encode_operand(&tm.b[pl], B + q * a.b_plane_bytes, PREC, a.N, a.K, a.ldb, BN, C::kSlab))
      return cudaErrorInvalidValue;
  }
  Epilogue ep;
  ep.M = a.M;
  ep.N = a.N;
  ep.K = a.K;
  ep.C = a.C;
  ep.c_plane = a.c_plane_elems;
  ep.m_dst = a.m_dst;
  ep.n_dst = a.n_dst;
  ep.alpha = a.alpha;
  {
    int e2 = 0;
    const double fr = std::frexp(a.alpha, &e2);  // alpha = fr * 2^e2, fr in [0.5, 1)
    ep.alpha_pow2 = (fr == 0.5) ? 1 : 0;
    ep.alpha_exp = e2 - 1;
  }
  ep.accumulate = a.accumulate;
  ep.c_final = a.c_final ? 1 : 0;
  const int64_t num_k = (a.K + C::kBK - 1) / C::kBK;
  const int split = a.split > 1 && a.partial ? a.split : 1;
  ep.split = split;
  ep.kc = int((num_k + split - 1) / split);
  ep.partial = a.partial;
  ep.p_plane = 0;
  {
    // largest column offset, to allow 32-bit column offsets (the row
    // offset stays 64-bit)
    int64_t hi = 0;
    for (int i = 0; i < a.n_dst.n; ++i) hi += (a.n_dst.dim[i] - 1) * a.n_dst.stride[i];
    ep.off32 = hi < (int64_t(1) << 31) ? 1 : 0;
  }
  ep.group_m = group_rows(a, a.K * C::kElem * C::kPlanes);
  if (split > 1 && (int64_t(split - 1) * ep.kc >= num_k)) return cudaErrorInvalidValue;  // empty split
  const int64_t tiles = ((a.M + kBM - 1) / kBM) * ((a.N + BN - 1) / BN) * split;
  if (tiles <= 0) return cudaErrorInvalidValue;
  static int resident = 0;  // CTAs of this configuration the whole GPU holds at once
  static std::once_flag occ_once;
  std::call_once(occ_once, [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_gemm_kernel<PREC, BN>, kThreads, C::kSmem);
    resident = std::max(1, sms) * std::max(1, per_sm);
  });
  const unsigned grid = unsigned(std::min<int64_t>(tiles, resident));
  count_launch();
  tc_gemm_kernel<PREC, BN><<<grid, kThreads, C::kSmem, stream>>>(tm, ep);
  if (split > 1) {
    const unsigned gx = unsigned((a.M + 255) / 256);
    const unsigned gy = unsigned(std::min<int64_t>(a.N, std::max<int64_t>(1, 4 * 152 / int64_t(gx))));
    count_launch();
    splitk_reduce_kernel<PREC><<<dim3(gx, gy), 256, 0, stream>>>(ep);
  }
  return cudaGetLastError();
}

// Shared by both launchers: the epilogue's destination description.
void fill_epilogue(const TcGemmArgs& a, Epilogue& ep) {
  ep.M = a.M;
  ep.N = a.N;
  ep.K = a.K;
  ep.C = a.C;
  ep.c_plane = a.c_plane_elems;
  ep.m_dst = a.m_dst;
  ep.n_dst = a.n_dst;
  ep.alpha = a.alpha;
  int e2 = 0;
  const double fr = std::frexp(a.alpha, &e2);  // alpha = fr * 2^e2, fr in [0.5, 1)
  ep.alpha_pow2 = (fr == 0.5) ? 1 : 0;
  ep.alpha_exp = e2 - 1;
  ep.accumulate = a.accumulate;
  ep.c_final = a.c_final ? 1 : 0;
  int64_t hi = 0;  // largest column offset: 32-bit column offsets allowed below 2^31
  for (int i = 0; i < a.n_dst.n; ++i) hi += (a.n_dst.dim[i] - 1) * a.n_dst.stride[i];
  ep.off32 = hi < (int64_t(1) << 31) ? 1 : 0;
}


// Fixed-point split modes: S slice planes per operand, K split in whole
// blocks of kOzBlockK.
template <int S, int BN>
cudaError_t launch_oz(const TcGemmArgs& a, cudaStream_t stream) {
  using C = OzCfg<S, BN>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(oz_gemm_kernel<S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::kSmem));
  });
  if (attr_err != cudaSuccess) return attr_err;
  TMaps tm;
  const char* A = static_cast<const char*>(a.A);
  const char* B = static_cast<const char*>(a.B);
  for (int pl = 0; pl < kMaxPlanes; ++pl) {
    const int q = pl < S ? pl : 0;
    if (!encode_operand(&tm.a[pl], A + q * a.a_plane_bytes, PREC_BF16, a.M, a.K, a.lda, kBM, C::kSlab))
      return cudaErrorInvalidValue;
    if (!encode_operand(&tm.b[pl], B + q * a.b_plane_bytes, PREC_BF16, a.N, a.K, a.ldb, BN, C::kSlab))
      return cudaErrorInvalidValue;
  }
  Epilogue ep;
  fill_epilogue(a, ep);
  ep.group_m = group_rows(a, a.K * 2 * S);
  const int64_t num_k = (a.K + C::kBK - 1) / C::kBK;
  const int64_t nblk = (a.K + kOzBlockK - 1) / kOzBlockK;
  const int split = a.split > 1 && a.partial ? a.split : 1;
  const int64_t per = (nblk + split - 1) / split;  // blocks per split
  ep.split = split;
  ep.kc = int(per * C::kBlockStages);
  ep.partial = a.partial;
  ep.p_plane = a.partial_plane;
  if (split > 1 && ((split - 1) * per >= nblk || a.partial_plane < int64_t(split) * a.N * a.M))
    return cudaErrorInvalidValue;  // an empty split, or lo partials overlapping hi
  if (num_k <= 0) return cudaErrorInvalidValue;
  const int64_t tiles = ((a.M + kBM - 1) / kBM) * ((a.N + BN - 1) / BN) * split;
  static int resident = 0;
  static std::once_flag occ_once;
  std::call_once(occ_once, [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oz_gemm_kernel<S, BN>, kOzThreads, C::kSmem);
    resident = std::max(1, sms) * std::max(1, per_sm);
  });
  const unsigned grid = unsigned(std::min<int64_t>(tiles, resident));
  count_launch();
  oz_gemm_kernel<S, BN><<<grid, kOzThreads, C::kSmem, stream>>>(tm, ep);
  if (split > 1) {
    const unsigned gx = unsigned((a.M + 255) / 256);
    const unsigned gy = unsigned(std::min<int64_t>(a.N, std::max<int64_t>(1, 4 * 152 / int64_t(gx))));
    count_launch();
    oz_splitk_reduce_kernel<<<dim3(gx, gy), 256, 0, stream>>>(ep);
  }
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_oz_prec(const TcGemmArgs& a, cudaStream_t stream) {
  const int bn = a.bn > 0 ? a.bn : (a.N > 64 ? 128 : (a.N > 16 ? 64 : 16));
  switch (bn) {
    case 128: return launch_oz<S, 128>(a, stream);
    case 64: return launch_oz<S, 64>(a, stream);
    case 16: return launch_oz<S, 16>(a, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int PREC>
cudaError_t launch_prec(const TcGemmArgs& a, cudaStream_t stream) {
  switch (a.bn) {  // a width chosen by the planner (heuristic or autotuned)
    case 0: break;
    case 256:
      if constexpr (PREC == PREC_BF16X6) return cudaErrorInvalidValue;  // one stage only
      else return launch_cfg<PREC, 256>(a, stream);
    case 192:  // N = 576 (chi = 24) in three full tiles
      if constexpr (PREC == PREC_BF16X6) return cudaErrorInvalidValue;
      else return launch_cfg<PREC, 192>(a, stream);
    case 160:
      if constexpr (PREC == PREC_BF16X6) return cudaErrorInvalidValue;
      else return launch_cfg<PREC, 160>(a, stream);
    case 128: return launch_cfg<PREC, 128>(a, stream);
    case 64: return launch_cfg<PREC, 64>(a, stream);
    case 16: return launch_cfg<PREC, 16>(a, stream);
    default: return cudaErrorInvalidValue;
  }
  // three-plane operands: a 256-wide B tile leaves room for one stage only
  if (a.N > 128 && PREC != PREC_BF16X6) return launch_cfg<PREC, (PREC == PREC_BF16X6 ? 128 : 256)>(a, stream);
  if (a.N > 64) return launch_cfg<PREC, 128>(a, stream);
  if (a.N > 16) return launch_cfg<PREC, 64>(a, stream);  // (a 32-wide variant spilled registers)
  return launch_cfg<PREC, 16>(a, stream);
}

}  // namespace

cudaError_t launch_gemm_tc(const TcGemmArgs& a, cudaStream_t stream) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaErrorInvalidValue;
  if (a.M > 0x7fffffff || a.N > 0x7fffffff || a.K > 0x7fffffff) return cudaErrorInvalidValue;
  switch (a.prec) {
    case PREC_TF32: return launch_prec<PREC_TF32>(a, stream);
    case PREC_BF16: return launch_prec<PREC_BF16>(a, stream);
    case PREC_BF16X3: return launch_prec<PREC_BF16X3>(a, stream);
    case PREC_BF16X6: return launch_prec<PREC_BF16X6>(a, stream);
    case PREC_OZ3: return launch_oz_prec<3>(a, stream);
    case PREC_OZ4: return launch_oz_prec<4>(a, stream);
    default: return cudaErrorNotSupported;
  }
}

__global__ void report_notconv_kernel(const int* state) {
  if (state[0] == 0) atomicOr(&g_device_status, 1 << MERA_ENOTCONV);
}

cudaError_t launch_report_notconv(const int* state, cudaStream_t stream) {
  count_launch();
  report_notconv_kernel<<<1, 1, 0, stream>>>(state);
  return cudaGetLastError();
}

cudaError_t read_device_status(int* status, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(status, g_device_status, sizeof(int));
  if (e != cudaSuccess || !clear) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
}

}  // namespace mera
