// Tensor-core GEMM for sm_103a: TMA -> shared memory (128-byte swizzle,
// K-major) -> tcgen05.mma (FP32 accumulator in tensor memory) -> scattered
// epilogue that writes the next contraction's operand layout directly.
//
// One CTA computes one 128 x BN output tile.  Warp roles:
//   warp 0      TMA producer (one elected lane), STAGES-deep ring
//   warp 1      tensor-memory allocator + MMA issuer (one lane)
//   warps 2..5  epilogue: tcgen05.ld of the accumulator, convert, store
// Every mbarrier wait is bounded; a wait that gives up records
// MERA_ETIMEOUT in a device status word and the CTA drains and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "../../include/mera.h"
#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace mera {

__device__ int g_device_status = 0;

namespace {

constexpr int kBM = 128;          // UMMA M (cta_group::1)
constexpr int kSlabBytes = 128;   // one swizzle row: 64 BF16 or 32 TF32 along K
constexpr int kThreads = 192;
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

// Bounded wait on the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1; i < kSpinCap; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0 && global_ns() - t0 > kTimeoutNs) break;
  }
  atomicOr(&g_device_status, 1 << MERA_ETIMEOUT);
  return false;
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

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (start address and offsets in 16-byte units).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t(1) << 16;             // leading-dimension offset (unused for this layout)
  d |= uint64_t(1024 >> 4) << 32;     // stride-dimension offset
  d |= uint64_t(1) << 46;             // descriptor version
  d |= uint64_t(2) << 61;             // 128-byte swizzle
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

struct Epilogue {
  int64_t M, N, K;
  void* C;
  int64_t c_plane;  // elements between hi and lo planes (BF16X3 operand)
  LegMap m_dst, n_dst;
  double alpha;
  int accumulate;
  int c_final;      // 1: FP64 output of the caller
};

template <int PREC, int BN>
struct Cfg {
  static constexpr int kElem = (PREC == PREC_TF32) ? 4 : 2;
  static constexpr int kBK = kSlabBytes / kElem;          // K per stage
  static constexpr int kPlanes = (PREC == PREC_BF16X3) ? 2 : 1;
  static constexpr int kABytes = kBM * kSlabBytes;        // one plane of A
  static constexpr int kBBytes = BN * kSlabBytes;
  static constexpr int kStageBytes = kPlanes * (kABytes + kBBytes);
  static constexpr int kStages = (PREC == PREC_BF16X3) ? (BN >= 256 ? 2 : 3) : 4;
  static constexpr int kTmemCols = BN < 32 ? 32 : BN;
  static constexpr uint32_t kFmt = (PREC == PREC_TF32) ? 2u : 1u;  // TF32 / BF16
  static constexpr size_t kSmem = 1024 + size_t(kStages) * kStageBytes + 1024 + BN * sizeof(int64_t);
};

template <int PREC, int BN>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                   const __grid_constant__ Epilogue ep) {
  using C = Cfg<PREC, BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint8_t* aux = smem + size_t(C::kStages) * C::kStageBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(aux);
  uint64_t* empty = full + C::kStages;
  uint64_t* accum = empty + C::kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int64_t* off_n = reinterpret_cast<int64_t*>(aux + 1024);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t tiles_n = (ep.N + BN - 1) / BN;
  const int64_t m0 = (int64_t(blockIdx.x) / tiles_n) * kBM;
  const int64_t n0 = (int64_t(blockIdx.x) % tiles_n) * BN;
  const int num_k = int((ep.K + C::kBK - 1) / C::kBK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
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
      int issued = 0;
      for (int kb = 0; kb < num_k; ++kb) {
        const int s = kb % C::kStages;
        if (kb >= C::kStages) {
          if (!mbar_wait(&empty[s], ((kb / C::kStages) & 1) ^ 1)) {
            *reinterpret_cast<volatile int*>(abort_flag) = 1;
            break;
          }
        }
        if (*reinterpret_cast<volatile int*>(abort_flag)) break;
        uint8_t* st = stage_base + size_t(s) * C::kStageBytes;
        mbar_arrive_expect_tx(&full[s], C::kStageBytes);
        const int x = kb * C::kBK;
        tma_load_2d(st, &tmA, x, int(m0), &full[s]);
        tma_load_2d(st + C::kABytes, &tmB, x, int(n0), &full[s]);
        if constexpr (C::kPlanes == 2) {
          tma_load_2d(st + C::kABytes + C::kBBytes, &tmA2, x, int(m0), &full[s]);
          tma_load_2d(st + 2 * C::kABytes + C::kBBytes, &tmB2, x, int(n0), &full[s]);
        }
        ++issued;
      }
      // drain: every issued stage must have landed before the CTA may exit
      for (int kb = (issued > C::kStages ? issued - C::kStages : 0); kb < issued; ++kb)
        mbar_wait(&full[kb % C::kStages], (kb / C::kStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer -------------------------------------------------------
      constexpr uint32_t idesc = make_idesc(C::kFmt, kBM, BN < 16 ? 16 : BN);
      for (int kb = 0; kb < num_k; ++kb) {
        const int s = kb % C::kStages;
        if (!mbar_wait(&full[s], (kb / C::kStages) & 1)) {
          *reinterpret_cast<volatile int*>(abort_flag) = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(stage_base + size_t(s) * C::kStageBytes);
        const uint32_t sb = sa + C::kABytes;
#pragma unroll
        for (int k = 0; k < kSlabBytes / 32; ++k) {
          const uint32_t koff = uint32_t(k * 32);
          const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
          tc_mma<PREC>(tmem, sw128_desc(sa + koff), sw128_desc(sb + koff), idesc, acc);
          if constexpr (C::kPlanes == 2) {
            const uint32_t sa2 = sb + C::kBBytes, sb2 = sa2 + C::kABytes;
            tc_mma<PREC>(tmem, sw128_desc(sa + koff), sw128_desc(sb2 + koff), idesc, 1u);   // hi * lo
            tc_mma<PREC>(tmem, sw128_desc(sa2 + koff), sw128_desc(sb + koff), idesc, 1u);   // lo * hi
          }
        }
        tc_commit(&empty[s]);
      }
      tc_commit(accum);
    }
  } else {
    // ---- epilogue (warps 2..5) -------------------------------------------------
    const int et = threadIdx.x - 64;  // 0..127
    for (int c = et; c < BN; c += 128) {
      const int64_t n = n0 + c;
      off_n[c] = n < ep.N ? legmap_offset(ep.n_dst, n) : 0;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const int quarter = warp % 4;  // tensor-memory lanes this warp may read
    const int row = quarter * 32 + lane;
    const int64_t m = m0 + row;
    const bool row_ok = m < ep.M;
    const int64_t off_m = row_ok ? legmap_offset(ep.m_dst, m) : 0;
    const bool ok = mbar_wait(accum, 0);
    tc_fence_after();
    if (ok && !*reinterpret_cast<volatile int*>(abort_flag)) {
      const float alpha = float(ep.alpha);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(c0), v);
        if (!row_ok) continue;
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
            } else {
              const __nv_bfloat16 hi = __float2bfloat16_rn(val);
              const __nv_bfloat16 lo = __float2bfloat16_rn(val - __bfloat162float(hi));
              static_cast<__nv_bfloat16*>(ep.C)[off] = hi;
              static_cast<__nv_bfloat16*>(ep.C)[off + ep.c_plane] = lo;
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
bool encode_operand(CUtensorMap* tm, const void* base, int prec, int64_t rows, int64_t K, int64_t ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int elem = (prec == PREC_TF32) ? 4 : 2;
  const CUtensorMapDataType dt = (prec == PREC_TF32) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[2] = {cuuint64_t(K), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(ld) * elem};
  cuuint32_t box[2] = {cuuint32_t(kSlabBytes / elem), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
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
  CUtensorMap tA, tB, tA2, tB2;
  const char* A = static_cast<const char*>(a.A);
  const char* B = static_cast<const char*>(a.B);
  if (!encode_operand(&tA, A, PREC, a.M, a.K, a.lda, kBM)) return cudaErrorInvalidValue;
  if (!encode_operand(&tB, B, PREC, a.N, a.K, a.ldb, BN)) return cudaErrorInvalidValue;
  if (C::kPlanes == 2) {
    if (!encode_operand(&tA2, A + a.a_plane_bytes, PREC, a.M, a.K, a.lda, kBM)) return cudaErrorInvalidValue;
    if (!encode_operand(&tB2, B + a.b_plane_bytes, PREC, a.N, a.K, a.ldb, BN)) return cudaErrorInvalidValue;
  } else {
    tA2 = tA;
    tB2 = tB;
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
  ep.accumulate = a.accumulate;
  ep.c_final = a.c_final ? 1 : 0;
  const int64_t tiles = ((a.M + kBM - 1) / kBM) * ((a.N + BN - 1) / BN);
  if (tiles <= 0 || tiles > 0x7fffffff) return cudaErrorInvalidValue;
  count_launch();
  tc_gemm_kernel<PREC, BN><<<unsigned(tiles), kThreads, C::kSmem, stream>>>(tA, tB, tA2, tB2, ep);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_prec(const TcGemmArgs& a, cudaStream_t stream) {
  if (a.N > 128) return launch_cfg<PREC, 256>(a, stream);
  if (a.N > 64) return launch_cfg<PREC, 128>(a, stream);
  if (a.N > 32) return launch_cfg<PREC, 64>(a, stream);
  if (a.N > 16) return launch_cfg<PREC, 32>(a, stream);
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
    default: return cudaErrorNotSupported;
  }
}

cudaError_t read_device_status(int* status, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(status, g_device_status, sizeof(int));
  if (e != cudaSuccess || !clear) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int));
}

}  // namespace mera
