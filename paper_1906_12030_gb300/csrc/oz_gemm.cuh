// Tensor-core GEMM of the fixed-point split modes (MERA_PREC_OZ3 / OZ4).
// Included by tc_gemm.cu inside its anonymous namespace: it shares that
// file's PTX wrappers (mbarrier, TMA, tcgen05) and its device status word.
//
// Operands are S BF16 slice planes written by the split kernel (oz_split.cu):
// along K every row is cut into blocks of kOzBlockK elements, and slice p of
// a block is an integer in [-256, 256] times 2^(e - 7 - 9p), e the exponent
// of the block's largest entry.  This is the error-free splitting of Ozaki,
// Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), with one exponent per
// row block instead of per row.  Within a block every product of the two
// leading slices is an integer multiple of 2^(eA + eB - 14) of magnitude at
// most 2^16, so the sum of a block's 256 of them stays below 2^24 units and
// the FP32 accumulator holds it exactly.  The kernel therefore keeps two
// accumulators per block in tensor memory:
//   G0  leading slice x leading slice (exact)
//   G1  every other product with slice orders summing to less than S (each
//       at most 2^-9 of G0's scale, so its FP32 rounding is ~2^-33 of it)
// and the epilogue adds each block's G0 and G1 into a running sum held as an
// unevaluated pair hi + lo of binary32 values (Knuth's TwoSum), ~48 bits.
// Products of slice orders summing to S or more are dropped: at most
// 2^(-9 S + 2) of the block's leading scale (OZ3 ~2^-25, OZ4 ~2^-34).
//
// Tensor memory: (G0, G1) x 2 buffers of width BN (<= 128), so the MMAs of
// block k+1 overlap the epilogue's reads of block k.  Warp roles as in
// tc_gemm_kernel (warp 0 TMA, warp 1 MMA) with eight epilogue warps; stages
// hold 64-byte slabs (32 BF16 along K) of every plane -- the A planes, then
// the B planes one after another -- so eight stages make one block.  With G1
// right after G0 in tensor memory, slice 0 of A meets slices 0 and 1 of B in
// one MMA of width 2 BN (one read of A for two products).
//
// Output: the caller's binary64 output (written or accumulated), raw hi + lo
// binary32 planes of the next operand (split afterwards), or, with a K split,
// hi + lo partial planes summed by oz_splitk_reduce_kernel.

// Eight epilogue warps (two per tensor-memory lane quarter): each thread then
// holds up to 64 running pairs in registers within the 200 that a 320-thread
// block allows (sixteen warps would cap it at 96 and spill).
constexpr int kOzEpiWarps = 8;
constexpr int kOzEpiThreads = 32 * kOzEpiWarps;
constexpr int kOzThreads = 64 + kOzEpiThreads;

template <int S, int BN>
struct OzCfg {
  static constexpr int kSlab = 64;                  // bytes along K per stage and plane
  static constexpr int kBK = kSlab / 2;             // 32 BF16
  static constexpr int kBlockStages = kOzBlockK / kBK;
  static constexpr int kABytes = kBM * kSlab;
  static constexpr int kBBytes = BN * kSlab;
  static constexpr int kStageBytes = S * (kABytes + kBBytes);
  static constexpr int kStages = kStageBudget / kStageBytes > 8 ? 8
                                 : (kStageBudget / kStageBytes < 2 ? 2 : kStageBudget / kStageBytes);
  static constexpr int kAccCols = BN < 32 ? 32 : BN;
  static constexpr int kTmemCols = 4 * kAccCols;    // (G0, G1) x 2
  static constexpr int kSubs = kOzEpiWarps / 4;     // warps per lane quarter
  static constexpr int kCols = BN < 32 ? BN : BN / kSubs;  // columns per epilogue thread
  static constexpr int kActiveSubs = BN < 32 ? 1 : kSubs;
  static constexpr size_t kSmem = 1024 + size_t(kStages) * kStageBytes + 1024 + BN * (sizeof(int64_t) + sizeof(int));
  static_assert(BN == 16 || BN == 64 || BN == 128, "fixed-point split tile widths");
  static_assert(kOzBlockK % kBK == 0, "block of whole stages");
};

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// hi + lo += x (exact, TwoSum) + y (rounded into lo).
__device__ __forceinline__ void dd_add(float& hi, float& lo, float x, float y) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, y));
}

// (hi, lo) -> the nearest binary32 pair with |lo| <= ulp(hi)/2 (TwoSum).
__device__ __forceinline__ void dd_norm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  const float bp = __fsub_rn(s, hi);
  lo = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(lo, bp));
  hi = s;
}

template <int S, int BN>
__global__ void __launch_bounds__(kOzThreads, 1)
    oz_gemm_kernel(const __grid_constant__ TMaps tm, const __grid_constant__ Epilogue ep) {
  using C = OzCfg<S, BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint8_t* aux = smem + size_t(C::kStages) * C::kStageBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(aux);
  uint64_t* empty = full + C::kStages;
  uint64_t* acc_full = empty + C::kStages;  // [2] MMA -> epilogue, one phase per block
  uint64_t* acc_empty = acc_full + 2;       // [2] epilogue -> MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* abort_snapshot = abort_flag + 1;
  volatile int* never = abort_flag + 2;
  int64_t* off_n = reinterpret_cast<int64_t*>(aux + 1024);
  int* off_n32 = reinterpret_cast<int*>(off_n + BN);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t tiles_n = (ep.N + BN - 1) / BN;
  const int64_t tiles_mn = ((ep.M + kBM - 1) / kBM) * tiles_n;
  const int64_t tiles = tiles_mn * ep.split;
  const int num_k = int((ep.K + C::kBK - 1) / C::kBK);  // stages over all of K
  // a work item covers stages [kb0, kb1): kc is a whole number of blocks

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kOzEpiWarps);
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
      // ---- producer: S planes of A and of B per stage ----------------------
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
          for (int pl = 0; pl < S; ++pl) {  // A planes, then the B planes one after another
            tma_load_2d(st + pl * C::kABytes, &tm.a[pl], x, m0, &full[s]);
            tma_load_2d(st + S * C::kABytes + pl * C::kBBytes, &tm.b[pl], x, n0, &full[s]);
          }
        }
      }
      for (uint32_t j = (it > uint32_t(C::kStages) ? it - C::kStages : 0); j < it; ++j)
        mbar_wait(&full[j % C::kStages], (j / C::kStages) & 1, never);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: one accumulator pair per block ------------------------
      constexpr uint32_t idesc = make_idesc(1u, kBM, BN);
      // slice 0 of A against slices 0 and 1 of B (adjacent in the stage) in
      // one MMA of width 2 BN, writing G0 and G1 (adjacent in tensor memory)
      constexpr bool kMerge = C::kAccCols == BN;
      constexpr uint32_t idesc2 = make_idesc(1u, kBM, kMerge ? 2 * BN : BN);
      constexpr uint32_t kBBase = uint32_t(S * C::kABytes);
      uint32_t it = 0, bc = 0;  // stages consumed, blocks issued
      bool alive = true;
      for (int64_t t = blockIdx.x; t < tiles && alive; t += gridDim.x) {
        const int kb0 = int(t / tiles_mn) * ep.kc, kb1 = min(kb0 + ep.kc, num_k);
        for (int blk = kb0; blk < kb1 && alive; blk += C::kBlockStages, ++bc) {
          const uint32_t b = bc & 1;
          if (bc >= 2 && !mbar_wait(&acc_empty[b], ((bc >> 1) - 1) & 1, abort_flag)) {
            alive = false;
            break;
          }
          tc_fence_after();
          const uint32_t g0 = tmem + b * 2u * uint32_t(C::kAccCols);
          const uint32_t g1 = g0 + uint32_t(C::kAccCols);
          const int blk_end = min(blk + C::kBlockStages, kb1);
          for (int kb = blk; kb < blk_end; ++kb, ++it) {
            const uint32_t s = it % C::kStages;
            if (!mbar_wait(&full[s], (it / C::kStages) & 1, abort_flag)) {
              alive = false;
              break;
            }
            tc_fence_after();
            const uint32_t s0 = smem_u32(stage_base + size_t(s) * C::kStageBytes);
#pragma unroll
            for (int k = 0; k < C::kSlab / 32; ++k) {
              const uint32_t koff = uint32_t(k * 32);
              const bool first = (kb == blk) && (k == 0);
#pragma unroll
              for (int pa = 0; pa < S; ++pa) {
#pragma unroll
                for (int pb = 0; pb + pa < S; ++pb) {
                  if (kMerge && pa == 0 && pb == 1) continue;  // issued with (0,0)
                  const uint32_t a_addr = s0 + pa * C::kABytes + koff;
                  const uint32_t b_addr = s0 + kBBase + pb * C::kBBytes + koff;
                  // G0 takes (0,0); G1 starts with (0,1), the first other product issued
                  const bool lead = (pa == 0 && pb == 0);
                  const uint32_t acc = (first && (lead || (pa == 0 && pb == 1))) ? 0u : 1u;
                  tc_mma<PREC_BF16>(lead ? g0 : g1, smem_desc<C::kSlab>(a_addr), smem_desc<C::kSlab>(b_addr),
                                    lead && kMerge ? idesc2 : idesc, acc);
                }
              }
            }
            tc_commit(&empty[s]);
          }
          tc_commit(&acc_full[b]);  // also after an abort, so that no epilogue warp waits forever
        }
      }
    }
  } else {
    // ---- epilogue (warps 2..9): running double-float sums in registers -------
    const int et = threadIdx.x - 64;
    const int quarter = warp % 4;
    const int sub = (warp - 2) / 4;
    const int row = quarter * 32 + lane;
    const bool active = sub < C::kActiveSubs;
    const int c0 = sub * C::kCols;  // first column of this warp's share
    const bool final_fast = ep.c_final && ep.split <= 1 && ep.off32 && ep.alpha_pow2;
    const bool raw_fast = !ep.c_final && ep.split <= 1 && ep.off32 && ep.alpha == 1.0;
    uint32_t bc = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int64_t ks = t / tiles_mn;
      int64_t row_t, col_t;
      tile_of(t % tiles_mn, tiles_mn / tiles_n, tiles_n, ep.group_m, row_t, col_t);
      const int64_t m0 = row_t * kBM, n0 = col_t * BN;
      const int kb0 = int(ks) * ep.kc, kb1 = min(kb0 + ep.kc, num_k);
      asm volatile("bar.sync 1, %0;" ::"n"(kOzEpiThreads) : "memory");
      if (et == 0) *abort_snapshot = *abort_flag;
      for (int c = et; c < BN; c += kOzEpiThreads) {
        const int64_t n = n0 + c;
        const int64_t o = n < ep.N ? legmap_offset32(ep.n_dst, uint32_t(n)) : 0;
        off_n[c] = o;
        off_n32[c] = int(o);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kOzEpiThreads) : "memory");
      if (*abort_snapshot) break;
      const int64_t m = m0 + row;
      const bool row_ok = m < ep.M;
      float hi[C::kCols], lo[C::kCols];
#pragma unroll
      for (int j = 0; j < C::kCols; ++j) hi[j] = lo[j] = 0.0f;
      bool ok = true;
      for (int blk = kb0; blk < kb1; blk += C::kBlockStages, ++bc) {
        const uint32_t b = bc & 1;
        ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (bc >> 1) & 1, abort_flag) ? 1 : 0) != 0;
        tc_fence_after();
        if (!ok) break;  // the next tile's snapshot sees the abort flag
        if (active) {
          const uint32_t ta = tmem + b * 2u * uint32_t(C::kAccCols) + uint32_t(c0) + (uint32_t(quarter * 32) << 16);
          // eight columns of G0 and G1 at a time: the running pairs already
          // take 2 kCols registers
#pragma unroll
          for (int h = 0; h < C::kCols; h += 8) {
            uint32_t v0[8], v1[8];
            tmem_ld8(ta + uint32_t(h), v0);
            tmem_ld8(ta + uint32_t(C::kAccCols) + uint32_t(h), v1);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) dd_add(hi[h + j], lo[h + j], __uint_as_float(v0[j]), __uint_as_float(v1[j]));
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
      }
      if (!ok || !active || !row_ok) continue;
#pragma unroll
      for (int j = 0; j < C::kCols; ++j) dd_norm(hi[j], lo[j]);
      if (ep.split > 1) {  // partial pair, summed by oz_splitk_reduce_kernel
        float* p = ep.partial + (ks * ep.N + n0 + c0) * ep.M + m;
#pragma unroll
        for (int j = 0; j < C::kCols; ++j, p += ep.M)
          if (n0 + c0 + j < ep.N) {
            p[0] = hi[j];
            p[ep.p_plane] = lo[j];
          }
        continue;
      }
      const int64_t off_m = legmap_offset32(ep.m_dst, uint32_t(m));
      const bool whole = n0 + c0 + C::kCols <= ep.N;
      if (ep.c_final) {
        double* __restrict__ r = static_cast<double*>(ep.C) + off_m;
#pragma unroll
        for (int j = 0; j < C::kCols; ++j) {
          if (!whole && n0 + c0 + j >= ep.N) continue;
          const int64_t o = final_fast ? int64_t(off_n32[c0 + j]) : off_n[c0 + j];
          const double x = final_fast ? f32_to_f64_pow2(hi[j], ep.alpha_exp) + f32_to_f64_pow2(lo[j], ep.alpha_exp)
                                      : ep.alpha * (double(hi[j]) + double(lo[j]));
          r[o] = ep.accumulate ? r[o] + x : x;
        }
      } else {
        float* __restrict__ r0 = static_cast<float*>(ep.C) + off_m;
        float* __restrict__ r1 = r0 + ep.c_plane;
        const float alpha = float(ep.alpha);
#pragma unroll
        for (int j = 0; j < C::kCols; ++j) {
          if (!whole && n0 + c0 + j >= ep.N) continue;
          const int64_t o = raw_fast ? int64_t(off_n32[c0 + j]) : off_n[c0 + j];
          if (raw_fast) {
            r0[o] = hi[j];
            r1[o] = lo[j];
          } else {  // alpha a power of two in the programs: exact
            r0[o] = __fmul_rn(alpha, hi[j]);
            r1[o] = __fmul_rn(alpha, lo[j]);
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

// Sum of the K-split partial pairs in a fixed order (double-float), then the
// same output as the GEMM epilogue.  One thread per row m over a chunk of
// columns.
__global__ void __launch_bounds__(256) oz_splitk_reduce_kernel(const __grid_constant__ Epilogue ep) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= ep.M) return;
  const int64_t off_m = legmap_offset32(ep.m_dst, uint32_t(m));
  const int64_t n_per = (ep.N + gridDim.y - 1) / gridDim.y;
  const int64_t n_lo = int64_t(blockIdx.y) * n_per, n_hi = min(ep.N, n_lo + n_per);
  for (int64_t n = n_lo; n < n_hi; ++n) {
    float hi = 0.0f, lo = 0.0f;
    for (int s = 0; s < ep.split; ++s) {
      const int64_t i = (int64_t(s) * ep.N + n) * ep.M + m;
      dd_add(hi, lo, ep.partial[i], ep.partial[i + ep.p_plane]);
    }
    dd_norm(hi, lo);
    const int64_t off = off_m + legmap_offset32(ep.n_dst, uint32_t(n));
    if (ep.c_final) {
      double* dst = static_cast<double*>(ep.C) + off;
      const double val = ep.alpha_pow2 ? f32_to_f64_pow2(hi, ep.alpha_exp) + f32_to_f64_pow2(lo, ep.alpha_exp)
                                       : ep.alpha * (double(hi) + double(lo));
      *dst = ep.accumulate ? (*dst + val) : val;
    } else {
      float* r = static_cast<float*>(ep.C) + off;
      r[0] = __fmul_rn(float(ep.alpha), hi);
      r[ep.c_plane] = __fmul_rn(float(ep.alpha), lo);
    }
  }
}
