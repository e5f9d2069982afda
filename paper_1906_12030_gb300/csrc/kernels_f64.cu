// Binary64 kernels: operand permute/cast, FP64 GEMM with scattered epilogue,
// deterministic reductions (trace, Hilbert-Schmidt products, norms) and the
// elementwise parts of the Newton-Schulz polar iteration.
#include "common.cuh"
#include "kernels.h"

namespace mera {

// ---------------------------------------------------------------------------
// Input tensor -> operand layout, cast to the operand precision.
//
// The copy is a permutation of the tensor's legs.  Let `a` be the leg that is
// contiguous in the destination and `b` the leg contiguous in the source.
// When a != b, 32 x 32 tiles over (a, b) go through shared memory so that the
// reads run along b and the writes along a, both coalesced; when a == b the
// copy runs along that leg directly.  The offsets of the remaining legs are
// decoded once per tile.
// ---------------------------------------------------------------------------
struct PermuteArgs {
  int n_other;
  int64_t dim[kMaxLeg], src_stride[kMaxLeg], dst_stride[kMaxLeg];  // legs other than a, b
  int64_t da, db;          // sizes of legs a and b
  int64_t a_src, a_dst;    // strides of leg a (a_dst is 1 unless every leg is degenerate)
  int64_t b_src, b_dst;    // strides of leg b (b_src is 1 likewise)
  int64_t outer;           // product of the other legs' sizes
};

// o < 2^31 (checked at launch), so the decode divides in 32 bits.
__device__ __forceinline__ void decode_other(const PermuteArgs& p, uint32_t o, int64_t& so, int64_t& dof) {
  so = 0;
  dof = 0;
#pragma unroll 1
  for (int i = p.n_other - 1; i >= 0; --i) {
    const uint32_t d = uint32_t(p.dim[i]);
    const uint32_t q = o / d;
    const int64_t x = int64_t(o - q * d);
    so += x * p.src_stride[i];
    dof += x * p.dst_stride[i];
    o = q;
  }
}

constexpr int kPermuteTile = 4352;  // doubles of shared memory per block (34.8 KB)

// Tiles of TA x TB (a, b) elements, TA, TB <= 32; several tiles (consecutive
// outer indices) per block pass so that a pass moves up to 1024 elements.
// Each thread's in-tile coordinates are fixed for the whole kernel and each
// tile's base offsets and extents are decoded once into shared memory, so
// the element loops do no division.  read_a_fast: the source is contiguous
// along a as well (a == b case, b is then another leg), so reads run along a.
template <int PREC>
__global__ void __launch_bounds__(256) permute_tile_kernel(const double* __restrict__ src, void* dst, int64_t plane,
                                                           const __grid_constant__ PermuteArgs p, int read_a_fast) {
  __shared__ double tile[kPermuteTile];
  __shared__ int64_t s_src[64], s_dst[64];
  __shared__ int s_alim[64], s_blim[64];
  const int TA = int(p.da < 32 ? p.da : 32), TB = int(p.db < 32 ? p.db : 32);
  const int per_tile = TA * TB;
  const int cap = kPermuteTile / (TA * (TB + 1));
  const int nb = cap < 64 ? cap : 64;  // tiles per pass (up to ~4096 elements)
  const uint32_t ca = uint32_t((p.da + TA - 1) / TA), cb = uint32_t((p.db + TB - 1) / TB);
  const int64_t total = p.outer * ca * cb;
  const int tid = threadIdx.x;
  const int tstride = TA * (TB + 1);
  for (int64_t t0 = int64_t(blockIdx.x) * nb; t0 < total; t0 += int64_t(gridDim.x) * nb) {
    const int ntiles = int(total - t0 < nb ? total - t0 : nb);
    if (tid < ntiles) {
      const uint32_t t = uint32_t(t0 + tid);
      const uint32_t o = t / (ca * cb);
      const uint32_t rem = t - o * ca * cb;
      const int64_t a0 = int64_t(rem / cb) * TA, b0 = int64_t(rem % cb) * TB;
      int64_t so, dof;
      decode_other(p, o, so, dof);
      s_src[tid] = so + a0 * p.a_src + b0 * p.b_src;
      s_dst[tid] = dof + a0 * p.a_dst + b0 * p.b_dst;
      s_alim[tid] = int(p.da - a0 < TA ? p.da - a0 : TA);
      s_blim[tid] = int(p.db - b0 < TB ? p.db - b0 : TB);
    }
    __syncthreads();
    const int count = ntiles * per_tile;
    // x / d for x <= 2^22 by a float reciprocal: (x + 0.5) / d is at least
    // 0.5 / d away from an integer, far more than the float rounding error
    const float inv_pt = 1.0f / float(per_tile), inv_ta = 1.0f / float(TA), inv_tb = 1.0f / float(TB);
    // reads: 8 independent loads per thread in flight before any shared store
    for (int e0 = 0; e0 < count; e0 += 256 * 8) {
      double v[8];
      int slot[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int e = e0 + tid + 256 * k;
        slot[k] = -1;
        v[k] = 0.0;
        if (e < count) {
          const int j = int((float(e) + 0.5f) * inv_pt), r = e - j * per_tile;
          int ia, ib;
          if (read_a_fast) {
            ib = int((float(r) + 0.5f) * inv_ta);
            ia = r - ib * TA;
          } else {
            ia = int((float(r) + 0.5f) * inv_tb);
            ib = r - ia * TB;
          }
          if (ia < s_alim[j] && ib < s_blim[j]) {
            v[k] = src[s_src[j] + ia * p.a_src + ib * p.b_src];
            slot[k] = j * tstride + ia * (TB + 1) + ib;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (slot[k] >= 0) tile[slot[k]] = v[k];
    }
    __syncthreads();
    // writes along a (contiguous in the destination)
    for (int e = tid; e < count; e += 256) {
      const int j = int((float(e) + 0.5f) * inv_pt), r = e - j * per_tile;
      const int ib = int((float(r) + 0.5f) * inv_ta), ia = r - ib * TA;
      if (ia < s_alim[j] && ib < s_blim[j])
        OperandStore<PREC>::store(dst, s_dst[j] + ib * p.b_dst + ia * p.a_dst, plane,
                                  tile[j * tstride + ia * (TB + 1) + ib]);
    }
    __syncthreads();
  }
}

cudaError_t launch_permute(const PermuteStep& st, const double* src, void* dst, int64_t plane_elems,
                           int prec, cudaStream_t stream) {
  if (st.rows <= 0 || st.cols <= 0) return cudaSuccess;
  // Every leg with its source and destination strides.
  int n = 0;
  int64_t dim[2 * kMaxLeg], ss[2 * kMaxLeg], ds[2 * kMaxLeg];
  int64_t acc = st.ld;
  for (int i = st.row_src.n - 1; i >= 0; --i) {
    dim[n] = st.row_src.dim[i];
    ss[n] = st.row_src.stride[i];
    ds[n] = acc;
    acc *= dim[n];
    ++n;
  }
  acc = 1;
  for (int i = st.col_src.n - 1; i >= 0; --i) {
    dim[n] = st.col_src.dim[i];
    ss[n] = st.col_src.stride[i];
    ds[n] = acc;
    acc *= dim[n];
    ++n;
  }
  // a: smallest destination stride, b: smallest source stride (legs of size
  // 1 are skipped unless every leg has size 1).
  int a = 0, b = 0;
  for (int i = 1; i < n; ++i) {
    const bool ai = dim[i] > 1, aa = dim[a] > 1;
    if ((ai && !aa) || (ai == aa && ds[i] < ds[a])) a = i;
    if ((ai && !(dim[b] > 1)) || (ai == (dim[b] > 1) && ss[i] < ss[b])) b = i;
  }
  // a == b: tile over (a, b2) with b2 the leg of next-smallest source
  // stride; reads then run along a too.  A tensor with one non-trivial leg
  // gets a dummy b of size 1.
  int read_a_fast = 0;
  if (a == b) {
    read_a_fast = 1;
    b = -1;
    for (int i = 0; i < n; ++i)
      if (i != a && dim[i] > 1 && (b < 0 || ss[i] < ss[b])) b = i;
  }
  PermuteArgs p{};
  p.da = dim[a];
  p.db = b >= 0 ? dim[b] : 1;
  p.a_src = ss[a];
  p.a_dst = ds[a];
  p.b_src = b >= 0 ? ss[b] : 0;
  p.b_dst = b >= 0 ? ds[b] : 0;
  p.outer = 1;
  // other legs, outermost first (order is irrelevant for correctness)
  for (int i = n - 1; i >= 0; --i) {
    if (i == a || i == b) continue;
    if (p.n_other >= kMaxLeg) return cudaErrorInvalidValue;
    p.dim[p.n_other] = dim[i];
    p.src_stride[p.n_other] = ss[i];
    p.dst_stride[p.n_other] = ds[i];
    p.outer *= dim[i];
    ++p.n_other;
  }
  count_launch();
  const int64_t ta = std::min<int64_t>(p.da, 32), tb = std::min<int64_t>(p.db, 32);
  const int64_t work = p.outer * ((p.da + ta - 1) / ta) * ((p.db + tb - 1) / tb);
  const int64_t per_pass = std::min<int64_t>(std::max<int64_t>(kPermuteTile / (ta * (tb + 1)), 1), 64);
  if (work >= (int64_t(1) << 31)) return cudaErrorInvalidValue;  // 32-bit tile indices
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>((work + per_pass - 1) / per_pass, 152 * 16)));
#define MERA_PERMUTE_LAUNCH(P) permute_tile_kernel<P><<<grid, 256, 0, stream>>>(src, dst, plane_elems, p, read_a_fast);
  switch (prec) {
    case PREC_F64: MERA_PERMUTE_LAUNCH(PREC_F64) break;
    case PREC_TF32: MERA_PERMUTE_LAUNCH(PREC_TF32) break;
    case PREC_BF16: MERA_PERMUTE_LAUNCH(PREC_BF16) break;
    case PREC_BF16X3: MERA_PERMUTE_LAUNCH(PREC_BF16X3) break;
    case PREC_BF16X6: MERA_PERMUTE_LAUNCH(PREC_BF16X6) break;
    default: return cudaErrorInvalidValue;
  }
#undef MERA_PERMUTE_LAUNCH
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 GEMM.  (16 T) x (16 T) tile per block of 256 threads, T x T outputs per
// thread at stride 16 (conflict-free shared-memory reads), K in steps of 16.
// T = 4 for large problems; T = 2 or 1 when the tile count would leave most
// of the 152 SMs idle (the small square products of the polar iteration).
// ---------------------------------------------------------------------------
constexpr int kBK = 16;

template <int T>
__global__ void __launch_bounds__(256) gemm_f64_kernel(const __grid_constant__ GemmF64Args p) {
  constexpr int R = 16 * T;
  __shared__ double As[kBK][R + 1];
  __shared__ double Bs[kBK][R + 1];
  __shared__ int64_t offm[R];
  __shared__ int64_t offn[R];
  if (p.skip_if && *p.skip_if) return;

  const int tid = threadIdx.x;
  const int64_t tiles_n = (p.N + R - 1) / R;
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile / tiles_n) * R;
  const int64_t n0 = (tile % tiles_n) * R;
  const int tx = tid % 16, ty = tid / 16;

  double acc[T][T];
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int j = 0; j < T; ++j) acc[i][j] = 0.0;

  const bool a_kfast = (p.a_k == 1);
  const bool b_kfast = (p.b_k == 1);

  for (int64_t k0 = 0; k0 < p.K; k0 += kBK) {
    // R rows x 16 k per operand, T elements per thread, along the unit stride.
#pragma unroll
    for (int i = 0; i < T; ++i) {
      int r, k;
      if (a_kfast) {
        k = tid % 16;
        r = tid / 16 + 16 * i;
      } else {
        r = tid % R;
        k = tid / R + (256 / R) * i;
      }
      const int64_t gm = m0 + r, gk = k0 + k;
      As[k][r] = (gm < p.M && gk < p.K) ? p.A[gm * p.a_m + gk * p.a_k] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < T; ++i) {
      int r, k;
      if (b_kfast) {
        k = tid % 16;
        r = tid / 16 + 16 * i;
      } else {
        r = tid % R;
        k = tid / R + (256 / R) * i;
      }
      const int64_t gn = n0 + r, gk = k0 + k;
      Bs[k][r] = (gn < p.N && gk < p.K) ? p.B[gn * p.b_n + gk * p.b_k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      double a[T], b[T];
#pragma unroll
      for (int i = 0; i < T; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < T; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  for (int t = tid; t < 2 * R; t += 256) {
    if (t < R) {
      const int64_t gm = m0 + t;
      offm[t] = gm < p.M ? legmap_offset32(p.m_dst, uint32_t(gm)) : 0;
    } else {
      const int64_t gn = n0 + t - R;
      offn[t - R] = gn < p.N ? legmap_offset32(p.n_dst, uint32_t(gn)) : 0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < T; ++i) {
    const int r = ty + 16 * i;
    if (m0 + r >= p.M) continue;
#pragma unroll
    for (int j = 0; j < T; ++j) {
      const int c = tx + 16 * j;
      if (n0 + c >= p.N) continue;
      double* dst = p.C + offm[r] + offn[c];
      const double v = p.alpha * acc[i][j];
      *dst = p.accumulate ? (*dst + v) : v;
    }
  }
}

cudaError_t launch_gemm_f64(const GemmF64Args& args, cudaStream_t stream) {
  if (args.M <= 0 || args.N <= 0) return cudaSuccess;
  if (args.M > 0x7fffffff || args.N > 0x7fffffff) return cudaErrorInvalidValue;  // 32-bit row/column decode
  auto tiles = [&](int64_t r) { return ((args.M + r - 1) / r) * ((args.N + r - 1) / r); };
  constexpr int64_t kFill = 2 * 152;  // enough blocks to occupy every SM twice
  count_launch();
  if (tiles(64) >= kFill || tiles(32) > 0x7fffffff) {
    if (tiles(64) > 0x7fffffff) return cudaErrorInvalidValue;
    gemm_f64_kernel<4><<<unsigned(tiles(64)), 256, 0, stream>>>(args);
  } else if (tiles(32) >= kFill) {
    gemm_f64_kernel<2><<<unsigned(tiles(32)), 256, 0, stream>>>(args);
  } else {
    gemm_f64_kernel<1><<<unsigned(tiles(16)), 256, 0, stream>>>(args);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic reductions: each block writes one partial, one block sums the
// partials in a fixed order.
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < NT / 32) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// mode 0: out = sum; mode 1: out = sqrt(sum)
__global__ void __launch_bounds__(1024) reduce_partials_kernel(const double* __restrict__ partials, int np,
                                                               double* out, int mode) {
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += partials[i];
  v = block_sum<1024>(v);
  if (threadIdx.x == 0) *out = mode == 1 ? sqrt(v) : v;
}

// 32 x 32 tiles of an n x n matrix, block (32, 8).  tile (ti, tj) covers rows
// [32 ti, 32 ti + 32) and columns [32 tj, ...).  The transposed tile of B is
// staged through shared memory so both reads are coalesced.
__global__ void __launch_bounds__(256) dot_t_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                    int64_t n, double* partials) {
  __shared__ double bt[32][33];
  const int64_t nt = (n + 31) / 32;
  double v = 0.0;
  for (int64_t t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const int64_t i0 = (t / nt) * 32, j0 = (t % nt) * 32;
    // bt[c][r] = B[j0 + r][i0 + c]
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int64_t gj = j0 + r, gi = i0 + threadIdx.x;
      bt[threadIdx.x][r] = (gj < n && gi < n) ? B[gj * n + gi] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int64_t gi = i0 + r, gj = j0 + threadIdx.x;
      if (gi < n && gj < n) v += A[gi * n + gj] * bt[r][threadIdx.x];
    }
    __syncthreads();
  }
  const int tid = threadIdx.y * 32 + threadIdx.x;
  // reuse block_sum with a flat thread index
  __shared__ double sh[8];
  double s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) sh[threadIdx.y] = s;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += sh[w];
    partials[blockIdx.x] = tot;
  }
}

static int reduction_blocks(int64_t tiles) { return int(std::min<int64_t>(std::max<int64_t>(tiles, 1), 4096)); }

cudaError_t launch_dot_transposed(const double* A, const double* B, int64_t n, double* partials, double* out,
                                  cudaStream_t stream) {
  const int64_t nt = (n + 31) / 32;
  const int nb = reduction_blocks(nt * nt);
  count_launch(2);
  dot_t_kernel<<<nb, dim3(32, 8), 0, stream>>>(A, B, n, partials);
  reduce_partials_kernel<<<1, 1024, 0, stream>>>(partials, nb, out, 0);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) trace_kernel(const double* __restrict__ X, int64_t n, double* out) {
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v += X[i * n + i];
  v = block_sum<1024>(v);
  if (threadIdx.x == 0) *out = v;
}

template <bool RESID>
__global__ void __launch_bounds__(256) sym_normalize_kernel(const double* __restrict__ X, double* rho, int64_t n,
                                                            const double* __restrict__ trace, double* partials) {
  __shared__ double xt[32][33];
  const double inv2t = 0.5 / *trace;
  const int64_t nt = (n + 31) / 32;
  double v = 0.0;
  for (int64_t t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const int64_t i0 = (t / nt) * 32, j0 = (t % nt) * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int64_t gj = j0 + r, gi = i0 + threadIdx.x;
      xt[threadIdx.x][r] = (gj < n && gi < n) ? X[gj * n + gi] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int64_t gi = i0 + r, gj = j0 + threadIdx.x;
      if (gi < n && gj < n) {
        const double nv = (X[gi * n + gj] + xt[r][threadIdx.x]) * inv2t;
        if constexpr (RESID) {
          const double d = nv - rho[gi * n + gj];
          v += d * d;
        }
        rho[gi * n + gj] = nv;
      }
    }
    __syncthreads();
  }
  if constexpr (RESID) {
    __shared__ double sh[8];
    double s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sh[threadIdx.y] = s;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double tot = 0.0;
      for (int w = 0; w < 8; ++w) tot += sh[w];
      partials[blockIdx.x] = tot;
    }
  }
}

cudaError_t launch_sym_normalize(const double* X, double* rho, int64_t n, double* partials, double* scalars,
                                 double* resid, cudaStream_t stream) {
  trace_kernel<<<1, 1024, 0, stream>>>(X, n, scalars);
  const int64_t nt = (n + 31) / 32;
  const int nb = reduction_blocks(nt * nt);
  if (resid) {
    count_launch(3);
    sym_normalize_kernel<true><<<nb, dim3(32, 8), 0, stream>>>(X, rho, n, scalars, partials);
    reduce_partials_kernel<<<1, 1024, 0, stream>>>(partials, nb, resid, 1);
  } else {
    count_launch(2);
    sym_normalize_kernel<false><<<nb, dim3(32, 8), 0, stream>>>(X, rho, n, scalars, partials);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Polar (Newton-Schulz) helpers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sumsq_kernel(const double* __restrict__ x, int64_t count, double* partials) {
  double v = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    v += x[i] * x[i];
  v = block_sum<256>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

__global__ void __launch_bounds__(256) scale_by_inverse_kernel(const double* __restrict__ src, double* dst,
                                                               int64_t count, const double* __restrict__ norm) {
  const double s = 1.0 / *norm;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[i] * s;
}

cudaError_t launch_frob_scale(const double* src, double* dst, int64_t count, double* partials, double* scalars,
                              cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((count + 255) / 256, 1024));
  count_launch(3);
  sumsq_kernel<<<nb, 256, 0, stream>>>(src, count, partials);
  reduce_partials_kernel<<<1, 1024, 0, stream>>>(partials, nb, scalars, 1);
  scale_by_inverse_kernel<<<nb, 256, 0, stream>>>(src, dst, count, scalars);
  return cudaGetLastError();
}

// Bm = (3 I - G) / 2 and partial sums of ||G - I||_F^2.
__global__ void __launch_bounds__(256) ns_combine_kernel(const double* __restrict__ G, double* Bm, int64_t n,
                                                         double* partials, const int* skip_if) {
  if (skip_if && *skip_if) return;
  double v = 0.0;
  const int64_t count = n * n;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
    const bool diag = (i / n) == (i % n);
    const double g = G[i];
    const double d = g - (diag ? 1.0 : 0.0);
    v += d * d;
    Bm[i] = (diag ? 1.5 : 0.0) - 0.5 * g;
  }
  v = block_sum<256>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// state[0] = done, state[1] = iterations executed, state[2] = converged after
// this iteration; resid = ||X^T X - I||_F of the iterate entering it.
__global__ void __launch_bounds__(1024) ns_check_kernel(const double* __restrict__ partials, int np, double* resid,
                                                        double tol, int* state) {
  if (state[0]) return;
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += partials[i];
  v = block_sum<1024>(v);
  if (threadIdx.x == 0) {
    const double r = sqrt(v);
    *resid = r;
    state[2] = (r <= tol || !(r == r)) ? 1 : 0;  // converged, or NaN: stop after this step
  }
}

__global__ void ns_finish_kernel(int* state) {
  if (state[0]) return;
  state[1] += 1;
  if (state[2]) state[0] = 1;
}

cudaError_t launch_ns_step(const double* G, double* Bm, int64_t n, double* partials, double* resid, double tol,
                           int* state, cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((n * n + 255) / 256, 1024));
  count_launch(2);
  ns_combine_kernel<<<nb, 256, 0, stream>>>(G, Bm, n, partials, state);
  ns_check_kernel<<<1, 1024, 0, stream>>>(partials, nb, resid, tol, state);
  return cudaGetLastError();
}

cudaError_t launch_ns_finish(int* state, cudaStream_t stream) {
  count_launch();
  ns_finish_kernel<<<1, 1, 0, stream>>>(state);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) scale_copy_kernel(const double* __restrict__ src, double* dst, int64_t count,
                                                         double alpha) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = alpha * src[i];
}

cudaError_t launch_scale_copy(const double* src, double* dst, int64_t count, double alpha, cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((count + 255) / 256, 1024));
  if (nb <= 0) return cudaSuccess;
  count_launch();
  scale_copy_kernel<<<nb, 256, 0, stream>>>(src, dst, count, alpha);
  return cudaGetLastError();
}

}  // namespace mera
