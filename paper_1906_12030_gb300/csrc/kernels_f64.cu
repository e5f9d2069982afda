// Binary64 kernels: operand permute/cast, FP64 GEMM with scattered epilogue,
// deterministic reductions (trace, Hilbert-Schmidt products, norms) and the
// elementwise parts of the polar iteration (quintic Newton-Schulz).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace mera {

// ---------------------------------------------------------------------------
// Input tensor -> operand layout, cast to the operand precision.
//
// The copy is a permutation of the tensor's legs.  The legs are grouped into
// A (those of smallest destination stride, up to kTile elements), B (those of
// smallest source stride among the rest, up to kTile elements) and the outer
// legs; a leg is split in two where that makes a group fill exactly.  Each
// block moves TA x TB tiles through shared memory: reads run along B (or
// along A when A is also contiguous in the source), writes along A, so both
// sides move runs of up to kTile elements.  The in-tile offsets come from
// tables in shared memory and the outer offsets are decoded once per tile.
// ---------------------------------------------------------------------------
constexpr int kTile = 64;

struct PermuteArgs {
  int n_other;
  int64_t dim[2 * kMaxLeg], src_stride[2 * kMaxLeg], dst_stride[2 * kMaxLeg];  // outer legs
  int ta, tb;              // tile extents (products of the A and B legs)
  int read_a;              // A is contiguous in the source too: read along A
  int64_t outer;           // number of tiles (product of the outer legs)
  int64_t a_src[kTile], a_dst[kTile], b_src[kTile], b_dst[kTile];  // in-tile offsets
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

template <int PREC>
__global__ void __launch_bounds__(256) permute_tile_kernel(const double* __restrict__ src, void* dst, int64_t plane,
                                                           const __grid_constant__ PermuteArgs p) {
  __shared__ double tile[kTile * (kTile + 1)];
  __shared__ int64_t s_as[kTile], s_ad[kTile], s_bs[kTile], s_bd[kTile];
  const int tid = threadIdx.x;
  const int ta = p.ta, tb = p.tb, count = ta * tb;
  if (tid < kTile) {
    s_as[tid] = tid < ta ? p.a_src[tid] : 0;
    s_ad[tid] = tid < ta ? p.a_dst[tid] : 0;
    s_bs[tid] = tid < tb ? p.b_src[tid] : 0;
    s_bd[tid] = tid < tb ? p.b_dst[tid] : 0;
  }
  __syncthreads();
  // x / d for x < 2^13 by a float reciprocal: (x + 0.5) / d is at least
  // 0.5 / d away from an integer, far more than the float rounding error
  const float inv_ta = 1.0f / float(ta), inv_tb = 1.0f / float(tb);
  const int pitch = tb + 1;  // tile[ia * pitch + ib]
  for (int64_t t = blockIdx.x; t < p.outer; t += gridDim.x) {
    int64_t so, dof;
    decode_other(p, uint32_t(t), so, dof);
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
          int ia, ib;
          if (p.read_a) {
            ib = int((float(e) + 0.5f) * inv_ta);
            ia = e - ib * ta;
          } else {
            ia = int((float(e) + 0.5f) * inv_tb);
            ib = e - ia * tb;
          }
          v[k] = src[so + s_as[ia] + s_bs[ib]];
          slot[k] = ia * pitch + ib;
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (slot[k] >= 0) tile[slot[k]] = v[k];
    }
    __syncthreads();
    // writes along A (contiguous in the destination)
    for (int e = tid; e < count; e += 256) {
      const int ib = int((float(e) + 0.5f) * inv_ta), ia = e - ib * ta;
      OperandStore<PREC>::store(dst, dof + s_ad[ia] + s_bd[ib], plane, tile[ia * pitch + ib]);
    }
    __syncthreads();
  }
}

namespace {

struct Leg {
  int64_t dim, ss, ds;
};

// Take legs from `pool` in order of `key` into a group of at most kTile
// elements; the first leg that does not fit whole is split when a divisor
// of its size fills the group further.  Returns the group's legs, inner first.
template <typename Key>
std::vector<Leg> take_group(std::vector<Leg>& pool, Key key) {
  std::stable_sort(pool.begin(), pool.end(), [&](const Leg& x, const Leg& y) { return key(x) < key(y); });
  std::vector<Leg> g;
  int64_t prod = 1;
  while (!pool.empty()) {
    Leg l = pool.front();
    if (prod * l.dim <= kTile) {
      g.push_back(l);
      prod *= l.dim;
      pool.erase(pool.begin());
      continue;
    }
    int64_t q = kTile / prod;
    while (q > 1 && l.dim % q) --q;
    if (q > 1) {  // inner part (q values) joins the group, outer part stays
      g.push_back({q, l.ss, l.ds});
      pool.front() = {l.dim / q, l.ss * q, l.ds * q};
      prod *= q;
    }
    break;
  }
  return g;
}

// In-tile offsets of a group: index i = sum over legs of x_leg * (product
// of the inner legs' sizes), inner leg fastest.
int fill_table(const std::vector<Leg>& g, int64_t* src_off, int64_t* dst_off) {
  int n = 1;
  src_off[0] = dst_off[0] = 0;
  for (const Leg& l : g) {
    for (int64_t x = 1; x < l.dim; ++x)
      for (int i = 0; i < n; ++i) {
        src_off[x * n + i] = src_off[i] + x * l.ss;
        dst_off[x * n + i] = dst_off[i] + x * l.ds;
      }
    n *= int(l.dim);
  }
  return n;
}

}  // namespace

cudaError_t launch_permute(const PermuteStep& st, const double* src, void* dst, int64_t plane_elems,
                           int prec, cudaStream_t stream) {
  if (st.rows <= 0 || st.cols <= 0) return cudaSuccess;
  // Every leg with its source and destination strides (size-1 legs dropped).
  std::vector<Leg> pool;
  int64_t acc = st.ld;
  for (int i = st.row_src.n - 1; i >= 0; --i) {
    if (st.row_src.dim[i] > 1) pool.push_back({st.row_src.dim[i], st.row_src.stride[i], acc});
    acc *= st.row_src.dim[i];
  }
  acc = 1;
  for (int i = st.col_src.n - 1; i >= 0; --i) {
    if (st.col_src.dim[i] > 1) pool.push_back({st.col_src.dim[i], st.col_src.stride[i], acc});
    acc *= st.col_src.dim[i];
  }
  // Ls: the leg contiguous in the source, Ld: the one contiguous in the
  // destination.  When they differ, Ls is kept out of A so that it leads B;
  // when they coincide, A leads with it and the reads run along A.
  PermuteArgs p{};
  std::vector<Leg> ga, gb;
  if (!pool.empty()) {
    size_t is = 0, id = 0;
    for (size_t i = 1; i < pool.size(); ++i) {
      if (pool[i].ss < pool[is].ss) is = i;
      if (pool[i].ds < pool[id].ds) id = i;
    }
    if (is == id) {
      p.read_a = 1;
      ga = take_group(pool, [](const Leg& l) { return l.ds; });
      gb = take_group(pool, [](const Leg& l) { return l.ss; });
    } else {
      const Leg ls = pool[is];
      pool.erase(pool.begin() + long(is));
      ga = take_group(pool, [](const Leg& l) { return l.ds; });
      pool.push_back(ls);
      gb = take_group(pool, [](const Leg& l) { return l.ss; });
    }
  }
  p.ta = fill_table(ga, p.a_src, p.a_dst);
  p.tb = fill_table(gb, p.b_src, p.b_dst);
  if (int(pool.size()) > 2 * kMaxLeg) return cudaErrorInvalidValue;
  p.outer = 1;
  p.n_other = 0;
  for (const Leg& l : pool) {  // outer legs (order is irrelevant for correctness)
    p.dim[p.n_other] = l.dim;
    p.src_stride[p.n_other] = l.ss;
    p.dst_stride[p.n_other] = l.ds;
    p.outer *= l.dim;
    ++p.n_other;
  }
  if (p.outer >= (int64_t(1) << 31)) return cudaErrorInvalidValue;  // 32-bit tile indices
  count_launch();
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(p.outer, 152 * 8)));
#define MERA_PERMUTE_LAUNCH(P) permute_tile_kernel<P><<<grid, 256, 0, stream>>>(src, dst, plane_elems, p);
  switch (prec) {
    case PREC_F64: MERA_PERMUTE_LAUNCH(PREC_F64) break;
    case PREC_TF32: MERA_PERMUTE_LAUNCH(PREC_TF32) break;
    case PREC_BF16: MERA_PERMUTE_LAUNCH(PREC_BF16) break;
    case PREC_BF16X3: MERA_PERMUTE_LAUNCH(PREC_BF16X3) break;
    case PREC_BF16X6: MERA_PERMUTE_LAUNCH(PREC_BF16X6) break;
    case PREC_OZ3:
    case PREC_OZ4:  // into the raw hi + lo planes; the split step follows
    case PREC_RAW: MERA_PERMUTE_LAUNCH(PREC_RAW) break;
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

// rho = (X + X^T) / (2 tr X) over pairs of 32 x 32 tiles (I, J), I <= J:
// both tiles are read once and both written once, so X is read once in all.
template <bool RESID>
__global__ void __launch_bounds__(256) sym_normalize_kernel(const double* __restrict__ X, double* rho, int64_t n,
                                                            const double* __restrict__ trace, double* partials) {
  __shared__ double sa[32][33], sb[32][33];
  const double inv2t = 0.5 / *trace;
  const int64_t nt = (n + 31) / 32;
  double v = 0.0;
  for (int64_t t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const int64_t I = t / nt, J = t % nt;
    if (I > J) continue;  // uniform over the block
    const int64_t i0 = I * 32, j0 = J * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int64_t ga = i0 + r, gb = j0 + threadIdx.x;  // tile (I, J)
      sa[r][threadIdx.x] = (ga < n && gb < n) ? X[ga * n + gb] : 0.0;
      const int64_t gc = j0 + r, gd = i0 + threadIdx.x;  // tile (J, I)
      sb[r][threadIdx.x] = (gc < n && gd < n) ? X[gc * n + gd] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
      {
        const int64_t gi = i0 + r, gj = j0 + threadIdx.x;
        if (gi < n && gj < n) {
          const double nv = (sa[r][threadIdx.x] + sb[threadIdx.x][r]) * inv2t;
          if constexpr (RESID) {
            const double d = nv - rho[gi * n + gj];
            v += d * d;
          }
          rho[gi * n + gj] = nv;
        }
      }
      if (I != J) {
        const int64_t gi = j0 + r, gj = i0 + threadIdx.x;
        if (gi < n && gj < n) {
          const double nv = (sb[r][threadIdx.x] + sa[threadIdx.x][r]) * inv2t;
          if constexpr (RESID) {
            const double d = nv - rho[gi * n + gj];
            v += d * d;
          }
          rho[gi * n + gj] = nv;
        }
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
// Polar (quintic Newton-Schulz) helpers.
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

// Gershgorin rescale of the first Newton-Schulz step: with G = X^T X and
// c = max_i sum_j |G_ij| >= lambda_max(G), X / sqrt(c) has every singular
// value in (0, 1] and the same polar factor, usually much closer to 1 than
// the Frobenius scaling leaves them.
__global__ void __launch_bounds__(1024) ns_gershgorin_kernel(const double* __restrict__ G, int64_t n, double* c) {
  __shared__ double sm[32];
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double r = 0.0;
    for (int64_t j = 0; j < n; ++j) r += fabs(G[i * n + j]);
    v = fmax(v, r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) *c = v;
  }
}

__global__ void __launch_bounds__(256) ns_prescale_kernel(double* G, int64_t gcount, double* X, int64_t xcount,
                                                          const double* __restrict__ c) {
  const double ig = 1.0 / *c, ix = 1.0 / sqrt(*c);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < gcount + xcount;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (i < gcount)
      G[i] *= ig;
    else
      X[i - gcount] *= ix;
  }
}

cudaError_t launch_ns_prescale(double* G, double* X, int64_t m, int64_t n, double* c, cudaStream_t stream) {
  count_launch(2);
  ns_gershgorin_kernel<<<1, 1024, 0, stream>>>(G, n, c);
  const int64_t total = n * n + m * n;
  const int nb = int(std::min<int64_t>((total + 255) / 256, 1024));
  ns_prescale_kernel<<<nb, 256, 0, stream>>>(G, n * n, X, m * n, c);
  return cudaGetLastError();
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

// The step X <- X p(X^T X) with the odd quintic x p(x^2),
//   p(g) = 5/2 - (5/2) g + g^2,  so that x p(x^2) = (5/2) x - (5/2) x^3 + x^5:
// it fixes 1 with zero slope (x p(x^2) - 1 ~ (5/2) (x - 1)^2: quadratic
// convergence, like the cubic (3 x - x^3) / 2), maps [0, 1] into
// [0, 1.061], below its repelling fixed point sqrt(3/2) = 1.225, and grows a
// small singular value 2.5-fold per step where the cubic grows it 1.5-fold.
// At three products per step against two that is 1.36 against 1.22 per
// product; the point is the reach of a step budget: 100 steps bring a
// singular value of 1e-38 of the largest to 1, the cubic's 1e-17.
// Bm = p(G) = (5/2)(I - G) + G2 (G2 = G G) and partial sums of ||G - I||_F^2.
__global__ void __launch_bounds__(256) ns_combine_kernel(const double* __restrict__ G, const double* __restrict__ G2,
                                                         double* Bm, int64_t n, double* partials, const int* skip_if) {
  if (skip_if && *skip_if) return;
  double v = 0.0;
  const int64_t count = n * n;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
    const bool diag = (i / n) == (i % n);
    const double d = G[i] - (diag ? 1.0 : 0.0);
    v += d * d;
    Bm[i] = fma(-2.5, d, G2[i]);
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

cudaError_t launch_ns_step(const double* G, const double* G2, double* Bm, int64_t n, double* partials,
                           double* resid, double tol, int* state, cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((n * n + 255) / 256, 1024));
  count_launch(2);
  ns_combine_kernel<<<nb, 256, 0, stream>>>(G, G2, Bm, n, partials, state);
  ns_check_kernel<<<1, 1024, 0, stream>>>(partials, nb, resid, tol, state);
  return cudaGetLastError();
}

cudaError_t launch_ns_finish(int* state, cudaStream_t stream) {
  count_launch();
  ns_finish_kernel<<<1, 1, 0, stream>>>(state);
  return cudaGetLastError();
}


// out = -X with X the iterate the Newton-Schulz state points at (buffer
// state[1] & 1), chosen on the device so that no host read is needed.  The
// sign flip is a bit operation (exact, off the FP64 pipe).
__global__ void __launch_bounds__(256) ns_output_kernel(const double* __restrict__ x0, const double* __restrict__ x1,
                                                        const int* __restrict__ state, double* out, int64_t count) {
  const double* src = (state[1] & 1) ? x1 : x0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = __longlong_as_double(__double_as_longlong(src[i]) ^ (1ll << 63));
}

cudaError_t launch_ns_output(const double* x0, const double* x1, const int* state, double* out, int64_t count,
                             cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((count + 255) / 256, 1024));
  if (nb <= 0) return cudaSuccess;
  count_launch();
  ns_output_kernel<<<nb, 256, 0, stream>>>(x0, x1, state, out, count);
  return cudaGetLastError();
}

// Riemannian gradient step on the Stiefel manifold (embedded metric):
// with A = X^T G, S = (A + A^T) / 2 and T = X S, the step direction is
// G - T; the kernel writes Yneg = -(X - eta (G - T)) for the polar retraction
// (the polar update returns -polar(-Y) = polar(Y)).
__global__ void __launch_bounds__(256) stiefel_sym_kernel(const double* __restrict__ A, double* S, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n * n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / n, c = i - r * n;
    S[i] = 0.5 * (A[i] + A[c * n + r]);
  }
}

__global__ void __launch_bounds__(256) stiefel_combine_kernel(const double* __restrict__ X, const double* __restrict__ G,
                                                              const double* __restrict__ T, double* Yneg, int64_t count,
                                                              double eta) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    Yneg[i] = eta * (G[i] - T[i]) - X[i];
}

cudaError_t launch_stiefel_sym(const double* A, double* S, int64_t n, cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((n * n + 255) / 256, 1024));
  count_launch();
  stiefel_sym_kernel<<<nb, 256, 0, stream>>>(A, S, n);
  return cudaGetLastError();
}

cudaError_t launch_stiefel_combine(const double* X, const double* G, const double* T, double* Yneg, int64_t count,
                                   double eta, cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((count + 255) / 256, 1024));
  count_launch();
  stiefel_combine_kernel<<<nb, 256, 0, stream>>>(X, G, T, Yneg, count, eta);
  return cudaGetLastError();
}

// Last kernel of a recorded Newton-Schulz loop body: go on while not
// converged and fewer than max_iter steps have run.
__global__ void ns_continue_kernel(const int* state, cudaGraphConditionalHandle h, int max_iter) {
  cudaGraphSetConditional(h, (state[0] == 0 && state[1] < max_iter) ? 1u : 0u);
}

cudaError_t launch_ns_continue(const int* state, cudaGraphConditionalHandle h, int max_iter, cudaStream_t stream) {
  count_launch();
  ns_continue_kernel<<<1, 1, 0, stream>>>(state, h, max_iter);
  return cudaGetLastError();
}


// out = g * (a + b) elementwise (b may be null), g a device scalar: the
// energy adjoint's sum of the two environment halves times the upstream
// gradient.
__global__ void __launch_bounds__(256) scaled_sum_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                         const double* __restrict__ g, double* __restrict__ out,
                                                         int64_t n) {
  const double gv = *g;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = gv * (b ? a[i] + b[i] : a[i]);
}

cudaError_t launch_scaled_sum(const double* a, const double* b, const double* g, double* out, int64_t n,
                              cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = unsigned(std::min<int64_t>((n + 255) / 256, 152 * 8));
  count_launch();
  scaled_sum_kernel<<<grid, 256, 0, stream>>>(a, b, g, out, n);
  return cudaGetLastError();
}

}  // namespace mera
