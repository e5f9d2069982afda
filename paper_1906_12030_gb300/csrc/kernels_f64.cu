// Binary64 kernels: operand permute/cast, FP64 GEMM with scattered epilogue,
// deterministic reductions (trace, Hilbert-Schmidt products, norms) and the
// elementwise parts of the Newton-Schulz polar iteration.
#include "common.cuh"
#include "kernels.h"

namespace mera {

// ---------------------------------------------------------------------------
// Input tensor -> operand layout.  One block row per destination row; the
// row's source offset is decoded once, then threads stride over columns.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(256) permute_kernel(const double* __restrict__ src, void* dst,
                                                      int64_t plane, const __grid_constant__ PermuteStep p) {
  for (int64_t r = blockIdx.y; r < p.rows; r += gridDim.y) {
    const int64_t roff = legmap_offset(p.row_src, r);
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < p.cols;
         c += int64_t(gridDim.x) * blockDim.x) {
      const double v = src[roff + legmap_offset(p.col_src, c)];
      OperandStore<PREC>::store(dst, r * p.ld + c, plane, v);
    }
  }
}

cudaError_t launch_permute(const PermuteStep& p, const double* src, void* dst, int64_t plane_elems,
                           int prec, cudaStream_t stream) {
  if (p.rows <= 0 || p.cols <= 0) return cudaSuccess;
  dim3 block(256);
  dim3 grid(unsigned(std::min<int64_t>((p.cols + 255) / 256, 64)), unsigned(std::min<int64_t>(p.rows, 65535)));
  count_launch();
  switch (prec) {
    case PREC_F64: permute_kernel<PREC_F64><<<grid, block, 0, stream>>>(src, dst, plane_elems, p); break;
    case PREC_TF32: permute_kernel<PREC_TF32><<<grid, block, 0, stream>>>(src, dst, plane_elems, p); break;
    case PREC_BF16: permute_kernel<PREC_BF16><<<grid, block, 0, stream>>>(src, dst, plane_elems, p); break;
    case PREC_BF16X3: permute_kernel<PREC_BF16X3><<<grid, block, 0, stream>>>(src, dst, plane_elems, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 GEMM.  64 x 64 tile per block of 256 threads, 4 x 4 outputs per
// thread at stride 16 (conflict-free shared-memory reads), K in steps of 16.
// ---------------------------------------------------------------------------
constexpr int kBM = 64, kBN = 64, kBK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(const __grid_constant__ GemmF64Args p) {
  __shared__ double As[kBK][kBM + 1];
  __shared__ double Bs[kBK][kBN + 1];
  __shared__ int64_t offm[kBM];
  __shared__ int64_t offn[kBN];

  const int tid = threadIdx.x;
  const int64_t tiles_n = (p.N + kBN - 1) / kBN;
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile / tiles_n) * kBM;
  const int64_t n0 = (tile % tiles_n) * kBN;
  const int tx = tid % 16, ty = tid / 16;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const bool a_kfast = (p.a_k == 1);
  const bool b_kfast = (p.b_k == 1);

  for (int64_t k0 = 0; k0 < p.K; k0 += kBK) {
    // A tile: 64 rows x 16 k.  Pick the thread mapping along the unit stride.
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r, k;
      if (a_kfast) {
        k = tid % 16;
        r = tid / 16 + 16 * i;
      } else {
        r = tid % 64;
        k = tid / 64 + 4 * i;
      }
      const int64_t gm = m0 + r, gk = k0 + k;
      As[k][r] = (gm < p.M && gk < p.K) ? p.A[gm * p.a_m + gk * p.a_k] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r, k;
      if (b_kfast) {
        k = tid % 16;
        r = tid / 16 + 16 * i;
      } else {
        r = tid % 64;
        k = tid / 64 + 4 * i;
      }
      const int64_t gn = n0 + r, gk = k0 + k;
      Bs[k][r] = (gn < p.N && gk < p.K) ? p.B[gn * p.b_n + gk * p.b_k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (tid < kBM) {
    const int64_t gm = m0 + tid;
    offm[tid] = gm < p.M ? legmap_offset(p.m_dst, gm) : 0;
  } else if (tid < kBM + kBN) {
    const int64_t gn = n0 + tid - kBM;
    offn[tid - kBM] = gn < p.N ? legmap_offset(p.n_dst, gn) : 0;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = ty + 16 * i;
    if (m0 + r >= p.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
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
  const int64_t tiles = ((args.M + kBM - 1) / kBM) * ((args.N + kBN - 1) / kBN);
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  count_launch();
  gemm_f64_kernel<<<unsigned(tiles), 256, 0, stream>>>(args);
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
        const double d = nv - rho[gi * n + gj];
        v += d * d;
        rho[gi * n + gj] = nv;
      }
    }
    __syncthreads();
  }
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

cudaError_t launch_sym_normalize(const double* X, double* rho, int64_t n, double* partials, double* scalars,
                                 double* resid, cudaStream_t stream) {
  count_launch(3);
  trace_kernel<<<1, 1024, 0, stream>>>(X, n, scalars);
  const int64_t nt = (n + 31) / 32;
  const int nb = reduction_blocks(nt * nt);
  sym_normalize_kernel<<<nb, dim3(32, 8), 0, stream>>>(X, rho, n, scalars, partials);
  reduce_partials_kernel<<<1, 1024, 0, stream>>>(partials, nb, resid ? resid : scalars + 1, 1);
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
                                                         double* partials) {
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

cudaError_t launch_ns_combine(const double* G, double* Bm, int64_t n, double* partials, double* resid,
                              cudaStream_t stream) {
  const int nb = int(std::min<int64_t>((n * n + 255) / 256, 1024));
  count_launch(2);
  ns_combine_kernel<<<nb, 256, 0, stream>>>(G, Bm, n, partials);
  reduce_partials_kernel<<<1, 1024, 0, stream>>>(partials, nb, resid, 1);
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
