// Launchers of the library's CUDA kernels (host-side declarations).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

#include <atomic>

namespace mera {

// Kernel launches issued by the library (all kernels, all devices).
extern std::atomic<long long> g_launch_count;
inline void count_launch(long long n = 1) { g_launch_count.fetch_add(n, std::memory_order_relaxed); }

// The driver context current on the calling thread (an opaque key for
// per-context caches: a device reset makes a new context).
void* current_cu_context();

// Input tensor -> operand layout, cast to the operand precision (in the
// fixed-point split modes: to the raw hi + lo binary32 planes).
cudaError_t launch_permute(const PermuteStep& p, const double* src, void* dst, int64_t plane_elems,
                           int prec, cudaStream_t stream);

// Fixed-point split modes: raw hi + lo binary32 planes (rows x ld, the lo
// plane raw_plane floats after the hi plane) -> `slices` BF16 planes of the
// operand (dst_plane elements apart), one exponent per row and block of
// kOzBlockK elements along K.  Columns K..ld-1 are not touched.
cudaError_t launch_oz_split(const float* raw, int64_t raw_plane, void* dst, int64_t dst_plane, int64_t rows,
                            int64_t K, int64_t ld, int slices, cudaStream_t stream);

// FP64 GEMM with a scattered epilogue:
//   C[m_dst(m) + n_dst(n)] (+)= alpha * sum_k A[m*a_m + k*a_k] * B[n*b_n + k*b_k]
struct GemmF64Args {
  const double* A;
  int64_t a_m, a_k;
  const double* B;
  int64_t b_n, b_k;
  int64_t M, N, K;
  double* C;
  LegMap m_dst, n_dst;
  double alpha;
  int accumulate;
  const int* skip_if = nullptr;  // device flag: the kernel returns at once when *skip_if != 0
};
cudaError_t launch_gemm_f64(const GemmF64Args& args, cudaStream_t stream);

// Number of per-block partial sums the reduction kernels below may write.
constexpr int kMaxPartials = 65536;

// *out = sum_ij A[i,j] * B[j,i] for n x n row-major A, B (deterministic).
cudaError_t launch_dot_transposed(const double* A, const double* B, int64_t n, double* partials,
                                  double* out, cudaStream_t stream);

// rho <- (X + X^T) / (2 tr X); *resid = ||rho_new - rho_old||_F (deterministic).
// `scalars` holds 2 doubles of scratch.
cudaError_t launch_sym_normalize(const double* X, double* rho, int64_t n, double* partials,
                                 double* scalars, double* resid, cudaStream_t stream);

// Polar-iteration helpers (all binary64, deterministic reductions).
// G = X^T X (n x n) and X (m x n) scaled by 1/c and 1/sqrt(c), c = max row
// abs sum of G (>= its largest eigenvalue), written to *c.
cudaError_t launch_ns_prescale(double* G, double* X, int64_t m, int64_t n, double* c, cudaStream_t stream);
cudaError_t launch_frob_scale(const double* src, double* dst, int64_t count, double* partials,
                              double* scalars, cudaStream_t stream);
// One gated quintic Newton-Schulz step's elementwise part: Bm = (5/2)(I - G)
// + G2 (G2 = G G), resid = ||G - I||_F, state[2] = (resid <= tol).  Skipped
// once state[0] is set.
cudaError_t launch_ns_step(const double* G, const double* G2, double* Bm, int64_t n, double* partials,
                           double* resid, double tol, int* state, cudaStream_t stream);
// Closes a step: state[1] += 1; state[0] = state[2].  Skipped once state[0] is set.
cudaError_t launch_ns_finish(int* state, cudaStream_t stream);
// out = -(state[1] odd ? x1 : x0): the polar result, selected on the device.
cudaError_t launch_ns_output(const double* x0, const double* x1, const int* state, double* out, int64_t count,
                             cudaStream_t stream);
// Stiefel gradient step helpers: S = (A + A^T)/2 (n x n) and
// Yneg = eta (G - T) - X (count elements).
cudaError_t launch_stiefel_sym(const double* A, double* S, int64_t n, cudaStream_t stream);
cudaError_t launch_stiefel_combine(const double* X, const double* G, const double* T, double* Yneg, int64_t count,
                                   double eta, cudaStream_t stream);
// out = g * (a + b) elementwise (b may be null), g a device scalar.
cudaError_t launch_scaled_sum(const double* a, const double* b, const double* g, double* out, int64_t n,
                              cudaStream_t stream);
// Sets the conditional handle of a recorded while loop to (state[0] == 0 and
// state[1] < max_iter).
cudaError_t launch_ns_continue(const int* state, cudaGraphConditionalHandle h, int max_iter, cudaStream_t stream);


}  // namespace mera
