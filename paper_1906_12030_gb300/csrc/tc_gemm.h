// Tensor-core (tcgen05 / TMEM / TMA) GEMM of the contraction programs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

namespace mera {

// C[m_dst(m) + n_dst(n)] (+)= alpha * sum_k A[m, k] * B[n, k]
// A: M x K operand matrix with row pitch lda elements (one or more planes),
// B: N x K with pitch ldb.  Operands are TF32 (stored as FP32), BF16, or
// BF16 planes of a split (BF16X3 hi/lo, BF16X6 hi/mid/lo, or the S slices of
// the fixed-point split modes OZ3/OZ4), plane p at p * *_plane_bytes.  FP32
// accumulation in tensor memory.  The destination is either the caller's
// FP64 output (c_final) or the next operand buffer in the same precision
// (c_plane_elems apart for the lower planes); in the fixed-point split modes
// it is the raw hi + lo binary32 pair of the next operand, split afterwards.
struct TcGemmArgs {
  int prec = 0;
  const void* A = nullptr;
  int64_t a_plane_bytes = 0, lda = 0;
  const void* B = nullptr;
  int64_t b_plane_bytes = 0, ldb = 0;
  int64_t M = 0, N = 0, K = 0;
  bool c_final = true;
  void* C = nullptr;
  int64_t c_plane_elems = 0;
  LegMap m_dst, n_dst;
  double alpha = 1.0;
  int accumulate = 0;
  int split = 1;             // K split (from tc_split_k); > 1 needs `partial`
  int bn = 0;                // tile width 16/64/128/256; 0: chosen from N
  float* partial = nullptr;  // FP32 scratch [split][N][M] (a second, lo plane in the fixed-point split modes)
  int64_t partial_plane = 0; // fixed-point split modes: floats from the hi to the lo plane of `partial`
};

cudaError_t launch_gemm_tc(const TcGemmArgs& args, cudaStream_t stream);

// Sets bit MERA_ENOTCONV of the device status word unless the Newton-Schulz
// state state[0] says the iteration converged (used where the host cannot
// look, e.g. inside a captured graph).
cudaError_t launch_report_notconv(const int* state, cudaStream_t stream);

// Device status word (bit MERA_ETIMEOUT set when a bounded wait gave up,
// bit MERA_ENOTCONV when a polar update inside a captured graph did not
// converge).
cudaError_t read_device_status(int* status, bool clear);

}  // namespace mera
