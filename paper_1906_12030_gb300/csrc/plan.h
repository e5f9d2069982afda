// Contraction programs of the binary-MERA diagrams (Fig. 4, Fig. A1).
//
// Each diagram is a closed tensor network with a few open legs.  The planner
// picks a pairwise contraction order by exhaustive dynamic programming over
// subsets (minimum flops, intermediates of rank <= 7), then fixes the memory
// layout of every intermediate so that its consumer reads it as a plain
// row-major matrix [free legs | contracted legs].  The producing GEMM writes
// its result straight into that layout (a scatter epilogue), so no transpose
// pass runs between contractions; only the caller's input tensors are copied
// once into operand layout (fused with the cast to the operand precision).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace mera {

enum Prec : int {
  PREC_F64 = 0,
  PREC_TF32 = 1,
  PREC_BF16 = 2,
  PREC_BF16X3 = 3,
  PREC_BF16X6 = 4,
  PREC_OZ3 = 5,  // fixed-point split into 3 BF16 slices per 256-element block of K, exact block sums
  PREC_OZ4 = 6,  // the same with 4 slices
  PREC_LAST = PREC_OZ4,
  // Not a mode: the storage format that the fixed-point split modes write
  // first (an unevaluated pair hi + lo of binary32 planes), before the split.
  PREC_RAW = 100
};
inline bool is_oz(int prec) { return prec == PREC_OZ3 || prec == PREC_OZ4; }
// K elements over which a fixed-point split shares one exponent per row; the
// GEMM sums the leading slice products of such a block exactly in FP32.
constexpr int kOzBlockK = 256;
enum Slot : int { SLOT_OP = 0, SLOT_RHO = 1, SLOT_U = 2, SLOT_W = 3 };
enum Op : int { OP_ASCEND = 0, OP_DESCEND = 1, OP_ENV_U = 2, OP_ENV_W = 3 };

constexpr int kMaxLeg = 8;

// Linear index -> element offset.  The index is decomposed over `n` legs,
// the last leg varying fastest; offset = sum idx_l * stride_l.
struct LegMap {
  int n = 0;
  int64_t dim[kMaxLeg] = {};
  int64_t stride[kMaxLeg] = {};
};

// Copy (and cast) an input tensor into operand layout:
// dst[r * ld + c] = src[row_src(r) + col_src(c)],  r < rows, c < cols.
struct PermuteStep {
  int slot = 0;
  int dst_buf = 0;     // the operand buffer, or (fixed-point split modes) its raw buffer
  int op_buf = 0;      // the operand buffer (== dst_buf unless a split step follows)
  int64_t rows = 0, cols = 0, ld = 0;
  int skip = 0;  // an earlier step of the same call already made this copy
  LegMap row_src, col_src;
};

// C[m, n] (+)= alpha * sum_k A[m*lda + k] * B[n*ldb + k], scattered to
// dst + m_dst(m) + n_dst(n).  c_buf == -1 targets the caller's output.
struct GemmStep {
  int a_buf = 0, b_buf = 0;
  int64_t M = 1, N = 1, K = 1, lda = 1, ldb = 1;
  int c_buf = -1;
  int64_t c_ld = 0;  // row pitch of the destination when it is an operand buffer
  LegMap m_dst, n_dst;
  double alpha = 1.0;
  int accumulate = 0;
  double flops = 0.0;
  int dominant = 0;   // one of the chi^9-class steps of its diagram
  int split = 1;      // K split over this many CTAs (tensor-core modes; partials summed by a TwoSum pair)
  int bn = 0;         // tensor-core tile width (16, 64, 128 or 256); 0 for the FP64 kernel
  int64_t a_off = 0, b_off = 0, c_off = 0;  // element offsets into A, B and the destination (slices)
  int p_buf = -1;     // FP32 partial-sum buffer [split][N][M] when split > 1
  int stat = 0;       // reads only u and w (directly or through such steps): its output is kept
                      // for the call, and a later run with the same u, w may skip the step
  std::string label;  // e.g. "aceiq*CDcdil->ADadelq" for inspection
};

// Fixed-point split modes: raw (hi + lo binary32 planes, written by a
// permute or GEMM step) -> S BF16 slice planes of the operand buffer, the
// exponent shared by each row's blocks of kOzBlockK elements along K.
struct SplitStep {
  int raw_buf = 0, dst_buf = 0;
  int64_t rows = 0, K = 0, ld = 0;
  int skip = 0;  // mirrors the skip of the permute step it follows
};

struct Step {
  int kind = 0;  // 0 permute, 1 gemm, 2 split (fixed-point split modes)
  PermuteStep p;
  GemmStep g;
  SplitStep x;
};

struct Buffer {
  int64_t rows = 0, ld = 0;   // operand matrix rows x pitch (elements per plane)
  int64_t offset = 0;         // byte offset in the workspace
  int64_t plane_bytes = 0;    // bytes of one plane (BF16X3 keeps hi, then lo)
  int64_t bytes = 0;          // plane_bytes * planes
  int raw = 0;                // 1: raw buffer of a fixed-point split mode (hi, lo binary32 planes)
  int resident = 0;           // kept for the whole call, outside the transient arena:
                              // 1 copy of a disentangler/isometry (a later call with the
                              // same u, w may reuse it), 2 copy of h or rho that several
                              // diagrams read in the same layout
};

// The program of one diagram.  Buffers are laid out in one arena.
struct Program {
  std::vector<Step> steps;
  std::vector<Buffer> bufs;
  size_t ws_bytes = 0;        // transient arena bytes (resident buffers excluded)
  size_t resident_bytes = 0;  // bytes of the resident buffers
  double flops = 0.0;
  int out_rank = 0;
};

// A whole operation (sum of diagrams, each scaled by alpha, the first one
// overwriting the output and the others accumulating).
struct OpProgram {
  std::vector<Program> diagrams;
  size_t ws_bytes = 0;
  size_t persistent_bytes = 0;  // leading workspace bytes holding the resident copies
  double flops = 0.0;
};

int elem_bytes(int prec);   // storage bytes of one operand element (one plane)
// Output-tile width of the tensor-core GEMM for an N-column product.
int tc_block_n(int prec, int64_t N);
// K split of a tensor-core GEMM: > 1 when too few output tiles would leave
// most SMs idle and K is long (each split keeps >= 4 k-blocks).
int tc_split_k(int prec, int64_t M, int64_t N, int64_t K, int bn = 0);

// Tile width of a tensor-core GEMM step: a width recorded by the autotuner
// for this (prec, M, N, K, caller-format output) if any, else tc_block_n.
int tc_tile_n(int prec, int64_t M, int64_t N, int64_t K, int c_final);
// Records a tuned width (0 forgets it) and discards the cached programs.
void set_tuned_tile(int prec, int64_t M, int64_t N, int64_t K, int c_final, int bn);
void clear_tuned_tiles();
int tuned_tile_count();
// Every recorded width as (prec, M, N, K, c_final, width), in key order.
std::vector<std::vector<int64_t>> tuned_tiles();
int planes(int prec);       // 2 for BF16X3 (hi, lo), 3 for BF16X6 (hi, mid, lo), 3 / 4 for OZ3 / OZ4, else 1

// Builds (and caches) the program; thread safe.  Returns nullptr on bad input.
const OpProgram* get_program(int op, int chi_b, int chi_t, int prec);

std::string program_json(const OpProgram& prog, int op, int chi_b, int chi_t, int prec);

// Rank-7 intermediates larger than this many bytes are sliced over one leg
// (the pair of chi^9 GEMMs around them runs once per value of that leg, on
// a one-slice buffer).  Setting it clears the program cache.
void set_slice_bytes(size_t bytes);
size_t slice_bytes();

}  // namespace mera
