// C ABI of the MERA library: argument checks, contraction-program execution,
// the scale-invariant fixed point, the polar update (quintic Newton-Schulz; a
// conditional while loop when recorded into a graph), the Stiefel gradient
// step, the energy, the native sweep driver (SVD or Riemannian updates),
// batched sweeps, recorded sweep graphs and the tile-width autotuner.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <atomic>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/mera.h"
#include "kernels.h"
#include "plan.h"
#include "tc_gemm.h"

namespace mera {

std::atomic<long long> g_launch_count{0};

namespace {

thread_local std::string g_err;

// Optional CUDA-event timing of every GEMM / permute launch, recorded on the
// launching stream.  Off by default; enabling it adds two event records per
// launch and no synchronisation until the totals are read.
struct Profiler {
  std::mutex mu;
  bool on = false;
  struct Rec {
    cudaEvent_t a, b;
    int kind;  // 0 gemm, 1 permute
    int dominant;
    double flops;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void clear() {
    for (auto& r : recs) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
};
Profiler g_prof;

struct ProfScope {
  cudaStream_t s;
  bool on;
  Profiler::Rec rec{};
  ProfScope(cudaStream_t st, int kind, int dominant, double flops) : s(st) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    on = g_prof.on;
    if (!on) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
      on = false;  // no per-step timing inside a captured graph
      return;
    }
    rec.a = g_prof.get();
    rec.b = g_prof.get();
    rec.kind = kind;
    rec.dominant = dominant;
    rec.flops = flops;
    cudaEventRecord(rec.a, s);
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(rec.b, s);
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.recs.push_back(rec);
  }
};

mera_status fail(mera_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

mera_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return MERA_OK;
  return fail(MERA_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
constexpr size_t align_up_const(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
size_t align_up(size_t x) { return align_up_const(x); }

bool chi_ok(int chi_b, int chi_t) {
  return chi_b >= 1 && chi_t >= 1 && chi_b <= MERA_MAX_CHI && chi_t <= MERA_MAX_CHI &&
         int64_t(chi_t) <= int64_t(chi_b) * chi_b;
}
bool prec_ok(int prec) { return prec >= MERA_PREC_F64 && prec <= MERA_PREC_OZ4; }

// Bytes of one element of a program buffer (raw buffers of the fixed-point
// split modes hold binary32 planes).
int64_t buf_elem_bytes(const Buffer& b, int prec) { return b.raw ? 4 : elem_bytes(prec); }

// Tensor-core GEMM arguments of one program step; `out` is the caller's
// output (root steps), `base` the workspace.
TcGemmArgs tc_args(const GemmStep& g, const Program& dg, int prec, char* base, double* out) {
  TcGemmArgs args;
  args.prec = prec;
  const int64_t eb = elem_bytes(prec);
  args.A = base + dg.bufs[g.a_buf].offset + g.a_off * eb;
  args.a_plane_bytes = dg.bufs[g.a_buf].plane_bytes;
  args.lda = g.lda;
  args.B = base + dg.bufs[g.b_buf].offset + g.b_off * eb;
  args.b_plane_bytes = dg.bufs[g.b_buf].plane_bytes;
  args.ldb = g.ldb;
  args.M = g.M;
  args.N = g.N;
  args.K = g.K;
  args.c_final = g.c_buf < 0;
  if (g.c_buf >= 0) {
    const Buffer& c = dg.bufs[g.c_buf];
    const int64_t ce = buf_elem_bytes(c, prec);
    args.C = base + c.offset + g.c_off * ce;
    args.c_plane_elems = c.plane_bytes / ce;
  } else {
    args.C = out + g.c_off;
    args.c_plane_elems = 0;
  }
  args.m_dst = g.m_dst;
  args.n_dst = g.n_dst;
  args.alpha = g.alpha;
  args.accumulate = g.accumulate;
  args.split = g.split;
  args.bn = g.bn;
  if (g.p_buf >= 0) {
    const Buffer& p = dg.bufs[g.p_buf];
    args.partial = reinterpret_cast<float*>(base + p.offset);
    args.partial_plane = p.plane_bytes / 4;
  }
  return args;
}

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Small scratch that reductions need (partials + scalars), bytes.
constexpr size_t kReduceBytes = align_up_const(size_t(4096 + 8) * sizeof(double));

// Bump allocator over the caller's workspace.
struct Arena {
  char* base;
  size_t cap, used = 0;
  char* take(size_t bytes) {
    char* p = base + used;
    used += align_up(bytes);
    return p;
  }
  char* ptr() const { return base + used; }
  size_t left() const { return used <= cap ? cap - used : 0; }
};

// Execute a contraction program; inputs[slot] are device pointers.
// reuse_resident: the u/w operand copies (resident == 1) and the u/w-only
// products left by the previous run of this same program (same u, w,
// workspace) are still valid; skip those steps.
mera_status run_program(const OpProgram& prog, const double* const inputs[4], double* out, int prec, char* ws,
                        cudaStream_t stream, bool reuse_resident = false) {
  for (const Program& dg : prog.diagrams) {
    for (const Step& st : dg.steps) {
      if (st.kind == 0) {
        const PermuteStep& p = st.p;
        const Buffer& b = dg.bufs[p.dst_buf];
        if (p.skip || (reuse_resident && dg.bufs[p.op_buf].resident == 1)) continue;
        const int64_t plane = b.plane_bytes / buf_elem_bytes(b, prec);
        ProfScope ps(stream, 1, 0, 0.0);
        cudaError_t e = launch_permute(p, inputs[p.slot], ws + b.offset, plane, b.raw ? PREC_RAW : prec, stream);
        if (e != cudaSuccess) return cuda_status(e, "permute");
        continue;
      }
      if (st.kind == 2) {  // fixed-point split of a raw buffer into its operand
        const SplitStep& x = st.x;
        const Buffer& r = dg.bufs[x.raw_buf];
        const Buffer& d = dg.bufs[x.dst_buf];
        if (x.skip || (reuse_resident && d.resident == 1)) continue;
        ProfScope ps(stream, 1, 0, 0.0);
        cudaError_t e = launch_oz_split(reinterpret_cast<const float*>(ws + r.offset), r.plane_bytes / 4,
                                        ws + d.offset, d.plane_bytes / elem_bytes(prec), x.rows, x.K, x.ld,
                                        planes(prec), stream);
        if (e != cudaSuccess) return cuda_status(e, "split");
        continue;
      }
      const GemmStep& g = st.g;
      if (reuse_resident && g.stat) continue;  // u/w-only product kept from the previous run
      const Buffer& a = dg.bufs[g.a_buf];
      const Buffer& b = dg.bufs[g.b_buf];
      ProfScope ps(stream, 0, g.dominant, g.flops);
      if (prec == PREC_F64) {
        GemmF64Args args;
        args.A = reinterpret_cast<const double*>(ws + a.offset) + g.a_off;
        args.a_m = g.lda;
        args.a_k = 1;
        args.B = reinterpret_cast<const double*>(ws + b.offset) + g.b_off;
        args.b_n = g.ldb;
        args.b_k = 1;
        args.M = g.M;
        args.N = g.N;
        args.K = g.K;
        args.C = (g.c_buf >= 0 ? reinterpret_cast<double*>(ws + dg.bufs[g.c_buf].offset) : out) + g.c_off;
        args.m_dst = g.m_dst;
        args.n_dst = g.n_dst;
        args.alpha = g.alpha;
        args.accumulate = g.accumulate;
        cudaError_t e = launch_gemm_f64(args, stream);
        if (e != cudaSuccess) return cuda_status(e, "gemm_f64");
      } else {
        const TcGemmArgs args = tc_args(g, dg, prec, ws, out);
        cudaError_t e = launch_gemm_tc(args, stream);
        if (e == cudaErrorNotSupported) return fail(MERA_EINVAL, "tensor-core GEMM unavailable for prec %d", prec);
        if (e != cudaSuccess) return cuda_status(e, "gemm_tc");
      }
    }
  }
  return MERA_OK;
}

// Workspace bytes of each composite operation.
size_t op_bytes(const OpProgram& p) { return align_up(p.ws_bytes); }

mera_status map_call(int op, const double* h, const double* rho, const double* u, const double* w, int chi_b,
                     int chi_t, double* out, int prec, void* ws, size_t ws_bytes, void* stream) {
  if (!chi_ok(chi_b, chi_t)) return fail(MERA_EINVAL, "bad bond dimensions chi_b=%d chi_t=%d", chi_b, chi_t);
  if (!prec_ok(prec)) return fail(MERA_EINVAL, "bad prec %d", prec);
  if (!u || !w || !out) return fail(MERA_EINVAL, "null tensor pointer");
  if ((op == OP_ASCEND || op == OP_ENV_U || op == OP_ENV_W) && !h) return fail(MERA_EINVAL, "null h");
  if ((op == OP_DESCEND || op == OP_ENV_U || op == OP_ENV_W) && !rho) return fail(MERA_EINVAL, "null rho");
  const OpProgram* prog = get_program(op, chi_b, chi_t, prec);
  if (!prog) return fail(MERA_EINVAL, "no contraction program");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (ws_bytes < op_bytes(*prog) || (!ws && op_bytes(*prog) > 0))
    return fail(MERA_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, op_bytes(*prog));
  const double* inputs[4] = {h, rho, u, w};
  return run_program(*prog, inputs, out, prec, static_cast<char*>(ws), static_cast<cudaStream_t>(stream));
}

}  // namespace
}  // namespace mera

using namespace mera;

// ---------------------------------------------------------------------------
extern "C" const char* mera_version(void) { return "mera-gb300 0.1 sm_103a"; }
extern "C" const char* mera_last_error(void) { return g_err.c_str(); }

static mera_status ws_size_impl(int op, int chi_b, int chi_t, int prec, size_t* bytes) {
  if (!bytes) return fail(MERA_EINVAL, "null bytes");
  if (!chi_ok(chi_b, chi_t) || !prec_ok(prec)) return fail(MERA_EINVAL, "bad sizes or prec");
  switch (op) {
    case MERA_OP_ASCEND:
    case MERA_OP_DESCEND:
    case MERA_OP_ENV_U:
    case MERA_OP_ENV_W: {
      const OpProgram* p = get_program(op, chi_b, chi_t, prec);
      if (!p) return fail(MERA_EINVAL, "no contraction program");
      *bytes = op_bytes(*p);
      return MERA_OK;
    }
    case MERA_OP_ENERGY: {
      const OpProgram* p = get_program(OP_ASCEND, chi_b, chi_t, prec);
      if (!p) return fail(MERA_EINVAL, "no contraction program");
      *bytes = op_bytes(*p) + align_up(ipow(chi_t, 6) * sizeof(double)) + kReduceBytes;
      return MERA_OK;
    }
    case MERA_OP_ENERGY_ADJOINT: {
      // transposes of h and rho, an environment half, then the largest map
      size_t maps = 0;
      for (int op2 : {OP_ASCEND, OP_DESCEND, OP_ENV_U, OP_ENV_W}) {
        const OpProgram* p = get_program(op2, chi_b, chi_t, prec);
        if (!p) return fail(MERA_EINVAL, "no contraction program");
        maps = std::max(maps, op_bytes(*p));
      }
      *bytes = align_up(ipow(chi_b, 6) * sizeof(double)) + align_up(ipow(chi_t, 6) * sizeof(double)) +
               align_up(std::max(ipow(chi_b, 4), ipow(chi_b, 2) * chi_t) * sizeof(double)) + maps;
      return MERA_OK;
    }
    case MERA_OP_FIXED_POINT: {
      if (chi_b != chi_t) return fail(MERA_EINVAL, "fixed point needs chi_b == chi_t");
      const OpProgram* p = get_program(OP_DESCEND, chi_b, chi_t, prec);
      if (!p) return fail(MERA_EINVAL, "no contraction program");
      *bytes = op_bytes(*p) + align_up(ipow(chi_t, 6) * sizeof(double)) + kReduceBytes;
      return MERA_OK;
    }
    default:
      return fail(MERA_EINVAL, "unknown op %d", op);
  }
}

extern "C" mera_status mera_workspace_size(int op, int chi_b, int chi_t, int prec, size_t* bytes) {
  return ws_size_impl(op, chi_b, chi_t, prec, bytes);
}

extern "C" mera_status mera_ascend(const double* h, const double* u, const double* w, int chi_b, int chi_t,
                                   double* h_out, int prec, void* ws, size_t ws_bytes, void* stream) {
  if (h_out && h_out == h) return fail(MERA_EINVAL, "h_out aliases h");
  return map_call(OP_ASCEND, h, nullptr, u, w, chi_b, chi_t, h_out, prec, ws, ws_bytes, stream);
}

extern "C" mera_status mera_descend(const double* rho, const double* u, const double* w, int chi_b, int chi_t,
                                    double* rho_out, int prec, void* ws, size_t ws_bytes, void* stream) {
  if (rho_out && rho_out == rho) return fail(MERA_EINVAL, "rho_out aliases rho");
  return map_call(OP_DESCEND, nullptr, rho, u, w, chi_b, chi_t, rho_out, prec, ws, ws_bytes, stream);
}

extern "C" mera_status mera_env_u(const double* h, const double* rho, const double* u, const double* w, int chi_b,
                                  int chi_t, double* env_out, int prec, void* ws, size_t ws_bytes, void* stream) {
  return map_call(OP_ENV_U, h, rho, u, w, chi_b, chi_t, env_out, prec, ws, ws_bytes, stream);
}

extern "C" mera_status mera_env_w(const double* h, const double* rho, const double* u, const double* w, int chi_b,
                                  int chi_t, double* env_out, int prec, void* ws, size_t ws_bytes, void* stream) {
  return map_call(OP_ENV_W, h, rho, u, w, chi_b, chi_t, env_out, prec, ws, ws_bytes, stream);
}

extern "C" mera_status mera_energy(const double* h, const double* rho, const double* u, const double* w, int chi_b,
                                   int chi_t, double* e_dev, int prec, void* ws, size_t ws_bytes, void* stream) {
  size_t need = 0;
  mera_status st = ws_size_impl(MERA_OP_ENERGY, chi_b, chi_t, prec, &need);
  if (st != MERA_OK) return st;
  if (!h || !rho || !u || !w || !e_dev) return fail(MERA_EINVAL, "null pointer");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < need) return fail(MERA_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
  const OpProgram* prog = get_program(OP_ASCEND, chi_b, chi_t, prec);
  Arena ar{static_cast<char*>(ws), ws_bytes};
  char* pws = ar.take(op_bytes(*prog));
  const int64_t n = ipow(chi_t, 3);
  double* a = reinterpret_cast<double*>(ar.take(n * n * sizeof(double)));
  double* partials = reinterpret_cast<double*>(ar.take(kReduceBytes));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double* inputs[4] = {h, nullptr, u, w};
  st = run_program(*prog, inputs, a, prec, pws, s);
  if (st != MERA_OK) return st;
  return cuda_status(launch_dot_transposed(a, rho, n, partials, e_dev, s), "energy dot");
}

extern "C" mera_status mera_fixed_point_rho(const double* u, const double* w, int chi, double* rho_inout, int n_iter,
                                            double* resid_dev, int prec, void* ws, size_t ws_bytes, void* stream) {
  size_t need = 0;
  mera_status st = ws_size_impl(MERA_OP_FIXED_POINT, chi, chi, prec, &need);
  if (st != MERA_OK) return st;
  if (!u || !w || !rho_inout) return fail(MERA_EINVAL, "null pointer");
  if (n_iter < 0) return fail(MERA_EINVAL, "negative n_iter");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < need) return fail(MERA_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_iter == 0) {
    if (resid_dev) return cuda_status(cudaMemsetAsync(resid_dev, 0, sizeof(double), s), "memset");
    return MERA_OK;
  }
  const OpProgram* prog = get_program(OP_DESCEND, chi, chi, prec);
  Arena ar{static_cast<char*>(ws), ws_bytes};
  char* pws = ar.take(op_bytes(*prog));
  const int64_t n = ipow(chi, 3);
  double* tmp = reinterpret_cast<double*>(ar.take(n * n * sizeof(double)));
  double* red = reinterpret_cast<double*>(ar.take(kReduceBytes));
  double* scalars = red + 4096;
  const double* inputs[4] = {nullptr, rho_inout, u, w};
  for (int it = 0; it < n_iter; ++it) {
    // u and w are fixed during the iteration: their operand copies are made once
    st = run_program(*prog, inputs, tmp, prec, pws, s, it > 0);
    if (st != MERA_OK) return st;
    // the residual is reported for the last step only
    cudaError_t e = launch_sym_normalize(tmp, rho_inout, n, red, scalars, it + 1 == n_iter ? resid_dev : nullptr, s);
    if (e != cudaSuccess) return cuda_status(e, "sym_normalize");
  }
  return MERA_OK;
}

// ---------------------------------------------------------------------------
// Polar update.
// ---------------------------------------------------------------------------
static size_t polar_bytes(int m, int n) {
  return 2 * align_up(size_t(m) * n * sizeof(double)) + 3 * align_up(size_t(n) * n * sizeof(double)) +
         kReduceBytes;
}

// Stiefel step: A, S (n x n), T, Yneg (m x n), then the polar update's scratch.
static size_t stiefel_bytes(int m, int n) {
  return 2 * align_up(size_t(n) * n * sizeof(double)) + 2 * align_up(size_t(m) * n * sizeof(double)) +
         polar_bytes(m, n);
}

extern "C" mera_status mera_polar_workspace_size(int m, int n, size_t* bytes) {
  if (!bytes || m < 1 || n < 1 || m < n || m > 1 << 16) return fail(MERA_EINVAL, "bad polar sizes");
  *bytes = polar_bytes(m, n);
  return MERA_OK;
}

// Records the whole polar update on the capturing stream s: scaling, the
// quintic Newton-Schulz steps X <- X ((5/2)(I - G) + G^2), G = X^T X, as a
// conditional while-loop node whose body ends with a kernel that decides on
// the device whether to go on, the result chosen on the device, and
// non-convergence set in the device status word.
static mera_status polar_record(const double* env, int m, int n, double* out, int max_iter, double tol, void* ws,
                                size_t ws_bytes, cudaStream_t s) {
  Arena ar{static_cast<char*>(ws), ws_bytes};
  double* X = reinterpret_cast<double*>(ar.take(size_t(m) * n * sizeof(double)));
  double* Xn = reinterpret_cast<double*>(ar.take(size_t(m) * n * sizeof(double)));
  double* G = reinterpret_cast<double*>(ar.take(size_t(n) * n * sizeof(double)));
  double* G2 = reinterpret_cast<double*>(ar.take(size_t(n) * n * sizeof(double)));
  double* Bm = reinterpret_cast<double*>(ar.take(size_t(n) * n * sizeof(double)));
  double* red = reinterpret_cast<double*>(ar.take(kReduceBytes));
  double* scalars = red + 4096;
  cudaError_t e = launch_frob_scale(env, X, int64_t(m) * n, red, scalars, s);
  if (e != cudaSuccess) return cuda_status(e, "polar init");
  LegMap row_n, col_1, row_m;  // G / Bm (n x n) and X (m x n) destinations
  row_n.n = 1; row_n.dim[0] = n; row_n.stride[0] = n;
  col_1.n = 1; col_1.dim[0] = n; col_1.stride[0] = 1;
  row_m.n = 1; row_m.dim[0] = m; row_m.stride[0] = n;
  // Device-gated iterations: once the residual is below tol, one more step
  // runs and every later kernel returns at once.
  int* state = reinterpret_cast<int*>(scalars + 4);  // done, iterations, converged-after-this-step
  if ((e = cudaMemsetAsync(state, 0, 3 * sizeof(int), s)) != cudaSuccess) return cuda_status(e, "polar state");
  // G = x^T x (skipped once converged)
  auto gram = [&](const double* x, cudaStream_t st) {
    GemmF64Args g;
    g.skip_if = state;
    g.A = x; g.a_m = 1; g.a_k = n;
    g.B = x; g.b_n = 1; g.b_k = n;
    g.M = n; g.N = n; g.K = m;
    g.C = G; g.m_dst = row_n; g.n_dst = col_1; g.alpha = 1.0; g.accumulate = 0;
    return launch_gemm_f64(g, st);
  };
  // One step src -> dst = src ((5/2)(I - G) + G^2), ending with the next
  // step's G.
  auto step = [&](const double* src, double* dst, cudaStream_t st) {
    GemmF64Args q;  // G2 = G G (skipped once converged)
    q.skip_if = state;
    q.A = G; q.a_m = n; q.a_k = 1;
    q.B = G; q.b_n = 1; q.b_k = n;
    q.M = n; q.N = n; q.K = n;
    q.C = G2; q.m_dst = row_n; q.n_dst = col_1; q.alpha = 1.0; q.accumulate = 0;
    cudaError_t r = launch_gemm_f64(q, st);
    if (r != cudaSuccess) return r;
    if ((r = launch_ns_step(G, G2, Bm, n, red, scalars + 1, tol, state, st)) != cudaSuccess) return r;
    GemmF64Args g;
    g.skip_if = state;
    g.A = src; g.a_m = n; g.a_k = 1;
    g.B = Bm; g.b_n = 1; g.b_k = n;
    g.M = m; g.N = n; g.K = n;
    g.C = dst; g.m_dst = row_m; g.n_dst = col_1; g.alpha = 1.0; g.accumulate = 0;
    if ((r = launch_gemm_f64(g, st)) != cudaSuccess) return r;
    if ((r = launch_ns_finish(state, st)) != cudaSuccess) return r;
    return gram(dst, st);
  };
  if ((e = gram(X, s)) != cudaSuccess) return cuda_status(e, "polar gemm");
  if ((e = launch_ns_prescale(G, X, m, n, scalars + 2, s)) != cudaSuccess) return cuda_status(e, "polar prescale");
  // while (not converged and fewer than max_iter steps): X -> Xn -> X
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, &edges, &nd)) != cudaSuccess)
    return cuda_status(e, "capture info");
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return cuda_status(e, "conditional handle");
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t loop = nullptr;
  if ((e = cudaGraphAddNode(&loop, cg, deps, edges, nd, &p)) != cudaSuccess) return cuda_status(e, "while node");
  cudaGraph_t body = p.conditional.phGraph_out[0];
  cudaStream_t bs = nullptr;
  if ((e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_status(e, "body stream");
  e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = step(X, Xn, bs);
  if (e == cudaSuccess) e = step(Xn, X, bs);
  if (e == cudaSuccess) e = launch_ns_continue(state, h, max_iter, bs);
  cudaGraph_t got = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(bs, &got);
  cudaStreamDestroy(bs);
  if (e != cudaSuccess || e2 != cudaSuccess) return cuda_status(e != cudaSuccess ? e : e2, "while body");
  if ((e = cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
      cudaSuccess)
    return cuda_status(e, "capture dependencies");
  e = launch_ns_output(X, Xn, state, out, int64_t(m) * n, s);  // -X of the last step, chosen on the device
  if (e != cudaSuccess) return cuda_status(e, "polar output");
  if ((e = launch_report_notconv(state, s)) != cudaSuccess) return cuda_status(e, "polar report");
  return MERA_OK;
}

namespace mera {
namespace polar_detail {

// Direct (uncaptured) polar updates launch an instantiated recording of the
// same steps, so that the host never waits for the device.  Instantiations
// are cached by everything the recording bakes in: the driver context, the
// pointers, the sizes and the stopping rule.
struct Key {
  void* ctx;
  const double* env;
  double* out;
  void* ws;
  size_t ws_bytes;
  int m, n, max_iter;
  double tol;
  bool operator<(const Key& o) const {
    return std::tie(ctx, env, out, ws, ws_bytes, m, n, max_iter, tol) <
           std::tie(o.ctx, o.env, o.out, o.ws, o.ws_bytes, o.m, o.n, o.max_iter, o.tol);
  }
};
struct Entry {
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernels in the recording
  unsigned long long used = 0;
};
constexpr size_t kMaxEntries = 256;
std::mutex mu;
std::map<Key, Entry> cache;
unsigned long long tick = 0;

}  // namespace polar_detail

// The driver context current on the calling thread (cuCtxGetCurrent through
// the runtime's driver entry point; nullptr if unavailable).
void* current_cu_context() {
  using GetCtx = int (*)(void**);
  static GetCtx fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetCtx>(p);
  });
  void* ctx = nullptr;
  if (fn) fn(&ctx);
  return ctx;
}

}  // namespace mera

extern "C" mera_status mera_polar_update(const double* env, int m, int n, double* out, int max_iter, double tol,
                                         void* ws, size_t ws_bytes, void* stream) {
  using namespace mera::polar_detail;
  if (!env || !out || env == out) return fail(MERA_EINVAL, "bad env/out pointers");
  if (m < 1 || n < 1 || m < n || m > 1 << 16) return fail(MERA_EINVAL, "polar needs m >= n >= 1 (m=%d n=%d)", m, n);
  const size_t need = polar_bytes(m, n);
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < need) return fail(MERA_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (max_iter <= 0) max_iter = 100;
  if (!(tol > 0)) tol = 1e-13 * std::sqrt(double(n));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return fail(MERA_ECUDA, "stream capture status");
  if (cap != cudaStreamCaptureStatusNone) return polar_record(env, m, n, out, max_iter, tol, ws, ws_bytes, s);
  // Direct call: launch the cached instantiation of the recording (made on
  // the first call with these arguments).
  const Key key{current_cu_context(), env, out, ws, ws_bytes, m, n, max_iter, tol};
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it == cache.end()) {
    if (cache.size() >= kMaxEntries) {  // forget the least recently used one
      auto old = cache.begin();
      for (auto c = cache.begin(); c != cache.end(); ++c)
        if (c->second.used < old->second.used) old = c;
      cudaGraphExecDestroy(old->second.exec);  // freed once any launch in flight completes
      cache.erase(old);
    }
    cudaStream_t ps = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_status(e, "polar recording stream");
    const long long l0 = g_launch_count.load();
    e = cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
    mera_status st = e == cudaSuccess ? polar_record(env, m, n, out, max_iter, tol, ws, ws_bytes, ps)
                                      : cuda_status(e, "polar begin capture");
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ps, &g) : cudaSuccess;
    cudaStreamDestroy(ps);
    const long long n_kernels = g_launch_count.load() - l0;
    g_launch_count.fetch_sub(n_kernels);  // counted when launched
    if (st != MERA_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e2 != cudaSuccess || !g) return cuda_status(e2 == cudaSuccess ? cudaErrorUnknown : e2, "polar end capture");
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "polar instantiate");
    it = cache.emplace(key, Entry{x, n_kernels, 0}).first;
  }
  it->second.used = ++tick;
  const cudaError_t e = cudaGraphLaunch(it->second.exec, s);
  if (e != cudaSuccess) return cuda_status(e, "polar launch");
  count_launch(it->second.launches);
  return MERA_OK;
}

extern "C" mera_status mera_stiefel_workspace_size(int m, int n, size_t* bytes) {
  if (!bytes || m < 1 || n < 1 || m < n) return fail(MERA_EINVAL, "bad stiefel sizes");
  *bytes = stiefel_bytes(m, n);
  return MERA_OK;
}

extern "C" mera_status mera_stiefel_step(const double* X, const double* G, int m, int n, double eta, double* out,
                                         void* ws, size_t ws_bytes, void* stream) {
  if (!X || !G || !out || G == out) return fail(MERA_EINVAL, "bad stiefel pointers");
  if (m < 1 || n < 1 || m < n || m > 1 << 16) return fail(MERA_EINVAL, "stiefel step needs m >= n >= 1");
  if (!(eta >= 0.0) || !std::isfinite(eta)) return fail(MERA_EINVAL, "bad step size");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < stiefel_bytes(m, n)) return fail(MERA_ENOMEM, "stiefel workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar{static_cast<char*>(ws), ws_bytes};
  double* A = reinterpret_cast<double*>(ar.take(size_t(n) * n * sizeof(double)));
  double* S = reinterpret_cast<double*>(ar.take(size_t(n) * n * sizeof(double)));
  double* T = reinterpret_cast<double*>(ar.take(size_t(m) * n * sizeof(double)));
  double* Y = reinterpret_cast<double*>(ar.take(size_t(m) * n * sizeof(double)));
  LegMap row_n, col_1, row_m;
  row_n.n = 1; row_n.dim[0] = n; row_n.stride[0] = n;
  col_1.n = 1; col_1.dim[0] = n; col_1.stride[0] = 1;
  row_m.n = 1; row_m.dim[0] = m; row_m.stride[0] = n;
  GemmF64Args g;
  // A = X^T G
  g.A = X; g.a_m = 1; g.a_k = n;
  g.B = G; g.b_n = 1; g.b_k = n;
  g.M = n; g.N = n; g.K = m;
  g.C = A; g.m_dst = row_n; g.n_dst = col_1; g.alpha = 1.0; g.accumulate = 0;
  cudaError_t e = launch_gemm_f64(g, s);
  if (e == cudaSuccess) e = launch_stiefel_sym(A, S, n, s);
  if (e != cudaSuccess) return cuda_status(e, "stiefel sym");
  // T = X S
  g.A = X; g.a_m = n; g.a_k = 1;
  g.B = S; g.b_n = 1; g.b_k = n;
  g.M = m; g.N = n; g.K = n;
  g.C = T; g.m_dst = row_m; g.n_dst = col_1;
  e = launch_gemm_f64(g, s);
  if (e == cudaSuccess) e = launch_stiefel_combine(X, G, T, Y, int64_t(m) * n, eta, s);
  if (e != cudaSuccess) return cuda_status(e, "stiefel combine");
  // retraction: polar(X - eta (G - T)) = -polar_update(-(X - eta (G - T)))
  return mera_polar_update(Y, m, n, out, 0, 0.0, ar.ptr(), ar.left(), stream);
}

// ---------------------------------------------------------------------------
// Sweep.
// ---------------------------------------------------------------------------
namespace mera {
namespace sweep_detail {

struct SweepLayout {
  size_t h_off[MERA_MAX_LAYERS];  // ascended Hamiltonians (layer >= 1)
  size_t rho_off[2];              // ping-pong descended densities
  size_t env_off, etmp_off, red_off, map_off, total;
  size_t map_bytes;
};

mera_status sweep_layout(int n_layers, const int* chi_b, const int* chi_t, int prec, SweepLayout* L) {
  if (n_layers < 1 || n_layers > MERA_MAX_LAYERS) return fail(MERA_EINVAL, "bad n_layers %d", n_layers);
  for (int t = 0; t < n_layers; ++t) {
    if (!chi_ok(chi_b[t], chi_t[t])) return fail(MERA_EINVAL, "bad dims in layer %d", t);
    if (t + 1 < n_layers && chi_t[t] != chi_b[t + 1]) return fail(MERA_EINVAL, "layer dims do not chain at %d", t);
  }
  if (chi_b[n_layers - 1] != chi_t[n_layers - 1]) return fail(MERA_EINVAL, "scale-invariant layer needs chi_b == chi_t");
  if (!prec_ok(prec)) return fail(MERA_EINVAL, "bad prec");
  size_t off = 0, map_bytes = 0, rho_max = 0, env_max = 0;
  for (int t = 0; t < n_layers; ++t) {
    L->h_off[t] = off;
    if (t >= 1) off += align_up(size_t(ipow(chi_b[t], 6)) * sizeof(double));
    rho_max = std::max(rho_max, size_t(ipow(chi_b[t], 6)));
    env_max = std::max(env_max, size_t(ipow(chi_b[t], 4)));
    for (int op : {OP_ASCEND, OP_DESCEND, OP_ENV_U, OP_ENV_W}) {
      const OpProgram* p = get_program(op, chi_b[t], chi_t[t], prec);
      if (!p) return fail(MERA_EINVAL, "no program for layer %d", t);
      map_bytes = std::max(map_bytes, op_bytes(*p));
    }
    const int64_t eb = int64_t(chi_b[t]) * chi_b[t];
    map_bytes = std::max(map_bytes, stiefel_bytes(int(eb), int(eb)));  // >= polar_bytes
    size_t fp = 0;
    if (t == n_layers - 1) {
      ws_size_impl(MERA_OP_FIXED_POINT, chi_b[t], chi_t[t], prec, &fp);
      map_bytes = std::max(map_bytes, fp);
    }
    if (t == 0) {
      ws_size_impl(MERA_OP_ENERGY, chi_b[t], chi_t[t], prec, &fp);
      map_bytes = std::max(map_bytes, fp);
    }
  }
  L->rho_off[0] = off;
  off += align_up(rho_max * sizeof(double));
  L->rho_off[1] = off;
  off += align_up(rho_max * sizeof(double));
  L->env_off = off;
  off += align_up(env_max * sizeof(double));
  L->etmp_off = off;
  off += align_up(sizeof(double) * 2);
  L->red_off = off;
  off += kReduceBytes;
  L->map_off = off;
  L->map_bytes = map_bytes;
  off += map_bytes;
  L->total = off;
  return MERA_OK;
}

__global__ void energy_per_spin_kernel(const double* tr, double shift, double* e) { *e = 0.5 * (*tr + shift); }

}  // namespace sweep_detail
}  // namespace mera

using namespace mera::sweep_detail;

extern "C" mera_status mera_sweep_workspace_size(int n_layers, const int* chi_b, const int* chi_t, int prec,
                                                 size_t* bytes) {
  if (!chi_b || !chi_t || !bytes) return fail(MERA_EINVAL, "null argument");
  SweepLayout L;
  mera_status st = sweep_layout(n_layers, chi_b, chi_t, prec, &L);
  if (st != MERA_OK) return st;
  *bytes = L.total;
  return MERA_OK;
}

// One sweep; update 0: polar (SVD) update of every tensor (Fig. 5); update
// 1: one Riemannian gradient step on the Stiefel manifold with step size
// eta (gradient 2 Gamma), retracted by the polar factor.
static mera_status sweep_impl(mera_state* S, const double* h1, double shift, int n_pow, int prec, void* ws,
                              size_t ws_bytes, double* e_dev, void* stream, int update, double eta) {
  if (!S || !h1 || !e_dev) return fail(MERA_EINVAL, "null argument");
  const int n = S->n_layers;
  SweepLayout L;
  mera_status st = sweep_layout(n, S->chi_b, S->chi_t, prec, &L);
  if (st != MERA_OK) return st;
  for (int t = 0; t < n; ++t)
    if (!S->u[t] || !S->w[t]) return fail(MERA_EINVAL, "null tensor in layer %d", t);
  if (!S->rho_star) return fail(MERA_EINVAL, "null rho_star");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < L.total) return fail(MERA_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
  char* base = static_cast<char*>(ws);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double* hs[MERA_MAX_LAYERS];
  hs[0] = h1;
  for (int t = 1; t < n; ++t) hs[t] = reinterpret_cast<double*>(base + L.h_off[t]);
  void* mws = base + L.map_off;
  const size_t mb = L.map_bytes;
  // 1. ascend the Hamiltonian density through the transitional layers
  for (int t = 0; t + 1 < n; ++t) {
    st = mera_ascend(hs[t], S->u[t], S->w[t], S->chi_b[t], S->chi_t[t], const_cast<double*>(hs[t + 1]), prec, mws,
                     mb, stream);
    if (st != MERA_OK) return st;
  }
  // 2. scale-invariant fixed point (warm start from the state's rho*)
  st = mera_fixed_point_rho(S->u[n - 1], S->w[n - 1], S->chi_t[n - 1], S->rho_star, n_pow, nullptr, prec, mws, mb,
                            stream);
  if (st != MERA_OK) return st;
  // 3./4. updates, scale-invariant layer first, then top-down
  double* env = reinterpret_cast<double*>(base + L.env_off);
  const double* rho_above = S->rho_star;
  int ping = 0;
  for (int t = n - 1; t >= 0; --t) {
    const int cb = S->chi_b[t], ct = S->chi_t[t];
    st = mera_env_u(hs[t], rho_above, S->u[t], S->w[t], cb, ct, env, prec, mws, mb, stream);
    if (st != MERA_OK) return st;
    st = update ? mera_stiefel_step(S->u[t], env, cb * cb, cb * cb, 2.0 * eta, S->u[t], mws, mb, stream)
                : mera_polar_update(env, cb * cb, cb * cb, S->u[t], 0, 0.0, mws, mb, stream);
    if (st != MERA_OK) return st;
    st = mera_env_w(hs[t], rho_above, S->u[t], S->w[t], cb, ct, env, prec, mws, mb, stream);
    if (st != MERA_OK) return st;
    st = update ? mera_stiefel_step(S->w[t], env, cb * cb, ct, 2.0 * eta, S->w[t], mws, mb, stream)
                : mera_polar_update(env, cb * cb, ct, S->w[t], 0, 0.0, mws, mb, stream);
    if (st != MERA_OK) return st;
    if (t > 0 && t < n - 1) {  // rho* sits on top of the last transitional layer
      double* dst = reinterpret_cast<double*>(base + L.rho_off[ping]);
      ping ^= 1;
      st = mera_descend(rho_above, S->u[t], S->w[t], cb, ct, dst, prec, mws, mb, stream);
      if (st != MERA_OK) return st;
      rho_above = dst;
    }
  }
  // 5. energy per spin with the new tensors
  double* etmp = reinterpret_cast<double*>(base + L.etmp_off);
  st = mera_energy(h1, rho_above, S->u[0], S->w[0], S->chi_b[0], S->chi_t[0], etmp, prec, mws, mb, stream);
  if (st != MERA_OK) return st;
  count_launch();
  energy_per_spin_kernel<<<1, 1, 0, s>>>(etmp, shift, e_dev);
  return cuda_status(cudaGetLastError(), "energy per spin");
}

extern "C" mera_status mera_sweep(mera_state* S, const double* h1, double shift, int n_pow, int prec, void* ws,
                                  size_t ws_bytes, double* e_dev, void* stream) {
  return sweep_impl(S, h1, shift, n_pow, prec, ws, ws_bytes, e_dev, stream, 0, 0.0);
}

extern "C" mera_status mera_sweep_riemannian(mera_state* S, const double* h1, double shift, int n_pow, int prec,
                                             double eta, void* ws, size_t ws_bytes, double* e_dev, void* stream) {
  if (!(eta > 0.0) || !std::isfinite(eta)) return fail(MERA_EINVAL, "bad step size");
  return sweep_impl(S, h1, shift, n_pow, prec, ws, ws_bytes, e_dev, stream, 1, eta);
}

// ---------------------------------------------------------------------------
// A sweep recorded once as a CUDA graph and replayed.
// ---------------------------------------------------------------------------
struct mera_graph_s;
extern "C" mera_status mera_graph_launch(mera_graph g, void* stream);
struct mera_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernels in the graph
};

extern "C" mera_status mera_sweep_graph_create(mera_state* S, const double* h1, double shift, int n_pow, int prec,
                                               void* ws, size_t ws_bytes, double* e_dev, void* stream,
                                               mera_graph* out) {
  if (!out) return fail(MERA_EINVAL, "null graph handle");
  *out = nullptr;
  if (!stream) return fail(MERA_EINVAL, "graph capture needs a stream other than the legacy default stream");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e, "begin capture");
  const long long l0 = g_launch_count.load();
  const mera_status st = mera_sweep(S, h1, shift, n_pow, prec, ws, ws_bytes, e_dev, stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (st != MERA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;  // message already recorded
  }
  if (e != cudaSuccess || !g) return cuda_status(e == cudaSuccess ? cudaErrorUnknown : e, "end capture");
  cudaGraphExec_t x = nullptr;
  if ((e = cudaGraphInstantiate(&x, g, 0)) != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e, "graph instantiate");
  }
  auto* h = new mera_graph_s;
  h->graph = g;
  h->exec = x;
  h->launches = g_launch_count.load() - l0;
  g_launch_count.fetch_sub(h->launches);  // counted when replayed
  *out = h;
  return MERA_OK;
}

extern "C" mera_status mera_graph_launch(mera_graph g, void* stream) {
  if (!g || !g->exec) return fail(MERA_EINVAL, "null graph");
  const cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e, "graph launch");
  count_launch(g->launches);
  return MERA_OK;
}

extern "C" mera_status mera_sweep_host(mera_state* S, const double* const* u_host, const double* const* w_host,
                                       const double* rho_host, const double* h1_host, double* h1_dev, double shift,
                                       int n_pow, int prec, void* ws, size_t ws_bytes, double* e_dev, double* e_host,
                                       mera_graph graph, void* stream) {
  if (!S || !u_host || !w_host || !rho_host || !h1_host || !h1_dev || !e_dev || !e_host)
    return fail(MERA_EINVAL, "null argument to mera_sweep_host");
  const int n = S->n_layers;
  if (n < 1 || n > MERA_MAX_LAYERS) return fail(MERA_EINVAL, "bad n_layers %d", n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto up = [&](double* dst, const double* src, int64_t count) {
    return cudaMemcpyAsync(dst, src, size_t(count) * sizeof(double), cudaMemcpyHostToDevice, s);
  };
  cudaError_t e = cudaSuccess;
  for (int t = 0; t < n && e == cudaSuccess; ++t) {
    if (!S->u[t] || !S->w[t] || !u_host[t] || !w_host[t]) return fail(MERA_EINVAL, "null tensor in layer %d", t);
    e = up(S->u[t], u_host[t], ipow(S->chi_b[t], 4));
    if (e == cudaSuccess) e = up(S->w[t], w_host[t], ipow(S->chi_b[t], 2) * S->chi_t[t]);
  }
  if (e == cudaSuccess) e = up(S->rho_star, rho_host, ipow(S->chi_t[n - 1], 6));
  if (e == cudaSuccess) e = up(h1_dev, h1_host, ipow(S->chi_b[0], 6));
  if (e != cudaSuccess) return cuda_status(e, "host to device copies");
  mera_status st = graph ? mera_graph_launch(graph, stream)
                         : mera_sweep(S, h1_dev, shift, n_pow, prec, ws, ws_bytes, e_dev, stream);
  if (st != MERA_OK) return st;
  return cuda_status(cudaMemcpyAsync(e_host, e_dev, sizeof(double), cudaMemcpyDeviceToHost, s), "energy copy");
}

extern "C" mera_status mera_graph_destroy(mera_graph g) {
  if (!g) return MERA_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return MERA_OK;
}

// ---------------------------------------------------------------------------
extern "C" mera_status mera_plan_json(int op, int chi_b, int chi_t, int prec, char* buf, size_t cap, size_t* len) {
  if (!chi_ok(chi_b, chi_t) || !prec_ok(prec) || op < 0 || op > 3) return fail(MERA_EINVAL, "bad arguments");
  const OpProgram* p = get_program(op, chi_b, chi_t, prec);
  if (!p) return fail(MERA_EINVAL, "no contraction program");
  const std::string js = program_json(*p, op, chi_b, chi_t, prec);
  if (len) *len = js.size();
  if (buf && cap > 0) {
    const size_t k = std::min(cap - 1, js.size());
    std::memcpy(buf, js.data(), k);
    buf[k] = '\0';
  }
  return MERA_OK;
}

extern "C" mera_status mera_flops(int op, int chi_b, int chi_t, double* flops) {
  if (!flops || !chi_ok(chi_b, chi_t)) return fail(MERA_EINVAL, "bad arguments");
  int base_op = op;
  if (op == MERA_OP_ENERGY) base_op = OP_ASCEND;
  if (op == MERA_OP_FIXED_POINT) base_op = OP_DESCEND;
  if (base_op < 0 || base_op > 3) return fail(MERA_EINVAL, "bad op");
  const OpProgram* p = get_program(base_op, chi_b, chi_t, MERA_PREC_F64);
  if (!p) return fail(MERA_EINVAL, "no contraction program");
  *flops = p->flops;
  return MERA_OK;
}

// ---------------------------------------------------------------------------
// Instrumentation.
// ---------------------------------------------------------------------------
extern "C" long long mera_launch_count(void) { return g_launch_count.load(); }

extern "C" mera_status mera_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  for (auto& r : g_prof.recs) cudaEventSynchronize(r.b);
  g_prof.clear();
  g_prof.on = on != 0;
  return MERA_OK;
}

extern "C" mera_status mera_profile_read(int kind, long long* launches, double* ms, double* flops) {
  if (kind < 0 || kind > 2) return fail(MERA_EINVAL, "bad profile kind %d", kind);
  std::lock_guard<std::mutex> lk(g_prof.mu);
  long long n = 0;
  double t = 0.0, f = 0.0;
  for (auto& r : g_prof.recs) {
    const bool match = (kind == 0 && r.kind == 0) || (kind == 1 && r.kind == 0 && r.dominant) || (kind == 2 && r.kind == 1);
    if (!match) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_status(e, "profile sync");
    float x = 0.f;
    e = cudaEventElapsedTime(&x, r.a, r.b);
    if (e != cudaSuccess) return cuda_status(e, "profile elapsed");
    ++n;
    t += x;
    f += r.flops;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (flops) *flops = f;
  return MERA_OK;
}

extern "C" mera_status mera_device_status(int* status, int clear) {
  if (!status) return fail(MERA_EINVAL, "null status");
  return cuda_status(read_device_status(status, clear != 0), "device status");
}

extern "C" mera_status mera_gemm_test(int prec, const double* A, const double* B, int M, int N, int K, double* C,
                                      void* ws, size_t ws_bytes, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1) return fail(MERA_EINVAL, "bad gemm test arguments");
  if (!prec_ok(prec)) return fail(MERA_EINVAL, "bad prec");
  const int64_t eb = elem_bytes(prec), np = planes(prec);
  const int64_t ld = (int64_t(K) * eb + 15) / 16 * 16 / eb;
  const size_t pa = align_up(size_t(M) * ld * eb), pb = align_up(size_t(N) * ld * eb);
  // fixed-point split modes: raw hi + lo binary32 planes of both operands first
  const size_t ra = is_oz(prec) ? align_up(size_t(M) * ld * 4) : 0, rb = is_oz(prec) ? align_up(size_t(N) * ld * 4) : 0;
  const size_t need = np * (pa + pb) + 2 * (ra + rb);
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < need) return fail(MERA_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* wa = static_cast<char*>(ws);
  char* wb = wa + np * pa;
  char* wra = wb + np * pb;
  char* wrb = wra + 2 * ra;
  // operands: A row-major M x K, B row-major N x K, copied to padded pitch
  PermuteStep pa_step, pb_step;
  pa_step.rows = M; pa_step.cols = K; pa_step.ld = ld;
  pa_step.row_src.n = 1; pa_step.row_src.dim[0] = M; pa_step.row_src.stride[0] = K;
  pa_step.col_src.n = 1; pa_step.col_src.dim[0] = K; pa_step.col_src.stride[0] = 1;
  pb_step = pa_step;
  pb_step.rows = N; pb_step.row_src.dim[0] = N;
  cudaError_t e = cudaSuccess;
  if (is_oz(prec)) {
    e = launch_permute(pa_step, A, wra, int64_t(ra / 4), PREC_RAW, s);
    if (e == cudaSuccess) e = launch_permute(pb_step, B, wrb, int64_t(rb / 4), PREC_RAW, s);
    if (e == cudaSuccess)
      e = launch_oz_split(reinterpret_cast<const float*>(wra), int64_t(ra / 4), wa, int64_t(pa / eb), M, K, ld, int(np), s);
    if (e == cudaSuccess)
      e = launch_oz_split(reinterpret_cast<const float*>(wrb), int64_t(rb / 4), wb, int64_t(pb / eb), N, K, ld, int(np), s);
  } else {
    e = launch_permute(pa_step, A, wa, int64_t(pa / eb), prec, s);
    if (e == cudaSuccess) e = launch_permute(pb_step, B, wb, int64_t(pb / eb), prec, s);
  }
  if (e != cudaSuccess) return cuda_status(e, "gemm test operands");
  LegMap md, nd;
  md.n = 1; md.dim[0] = M; md.stride[0] = N;
  nd.n = 1; nd.dim[0] = N; nd.stride[0] = 1;
  if (prec == PREC_F64) {
    GemmF64Args g;
    g.A = reinterpret_cast<const double*>(wa); g.a_m = ld; g.a_k = 1;
    g.B = reinterpret_cast<const double*>(wb); g.b_n = ld; g.b_k = 1;
    g.M = M; g.N = N; g.K = K; g.C = C; g.m_dst = md; g.n_dst = nd; g.alpha = 1.0; g.accumulate = 0;
    return cuda_status(launch_gemm_f64(g, s), "gemm test f64");
  }
  TcGemmArgs t;
  t.prec = prec; t.A = wa; t.a_plane_bytes = pa; t.lda = ld; t.B = wb; t.b_plane_bytes = pb; t.ldb = ld;
  t.M = M; t.N = N; t.K = K; t.c_final = true; t.C = C; t.m_dst = md; t.n_dst = nd; t.alpha = 1.0; t.accumulate = 0;
  t.bn = tc_block_n(prec, N);  // the planner's width for this N
  return cuda_status(launch_gemm_tc(t, s), "gemm test tc");
}

namespace mera {
// Records `msg` as the calling thread's last error and returns `st`; for
// entry points defined in other translation units.
mera_status set_last_error(mera_status st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace mera

extern "C" mera_status mera_op_transpose(const double* x, int d, double* out, void* stream) {
  if (!x || !out || x == out) return fail(MERA_EINVAL, "bad transpose pointers");
  if (d < 1 || d > MERA_MAX_CHI) return fail(MERA_EINVAL, "bad local dimension %d", d);
  const int64_t n = ipow(d, 3);
  PermuteStep st;  // out[r][c] = x[c][r]
  st.rows = n;
  st.cols = n;
  st.ld = n;
  st.row_src.n = 1; st.row_src.dim[0] = n; st.row_src.stride[0] = 1;
  st.col_src.n = 1; st.col_src.dim[0] = n; st.col_src.stride[0] = n;
  return cuda_status(launch_permute(st, x, out, 0, PREC_F64, static_cast<cudaStream_t>(stream)), "transpose");
}

extern "C" mera_status mera_energy_adjoint(const double* h, const double* rho, const double* u, const double* w,
                                           int chi_b, int chi_t, const double* g_dev, double* dh, double* drho,
                                           double* du, double* dw, int prec, void* ws, size_t ws_bytes,
                                           void* stream) {
  size_t need = 0;
  mera_status st = ws_size_impl(MERA_OP_ENERGY_ADJOINT, chi_b, chi_t, prec, &need);
  if (st != MERA_OK) return st;
  if (!h || !rho || !u || !w || !g_dev) return fail(MERA_EINVAL, "null input pointer");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < need) return fail(MERA_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Arena ar{static_cast<char*>(ws), ws_bytes};
  const int64_t nb = ipow(chi_b, 6), nt = ipow(chi_t, 6);
  double* ht = reinterpret_cast<double*>(ar.take(nb * sizeof(double)));
  double* rt = reinterpret_cast<double*>(ar.take(nt * sizeof(double)));
  double* half = reinterpret_cast<double*>(ar.take(std::max(ipow(chi_b, 4), ipow(chi_b, 2) * chi_t) * sizeof(double)));
  void* mws = ar.ptr();
  const size_t mb = ar.left();
  if ((st = mera_op_transpose(h, chi_b, ht, stream)) != MERA_OK) return st;
  if ((st = mera_op_transpose(rho, chi_t, rt, stream)) != MERA_OK) return st;
  cudaError_t e = cudaSuccess;
  if (dh) {  // dE/dh = D(rho^T)
    if ((st = mera_descend(rt, u, w, chi_b, chi_t, dh, prec, mws, mb, stream)) != MERA_OK) return st;
    if ((e = launch_scaled_sum(dh, nullptr, g_dev, dh, nb, s)) != cudaSuccess) return cuda_status(e, "scale");
  }
  if (drho) {  // dE/drho = A(h^T)
    if ((st = mera_ascend(ht, u, w, chi_b, chi_t, drho, prec, mws, mb, stream)) != MERA_OK) return st;
    if ((e = launch_scaled_sum(drho, nullptr, g_dev, drho, nt, s)) != cudaSuccess) return cuda_status(e, "scale");
  }
  if (du) {  // dE/du = Gamma_u(h, rho) + Gamma_u(h^T, rho^T)
    if ((st = mera_env_u(h, rho, u, w, chi_b, chi_t, du, prec, mws, mb, stream)) != MERA_OK) return st;
    if ((st = mera_env_u(ht, rt, u, w, chi_b, chi_t, half, prec, mws, mb, stream)) != MERA_OK) return st;
    if ((e = launch_scaled_sum(du, half, g_dev, du, ipow(chi_b, 4), s)) != cudaSuccess) return cuda_status(e, "sum");
  }
  if (dw) {  // dE/dw = Gamma_w(h, rho) + Gamma_w(h^T, rho^T)
    if ((st = mera_env_w(h, rho, u, w, chi_b, chi_t, dw, prec, mws, mb, stream)) != MERA_OK) return st;
    if ((st = mera_env_w(ht, rt, u, w, chi_b, chi_t, half, prec, mws, mb, stream)) != MERA_OK) return st;
    if ((e = launch_scaled_sum(dw, half, g_dev, dw, ipow(chi_b, 2) * chi_t, s)) != cudaSuccess)
      return cuda_status(e, "sum");
  }
  return MERA_OK;
}

extern "C" mera_status mera_sweep_batch(mera_state* states, int n, const double* const* h1, const double* shift,
                                        int n_pow, int prec, void* const* ws, const size_t* ws_bytes, double* e_dev,
                                        void* const* streams, int n_threads) {
  if (!states || n < 1 || !h1 || !shift || !ws || !ws_bytes || !e_dev || !streams)
    return fail(MERA_EINVAL, "null argument to mera_sweep_batch");
  // MERAs on one stream form a group that one host thread issues in index
  // order, so its members run one after another and may share scratch;
  // scratch handed to two streams would be written by concurrent sweeps.
  std::vector<std::vector<int>> groups;
  std::map<void*, size_t> group_of;
  std::map<void*, void*> stream_of_ws;
  for (int i = 0; i < n; ++i) {
    auto w = stream_of_ws.emplace(ws[i], streams[i]);
    if (!w.second && w.first->second != streams[i])
      return fail(MERA_EINVAL, "MERA %d: its scratch is also used on another stream", i);
    auto g = group_of.emplace(streams[i], groups.size());
    if (g.second) groups.emplace_back();
    groups[g.first->second].push_back(i);
  }
  n_threads = std::max(1, std::min(n_threads, int(groups.size())));
  std::vector<mera_status> st(static_cast<size_t>(n), MERA_OK);
  std::vector<std::string> msg(static_cast<size_t>(n));
  int dev = 0;
  cudaGetDevice(&dev);
  auto worker = [&](int t) {
    cudaSetDevice(dev);  // host threads start on device 0
    for (size_t g = size_t(t); g < groups.size(); g += size_t(n_threads))
      for (int i : groups[g]) {
        st[size_t(i)] = mera_sweep(&states[i], h1[i], shift[i], n_pow, prec, ws[i], ws_bytes[i], e_dev + i,
                                   streams[i]);
        if (st[size_t(i)] != MERA_OK) msg[size_t(i)] = g_err;
      }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < n_threads; ++t) pool.emplace_back(worker, t);
  worker(0);
  for (auto& th : pool) th.join();
  mera_status worst = MERA_OK;
  for (int i = 0; i < n; ++i) {
    if (st[size_t(i)] == MERA_OK) continue;
    if (worst == MERA_OK || (worst == MERA_ENOTCONV && st[size_t(i)] != MERA_ENOTCONV)) {
      worst = st[size_t(i)];
      g_err = "MERA " + std::to_string(i) + ": " + msg[size_t(i)];
    }
  }
  return worst;
}

// Contraction flops of one sweep (the stages of sweep_impl): per transitional
// layer an ascent of h, both environments, and a descent of rho (the bottom
// layer's last map is the energy, an ascent's network); the scale-invariant
// layer adds n_pow descents for rho*.
static double sweep_flops(int n, const int* cb, const int* ct, int n_pow) {
  double tot = 0.0;
  for (int k = 0; k < n; ++k) {
    double f[4] = {0, 0, 0, 0};
    for (int op = OP_ASCEND; op <= OP_ENV_W; ++op) {
      const OpProgram* p = get_program(op, cb[k], ct[k], MERA_PREC_F64);
      f[op] = p ? p->flops : 0.0;
    }
    tot += f[OP_ENV_U] + f[OP_ENV_W];
    if (k + 1 < n) tot += f[OP_ASCEND] + (k == 0 ? f[OP_ASCEND] : f[OP_DESCEND]);
    else tot += double(n_pow) * f[OP_DESCEND];
  }
  return tot;
}

// Lanes of a batch.  A MERA whose sweep alone fills the GPU (at least
// kFillFlops contraction flops: its GEMMs are persistent kernels over every
// SM, and two of them side by side only contend for the SMs and L2) joins
// one shared lane, so those run back to back.  The others get
// longest-processing-time-first list scheduling under a cap on the summed
// scratch: taken by decreasing scratch size (then cost), each opens a lane
// while lanes and budget remain, else joins the least-loaded lane among
// those whose scratch holds it or can grow to hold it within the budget.
// (A lane opened by a later MERA is never smaller than it; the shared lane
// of the GPU-filling MERAs can be, when a MERA with few flops has a large
// transitional layer.)
extern "C" mera_status mera_batch_lanes(int n, int n_layers, const int* chi_b, const int* chi_t, int prec, int n_pow,
                                        size_t budget_bytes, int max_lanes, int* lane, int* n_lanes,
                                        size_t* lane_bytes) {
  if (n < 1 || n_layers < 1 || n_layers > MERA_MAX_LAYERS || !chi_b || !chi_t || n_pow < 0 || max_lanes < 1 ||
      !lane || !n_lanes || !lane_bytes)
    return fail(MERA_EINVAL, "bad arguments to mera_batch_lanes");
  std::vector<size_t> need(static_cast<size_t>(n));
  std::vector<double> cost(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) {
    const int* cb = chi_b + size_t(i) * size_t(n_layers);
    const int* ct = chi_t + size_t(i) * size_t(n_layers);
    SweepLayout L;
    const mera_status st = sweep_layout(n_layers, cb, ct, prec, &L);
    if (st != MERA_OK) {
      g_err = "MERA " + std::to_string(i) + ": " + g_err;
      return st;
    }
    need[size_t(i)] = L.total;
    cost[size_t(i)] = sweep_flops(n_layers, cb, ct, n_pow);
  }
  std::vector<int> order(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) order[size_t(i)] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (need[size_t(a)] != need[size_t(b)]) return need[size_t(a)] > need[size_t(b)];
    return cost[size_t(a)] > cost[size_t(b)];
  });
  std::vector<size_t> bytes;
  std::vector<double> load;
  size_t used = 0;
  // a chi = 20 sweep (1.2e14) is GEMM-bound throughout; a chi = 16 one (2.0e13) still has latency-bound parts
  // (polar updates, small GEMMs) that overlap with other lanes
  constexpr double kFillFlops = 1e14;
  size_t big_need = 0;
  double big_load = 0.0;
  for (int i = 0; i < n; ++i)
    if (cost[size_t(i)] >= kFillFlops) {
      big_need = std::max(big_need, need[size_t(i)]);
      big_load += cost[size_t(i)];
    }
  if (big_need > 0) {  // the shared lane of the GPU-filling MERAs is lane 0
    if (big_need > budget_bytes)
      return fail(MERA_ENOMEM, "a MERA needs %zu bytes of scratch; the budget is %zu", big_need, budget_bytes);
    bytes.push_back(big_need);
    load.push_back(big_load);
    used = big_need;
  }
  for (int i : order) {
    const size_t b = need[size_t(i)];
    if (cost[size_t(i)] >= kFillFlops) {
      lane[i] = 0;
      continue;
    }
    if (int(bytes.size()) < max_lanes && b <= budget_bytes - used) {
      lane[i] = int(bytes.size());
      bytes.push_back(b);
      load.push_back(cost[size_t(i)]);
      used += b;
      continue;
    }
    size_t best = bytes.size();
    for (size_t l = 0; l < bytes.size(); ++l) {
      const size_t grow = b > bytes[l] ? b - bytes[l] : 0;
      if (grow > budget_bytes - used) continue;
      if (best == bytes.size() || load[l] < load[best]) best = l;
    }
    if (best == bytes.size())
      return fail(MERA_ENOMEM, "MERA %d needs %zu bytes of scratch; no lane holds it within the budget of %zu", i,
                  b, budget_bytes);
    if (b > bytes[best]) {
      used += b - bytes[best];
      bytes[best] = b;
    }
    lane[i] = int(best);
    load[best] += cost[size_t(i)];
  }
  *n_lanes = int(bytes.size());
  for (size_t l = 0; l < bytes.size(); ++l) lane_bytes[l] = bytes[l];
  return MERA_OK;
}

// Tile-width autotuner: every tensor-core GEMM step of the op's program that
// has more than one sensible width (N > 64) and no K split is timed with each
// width on the program's own buffers, and the fastest is recorded for that
// step shape; later programs use it.
extern "C" mera_status mera_autotune(int op, int chi_b, int chi_t, int prec, double* out_scratch,
                                     size_t out_elems, void* ws, size_t ws_bytes, void* stream, int* n_tuned) {
  if (!chi_ok(chi_b, chi_t)) return fail(MERA_EINVAL, "bad bond dimensions");
  if (prec == PREC_F64 || !prec_ok(prec)) return fail(MERA_EINVAL, "autotuning needs a tensor-core mode");
  if (op < OP_ASCEND || op > OP_ENV_W) return fail(MERA_EINVAL, "unknown op %d", op);
  const OpProgram* prog = get_program(op, chi_b, chi_t, prec);
  if (!prog) return fail(MERA_EINVAL, "no contraction program");
  const size_t out_need = size_t(op == OP_ASCEND ? ipow(chi_t, 6)
                                 : op == OP_DESCEND ? ipow(chi_b, 6)
                                 : op == OP_ENV_U ? ipow(chi_b, 4) : ipow(chi_b, 2) * chi_t);
  if (!out_scratch || out_elems < out_need) return fail(MERA_EINVAL, "output scratch too small");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(MERA_EINVAL, "workspace not 256-byte aligned");
  if (!ws || ws_bytes < op_bytes(*prog)) return fail(MERA_ENOMEM, "workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  struct Pick { int prec; int64_t M, N, K; int cf; int bn; };
  std::vector<Pick> picks;
  std::set<std::tuple<int64_t, int64_t, int64_t, int>> seen;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(MERA_ECUDA, "events");
  mera_status st = MERA_OK;
  for (const Program& dg : prog->diagrams) {
    for (const Step& stp : dg.steps) {
      if (stp.kind != 1) continue;
      const GemmStep& g = stp.g;
      const int cf = g.c_buf < 0 ? 1 : 0;
      if (g.N <= 64 || g.split > 1 || !seen.insert({g.M, g.N, g.K, cf}).second) continue;
      std::vector<int> cands = {128, 64};
      if (g.N > 128 && prec != PREC_BF16X6 && !is_oz(prec)) cands.insert(cands.begin(), {256, 192, 160});
      // the planner's own choice wins unless another width is clearly (3 %)
      // faster: single-step timings on scratch data carry noise
      const int heur = tc_block_n(prec, g.N);
      int best = 0;
      float best_ms = 0.0f, heur_ms = 0.0f;
      for (int bn : cands) {
        if (tc_split_k(prec, g.M, g.N, g.K, bn) > 1) continue;  // timed only without a K split
        TcGemmArgs a = tc_args(g, dg, prec, base, out_scratch);
        a.accumulate = 0;
        a.split = 1;
        a.partial = nullptr;
        a.bn = bn;
        cudaError_t e = launch_gemm_tc(a, s);  // warm
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = launch_gemm_tc(a, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          st = cuda_status(e, "autotune launch");
          break;
        }
        if (bn == heur) heur_ms = ms;
        if (best == 0 || ms < best_ms) {
          best = bn;
          best_ms = ms;
        }
      }
      if (st != MERA_OK) break;
      if (best && heur_ms > 0.0f && best != heur && best_ms > 0.97f * heur_ms) best = heur;
      if (best) picks.push_back({prec, g.M, g.N, g.K, cf, best});
    }
    if (st != MERA_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MERA_OK) return st;
  for (const Pick& p : picks) set_tuned_tile(p.prec, p.M, p.N, p.K, p.cf, p.bn);
  if (n_tuned) *n_tuned = int(picks.size());
  return MERA_OK;
}

extern "C" mera_status mera_autotune_reset(void) {
  clear_tuned_tiles();
  return MERA_OK;
}

// Recorded widths set or read directly: the autotuner's candidates only.
extern "C" mera_status mera_set_tile_width(int prec, long long M, long long N, long long K, int c_final, int bn) {
  if (!prec_ok(prec) || prec == PREC_F64) return fail(MERA_EINVAL, "tile widths apply to the tensor-core modes");
  if (M < 1 || N < 1 || K < 1 || (c_final != 0 && c_final != 1)) return fail(MERA_EINVAL, "bad GEMM shape");
  if (bn != 0) {
    const bool wide = prec != PREC_BF16X6 && !is_oz(prec);
    const bool ok = N > 128  ? (bn == 128 || bn == 64 || (wide && (bn == 256 || bn == 192 || bn == 160)))
                    : N > 64 ? (bn == 128 || bn == 64)
                             : false;
    if (!ok) return fail(MERA_EINVAL, "width %d is not an autotuner candidate for N = %lld", bn, N);
  }
  set_tuned_tile(prec, M, N, K, c_final, bn);
  return MERA_OK;
}

extern "C" mera_status mera_tile_widths(long long* out, int cap, int* n) {
  if (!n || cap < 0 || (cap > 0 && !out)) return fail(MERA_EINVAL, "bad arguments");
  const std::vector<std::vector<int64_t>> v = tuned_tiles();
  *n = int(v.size());
  for (size_t i = 0; i < v.size() && int(i) < cap; ++i)
    for (size_t j = 0; j < 6; ++j) out[6 * i + j] = static_cast<long long>(v[i][j]);
  return MERA_OK;
}

extern "C" mera_status mera_set_slice_bytes(size_t bytes) {
  set_slice_bytes(bytes);
  return MERA_OK;
}
