/*
 * mera.h -- C ABI of the GB300 (sm_103a) library for the scale-invariant
 * binary MERA of arXiv:1906.12030 ("TensorNetwork on TensorFlow:
 * Entanglement Renormalization for quantum critical lattice models").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Real arithmetic in IEEE binary64 at the boundary.  The Ising Hamiltonian
 *   (Eq. ham, Sec. II A) is real, so the complex conjugations of Eq. (iso)
 *   and Eq. (unitarity) drop out.
 * - Tensors are C-contiguous (row-major) with these leg orders:
 *     w[a][b][c]        isometry, a,b lower (fine) legs of size chi_b,
 *                       c upper (coarse) leg of size chi_t;   Eq. (iso)
 *     u[a][b][m][n]     disentangler, a,b lower legs, m,n upper legs, all
 *                       of size chi_b;                        Eq. (unitarity)
 *     X[i1][i2][i3][j1][j2][j3]
 *                       3-site operator (Hamiltonian density h or reduced
 *                       density matrix rho): ket legs, then bra legs.
 *   As matrices: w is (chi_b^2) x chi_t, u is (chi_b^2) x (chi_b^2), X is
 *   (d^3) x (d^3).
 * - Unless a parameter says "host", every tensor pointer is a DEVICE pointer
 *   owned by the caller (for example allocated through PyTorch).  Inputs are
 *   read-only.  Outputs must not alias inputs unless stated.
 * - Every compute call is asynchronous on the given stream (NULL = the legacy
 *   default stream).  Returned status codes report argument errors detected on
 *   the host and launch errors; results are valid once the stream is
 *   synchronised.
 * - Scratch memory is the caller's: `ws` must hold at least the byte count
 *   reported by mera_workspace_size for the same operation and sizes, and be
 *   256-byte aligned.  Apart from a status word and the fixed static array
 *   behind mera_ascend_noalloc, the library holds no device memory.
 * - prec selects the arithmetic of the contractions (the O(chi^9) part):
 *     MERA_PREC_F64    binary64 everywhere (FP64 units),
 *     MERA_PREC_TF32   tensor cores, TF32 operands, FP32 accumulation,
 *     MERA_PREC_BF16   tensor cores, BF16 operands, FP32 accumulation,
 *     MERA_PREC_BF16X3 tensor cores, each operand split into a BF16 pair
 *                      (hi + lo), three products hi*hi + hi*lo + lo*hi,
 *                      FP32 accumulation.
 *     MERA_PREC_BF16X6 tensor cores, each operand split into three BF16
 *                      parts (hi + mid + lo, 24 significant bits), the six
 *                      products whose parts' orders sum to at most 2, FP32
 *                      accumulation.
 *     MERA_PREC_OZ3    tensor cores, fixed-point split (Ozaki, Ogita, Oishi
 *                      and Rump, Numer. Algorithms 59, 2012): along the
 *                      contraction index every row of an operand is cut into
 *                      blocks of 256 elements sharing one exponent, and each
 *                      entry into three BF16 slices of 9 bits each relative
 *                      to the block's largest entry (~26 bits).  Within a
 *                      block the leading-slice products sum exactly in FP32;
 *                      block sums are accumulated as a pair of binary32
 *                      values (~48 bits); the six slice products whose
 *                      orders sum to at most 2 are kept.  Intermediates are
 *                      stored as that pair and split again.  Map errors of
 *                      ~1e-8 of the largest entry.
 *     MERA_PREC_OZ4    the same with four slices (~35 bits) and ten
 *                      products; map errors of ~1e-9.
 *   Polar updates, normalisation, traces and energies are binary64 always.
 */
#ifndef MERA_GB300_H
#define MERA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mera_status;
#define MERA_OK 0
#define MERA_EINVAL 1    /* bad size, pointer, alignment or mode            */
#define MERA_ENOMEM 2    /* workspace smaller than mera_workspace_size      */
#define MERA_ECUDA 3     /* CUDA launch / runtime error                     */
#define MERA_ENOTCONV 4  /* iteration cap reached; output still written     */
#define MERA_ETIMEOUT 5  /* a bounded device-side wait gave up              */

#define MERA_PREC_F64 0
#define MERA_PREC_TF32 1
#define MERA_PREC_BF16 2
#define MERA_PREC_BF16X3 3
#define MERA_PREC_BF16X6 4
#define MERA_PREC_OZ3 5
#define MERA_PREC_OZ4 6

/* Operation ids for mera_workspace_size / mera_plan_json. */
#define MERA_OP_ASCEND 0
#define MERA_OP_DESCEND 1
#define MERA_OP_ENV_U 2
#define MERA_OP_ENV_W 3
#define MERA_OP_ENERGY 4
#define MERA_OP_FIXED_POINT 5
#define MERA_OP_ENERGY_ADJOINT 6

/* Largest bond dimension accepted by any entry point. */
#define MERA_MAX_CHI 64
/* Most layers a mera_state may hold (tau* <= MERA_MAX_LAYERS). */
#define MERA_MAX_LAYERS 8

/* Library version string, e.g. "mera-gb300 0.1 sm_103a". */
const char* mera_version(void);

/* Text of the last error reported on the calling thread ("" if none). */
const char* mera_last_error(void);

/*
 * Scratch bytes needed by one call of `op` (MERA_OP_*) with lower bond
 * dimension chi_b, upper bond dimension chi_t and mode prec.  For
 * MERA_OP_FIXED_POINT chi_b == chi_t == chi.  Writes the count to *bytes.
 * Returns MERA_EINVAL for an unknown op/prec, chi outside [1, MERA_MAX_CHI],
 * chi_t > chi_b^2, or a NULL `bytes`.
 */
mera_status mera_workspace_size(int op, int chi_b, int chi_t, int prec, size_t* bytes);

/*
 * Ascending superoperator (Fig. 4a, Sec. II B): h_out = A(h) =
 * (A_even(h) + A_odd(h)) / 2, the 3-site operator h on the lattice below a
 * layer (u, w) lifted to the lattice above it.  A_even places h on the right
 * lower leg of one disentangler and both lower legs of the next; A_odd on
 * both lower legs of one and the left lower leg of the next.
 *   h      [chi_b^6]  input operator (any real operator, not only symmetric)
 *   u      [chi_b^4]  disentangler of the layer
 *   w      [chi_b^2 * chi_t] isometry of the layer
 *   h_out  [chi_t^6]  output, overwritten; must not alias h
 */
mera_status mera_ascend(const double* h, const double* u, const double* w, int chi_b, int chi_t,
                        double* h_out, int prec, void* ws, size_t ws_bytes, void* stream);

/*
 * Descending superoperator (Fig. 4b, Sec. II B): rho_out = D(rho) =
 * (D_even(rho) + D_odd(rho)) / 2, the Hilbert-Schmidt adjoint of A:
 * <A(h), rho> = <h, D(rho)> with <X,Y> = sum_ij X_ij Y_ij.
 *   rho     [chi_t^6]  3-site operator on the lattice above the layer
 *   rho_out [chi_b^6]  output on the lattice below, overwritten
 */
mera_status mera_descend(const double* rho, const double* u, const double* w, int chi_b, int chi_t,
                         double* rho_out, int prec, void* ws, size_t ws_bytes, void* stream);

/*
 * Scale-invariant fixed point (Sec. II B: rho* is the dominant eigenvector of
 * the scale-invariant descending superoperator, found by an iterative
 * method).  Runs n_iter power steps  rho <- S(D(rho)) / tr S(D(rho)),  with
 * S(X) = (X + X^T)/2 exchanging the ket and bra triples, in place.
 *   u, w       SI-layer tensors with chi_b = chi_t = chi
 *   rho_inout  [chi^6] start vector on entry (e.g. identity / chi^3, or the
 *              previous sweep's rho*), the iterate on return
 *   resid_dev  device double: ||rho_k - rho_{k-1}||_F of the last step
 *              (0 if n_iter == 0); may be NULL
 * Normalisation, symmetrisation and the residual are binary64 in every mode.
 */
mera_status mera_fixed_point_rho(const double* u, const double* w, int chi, double* rho_inout,
                                 int n_iter, double* resid_dev, int prec, void* ws,
                                 size_t ws_bytes, void* stream);

/*
 * Environment of the disentangler (Fig. 4d, Fig. A1b, Sec. II C): half the
 * sum of the four networks of E = tr(A(h) rho) with one bra-side
 * disentangler removed (two per causal-cone position).  For symmetric h and
 * rho, dE/du = 2 * env.
 *   h       [chi_b^6] operator below the layer;  rho [chi_t^6] above it
 *   env_out [chi_b^4] output in u's leg order, overwritten
 */
mera_status mera_env_u(const double* h, const double* rho, const double* u, const double* w,
                       int chi_b, int chi_t, double* env_out, int prec, void* ws, size_t ws_bytes,
                       void* stream);

/*
 * Environment of the isometry (Fig. 4c, Fig. A1a): half the sum of the six
 * networks of E with one bra-side isometry removed (three per position).
 * dE/dw = 2 * env for symmetric h and rho.
 *   env_out [chi_b^2 * chi_t] output in w's leg order, overwritten
 */
mera_status mera_env_w(const double* h, const double* rho, const double* u, const double* w,
                       int chi_b, int chi_t, double* env_out, int prec, void* ws, size_t ws_bytes,
                       void* stream);

/*
 * Update (Fig. 5, Sec. II C): out = -polar(env) = -U V^T where the m x n
 * matrix env (row-major; rows = lower legs, columns = upper legs) has the
 * thin SVD U S V^T.  Requires m >= n >= 1.  Binary64, computed on the device
 * by a quintic Newton-Schulz iteration X <- X ((5/2)(I - G) + G^2), G = X^T X
 * (every singular value x -> (5/2) x - (5/2) x^3 + x^5), from
 * X0 = env / ||env||_F rescaled so that every singular value is at most 1;
 * it converges quadratically to the polar factor for full column rank, and
 * a singular value 1e-38 of the largest reaches 1 within 100 steps.  An
 * exactly rank-deficient env has no unique polar factor: its null space stays
 * at zero.  Stops when ||X^T X - I||_F <= tol (tol <= 0 selects 1e-13 * sqrt(n))
 * or after max_iter steps (<= 0 selects 100); in the latter case the last
 * iterate is written and bit (1 << MERA_ENOTCONV) of the device status word
 * is set (mera_device_status).  Asynchronous like every compute call: the
 * steps run as a conditional while loop whose continuation the device
 * decides, so the host never waits.  The first call with a given (env, out,
 * ws, ws_bytes, m, n, max_iter, tol) in a CUDA context records and
 * instantiates that loop (host work only, no synchronisation) and keeps it
 * (at most 256 such instantiations, the least recently used one discarded);
 * later calls with the same arguments launch it.  Inside a stream capture
 * the loop is recorded into the caller's graph instead.  out [m*n] must not
 * alias env.
 */
mera_status mera_polar_update(const double* env, int m, int n, double* out, int max_iter,
                              double tol, void* ws, size_t ws_bytes, void* stream);

/* Scratch bytes for mera_polar_update with an m x n environment. */
mera_status mera_polar_workspace_size(int m, int n, size_t* bytes);

/*
 * Energy term (Sec. II B): *e_dev = tr(A(h) rho) = sum A(h)[I][J] rho[J][I]
 * with I, J the ket and bra triples.  e_dev is a device double.
 */
mera_status mera_energy(const double* h, const double* rho, const double* u, const double* w,
                        int chi_b, int chi_t, double* e_dev, int prec, void* ws, size_t ws_bytes,
                        void* stream);

/*
 * Blocked critical-Ising density (Eq. ham with spins blocked in pairs to a
 * local dimension 4, Sec. II B 3-site regrouping): writes, to HOST memory,
 * h1 = h3 - shift * 1 as a [4]^6 operator (4096 doubles) with
 * shift = lambda_max(h3) so that h1 is negative semidefinite, and *shift.
 * The field hz multiplies the Z terms; hz = 1 is the critical point.
 */
mera_status mera_ising_h1(double hz, double* h1_host, double* shift_host);

/* One MERA: layers bottom first, the last one scale invariant (Sec. II A). */
typedef struct {
  int n_layers;                    /* tau*, 1..MERA_MAX_LAYERS              */
  int chi_b[MERA_MAX_LAYERS];      /* lower bond dimension of each layer    */
  int chi_t[MERA_MAX_LAYERS];      /* upper bond dimension of each layer    */
  double* u[MERA_MAX_LAYERS];      /* device, chi_b^4, updated in place     */
  double* w[MERA_MAX_LAYERS];      /* device, chi_b^2*chi_t, in place       */
  double* rho_star;                /* device, chi_t[last]^6, warm start     */
} mera_state;

/*
 * One optimisation sweep (Sec. II C): ascend h1 through the transitional
 * layers, n_pow power steps for rho*, update the scale-invariant layer (u,
 * then w with the new u) from its environment with h_{tau*} and rho*, then
 * the transitional layers top-down (u, w, then descend rho one layer; the
 * layer just below the scale-invariant ones sees rho* itself), and
 * finally *e_dev = (tr(h1 rho1) + shift) / 2, the energy per spin with the
 * new tensors.  Layer dimensions must chain: chi_t[k] == chi_b[k+1], and
 * the last layer has chi_b == chi_t.  h1_dev is [chi_b[0]^6] on the device.
 * Asynchronous on the stream (no host synchronisation).  A polar update that
 * hits its iteration cap sets bit (1 << MERA_ENOTCONV) of the device status
 * word; the sweep is still completed.
 */
mera_status mera_sweep(mera_state* state, const double* h1_dev, double shift, int n_pow, int prec,
                       void* ws, size_t ws_bytes, double* e_dev, void* stream);

/*
 * Many independent MERAs, one sweep each (each its own Hamiltonian, bond
 * dimensions and precision-independent state): states[i] with h1[i]
 * (device, [chi_b[0]^6]) and shift[i], scratch ws[i] of ws_bytes[i]
 * (mera_sweep_workspace_size of that state), energy written to e_dev[i]
 * (device), work issued on streams[i].  MERAs that share a stream form a
 * lane: one host thread issues its members in index order, so they run one
 * after another and may share one scratch buffer (large enough for each of
 * them).  Lanes run concurrently: a pool of n_threads host threads issues
 * them, so that the launches of different lanes are issued in parallel.
 * Each MERA's result is exactly what mera_sweep gives for it alone.
 * Returns the most severe status of the batch; the error text names the
 * MERA.  MERA_EINVAL, before any
 * work, if one scratch pointer is given with two different streams (only
 * identical pointers are detected; partly overlapping buffers are the
 * caller's error).
 */
mera_status mera_sweep_batch(mera_state* states, int n, const double* const* h1, const double* shift,
                             int n_pow, int prec, void* const* ws, const size_t* ws_bytes, double* e_dev,
                             void* const* streams, int n_threads);

/*
 * Lanes for mera_sweep_batch under a device-memory budget (host only, no
 * device access).  MERA i has n_layers layers with dimensions
 * chi_b[i * n_layers + k], chi_t[i * n_layers + k]; its scratch is
 * mera_sweep_workspace_size and its cost the contraction flops of one sweep
 * with n_pow power steps.  MERAs whose sweep alone fills the GPU (at least
 * 1e14 flops, e.g. chi >= 20 with tau* = 3) all go to lane 0, one after
 * another: their GEMMs are persistent kernels over every SM, and two of them
 * side by side only contend (measured: 0.94x of one at a time for a 32-MERA
 * mix of chi 8..32 with one lane each).  The others get longest-processing-
 * time-first list scheduling: taken by decreasing scratch (then cost), each
 * opens a new lane while fewer than max_lanes exist and its scratch fits in
 * what is left of budget_bytes, otherwise it joins the lane with the least
 * cost so far among those whose scratch holds it or can grow to hold it
 * within the budget.
 * Outputs: lane[i] in [0, *n_lanes) for every MERA, and lane_bytes[l] (room
 * for n entries) the scratch of lane l, which covers each of its members;
 * the lane_bytes sum to at most budget_bytes.  MERA_ENOMEM if a MERA fits in
 * no lane within the budget (e.g. the largest alone exceeds it); MERA_EINVAL
 * for bad dimensions (the error text names the MERA) or arguments.
 */
mera_status mera_batch_lanes(int n, int n_layers, const int* chi_b, const int* chi_t, int prec, int n_pow,
                             size_t budget_bytes, int max_lanes, int* lane, int* n_lanes, size_t* lane_bytes);

/*
 * Riemannian alternative to the polar update (the paper notes gradients can be
 * obtained by automatic differentiation, Fig. A1 caption; the update itself is
 * the standard Stiefel-manifold step, not the paper's method).
 *
 * mera_stiefel_step: X (m x n, isometric: X^T X = 1, m >= n) and a Euclidean
 * gradient G (m x n), both row-major binary64 device arrays.  Writes
 *   out = polar(X - eta (G - X sym(X^T G))),  sym(A) = (A + A^T) / 2,
 * i.e. one gradient step of length eta along the Riemannian gradient of the
 * embedded metric, retracted to the manifold by the polar factor (computed
 * by the polar update's quintic Newton-Schulz iteration).  out may alias X, not G.
 * Scratch: mera_stiefel_workspace_size(m, n).  Non-convergence of the
 * retraction is reported as for mera_polar_update.
 *
 * mera_sweep_riemannian: mera_sweep with every tensor update replaced by
 * mera_stiefel_step(X, 2 Gamma, eta) (2 Gamma is the energy's gradient for
 * symmetric h and rho).  Same workspace as mera_sweep.
 */
mera_status mera_stiefel_workspace_size(int m, int n, size_t* bytes);
mera_status mera_stiefel_step(const double* X, const double* G, int m, int n, double eta, double* out, void* ws,
                              size_t ws_bytes, void* stream);
mera_status mera_sweep_riemannian(mera_state* S, const double* h1, double shift, int n_pow, int prec, double eta,
                                  void* ws, size_t ws_bytes, double* e_dev, void* stream);

/* Scratch bytes for mera_sweep on a state with these dimensions. */
mera_status mera_sweep_workspace_size(int n_layers, const int* chi_b, const int* chi_t, int prec,
                                      size_t* bytes);

/*
 * Contraction program of `op` as JSON text (orders, GEMM shapes, layouts,
 * flop counts) for inspection and host-side tests.  Writes at most `cap`
 * bytes including the terminating NUL to `buf` and the full length
 * (excluding NUL) to *len.  No device access.
 */
mera_status mera_plan_json(int op, int chi_b, int chi_t, int prec, char* buf, size_t cap,
                           size_t* len);

/*
 * Algorithmic flop count of one call of `op` (the pairwise contraction
 * program's GEMMs, 2 flops per multiply-add).  No device access.
 */
mera_status mera_flops(int op, int chi_b, int chi_t, double* flops);

/*
 * Device-side failure word of the current device: bit (1 << MERA_ETIMEOUT)
 * is set when a bounded wait inside a tensor-core kernel gave up (the kernel
 * then skipped its remaining work and returned; its outputs are invalid);
 * bit (1 << MERA_ENOTCONV) when a polar update (a direct call or one
 * recorded in a graph, below) did not converge within its step limit.
 * Synchronises with the device.  clear != 0 resets the word afterwards.
 */
mera_status mera_device_status(int* status, int clear);

/*
 * One sweep recorded as a CUDA graph and replayed (Sec. II C; no
 * counterpart in the paper's TensorFlow implementation).  Launching ~1200
 * kernels per sweep from the host bounds small-chi sweeps and batches of
 * MERAs; a replay issues them all with one call.
 *
 * mera_sweep_graph_create records mera_sweep(S, h1, shift, n_pow, prec, ws,
 * ws_bytes, e_dev) issued on `stream` (which must not be the legacy
 * default stream) into *graph; nothing is computed.  Every replay then
 * performs that sweep on the same buffers: S's tensors, h1, ws and e_dev are
 * captured by address and must stay allocated (and hold the state to update)
 * until mera_graph_destroy.  Inside the recording every polar update is a
 * conditional while-loop node: Newton-Schulz steps repeat until the device
 * sees convergence (at most 100 steps), with no host check, exactly as a
 * direct mera_polar_update runs it; non-convergence is reported through bit
 * MERA_ENOTCONV of mera_device_status.  A replay gives bit-identical results
 * to mera_sweep on the same inputs.
 * mera_graph_launch enqueues one replay on `stream` (any stream).
 */
typedef struct mera_graph_s* mera_graph;
mera_status mera_sweep_graph_create(mera_state* S, const double* h1, double shift, int n_pow, int prec, void* ws,
                                    size_t ws_bytes, double* e_dev, void* stream, mera_graph* graph);
mera_status mera_graph_launch(mera_graph graph, void* stream);
mera_status mera_graph_destroy(mera_graph graph);

/*
 * One sweep of a MERA whose tensors come from HOST memory (Sec. II C; the
 * host-buffer form of mera_sweep).  On `stream`: copies u_host[k]
 * (chi_b[k]^4 doubles) and w_host[k] (chi_b[k]^2 chi_t[k]) of every layer
 * into S's device tensors, rho_host (chi_t[last]^6) into S->rho_star and
 * h1_host (chi_b[0]^6) into h1_dev, then runs the sweep -- a replay of
 * `graph` when it is not NULL (a sweep recorded with mera_sweep_graph_create
 * on these same device buffers), else mera_sweep(S, h1_dev, shift, n_pow,
 * prec, ws, ws_bytes, e_dev) -- and copies the energy per spin *e_dev to
 * *e_host.  The updated tensors stay on the device.  Asynchronous: the host
 * buffers must stay valid until the stream has passed the copies, and they
 * should be page-locked for the copies to overlap nothing else on the host;
 * *e_host is valid once the stream is synchronised.
 */
mera_status mera_sweep_host(mera_state* S, const double* const* u_host, const double* const* w_host,
                            const double* rho_host, const double* h1_host, double* h1_dev, double shift, int n_pow,
                            int prec, void* ws, size_t ws_bytes, double* e_dev, double* e_host, mera_graph graph,
                            void* stream);

/* ------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; used to measure the kernels).
 * ---------------------------------------------------------------------- */

/* Number of CUDA kernels this library has launched since it was loaded. */
long long mera_launch_count(void);

/*
 * Turn per-launch CUDA-event timing of the contraction kernels on (1) or off
 * (0).  Both calls first wait for and discard earlier records.  While on,
 * every GEMM and operand-permute launch is bracketed by two events recorded
 * on its own stream.
 */
mera_status mera_profile_enable(int on);

#define MERA_PROF_GEMM 0          /* every contraction GEMM                 */
#define MERA_PROF_GEMM_DOMINANT 1 /* the chi^9-class GEMMs of each diagram  */
#define MERA_PROF_PERMUTE 2       /* input permute/cast kernels             */

/*
 * Totals over the records since mera_profile_enable(1): launches, summed
 * device milliseconds and summed algorithmic flops of the selected kind.
 * Waits for the recorded events.  Any pointer may be NULL.
 */
mera_status mera_profile_read(int kind, long long* launches, double* ms, double* flops);

/*
 * Ket/bra transpose of a 3-site operator: out[I][J] = x[J][I] with I, J the
 * ket and bra triples of local dimension d (x, out: d^6 doubles on the
 * device, distinct).  Used by the energy adjoint: dE/dh = D(rho^T) and
 * dE/drho = A(h^T) for E = tr(A(h) rho) (Sec. II B).
 */
mera_status mera_op_transpose(const double* x, int d, double* out, void* stream);

/*
 * Adjoint of the energy term E = tr(A(h) rho) (Sec. II B; the gradients that
 * Fig. A1's caption obtains by automatic differentiation), scaled by the
 * upstream gradient *g_dev (a device double):
 *   dh   = g D(rho^T)                          [chi_b^6]
 *   drho = g A(h^T)                            [chi_t^6]
 *   du   = g (Gamma_u(h, rho) + Gamma_u(h^T, rho^T))   [chi_b^4]
 *   dw   = g (Gamma_w(h, rho) + Gamma_w(h^T, rho^T))   [chi_b^2 chi_t]
 * with ^T the ket/bra transpose (A and D are adjoint; exchanging the ket and
 * bra sides of the network transposes h and rho, so the ket-side holes are
 * the environments of the transposed operators).  For symmetric h and rho,
 * du = 2 g Gamma_u and dw = 2 g Gamma_w.  Any of dh, drho, du, dw may be
 * NULL (not computed).  Nothing is kept between calls: every intermediate is
 * recomputed.  Scratch: mera_workspace_size(MERA_OP_ENERGY_ADJOINT, ...).
 */
mera_status mera_energy_adjoint(const double* h, const double* rho, const double* u, const double* w, int chi_b,
                                int chi_t, const double* g_dev, double* dh, double* drho, double* du, double* dw,
                                int prec, void* ws, size_t ws_bytes, void* stream);

/* Bytes of the device array that backs mera_ascend_noalloc (32 MiB). */
#define MERA_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/*
 * mera_ascend without a workspace argument (the paper has no counterpart;
 * this is an interface for callers that cannot allocate).  Some callers
 * cannot hand the library scratch memory: an application whose own pool
 * allocator owns all device memory and must not be bypassed, or a
 * latency-bound loop that cannot afford a cudaMalloc, which may synchronise
 * the device.  They pass only h, u, w and h_out, exactly as for
 * mera_ascend, whose result this returns.
 *
 * The scratch lives in a file-scope __device__ array of
 * MERA_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds
 * until the process exits (enough for chi_b = chi_t <= 8 in every mode but
 * the fixed-point split ones, which need up to 37 MiB there, and for the
 * 4 -> 16 first layer in every mode).  Sizes whose mera_workspace_size(
 * MERA_OP_ASCEND, ...) exceeds it are rejected with MERA_EINVAL and a
 * message.  No cudaMalloc, cudaFree or allocating library call is made.
 *
 * The first call on each device (and again after a device reset, which
 * makes a new context) looks up the array's device address on the current
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array: every byte a call reads
 * is first written by that same call, so nothing has to start at zero, but
 * two calls that overlap on the GPU (different streams, or different host
 * threads) race on it and give undefined results.
 */
mera_status mera_ascend_noalloc(const double* h, const double* u, const double* w, int chi_b, int chi_t,
                                double* h_out, int prec, void* stream);

/*
 * Tile-width autotuner (batching/tuning extension; no counterpart in the
 * paper).  Times every tensor-core GEMM step of op's program that has more
 * than one sensible output-tile width (N > 64) and no K split, with each
 * candidate width (256, 128, 64; 128 at most for MERA_PREC_BF16X6), on the
 * program's own buffers in `ws` (ws_bytes >= mera_workspace_size(op, ...))
 * and an output scratch of out_elems doubles (>= the op's output size); the
 * contents of both are overwritten.  The fastest width (the planner's own
 * choice unless another is at least 3 % faster) is recorded for the
 * step's shape (mode, M, N, K, output format) and used by every program built
 * afterwards (cached programs are discarded).  *n_tuned: shapes recorded.
 * Results do not depend on the width beyond rounding (K-split counts may
 * change with it).  mera_autotune_reset forgets all recorded widths.
 * Synchronises with the device; call it when no call of this library is in
 * flight.
 */
mera_status mera_autotune(int op, int chi_b, int chi_t, int prec, double* out_scratch, size_t out_elems, void* ws,
                          size_t ws_bytes, void* stream, int* n_tuned);
mera_status mera_autotune_reset(void);

/*
 * Recorded tile widths, set and read without timing (host only): to carry
 * the autotuner's results from one process to another, or to reproduce them
 * where timings would be distorted (under a profiler).
 * mera_set_tile_width records width bn for the GEMM shape (prec, M, N, K,
 * c_final: 1 when the step writes the caller's binary64 output); bn = 0
 * forgets it.  Accepted widths are the autotuner's candidates: 256 (not
 * MERA_PREC_BF16X6), 128 or 64 for N > 128; 128 or 64 for 64 < N <= 128;
 * none for N <= 64.  MERA_EINVAL otherwise, and for MERA_PREC_F64.
 * mera_tile_widths writes *n, the number of recorded shapes, and the first
 * min(*n, cap) of them to out as six values each: prec, M, N, K, c_final,
 * width.  mera_set_tile_width discards cached programs like mera_autotune;
 * call it when no call of this library is in flight.
 */
mera_status mera_set_tile_width(int prec, long long M, long long N, long long K, int c_final, int bn);
mera_status mera_tile_widths(long long* out, int cap, int* n);

/*
 * Memory knob (no counterpart in the paper): a rank-7 intermediate of the
 * chi^9 contraction pairs larger than `bytes` (default 16 GiB) is computed
 * one slice at a time -- the pair runs once per value of one of its free
 * legs on a buffer a factor chi smaller -- so that chi = 40 fits in HBM.
 * Results agree with the unsliced program up to rounding (a smaller slice
 * GEMM may split its K range where the whole one did not).  Changing it
 * discards the cached contraction programs;
 * call it when no call of this library is in flight.
 */
mera_status mera_set_slice_bytes(size_t bytes);

/*
 * Test hook (no counterpart in the paper): C = A * B^T through the GEMM
 * kernel of mode prec, with A row-major M x K, B row-major N x K and C
 * row-major M x N, all binary64 device arrays.  The operands are first cast
 * to the mode's operand format in `ws`, which needs
 * planes * (pad(M*ld) + pad(N*ld)) bytes (ld = K rounded up to 16 bytes,
 * pad = 256-byte multiple, planes = 2 for BF16X3, else 1).
 */
mera_status mera_gemm_test(int prec, const double* A, const double* B, int M, int N, int K, double* C,
                           void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MERA_GB300_H */
