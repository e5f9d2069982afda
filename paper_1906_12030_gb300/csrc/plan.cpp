// Contraction planner: diagram definitions, pairwise order, operand layouts.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <functional>
#include <limits>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <sstream>
#include <tuple>

namespace mera {

int elem_bytes(int prec) {
  switch (prec) {
    case PREC_F64: return 8;
    case PREC_TF32: return 4;
    default: return 2;
  }
}
int tc_block_n(int prec, int64_t N) {
  // the fixed-point split modes keep two accumulators per buffer in tensor
  // memory (4 x width columns of 512): 128 at most
  if (N > 128) {
    if (prec == PREC_BF16X6 || is_oz(prec)) return 128;
    // The widest tile unless a 192- or 160-wide one covers N with less
    // padding.  The kernel is bound by shared-memory reads, which per tile
    // are ~(128 + width) rows of K, so compare ceil(N / width) (128 + width):
    // N = 576 (chi = 24) takes three 192-wide tiles, N = 1600 (chi = 40)
    // keeps 256 (seven tiles, the last a quarter full, cost less than ten
    // 160-wide ones).
    int best = 256;
    int64_t cost = (N + 255) / 256 * (128 + 256);
    for (int bn : {192, 160}) {
      const int64_t c = (N + bn - 1) / bn * (128 + bn);
      if (c < cost) {
        best = bn;
        cost = c;
      }
    }
    return best;
  }
  if (N > 64) return 128;
  if (N > 16) return 64;
  return 16;
}

int tc_split_k(int prec, int64_t M, int64_t N, int64_t K, int bn_in) {
  if (prec == PREC_F64) return 1;
  constexpr int64_t kSMs = 152;
  const int64_t bn = bn_in > 0 ? bn_in : tc_block_n(prec, N);
  const int64_t tiles = ((M + 127) / 128) * ((N + bn - 1) / bn);
  if (is_oz(prec)) {
    // splits hold whole blocks of kOzBlockK (the kernel's exact-sum unit);
    // enough splits for about two waves, at least two blocks each
    const int64_t nblk = (K + kOzBlockK - 1) / kOzBlockK;
    if (tiles >= kSMs || nblk < 4) return 1;
    const int64_t want = std::min<int64_t>((2 * kSMs + tiles - 1) / tiles, nblk / 2);
    if (want < 2) return 1;
    const int64_t per = (nblk + want - 1) / want;  // blocks per split
    return int((nblk + per - 1) / per);             // splits actually non-empty
  }
  const int64_t bk = 128 / elem_bytes(prec);  // K per stage of the GEMM kernel
  const int64_t num_k = (K + bk - 1) / bk;
  if (tiles >= kSMs || num_k < 8) return 1;
  // At least two waves of work items; among the splits up to four times that
  // (and at least 4 k-blocks per split) the one whose last wave is fullest,
  // the smallest on ties.
  const int64_t s_lo = std::max<int64_t>(1, std::min<int64_t>((2 * kSMs + tiles - 1) / tiles, num_k / 4));
  const int64_t s_hi = std::max<int64_t>(s_lo, std::min<int64_t>(4 * s_lo, num_k / 4));
  int64_t best = s_lo;
  double best_eff = 0.0;
  for (int64_t s = s_lo; s <= s_hi; ++s) {
    const int64_t kc = (num_k + s - 1) / s;
    const int64_t sn = (num_k + kc - 1) / kc;  // splits actually non-empty
    const int64_t work = tiles * sn;
    const double eff = double(work) / double(((work + kSMs - 1) / kSMs) * kSMs);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = sn;
    }
  }
  return int(best);
}

int planes(int prec) {
  switch (prec) {
    case PREC_BF16X3: return 2;
    case PREC_BF16X6: return 3;
    case PREC_OZ3: return 3;
    case PREC_OZ4: return 4;
    default: return 1;
  }
}

// Bytes per element of an operand buffer, counting the raw (hi, lo binary32)
// buffer that the fixed-point split modes write before splitting.
double operand_elem_bytes(int prec) { return double(elem_bytes(prec) * planes(prec)) + (is_oz(prec) ? 8.0 : 0.0); }

namespace {

// ---------------------------------------------------------------------------
// Diagrams.  Leg letters: the upper legs of the isometries (p q r on the ket
// side, s t v on the bra side) have size chi_t, every other leg chi_b.
//   ket isometries   w[x,a,p] w[b,c,q] w[d,y,r]
//   bra isometries   w[x,A,s] w[B,C,t] w[D,y,v]
//   even position    u[e,i,a,b] u[j,k,c,d]  h[i,j,k,l,m,n]  u[e,l,A,B] u[m,n,C,D]
//   odd position     u[i,j,a,b] u[k,e,c,d]  h[i,j,k,l,m,n]  u[l,m,A,B] u[n,e,C,D]
// The density rho closes E = tr(A(h) rho) as rho[s,t,v,p,q,r].
// ---------------------------------------------------------------------------
struct TensorSpec {
  int slot;
  const char* legs;
};
struct Diagram {
  std::vector<TensorSpec> tensors;
  const char* out;
};

const char* kKetW[3] = {"xap", "bcq", "dyr"};
const char* kBraW[3] = {"xAs", "BCt", "Dyv"};
const char* kKetU[2][2] = {{"eiab", "jkcd"}, {"ijab", "kecd"}};  // even, odd
const char* kBraU[2][2] = {{"elAB", "mnCD"}, {"lmAB", "neCD"}};

std::vector<Diagram> diagrams_of(int op) {
  std::vector<Diagram> out;
  for (int cs = 0; cs < 2; ++cs) {
    if (op == OP_ASCEND || op == OP_DESCEND) {
      Diagram d;
      for (int k = 0; k < 3; ++k) d.tensors.push_back({SLOT_W, kKetW[k]});
      for (int k = 0; k < 2; ++k) d.tensors.push_back({SLOT_U, kKetU[cs][k]});
      if (op == OP_ASCEND) d.tensors.push_back({SLOT_OP, "ijklmn"});
      for (int k = 0; k < 2; ++k) d.tensors.push_back({SLOT_U, kBraU[cs][k]});
      for (int k = 0; k < 3; ++k) d.tensors.push_back({SLOT_W, kBraW[k]});
      if (op == OP_DESCEND) d.tensors.push_back({SLOT_RHO, "pqrstv"});
      d.out = (op == OP_ASCEND) ? "pqrstv" : "ijklmn";
      out.push_back(d);
    } else {
      const int holes = (op == OP_ENV_W) ? 3 : 2;
      for (int hole = 0; hole < holes; ++hole) {
        Diagram d;
        for (int k = 0; k < 3; ++k) d.tensors.push_back({SLOT_W, kKetW[k]});
        for (int k = 0; k < 2; ++k) d.tensors.push_back({SLOT_U, kKetU[cs][k]});
        d.tensors.push_back({SLOT_OP, "ijklmn"});
        for (int k = 0; k < 2; ++k)
          if (!(op == OP_ENV_U && k == hole)) d.tensors.push_back({SLOT_U, kBraU[cs][k]});
        for (int k = 0; k < 3; ++k)
          if (!(op == OP_ENV_W && k == hole)) d.tensors.push_back({SLOT_W, kBraW[k]});
        d.tensors.push_back({SLOT_RHO, "stvpqr"});
        d.out = (op == OP_ENV_W) ? kBraW[hole] : kBraU[cs][hole];
        out.push_back(d);
      }
    }
  }
  return out;
}

int label_id(char c) {
  if (c >= 'a' && c <= 'z') return c - 'a';
  return 26 + (c - 'A');
}
char label_char(int id) { return id < 26 ? char('a' + id) : char('A' + id - 26); }

// ---------------------------------------------------------------------------
// Pairwise order by dynamic programming over subsets of the input tensors.
// ---------------------------------------------------------------------------
struct Node {
  int left = -1, right = -1;  // children (node ids) or -1 for a leaf
  int tensor = -1;            // leaf: input tensor index
  uint64_t legs = 0;          // open legs (label bitmask)
};

struct Tree {
  std::vector<Node> nodes;
  int root = -1;
};

double size_of(uint64_t legs, const int64_t* dim) {
  double s = 1.0;
  for (int l = 0; l < 64; ++l)
    if (legs >> l & 1ull) s *= double(dim[l]);
  return s;
}

int popcount64(uint64_t x) { return __builtin_popcountll(x); }

Tree plan_order(const std::vector<uint64_t>& tmask, const int64_t* dim, int max_rank) {
  const int n = int(tmask.size());
  const uint32_t full = (1u << n) - 1;
  std::vector<uint64_t> open(1u << n, 0);
  for (uint32_t s = 1; s <= full; ++s) {
    int low = __builtin_ctz(s);
    open[s] = open[s & (s - 1)] ^ tmask[low];
  }
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> cost(1u << n, inf), peak(1u << n, 0.0);
  std::vector<uint32_t> split(1u << n, 0);
  for (int t = 0; t < n; ++t) {
    cost[1u << t] = 0.0;
    peak[1u << t] = 0.0;
  }
  std::vector<uint32_t> order;
  for (uint32_t s = 1; s <= full; ++s) order.push_back(s);
  std::stable_sort(order.begin(), order.end(),
                   [](uint32_t a, uint32_t b) { return __builtin_popcount(a) < __builtin_popcount(b); });
  for (uint32_t s : order) {
    if (__builtin_popcount(s) < 2) continue;
    if (popcount64(open[s]) > max_rank && s != full) continue;
    const uint32_t low = s & (~s + 1);
    const double out_size = size_of(open[s], dim);
    for (uint32_t s1 = (s - 1) & s; s1; s1 = (s1 - 1) & s) {
      if (!(s1 & low)) continue;  // each unordered split once
      const uint32_t s2 = s ^ s1;
      if (cost[s1] == inf || cost[s2] == inf) continue;
      const uint64_t shared = open[s1] & open[s2];
      if (!shared) continue;  // no outer products
      const double fl = 2.0 * size_of(open[s1] | open[s2], dim);
      const double c = cost[s1] + cost[s2] + fl;
      const double pk = std::max({peak[s1], peak[s2], s == full ? 0.0 : out_size});
      const bool better = c < cost[s] * (1 - 1e-12) ||
                          (c <= cost[s] * (1 + 1e-12) && pk < peak[s]);
      if (better) {
        cost[s] = c;
        peak[s] = pk;
        split[s] = s1;
      }
    }
  }
  Tree tr;
  if (cost[full] == inf) return tr;
  // Build nodes recursively.
  std::vector<std::pair<uint32_t, int>> stack;
  std::map<uint32_t, int> id_of;
  std::function<int(uint32_t)> build = [&](uint32_t s) -> int {
    Node nd;
    nd.legs = open[s];
    if (__builtin_popcount(s) == 1) {
      nd.tensor = __builtin_ctz(s);
      tr.nodes.push_back(nd);
      return int(tr.nodes.size()) - 1;
    }
    const int l = build(split[s]);
    const int r = build(s ^ split[s]);
    nd.left = l;
    nd.right = r;
    tr.nodes.push_back(nd);
    return int(tr.nodes.size()) - 1;
  };
  tr.root = build(full);
  return tr;
}

// ---------------------------------------------------------------------------
// Layouts.
// ---------------------------------------------------------------------------
std::vector<int> legs_list(uint64_t m) {
  std::vector<int> v;
  for (int l = 0; l < 64; ++l)
    if (m >> l & 1ull) v.push_back(l);
  return v;
}

std::string legs_str(const std::vector<int>& v) {
  std::string s;
  for (int l : v) s.push_back(label_char(l));
  return s;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Identity of an input copy: which input, and where each of its elements
// goes.  Two steps with the same key write the same bytes.
std::string permute_key(const PermuteStep& p) {
  std::ostringstream o;
  o << p.slot << ':' << p.rows << 'x' << p.cols << '/' << p.ld;
  for (const LegMap* m : {&p.row_src, &p.col_src}) {
    o << '|';
    for (int i = 0; i < m->n; ++i) o << m->dim[i] << '@' << m->stride[i] << ',';
  }
  return o.str();
}

struct Builder {
  const Diagram& dg;
  const int64_t* dim;
  int prec;
  double alpha;
  int accumulate;
  Tree tr;
  Program prog;
  // For every node: the layout its consumer wants (stride of every leg in
  // elements) and the operand buffer it lives in.
  std::vector<std::map<int, int64_t>> dst_stride;
  std::vector<int> buf_of;
  std::vector<int> raw_of;      // fixed-point split modes: raw buffer of each node's operand
  std::vector<int64_t> k_of;    // K of the GEMM that reads each node's operand
  // GEMM info per internal node
  struct G {
    int a = -1, b = -1;
    std::vector<int> mlegs, nlegs, klegs;
  };
  std::vector<G> g;
  // Slicing of rank-7 intermediates: slice_leg[P2] = leg, sliced_child[P2] =
  // P1 (the producer, emitted inside P2's slice loop).
  // slice_block[P2] = b: each slice covers b consecutive values of the leg.
  std::vector<int> slice_leg, sliced_child;
  std::vector<int64_t> slice_block;
  std::vector<char> is_static;  // the node's value depends on u and w only
  std::vector<char> deferred;
  size_t slice_threshold = 0;
  // Copies of h or rho that several diagrams of the operation read in the
  // same layout (keys of permute_key): kept outside the arena.
  const std::set<std::string>* shared = nullptr;

  Builder(const Diagram& d, const int64_t* dm, int p, double al, int acc, size_t sb,
          const std::set<std::string>* sh = nullptr)
      : dg(d), dim(dm), prec(p), alpha(al), accumulate(acc), slice_threshold(sb), shared(sh) {}

  int64_t prod(const std::vector<int>& legs) const {
    int64_t s = 1;
    for (int l : legs) s *= dim[l];
    return s;
  }

  // Leg decomposition of a row or column index; leg `cut` (if any) has
  // extent cut_dim instead of its full size (a slice block).
  LegMap legmap(const std::vector<int>& legs, const std::map<int, int64_t>& stride, int cut = -1,
                int64_t cut_dim = 0) const {
    LegMap m;
    m.n = int(legs.size());
    for (int i = 0; i < m.n; ++i) {
      m.dim[i] = legs[i] == cut ? cut_dim : dim[legs[i]];
      m.stride[i] = stride.at(legs[i]);
    }
    return m;
  }

  // Operand layout [free..., k...] row-major with padded row pitch.
  std::map<int, int64_t> operand_strides(const std::vector<int>& free, const std::vector<int>& k,
                                         int64_t ld) const {
    std::map<int, int64_t> st;
    int64_t s = 1;
    for (int i = int(k.size()) - 1; i >= 0; --i) {
      st[k[i]] = s;
      s *= dim[k[i]];
    }
    s = ld;
    for (int i = int(free.size()) - 1; i >= 0; --i) {
      st[free[i]] = s;
      s *= dim[free[i]];
    }
    return st;
  }

  int64_t pitch(int64_t cols) const {
    const int64_t align = std::max<int64_t>(1, 16 / elem_bytes(prec));
    return round_up(std::max<int64_t>(cols, 1), align);
  }

  // One GEMM step for node i; with slice leg l >= 0 the step covers the
  // values v*bl .. v*bl + bl - 1 of l only: the operand holding l is read
  // from row block v (l is its outermost row leg), the sliced intermediate
  // lives in a one-slice buffer, and the consumer writes its output at
  // offset v * bl * stride(l).
  void emit_gemm(int i, int l, int64_t v, int64_t bl, std::vector<int>& first_use, std::vector<int>& last_use) {
    const G& gi = g[i];
    Step s;
    s.kind = 1;
    GemmStep& gs = s.g;
    gs.a_buf = buf_of[gi.a];
    gs.b_buf = buf_of[gi.b];
    std::vector<int> ml = gi.mlegs, nl = gi.nlegs;
    const bool full_flops_dominant_hint = (l >= 0);
    gs.M = prod(ml);
    gs.N = prod(nl);
    gs.K = prod(gi.klegs);
    gs.lda = prog.bufs[gs.a_buf].ld;
    gs.ldb = prog.bufs[gs.b_buf].ld;
    gs.c_buf = (i == tr.root) ? -1 : (is_oz(prec) ? raw_of[i] : buf_of[i]);
    if (i != tr.root && is_static[i]) {
      gs.stat = 1;
      prog.bufs[buf_of[i]].resident = 1;
    }
    gs.c_ld = (i == tr.root) ? 0 : prog.bufs[buf_of[i]].ld;
    const bool is_producer = (l >= 0) && deferred[i];  // writes the one-slice buffer
    if (l >= 0) {
      const bool in_m = !ml.empty() && ml.front() == l;
      const bool in_n = !nl.empty() && nl.front() == l;
      const int64_t ns = dim[l] / bl;  // number of slices
      // The producer reads row block v of its operand on l's side; the
      // consumer's operand on that side is the one-slice buffer itself.
      if (in_m) {
        gs.M /= ns;
        gs.a_off = is_producer ? v * gs.M * gs.lda : 0;
      } else if (in_n) {
        gs.N /= ns;
        gs.b_off = is_producer ? v * gs.N * gs.ldb : 0;
      }
      gs.c_off = is_producer ? 0 : v * bl * dst_stride[i].at(l);
    }
    gs.m_dst = legmap(ml, dst_stride[i], l, bl);
    gs.n_dst = legmap(nl, dst_stride[i], l, bl);
    gs.alpha = (i == tr.root) ? alpha : 1.0;
    gs.accumulate = (i == tr.root) ? accumulate : 0;
    gs.flops = 2.0 * double(gs.M) * double(gs.N) * double(gs.K);
    gs.dominant = full_flops_dominant_hint ? 2 : 0;  // resolved after emission
    gs.bn = prec == PREC_F64 ? 0 : tc_tile_n(prec, gs.M, gs.N, gs.K, i == tr.root ? 1 : 0);
    gs.split = tc_split_k(prec, gs.M, gs.N, gs.K, gs.bn);
    if (gs.split > 1) {  // FP32 partials [split][N][M], live during this step only
      Buffer pb;
      pb.rows = int64_t(gs.split) * gs.N;
      pb.ld = gs.M;
      pb.plane_bytes = round_up(pb.rows * pb.ld * 4, 256);
      pb.bytes = pb.plane_bytes * (is_oz(prec) ? 2 : 1);  // hi, lo planes in the split modes
      prog.bufs.push_back(pb);
      gs.p_buf = int(prog.bufs.size()) - 1;
      first_use.push_back(-1);
      last_use.push_back(-1);
    }
    {
      std::vector<int> kl = gi.klegs;
      auto a_legs = gi.mlegs;
      a_legs.insert(a_legs.end(), kl.begin(), kl.end());
      auto b_legs = gi.nlegs;
      b_legs.insert(b_legs.end(), kl.begin(), kl.end());
      std::vector<std::pair<int64_t, int>> o;
      for (int x : gi.mlegs) o.push_back({dst_stride[i].at(x), x});
      for (int x : gi.nlegs) o.push_back({dst_stride[i].at(x), x});
      std::sort(o.begin(), o.end(), [](auto& x, auto& y) { return x.first > y.first; });
      std::vector<int> ol;
      for (auto& pr : o) ol.push_back(pr.second);
      gs.label = legs_str(a_legs) + "*" + legs_str(b_legs) + "->" + legs_str(ol);
      if (l >= 0) gs.label += std::string("[") + label_char(l) + "=" + std::to_string(v) + "]";
    }
    prog.flops += gs.flops;
    prog.steps.push_back(s);
    const int si = int(prog.steps.size()) - 1;
    if (last_use[gs.a_buf] < si) last_use[gs.a_buf] = si;
    if (last_use[gs.b_buf] < si) last_use[gs.b_buf] = si;
    if (gs.p_buf >= 0) first_use[gs.p_buf] = last_use[gs.p_buf] = si;
    if (gs.c_buf >= 0) {
      if (first_use[gs.c_buf] < 0) first_use[gs.c_buf] = si;
      if (last_use[gs.c_buf] < si) last_use[gs.c_buf] = si;
    }
  }

  // Fixed-point split modes: node i's raw buffer -> its operand buffer, once
  // the raw buffer is complete.
  void emit_split(int i, std::vector<int>& first_use, std::vector<int>& last_use) {
    if (!is_oz(prec) || i == tr.root) return;
    Step s;
    s.kind = 2;
    SplitStep& x = s.x;
    x.raw_buf = raw_of[i];
    x.dst_buf = buf_of[i];
    x.rows = prog.bufs[x.dst_buf].rows;
    x.ld = prog.bufs[x.dst_buf].ld;
    x.K = k_of[i];
    prog.steps.push_back(s);
    const int si = int(prog.steps.size()) - 1;
    if (last_use[x.raw_buf] < si) last_use[x.raw_buf] = si;
    if (first_use[x.dst_buf] < 0) first_use[x.dst_buf] = si;
    if (last_use[x.dst_buf] < si) last_use[x.dst_buf] = si;
  }

  bool build() {
    const int n = int(dg.tensors.size());
    std::vector<uint64_t> tmask(n, 0);
    for (int t = 0; t < n; ++t)
      for (const char* c = dg.tensors[t].legs; *c; ++c) tmask[t] |= 1ull << label_id(*c);
    tr = plan_order(tmask, dim, 7);
    if (tr.root < 0) return false;
    const size_t nn = tr.nodes.size();
    is_static.assign(nn, 0);
    for (size_t i = 0; i < nn; ++i) {  // children precede their parent in the node list
      const Node& nd = tr.nodes[i];
      if (nd.tensor >= 0) {
        const int slot = dg.tensors[nd.tensor].slot;
        is_static[i] = (slot == SLOT_U || slot == SLOT_W);
      } else {
        is_static[i] = is_static[nd.left] && is_static[nd.right];
      }
    }
    dst_stride.assign(nn, {});
    buf_of.assign(nn, -1);
    raw_of.assign(nn, -1);
    k_of.assign(nn, 0);
    g.assign(nn, {});
    // GEMM roles (bottom-up information only depends on leg sets).
    for (size_t i = 0; i < nn; ++i) {
      const Node& nd = tr.nodes[i];
      if (nd.tensor >= 0) continue;
      const uint64_t L = tr.nodes[nd.left].legs, R = tr.nodes[nd.right].legs;
      const uint64_t K = L & R;
      const double fl = size_of(L & ~K, dim), fr = size_of(R & ~K, dim);
      G& gi = g[i];
      gi.a = (fl >= fr) ? nd.left : nd.right;
      gi.b = (fl >= fr) ? nd.right : nd.left;
      gi.klegs = legs_list(K);
    }
    // Slicing pre-pass: a rank-7 intermediate T (the product of the two
    // chi^9 GEMMs) bigger than the threshold is cut over one of its legs
    // that stays free in the consumer, the largest one.
    slice_leg.assign(nn, -1);
    sliced_child.assign(nn, -1);
    slice_block.assign(nn, 1);
    deferred.assign(nn, 0);
    for (size_t i = 0; i < nn; ++i) {
      const Node& nd = tr.nodes[i];
      if (nd.tensor >= 0) continue;
      for (int c : {g[i].a, g[i].b}) {
        const Node& cn = tr.nodes[c];
        if (cn.tensor >= 0 || popcount64(cn.legs) != 7) continue;
        const double bytes = size_of(cn.legs, dim) * operand_elem_bytes(prec);
        if (bytes <= double(slice_threshold)) continue;
        const uint64_t K2 = tr.nodes[g[i].a].legs & tr.nodes[g[i].b].legs;
        int best = -1;
        for (int l : legs_list(cn.legs & ~K2))
          if (best < 0 || dim[l] > dim[best]) best = l;
        if (best < 0 || dim[best] < 2) continue;
        // the largest block of the leg (a divisor of its size) whose slice
        // stays within the threshold; whole slices keep the GEMMs large
        int64_t bl = 1;
        for (int64_t q = dim[best] - 1; q >= 1; --q)
          if (dim[best] % q == 0 && bytes * double(q) / double(dim[best]) <= double(slice_threshold)) {
            bl = q;
            break;
          }
        slice_leg[i] = best;
        slice_block[i] = bl;
        sliced_child[i] = c;
        deferred[c] = 1;
        break;
      }
    }
    // A sliced intermediate is produced inside its consumer's loop by one
    // GEMM per slice, so it cannot itself run a slice loop of its own: keep
    // its child whole in that case.
    for (size_t i = 0; i < nn; ++i)
      if (deferred[i] && slice_leg[i] >= 0) {
        deferred[sliced_child[i]] = 0;
        sliced_child[i] = -1;
        slice_leg[i] = -1;
      }
    // Root output layout: the caller's order of the open legs.
    {
      std::vector<int> out;
      for (const char* c = dg.out; *c; ++c) out.push_back(label_id(*c));
      int64_t s = 1;
      for (int i = int(out.size()) - 1; i >= 0; --i) {
        dst_stride[tr.root][out[i]] = s;
        s *= dim[out[i]];
      }
      prog.out_rank = int(out.size());
    }
    // Top-down: fix orders and operand layouts, then emit steps bottom-up.
    std::vector<int> topo;  // pre-order
    std::vector<int> st{tr.root};
    while (!st.empty()) {
      int i = st.back();
      st.pop_back();
      topo.push_back(i);
      if (tr.nodes[i].tensor < 0) {
        st.push_back(tr.nodes[i].left);
        st.push_back(tr.nodes[i].right);
      }
    }
    for (int i : topo) {
      const Node& nd = tr.nodes[i];
      if (nd.tensor >= 0) continue;
      G& gi = g[i];
      const uint64_t K = tr.nodes[gi.a].legs & tr.nodes[gi.b].legs;
      std::vector<int> mlegs = legs_list(tr.nodes[gi.a].legs & ~K);
      std::vector<int> nlegs = legs_list(tr.nodes[gi.b].legs & ~K);
      auto by_stride = [&](int x, int y) { return dst_stride[i].at(x) > dst_stride[i].at(y); };
      std::stable_sort(mlegs.begin(), mlegs.end(), by_stride);
      std::stable_sort(nlegs.begin(), nlegs.end(), by_stride);
      // Contracted-leg order: make the innermost one a row leg of the A
      // child's own GEMM when that child is an intermediate, so that the
      // child's epilogue writes consecutive addresses from consecutive rows.
      std::vector<int> klegs = gi.klegs;
      int prefer = -1;
      for (int c : {gi.a, gi.b}) {
        if (tr.nodes[c].tensor >= 0) continue;
        const G& gc = g[c];
        const uint64_t Kc = tr.nodes[gc.a].legs & tr.nodes[gc.b].legs;
        const uint64_t rows_c = tr.nodes[gc.a].legs & ~Kc;
        for (int l : klegs)
          if (rows_c >> l & 1ull) { prefer = l; break; }
        if (prefer >= 0) break;
      }
      if (prefer >= 0) {
        klegs.erase(std::find(klegs.begin(), klegs.end(), prefer));
        klegs.push_back(prefer);
      }
      if (slice_leg[i] >= 0) {  // the sliced leg outermost on T's side
        std::vector<int>& side = (sliced_child[i] == gi.a) ? mlegs : nlegs;
        auto it = std::find(side.begin(), side.end(), slice_leg[i]);
        if (it != side.end()) {
          side.erase(it);
          side.insert(side.begin(), slice_leg[i]);
        }
      }
      gi.mlegs = mlegs;
      gi.nlegs = nlegs;
      gi.klegs = klegs;
      const int64_t Kn = prod(klegs);
      const int64_t ld = pitch(Kn);
      dst_stride[gi.a] = operand_strides(mlegs, klegs, ld);
      dst_stride[gi.b] = operand_strides(nlegs, klegs, ld);
      // operand buffers for both children
      for (int c : {gi.a, gi.b}) {
        Buffer b;
        b.rows = (c == gi.a) ? prod(mlegs) : prod(nlegs);
        if (c == sliced_child[i]) b.rows = b.rows / dim[slice_leg[i]] * slice_block[i];  // one slice at a time
        b.ld = ld;
        b.plane_bytes = round_up(b.rows * ld * elem_bytes(prec), 256);
        b.bytes = b.plane_bytes * planes(prec);
        prog.bufs.push_back(b);
        buf_of[c] = int(prog.bufs.size()) - 1;
        k_of[c] = Kn;
        if (is_oz(prec)) {  // hi, lo binary32 planes in the same layout, split afterwards
          Buffer r = b;
          r.raw = 1;
          r.plane_bytes = round_up(b.rows * ld * 4, 256);
          r.bytes = 2 * r.plane_bytes;
          prog.bufs.push_back(r);
          raw_of[c] = int(prog.bufs.size()) - 1;
        }
      }
    }
    // Emit steps in post-order (children first).
    std::vector<int> post(topo.rbegin(), topo.rend());
    // reverse pre-order (root, right, left) gives a valid post-order.
    std::vector<int> first_use(prog.bufs.size(), -1), last_use(prog.bufs.size(), -1);
    for (int i : post) {
      const Node& nd = tr.nodes[i];
      if (nd.tensor >= 0) {
        const TensorSpec& ts = dg.tensors[nd.tensor];
        const G* parent_g = nullptr;
        (void)parent_g;
        Step s;
        s.kind = 0;
        PermuteStep& p = s.p;
        p.slot = ts.slot;
        p.op_buf = buf_of[i];
        p.dst_buf = is_oz(prec) ? raw_of[i] : buf_of[i];
        // which legs are rows vs cols of the destination: decided by strides
        // (cols = legs with stride < ld).
        const Buffer& b = prog.bufs[p.op_buf];
        std::vector<std::pair<int64_t, int>> legs;  // (dst stride, label)
        for (const char* c = ts.legs; *c; ++c) legs.push_back({dst_stride[i].at(label_id(*c)), label_id(*c)});
        std::sort(legs.begin(), legs.end(), [](auto& x, auto& y) { return x.first > y.first; });
        // source strides: the tensor's own row-major order
        std::map<int, int64_t> src;
        {
          int64_t sstr = 1;
          const int nl = int(std::char_traits<char>::length(ts.legs));
          for (int q = nl - 1; q >= 0; --q) {
            src[label_id(ts.legs[q])] = sstr;
            sstr *= dim[label_id(ts.legs[q])];
          }
        }
        std::vector<int> rl, cl;
        for (auto& pr : legs) (pr.first >= b.ld ? rl : cl).push_back(pr.second);
        p.rows = prod(rl);
        p.cols = prod(cl);
        p.ld = b.ld;
        p.row_src = legmap(rl, src);
        p.col_src = legmap(cl, src);
        prog.steps.push_back(s);
        const int si = int(prog.steps.size()) - 1;
        first_use[p.dst_buf] = si;
        if (ts.slot == SLOT_U || ts.slot == SLOT_W)
          prog.bufs[p.op_buf].resident = 1;
        else if (shared && shared->count(permute_key(p)))
          prog.bufs[p.op_buf].resident = 2;
        emit_split(i, first_use, last_use);
        continue;
      }
      if (deferred[i]) continue;  // emitted inside its consumer's slice loop
      if (slice_leg[i] < 0) {
        emit_gemm(i, -1, 0, 1, first_use, last_use);
        emit_split(i, first_use, last_use);
        continue;
      }
      const int l = slice_leg[i];
      const int64_t bl = slice_block[i];
      for (int64_t v = 0; v < dim[l] / bl; ++v) {
        emit_gemm(sliced_child[i], l, v, bl, first_use, last_use);
        emit_split(sliced_child[i], first_use, last_use);
        emit_gemm(i, l, v, bl, first_use, last_use);
      }
      emit_split(i, first_use, last_use);  // every slice of i's output written
    }
    double fmax = 0.0;
    for (const Step& st : prog.steps)
      if (st.kind == 1 && st.g.dominant != 2) fmax = std::max(fmax, st.g.flops);
    for (Step& st : prog.steps)
      if (st.kind == 1) st.g.dominant = (st.g.dominant == 2) || st.g.flops >= 0.25 * fmax;
    // Resident buffers (operand copies of u and w) are packed one after the
    // other and never reused, so a caller may run the program again with the
    // same u and w without repeating those copies.  Offsets here are
    // relative to the resident region; get_program adds its base.
    size_t res_top = 0;
    for (Buffer& b : prog.bufs)
      if (b.resident) {
        b.offset = int64_t(res_top);
        res_top += size_t(b.bytes);
      }
    prog.resident_bytes = res_top;
    // Arena: first-fit over [first_use, last_use] intervals.
    struct Iv { int64_t off, bytes; int lo, hi; };
    std::vector<Iv> placed;
    size_t top = 0;
    for (size_t bi = 0; bi < prog.bufs.size(); ++bi) {
      Buffer& b = prog.bufs[bi];
      if (b.resident) continue;
      const int lo = first_use[bi], hi = last_use[bi];
      std::vector<std::pair<int64_t, int64_t>> busy;
      for (auto& iv : placed)
        if (!(iv.hi < lo || hi < iv.lo)) busy.push_back({iv.off, iv.off + iv.bytes});
      std::sort(busy.begin(), busy.end());
      int64_t off = 0;
      for (auto& r : busy) {
        if (off + b.bytes <= r.first) break;
        off = std::max(off, r.second);
      }
      b.offset = off;
      placed.push_back({off, b.bytes, lo, hi});
      top = std::max<size_t>(top, size_t(off + b.bytes));
    }
    prog.ws_bytes = top;
    return true;
  }
};

struct Key {
  int op, chi_b, chi_t, prec;
  bool operator<(const Key& o) const {
    return std::tie(op, chi_b, chi_t, prec) < std::tie(o.op, o.chi_b, o.chi_t, o.prec);
  }
};

std::mutex g_mu;
std::map<Key, std::unique_ptr<OpProgram>> g_cache;
size_t g_slice_bytes = size_t(16) << 30;  // 16 GiB
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t, int64_t, int>, int> g_tuned;  // (prec, M, N, K, c_final) -> width

}  // namespace

const OpProgram* get_program(int op, int chi_b, int chi_t, int prec) {
  if (op < OP_ASCEND || op > OP_ENV_W) return nullptr;
  if (prec < PREC_F64 || prec > PREC_LAST) return nullptr;
  if (chi_b < 1 || chi_t < 1 || chi_b > 64 || chi_t > 64) return nullptr;
  if (chi_t > chi_b * chi_b) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  Key k{op, chi_b, chi_t, prec};
  auto it = g_cache.find(k);
  if (it != g_cache.end()) return it->second.get();
  int64_t dim[64];
  for (int l = 0; l < 64; ++l) dim[l] = chi_b;
  for (char c : std::string("pqrstv")) dim[label_id(c)] = chi_t;
  const std::vector<Diagram> ds = diagrams_of(op);
  auto build_all = [&](const std::set<std::string>* sh) -> std::unique_ptr<OpProgram> {
    auto pr = std::make_unique<OpProgram>();
    for (size_t d = 0; d < ds.size(); ++d) {
      Builder b(ds[d], dim, prec, 0.5, d == 0 ? 0 : 1, g_slice_bytes, sh);
      if (!b.build()) return nullptr;
      pr->flops += b.prog.flops;
      pr->diagrams.push_back(std::move(b.prog));
    }
    return pr;
  };
  auto prog = build_all(nullptr);
  if (!prog) return nullptr;
  // Copies of h or rho made more than once in the same layout are made once
  // and kept for the whole call, as long as they are small (each at most
  // 1 GiB, 4 GiB in all): at large chi a copy costs nothing next to the
  // chi^9 work, while keeping it would cost HBM.
  {
    std::map<std::string, int> count;
    std::map<std::string, int64_t> bytes;
    std::vector<std::string> order;
    for (const Program& pg : prog->diagrams)
      for (const Step& st : pg.steps)
        if (st.kind == 0 && (st.p.slot == SLOT_OP || st.p.slot == SLOT_RHO)) {
          const std::string k = permute_key(st.p);
          if (count[k]++ == 0) order.push_back(k);
          bytes[k] = pg.bufs[st.p.op_buf].bytes;
        }
    std::set<std::string> shared;
    int64_t budget = int64_t(4) << 30;
    for (const std::string& k : order)
      if (count[k] > 1 && bytes[k] <= (int64_t(1) << 30) && bytes[k] <= budget) {
        shared.insert(k);
        budget -= bytes[k];
      }
    if (!shared.empty()) {
      prog = build_all(&shared);
      if (!prog) return nullptr;
    }
  }
  // Workspace: [resident buffers][transient arena].  Resident buffers are
  // input copies (one per distinct copy: a later step making a copy that
  // already exists is skipped) and the outputs of u/w-only GEMM steps.
  size_t res_base = 0;
  {
    std::map<std::string, int64_t> made;  // key -> offset
    for (Program& pg : prog->diagrams) {
      std::vector<char> placed(pg.bufs.size(), 0);
      for (size_t si = 0; si < pg.steps.size(); ++si) {
        Step& st = pg.steps[si];
        if (st.kind != 0) continue;
        Buffer& bf = pg.bufs[st.p.op_buf];
        if (!bf.resident) continue;
        placed[size_t(st.p.op_buf)] = 1;
        const std::string k = permute_key(st.p);
        auto it = made.find(k);
        if (it != made.end()) {
          bf.offset = it->second;
          st.p.skip = 1;
          // the split of that copy (fixed-point split modes) is skipped with it
          if (si + 1 < pg.steps.size() && pg.steps[si + 1].kind == 2 && pg.steps[si + 1].x.dst_buf == st.p.op_buf)
            pg.steps[si + 1].x.skip = 1;
        } else {
          bf.offset = int64_t(res_base);
          made[k] = bf.offset;
          res_base += size_t(bf.bytes + 255) / 256 * 256;
        }
      }
      for (size_t b = 0; b < pg.bufs.size(); ++b)
        if (pg.bufs[b].resident && !placed[b]) {
          pg.bufs[b].offset = int64_t(res_base);
          res_base += size_t(pg.bufs[b].bytes + 255) / 256 * 256;
        }
    }
  }
  prog->persistent_bytes = res_base;
  size_t trans = 0;
  for (Program& pg : prog->diagrams) {
    for (Buffer& bf : pg.bufs)
      if (!bf.resident) bf.offset += int64_t(res_base);
    trans = std::max(trans, pg.ws_bytes);
  }
  prog->ws_bytes = res_base + trans;
  const OpProgram* out = prog.get();
  g_cache[k] = std::move(prog);
  return out;
}

int tc_tile_n(int prec, int64_t M, int64_t N, int64_t K, int c_final) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(prec, M, N, K, c_final));
    if (it != g_tuned.end()) return it->second;
  }
  return tc_block_n(prec, N);
}

void set_tuned_tile(int prec, int64_t M, int64_t N, int64_t K, int c_final, int bn) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto key = std::make_tuple(prec, M, N, K, c_final);
    if (bn > 0)
      g_tuned[key] = bn;
    else
      g_tuned.erase(key);
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
}

void clear_tuned_tiles() {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
}

int tuned_tile_count() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return int(g_tuned.size());
}

std::vector<std::vector<int64_t>> tuned_tiles() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::vector<std::vector<int64_t>> out;
  for (const auto& kv : g_tuned)
    out.push_back({std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                   std::get<4>(kv.first), kv.second});
  return out;
}

void set_slice_bytes(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_slice_bytes = bytes;
  g_cache.clear();
}

size_t slice_bytes() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_slice_bytes;
}

std::string program_json(const OpProgram& prog, int op, int chi_b, int chi_t, int prec) {
  std::ostringstream o;
  o.precision(17);
  auto lm = [&](const LegMap& m) {
    o << "{\"dim\":[";
    for (int i = 0; i < m.n; ++i) o << (i ? "," : "") << m.dim[i];
    o << "],\"stride\":[";
    for (int i = 0; i < m.n; ++i) o << (i ? "," : "") << m.stride[i];
    o << "]}";
  };
  o << "{\"op\":" << op << ",\"chi_b\":" << chi_b << ",\"chi_t\":" << chi_t << ",\"prec\":" << prec
    << ",\"ws_bytes\":" << prog.ws_bytes << ",\"flops\":" << prog.flops << ",\"elem_bytes\":" << elem_bytes(prec)
    << ",\"planes\":" << planes(prec) << ",\"persistent_bytes\":" << prog.persistent_bytes << ",\"diagrams\":[";
  for (size_t d = 0; d < prog.diagrams.size(); ++d) {
    const Program& p = prog.diagrams[d];
    o << (d ? "," : "") << "{\"ws_bytes\":" << p.ws_bytes << ",\"flops\":" << p.flops << ",\"bufs\":[";
    for (size_t b = 0; b < p.bufs.size(); ++b)
      o << (b ? "," : "") << "{\"rows\":" << p.bufs[b].rows << ",\"ld\":" << p.bufs[b].ld
        << ",\"offset\":" << p.bufs[b].offset << ",\"bytes\":" << p.bufs[b].bytes
        << ",\"plane_bytes\":" << p.bufs[b].plane_bytes << ",\"raw\":" << p.bufs[b].raw
        << ",\"resident\":" << p.bufs[b].resident << "}";
    o << "],\"steps\":[";
    for (size_t s = 0; s < p.steps.size(); ++s) {
      const Step& st = p.steps[s];
      o << (s ? "," : "");
      if (st.kind == 2) {
        o << "{\"kind\":\"split\",\"raw_buf\":" << st.x.raw_buf << ",\"dst_buf\":" << st.x.dst_buf
          << ",\"rows\":" << st.x.rows << ",\"K\":" << st.x.K << ",\"ld\":" << st.x.ld << ",\"skip\":" << st.x.skip
          << "}";
      } else if (st.kind == 0) {
        o << "{\"kind\":\"permute\",\"slot\":" << st.p.slot << ",\"dst_buf\":" << st.p.dst_buf
          << ",\"op_buf\":" << st.p.op_buf
          << ",\"rows\":" << st.p.rows << ",\"cols\":" << st.p.cols << ",\"ld\":" << st.p.ld
          << ",\"skip\":" << st.p.skip << ",\"row_src\":";
        lm(st.p.row_src);
        o << ",\"col_src\":";
        lm(st.p.col_src);
        o << "}";
      } else {
        const GemmStep& g = st.g;
        o << "{\"kind\":\"gemm\",\"label\":\"" << g.label << "\",\"a_buf\":" << g.a_buf << ",\"b_buf\":" << g.b_buf
          << ",\"M\":" << g.M << ",\"N\":" << g.N << ",\"K\":" << g.K << ",\"lda\":" << g.lda << ",\"ldb\":" << g.ldb
          << ",\"c_buf\":" << g.c_buf << ",\"alpha\":" << g.alpha << ",\"accumulate\":" << g.accumulate
          << ",\"flops\":" << g.flops << ",\"dominant\":" << g.dominant << ",\"split\":" << g.split
          << ",\"p_buf\":" << g.p_buf << ",\"a_off\":" << g.a_off << ",\"b_off\":" << g.b_off
          << ",\"c_off\":" << g.c_off << ",\"stat\":" << g.stat << ",\"bn\":" << g.bn << ",\"m_dst\":";
        lm(g.m_dst);
        o << ",\"n_dst\":";
        lm(g.n_dst);
        o << "}";
      }
    }
    o << "]}";
  }
  o << "]}";
  return o.str();
}

}  // namespace mera
