"""Host-side tests of the C-ABI library (no GPU needed).

* the shared library builds for sm_103a, loads and exports every entry point
  that include/mera.h declares;
* host-only entry points (Hamiltonian builder, planner, flop counts,
  argument checks) behave as documented;
* the contraction programs the planner emits -- pairwise orders, operand
  layouts, padded pitches, scattered epilogue strides, workspace arena --
  reproduce the oracle when executed step by step with numpy exactly as the
  kernels execute them.
"""
import os
import re

import numpy as np
import pytest

import mera_inputs as I
from oracle import mera_oracle as O

m = pytest.importorskip("paper_1906_12030_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mera.h")


def _declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:mera_status|const char\*|long long)\s+(mera_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol():
    lib = m.library()
    names = _declared_symbols()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    assert "sm_103a" in m.mera_version()


def test_ising_builder_matches_oracle():
    for hz in (1.0, 0.9, 1.1):
        h1, s = m.mera_ising_h1(hz)
        h1o, so = O.ising_h1(hz)
        assert abs(s - so) < 1e-13
        assert np.abs(h1 - h1o).max() < 1e-13


def test_argument_checks_without_device():
    with pytest.raises(m.MeraError):
        m.mera_workspace_size(99, 4, 4, 0)
    with pytest.raises(m.MeraError):
        m.mera_workspace_size(m.OP_ASCEND, 4, 17, 0)  # chi_t > chi_b^2
    with pytest.raises(m.MeraError):
        m.mera_workspace_size(m.OP_ASCEND, 0, 4, 0)
    with pytest.raises(m.MeraError):
        m.mera_workspace_size(m.OP_FIXED_POINT, 4, 3, 0)
    with pytest.raises(m.MeraError):
        m.mera_polar_workspace_size(3, 4)  # m < n
    assert m.mera_workspace_size(m.OP_ASCEND, 4, 4, m.PREC_BF16X3) > 0


@pytest.mark.parametrize("chi,per_diagram", [(4, 1.59e6), (8, 6.72e8), (16, 3.09e11), (32, 1.50e14)])
def test_min_flop_orders(chi, per_diagram):
    """4 chi^9 + 8 chi^8 + lower per diagram: the chi^9 cost of Sec. II B."""
    for op, nd in ((m.OP_ASCEND, 2), (m.OP_DESCEND, 2), (m.OP_ENV_U, 4), (m.OP_ENV_W, 6)):
        f = m.mera_flops(op, chi, chi)
        assert f / nd == pytest.approx(per_diagram, rel=0.01)
        assert f / nd >= 4 * chi ** 9


def test_sweep_flops_chi16():
    """tau* = 3, 20 power steps: 50 SI diagrams + 14 + 14, ~1.98e13 at chi = 16."""
    dims = I.layer_dims(16)
    total = 0.0
    for k, (cb, ct) in enumerate(dims):
        if k < len(dims) - 1:
            total += m.mera_flops(m.OP_ASCEND, cb, ct)
        else:
            total += 20 * m.mera_flops(m.OP_DESCEND, cb, ct)
        total += m.mera_flops(m.OP_ENV_U, cb, ct) + m.mera_flops(m.OP_ENV_W, cb, ct)
        if 0 < k < len(dims) - 1:
            total += m.mera_flops(m.OP_DESCEND, cb, ct)  # rho down one transitional layer
        elif k == 0:
            total += m.mera_flops(m.OP_ASCEND, cb, ct)   # energy tr(A(h1) rho2)
    assert total == pytest.approx(1.98e13, rel=0.01)


# --------------------------------------------------------------------------
# Emulate the programs with numpy.
# --------------------------------------------------------------------------
def _offsets(lm, count):
    idx = np.arange(count, dtype=np.int64)
    off = np.zeros(count, dtype=np.int64)
    for d, s in zip(reversed(lm["dim"]), reversed(lm["stride"])):
        off += (idx % d) * s
        idx //= d
    return off


def _emulate(plan, inputs, out_size, arena=None, reuse=False, keep=False):
    """Run a program in float64; buffers live in one flat arena (per plane).
    reuse: run it again on the arena of a previous run with the same u and w,
    skipping the u/w copies and the u/w-only products as the library does.
    keep: return (output, arena)."""
    eb = plan["elem_bytes"]
    out = np.zeros(out_size)
    if arena is None:
        arena = np.full(plan["ws_bytes"] // eb + 1, np.nan)
    for dg in plan["diagrams"]:
        bufs = dg["bufs"]
        partial = {st["p_buf"] for st in dg["steps"] if st["kind"] == "gemm" and st["p_buf"] >= 0}
        for i, b in enumerate(bufs):
            assert b["offset"] % 256 == 0
            assert b["offset"] + b["bytes"] <= plan["ws_bytes"]
            if i in partial:  # FP32 split-K partials [split][N][M]
                assert b["bytes"] >= b["rows"] * b["ld"] * 4
            else:
                assert b["ld"] * eb % 16 == 0  # TMA: row pitch multiple of 16 bytes
            if b.get("raw"):  # hi and lo binary32 planes
                assert b["bytes"] >= 2 * b["rows"] * b["ld"] * 4
        # stale data from an earlier diagram must never be read, except the
        # copies kept for the whole call (the leading persistent bytes)
        arena[plan["persistent_bytes"] // eb:] = np.nan
        for st in dg["steps"]:
            if st["kind"] == "permute" and st["skip"]:
                b = bufs[st["op_buf"]]
                assert b["resident"] and b["offset"] + b["bytes"] <= plan["persistent_bytes"]
                continue  # the same copy was made by an earlier step
            if st["kind"] == "split" and st["skip"]:
                assert bufs[st["dst_buf"]]["resident"]
                continue  # the split of that copy was made with it
            if reuse and st["kind"] == "permute" and bufs[st["op_buf"]]["resident"] == 1:
                continue  # u/w copy kept from the previous run
            if reuse and st["kind"] == "split" and bufs[st["dst_buf"]]["resident"] == 1:
                continue  # its split too
            if reuse and st["kind"] == "gemm" and st["stat"]:
                assert bufs[st["c_buf"]]["resident"] == 1 or bufs[st["c_buf"]]["raw"]
                continue  # u/w-only product kept from the previous run
            if st["kind"] == "split":
                # fixed-point split modes: raw hi + lo planes -> slices (same values here);
                # every entry of the K columns of every row must have been written
                r, d = bufs[st["raw_buf"]], bufs[st["dst_buf"]]
                assert r["raw"] and not d["raw"] and st["K"] <= st["ld"] == d["ld"] == r["ld"]
                assert st["rows"] == d["rows"] == r["rows"]
                idx = np.arange(st["rows"])[:, None] * st["ld"] + np.arange(st["K"])[None, :]
                vals = arena[r["offset"] // eb + idx]
                assert not np.isnan(vals).any()
                arena[d["offset"] // eb + idx] = vals
                continue
            if st["kind"] == "permute":
                src = inputs[st["slot"]].reshape(-1)
                b = bufs[st["dst_buf"]]
                rows, cols, ld = st["rows"], st["cols"], st["ld"]
                ro = _offsets(st["row_src"], rows)
                co = _offsets(st["col_src"], cols)
                base = b["offset"] // eb
                dst_idx = base + (np.arange(rows)[:, None] * ld + np.arange(cols)[None, :])
                arena[dst_idx] = src[ro[:, None] + co[None, :]]
            else:
                a, bb = bufs[st["a_buf"]], bufs[st["b_buf"]]
                M, N, K = st["M"], st["N"], st["K"]
                # operand reads (TMA boxes are clipped to rows x K of these planes)
                assert K <= st["lda"] == a["ld"] and K <= st["ldb"] == bb["ld"]
                # a slice step reads a row block of its operand: whole rows only
                assert st["a_off"] % st["lda"] == 0 and st["b_off"] % st["ldb"] == 0
                assert st["a_off"] // st["lda"] + M <= a["rows"] and st["b_off"] // st["ldb"] + N <= bb["rows"]
                A = arena[a["offset"] // eb + st["a_off"] + np.arange(M)[:, None] * st["lda"] + np.arange(K)[None, :]]
                B = arena[bb["offset"] // eb + st["b_off"] + np.arange(N)[:, None] * st["ldb"] + np.arange(K)[None, :]]
                assert not np.isnan(A).any() and not np.isnan(B).any()
                C = st["alpha"] * (A @ B.T)
                mo = _offsets(st["m_dst"], M)
                no = _offsets(st["n_dst"], N)
                idx = st["c_off"] + mo[:, None] + no[None, :]
                assert len(np.unique(idx)) == idx.size  # the scatter is a bijection
                if st["c_buf"] < 0:
                    assert idx.min() >= 0 and idx.max() < out_size
                    if st["accumulate"]:
                        out[idx] += C
                    else:
                        out[idx] = C
                else:
                    cb = bufs[st["c_buf"]]
                    # every scattered store stays inside its operand plane
                    assert idx.min() >= 0 and idx.max() < cb["rows"] * cb["ld"]
                    assert (idx % cb["ld"]).max() < bufs[st["c_buf"]]["ld"]
                    arena[cb["offset"] // eb + idx] = C
    return (out, arena) if keep else out


_SMALL = [(1, 1), (2, 1), (2, 2), (3, 3), (2, 3), (4, 3), (3, 5)]


@pytest.mark.parametrize("prec,chi_b,chi_t",
                         [(p, b, t) for p in (m.PREC_F64, m.PREC_BF16X3, m.PREC_BF16X6, m.PREC_OZ3) for b, t in _SMALL]
                         + [(m.PREC_BF16X3, 4, 16), (m.PREC_OZ4, 4, 16)])  # first-layer shape, with K-split steps
def test_programs_reproduce_oracle(prec, chi_b, chi_t):
    rng = np.random.default_rng(20)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b, symmetric=False)
    rho = I.random_operator(rng, chi_t, symmetric=False)
    hs, rs = I.random_operator(rng, chi_b), I.random_density(rng, chi_t)
    cases = [
        (m.OP_ASCEND, [h, None, u, w], O.ascend(h, u, w)),
        (m.OP_DESCEND, [None, rho, u, w], O.descend(rho, u, w)),
        (m.OP_ENV_U, [hs, rs, u, w], O.env_u(hs, rs, u, w)),
        (m.OP_ENV_W, [hs, rs, u, w], O.env_w(hs, rs, u, w)),
    ]
    for op, inputs, want in cases:
        plan = m.mera_plan_json(op, chi_b, chi_t, prec)
        got = _emulate(plan, inputs, want.size).reshape(want.shape)
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), op


@pytest.fixture
def forced_slicing():
    """Slice every rank-7 intermediate, whatever its size."""
    m.mera_set_slice_bytes(0)
    try:
        yield
    finally:
        m.mera_set_slice_bytes(16 << 30)


@pytest.mark.parametrize("prec,chi_b,chi_t", [(m.PREC_F64, 3, 3), (m.PREC_BF16X3, 2, 3), (m.PREC_F64, 4, 3),
                                              (m.PREC_BF16X6, 3, 5), (m.PREC_OZ3, 3, 4)])
def test_sliced_programs_reproduce_oracle(forced_slicing, prec, chi_b, chi_t):
    _check_sliced(prec, chi_b, chi_t)


@pytest.mark.parametrize("prec", [m.PREC_F64, m.PREC_BF16X3])
def test_block_sliced_programs_reproduce_oracle(prec):
    """A threshold of half the intermediate makes each slice cover two values
    of the sliced leg (chi = 4): the block form of the slice loop."""
    eb = {m.PREC_F64: 8, m.PREC_BF16X3: 4}[prec]
    m.mera_set_slice_bytes(4 ** 7 * eb // 2)
    try:
        n = _check_sliced(prec, 4, 4)
    finally:
        m.mera_set_slice_bytes(16 << 30)
    assert n["ascend"] == 2 * 2 * 2  # 2 diagrams x 2 slices x (producer, consumer)


def _check_sliced(prec, chi_b, chi_t):
    """Rank-7 intermediates computed one slice at a time (the memory plan
    that lets chi = 40 fit) still give the oracle's maps, and every diagram
    holding a chi^9 pair does slice it."""
    rng = np.random.default_rng(11)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b, symmetric=False)
    rho = I.random_operator(rng, chi_t, symmetric=False)
    hs, rs = I.random_operator(rng, chi_b), I.random_density(rng, chi_t)
    cases = {m.OP_ASCEND: ([h, None, u, w], O.ascend(h, u, w)),
             m.OP_DESCEND: ([None, rho, u, w], O.descend(rho, u, w)),
             m.OP_ENV_U: ([hs, rs, u, w], O.env_u(hs, rs, u, w)),
             m.OP_ENV_W: ([hs, rs, u, w], O.env_w(hs, rs, u, w))}
    counts = {}
    names = {m.OP_ASCEND: "ascend", m.OP_DESCEND: "descend", m.OP_ENV_U: "env_u", m.OP_ENV_W: "env_w"}
    for op, (inputs, want) in cases.items():
        plan = m.mera_plan_json(op, chi_b, chi_t, prec)
        sliced = [st for dg in plan["diagrams"] for st in dg["steps"] if st["kind"] == "gemm" and "=" in st["label"]]
        assert sliced, op
        counts[names[op]] = len(sliced)
        got = _emulate(plan, inputs, want.size).reshape(want.shape)
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), op
    return counts


def test_slicing_shrinks_the_chi40_workspace():
    """At chi = 40 the unsliced rank-7 intermediates alone take hundreds of
    GB; with the default threshold the descend workspace fits in HBM."""
    need = m.mera_workspace_size(m.OP_DESCEND, 40, 40, m.PREC_BF16X3)
    assert need < 200 * 2**30
    m.mera_set_slice_bytes(1 << 62)
    try:
        whole = m.mera_workspace_size(m.OP_DESCEND, 40, 40, m.PREC_BF16X3)
    finally:
        m.mera_set_slice_bytes(16 << 30)
    assert whole > 300 * 2**30


@pytest.mark.parametrize("prec", [m.PREC_BF16X3, m.PREC_OZ3])
def test_split_k_partials_do_not_overlap_live_buffers(prec):
    """Steps with few output tiles and long K get a K split; its FP32 partial
    buffer must not overlap the step's operands (the arena check above runs
    the same programs)."""
    plan = m.mera_plan_json(m.OP_ENV_W, 4, 16, prec)
    splits = [st for dg in plan["diagrams"] for st in dg["steps"] if st["kind"] == "gemm" and st["split"] > 1]
    assert splits, "the K = 65536 step of the 4 -> 16 env_w program should be split"
    for dg in plan["diagrams"]:
        bufs = dg["bufs"]
        for st in dg["steps"]:
            if st["kind"] != "gemm" or st["split"] <= 1:
                continue
            p = bufs[st["p_buf"]]
            for other in (st["a_buf"], st["b_buf"]) + ((st["c_buf"],) if st["c_buf"] >= 0 else ()):
                o = bufs[other]
                assert p["offset"] + p["bytes"] <= o["offset"] or o["offset"] + o["bytes"] <= p["offset"]


@pytest.mark.parametrize("op", [m.OP_DESCEND, m.OP_ENV_W])
def test_resident_operand_copies_are_never_reused(op):
    """The operand copies of u and w are kept for the whole call (the fixed
    point reuses them across its power steps), and so are copies of h or rho
    that several diagrams read in the same layout: distinct copies must not
    overlap each other, in any diagram, nor any transient buffer."""
    plan = m.mera_plan_json(op, 4, 4, m.PREC_BF16X3)
    resident, transient = [], []
    for dg in plan["diagrams"]:
        for b in dg["bufs"]:
            (resident if b["resident"] else transient).append((b["offset"], b["offset"] + b["bytes"]))
    assert resident
    resident = sorted(set(resident))  # a copy shared by several diagrams appears once
    for (a0, a1), (b0, b1) in zip(resident, resident[1:]):
        assert a1 <= b0
    for r0, r1 in resident:
        for t0, t1 in transient:
            assert r1 <= t0 or t1 <= r0


@pytest.mark.parametrize("op,chi", [(m.OP_DESCEND, 16), (m.OP_ENV_W, 16), (m.OP_ENV_U, 8)])
def test_identical_input_copies_are_made_once(op, chi):
    """Each distinct operand copy of an input is made once per call; every
    later step that would make the same copy is skipped and reads the first
    one (the emulation of these programs against the oracle covers the
    correctness; this checks the count)."""
    plan = m.mera_plan_json(op, chi, chi, m.PREC_BF16X3)
    made, skipped = set(), 0
    for dg in plan["diagrams"]:
        for st in dg["steps"]:
            if st["kind"] != "permute":
                continue
            key = (st["slot"], st["rows"], st["cols"], st["ld"], str(st["row_src"]), str(st["col_src"]))
            if st["skip"]:
                assert key in made
                skipped += 1
            else:
                assert key not in made or not dg["bufs"][st["dst_buf"]]["resident"]
                made.add(key)
    assert skipped > 0
    if op == m.OP_DESCEND:  # both diagrams read rho in the same layout
        rho_copies = [st for dg in plan["diagrams"] for st in dg["steps"]
                      if st["kind"] == "permute" and st["slot"] == 1 and not st["skip"]]
        assert len(rho_copies) == 1


@pytest.mark.parametrize("prec,chi", [(m.PREC_F64, 3), (m.PREC_BF16X3, 4), (m.PREC_OZ3, 4)])
def test_rerun_with_kept_uw_products(prec, chi):
    """The power iteration runs the descending program again with new rho and
    the same u, w, skipping the u/w copies and the u/w-only products it kept:
    the second run must still give the oracle's D(rho2), and every kept
    product must read only kept buffers."""
    rng = np.random.default_rng(31)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    r1, r2 = I.random_density(rng, chi), I.random_density(rng, chi)
    plan = m.mera_plan_json(m.OP_DESCEND, chi, chi, prec)
    n_stat = 0
    for dg in plan["diagrams"]:
        for st in dg["steps"]:
            if st["kind"] == "gemm" and st["stat"]:
                n_stat += 1
                assert dg["bufs"][st["a_buf"]]["resident"] == 1 and dg["bufs"][st["b_buf"]]["resident"] == 1
    assert n_stat == 8  # four u/w products in each of the two diagrams
    out1, arena = _emulate(plan, [None, r1, u, w], chi ** 6, keep=True)
    out2 = _emulate(plan, [None, r2, u, w], chi ** 6, arena=arena, reuse=True)
    for got, rho in ((out1, r1), (out2, r2)):
        want = O.descend(rho, u, w).reshape(-1)
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


def test_plans_carry_tile_widths():
    """Tensor-core steps carry the tile width the kernel will use (from N when
    nothing is tuned); FP64 steps carry none."""
    m.mera_autotune_reset()
    plan = m.mera_plan_json(m.OP_ASCEND, 16, 16, m.PREC_BF16X3)
    for dg in plan["diagrams"]:
        for st in dg["steps"]:
            if st["kind"] == "gemm":
                want = 256 if st["N"] > 128 else 128 if st["N"] > 64 else 64 if st["N"] > 16 else 16
                assert st["bn"] == want
    plan = m.mera_plan_json(m.OP_ASCEND, 4, 4, m.PREC_F64)
    assert all(st["bn"] == 0 for dg in plan["diagrams"] for st in dg["steps"] if st["kind"] == "gemm")


def _batch_dims(chis):
    return [([b for b, _ in I.layer_dims(c)], [t for _, t in I.layer_dims(c)]) for c in chis]


def _sweep_need(dims, prec):
    return [m.mera_sweep_workspace_size(b, t, prec) for b, t in dims]


def test_batch_lanes_one_per_mera_when_memory_allows():
    dims = _batch_dims([8, 12, 16, 8])
    need = _sweep_need(dims, m.PREC_BF16X3)
    lanes, lane_bytes = m.mera_batch_lanes(dims, m.PREC_BF16X3, sum(need), max_lanes=32)
    assert sorted(lanes) == [0, 1, 2, 3]
    assert [lane_bytes[k] for k in lanes] == need


def test_batch_lanes_single_lane_at_the_largest_scratch():
    dims = _batch_dims([8, 16, 12, 16, 4])
    need = _sweep_need(dims, m.PREC_BF16X3)
    lanes, lane_bytes = m.mera_batch_lanes(dims, m.PREC_BF16X3, max(need), max_lanes=32)
    assert lanes == [0] * 5 and lane_bytes == [max(need)]
    with pytest.raises(m.MeraError, match="budget"):
        m.mera_batch_lanes(dims, m.PREC_BF16X3, max(need) - 1)


@pytest.mark.parametrize("budget_gb,max_lanes", [(40, 32), (120, 32), (200, 3), (200, 32), (1000, 8)])
def test_batch_lanes_respect_budget_and_cover_every_member(budget_gb, max_lanes):
    """32 MERAs with chi drawn from {8, 12, 16, 20, 24, 32}: lanes never exceed
    the budget or the lane cap, and each lane's scratch holds every member."""
    rng = np.random.default_rng(3)
    chis = [int(rng.choice([8, 12, 16, 20, 24, 32])) for _ in range(32)]
    dims = _batch_dims(chis)
    need = _sweep_need(dims, m.PREC_BF16X3)
    budget = budget_gb << 30
    if max(need) > budget:
        with pytest.raises(m.MeraError):
            m.mera_batch_lanes(dims, m.PREC_BF16X3, budget, max_lanes)
        return
    lanes, lane_bytes = m.mera_batch_lanes(dims, m.PREC_BF16X3, budget, max_lanes)
    assert 1 <= len(lane_bytes) <= max_lanes and sum(lane_bytes) <= budget
    assert set(lanes) == set(range(len(lane_bytes)))
    assert all(lane_bytes[k] >= n for k, n in zip(lanes, need))


def test_batch_lanes_balance_equal_meras():
    """Equal MERAs over k lanes: the list schedule deals them out evenly."""
    dims = _batch_dims([12] * 11)
    need = _sweep_need(dims, m.PREC_F64)[0]
    lanes, lane_bytes = m.mera_batch_lanes(dims, m.PREC_F64, 100 * need, max_lanes=4)
    counts = sorted(lanes.count(k) for k in range(len(lane_bytes)))
    assert len(lane_bytes) == 4 and counts == [2, 3, 3, 3]


def test_batch_lanes_reject_bad_dimensions():
    dims = _batch_dims([8, 8])
    dims[1] = ([4, 16, 8], [16, 9, 8])    # layers do not chain
    with pytest.raises(m.MeraError, match="MERA 1"):
        m.mera_batch_lanes(dims, m.PREC_F64, 1 << 40)


def _gemm_steps(op, chi, prec):
    return [st for dg in m.mera_plan_json(op, chi, chi, prec)["diagrams"] for st in dg["steps"] if st["kind"] == "gemm"]


def test_recorded_tile_widths_set_read_and_reach_the_plan():
    prec = m.PREC_BF16X3
    m.mera_autotune_reset()
    try:
        st = next(s for s in _gemm_steps(m.OP_ASCEND, 16, prec) if s["N"] > 128 and s["split"] == 1)
        cf = int(st["c_buf"] < 0)
        new = 128 if st["bn"] != 128 else 64
        m.mera_set_tile_width(prec, st["M"], st["N"], st["K"], cf, new)
        assert m.mera_tile_widths() == [(prec, st["M"], st["N"], st["K"], cf, new)]
        same = [s for s in _gemm_steps(m.OP_ASCEND, 16, prec)
                if (s["M"], s["N"], s["K"], int(s["c_buf"] < 0)) == (st["M"], st["N"], st["K"], cf)]
        assert same and all(s["bn"] == new for s in same)
        m.mera_set_tile_width(prec, st["M"], st["N"], st["K"], cf, 0)      # forget
        assert m.mera_tile_widths() == []
        assert all(s["bn"] == st["bn"] for s in _gemm_steps(m.OP_ASCEND, 16, prec)
                   if (s["M"], s["N"], s["K"], int(s["c_buf"] < 0)) == (st["M"], st["N"], st["K"], cf))
    finally:
        m.mera_autotune_reset()


@pytest.mark.parametrize("prec,N,bn", [(m.PREC_F64, 256, 128), (m.PREC_BF16X3, 64, 64), (m.PREC_BF16X3, 100, 256),
                                       (m.PREC_BF16X6, 512, 256), (m.PREC_TF32, 512, 96)])
def test_tile_widths_outside_the_candidates_are_rejected(prec, N, bn):
    with pytest.raises(m.MeraError):
        m.mera_set_tile_width(prec, 4096, N, 256, 0, bn)
    assert m.mera_tile_widths() == []


def _imports(path):
    import ast

    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def test_product_and_oracle_share_no_code():
    """The package never imports the oracle, the oracle never imports the
    package, and the native sources never name the oracle."""
    pkg = os.path.join(ROOT, "paper_1906_12030_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            assert "oracle" not in _imports(os.path.join(pkg, name)), name
    for name in os.listdir(os.path.join(ROOT, "oracle")):
        if name.endswith(".py"):
            assert "paper_1906_12030_gb300" not in _imports(os.path.join(ROOT, "oracle", name)), name
    csrc = os.path.join(pkg, "csrc")
    for name in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, name), errors="replace").read().lower(), name
    assert _imports(os.path.join(ROOT, "mera_inputs.py")) <= {"__future__", "numpy"}


def test_plain_c_consumer_builds_and_runs(tmp_path):
    """tests/c/abi_consumer.c: the header compiles as strict C11, the library
    links from C, and the host-only entry points answer as documented."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(m.library_path())
    exe = str(tmp_path / "abi_consumer")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_consumer.c"), "-L", lib_dir, "-lmera", "-lm",
                    f"-Wl,-rpath,{lib_dir}", "-o", exe], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "abi consumer ok"


def test_library_exports_nothing_undeclared():
    """Every exported mera_* symbol of the shared library is declared (and so
    documented) in include/mera.h."""
    import shutil
    import subprocess

    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("no nm")
    out = subprocess.run([nm, "-D", "--defined-only", m.library_path()], check=True, capture_output=True,
                         text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("mera_")}
    assert exported == set(_declared_symbols())


def test_parity_growth_map_keeps_every_charge():
    """grow._leg_map with the parity: one-to-one, and each old basis state
    lands on a new state of the same charge (bond legs: the first ceil(dim/2)
    states even)."""
    from paper_1906_12030_gb300 import grow

    for old, new in ((2, 3), (4, 6), (5, 8), (8, 16), (16, 32), (3, 3)):
        mp = grow._leg_map(old, new, True)
        assert len(set(mp)) == old and max(mp) < new
        po, pn = I.parity_labels(old), I.parity_labels(new)
        assert all(po[i] == pn[j] for i, j in enumerate(mp))
        assert grow._leg_map(old, new, False) == list(range(old))


def test_batch_lanes_put_gpu_filling_meras_in_one_lane():
    """MERAs whose sweep fills the GPU (>= 1e14 flops: chi >= 20 here) share
    lane 0 and run one after another; the others get lanes of their own while
    the budget lasts."""
    chis = [8, 32, 12, 16, 24, 8, 20, 12]
    dims = _batch_dims(chis)
    need = _sweep_need(dims, m.PREC_BF16X3)
    lanes, lane_bytes = m.mera_batch_lanes(dims, m.PREC_BF16X3, sum(need), max_lanes=32)
    big = [i for i, c in enumerate(chis) if c >= 20]
    small = [i for i, c in enumerate(chis) if c < 20]
    assert all(lanes[i] == 0 for i in big)
    assert sorted(lanes[i] for i in small) == list(range(1, len(small) + 1))
    assert lane_bytes[0] == max(need[i] for i in big)
    assert all(lane_bytes[lanes[i]] >= need[i] for i in range(len(chis)))


def test_batch_lanes_shared_lane_grows_for_a_joining_mera():
    """With n_pow = 20000 the MERA with a chi = 12 scale-invariant layer is
    GPU-filling (lane 0) while the one with a 16 -> 8 transitional layer is
    not, though its scratch is larger.  With one lane allowed, it joins lane
    0, whose scratch must grow to hold it."""
    dims = [([4, 8, 12], [8, 12, 12]), ([4, 16, 8], [16, 8, 8])]
    need = _sweep_need(dims, m.PREC_BF16X3)
    assert need[1] > need[0]
    lanes, lane_bytes = m.mera_batch_lanes(dims, m.PREC_BF16X3, sum(need), max_lanes=1, n_pow=20000)
    assert lanes == [0, 0] and lane_bytes == [need[1]]
    with pytest.raises(m.MeraError, match="budget"):
        m.mera_batch_lanes(dims, m.PREC_BF16X3, need[1] - 1, max_lanes=1, n_pow=20000)


def test_batch_lanes_hold_every_member_for_random_batches():
    """Random batches of three-layer MERAs (transitional layers that grow or
    shrink the bond dimension), power-step counts from 20 to 20000, budgets
    from tight to loose and one to three lanes: every lane's scratch holds
    each of its members and the lanes fit in the budget, or the call reports
    MERA_ENOMEM."""
    shapes = [([4, a, b], [a, b, b]) for a in (4, 8, 12, 16) for b in (2, 4, 6, 8, 12, 16) if b <= a * a]
    need_of = dict(zip(range(len(shapes)), _sweep_need(shapes, m.PREC_BF16X3)))
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(300):
        idx = [int(i) for i in rng.integers(0, len(shapes), int(rng.integers(2, 6)))]
        dims = [shapes[i] for i in idx]
        need = [need_of[i] for i in idx]
        n_pow = int(rng.choice([20, 2000, 20000]))
        max_lanes = int(rng.integers(1, 4))
        budget = max(need) + int(sum(need) * rng.uniform(0.0, 1.0))
        try:
            lanes, lane_bytes = m.mera_batch_lanes(dims, m.PREC_BF16X3, budget, max_lanes, n_pow=n_pow)
        except m.MeraError as e:
            assert "budget" in str(e)
            continue
        assert len(lane_bytes) <= max_lanes and sum(lane_bytes) <= budget
        assert all(lane_bytes[lanes[i]] >= need[i] for i in range(len(dims)))
        checked += 1
    assert checked > 200
