"""Host-side tests of the C library (no GPU needed).

* the library loads and exports every symbol declared in include/heff.h;
* heff_qn_block_layout enumerates exactly the oracle's allowed blocks, in the same
  lexicographic order, with dense row-major offsets;
* the plan's canonical flop count equals the oracle's count;
* the plan's schedule tables, executed by a numpy interpreter, reproduce the oracle's
  y = K x (FP64, 1e-12) for spin and electron problems, including ragged sectors;
* argument validation returns the documented error codes.
"""
import os
import re

import numpy as np
import pytest

import workloads as wl
from oracle import heff as oh
from oracle.blocks import Index, allowed_keys
from paper_2007_05540_gb300 import heff
from tests.helpers import library_problem, interpret_plan, oracle_flat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    src = open(os.path.join(ROOT, "include", "heff.h")).read()
    declared = set(re.findall(r"\b(heff_[a-z0-9_]+)\s*\(", src))
    assert len(declared) >= 15
    for name in sorted(declared):
        assert hasattr(heff._lib, name), name
    assert set(heff.EXPORTED) == declared   # every declared entry has a binding, and no more
    assert heff.heff_version().startswith("heff-gb300")


@pytest.mark.parametrize("name", ["spin_m24", "electron_m40"])
def test_layout_matches_oracle_enumeration(name):
    w = wl.workload_by_name(name)
    lays, _ = library_problem(w)
    Ll, W1l, W2l, Rl, xl = lays
    alpha, beta = Index(w.alpha_q, w.alpha_d), Index(w.beta_q, w.beta_d)
    phys = Index(w.phys, np.ones(len(w.phys)))
    ch = lambda q: Index(q, np.ones(len(q)))
    cases = [
        (xl, [alpha, phys, phys, beta], (1, 1, 1, -1)),
        (Ll, [alpha, ch(w.ql), alpha], (-1, 1, 1)),
        (Rl, [beta, ch(w.qr), beta], (-1, 1, 1)),
        (W1l, [ch(w.ql), phys, phys, ch(w.qm)], (1, 1, -1, -1)),
    ]
    for lay, idx, flows in cases:
        keys = allowed_keys(idx, flows, np.zeros(w.nq))
        assert [tuple(k) for k in lay.keys] == keys
        sizes = [int(np.prod([ix.dims[s] for ix, s in zip(idx, k)])) for k in keys]
        assert list(lay.offsets) == list(np.concatenate([[0], np.cumsum(sizes)[:-1]]))
        assert lay.nelem == sum(sizes)


def _plan(w, lays, bufs, precision="fp64", io="f64"):
    Ll, W1l, W2l, Rl, xl = lays
    return heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], precision, io)


@pytest.mark.parametrize("name", ["spin_m24", "spin_m64", "electron_m40", "electron_m96", "spin_j1j2_6x6_m200",
                                  "electron_hubbard_4x8_m96", "spin_j1j2_20x10_m200", "electron_tri_xc6_m96"])
def test_canonical_flops_match_oracle(name):
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs)
    L, W1, W2, R, x = oh.problem_from_workload(w)
    assert P.flops_canonical == oh.canonical_flops(L, W1, W2, R, x)["total"]


@pytest.mark.parametrize("name,prec", [("spin_m24", "fp64"), ("spin_m64", "fp64"),
                                       ("electron_m40", "fp64"), ("spin_m64", "bf16x3"),
                                       ("electron_m96", "bf16x3"), ("electron_hubbard_4x8_m96", "bf16x3"),
                                       ("spin_m200", "tf32x3"), ("electron_tri_xc6_m96", "bf16x3")])
def test_plan_schedule_reproduces_oracle(name, prec):
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs, prec, "f64" if prec == "fp64" else "f32")
    L, W1, W2, R, x = oh.problem_from_workload(w)
    y_ref = oracle_flat(lays[4], oh.heff_apply(L, W1, W2, R, x))
    y = interpret_plan(P, bufs, bufs["x"][0])
    assert not np.isnan(y).any()
    assert np.abs(y - y_ref).max() < 1e-12 * np.abs(y_ref).max()


def test_plan_rejects_bad_arguments():
    w = wl.workload_by_name("spin_m24")
    lays, bufs = library_problem(w)
    Ll, W1l, W2l, Rl, xl = lays
    with pytest.raises(heff.HeffError) as e:
        heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], "fp64", "f32")
    assert e.value.code == -3
    with pytest.raises(heff.HeffError) as e:          # L and R swapped: charge mismatch
        heff.Plan(Rl, W1l, W2l, Ll, xl, bufs["W1"], bufs["W2"], "fp64", "f64")
    assert e.value.code == -2
    with pytest.raises(heff.HeffError) as e:
        heff.heff_qn_block_layout([(np.array([[0]]), np.array([0]), 1)])
    assert e.value.code == -1


def test_host_only_plan_refuses_compute():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    w = wl.workload_by_name("spin_m24")
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs)
    t = torch.zeros(16, dtype=torch.float64)
    rc = heff._lib.heff_apply_prepared(P.handle, heff._ptr(t), heff._ptr(t + 1), heff._ptr(t), 128, None)
    assert rc == -3
    assert "without a CUDA device" in heff.heff_last_error()


def test_gradient_workspace_limit_splits_left_sectors():
    """A workspace limit streams the gradient intermediates in left-sector chunks; the
    workspace stays within the limit, and a limit below one sector's need is refused."""
    w = wl.workload_by_name("spin_m200")
    lays, bufs = library_problem(w)
    hs = [t.handle for t in lays]

    def make(limit):
        return heff.heff_grad_plan_create(*hs, bufs["W1"], bufs["W2"], limit)
    g = make(0)
    whole = heff.heff_grad_workspace_size(g)
    assert heff.heff_grad_chunks(g) == 1
    heff.heff_grad_plan_destroy(g)
    last = 1
    for frac in (0.75, 0.5, 0.4):
        g = make(int(whole * frac))
        n = heff.heff_grad_chunks(g)
        assert heff.heff_grad_workspace_size(g) <= int(whole * frac)
        assert n >= last and n >= 2
        last = n
        heff.heff_grad_plan_destroy(g)
    with pytest.raises(heff.HeffError) as e:
        make(int(whole * 0.05))
    assert e.value.code == -7
    assert "minimum" in heff.heff_last_error()


def test_block_product_precision_switch_keeps_the_work():
    """Re-tiling the environment-update and gradient block lists for the tensor cores
    (128 x 128 output tiles) and back leaves their flop counts unchanged; other precisions
    are refused."""
    w = wl.workload_by_name("spin_m200")
    lays, bufs = library_problem(w)
    hs = [t.handle for t in lays]
    g = heff.heff_grad_plan_create(*hs, bufs["W1"], bufs["W2"], 0)
    for prec in ("bf16x3", "fp64", "bf16x3"):
        heff.heff_grad_plan_set_precision(g, prec)
    with pytest.raises(heff.HeffError) as e:
        heff.heff_grad_plan_set_precision(g, "tf32x3")
    assert e.value.code == -3
    heff.heff_grad_plan_destroy(g)
    Ll = lays[0]
    ones = lambda n: np.ones(n, dtype=np.int32)
    gq, gd = wl.binomial_sectors(220, 11, 3, parity=0)
    site = heff.Layout([(w.alpha_q, w.alpha_d, 1), (w.phys, ones(2), 1), (gq, gd, -1)])
    Wl = heff.Layout([(w.ql, ones(len(w.ql)), 1), (w.phys, ones(2), 1), (w.phys, ones(2), -1),
                      (w.qm, ones(len(w.qm)), -1)])
    new = heff.Layout([(gq, gd, -1), (w.qm, ones(len(w.qm)), 1), (gq, gd, 1)])
    P = heff.heff_env_plan_create(Ll.handle, site.handle, Wl.handle, new.handle, Wl.assemble(lambda k: w.W1[k]),
                                  "left")
    f0 = heff.heff_env_flops(P)
    heff.heff_env_plan_set_precision(P, "bf16x3")
    assert heff.heff_env_flops(P) == f0 > 0
    heff.heff_env_plan_set_precision(P, "fp64")
    assert heff.heff_env_flops(P) == f0
    heff.heff_env_plan_destroy(P)


def _row_block_mask(xl, sectors):
    """Flat mask of the y blocks whose left sector is in `sectors`."""
    mask = np.zeros(xl.nelem, dtype=bool)
    for key, off, size in xl.blocks():
        if key[0] in set(int(s) for s in sectors):
            mask[off:off + size] = True
    return mask


@pytest.mark.parametrize("name,prec,S", [("spin_m64", "fp64", 3), ("electron_m40", "bf16x3", 2),
                                         ("electron_m96", "fp64", 5)])
def test_row_shards_partition_and_sum_to_oracle(name, prec, S):
    """Row shards own disjoint left sectors covering y; each writes exactly its blocks,
    and the sum of the shards' outputs is the oracle's y."""
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    Ll, W1l, W2l, Rl, xl = lays
    io = "f64" if prec == "fp64" else "f32"
    whole = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], prec, io)
    L, W1, W2, R, x = oh.problem_from_workload(w)
    y_ref = oracle_flat(xl, oh.heff_apply(L, W1, W2, R, x))
    total = np.zeros(xl.nelem)
    seen, canon = [], 0.0
    for r in range(S):
        P = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], prec, io, shard=(r, S))
        secs = heff.heff_plan_shard_sectors(P.handle)
        seen.extend(int(s) for s in secs)
        canon += P.flops_canonical
        y = interpret_plan(P, bufs, bufs["x"][0])
        mine = _row_block_mask(xl, secs)
        assert not np.isnan(y[mine]).any()
        assert np.isnan(y[~mine]).all()            # other shards' blocks are not written
        total[mine] += y[mine]
    assert sorted(seen) == list(range(len(w.alpha_d)))
    assert canon == pytest.approx(whole.flops_canonical, rel=1e-12)
    assert np.abs(total - y_ref).max() < 1e-12 * np.abs(y_ref).max()


def test_row_shard_arguments_checked():
    w = wl.workload_by_name("spin_m24")
    lays, bufs = library_problem(w)
    for shard in ((2, 2), (-1, 2), (1, 0)):
        with pytest.raises(heff.HeffError) as e:
            heff.Plan(*lays, bufs["W1"], bufs["W2"], "fp64", "f64", shard=shard)
        assert e.value.code == -1
    P = heff.Plan(*lays, bufs["W1"], bufs["W2"], "fp64", "f64", shard=(0, 1))
    assert list(heff.heff_plan_shard_sectors(P.handle)) == list(range(len(w.alpha_d)))


def test_select_tiles_swaps_task_lists():
    """All tile variants are planned; selecting one swaps its task list in (the schedule
    still reproduces the oracle), unknown variants and FP64 plans are refused."""
    w = wl.workload_by_name("spin_m64")
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs, "bf16x3", "f32")
    assert (P.stats[15], P.stats[22]) == (256, 256)
    L, W1, W2, R, x = oh.problem_from_workload(w)
    y_ref = oracle_flat(lays[4], oh.heff_apply(L, W1, W2, R, x))
    for code in (heff.TILE_128, heff.TILE_PAIR_256, heff.TILE_256):
        heff.heff_plan_select_tiles(P.handle, code, code)
        st = heff.heff_plan_stats(P.handle)
        assert (st[15], st[22]) == (code, code)
        P.stats = st
        y = interpret_plan(P, bufs, bufs["x"][0])
        assert np.abs(y - y_ref).max() < 1e-12 * np.abs(y_ref).max()
    with pytest.raises(heff.HeffError):
        heff.heff_plan_select_tiles(P.handle, 64, 0)
    P64 = _plan(w, lays, bufs, "fp64", "f64")
    with pytest.raises(heff.HeffError):
        heff.heff_plan_select_tiles(P64.handle, 128, 0)


@pytest.mark.parametrize("name", ["spin_m200", "electron_m96", "spin_m1024_s8"])
def test_pair_entries_share_b_rows_and_segments(name):
    """CTA-pair lists: tasks 2e and 2e + 1 load the same B rows with the same K segments (one
    B box serves both); a ghost partner has no rows; every real tile of the single-CTA list
    appears exactly once."""
    w = wl.spin_heff_workload(1024, 8, 21, name=name) if name == "spin_m1024_s8" else wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs, "bf16x3", "f32")
    for which in (3, 5):
        single = heff.heff_plan_export(P.handle, which)
        heff.heff_plan_select_tiles(P.handle, heff.TILE_PAIR_256, heff.TILE_PAIR_256)
        pairs = heff.heff_plan_export(P.handle, which)
        segs = heff.heff_plan_export(P.handle, which + 1)
        heff.heff_plan_select_tiles(P.handle, heff.TILE_256, heff.TILE_256)
        assert len(pairs) % 2 == 0
        seg = lambda t: segs[t["seg_begin"]:t["seg_begin"] + t["seg_count"]].tolist()
        for a, b in zip(pairs[0::2], pairs[1::2]):
            if a["seg_count"] == 0 or b["seg_count"] == 0:
                assert a["seg_count"] == b["seg_count"] == 0          # no ring use on either side
                continue
            assert a["b_row"] == b["b_row"] and a["n"] == b["n"] and a["ktotal"] == b["ktotal"]
            assert seg(a) == seg(b)
            assert a["m"] > 0                                          # rank 0 is never a ghost
        key = lambda t: (int(t["a_row"]), int(t["b_row"]), int(t["c_off"]), int(t["m"]), int(t["n"]))
        real = sorted(key(t) for t in pairs if t["m"] > 0)
        assert real == sorted(key(t) for t in single if t["m"] > 0)


def test_product_state_reaches_total_charge():
    from paper_2007_05540_gb300 import dmrg
    sp = wl.spin_phys()
    st = dmrg.product_state(sp, 16, (0,))
    assert sum(int(sp[s][0]) for s in st) == 0 and len(st) == 16
    el = wl.electron_phys()
    st = dmrg.product_state(el, 6, (6, 0))
    assert tuple(map(int, el[st].sum(axis=0))) == (6, 0)
    with pytest.raises(ValueError):
        dmrg.product_state(sp, 3, (0,))          # odd chain cannot reach 2Sz = 0



def test_wait_status_entries_check_arguments_before_touching_the_device():
    """heff_workspace_status / heff_wait_selftest reject bad arguments on the host (no CUDA
    call is made); an FP64 plan has no device-side waits, so its status is HEFF_OK unread."""
    import types

    import torch
    w = wl.workload_by_name("spin_m24")
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs, "bf16x3", "f32")
    small = torch.empty(16, dtype=torch.uint8)          # host memory, never dereferenced
    st = types.SimpleNamespace(cuda_stream=0)            # legacy stream handle, never used
    assert heff.heff_workspace_status(None, small, st) == -1                 # INVALID_ARG
    assert heff.heff_workspace_status(P.handle, small, st) == -7             # WORKSPACE: too small
    for kind in (2, -1):
        with pytest.raises(heff.HeffError) as e:
            heff.heff_wait_selftest(P.handle, small, kind, st)
        assert e.value.code == -1
    with pytest.raises(heff.HeffError) as e:
        heff.heff_wait_selftest(P.handle, small, 0, st)
    assert e.value.code == -7
    P64 = _plan(w, lays, bufs, "fp64", "f64")
    assert heff.heff_workspace_status(P64.handle, small, st) == 0
    with pytest.raises(heff.HeffError) as e:
        heff.heff_wait_selftest(P64.handle, small, 0, st)
    assert e.value.code == -1


def test_ground_state_and_block_status_entries_check_arguments():
    """heff_ground_state, heff_env_status and heff_grad_status reject bad arguments on the host
    before any CUDA call; FP64 block products have no device-side waits (status HEFF_OK)."""
    import types

    import torch
    w = wl.workload_by_name("spin_m24")
    lays, bufs = library_problem(w)
    st = types.SimpleNamespace(cuda_stream=0)
    t = torch.zeros(64, dtype=torch.float64)             # host memory, never dereferenced
    small = torch.empty(16, dtype=torch.uint8)
    Pb = _plan(w, lays, bufs, "bf16x3", "f64")
    P32 = _plan(w, lays, bufs, "bf16x3", "f32")
    # null tensors / output
    with pytest.raises(heff.HeffError) as e:
        heff.heff_ground_state(Pb.handle, None, None, t, t, t, t, 10, 2, 1e-8, t, small, None, small, st)
    assert e.value.code == -1
    # io dtype: the eigensolvers need FP64 tensors
    with pytest.raises(heff.HeffError) as e:
        heff.heff_ground_state(P32.handle, None, t, t, t, t, t, 10, 2, 1e-8, t, small, None, small, st)
    assert e.value.code == -3
    # step count, cycles, tolerance
    for n_iter, cycles, tol in ((0, 2, 1e-8), (127, 2, 1e-8), (10, 0, 1e-8), (10, 2, -1.0)):
        with pytest.raises(heff.HeffError) as e:
            heff.heff_ground_state(Pb.handle, None, t, t, t, t, t, n_iter, cycles, tol, t, small, None, small, st)
        assert e.value.code == -1
    # the FP64 plan must be FP64
    with pytest.raises(heff.HeffError) as e:
        heff.heff_ground_state(Pb.handle, Pb.handle, t, t, t, t, t, 10, 2, 1e-8, t, small, small, small, st)
    assert e.value.code == -1
    # a workspace below heff_ground_state_workspace_size
    assert heff.heff_ground_state_workspace_size(Pb.handle, 10) > small.numel()
    with pytest.raises(heff.HeffError) as e:
        heff.heff_ground_state(Pb.handle, None, t, t, t, t, t, 10, 2, 1e-8, t, small, None, small, st)
    assert e.value.code == -7
    # status calls
    hs = [x.handle for x in lays]
    g = heff.heff_grad_plan_create(*hs, bufs["W1"], bufs["W2"], 0)
    assert heff.heff_grad_status(g, small, st) == 0                       # FP64 products: no waits
    heff.heff_grad_plan_set_precision(g, "bf16x3")
    assert heff.heff_grad_status(g, small, st) == -7                      # too small
    assert heff.heff_grad_status(None, small, st) == -1
    heff.heff_grad_plan_destroy(g)


def test_empty_two_site_space_plan():
    """A target charge that no x block satisfies: an empty layout, and a plan with no work."""
    w = wl.workload_by_name("spin_m24")
    lays = heff.heff_layouts((w.alpha_q, w.alpha_d), (w.beta_q, w.beta_d), w.phys, w.ql, w.qm, w.qr,
                             target=np.array([1001], dtype=np.int32))
    assert lays[4].nblocks == 0 and lays[4].nelem == 0
    W1 = lays[1].assemble(lambda k: w.W1[k])
    W2 = lays[2].assemble(lambda k: w.W2[k])
    for prec, io in (("fp64", "f64"), ("bf16x3", "f32"), ("tf32x3", "f32")):
        P = heff.Plan(*lays, W1, W2, prec, io)
        assert P.flops_canonical == 0.0
        st = P.stats
        assert st[3] == 0 and st[4] == 0 and st[5] == 0      # no GEMM tasks, no pack tiles


def test_check_mpo_arguments():
    """heff_plan_check_mpo rejects null tensors on the host and needs a plan with a device."""
    import types

    import torch
    w = wl.workload_by_name("spin_m24")
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs, "fp64", "f64")
    assert len(np.flatnonzero(bufs["W1"] == 0.0)) > 0          # the schedule drops entries
    t = torch.zeros(8, dtype=torch.float64)                     # host memory, never dereferenced
    st = types.SimpleNamespace(cuda_stream=0)
    with pytest.raises(heff.HeffError) as e:
        heff.heff_plan_check_mpo(P.handle, None, t, st)
    assert e.value.code == -1
    if not torch.cuda.is_available():                           # a host-only plan
        with pytest.raises(heff.HeffError) as e:
            heff.heff_plan_check_mpo(P.handle, t, t, st)
        assert e.value.code == -3
