"""Batched applies (many x sharing L, W1, W2, R), the tile autotuner and CUDA-graph capture.

* heff_plan_autotune picks a tile variant per GEMM, and every variant gives bitwise the
  same results (a tile's K accumulation order does not depend on the N tiling or on CTA
  pairing);
* heff_apply_batched captured once in a CUDA graph and replayed gives bitwise the
  results of the uncaptured call, and each batch entry matches the oracle;
* the same at the electron workload's full size with 32 vectors (sampled sectors);
* a batch of 70 vectors (two launches per kernel, 64 entries and 6) equals the single
  applies bitwise.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import heff as oh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff              # noqa: E402
from tests.helpers import library_problem, oracle_flat  # noqa: E402


def _setup(name, nb, prec="bf16x3"):
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w, batches=tuple(range(nb)))
    plan = heff.Plan(*lays, bufs["W1"], bufs["W2"], prec, "f32", max_batch=nb)
    d = {k: torch.from_numpy(np.asarray(bufs[k])).to("cuda", torch.float32) for k in ("L", "W1", "W2", "R")}
    xs = [torch.from_numpy(x).to("cuda", torch.float32) for x in bufs["x"]]
    return w, lays, plan, d, xs


def _batched(plan, d, xs, ws):
    ys = [torch.full_like(x, float("nan")) for x in xs]
    heff.heff_apply_batched(plan.handle, d["L"], d["W1"], d["W2"], d["R"], xs, ys, ws)
    torch.cuda.synchronize()
    return ys


def test_autotune_keeps_results_bitwise():
    w, lays, plan, d, xs = _setup("spin_m1024", 1)
    ws = plan.workspace()
    before = _batched(plan, d, xs, ws)[0].cpu().numpy()
    y = torch.empty_like(xs[0])
    tn = heff.heff_plan_autotune(plan.handle, d["L"], d["W1"], d["W2"], d["R"], xs[0], y, ws)
    assert all(t in (heff.TILE_128, heff.TILE_256, heff.TILE_PAIR_256) for t in tn)
    after = _batched(plan, d, xs, ws)[0].cpu().numpy()
    print("autotuned tile widths", tn)
    assert np.array_equal(before, after)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("name", ["spin_m200", "electron_m256", "spin_j1j2_6x6_m200", "spin_m1024"])
def test_tile_variants_bitwise_equal(name, prec):
    """Every tile variant (N = 256, N = 128, N = 256 in CTA pairs that run one M = 256 tile
    with pair MMAs, each CTA loading its own half of the B rows) gives bitwise the same y for
    a batch of 3 (a tile's K order is the same in all of them), and batch entry 0 matches the
    oracle."""
    w, lays, plan, d, xs = _setup(name, 3, prec)
    ws = plan.workspace()
    out = {}
    for code in (heff.TILE_256, heff.TILE_128, heff.TILE_PAIR_256):
        heff.heff_plan_select_tiles(plan.handle, code, code)
        out[code] = [t.cpu().numpy() for t in _batched(plan, d, xs, ws)]
    for code in (heff.TILE_128, heff.TILE_PAIR_256):
        for b in range(3):
            assert np.array_equal(out[code][b], out[heff.TILE_256][b]), (code, b)
    L, W1, W2, R, x = oh.problem_from_workload(w, 0)
    y_ref = oracle_flat(lays[4], oh.heff_apply(L, W1, W2, R, x))
    y = out[heff.TILE_PAIR_256][0].astype(np.float64)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < (1e-3 if prec == "bf16x3" else 1e-5)


def test_batched_graph_capture_matches_eager_and_oracle():
    nb = 4
    w, lays, plan, d, xs = _setup("electron_m256", nb)
    ws = plan.workspace()
    y = torch.empty_like(xs[0])
    heff.heff_plan_autotune(plan.handle, d["L"], d["W1"], d["W2"], d["R"], xs[0], y, ws)
    eager = [t.cpu().numpy() for t in _batched(plan, d, xs, ws)]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):      # warm-up on the capture stream
        heff.heff_apply_batched(plan.handle, d["L"], d["W1"], d["W2"], d["R"], xs, ys, ws, stream)
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    for t in ys:
        t.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        heff.heff_apply_batched(plan.handle, d["L"], d["W1"], d["W2"], d["R"], xs, ys, ws, stream)
    for _ in range(2):
        for t in ys:
            t.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for b in range(nb):
            assert np.array_equal(ys[b].cpu().numpy(), eager[b])
    for b in range(nb):
        L, W1, W2, R, x = oh.problem_from_workload(w, b)
        ref = oracle_flat(lays[4], oh.heff_apply(L, W1, W2, R, x))
        err = np.linalg.norm(eager[b] - ref) / np.linalg.norm(ref)
        assert err < 1e-3, err


def test_electron_full_size_batch_of_32_sampled():
    nb = 32
    w, lays, plan, d, xs = _setup("electron_m2048", nb)
    ws = plan.workspace()
    ys = _batched(plan, d, xs, ws)
    keep = {0, 30, 60}
    mask = np.zeros(lays[4].nelem, dtype=bool)
    for key, off, size in lays[4].blocks():
        if key[0] in keep:
            mask[off:off + size] = True
    for b in (0, 17, 31):
        L, W1, W2, R, x = oh.problem_from_workload(w, b)
        ref = oracle_flat(lays[4], oh.heff_apply(L, W1, W2, R, x, left_sectors=keep))
        yb = ys[b].double().cpu().numpy()
        assert not np.isnan(yb).any()
        err = np.linalg.norm(yb[mask] - ref[mask]) / np.linalg.norm(ref[mask])
        print(f"electron m=2048 batch entry {b}: rel err {err:.2e}")
        assert err < 1e-3


@pytest.mark.parametrize("pinned", [True, False])
def test_apply_host_equals_device_apply(pinned):
    """heff_apply_host (host inputs -> staging -> apply -> host y) gives bitwise the result
    of heff_apply on device copies of the same inputs, on two alternating streams."""
    w, lays, plan, d, xs = _setup("spin_m1024", 1)
    ws = [plan.workspace(), plan.workspace()]
    y_dev = torch.empty_like(xs[0])
    heff.heff_apply(plan.handle, d["L"], d["W1"], d["W2"], d["R"], xs[0], y_dev, ws[0])
    torch.cuda.synchronize()
    host = {k: v.cpu() for k, v in d.items()}
    host["x"] = xs[0].cpu()
    if pinned:
        host = {k: v.pin_memory() for k, v in host.items()}
    ys = [torch.full((xs[0].numel(),), float("nan"), dtype=torch.float32) for _ in range(2)]
    if pinned:
        ys = [t.pin_memory() for t in ys]
    staging = [torch.empty(heff.heff_apply_host_staging_size(plan.handle), dtype=torch.uint8, device="cuda")
               for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(4):
        j = k % 2
        heff.heff_apply_host(plan.handle, host["L"], host["W1"], host["W2"], host["R"], host["x"], ys[j],
                             staging[j], ws[j], streams[j])
    torch.cuda.synchronize()
    ref = y_dev.cpu()
    for t in ys:
        assert torch.equal(t, ref)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_batch_of_more_than_one_launch(prec):
    """70 vectors run as two launches per kernel (64 entries, then 6): the later launch's
    pack, GEMM 1 and GEMM 2 address their entries by the absolute batch index in the
    interleaved hi/lo operand rows.  Every entry equals its own apply bitwise, and entries
    0, 64 and 69 match the oracle."""
    nb = 70
    w, lays, plan, d, xs = _setup("spin_m64", nb, prec)
    ws = plan.workspace()
    ys = _batched(plan, d, xs, ws)
    for b in (0, 1, 63, 64, 65, 69):
        y1 = torch.full_like(xs[b], float("nan"))
        heff.heff_apply(plan.handle, d["L"], d["W1"], d["W2"], d["R"], xs[b], y1, ws)
        torch.cuda.synchronize()
        assert torch.equal(ys[b], y1), b
    for b in (0, 64, 69):
        L, W1, W2, R, x = oh.problem_from_workload(w, b)
        y_ref = oracle_flat(lays[4], oh.heff_apply(L, W1, W2, R, x))
        y = ys[b].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < (1e-3 if prec == "bf16x3" else 1e-5)
