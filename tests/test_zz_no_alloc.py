"""heff_apply_noalloc: the entry point for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: code running under another
framework's memory manager that has already reserved the device memory it may use, or
code on a latency-critical path where cudaMalloc's implicit device synchronisation is
not acceptable.  heff_apply_noalloc serves them from a workspace array compiled into the
library (HEFF_NOALLOC_WORKSPACE_BYTES per GPU).  The paper has no counterpart of it.

The test calls it through the C ABI twice in a row and compares each result with
heff_apply on a caller-owned workspace, within the parity tolerance of the precision.
It sits in its own file, collected last, so that if it fails a run stopping at the first
failure has already run every other test; it needs no state from other tests.
"""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected only with -m gpu on CPU
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff           # noqa: E402
from tests.helpers import library_problem          # noqa: E402

TOL = {"fp64": 1e-10, "bf16x3": 1e-3, "tf32x3": 1e-5}


def _setup(name, prec):
    io = "f64" if prec == "fp64" else "f32"
    dt = torch.float64 if io == "f64" else torch.float32
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    Ll, W1l, W2l, Rl, xl = lays
    plan = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], prec, io)
    dev = {k: torch.from_numpy(np.asarray(bufs[k] if k != "x" else bufs["x"][0])).to("cuda", dt)
           for k in ("L", "W1", "W2", "R", "x")}
    return plan, dev


@pytest.mark.parametrize("name,prec", [("spin_m1024", "bf16x3"), ("spin_m200", "fp64"),
                                       ("electron_m256", "tf32x3")])
def test_noalloc_matches_apply_on_two_calls(name, prec):
    plan, d = _setup(name, prec)
    assert plan.workspace_bytes <= heff.NOALLOC_WORKSPACE_BYTES
    ws = plan.workspace()
    ref = torch.full_like(d["x"], float("nan"))
    heff.heff_apply(plan.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], ref, ws)
    torch.cuda.synchronize()
    ref = ref.double().cpu().numpy()
    assert not np.isnan(ref).any()
    for _ in range(2):
        y = torch.full_like(d["x"], float("nan"))
        heff.heff_apply_noalloc(plan.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], y)
        torch.cuda.synchronize()
        assert heff.heff_apply_noalloc_status(plan.handle) == 0    # no bounded wait expired
        y = y.double().cpu().numpy()
        assert not np.isnan(y).any()
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert err < TOL[prec], f"{name} {prec}: rel err {err:.3e}"


def test_noalloc_rejects_plans_beyond_the_builtin_workspace():
    plan, d = _setup("spin_m4096", "bf16x3")
    assert plan.workspace_bytes > heff.NOALLOC_WORKSPACE_BYTES
    y = torch.empty_like(d["x"])
    with pytest.raises(heff.HeffError) as e:
        heff.heff_apply_noalloc(plan.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], y)
    assert e.value.code == -7
    assert "HEFF_NOALLOC_WORKSPACE_BYTES" in str(e.value)
