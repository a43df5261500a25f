"""Row shards of one apply (left sectors of y split over S plans) on one GPU.

Each shard plan writes exactly its y blocks; summing the shards' outputs (zero-filled
buffers, as an all-reduce would across GPUs) reproduces the whole plan's y bitwise,
because every y tile is computed by the same task with the same contraction order.
"""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff              # noqa: E402
from tests.helpers import library_problem             # noqa: E402


@pytest.mark.parametrize("name,prec,S", [("spin_m1024", "bf16x3", 3), ("electron_m256", "tf32x3", 2),
                                         ("spin_m384", "fp64", 4)])
def test_row_shards_sum_to_whole_apply(name, prec, S):
    w = wl.workload_by_name(name)
    lays, bufs = library_problem(w)
    io = "f64" if prec == "fp64" else "f32"
    dt = torch.float64 if io == "f64" else torch.float32
    d = {k: torch.from_numpy(np.asarray(bufs[k])).to("cuda", dt) for k in ("L", "W1", "W2", "R")}
    x = torch.from_numpy(bufs["x"][0]).to("cuda", dt)
    whole = heff.Plan(*lays, bufs["W1"], bufs["W2"], prec, io)
    y = torch.empty_like(x)
    heff.heff_apply(whole.handle, d["L"], d["W1"], d["W2"], d["R"], x, y, whole.workspace())
    total = torch.zeros_like(x)
    owned = np.zeros(lays[4].nelem, dtype=bool)
    for r in range(S):
        P = heff.Plan(*lays, bufs["W1"], bufs["W2"], prec, io, shard=(r, S))
        ys = torch.zeros_like(x)
        heff.heff_apply(P.handle, d["L"], d["W1"], d["W2"], d["R"], x, ys, P.workspace())
        total += ys
        secs = set(int(s) for s in heff.heff_plan_shard_sectors(P.handle))
        for key, off, size in lays[4].blocks():
            if key[0] in secs:
                assert not owned[off:off + size].any()
                owned[off:off + size] = True
    torch.cuda.synchronize()
    assert owned.all()
    assert torch.equal(total, y)
