"""Device-side bounded waits give up instead of hanging, and the host learns of it.

A single-block kernel waits, with the GEMM kernels' own mbarrier wait (kind 0) or at the
SVD sweeps' grid barrier (kind 1), on something nothing completes.  The wait must expire
after its cycle limit (about 1.5 s / 1 s), set the workspace's sticky error flag, which
heff_workspace_status reports as HEFF_ERR_TIMEOUT and clears, and leave the context
usable: an apply afterwards still matches the oracle.  No kernel faults or traps.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected only with -m gpu on CPU
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff                       # noqa: E402
from tests.helpers import oracle_flat                           # noqa: E402
from tests.test_gpu_parity import Lib, _compare, _oracle, TOL  # noqa: E402

import workloads as wl                                          # noqa: E402

HEFF_ERR_TIMEOUT = -6


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_expires_and_context_stays_usable(kind):
    w = wl.workload_by_name("spin_m64")
    lib = Lib(w, "bf16x3")
    y_ref = oracle_flat(lib.lays[4], _oracle(w))
    _compare(lib.apply(), y_ref, TOL["bf16x3"])
    assert heff.heff_workspace_status(lib.plan.handle, lib.ws) == 0

    ms = heff.heff_wait_selftest(lib.plan.handle, lib.ws, kind)
    print(f"kind {kind}: wait expired after {ms:.1f} ms")
    # the limits are 3 * 2^30 (kind 0) and 2^31 (kind 1) SM cycles: ~0.5-2.5 s at the
    # clocks a GB300 runs (2.07 GHz at most)
    assert 300.0 < ms < 5000.0, ms
    assert heff.heff_workspace_status(lib.plan.handle, lib.ws) == HEFF_ERR_TIMEOUT
    assert "expired" in heff.heff_last_error()
    assert heff.heff_workspace_status(lib.plan.handle, lib.ws) == 0   # read clears it

    _compare(lib.apply(), y_ref, TOL["bf16x3"])
    assert heff.heff_workspace_status(lib.plan.handle, lib.ws) == 0


def test_workspace_status_fp64_plan_has_no_waits():
    w = wl.workload_by_name("spin_m64")
    lib = Lib(w, "fp64")
    _compare(lib.apply(), oracle_flat(lib.lays[4], _oracle(w)), TOL["fp64"])
    assert heff.heff_workspace_status(lib.plan.handle, lib.ws) == 0
    with pytest.raises(heff.HeffError):
        heff.heff_wait_selftest(lib.plan.handle, lib.ws, 0)
