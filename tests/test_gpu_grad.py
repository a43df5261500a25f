"""GPU Rayleigh-quotient gradients (heff_backward) against the oracle.

The oracle's gradients are pinned by central finite differences, Euler homogeneity and
the closed form for dx (tests/test_oracle_eig_svd_dmrg_grad.py).  Here the GPU results
(FP64 apply plan) must equal them to 1e-11 relative; the gradient with respect to the
tagged J2 coupling (through W1 and W2 only) must equal a central difference of the GPU
rho; with a BF16x3 apply plan only rho and dx carry the split-precision error.  With a
workspace limit the intermediates are streamed in left-sector chunks: the results equal the
unchunked ones (rho, dx and dL bitwise; dR and the W gradients, sums over the chunks, to
1e-13), including at m = 4096, where the oracle's rho and Euler homogeneity also hold.
"""
import numpy as np
import pytest

import workloads as wl
from workloads.fill import spin_window, SPIN_COUPLINGS
from oracle import heff as oh, grad as ograd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff              # noqa: E402
from tests.helpers import library_problem             # noqa: E402


def _dev(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float64)).to("cuda")


class GradRun:
    def __init__(self, w, prec="fp64", ws_limit=0, problem=None, plan=None, gprec="fp64"):
        self.w = w
        self.lays, self.bufs = problem if problem is not None else library_problem(w)
        Ll, W1l, W2l, Rl, xl = self.lays
        self.plan = plan if plan is not None else heff.Plan(Ll, W1l, W2l, Rl, xl, self.bufs["W1"], self.bufs["W2"],
                                                            prec, "f64")
        self.g = heff.heff_grad_plan_create(Ll.handle, W1l.handle, W2l.handle, Rl.handle, xl.handle,
                                            self.bufs["W1"], self.bufs["W2"], ws_limit)
        heff.heff_grad_plan_set_precision(self.g, gprec)
        self.aws = self.plan.workspace()
        self.gws = torch.empty(heff.heff_grad_workspace_size(self.g), dtype=torch.uint8, device="cuda")

    def run(self, W1=None, W2=None):
        b = self.bufs
        d = {k: _dev(b[k]) for k in ("L", "R")}
        d["W1"] = _dev(b["W1"] if W1 is None else W1)
        d["W2"] = _dev(b["W2"] if W2 is None else W2)
        x = _dev(b["x"][0])
        rho = torch.empty((), dtype=torch.float64, device="cuda")
        out = [torch.full_like(t, float("nan")) for t in (x, d["L"], d["R"], d["W1"], d["W2"])]
        heff.heff_backward(self.g, self.plan.handle, d["L"], d["W1"], d["W2"], d["R"], x, rho, *out,
                           self.aws, self.gws)
        torch.cuda.synchronize()
        return float(rho), [t.cpu().numpy() for t in out]

    def __del__(self):
        heff.heff_grad_plan_destroy(self.g)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", ["spin_m64", "electron_m96", "spin_m200"])
def test_backward_matches_oracle(name):
    w = wl.workload_by_name(name)
    r = GradRun(w)
    rho, (dx, dL, dR, dW1, dW2) = r.run()
    L, W1, W2, R, x = oh.problem_from_workload(w)
    ref = ograd.grad_all(L, W1, W2, R, x)
    Ll, W1l, W2l, Rl, xl = r.lays
    assert abs(rho - ref["rho"]) < 1e-12 * abs(ref["rho"])
    errs = {
        "dx": _rel(dx, xl.assemble(lambda k: ref["dx"].blocks[k])),
        "dL": _rel(dL, Ll.assemble(lambda k: ref["dL"].blocks[k])),
        "dR": _rel(dR, Rl.assemble(lambda k: ref["dR"].blocks[k])),
        "dW1": _rel(dW1, W1l.assemble(lambda k: ref["dW1"][k])),
        "dW2": _rel(dW2, W2l.assemble(lambda k: ref["dW2"][k])),
    }
    print(name, {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < 1e-11, (k, v)
    # Euler homogeneity on the GPU results: rho is linear in L, R, W1, W2; degree 0 in x
    b = r.bufs
    for g_, t_ in ((dL, b["L"]), (dR, b["R"]), (dW1, b["W1"]), (dW2, b["W2"])):
        assert abs(float(np.dot(g_, t_)) - rho) < 1e-11 * abs(rho)
    assert abs(float(np.dot(dx, b["x"][0]))) < 1e-11 * abs(rho) * np.linalg.norm(b["x"][0])


def test_backward_j2_coupling_central_difference():
    w = wl.workload_by_name("spin_m64")
    r = GradRun(w)
    W1l, W2l = r.lays[1], r.lays[2]

    def Ws(J2):
        c = list(SPIN_COUPLINGS)
        c[1] = J2
        win = spin_window(tuple(c))
        return W1l.assemble(lambda k: win["W1"][k]), W2l.assemble(lambda k: win["W2"][k])
    J2, h = SPIN_COUPLINGS[1], 1e-6
    rho, (dx, dL, dR, dW1, dW2) = r.run()
    W1p, W2p = Ws(J2 + h)
    W1m, W2m = Ws(J2 - h)
    an = float(np.dot(dW1, (W1p - W1m) / (2 * h)) + np.dot(dW2, (W2p - W2m) / (2 * h)))
    fd = (r.run(W1p, W2p)[0] - r.run(W1m, W2m)[0]) / (2 * h)
    print(f"d rho / d J2: analytic {an:.10f}  central difference {fd:.10f}")
    assert abs(an - fd) < 1e-7 * max(1.0, abs(fd))


def test_backward_with_split_precision_apply():
    w = wl.workload_by_name("spin_m200")
    exact = GradRun(w, "fp64").run()
    rho, grads = GradRun(w, "bf16x3").run()
    assert abs(rho - exact[0]) < 1e-4 * abs(exact[0])
    assert _rel(grads[0], exact[1][0]) < 1e-3                 # dx uses the BF16x3 apply
    for a, b in zip(grads[1:], exact[1][1:]):                 # L, R, W gradients: FP64 only
        assert _rel(a, b) < 1e-13


def test_autograd_function():
    w = wl.workload_by_name("spin_m64")
    r = GradRun(w)
    b = r.bufs
    ts = {k: _dev(b[k]).requires_grad_(True) for k in ("L", "W1", "W2", "R")}
    x = _dev(b["x"][0]).requires_grad_(True)
    rho = heff.RayleighQuotient.apply((r.g, r.plan.handle, r.aws, r.gws), x, ts["L"], ts["W1"], ts["W2"],
                                      ts["R"])
    (3.0 * rho).backward()
    _, (dx, dL, dR, dW1, dW2) = r.run()
    assert np.allclose(x.grad.cpu().numpy(), 3.0 * dx, rtol=0, atol=1e-14 * np.abs(dx).max() + 1e-300)
    assert np.allclose(ts["L"].grad.cpu().numpy(), 3.0 * dL)
    assert np.allclose(ts["W2"].grad.cpu().numpy(), 3.0 * dW2)


def _chunked_limit(r_whole):
    """The smallest accepted workspace limit on a 0.8x ladder below the whole size (the
    most chunks); at least two chunks are required."""
    lays, bufs = r_whole.lays, r_whole.bufs
    Ll, W1l, W2l, Rl, xl = lays
    lim = heff.heff_grad_workspace_size(r_whole.g)
    best = None
    while lim > 0:
        lim = int(lim * 0.8)
        try:
            g = heff.heff_grad_plan_create(Ll.handle, W1l.handle, W2l.handle, Rl.handle, xl.handle,
                                           bufs["W1"], bufs["W2"], lim)
        except heff.HeffError as e:
            assert e.code == -7
            break
        if heff.heff_grad_chunks(g) >= 2:
            best = lim
        heff.heff_grad_plan_destroy(g)
    assert best is not None, "no limit gives two chunks"
    return best


def _compare_streamed(whole, streamed):
    rho0, g0 = whole
    rho1, g1 = streamed
    assert rho1 == rho0
    assert np.array_equal(g1[0], g0[0])                        # dx
    assert np.array_equal(g1[1], g0[1])                        # dL: complete within a chunk
    for k, a, b in zip(("dR", "dW1", "dW2"), g1[2:], g0[2:]):  # sums over the chunks
        assert _rel(a, b) < 1e-13, (k, _rel(a, b))


@pytest.mark.parametrize("name", ["spin_m200", "electron_m256"])
def test_backward_streamed_chunks_equal_whole(name):
    w = wl.workload_by_name(name)
    whole = GradRun(w)
    lim = _chunked_limit(whole)
    st = GradRun(w, ws_limit=lim, problem=(whole.lays, whole.bufs), plan=whole.plan)
    n = heff.heff_grad_chunks(st.g)
    assert n >= 2 and heff.heff_grad_workspace_size(st.g) <= lim
    print(name, "chunks", n, "workspace", heff.heff_grad_workspace_size(st.g), "of", heff.heff_grad_workspace_size(whole.g))
    _compare_streamed(whole.run(), st.run())


def test_backward_streamed_at_m4096():
    w = wl.workload_by_name("spin_m4096")
    whole = GradRun(w)
    st = GradRun(w, ws_limit=256 << 20, problem=(whole.lays, whole.bufs), plan=whole.plan)
    n = heff.heff_grad_chunks(st.g)
    ws0, ws1 = heff.heff_grad_workspace_size(whole.g), heff.heff_grad_workspace_size(st.g)
    print(f"m=4096 gradients: {n} chunks, workspace {ws1 / 1e6:.0f} MB instead of {ws0 / 1e6:.0f} MB")
    assert n >= 2 and ws1 <= 256 << 20
    r0, r1 = whole.run(), st.run()
    _compare_streamed(r0, r1)
    rho, (dx, dL, dR, dW1, dW2) = r1
    b = whole.bufs
    for g_, t_ in ((dL, b["L"]), (dR, b["R"]), (dW1, b["W1"]), (dW2, b["W2"])):
        assert abs(float(np.dot(g_, t_)) - rho) < 1e-11 * abs(rho)
    x0 = b["x"][0]
    assert abs(float(np.dot(dx, x0))) < 1e-11 * abs(rho) * np.linalg.norm(x0)
    L, W1, W2, R, x = oh.problem_from_workload(w)
    y = oh.heff_apply(L, W1, W2, R, x)
    rho_o = sum(float(np.vdot(x.blocks[k], y.blocks[k])) for k in x.blocks) / \
        sum(float(np.vdot(v, v)) for v in x.blocks.values())
    print(f"m=4096 rho {rho:.15f} oracle {rho_o:.15f}")
    assert abs(rho - rho_o) < 1e-11 * abs(rho_o)


# ---------------------------------------------------------------- tensor-core block products
@pytest.mark.parametrize("name", ["spin_m200", "electron_m256"])
def test_backward_bf16x3_matches_oracle(name):
    """BF16x3 apply and BF16x3 block products (FP32-accumulated): every gradient within the
    BF16 path's 1e-3 of the oracle (norm-wise), Euler homogeneity to the same accuracy, and
    the error flag clear."""
    w = wl.workload_by_name(name)
    r = GradRun(w, "bf16x3", gprec="bf16x3")
    rho, (dx, dL, dR, dW1, dW2) = r.run()
    assert heff.heff_grad_status(r.g, r.gws) == 0
    L, W1, W2, R, x = oh.problem_from_workload(w)
    ref = ograd.grad_all(L, W1, W2, R, x)
    Ll, W1l, W2l, Rl, xl = r.lays
    errs = {
        "dx": _rel(dx, xl.assemble(lambda k: ref["dx"].blocks[k])),
        "dL": _rel(dL, Ll.assemble(lambda k: ref["dL"].blocks[k])),
        "dR": _rel(dR, Rl.assemble(lambda k: ref["dR"].blocks[k])),
        "dW1": _rel(dW1, W1l.assemble(lambda k: ref["dW1"][k])),
        "dW2": _rel(dW2, W2l.assemble(lambda k: ref["dW2"][k])),
    }
    print(name, "bf16x3", {k: f"{v:.1e}" for k, v in errs.items()}, f"rho err {abs(rho - ref['rho']):.1e}")
    assert abs(rho - ref["rho"]) < 1e-3 * abs(ref["rho"])
    for k, v in errs.items():
        assert v < 1e-3, (k, v)
    b = r.bufs
    for g_, t_ in ((dL, b["L"]), (dR, b["R"]), (dW1, b["W1"]), (dW2, b["W2"])):
        assert abs(float(np.dot(g_, t_)) - rho) < 1e-3 * abs(rho)


def test_backward_bf16x3_streamed_at_m4096_close_to_fp64():
    w = wl.workload_by_name("spin_m4096")
    f64 = GradRun(w, ws_limit=256 << 20)
    tc = GradRun(w, "bf16x3", ws_limit=256 << 20, problem=(f64.lays, f64.bufs), gprec="bf16x3")
    r0, r1 = f64.run(), tc.run()
    assert heff.heff_grad_status(tc.g, tc.gws) == 0
    errs = [_rel(a, b) for a, b in zip(r1[1], r0[1])]
    print("m=4096 bf16x3 vs fp64 gradients:", [f"{e:.1e}" for e in errs], f"rho {abs(r1[0] - r0[0]) / abs(r0[0]):.1e}")
    assert abs(r1[0] - r0[0]) < 1e-3 * abs(r0[0])
    assert max(errs) < 1e-3
