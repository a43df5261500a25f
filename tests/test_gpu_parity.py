"""GPU parity of the CUDA H_eff path against the FP64 oracle (through the C ABI).

Tolerances: FP64 path 1e-10; TF32 split (3xTF32) 1e-5; BF16 with
compensation (BF16x3) 1e-3, as norm-wise relative errors ||y - y_oracle|| / ||y_oracle||,
with every element also within 20x the tolerance of max|y_oracle|; all output elements
at small sizes, every element of sampled output sectors at the benchmark's full sizes.
y is pre-filled with NaN so an output block the kernels fail to write is caught.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import heff as oh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected only with -m gpu on CPU
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff                       # noqa: E402
from tests.helpers import library_problem, oracle_flat         # noqa: E402

TOL = {"fp64": 1e-10, "tf32x3": 1e-5, "bf16x3": 1e-3}
IO = {"fp64": "f64", "tf32x3": "f32", "bf16x3": "f32"}


def _dev(a, io):
    return torch.from_numpy(np.asarray(a)).to("cuda", torch.float64 if io == "f64" else torch.float32)


class Lib:
    """The library problem for one workload and precision, resident on the GPU."""

    def __init__(self, w, prec, batches=(0,), max_batch=1):
        self.w, self.prec, self.io = w, prec, IO[prec]
        self.lays, self.bufs = library_problem(w, batches)
        Ll, W1l, W2l, Rl, xl = self.lays
        self.plan = heff.Plan(Ll, W1l, W2l, Rl, xl, self.bufs["W1"], self.bufs["W2"], prec, self.io,
                              max_batch)
        self.L, self.W1, self.W2, self.R = (_dev(self.bufs[k], self.io) for k in ("L", "W1", "W2", "R"))
        self.xs = [_dev(x, self.io) for x in self.bufs["x"]]
        self.ws = self.plan.workspace()

    def apply(self, b=0):
        y = torch.full_like(self.xs[b], float("nan"))
        heff.heff_apply(self.plan.handle, self.L, self.W1, self.W2, self.R, self.xs[b], y, self.ws)
        torch.cuda.synchronize()
        return y.double().cpu().numpy()


def _oracle(w, batch=0, left_sectors=None):
    L, W1, W2, R, x = oh.problem_from_workload(w, batch)
    return oh.heff_apply(L, W1, W2, R, x, left_sectors=left_sectors)


def _compare(y, y_ref, tol, mask=None):
    """Relative error of y against the oracle: ||y - y_ref||_2 / ||y_ref||_2 < tol, and every
    element within ELEM * tol of max|y_ref| (FP32 accumulation over K ~ 1e4 terms puts single
    elements a few times above the norm-wise error; a wrong block would be O(1) off)."""
    ELEM = 20.0
    if mask is not None:
        y, y_ref = y[mask], y_ref[mask]
    assert not np.isnan(y).any(), "unwritten output elements"
    nerr = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    merr = np.abs(y - y_ref).max() / np.abs(y_ref).max()
    assert nerr < tol, f"norm-wise rel err {nerr:.3e} >= {tol:.0e}"
    assert merr < ELEM * tol, f"element-wise err {merr:.3e} >= {ELEM * tol:.0e} of max|y|"
    print(f"rel err: norm {nerr:.3e}  max-element {merr:.3e}")
    return nerr


SMALL = ["spin_m64", "spin_m200", "electron_m96", "electron_m256", "spin_m1024_s8", "spin_j1j2_6x6_m200",
         "electron_hubbard_4x8_m96", "spin_j1j2_20x10_m200", "electron_tri_xc6_m96", "spin_j1j2_20x10c_m200",
         "electron_tri_xc6c_m96", "spin_j1j2_20x10ci_m200", "electron_tri_xc6ci_m96"]


def _workload(name):
    if name == "spin_m1024_s8":   # few, large sectors: several M and N tiles with ragged tails
        return wl.spin_heff_workload(1024, 8, 21, name=name)
    return wl.workload_by_name(name)


# The tensor cores' FP32 accumulation is biased toward zero over long contractions; GEMM 2
# therefore accumulates in chunks and adds them with round-to-nearest (tc_gemm.cu).  Before
# that change the TF32 split missed its 1e-5 bound (0.9e-5 - 3e-5) at contraction lengths
# above ~5000; every case below must now meet the stated bounds.
def _check(y, y_ref, tol, mask=None):
    return _compare(y, y_ref, tol, mask)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("name", SMALL)
def test_apply_matches_oracle(name, prec):
    w = _workload(name)
    lib = Lib(w, prec)
    y_ref = oracle_flat(lib.lays[4], _oracle(w))
    _check(lib.apply(), y_ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_batched_matches_oracle_and_single(prec):
    w = wl.workload_by_name("electron_m96")
    lib = Lib(w, prec, batches=(0, 1, 2), max_batch=3)
    ys = [torch.full_like(x, float("nan")) for x in lib.xs]
    heff.heff_apply_batched(lib.plan.handle, lib.L, lib.W1, lib.W2, lib.R, lib.xs, ys, lib.ws)
    torch.cuda.synchronize()
    for b in range(3):
        y_ref = oracle_flat(lib.lays[4], _oracle(w, b))
        yb = ys[b].double().cpu().numpy()
        _compare(yb, y_ref, TOL[prec])
        assert np.array_equal(yb, lib.apply(b))        # batched = single apply, bitwise


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_prepared_apply_repeatable(prec):
    w = wl.workload_by_name("spin_m200")
    lib = Lib(w, prec)
    heff.heff_prepare(lib.plan.handle, lib.L, lib.W1, lib.W2, lib.R, lib.ws)
    outs = []
    for _ in range(2):
        y = torch.full_like(lib.xs[0], float("nan"))
        heff.heff_apply_prepared(lib.plan.handle, lib.xs[0], y, lib.ws)
        torch.cuda.synchronize()
        outs.append(y.double().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])            # deterministic: no races in the epilogue
    assert np.array_equal(outs[0], lib.apply())


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_zero_input_and_linearity(prec):
    w = wl.workload_by_name("spin_m64")
    lib = Lib(w, prec)
    x0 = lib.xs[0]
    lib.xs[0] = torch.zeros_like(x0)
    assert np.array_equal(lib.apply(), np.zeros(x0.numel()))
    lib.xs[0] = 2.0 * x0
    y2 = lib.apply()
    lib.xs[0] = x0
    y1 = lib.apply()
    np.testing.assert_allclose(y2, 2.0 * y1, rtol=0, atol=TOL[prec] * np.abs(y1).max() * 4)


def test_single_sector_bonds():
    # degenerate: one sector per bond (the charge structure reduces to dense tensors)
    w = wl.spin_heff_workload(40, 1, 3, name="one_sector")
    for prec in ("fp64", "bf16x3"):
        lib = Lib(w, prec)
        _compare(lib.apply(), oracle_flat(lib.lays[4], _oracle(w)), TOL[prec])


def test_workspace_errors():
    w = wl.workload_by_name("spin_m64")
    lib = Lib(w, "fp64")
    y = torch.empty_like(lib.xs[0])
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(heff.HeffError) as e:
        heff.heff_apply(lib.plan.handle, lib.L, lib.W1, lib.W2, lib.R, lib.xs[0], y, small)
    assert e.value.code == -7
    with pytest.raises(heff.HeffError) as e:
        heff.heff_apply(lib.plan.handle, lib.L, lib.W1, lib.W2, lib.R, lib.xs[0], lib.xs[0], lib.ws)
    assert e.value.code == -1


# spin_paper_m4096: the Table II block-size model (27 sectors, centre block 1024 rows), the
# largest single-sector GEMMs of any workload; sector 13 is the centre, 0 and 26 the edges
FULL = [("spin_m4096", (0, 19, 20, 39)), ("spin_m1024", (0, 14, 15, 29)),
        ("electron_m2048", (0, 30, 31, 60)), ("spin_j1j2_6x6_m4096", (0, 19, 20, 39)),
        ("spin_paper_m4096", (0, 12, 13, 26)), ("spin_j1j2_20x10c_m4096", (0, 19, 20, 39))]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp64"])
@pytest.mark.parametrize("name,sectors", FULL)
def test_full_size_sampled_sectors(name, sectors, prec):
    # benchmark sizes and launch configuration; every element of the output blocks whose
    # left sector is in `sectors` is compared with the oracle restricted to those blocks
    w = wl.workload_by_name(name)
    lib = Lib(w, prec)
    y = lib.apply()
    keep = set(sectors)
    y_ref = oracle_flat(lib.lays[4], _oracle(w, left_sectors=keep))
    xl = lib.lays[4]
    mask = np.zeros(xl.nelem, dtype=bool)
    for key, off, size in xl.blocks():
        if key[0] in keep:
            mask[off:off + size] = True
    assert not np.isnan(y).any()
    _check(y, y_ref, TOL[prec], mask)


def test_empty_two_site_space():
    """A target charge no x block satisfies: the plan has no work, every apply entry is a
    no-op that returns success (also with NULL x and y), and the eigensolvers refuse it."""
    w = wl.workload_by_name("spin_m24")
    lays = heff.heff_layouts((w.alpha_q, w.alpha_d), (w.beta_q, w.beta_d), w.phys, w.ql, w.qm, w.qr,
                             target=np.array([1001], dtype=np.int32))
    assert lays[4].nelem == 0 and lays[0].nelem > 0
    W1 = lays[1].assemble(lambda k: w.W1[k])
    W2 = lays[2].assemble(lambda k: w.W2[k])
    L = torch.from_numpy(lays[0].assemble(lambda k: w.L_block((k[0], k[1], k[2])))).cuda()
    R = torch.from_numpy(lays[3].assemble(lambda k: w.R_block((k[0], k[1], k[2])))).cuda()
    d1, d2 = torch.from_numpy(W1).cuda(), torch.from_numpy(W2).cuda()
    x = torch.empty(0, dtype=torch.float64, device="cuda")
    y = torch.empty(0, dtype=torch.float64, device="cuda")
    for prec in ("fp64", "bf16x3"):
        io = torch.float64 if prec == "fp64" else torch.float32
        P = heff.Plan(*lays, W1, W2, prec, "f64" if prec == "fp64" else "f32")
        assert P.flops_canonical == 0.0
        ws = P.workspace()
        args = [t.to(io) for t in (L, d1, d2, R)]
        heff.heff_apply(P.handle, *args, x.to(io), y.to(io), ws)
        heff.heff_apply_batched(P.handle, *args, [x.to(io)], [y.to(io)], ws)
        torch.cuda.synchronize()
    P = heff.Plan(*lays, W1, W2, "fp64", "f64")
    lz = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    res = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(heff.HeffError) as e:
        heff.heff_lanczos(P.handle, L, d1, d2, R, x, 1, y, res, P.workspace(), lz)
    assert e.value.code == -1


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_check_mpo_counts_entries_the_plan_dropped(prec):
    """The device MPO tensors the plan was made from fit it (0); a value placed where the host
    copy was zero (an entry the schedule dropped, which the apply would ignore) is counted,
    in W1 and in W2."""
    w = wl.workload_by_name("spin_m64")
    lib = Lib(w, prec)
    assert heff.heff_plan_check_mpo(lib.plan.handle, lib.W1, lib.W2) == 0
    z1 = np.flatnonzero(np.asarray(lib.bufs["W1"]) == 0.0)
    z2 = np.flatnonzero(np.asarray(lib.bufs["W2"]) == 0.0)
    assert len(z1) > 0 and len(z2) > 0
    W1, W2 = lib.W1.clone(), lib.W2.clone()
    W1[int(z1[0])] = 0.5
    assert heff.heff_plan_check_mpo(lib.plan.handle, W1, W2) == 1
    W2[int(z2[-1])] = -2.0
    W2[int(z2[0])] = 1e-30
    assert heff.heff_plan_check_mpo(lib.plan.handle, W1, W2) == 3
