"""GPU FP64 Lanczos (heff_lanczos) against the oracle's Lanczos and exact eigenpairs.

* FP64 path: the lowest Ritz value after n steps from the same start vector equals the
  oracle's (Section II-C eigensolver; Lanczos with full reorthogonalisation) to 1e-10
  relative, and the Ritz vectors agree;
* BF16x3 / TF32x3 matvecs inside the FP64 Lanczos: the Ritz value is within the split
  precision of the exact lowest eigenvalue; one FP64 Rayleigh quotient of the returned
  vector (a single FP64 apply) brings the energy within 1e-8 relative of it (the
  second-order accuracy of the Rayleigh quotient in the eigenvector error).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import heff as oh, eig

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import heff               # noqa: E402
from tests.helpers import library_problem              # noqa: E402


class LzProblem:
    def __init__(self, name):
        self.w = wl.workload_by_name(name)
        self.lays, self.bufs = library_problem(self.w)
        self.d = {k: torch.from_numpy(np.asarray(self.bufs[k])).to("cuda", torch.float64)
                  for k in ("L", "W1", "W2", "R")}
        self.x0 = torch.from_numpy(self.bufs["x"][0]).to("cuda", torch.float64)
        self.plans = {}

    def plan(self, prec):
        if prec not in self.plans:
            Ll, W1l, W2l, Rl, xl = self.lays
            self.plans[prec] = heff.Plan(Ll, W1l, W2l, Rl, xl, self.bufs["W1"], self.bufs["W2"], prec, "f64")
        return self.plans[prec]

    def lanczos(self, prec, n_iter):
        P = self.plan(prec)
        ws = P.workspace()
        lz = torch.empty(heff.heff_lanczos_workspace_size(P.handle, n_iter), dtype=torch.uint8, device="cuda")
        x = torch.empty_like(self.x0)
        res = torch.zeros(3 + 2 * (n_iter + 1), dtype=torch.float64, device="cuda")
        d = self.d
        heff.heff_lanczos(P.handle, d["L"], d["W1"], d["W2"], d["R"], self.x0, n_iter, x, res, ws, lz)
        torch.cuda.synchronize()
        return res.cpu().numpy(), x

    def rayleigh_fp64(self, x):
        P = self.plan("fp64")
        ws = P.workspace()
        y = torch.empty_like(x)
        d = self.d
        heff.heff_apply(P.handle, d["L"], d["W1"], d["W2"], d["R"], x, y, ws)
        torch.cuda.synchronize()
        return float(torch.dot(x, y) / torch.dot(x, x))

    def oracle(self, n_iter):
        L, W1, W2, R, x = oh.problem_from_workload(self.w)

        def mv(v):
            return oh.heff_apply(L, W1, W2, R, x.copy().set_flat(v)).flat()
        return eig.lanczos(mv, x.flat(), n_iter)

    def exact_lowest(self):
        L, W1, W2, R, x = oh.problem_from_workload(self.w)
        K = oh.heff_matrix_dense(L.to_dense(), W1, W2, R.to_dense())
        mask = x.to_dense().reshape(-1) != 0
        return float(np.linalg.eigvalsh(K[mask][:, mask])[0])


@pytest.mark.parametrize("name,n_iter", [("spin_m64", 20), ("electron_m96", 25), ("spin_m1024", 30)])
def test_fp64_lanczos_matches_oracle(name, n_iter):
    p = LzProblem(name)
    res, x = p.lanczos("fp64", n_iter)
    th_o, x_o, info = p.oracle(n_iter)
    th = res[0]
    assert int(res[2]) == info["n"]
    assert abs(th - th_o) < 1e-10 * abs(th_o), (th, th_o)
    np.testing.assert_allclose(res[3:3 + info["n"]], info["alpha"], rtol=0, atol=1e-9 * abs(th_o))
    ov = abs(float(np.dot(x.cpu().numpy(), x_o)))
    assert ov > 1 - 1e-8, ov
    print(f"{name}: theta {th:.15f} oracle {th_o:.15f} rel {abs(th - th_o) / abs(th_o):.2e}")


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-3), ("tf32x3", 1e-4)])
@pytest.mark.parametrize("name", ["spin_m24", "electron_m40"])
def test_mixed_lanczos_with_fp64_refinement(name, prec, tol):
    p = LzProblem(name)
    E0 = p.exact_lowest()
    n_iter = min(120, p.lays[4].nelem)
    res, x = p.lanczos(prec, n_iter)
    th = res[0]
    err_mixed = abs(th - E0) / abs(E0)
    assert err_mixed < tol, err_mixed
    th_rq = p.rayleigh_fp64(x)
    err_rq = abs(th_rq - E0) / abs(E0)
    print(f"{name} {prec}: E0 {E0:.12f} mixed Ritz err {err_mixed:.2e} refined err {err_rq:.2e}")
    assert err_rq < 1e-8, err_rq


def test_fp64_lanczos_converges_to_exact_lowest_eigenvalue():
    p = LzProblem("spin_m24")
    E0 = p.exact_lowest()
    res, x = p.lanczos("fp64", min(120, p.lays[4].nelem))
    assert abs(res[0] - E0) < 1e-11 * abs(E0)
    assert res[1] < 1e-6 * abs(E0)          # Lanczos residual estimate of a converged pair


def test_lanczos_rejects_f32_plans():
    w = wl.workload_by_name("spin_m64")
    lays, bufs = library_problem(w)
    P = heff.Plan(*lays, bufs["W1"], bufs["W2"], "bf16x3", "f32")
    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(heff.HeffError) as e:
        heff.heff_lanczos(P.handle, t, t, t, t, t, 5, t, t, ws, ws)
    assert e.value.code == -3


def test_restart_from_converged_vector_breaks_down_cleanly():
    """Started from a converged Ritz vector the Krylov space is invariant after one step
    (the situation at the turn of a DMRG sweep): the result must be that vector and its
    Rayleigh quotient, finite, with a Krylov dimension of 1."""
    p = LzProblem("spin_m24")
    res, x = p.lanczos("fp64", min(120, p.lays[4].nelem))
    p.x0 = x.clone()
    res2, x2 = p.lanczos("fp64", 10)
    assert np.isfinite(res2[:3]).all() and torch.isfinite(x2).all()
    assert res2[2] <= 2
    assert abs(res2[0] - res[0]) < 1e-10 * abs(res[0])
    ov = abs(float(torch.dot(x2, x)))
    assert ov > 1 - 1e-10, ov


def test_zero_start_vector_gives_empty_krylov_space():
    """A zero start vector spans nothing: Krylov dimension 0, theta and the residual
    estimate 0, a zero output vector, all finite (nothing reads past the empty basis)."""
    p = LzProblem("spin_m24")
    p.x0 = torch.zeros_like(p.x0)
    res, x = p.lanczos("fp64", 10)
    assert res[2] == 0 and res[0] == 0.0 and res[1] == 0.0
    assert torch.count_nonzero(x) == 0


# ---------------------------------------------------------------- Davidson (Algorithm 1)
def _davidson(p, prec, max_vecs, tol, x0=None, seed=7):
    P = p.plan(prec)
    ws = P.workspace()
    dw = torch.empty(heff.heff_davidson_workspace_size(P.handle, max_vecs), dtype=torch.uint8, device="cuda")
    x0 = p.x0 if x0 is None else x0
    rnd = torch.from_numpy(np.random.default_rng(seed).standard_normal(x0.numel())).cuda()
    x = torch.empty_like(x0)
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    d = p.d
    heff.heff_davidson(P.handle, d["L"], d["W1"], d["W2"], d["R"], x0, rnd, max_vecs, tol, x, res, ws, dw)
    torch.cuda.synchronize()
    return res.cpu().numpy(), x


@pytest.mark.parametrize("name,max_vecs", [("spin_m24", 12), ("electron_m40", 16), ("spin_m64", 2),
                                           ("spin_m1024", 2), ("spin_m200", 6)])
def test_fp64_davidson_matches_oracle_algorithm_1(name, max_vecs):
    """Same start vector, same stopping rule: the GPU Davidson (two classical Gram-Schmidt
    passes) and the oracle's (modified Gram-Schmidt) agree to rounding."""
    p = LzProblem(name)
    res, x = _davidson(p, "fp64", max_vecs, 1e-10)
    L, W1, W2, R, xo = oh.problem_from_workload(p.w)

    def mv(v):
        return oh.heff_apply(L, W1, W2, R, xo.copy().set_flat(v)).flat()
    lam_o, x_o = eig.davidson(mv, xo.flat(), max_vecs, tol=1e-10)
    assert abs(res[0] - lam_o) < 1e-10 * abs(lam_o), (res[0], lam_o)
    ov = abs(float(np.dot(x.cpu().numpy(), x_o)))
    assert ov > 1 - 1e-8, ov
    assert 1 <= res[2] <= max_vecs
    print(f"{name} davidson({max_vecs}): lambda {res[0]:.15f} oracle {lam_o:.15f} |q| {res[1]:.2e} vecs {int(res[2])}")


def test_davidson_converges_to_exact_lowest_eigenvalue():
    p = LzProblem("spin_m24")
    E0 = p.exact_lowest()
    res, x = _davidson(p, "fp64", 60, 1e-10)
    assert abs(res[0] - E0) < 1e-10 * abs(E0)
    assert res[1] < 1e-9 * abs(E0)


def test_davidson_from_an_eigenvector_stays_finite():
    """Started from a converged eigenvector with tol = 0 the correction q is rounding noise
    (the case Algorithm 1's randomisation guards); the result must stay that eigenpair."""
    p = LzProblem("spin_m24")
    res, x = p.lanczos("fp64", min(120, p.lays[4].nelem))
    r2, x2 = _davidson(p, "fp64", 4, 0.0, x0=x.clone())
    assert np.isfinite(r2).all() and torch.isfinite(x2).all()
    assert abs(r2[0] - res[0]) < 1e-10 * abs(res[0])
    assert abs(float(torch.dot(x2, x))) > 1 - 1e-10


def test_davidson_with_bf16x3_matvecs():
    """BF16x3 matvecs inside the FP64 Davidson (the subspace that converges in FP64 above):
    the Ritz value carries the split precision, the FP64 Rayleigh quotient of the vector
    does not."""
    p = LzProblem("spin_m24")
    E0 = p.exact_lowest()
    res, x = _davidson(p, "bf16x3", 60, 1e-7)
    assert abs(res[0] - E0) < 1e-3 * abs(E0)
    assert abs(p.rayleigh_fp64(x) - E0) < 1e-8 * abs(E0)


# ---------------------------------------------------------------- ground state to a tolerance
def _ground_state(p, prec, refine, n_iter=120, cycles=8, tol=1e-9):
    P = p.plan(prec)
    P64 = p.plan("fp64") if refine else None
    ws = P.workspace()
    ws64 = P64.workspace() if refine else None
    gs = torch.empty(heff.heff_ground_state_workspace_size(P.handle, n_iter), dtype=torch.uint8, device="cuda")
    x = torch.empty_like(p.x0)
    d = p.d
    r = heff.heff_ground_state(P.handle, P64.handle if refine else None, d["L"], d["W1"], d["W2"], d["R"], p.x0,
                               n_iter, cycles, tol, x, ws, ws64, gs)
    return r, x


@pytest.mark.parametrize("name", ["spin_m24", "electron_m40"])
def test_ground_state_equals_lowest_eigenvalue_of_dense_K(name):
    """Converged to the tolerance, the FP64 path's energy equals the lowest eigenvalue of the
    oracle's dense K (Section II-C) to 1e-10, and the split-precision path with its FP64
    Rayleigh quotient equals it to 1e-8."""
    p = LzProblem(name)
    L, W1, W2, R, x = oh.problem_from_workload(p.w)
    K = oh.heff_matrix_dense(L.to_dense(), W1, W2, R.to_dense())
    # the lowest eigenvalue restricted to the allowed blocks (K maps them into themselves)
    mask = x.to_dense().reshape(-1) != 0
    E_ex = np.linalg.eigvalsh(K[np.ix_(mask, mask)])[0]
    r64, _ = _ground_state(p, "fp64", False, n_iter=60, cycles=10, tol=1e-11)
    rb, _ = _ground_state(p, "bf16x3", True, n_iter=60, cycles=10, tol=1e-10)
    print(f"{name}: exact {E_ex:.14f} fp64 {r64['energy']:.14f} ({r64['cycles']} cycles) bf16x3+fp64 RQ "
          f"{rb['energy']:.14f} (Ritz {rb['ritz']:.14f}, FP64 residual {rb['residual_fp64']:.2e})")
    assert abs(r64["energy"] - E_ex) < 1e-10 * abs(E_ex)
    assert r64["residual_fp64"] < 1e-8
    assert abs(rb["energy"] - E_ex) < 1e-8 * abs(E_ex)


def test_ground_state_mixed_energy_within_1e8_of_fp64_path_m1024():
    """The full m = 1024 spin workload (30 sectors, k = 14): both paths converged to a
    residual estimate of 1e-9 |E| by restarted Lanczos from the same start vector; the
    BF16x3 path's energy (its Ritz vector's FP64 Rayleigh quotient, one FP64 apply) is within
    1e-8 relative of the FP64 path's, while its own Ritz value carries the split's bias."""
    p = LzProblem("spin_m1024")
    r64, x64 = _ground_state(p, "fp64", False)
    rb, xb = _ground_state(p, "bf16x3", True)
    rel = abs(rb["energy"] - r64["energy"]) / abs(r64["energy"])
    print(f"m=1024: fp64 {r64['energy']:.14f} ({r64['matvecs']} matvecs, FP64 residual {r64['residual_fp64']:.2e}); "
          f"bf16x3 {rb['energy']:.14f} ({rb['matvecs']} matvecs, Ritz {rb['ritz']:.14f}, FP64 residual "
          f"{rb['residual_fp64']:.2e}); rel diff {rel:.2e}")
    assert r64["residual_estimate"] <= 1e-9 and rb["residual_estimate"] <= 1e-9
    assert r64["residual_fp64"] < 1e-7
    assert rel <= 1e-8
    # the same eigenvector: |<x_fp64|x_mixed>| = 1 to the split's accuracy
    assert abs(abs(float(torch.dot(x64, xb))) - 1.0) < 1e-6
