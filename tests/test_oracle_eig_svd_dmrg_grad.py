"""Pins of the oracle's eigensolvers, SVD truncation, DMRG and gradients.

* Lanczos and Algorithm 1 (Davidson) against numpy.linalg.eigh of dense
  matrices (including the dense K of a small H_eff);
* truncated block SVD: squared reconstruction error = discarded weight;
  isometric left factor;
* two-site DMRG against exact diagonalisation (16-site Heisenberg chain, a
  J1-J2 cylinder, a Hubbard chain) and the variational bound;
* Rayleigh-quotient gradients against central finite differences (h = 1e-6),
  Euler homogeneity (rho is linear in L, R, W1, W2 and of degree 0 in x)
  and the closed form d rho/dx = 2 (Kx - rho x)/<x|x>.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import kron, heff, eig, svd, dmrg, grad, mps
from oracle.blocks import BlockTensor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_sym(n, seed):
    A = np.random.default_rng(seed).standard_normal((n, n))
    return (A + A.T) / 2


def test_lanczos_full_krylov_equals_eigh():
    A = _rand_sym(40, 0)
    v0 = np.random.default_rng(1).standard_normal(40)
    th, x, info = eig.lanczos(lambda v: A @ v, v0, 40)
    w = np.linalg.eigvalsh(A)
    assert abs(th - w[0]) < 1e-10
    assert np.linalg.norm(A @ x - th * x) < 1e-7


def test_davidson_equals_eigh():
    A = _rand_sym(30, 2)
    v0 = np.random.default_rng(3).standard_normal(30)
    lam, x = eig.davidson(lambda v: A @ v, v0, 30, tol=1e-12)
    assert abs(lam - np.linalg.eigvalsh(A)[0]) < 1e-10
    assert np.linalg.norm(A @ x - lam * x) < 1e-8


def test_davidson_subspace_two_restarts_decrease():
    # Algorithm 1 with 2 vectors per call, restarted from its own output:
    # the Ritz value decreases monotonically toward the lowest eigenvalue.
    A = _rand_sym(25, 4)
    x = np.random.default_rng(5).standard_normal(25)
    prev = np.inf
    for it in range(300):
        lam, x = eig.davidson(lambda v: A @ v, x, 2, seed=it)
        assert lam <= prev + 1e-12
        prev = lam
    assert abs(lam - np.linalg.eigvalsh(A)[0]) < 1e-6


@pytest.mark.parametrize("name", ["spin_m24", "electron_m40"])
def test_lanczos_on_heff_matches_dense_K(name):
    w = wl.workload_by_name(name)
    L, W1, W2, R, x = heff.problem_from_workload(w)
    K = heff.heff_matrix_dense(L.to_dense(), W1, W2, R.to_dense())
    mask = x.to_dense().reshape(-1) != 0   # the allowed-block subspace
    Kb = K[mask][:, mask]
    assert np.abs(Kb - Kb.T).max() < 1e-12
    keys = sorted(x.blocks)
    flat = lambda t: np.concatenate([t.blocks[k].reshape(-1) for k in keys])

    def mv(v):
        t = x.copy().set_flat(v)
        return heff.heff_apply(L, W1, W2, R, t).flat()
    th, _, _ = eig.lanczos(mv, flat(x), 200)
    assert abs(th - np.linalg.eigvalsh(Kb)[0]) < 1e-9 * abs(th)


def _rand_two_site(seed, m=6):
    n = 6
    sites = mps.random_mps(wl.spin_phys(), n, (0,), m, seed)
    return mps.two_site(sites[2], sites[3])


def test_svd_truncation_error_equals_discarded_weight():
    x = _rand_two_site(0, 8)
    x.scale(1.0 / x.norm())
    A, B, s, disc = svd.svd_split(x, 5, cutoff=0.0, absorb="right")
    y = mps.two_site(A, B)
    err2 = x.copy().axpy(-1.0, y).norm() ** 2
    assert disc > 1e-6
    assert abs(err2 - disc) < 1e-12
    # the left factor is an isometry per sector
    for c in range(A.indices[2].nsec):
        M = np.vstack([blk[:, 0, :] for (i, s1, cc), blk in sorted(A.blocks.items()) if cc == c])
        assert np.abs(M.T @ M - np.eye(M.shape[1])).max() < 1e-12


def test_svd_without_truncation_is_exact():
    x = _rand_two_site(1, 6)
    A, B, s, disc = svd.svd_split(x, 10 ** 6, cutoff=0.0, absorb="left")
    y = mps.two_site(A, B)
    assert x.copy().axpy(-1.0, y).norm() < 1e-12 * x.norm()
    assert abs(disc) < 1e-14


def test_svd_cutoff_drops_small_values():
    x = _rand_two_site(2, 6)
    x.scale(1.0 / x.norm())
    A, B, s, disc = svd.svd_split(x, 10 ** 6, cutoff=0.05, absorb="right")
    assert (s >= 0.05).all()


def _ed_golden():
    with open(os.path.join(GOLDEN, "ed_energies.json")) as f:
        return json.load(f)


def test_dmrg_heisenberg_16_equals_ed():
    # 1D spin-1/2 Heisenberg chain, L = 16, OBC, MPO bond dim 5, m = 64
    n = 16
    mpo = wl.heisenberg_mpo(n, wl.chain_pairs(n, [1.0]))
    assert max(mpo.bond_dim(b) for b in range(n + 1)) == 5
    E_ed = _ed_golden()["heisenberg_chain_L16_obc_Sz0"]["E0"]
    r = dmrg.dmrg(mpo, (0,), [16, 64, 64], n_iter=20)
    E = r["sweep_energies"][-1]
    assert E >= E_ed - 1e-12 * abs(E_ed)          # variational bound
    assert abs(E - E_ed) < 1e-10 * abs(E_ed)


def test_dmrg_davidson_heisenberg_equals_ed():
    n = 10
    mpo = wl.heisenberg_mpo(n, wl.chain_pairs(n, [1.0]))
    E_ed = kron.ground_energy(kron.heisenberg_hamiltonian(n, wl.chain_pairs(n, [1.0])),
                              kron.basis_charges(n, wl.spin_phys()), (0,))
    r = dmrg.dmrg(mpo, (0,), [32] * 8, solver="davidson", davidson_vecs=2)
    assert abs(r["sweep_energies"][-1] - E_ed) < 1e-8 * abs(E_ed)


def test_dmrg_j1j2_cylinder_equals_ed():
    Lx, Ly = 3, 4
    pairs = wl.cylinder_pairs(Lx, Ly, 1.0, 0.5)
    n = Lx * Ly
    mpo = wl.heisenberg_mpo(n, pairs)
    E_ed = _ed_golden()["j1j2_cylinder_3x4_J2_0.5_Sz0"]["E0"]
    r = dmrg.dmrg(mpo, (0,), [16, 64, 64], n_iter=25)
    assert abs(r["sweep_energies"][-1] - E_ed) < 1e-9 * abs(E_ed)


def test_dmrg_hubbard_equals_ed():
    n = 6
    hops = [(i, i + 1, 1.0) for i in range(n - 1)]
    mpo = wl.hubbard_mpo(n, hops, 8.0)
    E_ed = _ed_golden()["hubbard_chain_L6_U8_half_filling"]["E0"]
    r = dmrg.dmrg(mpo, (6, 0), [16, 64, 64], n_iter=25)
    assert abs(r["sweep_energies"][-1] - E_ed) < 1e-9 * abs(E_ed)


def test_product_state_mps_is_the_basis_state_and_dmrg_from_it_reaches_ed():
    # the Neel product state as an MPS contracts to one basis vector of the Kronecker basis,
    # and two-site DMRG started from it reaches the exact ground energy (3 x 4 J1-J2)
    Lx, Ly = 3, 4
    n = Lx * Ly
    states = [i % 2 for i in range(n)]
    sites = mps.product_mps(wl.spin_phys(), states)
    psi = mps.to_dense_state(sites)
    idx = 0
    for s in states:
        idx = idx * 2 + s
    assert np.array_equal(np.flatnonzero(psi), [idx]) and psi[idx] == 1.0
    mpo = wl.heisenberg_mpo(n, wl.cylinder_pairs(Lx, Ly, 1.0, 0.5))
    E_ed = _ed_golden()["j1j2_cylinder_3x4_J2_0.5_Sz0"]["E0"]
    r = dmrg.dmrg(mpo, (0,), [16, 64, 64, 64], n_iter=25, states=states)
    assert r["sweep_energies"][-1] >= E_ed - 1e-12 * abs(E_ed)
    assert abs(r["sweep_energies"][-1] - E_ed) < 1e-9 * abs(E_ed)
    with pytest.raises(ValueError):
        dmrg.dmrg(mpo, (2,), [4], states=states)      # the product state has 2Sz = 0


def test_golden_dmrg_sweeps_variational_and_decreasing():
    # the stored 6 x 6 sweep energies do not increase from sweep to sweep, and the last lies
    # below the energy of the Neel start state (DMRG improves on its start variationally)
    with open(os.path.join(GOLDEN, "dmrg_sweeps.json")) as f:
        g = json.load(f)["j1j2_cylinder_6x6_J2_0.5_neel_start"]
    e = g["sweep_energies"]
    assert all(b <= a + 1e-12 for a, b in zip(e, e[1:]))
    pairs = wl.cylinder_pairs(6, 6, 1.0, 0.5)
    # Neel energy along the snake: sum over bonds of J <Sz_i Sz_j> = +-J/4
    neel = sum(J * (0.25 if (i % 2) == (j % 2) else -0.25) for i, j, J in pairs)
    assert e[-1] < neel


def test_golden_ed_values_reproduce():
    g = _ed_golden()
    n = 12
    pairs = wl.cylinder_pairs(3, 4, 1.0, 0.5)
    E = kron.ground_energy(kron.heisenberg_hamiltonian(n, pairs),
                           kron.basis_charges(n, wl.spin_phys()), (0,))
    assert abs(E - g["j1j2_cylinder_3x4_J2_0.5_Sz0"]["E0"]) < 1e-10


# ---------------------------------------------------------------- gradients

def _grad_problem(name="spin_m64"):
    w = wl.workload_by_name(name)
    return w, heff.problem_from_workload(w)


def _rho(L, W1, W2, R, x):
    return grad.rayleigh(L, W1, W2, R, x)[0]


def test_grad_homogeneity_and_closed_form():
    w, (L, W1, W2, R, x) = _grad_problem()
    g = grad.grad_all(L, W1, W2, R, x)
    rho = g["rho"]
    assert abs(L.vdot(g["dL"]) - rho) < 1e-11 * abs(rho)
    assert abs(R.vdot(g["dR"]) - rho) < 1e-11 * abs(rho)
    assert abs(np.sum(W1 * g["dW1"]) - rho) < 1e-11 * abs(rho)
    assert abs(np.sum(W2 * g["dW2"]) - rho) < 1e-11 * abs(rho)
    assert abs(x.vdot(g["dx"])) < 1e-11 * abs(rho) * x.norm()


def test_grad_central_differences():
    w, (L, W1, W2, R, x) = _grad_problem()
    g = grad.grad_all(L, W1, W2, R, x)
    h = 1e-6
    rng = np.random.default_rng(0)
    # x
    for _ in range(4):
        k = sorted(x.blocks)[rng.integers(len(x.blocks))]
        idx = tuple(rng.integers(s) for s in x.blocks[k].shape)
        xp, xm = x.copy(), x.copy()
        xp.blocks[k][idx] += h
        xm.blocks[k][idx] -= h
        fd = (_rho(L, W1, W2, R, xp) - _rho(L, W1, W2, R, xm)) / (2 * h)
        assert abs(fd - g["dx"].blocks[k][idx]) < 1e-6 * max(1.0, abs(fd))
    # L, R
    for T, dT, pos in [(L, g["dL"], 0), (R, g["dR"], 3)]:
        for _ in range(4):
            k = sorted(T.blocks)[rng.integers(len(T.blocks))]
            idx = tuple(rng.integers(s) for s in T.blocks[k].shape)
            Tp, Tm = T.copy(), T.copy()
            Tp.blocks[k][idx] += h
            Tm.blocks[k][idx] -= h
            args_p = [L, W1, W2, R, x]
            args_m = [L, W1, W2, R, x]
            args_p[pos], args_m[pos] = Tp, Tm
            fd = (_rho(*args_p) - _rho(*args_m)) / (2 * h)
            assert abs(fd - dT.blocks[k][idx]) < 1e-6 * max(1.0, abs(fd))
    # W1, W2 on their nonzero entries
    for Wi, dW, pos in [(W1, g["dW1"], 1), (W2, g["dW2"], 2)]:
        nz = np.argwhere(Wi != 0)
        for t in nz[rng.choice(len(nz), 5, replace=False)]:
            t = tuple(t)
            Wp, Wm = Wi.copy(), Wi.copy()
            Wp[t] += h
            Wm[t] -= h
            args_p = [L, W1, W2, R, x]
            args_m = [L, W1, W2, R, x]
            args_p[pos], args_m[pos] = Wp, Wm
            fd = (_rho(*args_p) - _rho(*args_m)) / (2 * h)
            assert abs(fd - dW[t]) < 1e-6 * max(1.0, abs(fd))


def test_grad_coupling_j2_central_difference():
    # rho is quadratic in J2 (W1, W2 affine in J2): central FD is exact up to rounding
    from workloads.fill import spin_window, SPIN_COUPLINGS
    w = wl.workload_by_name("spin_m64")
    L, _, _, R, x = heff.problem_from_workload(w)

    def Ws(J2):
        c = list(SPIN_COUPLINGS)
        c[1] = J2
        win = spin_window(tuple(c))
        return win["W1"], win["W2"]
    J2, h = SPIN_COUPLINGS[1], 1e-6
    W1, W2 = Ws(J2)
    W1p, W2p = Ws(J2 + h)
    W1m, W2m = Ws(J2 - h)
    g = grad.grad_all(L, W1, W2, R, x)
    dW1dJ = (W1p - W1m) / (2 * h)
    dW2dJ = (W2p - W2m) / (2 * h)
    an = float(np.sum(g["dW1"] * dW1dJ) + np.sum(g["dW2"] * dW2dJ))
    fd = (_rho(L, W1p, W2p, R, x) - _rho(L, W1m, W2m, R, x)) / (2 * h)
    assert abs(an - fd) < 1e-7 * max(1.0, abs(fd))
