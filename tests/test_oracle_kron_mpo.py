"""Pins of the Kronecker-product Hamiltonians and of the FSA MPOs.

The Kronecker builders are pinned by textbook closed forms and by the
canonical anticommutation relations; the MPOs (Section II-B) are then pinned
by contracting them to dense matrices and comparing with those builders for
the Section V models (Heisenberg/J1-J2, Hubbard).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import kron


def test_two_site_heisenberg_singlet():
    # singlet energy of J S1.S2 is -3J/4
    H = kron.heisenberg_hamiltonian(2, [(0, 1, 1.0)])
    assert abs(kron.ground_energy(H) + 0.75) < 1e-14


def test_four_site_heisenberg_ring():
    # 4-site periodic Heisenberg ring: E0 = -2 J
    H = kron.heisenberg_hamiltonian(4, [(0, 1, 1.0), (1, 2, 1.0), (2, 3, 1.0), (0, 3, 1.0)])
    assert abs(kron.ground_energy(H) + 2.0) < 1e-13


@pytest.mark.parametrize("U", [0.0, 4.0, 8.0, 8.5])
def test_two_site_hubbard(U):
    # half-filled Hubbard dimer, singlet sector: E0 = (U - sqrt(U^2 + 16 t^2)) / 2
    H = kron.hubbard_hamiltonian(2, [(0, 1, 1.0)], U)
    q = kron.basis_charges(2, wl.electron_phys())
    E = kron.ground_energy(H, q, (2, 0))
    assert abs(E - (U - np.sqrt(U * U + 16.0)) / 2.0) < 1e-13


def test_free_fermions_match_single_particle_levels():
    # U = 0: the ground energy is the sum of the lowest single-particle levels
    n, hops = 4, [(0, 1, 1.0), (1, 2, 0.8), (2, 3, 1.0), (0, 3, 0.3), (0, 2, 0.2)]
    T = np.zeros((n, n))
    for i, j, t in hops:
        T[i, j] -= t
        T[j, i] -= t
    eps = np.sort(np.linalg.eigvalsh(T))
    H = kron.hubbard_hamiltonian(n, hops, 0.0)
    q = kron.basis_charges(n, wl.electron_phys())
    for nup, ndn in [(2, 2), (1, 2), (3, 1)]:
        E = kron.ground_energy(H, q, (nup + ndn, nup - ndn))
        assert abs(E - eps[:nup].sum() - eps[:ndn].sum()) < 1e-12


def test_fermion_anticommutation():
    c = kron.fermion_operators(3)
    modes = [c[i][s] for i in range(3) for s in range(2)]
    dim = 4 ** 3
    I = np.eye(dim)
    for a, A in enumerate(modes):
        for b, B in enumerate(modes):
            Ad, Bd = A.toarray(), B.toarray()
            assert np.abs(Ad @ Bd + Bd @ Ad).max() < 1e-14
            acomm = Ad @ Bd.T + Bd.T @ Ad
            assert np.abs(acomm - (I if a == b else 0.0)).max() < 1e-14


def test_site_basis_of_fermions():
    # |up dn> = c+_up c+_dn |0>  on a single site (state index 3 from index 0)
    c = kron.fermion_operators(1)
    vac = np.zeros(4)
    vac[0] = 1.0
    v = c[0][0].T.toarray() @ (c[0][1].T.toarray() @ vac)
    assert np.allclose(v, [0, 0, 0, 1])


@pytest.mark.parametrize("n,couplings", [(6, [1.0]), (7, [1.0, 0.5, 0.2, 0.1]), (5, [0.0, 1.0])])
def test_chain_mpo_equals_kron(n, couplings):
    pairs = wl.chain_pairs(n, couplings)
    mpo = wl.heisenberg_mpo(n, pairs)
    Hm = kron.mpo_to_dense(mpo)
    Hk = kron.heisenberg_hamiltonian(n, pairs).toarray()
    assert np.abs(Hm - Hk).max() < 1e-13


@pytest.mark.parametrize("Lx,Ly", [(3, 2), (2, 3), (2, 4)])
def test_j1j2_cylinder_mpo_equals_kron(Lx, Ly):
    pairs = wl.cylinder_pairs(Lx, Ly, 1.0, 0.5)
    n = Lx * Ly
    mpo = wl.heisenberg_mpo(n, pairs)
    Hm = kron.mpo_to_dense(mpo)
    Hk = kron.heisenberg_hamiltonian(n, pairs).toarray()
    assert np.abs(Hm - Hk).max() < 1e-12


def test_hubbard_mpo_equals_kron():
    hops = [(0, 1, 1.0), (1, 2, 0.7), (0, 2, 0.3), (2, 3, 1.1), (0, 3, 0.2)]
    mpo = wl.hubbard_mpo(4, hops, 8.5)
    Hm = kron.mpo_to_dense(mpo)
    Hk = kron.hubbard_hamiltonian(4, hops, 8.5).toarray()
    assert np.abs(Hm - Hk).max() < 1e-12


@pytest.mark.parametrize("Lx,Ly", [(3, 2), (2, 3)])
def test_hubbard_cylinder_mpo_equals_kron(Lx, Ly):
    # the nearest-neighbour hops of the snake-ordered cylinder (periodic in y) give the
    # Hubbard cylinder of Section V; its MPO must contract to the Kronecker Hamiltonian
    n = Lx * Ly
    hops = wl.cylinder_hops(Lx, Ly, 1.0)
    assert len(hops) == (Lx - 1) * Ly + Lx * (Ly if Ly > 2 else Ly - 1)
    mpo = wl.hubbard_mpo(n, hops, 8.0)
    Hm = kron.mpo_to_dense(mpo)
    Hk = kron.hubbard_hamiltonian(n, hops, 8.0).toarray()
    assert np.abs(Hm - Hk).max() < 1e-12


@pytest.mark.parametrize("Lx,Ly", [(3, 2), (2, 3)])
def test_triangular_hubbard_cylinder_mpo_equals_kron(Lx, Ly):
    # the paper's electron lattice: triangular, six neighbours per bulk site (x, y and the
    # (1, 1) diagonal), periodic in y; its MPO must contract to the Kronecker Hamiltonian
    n = Lx * Ly
    hops = wl.triangular_hops(Lx, Ly, 1.0)
    assert len(hops) == (Ly if Ly > 2 else Ly - 1) * Lx + 2 * (Lx - 1) * Ly
    mpo = wl.hubbard_mpo(n, hops, 8.5)
    Hm = kron.mpo_to_dense(mpo)
    Hk = kron.hubbard_hamiltonian(n, hops, 8.5).toarray()
    assert np.abs(Hm - Hk).max() < 1e-12


@pytest.mark.parametrize("which", ["spin", "electron"])
def test_mpo_charge_rule_and_transpose_symmetry(which):
    w = wl.spin_heff_workload(64, 8, 0) if which == "spin" else wl.electron_heff_workload(96, 3, 6, 24)
    for W, ql, qr in [(w.W1, w.ql, w.qm), (w.W2, w.qm, w.qr)]:
        for wl_, t, s, wr in np.argwhere(W != 0):
            assert np.array_equal(ql[wl_] + w.phys[t] - w.phys[s], qr[wr])
    # W[wl,t,s,wr] = W[conj wl, s, t, conj wr] (Hermitian MPO, real)
    from workloads.fill import spin_window, electron_window
    win = spin_window() if which == "spin" else electron_window()
    W1 = win["W1"]
    cl, cm = win["conj_l"], win["conj_m"]
    W1t = W1[cl][:, :, :, cm].transpose(0, 2, 1, 3)
    assert np.abs(W1 - W1t).max() == 0.0


@pytest.mark.parametrize("name", ["spin_j1j2_6x6_m200", "spin_j1j2_20x10_m200", "electron_hubbard_4x8_m96",
                                  "electron_tri_xc6_m96", "spin_j1j2_20x10c_m200", "electron_tri_xc6c_m96",
                                  "spin_j1j2_20x10ci_m200", "electron_tri_xc6ci_m96"])
def test_lattice_windows_charge_rule_and_hermiticity(name):
    # the lattice MPO windows obey the charge rule of every nonzero entry and are Hermitian
    # under the channel transposition map, as the chain windows are
    w = wl.workload_by_name(name)
    for W, ql, qr in [(w.W1, w.ql, w.qm), (w.W2, w.qm, w.qr)]:
        for wl_, t, s, wr in np.argwhere(W != 0):
            assert np.array_equal(ql[wl_] + w.phys[t] - w.phys[s], qr[wr])
    from workloads.fill import lattice_window
    win = {"spin_j1j2_6x6_m200": lambda: lattice_window(), "spin_j1j2_20x10_m200": lambda: lattice_window(20, 10),
           "electron_hubbard_4x8_m96": wl.hubbard_lattice_window,
           "electron_tri_xc6_m96": wl.triangular_hubbard_window,
           "spin_j1j2_20x10c_m200": lambda: lattice_window(20, 10, compress=True),
           "electron_tri_xc6c_m96": lambda: wl.triangular_hubbard_window(compress=True),
           "spin_j1j2_20x10ci_m200": lambda: lattice_window(20, 10, compress="interpolative"),
           "electron_tri_xc6ci_m96": lambda: wl.triangular_hubbard_window(compress="interpolative")}[name]()
    for W, c0, c1 in [(win["W1"], win["conj_l"], win["conj_m"]), (win["W2"], win["conj_m"], win["conj_r"])]:
        Wt = W[c0][:, :, :, c1].transpose(0, 2, 1, 3)
        assert np.abs(W - Wt).max() < 1e-14


def test_bulk_window_bond_dims():
    from workloads.fill import spin_window, electron_window
    assert spin_window()["W1"].shape == (14, 2, 2, 14)
    assert electron_window()["W1"].shape == (22, 4, 4, 22)
    # 4 x 8 Hubbard cylinder: at most four left sites with a hop across a bond, four
    # fermion channels each, plus the start and done channels
    win = wl.hubbard_lattice_window()
    assert win["W1"].shape == (18, 4, 4, 18) and win["W2"].shape == (18, 4, 4, 18)
    # the paper's lattices (uncompressed automaton MPOs): 20 x 10 J1-J2 spins, 6 x 6
    # triangular Hubbard (XC6)
    assert wl.lattice_window(20, 10)["W1"].shape == (38, 2, 2, 38)
    assert wl.triangular_hubbard_window()["W1"].shape == (30, 4, 4, 30)


# ---------------------------------------------------------------- MPO compression (Section VI-B)
def _operator_schmidt_rank(H, n, b, d):
    """Rank of H as a sum of (operator on sites < b) x (operator on sites >= b): the minimal
    MPO bond dimension at bond b, from the dense Hamiltonian."""
    dl, dr = d ** b, d ** (n - b)
    M = H.reshape(dl, dr, dl, dr).transpose(0, 2, 1, 3).reshape(dl * dl, dr * dr)
    s = np.linalg.svd(M, compute_uv=False)
    return int(np.sum(s > 1e-10 * s[0]))


@pytest.mark.parametrize("method", ["svd", "interpolative"])
@pytest.mark.parametrize("case", ["j1j2_3x4", "tri_hubbard_2x3", "chain_range3"])
def test_compressed_mpo_equals_kronecker_hamiltonian_with_minimal_bonds(case, method):
    if case == "j1j2_3x4":
        n, d = 12, 2
        pairs = wl.cylinder_pairs(3, 4, 1.0, 0.5)
        mpo, Hk = wl.heisenberg_mpo(n, pairs), kron.heisenberg_hamiltonian(n, pairs).toarray()
        supports = [(i, j) for i, j, _ in pairs]
    elif case == "tri_hubbard_2x3":
        n, d = 6, 4
        hops = wl.triangular_hops(2, 3, 1.0)
        mpo, Hk = wl.hubbard_mpo(n, hops, 8.5), kron.hubbard_hamiltonian(n, hops, 8.5).toarray()
        supports = [(i, j) for i, j, _ in hops] + [(i, i) for i in range(n)]
    else:
        n, d = 10, 2
        pairs = wl.chain_pairs(n, [1.0, 0.5, 0.2])
        mpo, Hk = wl.heisenberg_mpo(n, pairs), kron.heisenberg_hamiltonian(n, pairs).toarray()
        supports = [(i, j) for i, j, _ in pairs]
    c = wl.compress_mpo(mpo, 1e-13, method=method)
    # the same operator ...
    assert np.abs(kron.mpo_to_dense(c) - Hk).max() < 1e-12
    # ... with the fewest channels any MPO of it can have at every bond: the operator
    # Schmidt rank of H across the bond, plus the start / done channels the compression keeps
    # even where their operator is zero (no term lies wholly right / left of the bond)
    for b in range(1, n):
        zero_done = not any(j < b for i, j in supports)
        zero_start = not any(i >= b for i, j in supports)
        assert c.bond_dim(b) <= mpo.bond_dim(b)
        assert c.bond_dim(b) == _operator_schmidt_rank(Hk, n, b, d) + zero_done + zero_start, b
    assert any(c.bond_dim(b) < mpo.bond_dim(b) for b in range(1, n))
    # compressing again changes no bond
    cc = wl.compress_mpo(c, 1e-13, method=method)
    assert [cc.bond_dim(b) for b in range(n + 1)] == [c.bond_dim(b) for b in range(n + 1)]


@pytest.mark.parametrize("method", ["svd", "interpolative"])
def test_compressed_mpo_charge_rule_and_transpose_symmetry(method):
    for mpo in (wl.heisenberg_mpo(36, wl.cylinder_pairs(6, 6, 1.0, 0.5)),
                wl.hubbard_mpo(36, wl.triangular_hops(6, 6, 1.0), 8.5)):
        c = wl.compress_mpo(mpo, method=method)
        for n in range(c.n_sites):
            W, ql, qr = c.W[n], c.charges[n], c.charges[n + 1]
            for wl_, t, s, wr in np.argwhere(W != 0):
                assert np.array_equal(ql[wl_] + c.phys[t] - c.phys[s], qr[wr])
            Wt = W[c.conj[n]][:, :, :, c.conj[n + 1]].transpose(0, 2, 1, 3)
            assert np.abs(W - Wt).max() < 1e-14
        assert c.start_index(0) == 0 and c.done_index(c.n_sites) == 0


def test_interpolative_compression_keeps_w_sparse():
    # the same channel counts as the SVD basis, with the kept channels the automaton's own:
    # far fewer nonzeros per site tensor
    mpo = wl.heisenberg_mpo(200, wl.cylinder_pairs(20, 10, 1.0, 0.5))
    cs, ci = wl.compress_mpo(mpo, method="svd"), wl.compress_mpo(mpo, method="interpolative")
    assert [cs.bond_dim(b) for b in range(201)] == [ci.bond_dim(b) for b in range(201)]
    nnz = lambda m: sum(np.count_nonzero(w) for w in m.W)
    assert nnz(ci) < 0.3 * nnz(cs)
    assert all(lab[0] in ("start", "open", "done") for b in range(201) for lab in ci.channels[b])


def test_compressed_paper_lattice_bond_dims():
    # Section VI-B: the 6 x 6 triangular Hubbard MPO compressed at 1e-13 has k = 26; the
    # paper's 20 x 10 J1-J2 cylinder ends near k = 30 (32 here: the J1-J2 couplings of a
    # width-10 snake cylinder leave 10 independent open sites, 3 channels each, + 2)
    assert wl.triangular_hubbard_window(compress=True)["W1"].shape == (26, 4, 4, 26)
    assert wl.lattice_window(20, 10, compress=True)["W1"].shape == (32, 2, 2, 32)
    assert wl.lattice_window(compress=True)["W1"].shape == (20, 2, 2, 20)
