"""Pins of the oracle's H_eff apply and environment extension.

* y = K x with K = Q^T H Q (Section II-C, the defining equation of the
  projected Hamiltonian) built from a random canonical MPS and the dense
  Kronecker Hamiltonian: pins the environments, the MPO and the block apply
  together against the paper's definition.
* block apply = dense einsum of the two-site definition;
* Hermiticity, linearity, charge conservation;
* the L = I, R = I special case reduces to the two-site MPO operator acting on
  the physical indices;
* a hand-counted flop total for a one-sector problem.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import kron, mps, env, heff
from oracle.blocks import BlockTensor, Index, allowed_keys


def _canonical_setup(mpo, total, n, j, m, seed):
    sites = mps.random_mps(mpo.phys, n, total, m, seed)
    for k in range(n - 1, j + 1, -1):
        sites = mps.right_orthonormalize(sites, k)
    for k in range(0, j):
        sites = mps.left_orthonormalize(sites, k)
    nq = mpo.phys.shape[1]
    L = env.left_boundary(nq)
    for k in range(j):
        L = env.extend_left(L, sites[k], mpo.W[k], mpo.charges[k + 1])
    R = env.right_boundary(total, mpo.charges[n], mpo.done_index(n))
    for k in range(n - 1, j + 1, -1):
        R = env.extend_right(R, sites[k], mpo.W[k], mpo.charges[k])
    return sites, L, R


def _projected_K(mpo, H, sites, n, j):
    d = mpo.phys.shape[0]
    QL = mps.left_part_dense(sites, j) if j > 0 else np.ones((1, 1))
    QR = mps.right_part_dense(sites, j + 2) if j + 2 < n else np.ones((1, 1))
    Q = np.einsum("Pa,st,uv,bR->PsuRatvb", QL, np.eye(d), np.eye(d), QR)
    Q = Q.reshape(QL.shape[0] * d * d * QR.shape[1], QL.shape[1] * d * d * QR.shape[0])
    return Q.T @ H @ Q


@pytest.mark.parametrize("j", [0, 3, 6])
def test_heff_equals_projected_hamiltonian_spins(j):
    n = 8
    pairs = wl.chain_pairs(n, [1.0, 0.5, 0.2, 0.1])
    mpo = wl.heisenberg_mpo(n, pairs)
    H = kron.heisenberg_hamiltonian(n, pairs).toarray()
    sites, L, R = _canonical_setup(mpo, (0,), n, j, 6, 11 + j)
    x = mps.two_site(sites[j], sites[j + 1])
    rng = np.random.default_rng(j)
    for k in x.blocks:
        x.blocks[k] = rng.standard_normal(x.blocks[k].shape)
    y = heff.heff_apply(L, mpo.W[j], mpo.W[j + 1], R, x)
    K = _projected_K(mpo, H, sites, n, j)
    xd, yd = x.to_dense().reshape(-1), y.to_dense().reshape(-1)
    assert np.abs(K @ xd - yd).max() < 1e-12 * max(1.0, np.abs(yd).max())


def test_heff_equals_projected_hamiltonian_j1j2_cylinder():
    Lx, Ly = 3, 3
    n = Lx * Ly
    pairs = wl.cylinder_pairs(Lx, Ly, 1.0, 0.5)
    mpo = wl.heisenberg_mpo(n, pairs)
    H = kron.heisenberg_hamiltonian(n, pairs).toarray()
    j = 4
    sites, L, R = _canonical_setup(mpo, (1,), n, j, 5, 3)
    x = mps.two_site(sites[j], sites[j + 1])
    y = heff.heff_apply(L, mpo.W[j], mpo.W[j + 1], R, x)
    K = _projected_K(mpo, H, sites, n, j)
    assert np.abs(K @ x.to_dense().reshape(-1) - y.to_dense().reshape(-1)).max() < 1e-12


@pytest.mark.parametrize("j,total", [(1, (4, 0)), (0, (3, 1)), (2, (4, 2))])
def test_heff_equals_projected_hamiltonian_hubbard(j, total):
    n = 4
    hops = [(0, 1, 1.0), (1, 2, 1.0), (2, 3, 1.0), (0, 2, 0.5), (1, 3, 0.4)]
    mpo = wl.hubbard_mpo(n, hops, 8.0)
    H = kron.hubbard_hamiltonian(n, hops, 8.0).toarray()
    sites, L, R = _canonical_setup(mpo, total, n, j, 8, 5)
    x = mps.two_site(sites[j], sites[j + 1])
    rng = np.random.default_rng(9)
    for k in x.blocks:
        x.blocks[k] = rng.standard_normal(x.blocks[k].shape)
    y = heff.heff_apply(L, mpo.W[j], mpo.W[j + 1], R, x)
    K = _projected_K(mpo, H, sites, n, j)
    yd = y.to_dense().reshape(-1)
    assert np.abs(K @ x.to_dense().reshape(-1) - yd).max() < 1e-12 * max(1.0, np.abs(yd).max())


@pytest.mark.parametrize("name", ["spin_m64", "electron_m96", "electron_hubbard_4x8_m96"])
def test_block_apply_equals_dense_einsum(name):
    w = wl.workload_by_name(name)
    L, W1, W2, R, x = heff.problem_from_workload(w)
    y = heff.heff_apply(L, W1, W2, R, x)
    yd = heff.heff_apply_dense(L.to_dense(), W1, W2, R.to_dense(), x.to_dense())
    assert np.abs(y.to_dense() - yd).max() < 1e-12 * np.abs(yd).max()
    # no weight outside allowed blocks: the dense result re-blocked is the same
    yb = BlockTensor.from_dense(x.indices, x.flows, x.target, yd)
    assert abs(np.linalg.norm(yd) - yb.norm()) < 1e-12 * np.linalg.norm(yd)


@pytest.mark.parametrize("name", ["spin_m64", "electron_m96", "electron_hubbard_4x8_m96"])
def test_heff_hermitian_and_linear(name):
    w = wl.workload_by_name(name)
    L, W1, W2, R, u = heff.problem_from_workload(w, batch=0)
    _, _, _, _, v = heff.problem_from_workload(w, batch=1)
    Ku = heff.heff_apply(L, W1, W2, R, u)
    Kv = heff.heff_apply(L, W1, W2, R, v)
    a = u.vdot(Kv)
    b = Ku.vdot(v)
    assert abs(a - b) < 1e-12 * max(abs(a), 1.0)
    comb = u.copy().scale(2.5).axpy(-0.75, v)
    Kc = heff.heff_apply(L, W1, W2, R, comb)
    ref = Ku.copy().scale(2.5).axpy(-0.75, Kv)
    assert Kc.copy().axpy(-1.0, ref).norm() < 1e-12 * ref.norm()


def test_identity_environments_reduce_to_two_site_operator():
    # L = delta on the start channel, R = delta on the done channel:
    # y[a, t1, t2, b] = sum_s W12[start, t1, t2, s1, s2, done] x[a, s1, s2, b]
    w = wl.workload_by_name("spin_m64")
    L, W1, W2, R, x = heff.problem_from_workload(w)
    for (ip, wl_, i) in list(L.blocks):
        if wl_ != w.start_l:
            L.blocks[(ip, wl_, i)][:] = 0.0
    for (jp, wr, j) in list(R.blocks):
        if wr != w.done_r:
            R.blocks[(jp, wr, j)][:] = 0.0
    y = heff.heff_apply(L, W1, W2, R, x)
    W12 = np.einsum("atsm,muvr->atusvr", W1, W2)[w.start_l, :, :, :, :, w.done_r]
    xd = x.to_dense()
    ref = np.einsum("tusv,asvb->atub", W12, xd)
    assert np.abs(y.to_dense() - ref).max() < 1e-13
    # the two-site operator of the chain MPO is J_1 S1.S2: check its spectrum
    S = W12.reshape(4, 4)
    assert np.allclose(np.sort(np.linalg.eigvalsh(S)), [-0.75, 0.25, 0.25, 0.25])


def test_hand_counted_flops():
    # one-sector bonds (dims 3 and 2, charge 0), identity MPO (k = 1)
    alpha = Index([[0]], [3])
    beta = Index([[0]], [2])
    phys = Index([[1], [-1]], [1, 1])
    ch = Index([[0]], [1])
    rng = np.random.default_rng(0)
    fill = lambda k: rng.standard_normal(1)
    L = BlockTensor.from_fill([alpha, ch, alpha], (-1, 1, 1), [0], lambda k: rng.standard_normal(9))
    R = BlockTensor.from_fill([beta, ch, beta], (-1, 1, 1), [0], lambda k: rng.standard_normal(4))
    x = BlockTensor.from_fill([alpha, phys, phys, beta], (1, 1, 1, -1), [0],
                              lambda k: rng.standard_normal(6))
    W = np.zeros((1, 2, 2, 1))
    W[0, 0, 0, 0] = W[0, 1, 1, 0] = 1.0
    # x blocks: (up, dn) and (dn, up); GEMM1: 2 * (2*3*3*2) = 72; GEMM2: 2 * (2*3*2*2) = 48
    c = heff.canonical_flops(L, W, W, R, x)
    assert c == {"gemm1": 72, "gemm2": 48, "total": 120}
    cnt = {}
    heff.heff_apply(L, W, W, R, x, count=cnt)
    assert cnt["gemm1"] == 72 and cnt["gemm2"] == 48


def test_canonical_flops_matches_apply_count():
    w = wl.workload_by_name("electron_m96")
    L, W1, W2, R, x = heff.problem_from_workload(w)
    cnt = {}
    heff.heff_apply(L, W1, W2, R, x, count=cnt)
    c = heff.canonical_flops(L, W1, W2, R, x)
    assert c["gemm1"] == cnt["gemm1"] and c["gemm2"] == cnt["gemm2"]


def test_allowed_keys_brute_force():
    a = Index([[1], [-1], [3]], [2, 1, 4])
    p = Index([[1], [-1]], [1, 1])
    keys = allowed_keys([a, p, p, a], (1, 1, 1, -1), [0])
    brute = [(i, s, t, j) for i in range(3) for s in range(2) for t in range(2) for j in range(3)
             if a.charges[i, 0] + p.charges[s, 0] + p.charges[t, 0] - a.charges[j, 0] == 0]
    assert keys == brute


def test_extend_left_right_equal_dense():
    n = 6
    pairs = wl.chain_pairs(n, [1.0, 0.5])
    mpo = wl.heisenberg_mpo(n, pairs)
    sites = mps.random_mps(mpo.phys, n, (0,), 4, 2)
    L = env.left_boundary(1)
    Ld = L.to_dense()
    for k in range(3):
        L = env.extend_left(L, sites[k], mpo.W[k], mpo.charges[k + 1])
        Ld = env.extend_left_dense(Ld, sites[k].to_dense(), mpo.W[k])
        assert np.abs(L.to_dense() - Ld).max() < 1e-12
    R = env.right_boundary((0,), mpo.charges[n], mpo.done_index(n))
    Rd = R.to_dense()
    for k in range(n - 1, 2, -1):
        R = env.extend_right(R, sites[k], mpo.W[k], mpo.charges[k])
        Rd = env.extend_right_dense(Rd, sites[k].to_dense(), mpo.W[k])
        assert np.abs(R.to_dense() - Rd).max() < 1e-12


def test_left_canonical_identity_channel():
    # For left-canonical sites the start channel of L stays the identity (A^T A = I)
    n = 6
    mpo = wl.heisenberg_mpo(n, wl.chain_pairs(n, [1.0]))
    sites = mps.random_mps(mpo.phys, n, (0,), 5, 4)
    for k in range(0, 4):
        sites = mps.left_orthonormalize(sites, k)
    L = env.left_boundary(1)
    for k in range(4):
        L = env.extend_left(L, sites[k], mpo.W[k], mpo.charges[k + 1])
    Ld = L.to_dense()
    s = mpo.start_index(4)
    assert np.abs(Ld[:, s, :] - np.eye(Ld.shape[0])).max() < 1e-12
