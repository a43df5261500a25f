"""Two-site DMRG sweeps on the GPU (paper_2007_05540_gb300.dmrg) against exact
diagonalisation (tests/golden/ed_energies.json, written by tests/golden/make_golden.py from
the oracle's Kronecker-product Hamiltonians).

The driver chains the library's two-site contraction, Lanczos, SVD truncation and
environment update from a product state; the energies after the sweeps must reach the
exact ground energy (variationally, from above) to the accuracy the bond cap allows, and
with BF16x3 matvecs the FP64 Rayleigh quotient of the final vector must agree as well.
"""
import json
import os

import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_05540_gb300 import dmrg   # noqa: E402


def _ed(key):
    with open(os.path.join(os.path.dirname(__file__), "golden", "ed_energies.json")) as f:
        return json.load(f)[key]["E0"]


def test_heisenberg_chain_16_reaches_ed():
    n = 16
    mpo = wl.heisenberg_mpo(n, wl.chain_pairs(n, [1.0]))
    E_ed = _ed("heisenberg_chain_L16_obc_Sz0")
    r = dmrg.dmrg(mpo, (0,), [16, 32, 64, 64, 64], n_iter=20)
    E = r["energy"]
    print(f"L=16 chain: sweeps {['%.12f' % e for e in r['sweep_energies']]} ED {E_ed:.12f} bonds {r['bond_dims']}")
    assert E >= E_ed - 1e-12 * abs(E_ed)
    assert abs(E - E_ed) < 1e-9 * abs(E_ed)


def test_heisenberg_chain_16_bf16x3_matvecs_with_fp64_energy():
    n = 16
    mpo = wl.heisenberg_mpo(n, wl.chain_pairs(n, [1.0]))
    E_ed = _ed("heisenberg_chain_L16_obc_Sz0")
    r = dmrg.dmrg(mpo, (0,), [16, 32, 64, 64, 64], precision="bf16x3", n_iter=20)
    print(f"L=16 chain bf16x3: last Ritz {r['energy']:.12f} FP64 energy {r['refined_energy']:.12f} ED {E_ed:.12f}")
    assert abs(r["energy"] - E_ed) < 1e-4 * abs(E_ed)
    assert abs(r["refined_energy"] - E_ed) < 1e-8 * abs(E_ed)


def test_heisenberg_chain_16_tensor_core_environments():
    """BF16x3 matvecs and environment updates on the tensor cores (FP32-accumulated, about
    1e-5 relative per update, compounding over the sweeps' updates): the FP64 energy of the
    final vector in those environments stays within 1e-4 of the exact ground energy."""
    n = 16
    mpo = wl.heisenberg_mpo(n, wl.chain_pairs(n, [1.0]))
    E_ed = _ed("heisenberg_chain_L16_obc_Sz0")
    r = dmrg.dmrg(mpo, (0,), [16, 32, 64, 64, 64], precision="bf16x3", n_iter=20, env_precision="bf16x3")
    print(f"L=16 chain, tensor-core environments: FP64 energy {r['refined_energy']:.12f} ED {E_ed:.12f} "
          f"(rel {abs(r['refined_energy'] - E_ed) / abs(E_ed):.1e})")
    assert abs(r["refined_energy"] - E_ed) < 1e-4 * abs(E_ed)


def test_j1j2_cylinder_3x4_reaches_ed():
    pairs = wl.cylinder_pairs(3, 4, 1.0, 0.5)
    mpo = wl.heisenberg_mpo(12, pairs)
    E_ed = _ed("j1j2_cylinder_3x4_J2_0.5_Sz0")
    r = dmrg.dmrg(mpo, (0,), [16, 32, 64, 64, 64], n_iter=25)
    print(f"3x4 J1-J2: {r['energy']:.12f} ED {E_ed:.12f}")
    assert abs(r["energy"] - E_ed) < 1e-9 * abs(E_ed)


@pytest.mark.parametrize("method", ["svd", "interpolative"])
def test_j1j2_cylinder_3x4_compressed_mpo_reaches_ed(method):
    """The same lattice with its MPO compressed at the SVD cutoff 1e-13 (Section VI-B):
    fewer channels, the same Hamiltonian, the same ground energy."""
    pairs = wl.cylinder_pairs(3, 4, 1.0, 0.5)
    mpo = wl.compress_mpo(wl.heisenberg_mpo(12, pairs), method=method)
    E_ed = _ed("j1j2_cylinder_3x4_J2_0.5_Sz0")
    r = dmrg.dmrg(mpo, (0,), [16, 32, 64, 64, 64], n_iter=25)
    print(f"3x4 J1-J2, compressed MPO (k <= {max(mpo.bond_dim(b) for b in range(13))}): {r['energy']:.12f} "
          f"ED {E_ed:.12f}")
    assert abs(r["energy"] - E_ed) < 1e-9 * abs(E_ed)


def test_j1j2_cylinder_6x6_sweeps_match_oracle():
    """The paper's spin model on a 6 x 6 cylinder (36-site snake MPS): every sweep's energy
    equals the oracle's two-site DMRG from the same Neel product state with the same bond
    caps, Lanczos step count and SVD cutoff (tests/golden/dmrg_sweeps.json, written by the
    oracle)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "dmrg_sweeps.json")) as f:
        g = json.load(f)["j1j2_cylinder_6x6_J2_0.5_neel_start"]
    mpo = wl.heisenberg_mpo(36, wl.cylinder_pairs(6, 6, 1.0, 0.5))
    r = dmrg.dmrg(mpo, (0,), g["m_schedule"], n_iter=g["lanczos_steps"], cutoff=g["svd_cutoff"],
                  states=g["states"])
    ref = g["sweep_energies"]
    print(f"6x6 J1-J2: GPU {['%.12f' % e for e in r['sweep_energies']]}")
    print(f"        oracle {['%.12f' % e for e in ref]}  bonds {r['bond_dims']}")
    assert len(r["sweep_energies"]) == len(ref)
    for e, e_ref in zip(r["sweep_energies"], ref):
        assert abs(e - e_ref) < 1e-10 * abs(e_ref)


def test_hubbard_chain_6_reaches_ed():
    n = 6
    mpo = wl.hubbard_mpo(n, [(i, i + 1, 1.0) for i in range(n - 1)], 8.0)
    E_ed = _ed("hubbard_chain_L6_U8_half_filling")
    r = dmrg.dmrg(mpo, (6, 0), [16, 64, 64, 64], n_iter=25)
    print(f"Hubbard L=6: {r['energy']:.12f} ED {E_ed:.12f}")
    assert abs(r["energy"] - E_ed) < 1e-9 * abs(E_ed)


def test_heisenberg_chain_10_davidson_subspace_2_reaches_ed():
    """The paper's sweep setting: Algorithm 1 with a subspace of 2 at every bond."""
    from oracle import kron
    n = 10
    mpo = wl.heisenberg_mpo(n, wl.chain_pairs(n, [1.0]))
    E_ed = kron.ground_energy(kron.heisenberg_hamiltonian(n, wl.chain_pairs(n, [1.0])),
                              kron.basis_charges(n, wl.spin_phys()), (0,))
    r = dmrg.dmrg(mpo, (0,), [32] * 10, solver="davidson", davidson_vecs=2)
    print(f"L=10 chain, Davidson(2): sweeps {['%.12f' % e for e in r['sweep_energies']]} ED {E_ed:.12f}")
    assert r["energy"] >= E_ed - 1e-12 * abs(E_ed)
    assert abs(r["energy"] - E_ed) < 1e-8 * abs(E_ed)
