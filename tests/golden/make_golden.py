"""Write the stored expected values under tests/golden/ (oracle only).

Run from the repository root:  python tests/golden/make_golden.py

ed_energies.json: exact ground energies; each entry records the model, its lattice
and charge sector; the values come from ``oracle.kron`` (sparse Kronecker Hamiltonian
+ Lanczos eigensolver), whose builders are pinned by closed forms in
tests/test_oracle_kron_mpo.py.

dmrg_sweeps.json: the energy after every full sweep of the oracle's two-site DMRG
(``oracle.dmrg``, Section II-C) on the 6 x 6 J1-J2 cylinder (J2 = 0.5, snake order,
open in x and periodic in y) from the Neel product state, with the bond cap of each
sweep, the Lanczos step count and the SVD cutoff recorded beside the values.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl          # noqa: E402
from oracle import kron         # noqa: E402
from oracle import dmrg         # noqa: E402


def main():
    out = {}
    n = 16
    pairs = wl.chain_pairs(n, [1.0])
    H = kron.heisenberg_hamiltonian(n, pairs)
    out["heisenberg_chain_L16_obc_Sz0"] = {
        "model": "spin-1/2 Heisenberg chain J=1, open BC (Section V spin model, 1D)",
        "sector": "2Sz=0", "E0": kron.ground_energy(H, kron.basis_charges(n, wl.spin_phys()), (0,))}
    pairs = wl.cylinder_pairs(3, 4, 1.0, 0.5)
    H = kron.heisenberg_hamiltonian(12, pairs)
    out["j1j2_cylinder_3x4_J2_0.5_Sz0"] = {
        "model": "J1-J2 Heisenberg, J2/J1=0.5, 3x4 cylinder (open x, periodic y), snake order "
                 "(Section V spin model)",
        "sector": "2Sz=0", "E0": kron.ground_energy(H, kron.basis_charges(12, wl.spin_phys()), (0,))}
    hops = [(i, i + 1, 1.0) for i in range(5)]
    H = kron.hubbard_hamiltonian(6, hops, 8.0)
    out["hubbard_chain_L6_U8_half_filling"] = {
        "model": "Hubbard chain t=1, U=8, open BC (Section V electron model, 1D)",
        "sector": "N=6, 2Sz=0",
        "E0": kron.ground_energy(H, kron.basis_charges(6, wl.electron_phys()), (6, 0))}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ed_energies.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out, indent=1))

    sweeps = {}
    Lx, Ly = 6, 6
    n = Lx * Ly
    mpo = wl.heisenberg_mpo(n, wl.cylinder_pairs(Lx, Ly, 1.0, 0.5))
    states = [i % 2 for i in range(n)]            # up, down, up, ... along the snake: 2Sz = 0
    schedule, n_iter, cutoff = [16, 32, 64, 64], 20, 1e-12
    r = dmrg.dmrg(mpo, (0,), schedule, n_iter=n_iter, cutoff=cutoff, states=states)
    sweeps["j1j2_cylinder_6x6_J2_0.5_neel_start"] = {
        "model": "J1-J2 Heisenberg, J2/J1=0.5, 6x6 cylinder (open x, periodic y), snake order "
                 "(Section V spin model)",
        "sector": "2Sz=0", "states": states, "m_schedule": schedule, "lanczos_steps": n_iter,
        "svd_cutoff": cutoff, "sweep_energies": [float(e) for e in r["sweep_energies"]]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dmrg_sweeps.json")
    with open(path, "w") as f:
        json.dump(sweeps, f, indent=1, sort_keys=True)
    print(json.dumps(sweeps, indent=1))


if __name__ == "__main__":
    main()
