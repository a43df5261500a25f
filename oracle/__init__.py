"""Plain FP64 CPU oracle for the two-site DMRG effective-Hamiltonian path.

TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports, links or calls
this package; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.  It shares no code with the CUDA path: the two
meet only through the seeded input generators in ``workloads``.

Every function is a direct restatement of the paper's definitions (Levy,
Solomonik, Clark, "Distributed-Memory DMRG via Sparse and Dense Parallel
Tensor Contractions"), written for readability, not speed:

* ``blocks``   quantum-number block tensors (Section II-D: a tensor is a list of
               dense blocks, one per allowed label tuple)
* ``heff``     the two-site H_eff matvec (Section II-C equation for K, two-site
               form of Section III, Fig. 1d) by blocks and by dense einsum
* ``env``      environment extension (Section II-C definition of A and B)
* ``kron``     dense / sparse Hamiltonians by Kronecker products and exact
               diagonalisation (ground truth for the MPOs and DMRG)
* ``mps``      random block-sparse MPS, canonical forms, two-site tensor
* ``eig``      Lanczos and the Davidson routine of Algorithm 1
* ``svd``      block SVD split with truncation (Section IV, Fig. 1e)
* ``dmrg``     two-site DMRG sweeps (Section II-C, III)
* ``grad``     gradients of the Rayleigh quotient <x|K|x>/<x|x>

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms, exact diagonalisation, brute force or invariants; none is
"parity unpinned".
"""
