"""Two-site DMRG (Section II-C and III).

One optimisation step at bond (j, j+1): form x = T^(j) T^(j+1), find the
lowest eigenpair of H_eff (Lanczos or Algorithm 1), split x by a truncated
block SVD (absorbing the singular values in the sweep direction), and extend
the environment by the new canonical site.  Sweeps run left-to-right then
right-to-left, with the bond dimension grown by a schedule (Section III: the
bond dimension is increased gradually over sweeps).
"""
import numpy as np

from .blocks import BlockTensor
from .heff import heff_apply
from .env import left_boundary, right_boundary, extend_left, extend_right
from .mps import random_mps, product_mps, right_orthonormalize, two_site
from .eig import lanczos, davidson
from .svd import svd_split


class _Shape:
    """Flat-vector view of a block tensor for the eigensolvers."""

    def __init__(self, like):
        self.like = like
        self.keys = sorted(like.blocks)

    def to_flat(self, t):
        return np.concatenate([t.blocks[k].reshape(-1) for k in self.keys])

    def to_tensor(self, v):
        t = BlockTensor(self.like.indices, self.like.flows, self.like.target)
        o = 0
        for k in self.keys:
            n = self.like.blocks[k].size
            t.blocks[k] = v[o:o + n].reshape(self.like.blocks[k].shape)
            o += n
        return t


def dmrg(mpo, total, m_schedule, solver="lanczos", n_iter=30, cutoff=1e-12,
         seed=0, davidson_vecs=2, m_init=8, states=None):
    """Run sweeps; ``m_schedule`` lists the bond cap of each full sweep.

    The start is a random MPS with bond cap ``m_init`` brought to right-canonical form,
    or, when ``states`` lists one local state per site (charges adding up to ``total``),
    that product state (bond dimension 1, already canonical); two-site updates grow the
    bonds from there.

    Returns a dict with the energy after every step, per-sweep energies and
    the final MPS.
    """
    n = mpo.n_sites
    nq = mpo.phys.shape[1]
    if states is not None:
        sites = product_mps(mpo.phys, states)
        qt = sites[-1].indices[2].charges[0]
        if not np.array_equal(qt, np.asarray(total).reshape(-1)):
            raise ValueError(f"product state has total charge {tuple(qt)}, not {tuple(total)}")
    else:
        sites = random_mps(mpo.phys, n, total, m_init, seed)
        for k in range(n - 1, 0, -1):
            sites = right_orthonormalize(sites, k)
        sites[0].scale(1.0 / sites[0].norm())
    Ls = [None] * (n + 1)
    Rs = [None] * (n + 2)
    Ls[0] = left_boundary(nq)
    Rs[n] = right_boundary(total, mpo.charges[n], mpo.done_index(n))
    for k in range(n - 1, 1, -1):
        Rs[k] = extend_right(Rs[k + 1], sites[k], mpo.W[k], mpo.charges[k])
    energies, sweep_E = [], []
    step = 0

    def solve(j, x):
        nonlocal step
        L, W1, W2, R = Ls[j], mpo.W[j], mpo.W[j + 1], Rs[j + 2]
        shp = _Shape(x)
        mv = lambda v: shp.to_flat(heff_apply(L, W1, W2, R, shp.to_tensor(v)))
        v0 = shp.to_flat(x)
        if solver == "lanczos":
            E, v, _ = lanczos(mv, v0, n_iter)
        else:
            E, v = davidson(mv, v0, davidson_vecs, seed=seed + step)
        step += 1
        return E, shp.to_tensor(v)

    for m in m_schedule:
        for j in range(0, n - 1):
            x = two_site(sites[j], sites[j + 1])
            E, x = solve(j, x)
            energies.append(E)
            A, B, s, disc = svd_split(x, m, cutoff, absorb="right")
            sites[j], sites[j + 1] = A, B
            Ls[j + 1] = extend_left(Ls[j], A, mpo.W[j], mpo.charges[j + 1])
        for j in range(n - 2, -1, -1):
            x = two_site(sites[j], sites[j + 1])
            E, x = solve(j, x)
            energies.append(E)
            A, B, s, disc = svd_split(x, m, cutoff, absorb="left")
            sites[j], sites[j + 1] = A, B
            Rs[j + 1] = extend_right(Rs[j + 2], B, mpo.W[j + 1], mpo.charges[j + 1])
        sweep_E.append(energies[-1])
    return {"energies": energies, "sweep_energies": sweep_E, "sites": sites}
