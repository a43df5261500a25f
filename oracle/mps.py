"""Block-sparse matrix product states (Section II-B, II-D).

Site tensors are block tensors T[a, s, b] with flows (+1, +1, -1): a block
(i, s, j) is allowed when q(j) = q(i) + q(s), so a bond charge counts the
charge of all sites to its left.  The last bond carries the total charge.
Canonical forms (Section II-C) come from block QR factorisations: for a
left-canonical site, the rows (a, s) that share the charge of b form one
matrix per sector, whose orthonormal factor is kept; a right-canonical site
uses the columns (s, b) sharing the charge of a.
"""
import numpy as np

from .blocks import BlockTensor, Index


def bond_structure(phys, n, total, m):
    """Bond indices of an MPS with bond dimension capped at ``m``.

    Bond b (left of site b) gets every charge reachable from both ends, with
    dimension min(m, #left basis states, #right basis states) of that charge.
    """
    phys = np.asarray(phys, dtype=np.int64)
    nq = phys.shape[1]
    total = np.asarray(total, dtype=np.int64)

    def counts_from(charges_list):
        c = {tuple(np.zeros(nq, dtype=np.int64)): 1}
        out = [dict(c)]
        for _ in charges_list:
            nc = {}
            for q, v in c.items():
                for p in phys:
                    k = tuple(np.asarray(q) + p)
                    nc[k] = nc.get(k, 0) + v
            c = nc
            out.append(dict(c))
        return out

    left = counts_from(range(n))                 # left[b]: charges of sites < b
    right = counts_from(range(n))                # right[r]: charges of r sites
    bonds = []
    for b in range(n + 1):
        sec_q, sec_d = [], []
        for q, cl in sorted(left[b].items()):
            rest = tuple(total - np.asarray(q))
            cr = right[n - b].get(rest, 0)
            if cr > 0:
                sec_q.append(q)
                sec_d.append(min(m, cl, cr))
        bonds.append(Index(np.array(sec_q, dtype=np.int64).reshape(-1, nq), sec_d))
    return bonds


def random_mps(phys, n, total, m, seed):
    """Random block MPS (Gaussian blocks) with the bond structure above."""
    rng = np.random.default_rng(seed)
    phys_ix = Index(phys, np.ones(len(phys), dtype=np.int64))
    bonds = bond_structure(phys, n, total, m)
    sites = []
    for k in range(n):
        t = BlockTensor([bonds[k], phys_ix, bonds[k + 1]], (1, 1, -1))
        for key in t.keys():
            t.blocks[key] = rng.standard_normal(t.shape(key))
        sites.append(t)
    return sites


def product_mps(phys, states):
    """MPS of the product state with local state ``states[k]`` on site k (Section II-B: a
    bond dimension 1 MPS): bond b has the single sector of the charge of sites < b, and
    every site holds one 1 x 1 x 1 block equal to 1.  It is left- and right-canonical."""
    phys = np.asarray(phys, dtype=np.int64)
    nq = phys.shape[1]
    phys_ix = Index(phys, np.ones(len(phys), dtype=np.int64))
    q = np.zeros(nq, dtype=np.int64)
    bonds = [Index(q.reshape(1, nq).copy(), [1])]
    for st in states:
        q = q + phys[int(st)]
        bonds.append(Index(q.reshape(1, nq).copy(), [1]))
    sites = []
    for k, st in enumerate(states):
        t = BlockTensor([bonds[k], phys_ix, bonds[k + 1]], (1, 1, -1))
        t.blocks[(0, int(st), 0)] = np.ones((1, 1, 1))
        sites.append(t)
    return sites


def _rows_by_right(T, j):
    """Stack the blocks (i, s, j) into one matrix [sum m_i x m_j]."""
    parts = [(key, blk[:, 0, :]) for key, blk in sorted(T.blocks.items()) if key[2] == j]
    return parts


def left_orthonormalize(sites, k):
    """Make site k left-canonical by block QR; push R into site k+1."""
    T = sites[k]
    bond = T.indices[2]
    new_dims = np.array(bond.dims)
    Qs, Rs = {}, {}
    for j in range(bond.nsec):
        parts = _rows_by_right(T, j)
        if not parts:
            new_dims[j] = 0
            continue
        M = np.vstack([p for _, p in parts])
        Q, R = np.linalg.qr(M)
        Qs[j] = (parts, Q)
        Rs[j] = R
        new_dims[j] = Q.shape[1]
    keep = np.where(new_dims > 0)[0]
    remap = {int(j): n for n, j in enumerate(keep)}
    newbond = Index(bond.charges[keep], new_dims[keep])
    A = BlockTensor([T.indices[0], T.indices[1], newbond], T.flows, T.target)
    for j, (parts, Q) in Qs.items():
        o = 0
        for key, p in parts:
            A.blocks[(key[0], key[1], remap[j])] = Q[o:o + p.shape[0]][:, None, :].copy()
            o += p.shape[0]
    sites[k] = A
    if k + 1 < len(sites):
        B = sites[k + 1]
        nb = BlockTensor([newbond, B.indices[1], B.indices[2]], B.flows, B.target)
        for key, blk in B.blocks.items():
            if key[0] in remap:
                R = Rs[key[0]]
                nb.blocks[(remap[key[0]], key[1], key[2])] = np.einsum("ij,jsk->isk", R, blk)
        sites[k + 1] = nb
    return sites


def right_orthonormalize(sites, k):
    """Make site k right-canonical by block LQ; push L into site k-1."""
    T = sites[k]
    bond = T.indices[0]
    new_dims = np.array(bond.dims)
    Qs, Ls = {}, {}
    for i in range(bond.nsec):
        parts = [(key, blk[:, 0, :]) for key, blk in sorted(T.blocks.items()) if key[0] == i]
        if not parts:
            new_dims[i] = 0
            continue
        M = np.hstack([p for _, p in parts])
        Q, R = np.linalg.qr(M.T)                 # M = R^T Q^T
        Qs[i] = (parts, Q.T)
        Ls[i] = R.T
        new_dims[i] = Q.shape[1]
    keep = np.where(new_dims > 0)[0]
    remap = {int(i): n for n, i in enumerate(keep)}
    newbond = Index(bond.charges[keep], new_dims[keep])
    Bt = BlockTensor([newbond, T.indices[1], T.indices[2]], T.flows, T.target)
    for i, (parts, Qt) in Qs.items():
        o = 0
        for key, p in parts:
            Bt.blocks[(remap[i], key[1], key[2])] = Qt[:, o:o + p.shape[1]][:, None, :].copy()
            o += p.shape[1]
    sites[k] = Bt
    if k - 1 >= 0:
        A = sites[k - 1]
        na = BlockTensor([A.indices[0], A.indices[1], newbond], A.flows, A.target)
        for key, blk in A.blocks.items():
            if key[2] in remap:
                Lm = Ls[key[2]]
                na.blocks[(key[0], key[1], remap[key[2]])] = np.einsum("isj,jk->isk", blk, Lm)
        sites[k - 1] = na
    return sites


def two_site(A, B):
    """x[a, s1, s2, b] = sum_c A[a, s1, c] B[c, s2, b] (Section III)."""
    x = BlockTensor([A.indices[0], A.indices[1], B.indices[1], B.indices[2]],
                    (1, 1, 1, -1), A.target)
    for key in x.keys():
        x.blocks[key] = np.zeros(x.shape(key))
    for (i, s1, c), Ab in A.blocks.items():
        for (c2, s2, j), Bb in B.blocks.items():
            if c2 == c:
                x.blocks[(i, s1, s2, j)][:, 0, 0, :] += Ab[:, 0, :] @ Bb[:, 0, :]
    return x


def to_dense_state(sites):
    """Contract the MPS into the full vector psi[s_0, ..., s_{n-1}]."""
    acc = None
    for T in sites:
        Td = T.to_dense()                          # [m_l, d, m_r]
        if acc is None:
            acc = Td.reshape(Td.shape[1], Td.shape[2]) if Td.shape[0] == 1 else Td
        else:
            acc = np.einsum("Pa,asb->Psb", acc, Td).reshape(-1, Td.shape[2])
    return acc.reshape(-1)


def left_part_dense(sites, k):
    """Q_L[s_0..s_{k-1}, a]: the contraction of sites 0..k-1 (k >= 1)."""
    acc = sites[0].to_dense()[0]                   # [d, m1]
    for T in sites[1:k]:
        Td = T.to_dense()
        acc = np.einsum("Pa,asb->Psb", acc, Td).reshape(-1, Td.shape[2])
    return acc


def right_part_dense(sites, k):
    """Q_R[b, s_k..s_{n-1}]: the contraction of sites k..n-1."""
    acc = sites[-1].to_dense()[:, :, 0]            # [m, d]
    for T in reversed(sites[k:-1]):
        Td = T.to_dense()
        acc = np.einsum("asb,bP->asP", Td, acc).reshape(Td.shape[0], -1)
    return acc
