"""Hamiltonians by Kronecker products, and exact diagonalisation.

Independent of any MPO: operators are built as sparse matrices on the full
product space (site 0 is the most significant factor, matching the MPS
contraction order of Section II-B), and the Hamiltonians of Section V are
summed term by term:

* Heisenberg:  H = sum_(i,j) J_ij S_i . S_j, with
  S_i . S_j = (S+_i S-_j + S-_i S+_j)/2 + Sz_i Sz_j;
* Hubbard:     H = -sum_(i,j),s t_ij (c+_is c_js + h.c.) + U sum_i n_i,up n_i,dn,
  with fermionic operators from the Jordan-Wigner construction over the mode
  order (site 0 up, site 0 dn, site 1 up, ...).

The ground energy in a fixed charge sector comes from ``scipy.sparse.linalg.eigsh``
(or ``numpy.linalg.eigh`` for small sectors).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def _site_op(op, i, n, d, fill=None):
    mats = []
    for k in range(n):
        if k == i:
            mats.append(sp.csr_matrix(op))
        elif fill is not None and k < i:
            mats.append(sp.csr_matrix(fill))
        else:
            mats.append(sp.identity(d, format="csr"))
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m, format="csr")
    return out


def heisenberg_hamiltonian(n, pairs, field_z=0.0):
    """Sparse H = sum J S_i.S_j (+ h sum Sz_i) on n spin-1/2 sites."""
    spl = np.array([[0.0, 1.0], [0.0, 0.0]])
    sml = spl.T
    szl = np.diag([0.5, -0.5])
    Sp = [_site_op(spl, i, n, 2) for i in range(n)]
    Sm = [_site_op(sml, i, n, 2) for i in range(n)]
    Sz = [_site_op(szl, i, n, 2) for i in range(n)]
    H = sp.csr_matrix((2 ** n, 2 ** n))
    for (i, j, J) in pairs:
        H = H + J * (0.5 * (Sp[i] @ Sm[j] + Sm[i] @ Sp[j]) + Sz[i] @ Sz[j])
    if field_z:
        for i in range(n):
            H = H + field_z * Sz[i]
    return H.tocsr()


def fermion_operators(n):
    """Annihilators c[i][s] (s=0 up, 1 dn) on n sites, 4 states per site.

    Each site's space is spanned by |0>, |up>, |dn>, |up dn> and the
    Jordan-Wigner string runs over all modes before (i, s) in the order
    (0,up), (0,dn), (1,up), ...  Built mode by mode on a 2^(2n) space and
    then regrouped, so it does not rely on any local sign convention.
    """
    nm = 2 * n
    a = np.array([[0.0, 1.0], [0.0, 0.0]])        # annihilates an occupied mode
    z = np.diag([1.0, -1.0])                       # parity of one mode
    modes = []
    for k in range(nm):
        mats = [z] * k + [a] + [np.eye(2)] * (nm - k - 1)
        out = sp.csr_matrix(mats[0])
        for m in mats[1:]:
            out = sp.kron(out, sp.csr_matrix(m), format="csr")
        modes.append(out)
    # per-site mode basis |n_up n_dn> with n=0 first in the kron (occupied=index 1)
    # maps to the site basis (|0>,|up>,|dn>,|updn>) = (00, 10, 01, 11):
    # kron index = 2*n_up + n_dn -> site index
    perm_site = {0: 0, 2: 1, 1: 2, 3: 3}
    dim = 4 ** n
    # build the permutation from the kron ordering of 2n modes to site states
    idx = np.arange(dim)
    new = np.zeros(dim, dtype=np.int64)
    for b in range(dim):
        # bits of b in the mode-kron order: mode 0 is most significant
        site_states = []
        for i in range(n):
            nu = (b >> (nm - 1 - 2 * i)) & 1
            nd = (b >> (nm - 2 - 2 * i)) & 1
            site_states.append(perm_site[2 * nu + nd])
        v = 0
        for s in site_states:
            v = v * 4 + s
        new[b] = v
    P = sp.csr_matrix((np.ones(dim), (new, idx)), shape=(dim, dim))
    ops = []
    for i in range(n):
        ops.append([(P @ modes[2 * i] @ P.T).tocsr(), (P @ modes[2 * i + 1] @ P.T).tocsr()])
    return ops


def hubbard_hamiltonian(n, hops, U):
    """Sparse Hubbard H on n sites (4 states each)."""
    c = fermion_operators(n)
    dim = 4 ** n
    H = sp.csr_matrix((dim, dim))
    for (i, j, t) in hops:
        for s in range(2):
            hop = c[i][s].T @ c[j][s]
            H = H - t * (hop + hop.T)
    for i in range(n):
        nu = c[i][0].T @ c[i][0]
        nd = c[i][1].T @ c[i][1]
        H = H + U * (nu @ nd)
    return H.tocsr()


def basis_charges(n, phys):
    """Total charge of every product basis state (site 0 most significant)."""
    phys = np.asarray(phys)
    d, nq = phys.shape
    q = np.zeros((1, nq), dtype=np.int64)
    for _ in range(n):
        q = (q[:, None, :] + phys[None, :, :]).reshape(-1, nq)
    return q


def ground_energy(H, charges=None, sector=None, k=1):
    """Lowest eigenvalue(s) of H, optionally within one charge sector."""
    if sector is not None:
        sel = np.where((charges == np.asarray(sector)).all(axis=1))[0]
        H = H[sel][:, sel]
    n = H.shape[0]
    if n <= 2000:
        w = np.linalg.eigvalsh(H.toarray() if sp.issparse(H) else H)
        return w[:k] if k > 1 else float(w[0])
    w = sla.eigsh(H, k=max(k, 1), which="SA", tol=1e-13, maxiter=100000)[0]
    w = np.sort(w)
    return w[:k] if k > 1 else float(w[0])


def mpo_to_dense(mpo):
    """Contract an MPO (dense site tensors) into the full matrix."""
    W0 = mpo.W[0]
    acc = W0[0]                                  # [d, d, k1]
    acc = acc.reshape(W0.shape[1], W0.shape[2], W0.shape[3])
    for Wn in mpo.W[1:]:
        # acc[T, S, w] * Wn[w, t, s, w'] -> [T t, S s, w']
        D1, D2, k = acc.shape
        d = Wn.shape[1]
        acc = np.einsum("ABw,wtsv->AtBsv", acc, Wn).reshape(D1 * d, D2 * d, Wn.shape[3])
    return acc[:, :, 0]
