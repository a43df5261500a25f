"""Matrix product operators (Section II-B) for the paper's lattice models.

The paper builds its MPOs with ITensor's AutoMPO (Section V); that tool is not
available here, so this module writes the standard finite-state-automaton (FSA)
form of a Hamiltonian made of on-site terms and two-site product terms
``c * A_i (string ops on i < l < j) B_j``.  At the bond after site ``b`` the
channels are

* ``start``: nothing placed yet (identity so far),
* ``(i, A)``: operator ``A`` placed on site ``i <= b`` and waiting for a
  partner site ``j > b`` (one channel per open site and operator type),
* ``done``: a term finished on the left.

Site tensors are dense arrays ``W[wl, t, s, wr] = <t| O |s>`` for the
operator ``O`` on the transition ``wl -> wr``.  The channel charge is the total
charge change of the operators placed so far, so every nonzero entry obeys
``q(wl) + q(t) - q(s) = q(wr)``.  Channel ``(i, A)`` transposes into
``(i, A^T)``; that map (``conj``) keeps environment tensors built from it
symmetric.
"""
from dataclasses import dataclass, field
import numpy as np


@dataclass
class MPO:
    """A site-dependent MPO.

    ``W[n]`` has shape ``[k_n, d, d, k_{n+1}]``; ``channels[b]`` lists the
    labels of bond ``b`` (bond 0 is the left boundary, bond N the right
    boundary); ``charges[b]`` is an int32 ``[k_b, nq]`` array; ``conj[b]`` maps
    each channel to its transpose partner; ``phys`` holds the site charges.
    """
    W: list
    channels: list
    charges: list
    conj: list
    phys: np.ndarray
    op_charge: dict = field(default_factory=dict)

    @property
    def n_sites(self):
        return len(self.W)

    def bond_dim(self, b):
        return len(self.channels[b])

    def start_index(self, b):
        return self.channels[b].index(("start",))

    def done_index(self, b):
        return self.channels[b].index(("done",))


def spin_ops():
    """Spin-1/2 operators on the basis (up, down) and their 2Sz charge change."""
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    sm = sp.T.copy()
    sz = np.diag([0.5, -0.5])
    ops = {"Id": (np.eye(2), (0,)), "Sp": (sp, (2,)), "Sm": (sm, (-2,)), "Sz": (sz, (0,))}
    transpose = {"Sp": "Sm", "Sm": "Sp", "Sz": "Sz"}
    return ops, transpose


def electron_ops():
    """Hubbard site operators on |0>, |up>, |dn>, |up dn> = c+_up c+_dn |0>.

    ``adag_dn`` carries the sign from passing the up mode of the same site.
    ``F`` is the site parity used for Jordan-Wigner strings.  Returns the
    local creation/annihilation operators dressed for hopping terms:
    ``adagF_s = a+_s F`` opens a ``c+_i c_j`` term and ``Fa_s = F a_s`` opens
    its Hermitian conjugate; ``a_s`` and ``adag_s`` close them.
    """
    adag_up = np.zeros((4, 4))
    adag_up[1, 0] = 1.0
    adag_up[3, 2] = 1.0
    adag_dn = np.zeros((4, 4))
    adag_dn[2, 0] = 1.0
    adag_dn[3, 1] = -1.0
    F = np.diag([1.0, -1.0, -1.0, 1.0])
    nn = np.diag([0.0, 0.0, 0.0, 1.0])
    ops = {
        "Id": (np.eye(4), (0, 0)),
        "F": (F, (0, 0)),
        "NN": (nn, (0, 0)),
        "adagF_up": (adag_up @ F, (1, 1)),
        "Fa_up": (F @ adag_up.T, (-1, -1)),
        "adagF_dn": (adag_dn @ F, (1, -1)),
        "Fa_dn": (F @ adag_dn.T, (-1, 1)),
        "a_up": (adag_up.T.copy(), (-1, -1)),
        "adag_up": (adag_up, (1, 1)),
        "a_dn": (adag_dn.T.copy(), (-1, 1)),
        "adag_dn": (adag_dn, (1, -1)),
    }
    transpose = {"adagF_up": "Fa_up", "Fa_up": "adagF_up",
                 "adagF_dn": "Fa_dn", "Fa_dn": "adagF_dn"}
    return ops, transpose


def pair_term_mpo(n_sites, phys, ops, transpose, terms, onsite, string_op="Id"):
    """FSA MPO for ``sum_terms c * A_i S.. S B_j + sum_onsite c * O_i``.

    ``terms``: list of ``(i, j, c, A, B)`` with ``i < j``; ``onsite``: list of
    ``(i, c, O)``; ``string_op`` is placed on every site strictly between i
    and j.  Operators are names in ``ops`` (``name -> (matrix, charge)``).
    """
    d = phys.shape[0]
    nq = phys.shape[1]
    ident = ops["Id"][0]
    string = ops[string_op][0]
    # open channels at bond b (after site b-1, i.e. between sites b-1 and b)
    open_at = [set() for _ in range(n_sites + 1)]
    for (i, j, c, A, B) in terms:
        if not (0 <= i < j < n_sites):
            raise ValueError("term sites out of order")
        for b in range(i + 1, j + 1):
            open_at[b].add((i, A))
    channels = []
    for b in range(n_sites + 1):
        ch = []
        if b < n_sites:
            ch.append(("start",))
        for (i, A) in sorted(open_at[b], key=lambda t: (t[0], t[1])):
            ch.append(("open", i, A))
        if b > 0:
            ch.append(("done",))
        channels.append(ch)
    charges = []
    conj = []
    for b in range(n_sites + 1):
        qb = np.zeros((len(channels[b]), nq), dtype=np.int32)
        cb = []
        for w, lab in enumerate(channels[b]):
            if lab[0] == "open":
                qb[w] = ops[lab[2]][1]
                partner = ("open", lab[1], transpose[lab[2]])
                cb.append(channels[b].index(partner) if partner in channels[b] else -1)
            else:
                cb.append(w)
        charges.append(qb)
        conj.append(np.array(cb, dtype=np.int32))
    W = []
    for n in range(n_sites):
        cl, cr = channels[n], channels[n + 1]
        Wn = np.zeros((len(cl), d, d, len(cr)))
        idx_l = {lab: w for w, lab in enumerate(cl)}
        idx_r = {lab: w for w, lab in enumerate(cr)}
        if ("start",) in idx_l and ("start",) in idx_r:
            Wn[idx_l[("start",)], :, :, idx_r[("start",)]] += ident
        if ("done",) in idx_l and ("done",) in idx_r:
            Wn[idx_l[("done",)], :, :, idx_r[("done",)]] += ident
        if ("start",) in idx_l and ("done",) in idx_r:
            for (i, c, O) in onsite:
                if i == n:
                    Wn[idx_l[("start",)], :, :, idx_r[("done",)]] += c * ops[O][0]
        for lab in cr:
            if lab[0] == "open" and lab[1] == n and ("start",) in idx_l:
                Wn[idx_l[("start",)], :, :, idx_r[lab]] += ops[lab[2]][0]
        for lab in cl:
            if lab[0] == "open":
                if lab in idx_r:
                    Wn[idx_l[lab], :, :, idx_r[lab]] += string
        for (i, j, c, A, B) in terms:
            if j == n:
                Wn[idx_l[("open", i, A)], :, :, idx_r[("done",)]] += c * ops[B][0]
        W.append(Wn)
    op_charge = {name: val[1] for name, val in ops.items()}
    return MPO(W=W, channels=channels, charges=charges, conj=conj, phys=phys,
               op_charge=op_charge)


def heisenberg_pairs(pairs):
    """Expand weighted site pairs ``(i, j, J)`` into S.S product terms."""
    terms = []
    for (i, j, J) in pairs:
        a, b = (i, j) if i < j else (j, i)
        terms.append((a, b, 0.5 * J, "Sp", "Sm"))
        terms.append((a, b, 0.5 * J, "Sm", "Sp"))
        terms.append((a, b, J, "Sz", "Sz"))
    return terms


def chain_pairs(n_sites, couplings, periodic=False):
    """Pairs ``(i, i+r, J_r)`` for ``couplings = [J_1, J_2, ...]``."""
    pairs = []
    for r, J in enumerate(couplings, start=1):
        for i in range(n_sites):
            j = i + r
            if j >= n_sites:
                if not periodic:
                    continue
                j -= n_sites
            if J != 0.0 and i != j:
                pairs.append((min(i, j), max(i, j), J))
    return pairs


def snake_index(x, y, Ly):
    """Snake ordering of an Lx x Ly cylinder: columns alternate direction."""
    return x * Ly + (y if x % 2 == 0 else Ly - 1 - y)


def cylinder_pairs(Lx, Ly, J1, J2=0.0):
    """J1 (nearest) and J2 (diagonal) bonds of a square cylinder.

    Open in x, periodic in y, snake-ordered; duplicate pairs (Ly <= 2) are
    merged into one pair carrying the summed coupling.
    """
    acc = {}

    def add(p, q, J):
        if J == 0.0 or p == q:
            return
        key = (min(p, q), max(p, q))
        acc[key] = acc.get(key, 0.0) + J

    seen = set()
    for x in range(Lx):
        for y in range(Ly):
            s = snake_index(x, y, Ly)
            nbrs = []
            if Ly > 1:
                nbrs.append(("J1", x, (y + 1) % Ly))
            if x + 1 < Lx:
                nbrs.append(("J1", x + 1, y))
                if Ly > 1:
                    nbrs.append(("J2", x + 1, (y + 1) % Ly))
                    nbrs.append(("J2", x + 1, (y - 1) % Ly))
            for kind, xx, yy in nbrs:
                t = snake_index(xx, yy, Ly)
                geo = (kind, min((x, y), (xx, yy)), max((x, y), (xx, yy)))
                if geo in seen:
                    continue
                seen.add(geo)
                add(s, t, J1 if kind == "J1" else J2)
    return [(p, q, J) for (p, q), J in sorted(acc.items())]


def cylinder_hops(Lx, Ly, t=1.0):
    """Nearest-neighbour hops ``(i, j, t)`` of a snake-ordered square cylinder (open in x,
    periodic in y), for the Hubbard MPO."""
    return cylinder_pairs(Lx, Ly, t, 0.0)


def triangular_hops(Lx, Ly, t=1.0):
    """Nearest-neighbour hops ``(i, j, t)`` of a triangular lattice on a snake-ordered
    cylinder (open in x, periodic in y): the square-grid bonds along x and y plus the
    (1, 1) diagonal, six neighbours per bulk site.  Duplicate pairs (Ly <= 2) are merged."""
    acc = {}

    def add(p, q):
        if p == q:
            return
        key = (min(p, q), max(p, q))
        acc[key] = acc.get(key, 0.0) + t

    seen = set()
    for x in range(Lx):
        for y in range(Ly):
            nbrs = []
            if Ly > 1:
                nbrs.append((x, (y + 1) % Ly))
            if x + 1 < Lx:
                nbrs.append((x + 1, y))
                if Ly > 1:
                    nbrs.append((x + 1, (y + 1) % Ly))
            for xx, yy in nbrs:
                geo = (min((x, y), (xx, yy)), max((x, y), (xx, yy)))
                if geo in seen:
                    continue
                seen.add(geo)
                add(snake_index(x, y, Ly), snake_index(xx, yy, Ly))
    return [(p, q, v) for (p, q), v in sorted(acc.items())]


def heisenberg_mpo(n_sites, pairs, field_z=0.0):
    """Heisenberg MPO for weighted pairs (optionally a uniform Sz field)."""
    from .sectors import spin_phys
    ops, tr = spin_ops()
    onsite = [(i, field_z, "Sz") for i in range(n_sites)] if field_z else []
    return pair_term_mpo(n_sites, spin_phys(), ops, tr, heisenberg_pairs(pairs), onsite)


def hubbard_mpo(n_sites, hops, U):
    """Hubbard MPO: -t (c+_i c_j + h.c.) per hop ``(i, j, t)`` and U n_up n_dn."""
    from .sectors import electron_phys
    ops, tr = electron_ops()
    terms = []
    for (i, j, t) in hops:
        a, b = (i, j) if i < j else (j, i)
        for s in ("up", "dn"):
            terms.append((a, b, -t, "adagF_" + s, "a_" + s))
            terms.append((a, b, -t, "Fa_" + s, "adag_" + s))
    onsite = [(i, U, "NN") for i in range(n_sites)] if U != 0.0 else []
    return pair_term_mpo(n_sites, electron_phys(), ops, tr, terms, onsite, string_op="F")


def bulk_window(mpo, site):
    """The two site tensors at ``site``, ``site+1`` and their three bonds."""
    return {
        "W1": mpo.W[site], "W2": mpo.W[site + 1],
        "ql": mpo.charges[site], "qm": mpo.charges[site + 1], "qr": mpo.charges[site + 2],
        "conj_l": mpo.conj[site], "conj_m": mpo.conj[site + 1], "conj_r": mpo.conj[site + 2],
        "start_l": mpo.start_index(site), "done_r": mpo.done_index(site + 2),
        "labels_l": mpo.channels[site], "labels_m": mpo.channels[site + 1],
        "labels_r": mpo.channels[site + 2],
    }
