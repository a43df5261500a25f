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


def compress_mpo(mpo, cutoff=1e-13, method="svd"):
    """SVD compression of an MPO's channels (Section VI-B: the electron MPO is compressed with
    an SVD cutoff of 1e-13).

    ``method="interpolative"`` gives the same channel counts but keeps a subset of the
    original channels instead of rotating to singular vectors: in each pass the rank-revealing
    (column-pivoted) QR of a sector's vectors picks the independent channels (the pivots whose
    |R_ii| exceed the cutoff times the bond's largest), the others are written as combinations
    of them, and only the neighbouring site's tensor absorbs those combinations.  The kept
    channels' own rows (or columns) stay the automaton's sparse operators, so W stays far
    sparser than in the SVD basis.

    The ``start`` and ``done`` channels are kept as they are; the other channels of every
    bond are replaced by a minimal set of linear combinations, charge sector by charge sector
    (channels of one sector share their charge, so the charge rule of every entry is kept).
    Pass 1 (left to right) makes the left operators of every bond independent: at site n the
    columns of W[n] that belong to one sector, as vectors over (wl, t, s), are decomposed as
    U S V^T; the singular values above ``cutoff`` times the bond's largest are kept, W[n]
    takes U's columns and S V^T is carried into the rows of W[n+1].  Pass 2 (right to left)
    does the same with the rows of W[n] as vectors over (t, s, wr), making the right operators
    independent; W[n] takes V^T's rows and U S goes into the columns of W[n-1].  Each pass
    multiplies the other side's operators by a matrix of full column rank, so independence
    won in pass 1 survives pass 2, and the channel count of every bond ends at the rank of
    the operator Schmidt decomposition of H across it.

    Hermitian structure: the MPO obeys W[conj wl, s, t, conj wr] = W[wl, t, s, wr] with the
    channel map ``conj`` (operator A <-> its transpose).  The factors of a sector q are
    computed once and applied to the sector -q through the partner channels, so the new
    channel j of sector q and channel j of sector -q are transposition partners (channels of
    charge 0 must be their own partners).  Returns a new ``MPO`` with channel labels
    ``("start",)``, ``("c", charge, j)``, ``("done",)``.
    """
    N = len(mpo.W)
    W = [np.array(w, dtype=np.float64, copy=True) for w in mpo.W]
    nq = mpo.charges[0].shape[1]
    d = mpo.phys.shape[0]
    special = [{w for w, lab in enumerate(mpo.channels[b]) if lab in (("start",), ("done",))}
               for b in range(N + 1)]
    # per bond: ordered list of (charge, [channel indices]) for the non-special channels, the
    # charge-conjugation partner of every channel, and the special channels' indices
    chan = [list(range(len(mpo.channels[b]))) for b in range(N + 1)]
    q_of = [np.array(mpo.charges[b], dtype=np.int64) for b in range(N + 1)]
    conj = [np.array(mpo.conj[b], dtype=np.int64) for b in range(N + 1)]

    def sectors(b):
        groups = {}
        for w in chan[b]:
            if w in special[b]:
                continue
            groups.setdefault(tuple(int(v) for v in q_of[b][w]), []).append(w)
        return groups

    def plan_bond(b, groups):
        """Canonical sectors (q >= -q) with their partner lists; checks the partner map."""
        out = []
        for q, ws in sorted(groups.items()):
            mq = tuple(-v for v in q)
            if q < mq:
                continue
            partners = [int(conj[b][w]) for w in ws]
            if any(p < 0 for p in partners):
                raise ValueError(f"bond {b}: channel without a transposition partner")
            if q == mq:
                if partners != ws:
                    raise ValueError(f"bond {b}: charge-0 channels must be their own partners")
                out.append((q, ws, None))
            else:
                if sorted(partners) != sorted(groups.get(mq, [])):
                    raise ValueError(f"bond {b}: partners of sector {q} are not sector {mq}")
                out.append((q, ws, partners))
        return out

    def rebuild_bond(b, new_sectors, left_site, right_site, left_cols, right_rows):
        """Replace the channels of bond b: new_sectors = [(q, count)] in order; left_cols[q] /
        right_rows[q]: the new columns of W[b-1] ([k, d, d, count]) and rows of W[b]."""
        keep = sorted(special[b])
        st = [w for w in keep if mpo.channels[b][w] == ("start",)]
        dn = [w for w in keep if mpo.channels[b][w] == ("done",)]
        labels, charges, conjn, cols, rows = [], [], [], [], []
        for w in st:
            labels.append(("start",)); charges.append(q_of[b][w])
            cols.append(W[b - 1][..., w:w + 1] if left_site else None)
            rows.append(W[b][w:w + 1] if right_site else None)
        base = {}
        for q, cnt in new_sectors:
            base[q] = len(labels)
            for j in range(cnt):
                labels.append(("c", q, j)); charges.append(np.array(q, dtype=np.int64))
            cols.append(left_cols[q] if left_site else None)
            rows.append(right_rows[q] if right_site else None)
        for w in dn:
            labels.append(("done",)); charges.append(q_of[b][w])
            cols.append(W[b - 1][..., w:w + 1] if left_site else None)
            rows.append(W[b][w:w + 1] if right_site else None)
        for lab in labels:
            if lab[0] == "c":
                mq = tuple(-v for v in lab[1])
                conjn.append(base[mq] + lab[2])
            else:
                conjn.append(len(conjn))
        if left_site:
            W[b - 1] = np.concatenate(cols, axis=3)
        if right_site:
            W[b] = np.concatenate(rows, axis=0)
        q_of[b] = np.array(charges, dtype=np.int64).reshape(-1, nq)
        conj[b] = np.array(conjn, dtype=np.int64)
        chan[b] = list(range(len(labels)))
        special[b] = {i for i, lab in enumerate(labels) if lab[0] != "c"}
        return labels

    labels = [list(mpo.channels[b]) for b in range(N + 1)]
    if method == "interpolative":
        return _compress_interpolative(mpo, W, special, q_of, conj, sectors, plan_bond, cutoff)
    if method != "svd":
        raise ValueError(f"unknown compression method {method!r}")
    # pass 1: left to right over the bonds 1..N-1 (right bond of site n = b - 1)
    for b in range(1, N):
        n = b - 1
        groups = sectors(b)
        canon = plan_bond(b, groups)
        k_l = W[n].shape[0]
        dec = {}
        for q, ws, partners in canon:
            M = W[n][..., ws].reshape(k_l * d * d, len(ws))
            U, S, Vt = np.linalg.svd(M, full_matrices=False)
            dec[q] = (ws, partners, U, S, Vt)
        smax = max((v[3][0] for v in dec.values() if len(v[3])), default=0.0)
        new_sectors, left_cols, right_rows = [], {}, {}
        for q, (ws, partners, U, S, Vt) in sorted(dec.items()):
            r = int(np.sum(S > cutoff * smax))
            T = S[:r, None] * Vt[:r]                             # new row j = sum_i T[j, i] old row i
            for qq, lst in ((q, ws),) + ((((tuple(-v for v in q)), partners),) if partners is not None else ()):
                M = W[n][..., lst].reshape(k_l * d * d, len(lst))
                # new columns: M T^+ (exact: M = U S V^T, T = S_r V_r^T); for the partner
                # sector the same T applies to the partner channels
                C = M @ (Vt[:r].T / S[:r][None, :])
                left_cols[qq] = C.reshape(k_l, d, d, r)
                right_rows[qq] = np.tensordot(T, W[b][lst], axes=(1, 0))
        order = sorted(set(left_cols))
        new_sectors = [(q, left_cols[q].shape[3]) for q in order]
        labels[b] = rebuild_bond(b, new_sectors, True, True, left_cols, right_rows)
    # pass 2: right to left over the bonds N-1..1 (left bond of site n = b)
    for b in range(N - 1, 0, -1):
        n = b
        groups = sectors(b)
        canon = plan_bond(b, groups)
        k_r = W[n].shape[3]
        dec = {}
        for q, ws, partners in canon:
            M = W[n][ws].reshape(len(ws), d * d * k_r)
            U, S, Vt = np.linalg.svd(M, full_matrices=False)
            dec[q] = (ws, partners, U, S, Vt)
        smax = max((v[3][0] for v in dec.values() if len(v[3])), default=0.0)
        left_cols, right_rows = {}, {}
        for q, (ws, partners, U, S, Vt) in sorted(dec.items()):
            r = int(np.sum(S > cutoff * smax))
            T = U[:, :r] * S[None, :r]                           # old row i = sum_j T[i, j] new row j
            for qq, lst in ((q, ws),) + ((((tuple(-v for v in q)), partners),) if partners is not None else ()):
                M = W[n][lst].reshape(len(lst), d * d * k_r)
                R_new = (U[:, :r].T / S[:r][:, None]) @ M         # T^+ M
                right_rows[qq] = R_new.reshape(r, d, d, k_r)
                left_cols[qq] = np.tensordot(W[b - 1][..., lst], T, axes=(3, 0))
        order = sorted(set(left_cols))
        new_sectors = [(q, left_cols[q].shape[3]) for q in order]
        labels[b] = rebuild_bond(b, new_sectors, True, True, left_cols, right_rows)
    charges = [np.asarray(q_of[b], dtype=np.int32).reshape(-1, nq) for b in range(N + 1)]
    conjs = [np.asarray(conj[b], dtype=np.int32) for b in range(N + 1)]
    # drop round-off below the cutoff's scale so that structurally zero blocks stay zero
    for n in range(N):
        scale = np.abs(W[n]).max()
        W[n][np.abs(W[n]) < 1e-15 * scale] = 0.0
    return MPO(W=W, channels=labels, charges=charges, conj=conjs, phys=mpo.phys, op_charge=dict(mpo.op_charge))


def _pivoted_subset(M, cutoff, scale):
    """Rank-revealing selection on the columns of M: (kept column indices, C) with
    M = M[:, kept] @ C (C[:, kept] = identity up to rounding)."""
    import scipy.linalg as sl
    if M.shape[1] == 0:
        return [], np.zeros((0, 0))
    _, R, piv = sl.qr(M, mode="economic", pivoting=True)
    diag = np.abs(np.diag(R))
    r = int(np.sum(diag > cutoff * scale)) if scale > 0 else 0
    kept = sorted(int(p) for p in piv[:r])
    if r == 0:
        return [], np.zeros((0, M.shape[1]))
    C, *_ = np.linalg.lstsq(M[:, kept], M, rcond=None)
    C[np.abs(C) < 1e-14] = 0.0
    for i, k in enumerate(kept):                      # exact identity on the kept columns
        C[:, k] = 0.0
        C[i, k] = 1.0
    return kept, C


def _compress_interpolative(mpo, W, special, q_of, conj, sectors, plan_bond, cutoff):
    """The two passes of compress_mpo with a subset of the original channels kept."""
    import scipy.linalg as sl
    N = len(W)
    d = mpo.phys.shape[0]
    labels = [list(mpo.channels[b]) for b in range(N + 1)]

    def largest(mats):
        vals = [np.abs(np.diag(sl.qr(M, mode="r", pivoting=True)[0])).max() for M in mats if M.size]
        return max(vals) if vals else 0.0

    def apply(b, choice):
        """choice[q] = (kept channel list, C) for every sector of bond b, including the -q
        partners; rebuild bond b keeping the start / done channels and the kept ones."""
        keep = sorted(special[b] | {w for q, (ks, _) in choice.items() for w in ks})
        pos = {w: i for i, w in enumerate(keep)}
        return keep, pos

    for pass_ in (1, 2):
        bonds = range(1, N) if pass_ == 1 else range(N - 1, 0, -1)
        for b in bonds:
            groups = sectors(b)
            canon = plan_bond(b, groups)
            mats = {}
            for q, ws, partners in canon:
                if pass_ == 1:       # columns of W[b-1] as vectors over (wl, t, s)
                    mats[q] = W[b - 1][..., ws].reshape(-1, len(ws))
                else:                # rows of W[b] as vectors over (t, s, wr): columns of the transpose
                    mats[q] = W[b][ws].reshape(len(ws), -1).T
            scale = largest(mats.values())
            choice = {}
            for q, ws, partners in canon:
                kept_i, C = _pivoted_subset(mats[q], cutoff, scale)
                choice[q] = ([ws[i] for i in kept_i], ws, C)
                if partners is not None:
                    choice[tuple(-v for v in q)] = ([partners[i] for i in kept_i], partners, C)
            # combine: pass 1 moves the dropped columns' weight into the rows of W[b] of the
            # kept channels (new row k = sum_j C[k, j] row j); pass 2 moves the dropped rows'
            # weight into the columns of W[b-1] (new col k = sum_i col i C[k, i])
            for q, (kept, ws, C) in choice.items():
                if pass_ == 1:
                    W[b][kept] = np.tensordot(C, W[b][ws], axes=(1, 0))
                else:
                    W[b - 1][..., kept] = np.tensordot(W[b - 1][..., ws], C.T, axes=(3, 0))
            keep = sorted(special[b] | {w for (kept, _, _) in choice.values() for w in kept})
            W[b - 1] = W[b - 1][..., keep]
            W[b] = W[b][keep]
            old_to_new = {w: i for i, w in enumerate(keep)}
            q_of[b] = q_of[b][keep]
            conj[b] = np.array([old_to_new[int(conj[b][w])] for w in keep], dtype=np.int64)
            labels[b] = [labels[b][w] for w in keep]
            special[b] = {old_to_new[w] for w in special[b]}
    charges = [np.asarray(q_of[b], dtype=np.int32).reshape(-1, mpo.charges[0].shape[1]) for b in range(N + 1)]
    conjs = [np.asarray(conj[b], dtype=np.int32) for b in range(N + 1)]
    for n in range(N):
        scale = np.abs(W[n]).max()
        W[n][np.abs(W[n]) < 1e-15 * scale] = 0.0
    return MPO(W=W, channels=labels, charges=charges, conj=conjs, phys=mpo.phys, op_charge=dict(mpo.op_charge))
