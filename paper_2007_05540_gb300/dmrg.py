"""Two-site DMRG sweeps on the GPU (Section II-C), chained from the library's entry points.

Every numerical step runs in the library's kernels, with the tensors resident in device
memory: per bond (i, i+1) of a sweep

    x0 = A_i . B_{i+1}                        heff_two_site_apply  (Fig. 1d)
    lowest eigenpair of K on the bond          heff_lanczos, or heff_davidson (Algorithm 1)
    x = U S V^T, truncated to m                heff_svd_*           (Fig. 1e, Section II-C)
    A_i <- U, B_{i+1} <- S V^T  (left -> right; mirrored right -> left)
    L_{i+1} from L_i, A_i  or  R_{i+1} from R_{i+2}, B_{i+1}        heff_env_update

The host builds the charge-sector layouts and plans of each bond and keeps the bond
structure (sector charges and dimensions) that the truncation returns.  The sweeps
start from a product state with the requested total charge (all sites then both left-
and right-canonical), so no orthonormalisation of a random state is needed; two-site
updates grow the bonds up to the schedule's m.  Only the matvecs use the plan's
precision; vectors, orthogonalisation, the SVD and the environments are FP64 buffers, and
the environment updates' block products run in FP64 or, with ``env_precision="bf16x3"``, on
the tensor cores (FP32-accumulated, about 1e-5 relative per update).  With a split
precision the energy of the final bond's vector is recomputed with an FP64 apply.
"""
import numpy as np

from . import heff


def _ones(n):
    return np.ones(n, dtype=np.int32)


def product_state(phys, n_sites, total):
    """Site states whose charges add up to ``total``: at every site the state that keeps
    the running charge closest to the straight line from 0 to ``total``."""
    phys = np.asarray(phys)
    total = np.asarray(total, dtype=np.float64)
    cum = np.zeros(phys.shape[1])
    states = []
    for i in range(n_sites):
        target = total * (i + 1) / n_sites
        best = min(range(len(phys)), key=lambda s: (float(np.sum((cum + phys[s] - target) ** 2)), s))
        states.append(best)
        cum = cum + phys[best]
    if not np.array_equal(cum, total):
        raise ValueError(f"no product state reaches total charge {tuple(total)} (got {tuple(cum)})")
    return states


class GpuDMRG:
    """Two-site DMRG for an MPO (``W[n]`` of shape [k_n, d, d, k_{n+1}], ``charges[b]`` the
    channel charges of bond b, ``phys`` the site charges, ``start_index(0)`` and
    ``done_index(N)`` the boundary channels) in the sector of total charge ``total``."""

    def __init__(self, mpo, total, precision="fp64", n_iter=20, cutoff=1e-12, states=None, device="cuda",
                 solver="lanczos", davidson_vecs=2, seed=0, env_precision="fp64"):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.mpo = mpo
        self.N = mpo.n_sites
        self.phys = np.asarray(mpo.phys, dtype=np.int32)
        self.nq = self.phys.shape[1]
        self.total = np.asarray(total, dtype=np.int32).reshape(self.nq)
        self.precision = precision
        self.env_precision = env_precision
        self.n_iter = int(n_iter)
        self.cutoff = float(cutoff)
        if solver not in ("lanczos", "davidson"):
            raise ValueError(f"unknown solver {solver!r}")
        self.solver = solver
        self.davidson_vecs = int(davidson_vecs)
        self.rng = np.random.default_rng(seed)     # the randomisation vectors of Algorithm 1
        self.ch = [np.asarray(q, dtype=np.int32).reshape(-1, self.nq) for q in mpo.charges]
        d = len(self.phys)
        # MPO tensors in their layouts (host copy for the schedules, device copy for compute)
        self.W = []
        for n in range(self.N):
            lay = heff.Layout([(self.ch[n], _ones(len(self.ch[n])), 1), (self.phys, _ones(d), 1),
                               (self.phys, _ones(d), -1), (self.ch[n + 1], _ones(len(self.ch[n + 1])), -1)])
            host = lay.assemble(lambda k, n=n: mpo.W[n][k])
            self.W.append((lay, host, torch.from_numpy(host).to(self.dev)))
        # product state: bond b has one sector (the running charge), every site one block = 1
        states = product_state(self.phys, self.N, self.total) if states is None else list(states)
        q = np.zeros(self.nq, dtype=np.int32)
        self.bonds = [(q.reshape(1, self.nq).copy(), np.ones(1, dtype=np.int32))]
        for s in states:
            q = q + self.phys[s]
            self.bonds.append((q.reshape(1, self.nq).copy(), np.ones(1, dtype=np.int32)))
        self.sites = []
        for n in range(self.N):
            lay = self._site_layout(self.bonds[n], self.bonds[n + 1])
            self.sites.append((lay, torch.ones(lay.nelem, dtype=torch.float64, device=self.dev)))
        # environments: L[0] on the start channel, R[N] on the done channel, R[N-1..2] grown
        self.L = [None] * (self.N + 1)
        self.R = [None] * (self.N + 1)
        self.L[0] = self._boundary(self.bonds[0], 0, mpo.start_index(0))
        self.R[self.N] = self._boundary(self.bonds[self.N], self.N, mpo.done_index(self.N))
        for j in range(self.N - 1, 1, -1):
            self.R[j] = self._extend(self.R[j + 1], self.sites[j], j, "right", self.bonds[j])
        self.energies = []
        self.discarded = []

    # ------------------------------------------------------------------ layouts
    def _site_layout(self, left, right):
        return heff.Layout([(left[0], left[1], 1), (self.phys, _ones(len(self.phys)), 1), (right[0], right[1], -1)])

    def _env_layout(self, bond, b):
        return heff.Layout([(bond[0], bond[1], -1), (self.ch[b], _ones(len(self.ch[b])), 1), (bond[0], bond[1], 1)])

    def _boundary(self, bond, b, channel):
        lay = self._env_layout(bond, b)
        host = lay.assemble(lambda k: np.ones(1) if k[1] == channel else np.zeros(1))
        return lay, self.torch.from_numpy(host).to(self.dev)

    def _extend(self, env, site, n, side, new_bond):
        """Environment grown over site n: side "left" gives L_{n+1} from L_n, "right" gives
        R_n from R_{n+1}; ``new_bond`` is the bond the result lives on."""
        torch = self.torch
        b = n + 1 if side == "left" else n
        new_l = self._env_layout(new_bond, b)
        W_l, W_host, W_dev = self.W[n]
        plan = heff.heff_env_plan_create(env[0].handle, site[0].handle, W_l.handle, new_l.handle, W_host, side)
        try:
            heff.heff_env_plan_set_precision(plan, self.env_precision)
            ws = torch.empty(max(heff.heff_env_workspace_size(plan), 256), dtype=torch.uint8, device=self.dev)
            out = torch.empty(new_l.nelem, dtype=torch.float64, device=self.dev)
            heff.heff_env_update(plan, env[1], site[1], W_dev, out, ws)
        finally:
            heff.heff_env_plan_destroy(plan)
        return new_l, out

    # ------------------------------------------------------------------ one bond
    def bond_step(self, i, m_max, direction):
        """Optimise sites (i, i+1) and move the orthogonality centre in ``direction``
        ("right" or "left").  Returns (energy, discarded weight)."""
        torch = self.torch
        alpha, beta = self.bonds[i], self.bonds[i + 2]
        Ll, W1l, W2l, Rl, xl = heff.heff_layouts(alpha, beta, self.phys, self.ch[i], self.ch[i + 1],
                                                 self.ch[i + 2])
        x0 = torch.empty(xl.nelem, dtype=torch.float64, device=self.dev)
        ts = heff.heff_two_site_create(self.sites[i][0].handle, self.sites[i + 1][0].handle, xl.handle)
        try:
            heff.heff_two_site_apply(ts, self.sites[i][1], self.sites[i + 1][1], x0)
        finally:
            heff.heff_two_site_destroy(ts)
        plan = heff.Plan(Ll, W1l, W2l, Rl, xl, self.W[i][1], self.W[i + 1][1], self.precision, "f64")
        ws = plan.workspace(self.dev)
        x = torch.empty_like(x0)
        Lenv, Renv = self.L[i][1], self.R[i + 2][1]
        if self.solver == "lanczos":
            n_it = max(1, min(self.n_iter, xl.nelem, 126))
            lz = torch.empty(heff.heff_lanczos_workspace_size(plan.handle, n_it), dtype=torch.uint8,
                             device=self.dev)
            res = torch.zeros(3 + 2 * (n_it + 1), dtype=torch.float64, device=self.dev)
            heff.heff_lanczos(plan.handle, Lenv, self.W[i][2], self.W[i + 1][2], Renv, x0, n_it, x, res, ws, lz)
        else:
            nv = max(1, min(self.davidson_vecs, xl.nelem, 64))
            dw = torch.empty(heff.heff_davidson_workspace_size(plan.handle, nv), dtype=torch.uint8, device=self.dev)
            rnd = torch.from_numpy(self.rng.standard_normal(xl.nelem)).to(self.dev)
            res = torch.zeros(3, dtype=torch.float64, device=self.dev)
            heff.heff_davidson(plan.handle, Lenv, self.W[i][2], self.W[i + 1][2], Renv, x0, rnd, nv, 1e-10, x, res,
                               ws, dw)
        energy = float(res[0].item())
        # split and truncate
        s = heff.heff_svd_create(xl.handle)
        try:
            sws = torch.empty(heff.heff_svd_workspace_size(s), dtype=torch.uint8, device=self.dev)
            heff.heff_svd_compute(s, x, sws)
            maxsec = len(alpha[1]) * len(self.phys) + 1
            q, dims, disc, _ = heff.heff_svd_truncate(s, m_max, self.cutoff, self.nq, maxsec)
            new_bond = (np.ascontiguousarray(q, dtype=np.int32), np.ascontiguousarray(dims, dtype=np.int32))
            A_l = self._site_layout(alpha, new_bond)
            B_l = self._site_layout(new_bond, beta)
            A = torch.empty(A_l.nelem, dtype=torch.float64, device=self.dev)
            B = torch.empty(B_l.nelem, dtype=torch.float64, device=self.dev)
            heff.heff_svd_write(s, A_l.handle, B_l.handle, A, B, direction == "right", sws)
        finally:
            heff.heff_svd_destroy(s)
        self.bonds[i + 1] = new_bond
        self.sites[i] = (A_l, A)
        self.sites[i + 1] = (B_l, B)
        if direction == "right":
            self.L[i + 1] = self._extend(self.L[i], self.sites[i], i, "left", new_bond)
        else:
            self.R[i + 1] = self._extend(self.R[i + 2], self.sites[i + 1], i + 1, "right", new_bond)
        self._last = (plan, (Ll, W1l, W2l, Rl, xl), x, i)
        return energy, disc

    def sweep(self, m_max):
        """One full sweep (left to right, then right to left); returns the last energy."""
        e = None
        for i in range(self.N - 1):
            e, disc = self.bond_step(i, m_max, "right")
            self.discarded.append(disc)
        for i in range(self.N - 2, -1, -1):
            e, disc = self.bond_step(i, m_max, "left")
            self.discarded.append(disc)
        self.energies.append(e)
        return e

    def refined_energy(self):
        """<x|K|x>/<x|x> of the last optimised bond's vector with an FP64 apply."""
        torch = self.torch
        _, lays, x, i = self._last
        Ll, W1l, W2l, Rl, xl = lays
        # the environments of that bond are L[i] and R[i+2] as they were when it was solved
        P = heff.Plan(Ll, W1l, W2l, Rl, xl, self.W[i][1], self.W[i + 1][1], "fp64", "f64")
        ws = P.workspace(self.dev)
        y = torch.empty_like(x)
        heff.heff_apply(P.handle, self.L[i][1], self.W[i][2], self.W[i + 1][2], self.R[i + 2][1], x, y, ws)
        return float(torch.dot(x, y) / torch.dot(x, x))

    def bond_dims(self):
        return [int(np.sum(b[1])) for b in self.bonds]


def dmrg(mpo, total, m_schedule, precision="fp64", n_iter=20, cutoff=1e-12, device="cuda", solver="lanczos",
         davidson_vecs=2, states=None, env_precision="fp64"):
    """Run one full sweep per entry of ``m_schedule`` (the bond cap of that sweep); the
    eigensolver is Lanczos (n_iter steps) or Algorithm 1's Davidson (davidson_vecs vectors).
    ``states`` (one local state per site) chooses the product state the sweeps start from.
    Returns dict(sweep_energies, energy, refined_energy, bond_dims, max_discarded)."""
    run = GpuDMRG(mpo, total, precision, n_iter, cutoff, states=states, device=device, solver=solver,
                  davidson_vecs=davidson_vecs, env_precision=env_precision)
    for m in m_schedule:
        run.sweep(int(m))
    out = {"sweep_energies": list(run.energies), "energy": run.energies[-1], "bond_dims": run.bond_dims(),
           "max_discarded": float(max(run.discarded)) if run.discarded else 0.0}
    out["refined_energy"] = run.refined_energy() if precision != "fp64" else out["energy"]
    return out
