"""Quantum-number block tensors (Section II-D).

An order-r tensor is a list of label tuples ``q^(l)`` and one dense block per
tuple.  Here a tensor index is a list of sectors (charge vector, dimension)
and a flow ``+1/-1``; a block, keyed by its tuple of sector numbers, is
allowed when ``sum_k flow_k * charge_k == target`` (charge conservation, which
Schur's lemma forces on every tensor of a symmetric MPS/MPO).
"""
import itertools
import numpy as np


class Index:
    """One tensor index: ``charges[nsec, nq]`` and ``dims[nsec]``."""

    def __init__(self, charges, dims):
        self.charges = np.asarray(charges, dtype=np.int64).reshape(len(dims), -1)
        self.dims = np.asarray(dims, dtype=np.int64)

    @property
    def nsec(self):
        return len(self.dims)

    @property
    def total(self):
        return int(self.dims.sum())

    def offsets(self):
        return np.concatenate([[0], np.cumsum(self.dims)[:-1]]).astype(np.int64)

    def find(self, q):
        """Sector number with charge ``q`` or -1."""
        q = np.asarray(q)
        hits = np.where((self.charges == q).all(axis=1))[0]
        return int(hits[0]) if len(hits) else -1


def allowed_keys(indices, flows, target):
    """All sector tuples obeying the charge rule, in lexicographic order."""
    target = np.asarray(target)
    out = []
    for key in itertools.product(*[range(ix.nsec) for ix in indices]):
        tot = sum(f * ix.charges[k] for f, ix, k in zip(flows, indices, key))
        if np.array_equal(tot, target):
            out.append(key)
    return out


class BlockTensor:
    """Dictionary of dense blocks keyed by sector tuple."""

    def __init__(self, indices, flows, target=None, blocks=None):
        self.indices = list(indices)
        self.flows = tuple(flows)
        nq = self.indices[0].charges.shape[1]
        self.target = np.zeros(nq, dtype=np.int64) if target is None else np.asarray(target)
        self.blocks = {} if blocks is None else dict(blocks)

    def keys(self):
        return allowed_keys(self.indices, self.flows, self.target)

    def shape(self, key):
        return tuple(int(ix.dims[k]) for ix, k in zip(self.indices, key))

    def copy(self):
        return BlockTensor(self.indices, self.flows, self.target,
                           {k: v.copy() for k, v in self.blocks.items()})

    @classmethod
    def from_fill(cls, indices, flows, target, fill):
        """Allocate every allowed block and fill it with ``fill(key)``."""
        t = cls(indices, flows, target)
        for key in t.keys():
            t.blocks[key] = np.asarray(fill(key), dtype=np.float64).reshape(t.shape(key))
        return t

    @classmethod
    def zeros(cls, indices, flows, target=None):
        t = cls(indices, flows, target)
        for key in t.keys():
            t.blocks[key] = np.zeros(t.shape(key))
        return t

    def to_dense(self):
        """Embed every block at its sector offsets (zeros elsewhere)."""
        dense = np.zeros([ix.total for ix in self.indices])
        offs = [ix.offsets() for ix in self.indices]
        for key, blk in self.blocks.items():
            sl = tuple(slice(int(o[k]), int(o[k]) + int(ix.dims[k]))
                       for o, ix, k in zip(offs, self.indices, key))
            dense[sl] = blk
        return dense

    @classmethod
    def from_dense(cls, indices, flows, target, dense):
        t = cls(indices, flows, target)
        offs = [ix.offsets() for ix in t.indices]
        for key in t.keys():
            sl = tuple(slice(int(o[k]), int(o[k]) + int(ix.dims[k]))
                       for o, ix, k in zip(offs, t.indices, key))
            t.blocks[key] = np.array(dense[sl])
        return t

    def vdot(self, other):
        return float(sum(np.vdot(v, other.blocks[k]) for k, v in self.blocks.items()
                         if k in other.blocks))

    def norm(self):
        return float(np.sqrt(sum(float(np.vdot(v, v)) for v in self.blocks.values())))

    def axpy(self, a, other):
        """self += a * other (blocks of other must be blocks of self)."""
        for k, v in other.blocks.items():
            self.blocks[k] = self.blocks[k] + a * v
        return self

    def scale(self, a):
        for k in self.blocks:
            self.blocks[k] = a * self.blocks[k]
        return self

    def flat(self):
        keys = sorted(self.blocks)
        return np.concatenate([self.blocks[k].reshape(-1) for k in keys]) if keys else np.zeros(0)

    def set_flat(self, v):
        keys = sorted(self.blocks)
        o = 0
        for k in keys:
            n = self.blocks[k].size
            self.blocks[k] = v[o:o + n].reshape(self.blocks[k].shape).copy()
            o += n
        return self
