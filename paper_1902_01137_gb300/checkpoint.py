"""Checkpoint and resume of long runs.

A long estimate is traced as a sequence of segments. Segment k is one
call (camera, flux or batch) with its own seed, derived from the run's
seed and k (counter-based random numbers: a segment's paths depend on
nothing else). Its FP64 sums (Sum x, Sum x^2, path count per tally entry)
are added on the host in segment order, so a run stopped after any segment
and resumed from its checkpoint ends with exactly the sums of an
uninterrupted run.

A checkpoint holds the run's seed, the next segment index and the
accumulated sums. With a learned proposal it also holds the network's
parameters and its Adam state (moments and step count). Files are written
to a temporary name and renamed into place, so a crash while saving leaves
the previous checkpoint intact.
"""
from __future__ import annotations

import os

import numpy as np

_SEGMENT_STRIDE = 0xD1B54A32D192ED03   # odd 64-bit constant spacing segment seeds


def segment_seed(seed: int, k: int) -> int:
    """Seed of segment k of a run with seed `seed`."""
    return (seed + (k + 1) * _SEGMENT_STRIDE) % (1 << 64)


class Accumulator:
    """FP64 sums of a segmented run (shape of one tally: entries x quantities)."""

    def __init__(self, shape, seed: int):
        self.seed = int(seed)
        self.next_segment = 0
        self.s1 = np.zeros(shape, dtype=np.float64)
        self.s2 = np.zeros(shape, dtype=np.float64)
        self.n = np.zeros(shape, dtype=np.float64)

    def add(self, s1, s2, n):
        """Add one segment's sums (in segment order) and advance."""
        self.s1 += np.asarray(s1, dtype=np.float64).reshape(self.s1.shape)
        self.s2 += np.asarray(s2, dtype=np.float64).reshape(self.s2.shape)
        self.n += np.broadcast_to(np.asarray(n, dtype=np.float64), self.n.shape)
        self.next_segment += 1

    def next_seed(self) -> int:
        return segment_seed(self.seed, self.next_segment)

    def mean_se(self):
        with np.errstate(invalid="ignore", divide="ignore"):
            m = self.s1 / self.n
            var = np.maximum(self.s2 / self.n - m * m, 0.0)
            se = np.where(self.n > 1, np.sqrt(var / np.maximum(self.n - 1, 1)), 0.0)
        return m, se

    def save(self, path: str, proposal=None):
        """Write the checkpoint (atomically: temporary file, then rename)."""
        state = {"seed": np.uint64(self.seed), "next_segment": np.int64(self.next_segment),
                 "s1": self.s1, "s2": self.s2, "n": self.n}
        if proposal is not None:
            mm, vv, st = proposal.adam_state
            state.update(params=proposal.params, adam_m=mm, adam_v=vv, adam_step=np.int64(st))
        tmp = path + ".tmp"
        with open(tmp, "wb") as f:
            np.savez(f, **state)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)

    @classmethod
    def load(cls, path: str, proposal=None) -> "Accumulator":
        """Read a checkpoint; with `proposal`, restore the network and its Adam state."""
        z = np.load(path)
        acc = cls(z["s1"].shape, int(z["seed"]))
        acc.next_segment = int(z["next_segment"])
        acc.s1[...] = z["s1"]
        acc.s2[...] = z["s2"]
        acc.n[...] = z["n"]
        if proposal is not None:
            if "params" not in z:
                raise ValueError("checkpoint holds no proposal state")
            proposal.params = z["params"]
            proposal.adam_state = (z["adam_m"], z["adam_v"], int(z["adam_step"]))
        return acc
