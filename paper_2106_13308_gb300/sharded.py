"""Sampling parallelism over GPUs (Sec. 4, "Sampling Parallelization"): one
process per GPU, each holding a replica of the model, draws its shard of every
iteration's batch; one all-reduce of the shard sums per iteration gives every
replica the same global-baseline gradient and the same Adam step.

Rank r of L draws B_local samples as global samples r B_local ..
(r + 1) B_local - 1 of the batch (its context's sample offset), so the union of
the shards is exactly the batch of B_tot = L B_local samples that one context
would draw.  Per iteration:

  1. ``shard_sums``: the shard's samples, local energies, and
     S1 = sum (E_b - c) g_b, S0 = sum g_b (float32, 2d values) with the FP64
     scalars {sum (E_b - c), sum (E_b - c)^2, B} (c: the shift);
  2. all-reduce (sum) of both buffers over the ranks;
  3. ``shard_apply``: gradient (S1 - (Ebar - c) S0) / B_tot, Adam.

The shift c must be the same on every rank.  It is the global mean energy of
the iteration two before (0 for the first two iterations): that iteration's
statistics are read back behind an event recorded when they were written, so
the host never waits on the iteration that is still running, and every rank
reads the same reduced value.

The collective is whatever torch.distributed provides for the tensors' device
(NCCL for CUDA tensors, gloo for CPU tensors); this module only sequences the
calls.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


class ShardedRun:
    """Drives `model` (a vqmc.VQMC, or any object with set_sample_offset /
    shard_sums / shard_apply) as one shard of a data-parallel run."""

    def __init__(self, model, batch_local: int, group=None):
        self.model = model
        self.B = int(batch_local)
        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        model.set_sample_offset(self.rank * self.B)
        self.shift = 0.0
        self._pending = []  # (event or None, stats tensor) of the last iterations, oldest first

    @property
    def batch_total(self) -> int:
        return self.B * self.world

    def _reduce(self, t):
        if self.world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def step(self):
        """One data-parallel iteration; returns the FP64 {mean, var} tensor of
        the whole batch (on the model's device, not yet synchronised)."""
        if len(self._pending) >= 2:
            ev, st = self._pending.pop(0)
            if ev is not None:
                ev.synchronize()
            self.shift = float(st[0])
        sums, scal = self.model.shard_sums(self.B, self.shift)
        self._reduce(sums)
        self._reduce(scal)
        _, stats = self.model.shard_apply(sums, scal, self.shift)
        if stats.is_cuda:
            # a copy to pinned memory and an event behind it: reading it two
            # iterations later waits for this iteration only
            host = torch.empty(stats.shape, dtype=stats.dtype, pin_memory=True)
            host.copy_(stats, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream())
            self._pending.append((ev, host))
        else:
            self._pending.append((None, stats))
        return stats
