"""The IVF index split by inverted lists over the ranks of a process group.

Every rank holds one shard (``dade_index_subset``: the lists dealt to it by
``dade_shard_lists``, plus the replicated mean, basis, eps table and
centroids), runs the whole query batch on it (rotation, probe of the global
lists, DADE scan of the probed lists it holds, Section 3.4), and the ranks
exchange their [nq, K] results in one all-gather; ``dade_merge_shards`` then
keeps the K nearest.  A shard's threshold is the K-th distance among its own
lists, never below the unsharded search's threshold at the same point of the
scan, so a shard prunes no more than the unsharded search would: every
position of the merged result is at least as near as the unsharded one's,
and in FD mode the two are equal.

The exchange is the only collective: one all-gather of nq x K x 12 bytes per
rank (ids and distances), NCCL for CUDA tensors (plain peer copies; no
multicast), gloo for CPU tensors.
"""
from __future__ import annotations

from . import dade


def gather_results(ids, dists, group=None):
    """All-gather every rank's [nq, K] ids and distances into [G, nq, K] in
    rank order (the layout dade_merge_shards reads)."""
    import torch
    import torch.distributed as dist

    g = dist.get_world_size(group)
    ids, dists = ids.contiguous(), dists.contiguous()
    if dist.get_backend(group) == "nccl":
        gi = ids.new_empty((g,) + tuple(ids.shape))
        gd = dists.new_empty((g,) + tuple(dists.shape))
        dist.all_gather_into_tensor(gi, ids, group=group)
        dist.all_gather_into_tensor(gd, dists, group=group)
        return gi, gd
    li = [torch.empty_like(ids) for _ in range(g)]
    ld = [torch.empty_like(dists) for _ in range(g)]
    dist.all_gather(li, ids, group=group)
    dist.all_gather(ld, dists, group=group)
    return torch.stack(li), torch.stack(ld)


class ShardedIndex:
    """This rank's shard of a full index and the sharded query step.

    ``index``: the full index (built or loaded on this rank's GPU; it may be
    closed once the shard exists).  ``owner``: the list partition, by default
    ``dade_shard_lists`` over the list sizes, which every rank computes alike.
    """

    def __init__(self, index, rank: int, world: int, owner=None):
        self.rank, self.world = int(rank), int(world)
        self.owner = dade.shard_lists(index.list_sizes(), self.world) if owner is None else owner
        self.local = index.subset(self.owner, self.rank)

    def query(self, q, k, nprobe, alpha, delta_d, ids, dists, group=None, **opts):
        """The sharded step: this rank's search of the whole batch q (device
        [nq, D]), the all-gather, and the merge into ids / dists (device
        [nq, k]).  Options as for Index.query."""
        import torch

        nq = q.shape[0]
        li = torch.empty(nq, k, dtype=torch.int64, device=q.device)
        ld = torch.empty(nq, k, dtype=torch.float32, device=q.device)
        self.local.query(q, k, nprobe, alpha, delta_d, li, ld, **opts)
        gi, gd = gather_results(li, ld, group)
        dade.merge_shards(gi, gd, ids, dists)
        return ids, dists

    def close(self):
        self.local.close()
