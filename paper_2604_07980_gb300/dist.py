"""Host-side sharding of the matching path across ranks (one process per GPU).

Frames are independent units of work, so ranks split them with no data-path
collective: a rank either processes its own batch (weak scaling, the
benchmark's mode, with a per-rank input seed) or a contiguous share of a common
batch (strong scaling).  Only reporting needs communication: the slowest
rank's time, and, when results are wanted in one place, the per-box outputs
gathered in frame order.
"""
from __future__ import annotations

import numpy as np


def rank_seed(base_seed: int, rank: int) -> int:
    """Input seed of a rank's own batch in weak-scaling mode."""
    return int(base_seed) + 7919 * int(rank)


def frame_shard(n_frames: int, world: int, rank: int) -> range:
    """Contiguous frames of `rank` when `n_frames` are split over `world` ranks
    (sizes differ by at most one; the lower ranks take the extra frames)."""
    if world < 1 or not 0 <= rank < world or n_frames < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_frames, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def boxes_of_frames(boxes: np.ndarray, frames: range) -> tuple[np.ndarray, np.ndarray]:
    """Boxes (int32 [n, 5], frame index in column 4) of the given frames,
    renumbered to local frame indices, and their positions in `boxes`."""
    sel = np.nonzero((boxes[:, 4] >= frames.start) & (boxes[:, 4] < frames.stop))[0]
    local = boxes[sel].copy()
    local[:, 4] -= frames.start
    return local, sel


def max_over_ranks(value: float, dist=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    backend = dist.get_backend()
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_outputs(local: dict, positions: np.ndarray, n_total: int, dist) -> dict | None:
    """Assemble per-box outputs of all ranks on rank 0 in global box order."""
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (positions, {k: np.asarray(v) for k, v in local.items()}))
    if dist.get_rank() != 0:
        return None
    out = {}
    for pos, vals in parts:
        for k, v in vals.items():
            if k not in out:
                out[k] = np.zeros((n_total,) + v.shape[1:], dtype=v.dtype)
            out[k][pos] = v
    return out
