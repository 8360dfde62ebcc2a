"""Split frame: one level-of-detail frame shared by the GPUs of a node.

Every rank holds a replica of the octree.  The frame's node selection is computed in full on every
rank (it is cheap and deterministic); rank k draws only the selected nodes whose index in the node
table is congruent to k modulo the number of ranks (gblod_render_part), into a partial 64-bit
fixed-point image.  The partial images are summed by one int64 sum-reduce (the only exchange of
the path: height x width x 8 bytes, 16.6 MB at 1920 x 1080), which is exact and order-free because
the accumulation is an integer sum whose total fits in 64 bits, and the sum is tone-mapped once.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def part_of(node_index: int, n_parts: int) -> int:
    """The part (rank) that draws a selected node."""
    return int(node_index) % int(n_parts)


def reduce_partials(acc: torch.Tensor, group=None) -> torch.Tensor:
    """In-place exact sum of every rank's int64 partial image (two's-complement int64 addition is
    uint64 addition, so the reinterpreted sum is the 64-bit image)."""
    assert acc.dtype == torch.int64
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    return acc


def render_split(renderer, octree, cam: dict, params=None, rank: int = 0, world: int = 1, group=None,
                 image: bool = True, stream=None):
    """Renders part `rank` of `world`, sums the parts over the group and tone-maps the sum on every
    rank.  Returns (uint8 image or None, int64 accumulation image of the whole frame)."""
    acc = renderer.render_part(octree, cam, rank, world, params, stream=stream)
    reduce_partials(acc, group)
    img = renderer.tonemap(acc, params, stream=stream) if image else None
    return img, acc
