"""Row-band partition of one large texture over ranks, one GPU each.

Every texel of a layer is edited from its own atlas entry (position, triangle) and the stroke
(Section 4.3.1), so a texture splits into bands of rows with no exchange during an edit: each rank
builds a band atlas (lcl_atlas_bind_band + lcl_atlas_build: the same rows as the whole atlas),
holds the same rows of every layer, receives every stroke and lasso (a few bytes each, the same on
every rank) and renders the depth maps whole.  Overlays are per texel.  Per-label texel counts and
areas are sums over texels, so each rank's tables cover its rows and one all-reduce (SUM) of the
integer tables gives the whole texture's, exactly.

This module holds the host logic of that partition; the per-texel work runs in liblcl.so."""
from __future__ import annotations


def band_rows(height: int, tile: int, world: int, rank: int):
    """Rows [y0, y1) of rank `rank` of `world`: the texture's tile rows dealt out as evenly as
    possible (the first height_in_tiles % world ranks take one more), so bands start on tile
    boundaries and every band but the last is a whole number of tiles.  Raises ValueError if
    there are fewer tile rows than ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    tiles_y = -(-height // tile)
    if tiles_y < world:
        raise ValueError(f"{tiles_y} tile rows cannot be split over {world} ranks")
    per, extra = divmod(tiles_y, world)
    first = rank * per + min(rank, extra)
    count = per + (1 if rank < extra else 0)
    return first * tile, min(height, (first + count) * tile)


def reduce_tables(tables, group=None):
    """Sums per-label tables over the ranks in place (torch.distributed all-reduce, SUM).  The
    tables are int64 tensors holding uint64 sums: two's-complement addition is addition modulo
    2^64, so the bits of the result are the uint64 sums.  No-op with a single rank."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return tables
    for t in tables:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tables
