"""Splitting one frame across ranks by rows of 16x16 tiles.

Every pixel of a CrowdSplat frame depends only on the splats whose support
box contains it, so a frame shards by image rows with no exchange before the
final gather: rank k renders the tile rows it owns (cull, projection, binning
and compositing restricted to its rows) and one gather assembles the image.
Rows are dealt out in whole tiles so no tile straddles two ranks.
"""
from __future__ import annotations

from dataclasses import replace


def row_ranges(height: int, world: int, tile: int = 16):
    """[(row0, row1)] per rank: contiguous pixel rows, whole tiles, sizes
    differing by at most one tile row."""
    if world < 1 or height < 1:
        raise ValueError("height and world must be >= 1")
    tiles = (height + tile - 1) // tile
    base, extra = divmod(tiles, world)
    out, t = [], 0
    for k in range(world):
        n = base + (1 if k < extra else 0)
        r0, r1 = min(height, t * tile), min(height, (t + n) * tile)
        out.append((r0, r1))
        t += n
    return out


def sub_camera(cam, row0: int, row1: int):
    """Camera that renders rows [row0, row1) of `cam`'s image: same pose and
    focal lengths, principal point moved up by row0, height row1 - row0.
    Pixel centres of the sub-image coincide with those rows of the full one
    (values agree up to FP32 rounding of the shifted principal point)."""
    if not (0 <= row0 < row1 <= cam.height):
        raise ValueError("row range outside the image")
    return replace(cam, cy=cam.cy - row0, height=row1 - row0)
