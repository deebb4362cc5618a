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


def sub_camera(cam, row0: int, row1: int, tile: int = 16):
    """Camera that renders rows [row0, row1) of `cam`'s image as a window of
    the full image: same pose, focal lengths and principal point, the full
    image's size and field of view (the EWA clamp depends on it), and pixel
    centres at their full-image positions.  With row0 on the tile grid the
    window's pixels are bit for bit the full frame's rows."""
    if not (0 <= row0 < row1 <= cam.height):
        raise ValueError("row range outside the image")
    if row0 % tile:
        raise ValueError(f"row0 must be a multiple of the tile size {tile}")
    return replace(cam, height=row1 - row0, win_x0=0, win_y0=row0, full_width=cam.width, full_height=cam.height)
