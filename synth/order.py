"""Pixel numberings of a grid graph.

The solver accepts any numbering of the pixels; the numbering decides how many stencil
neighbours of a pixel fall in the same run of consecutive pixels (a tile of the GPU kernels).
A row-major latitude-longitude image puts the north and south neighbours a whole image row
away.  ``blocked_order`` walks the image in bh x bw blocks (block rows top to bottom, blocks
left to right, pixels row-major inside a block), so that only the pixels on a block's border
have neighbours outside it, as HEALPix's hierarchical NESTED numbering does (App. A).

A relabelled problem is the same problem: with P the permutation matrix, L -> P L P^T and
every map -> its columns permuted, so the posterior mean is permuted the same way.
"""

from dataclasses import replace

import numpy as np

from .grids import GridGraph, _csr_from_neighbours


def blocked_order(H: int, W: int, bh: int = 16, bw: int = 16) -> np.ndarray:
    """perm with perm[i_new] = i_old (row-major index r * W + c) for bh x bw blocks."""
    if H % bh or W % bw:
        raise ValueError(f"{H} x {W} image is not a whole number of {bh} x {bw} blocks")
    br, bc, r, c = np.meshgrid(np.arange(H // bh), np.arange(W // bw), np.arange(bh),
                               np.arange(bw), indexing="ij")
    return ((br * bh + r) * W + (bc * bw + c)).reshape(-1).astype(np.int64)


def inverse(perm: np.ndarray) -> np.ndarray:
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size, dtype=perm.dtype)
    return inv


def permute_graph(g: GridGraph, perm: np.ndarray, tag: str = "blocked") -> GridGraph:
    """The graph with pixel perm[i] renamed i (Laplacian CSR rebuilt, columns sorted)."""
    perm = np.asarray(perm, dtype=np.int64)
    if perm.shape != (g.n,) or not np.array_equal(np.sort(perm), np.arange(g.n)):
        raise ValueError("perm is not a permutation of the pixels")
    inv = inverse(perm)
    old = g.nbr[perm]
    nbr = np.where(old >= 0, inv[np.maximum(old, 0)], -1)
    nbr_w = g.nbr_w[perm]
    rowptr, col, val = _csr_from_neighbours(nbr, nbr_w)
    return GridGraph(f"{g.kind}+{tag}", g.H, g.W, nbr, nbr_w, rowptr, col, val)


def permute_problem(p, perm: np.ndarray, tag: str = "blocked"):
    """The problem with its pixels renumbered (graph, noise maps, observations, true sky)."""
    perm = np.asarray(perm, dtype=np.int64)
    meta = dict(p.meta)
    meta["pixel_order"] = tag
    return replace(p, name=f"{p.name}_{tag}", graph=permute_graph(p.graph, perm, tag),
                   D=np.ascontiguousarray(p.D[:, perm]),
                   Yobs=np.ascontiguousarray(p.Yobs[:, :, perm]),
                   X_true=np.ascontiguousarray(p.X_true[:, perm]), meta=meta)


def outside_tile_fraction(rowptr, col, tile: int = 256) -> float:
    """Share of the off-diagonal Laplacian entries whose column lies outside the row's tile of
    ``tile`` consecutive pixels."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    row = np.repeat(np.arange(rowptr.size - 1, dtype=np.int64), np.diff(rowptr))
    off = col != row
    return float(np.mean((col[off] // tile) != (row[off] // tile)))
