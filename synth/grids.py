"""Pixel graphs used as stand-ins for the HEALPix neighbour structure (App. A, App. C).

Two grids are generated:

* ``periodic_lattice(H, W)``: flat H x W lattice, 4 neighbours with wrap-around, unit weights.
* ``latlong_sphere(H, W)``: H latitude rows x W longitude columns.  Row r sits at latitude
  phi_r = -pi/2 + (r + 1/2) pi / H.  East-west edges (periodic in longitude) carry weight
  cos(phi_r); north-south edges between rows r and r+1 carry cos((phi_r + phi_{r+1}) / 2);
  no edge crosses a pole.

Pixel index is ``i = r * W + c``.  The Laplacian of the weighted graph is produced in CSR form
(diagonal included, columns sorted per row) because it is an input the solver library takes
from its caller, exactly like a HEALPix neighbour list would be: row i holds the sum of the
weights of the edges at i on the diagonal and minus the edge weight at each neighbour.
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class GridGraph:
    kind: str            # "lattice" or "sphere"
    H: int
    W: int
    nbr: np.ndarray      # (n, 4) int64 neighbour index (E, W, S, N order), -1 where absent
    nbr_w: np.ndarray    # (n, 4) float64 edge weight, 0 where absent
    rowptr: np.ndarray   # CSR of the graph Laplacian (int32, n + 1)
    col: np.ndarray      # (int32, nnz)
    val: np.ndarray      # (float64, nnz)

    @property
    def n(self) -> int:
        return self.H * self.W

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _csr_from_neighbours(nbr, nbr_w):
    """Laplacian CSR from a padded neighbour table (duplicates are not expected)."""
    n = nbr.shape[0]
    valid = nbr >= 0
    cols = np.concatenate([np.arange(n, dtype=np.int64)[:, None], nbr], axis=1)
    vals = np.concatenate([nbr_w.sum(axis=1, where=valid)[:, None], -nbr_w], axis=1)
    ok = np.concatenate([np.ones((n, 1), dtype=bool), valid], axis=1)
    # absent slots sort last
    key = np.where(ok, cols, np.iinfo(np.int64).max)
    order = np.argsort(key, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vals = np.take_along_axis(vals, order, axis=1)
    ok = np.take_along_axis(ok, order, axis=1)
    counts = ok.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("graph too large for int32 CSR")
    return rowptr.astype(np.int32), cols[ok].astype(np.int32), vals[ok].astype(np.float64)


def laplacian_csr_from_edges(n, u, v, w):
    """CSR (rowptr, col, val) of sum_e w_e (e_u - e_v)(e_u - e_v)^T for a general edge list."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    deg = np.zeros(n, dtype=np.float64)
    np.add.at(deg, u, w)
    np.add.at(deg, v, w)
    rows = np.concatenate([np.arange(n, dtype=np.int64), u, v])
    cols = np.concatenate([np.arange(n, dtype=np.int64), v, u])
    vals = np.concatenate([deg, -w, -w])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    key = rows * n + cols
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    idx = np.cumsum(first) - 1
    mvals = np.zeros(int(first.sum()), dtype=np.float64)
    np.add.at(mvals, idx, vals)
    counts = np.bincount(rows[first], minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(np.int32), cols[first].astype(np.int32), mvals


def periodic_lattice(H: int, W: int) -> GridGraph:
    if H < 3 or W < 3:
        raise ValueError("periodic lattice needs H, W >= 3 (no parallel edges)")
    r = np.repeat(np.arange(H, dtype=np.int64), W)
    c = np.tile(np.arange(W, dtype=np.int64), H)
    nbr = np.stack([r * W + (c + 1) % W,
                    r * W + (c - 1) % W,
                    ((r + 1) % H) * W + c,
                    ((r - 1) % H) * W + c], axis=1)
    nbr_w = np.ones((H * W, 4), dtype=np.float64)
    rowptr, col, val = _csr_from_neighbours(nbr, nbr_w)
    return GridGraph("lattice", H, W, nbr, nbr_w, rowptr, col, val)


def sphere_latitudes(H: int) -> np.ndarray:
    return -np.pi / 2 + (np.arange(H) + 0.5) * np.pi / H


def latlong_sphere(H: int, W: int) -> GridGraph:
    if H < 2 or W < 3:
        raise ValueError("sphere grid needs H >= 2, W >= 3")
    phi = sphere_latitudes(H)
    w_ew = np.cos(phi)                        # per row
    w_ns = np.cos(0.5 * (phi[:-1] + phi[1:]))  # between row r and r + 1
    r = np.repeat(np.arange(H, dtype=np.int64), W)
    c = np.tile(np.arange(W, dtype=np.int64), H)
    has_s = r < H - 1
    has_n = r > 0
    nbr = np.stack([r * W + (c + 1) % W,
                    r * W + (c - 1) % W,
                    np.where(has_s, (r + 1) * W + c, -1),
                    np.where(has_n, (r - 1) * W + c, -1)], axis=1)
    nbr_w = np.stack([w_ew[r], w_ew[r],
                      np.where(has_s, w_ns[np.minimum(r, H - 2)], 0.0),
                      np.where(has_n, w_ns[np.maximum(r - 1, 0)], 0.0)], axis=1)
    rowptr, col, val = _csr_from_neighbours(nbr, nbr_w)
    return GridGraph("sphere", H, W, nbr, nbr_w, rowptr, col, val)
