"""Every block row of a full-size operator, from the oracle, chunk by chunk.

The oracle assembles a set of elements together with their face neighbours;
the block rows of the set's own elements are then exactly the rows of the
full assembly (a row couples an element only to itself and its face
neighbours). Covering the mesh with compact chunks of its logical element
grid gives (M v)_rows and (A v)_rows for every row of the full-size problem
with bounded memory, in worker processes started with `spawn` (safe after
CUDA has been initialised in the parent). Only oracle/ and the seeded input
generators are used here; nothing comes from the CUDA path except the vectors
being checked.
"""
import multiprocessing as mp
import os
import tempfile

import numpy as np

_W = {}


def _face_keys(elements, ids, dim):
    """Sorted corner-vertex tuples of the 2d faces of the elements `ids`."""
    keys = []
    for k in range(dim):
        for side in (0, 1):
            corners = [c for c in range(1 << dim) if ((c >> k) & 1) == side]
            keys.append(np.sort(elements[ids][:, corners], axis=1))
    return np.concatenate(keys)


_INC = {}


def _incidence(elements):
    """Vertex -> element incidence of a connectivity array (sorted vertex ids
    and the flat positions they come from), cached per array."""
    key = (elements.__array_interface__["data"][0], elements.shape)
    if key not in _INC:
        flat = elements.ravel()
        order = np.argsort(flat, kind="stable")
        _INC.clear()
        _INC[key] = (order, flat[order])
    return _INC[key]


def face_neighbours(elements, chunk, dim):
    """The chunk's elements plus every element sharing a face (the same
    2^(d-1) corner vertices) with one of them, sorted."""
    chunk = np.asarray(chunk, dtype=np.int64)
    E, V = elements.shape
    order, sv = _incidence(elements)
    verts = np.unique(elements[chunk].ravel())
    lo = np.searchsorted(sv, verts, side="left")
    hi = np.searchsorted(sv, verts, side="right")
    cand = np.unique(np.concatenate([order[a:b] // V for a, b in zip(lo, hi)]))
    cand = np.setdiff1d(cand, chunk)
    if len(cand) == 0:
        return np.sort(chunk)
    own = set(map(tuple, _face_keys(elements, chunk, dim).tolist()))
    ck = _face_keys(elements, cand, dim).reshape(2 * dim, len(cand), -1)
    hit = np.zeros(len(cand), dtype=bool)
    for f in range(2 * dim):
        hit |= np.array([tuple(r) in own for r in ck[f].tolist()])
    return np.unique(np.concatenate([chunk, cand[hit]]))


def grid_chunks(grid_shape, pieces):
    """Element ids (x fastest) of a logical grid split into compact blocks:
    pieces[k] pieces along axis k."""
    dim = len(grid_shape)
    edges = [np.linspace(0, grid_shape[k], pieces[k] + 1).astype(int) for k in range(dim)]
    strides = np.cumprod((1,) + tuple(grid_shape[:-1]))
    chunks = []
    for idx in np.ndindex(*pieces):
        ranges = [np.arange(edges[k][idx[k]], edges[k][idx[k] + 1]) for k in range(dim)]
        mesh = np.meshgrid(*ranges, indexing="ij")
        ids = sum(mesh[k].ravel() * strides[k] for k in range(dim))
        chunks.append(np.sort(ids.astype(np.int64)))
    return chunks


def _init(make_expr, vec_path):
    from paper_2602_16312_gb300 import workloads as W  # noqa: F401
    _W["wl"] = eval(make_expr, {"W": W})
    _W["vecs"] = np.load(vec_path, mmap_mode="r")


def _rows(args):
    chunk, which = args
    from oracle import sipg
    wl = _W["wl"]
    vecs = _W["vecs"]
    B = (wl.degree + 1) ** wl.mesh.dim
    idx = face_neighbours(wl.mesh.elements, chunk, wl.mesh.dim)
    disc = sipg.assemble(wl.mesh.vertices, wl.mesh.elements[idx], wl.conductivity[idx], wl.degree,
                         wl.penalty_mode, wl.penalty_coeff)
    loc = np.searchsorted(idx, chunk)
    rows = (loc[:, None] * B + np.arange(B)[None, :]).ravel()
    cols = (idx[:, None] * B + np.arange(B)[None, :]).ravel()
    Mr = disc.M[rows]
    Ar = disc.A[rows]
    out = []
    for k, ops in which:
        v = np.asarray(vecs[k][cols])
        out.append(((Mr @ v) if "M" in ops else None, (Ar @ v) if "A" in ops else None))
    return chunk, out


def oracle_products(make_expr, grid_shape, pieces, vectors, which, workers=None):
    """For the workload `make_expr` (an expression over the workloads module W)
    and global vectors `vectors` (list of arrays of n_dofs), the full
    products M v and A v as the oracle assembles them, for the requested
    (vector index, "M" / "A" / "MA") pairs in `which`. Returns a list of
    (Mv or None, Av or None) in the order of `which`."""
    chunks = grid_chunks(grid_shape, pieces)
    n = len(vectors[0])
    tmp = tempfile.mkdtemp(prefix="oracle_rows_")
    path = os.path.join(tmp, "vecs.npy")
    np.save(path, np.stack([np.asarray(v, dtype=np.float64) for v in vectors]))
    res = [[np.zeros(n) if "M" in ops else None, np.zeros(n) if "A" in ops else None] for _, ops in which]
    if workers is None:
        workers = max(1, min(len(chunks), os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    try:
        with ctx.Pool(workers, initializer=_init, initargs=(make_expr, path)) as pool:
            for chunk, out in pool.imap_unordered(_rows, [(c, which) for c in chunks]):
                B = n // (int(np.prod(grid_shape)))
                rows = (chunk[:, None] * B + np.arange(B)[None, :]).ravel()
                for j, (mv, av) in enumerate(out):
                    if mv is not None:
                        res[j][0][rows] = mv
                    if av is not None:
                        res[j][1][rows] = av
    finally:
        os.remove(path)
        os.rmdir(tmp)
    return [tuple(r) for r in res]
