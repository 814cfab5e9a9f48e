"""The CPU oracle over many host cores, for parity checks at the benchmark's full sizes.

Test infrastructure only.  The oracle itself is unchanged: each spawned process runs the plain C
oracle on its own share of the work and writes its slice of the result into a file-backed array,
so that the whole CSR value array (tens of millions of entries) is compared element by element
with the GPU's.  The shares are contiguous row ranges; a process assembles every cell that
touches its range (oracle_assemble_rows / oracle_action restricted to those cells), so every row
of the range receives all of its contributions, in the oracle's own cell order.

Processes are started with the spawn method, so a CUDA context in the calling process is never
inherited.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np

import oracle as O


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _touching(cmap, r0, r1):
    """Cells with at least one node in [r0, r1)."""
    hit = np.zeros(cmap.shape[0], dtype=bool)
    for i in range(cmap.shape[1]):
        c = cmap[:, i]
        hit |= (c >= r0) & (c < r1)
    return np.nonzero(hit)[0]


def _load(d, name, mode="r"):
    return np.load(os.path.join(d, name + ".npy"), mmap_mode=mode)


def _mat_worker(task):
    d, dim, p, form, nrows, r0, r1, has_kappa = task
    cmap, cv, xy = _load(d, "cmap"), _load(d, "cv"), _load(d, "coords")
    rowptr, colidx = _load(d, "rowptr"), _load(d, "colidx")
    kappa = np.ascontiguousarray(_load(d, "kappa")) if has_kappa else None
    cells = _touching(cmap, r0, r1)
    rows = np.arange(r0, r1, dtype=np.int64)
    b0, b1 = int(rowptr[r0]), int(rowptr[r1])
    srp = np.ascontiguousarray(rowptr[r0:r1 + 1] - b0, dtype=np.int64)
    sci = np.ascontiguousarray(colidx[b0:b1], dtype=np.int32)
    vals, absv = O.assemble_rows(dim, p, form, np.ascontiguousarray(cmap[cells]), np.ascontiguousarray(xy),
                                 np.ascontiguousarray(cv[cells]), nrows, rows, srp, sci, kappa=kappa)
    out_v, out_a = _load(d, "vals", "r+"), _load(d, "absv", "r+")
    out_v[b0:b1] = vals
    out_a[b0:b1] = absv
    out_v.flush()
    out_a.flush()
    return r1 - r0


def _action_worker(task):
    d, dim, p, form, r0, r1, has_kappa = task
    cmap, cv, xy, x = _load(d, "cmap"), _load(d, "cv"), _load(d, "coords"), _load(d, "x")
    kappa = np.ascontiguousarray(_load(d, "kappa")) if has_kappa else None
    cells = _touching(cmap, r0, r1)
    y, ay = O.action(dim, p, form, np.ascontiguousarray(cmap[cells]), np.ascontiguousarray(xy),
                     np.ascontiguousarray(cv[cells]), np.ascontiguousarray(x), kappa=kappa)
    out_y, out_a = _load(d, "y", "r+"), _load(d, "ay", "r+")
    out_y[r0:r1] = y[r0:r1]
    out_a[r0:r1] = ay[r0:r1]
    out_y.flush()
    out_a.flush()
    return r1 - r0


def _ranges(nrows, parts):
    cuts = np.linspace(0, nrows, parts + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


class _Stage:
    """A scratch folder of .npy inputs and outputs shared with the worker processes."""

    def __init__(self, **arrays):
        self.dir = tempfile.mkdtemp(prefix="oracle_pool_")
        for k, v in arrays.items():
            if v is not None:
                np.save(os.path.join(self.dir, k + ".npy"), np.ascontiguousarray(v))

    def out(self, name, n):
        a = np.lib.format.open_memmap(os.path.join(self.dir, name + ".npy"), mode="w+", dtype=np.float64, shape=(n,))
        a[:] = 0.0
        a.flush()
        del a

    def get(self, name):
        return np.array(_load(self.dir, name))

    def close(self):
        shutil.rmtree(self.dir, ignore_errors=True)


def _run(fn, tasks, procs):
    O.build()
    with mp.get_context("spawn").Pool(processes=procs) as pool:
        return sum(pool.map(fn, tasks, chunksize=1))


def assemble_mat_full(dim, p, form, cmap, coords, cell_vertex, rowptr, colidx, kappa=None, procs=None):
    """Oracle CSR values and per-entry scales on the caller's (oracle-identical) pattern."""
    procs = procs or _cores()
    nrows = len(rowptr) - 1
    st = _Stage(cmap=cmap.astype(np.int32), cv=cell_vertex.astype(np.int32), coords=coords,
                rowptr=rowptr.astype(np.int64), colidx=colidx.astype(np.int32), kappa=kappa)
    try:
        st.out("vals", len(colidx))
        st.out("absv", len(colidx))
        tasks = [(st.dir, dim, p, form, nrows, a, b, kappa is not None) for a, b in _ranges(nrows, 4 * procs)]
        assert _run(_mat_worker, tasks, procs) == nrows
        return st.get("vals"), st.get("absv")
    finally:
        st.close()


def action_full(dim, p, form, cmap, coords, cell_vertex, x, kappa=None, procs=None):
    """Oracle y = A x cell by cell, and its per-entry scale, over every row."""
    procs = procs or _cores()
    n = len(x)
    st = _Stage(cmap=cmap.astype(np.int32), cv=cell_vertex.astype(np.int32), coords=coords, x=x, kappa=kappa)
    try:
        st.out("y", n)
        st.out("ay", n)
        tasks = [(st.dir, dim, p, form, a, b, kappa is not None) for a, b in _ranges(n, 4 * procs)]
        assert _run(_action_worker, tasks, procs) == n
        return st.get("y"), st.get("ay")
    finally:
        st.close()


def _item_worker(task):
    dim, p, form, cmap, coords, cv, rowptr, colidx, f = task
    vals, absv = O.assemble_mat(dim, p, form, cmap, coords, cv, rowptr, colidx)
    b, babs = O.assemble_vec(dim, p, p, cmap, len(f), coords, cv, f, cmap)
    return vals, absv, b, babs


def assemble_items(items, procs=None):
    """Oracle Mat and right-hand side (f v dx, f in the same space) of several small problems:
    items = [(dim, p, form, cmap, coords, cell_vertex, rowptr, colidx, f)], one process each."""
    O.build()
    with mp.get_context("spawn").Pool(processes=min(procs or _cores(), max(1, len(items)))) as pool:
        return pool.map(_item_worker, items, chunksize=1)
