"""Worker processes for the oracle's chunked element sums (test
infrastructure, like the rest of the package).

`ReducedModel.eval` sums the elastic terms of Eq. 11 over chunks of cubature
tets (`reduced.chunk_terms`).  On the largest meshes (960,000 tets) one
evaluation takes about a minute on one core, almost all of it in the
per-chunk element Hessians, so `ElementPool` evaluates the same chunks in
worker processes and hands the per-chunk results back in chunk order; the
model adds them in that order, so the arithmetic is the serial loop's.

The workers are started with the "spawn" method (never forked: a process
forked after the parent has touched a GPU can hang), each with one BLAS
thread.  The mesh arrays, the positions x and the Jacobian J live in shared
memory; `chunk_terms(x, J, chunk)` copies x and J there and returns the list
of (g, K) parts.

    pool = ElementPool(model, workers=16)
    model.pool = pool        # model.eval now uses the workers
    ...
    pool.close()
"""
import atexit
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import shared_memory

import numpy as np

from . import reduced

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

# worker-side views of the shared arrays
_W = {}


def _attach(specs):
    out = {}
    for key, (name, shape, dtype) in specs.items():
        shm = shared_memory.SharedMemory(name=name)
        out[key] = (shm, np.ndarray(shape, dtype=np.dtype(dtype), buffer=shm.buf))
    return out


def _init(specs, mu, lam):
    _W["arrays"] = _attach(specs)
    _W["mu"], _W["lam"] = mu, lam


def _work(s0, s1):
    a = {k: v[1] for k, v in _W["arrays"].items()}
    xv = a["x"].reshape(-1, 3)
    return reduced.chunk_terms(xv, a["J"], a["tets"][s0:s1], a["DmInv"][s0:s1],
                               a["vol"][s0:s1], a["w"][s0:s1], _W["mu"], _W["lam"])


class ElementPool:
    def __init__(self, model, workers=None):
        self.workers = int(workers or os.cpu_count() or 1)
        self.S = int(model.tets.shape[0])
        arrays = {"tets": model.tets, "DmInv": model.DmInv, "vol": model.vol, "w": model.w,
                  "x": np.zeros(model.n), "J": np.zeros((model.n, model.r))}
        self._shm, specs = [], {}
        self.views = {}
        for key, a in arrays.items():
            a = np.ascontiguousarray(a)
            shm = shared_memory.SharedMemory(create=True, size=max(a.nbytes, 1))
            view = np.ndarray(a.shape, dtype=a.dtype, buffer=shm.buf)
            view[...] = a
            self._shm.append(shm)
            self.views[key] = view
            specs[key] = (shm.name, a.shape, a.dtype.str)
        # one BLAS thread per worker: set while the workers start, then restored
        saved = {v: os.environ.get(v) for v in _THREAD_VARS}
        for v in _THREAD_VARS:
            os.environ[v] = "1"
        try:
            self.ex = ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"),
                                          initializer=_init,
                                          initargs=(specs, model.mu, model.lam))
            list(self.ex.map(_noop, range(self.workers)))   # start every worker now
        finally:
            for v, val in saved.items():
                if val is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = val
        atexit.register(self.close)

    def chunk_terms(self, x, J, chunk):
        """[(g_part, K_part)] of the chunks [s, s + chunk), in chunk order."""
        self.views["x"][...] = x
        self.views["J"][...] = J
        futs = [self.ex.submit(_work, s, min(s + chunk, self.S))
                for s in range(0, self.S, chunk)]
        return [f.result() for f in futs]

    def close(self):
        if getattr(self, "ex", None) is not None:
            self.ex.shutdown(wait=True, cancel_futures=True)
            self.ex = None
        self.views = {}                # the views must go before the blocks close
        for shm in getattr(self, "_shm", []):
            try:
                shm.close()
                shm.unlink()
            except FileNotFoundError:
                pass
        self._shm = []


def _noop(_):
    return os.getpid()
