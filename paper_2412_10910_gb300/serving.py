"""Continuous-batching solve server on one GPU.

Every mesh family gets a FamilyEngine: its hierarchy (built once and cached on
the device), a CUDA stream and a PCG over 16 independent right-hand-side
slots (nnmg_batch_* in include/nnmg.h).  Between two PCG iterations an engine
retires the columns that converged, returns finished requests and admits
queued requests into the freed slots, so requests that arrive while others are
being solved join the running solve (iteration-level batching).  Engines of
different families step concurrently on their own streams.  A family is built
only if its device bytes fit the memory budget; the bytes are known before
anything is allocated (nnmg_estimate_bytes numbers the meshes on the host), so
a family that does not fit waits without touching device memory, and idle
families are evicted (least recently used) to make room.

The scheduler is host code; every arithmetic step runs in libnnmg's kernels.
"""
from __future__ import annotations

import collections
import concurrent.futures
import ctypes as C
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import _abi
from . import nnmg as _nnmg


@dataclass
class Request:
    rid: int
    family: str
    b: np.ndarray                  # host [rows, nrhs] float64
    arrival: float = 0.0           # seconds after the start of the run
    x: np.ndarray | None = None
    iters: list = field(default_factory=list)
    relres: list = field(default_factory=list)
    status: list = field(default_factory=list)
    t_admit: float | None = None
    t_done: float | None = None
    cols_left: int = 0

    @property
    def nrhs(self):
        return self.b.shape[1]


@dataclass
class FamilySpec:
    levels: list
    degree: int
    cheb: int = 3
    n_components: int = 1
    lame: tuple = (1.0, 1.0)


_copy_pool = None
COPY_THREADS = min(8, os.cpu_count() or 1)


def parallel_copy(dst, src, chunk_bytes=2 << 20):
    """dst[...] = src, split along the first axis into pieces of about
    chunk_bytes copied by COPY_THREADS host threads (numpy copies release the
    GIL): a request's right-hand sides and solutions are tens to hundreds of
    MB, and one thread copies them at a fraction of the host's bandwidth."""
    global _copy_pool
    k = int(min(COPY_THREADS, max(1, dst.nbytes // chunk_bytes)))
    if k <= 1:
        np.copyto(dst, src)
        return
    if _copy_pool is None:
        _copy_pool = concurrent.futures.ThreadPoolExecutor(max_workers=COPY_THREADS)
    b = np.linspace(0, dst.shape[0], k + 1).astype(np.int64)
    futs = [_copy_pool.submit(np.copyto, dst[lo:hi], src[lo:hi]) for lo, hi in zip(b[:-1], b[1:])]
    for f in futs:
        f.result()


def batch_width(n, nslots):
    """Columns of the batch that holds n occupied slots: 1 for n <= 1, else n
    rounded up to an even count (paired FP32 kernels and 8-byte rows), at
    most nslots."""
    return 1 if n <= 1 else min(nslots, n + (n & 1))


def pack_plan(owner, width, needed, nslots):
    """How to repack a batch before a step: the occupied slots of
    owner[:width] move, in order, to the first positions and the batch becomes
    batch_width(needed) columns wide.  Returns (new_width, src) for
    nnmg_batch_repack (src[j] = old slot of new column j, -1 empty), or None
    if the batch already has that form."""
    occ = [q for q in range(width) if owner[q] is not None]
    w = batch_width(max(needed, len(occ)), nslots)
    if w == width and occ == list(range(len(occ))):
        return None
    return w, occ + [-1] * (w - len(occ))


class FamilyEngine:
    """One mesh family: cached hierarchy, own stream, 16-slot PCG.

    Right-hand sides and solutions pass through pinned per-slot staging
    buffers, so admission and retirement copies are asynchronous; the host
    waits once per poll.  When nothing is queued for the family, a step runs
    up to `iters_per_step` iterations before the next host round trip.
    Before every step the occupied slots are packed into the first columns and
    the batch is cut to the width they need (nnmg_batch_repack), because a
    PCG iteration costs in proportion to its columns on the larger meshes."""

    def __init__(self, name, spec, nslots=16, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8, maxit=200,
                 iters_per_step=4, warm_widths=True):
        import torch
        self.name = name
        self.spec = spec
        self.H = _nnmg.Hierarchy(spec.levels, spec.degree, spec.n_components, spec.lame,
                                 spec.cheb, max_nrhs=nslots)
        self.top = self.H.n_levels - 1
        self.rows = self.H.rows(self.top)
        self.free_dofs = self.H.info(self.top)[1] * spec.n_components
        self.nslots = nslots
        self.stream = torch.cuda.Stream()
        self.sptr = C.c_void_p(self.stream.cuda_stream)
        self.lib = _abi.load()
        self.owner = [None] * nslots          # slot -> (request, column)
        self.queue = collections.deque()
        self.inflight = False
        self.last_used = time.perf_counter()
        self.iters_per_step = iters_per_step
        self.iterations = 0          # PCG iterations run by this engine
        self.column_iterations = 0   # sum over those iterations of the occupied slots
        self.width_iterations = 0    # sum over those iterations of the batch width
        # pinned staging: a request's right-hand sides as one [rows][nrhs]
        # block at the offset of its first slot; solutions one column per slot
        self.b_stage = torch.empty(nslots * self.rows, dtype=torch.float64, pin_memory=True)
        self.x_stage = torch.empty(nslots, self.rows, dtype=torch.float64, pin_memory=True)
        self.host_copy_s = 0.0       # host time spent staging b and x
        self.pending = collections.deque()     # (event, retired columns) in stream order
        self.staged = [False] * nslots         # x_stage[slot] awaits its host copy
        self._chk(self.lib.nnmg_batch_reset(self.H.h, mode, nslots, rtol, maxit, self.sptr), "reset")
        self.width = nslots                   # columns of the device batch
        self.repacks = 0
        if warm_widths:
            self._warm_widths()
        self._active = np.zeros(nslots, dtype=np.int32)
        self._iters = np.zeros(nslots, dtype=np.int32)
        self._rel = np.zeros(nslots)
        self._status = np.zeros(nslots, dtype=np.int32)

    def bytes(self):
        return self.H.hierarchy_bytes() + self.H.solve_bytes(self.nslots)

    @staticmethod
    def estimate_bytes(name, spec, nslots=16, **kw):
        """Device bytes of the engine, computed on the host before it is built."""
        hb, sb = _nnmg.nnmg_estimate_bytes(spec.levels, spec.degree, spec.n_components,
                                           nrhs=nslots, lame=spec.lame, cheb_degree=spec.cheb,
                                           max_nrhs=nslots)
        return hb + sb

    def _chk(self, st, what):
        if st != 0:
            raise _nnmg.NNMGError(st, f"{self.name}: {what}")

    def free_slots(self):
        return sum(o is None for o in self.owner)

    def busy(self):
        return (self.inflight or any(o is not None for o in self.owner) or bool(self.queue)
                or bool(self.pending))

    def _warm_widths(self):
        """Step every batch width twice with no column occupied, so that its
        kernel choices are tuned and its iteration graph is captured before
        serving (a width's first use would otherwise stall its requests)."""
        ready = C.c_int(0)
        for w in sorted({batch_width(n, self.nslots) for n in range(1, self.nslots + 1)}):
            self._chk(self.lib.nnmg_batch_repack(self.H.h, w, (C.c_int * w)(*([-1] * w)),
                                                 self.sptr), "repack")
            self.width = w
            for _ in range(2):
                self._chk(self.lib.nnmg_batch_step(self.H.h, 1, self.sptr), "step")
                self._chk(self.lib.nnmg_batch_poll(self.H.h, 1, C.byref(ready), None, None, None,
                                                   None), "poll")

    def _pack(self, needed):
        plan = pack_plan(self.owner, self.width, needed, self.nslots)
        if plan is None:
            return
        w, src = plan
        arr = (C.c_int * w)(*src)
        self._chk(self.lib.nnmg_batch_repack(self.H.h, w, arr, self.sptr), "repack")
        self.owner = [self.owner[q] for q in src if q >= 0]
        self.owner += [None] * (self.nslots - len(self.owner))
        self.width = w
        self.repacks += 1

    def admit(self, now):
        """Move queued requests into free slots while whole requests fit, then
        pack the batch to the width its columns need."""
        take = []
        free = self.free_slots()
        while self.queue and self.queue[0].nrhs <= free:
            take.append(self.queue.popleft())
            free -= take[-1].nrhs
        occupied = self.nslots - self.free_slots()
        if occupied == 0 and not take:
            return
        self._pack(occupied + sum(r.nrhs for r in take))
        for req in take:
            m = req.nrhs
            req.t_admit = now
            req.x = np.zeros((m, self.rows)).T     # [rows, nrhs], columns contiguous
            req.iters = [0] * m
            req.relres = [0.0] * m
            req.status = [0] * m
            req.cols_left = m
            s0 = self.owner.index(None)            # packed: the free slots follow
            assert all(o is None for o in self.owner[s0:s0 + m])
            for j in range(m):
                self.owner[s0 + j] = (req, j)
            t = time.perf_counter()
            block = self.b_stage[s0 * self.rows:(s0 + m) * self.rows]
            parallel_copy(block.numpy().reshape(self.rows, m), req.b)
            self.host_copy_s += time.perf_counter() - t
            self._chk(self.lib.nnmg_batch_admit_cols(self.H.h, s0, m, block.data_ptr(), m, 1,
                                                     self.sptr), "admit")

    def step(self):
        if any(o is not None for o in self.owner) and not self.inflight:
            n = 1 if self.queue else self.iters_per_step
            self._chk(self.lib.nnmg_batch_step(self.H.h, n, self.sptr), "step")
            self.iterations += n
            self.column_iterations += n * sum(o is not None for o in self.owner)
            self.width_iterations += n * self.width
            self.inflight = True
            self.last_used = time.perf_counter()

    def _drain(self, block=False):
        """Finish the retirements whose device copies are done: solution
        columns from the staging buffers into the requests; returns the
        requests that are complete."""
        done = []
        while self.pending and (block or self.pending[0][0].query()):
            ev, cols = self.pending.popleft()
            ev.synchronize()
            t = time.perf_counter()
            for slot, req, j, its, rel, st in cols:
                parallel_copy(req.x[:, j], self.x_stage[slot].numpy())
                self.staged[slot] = False
                req.iters[j], req.relres[j], req.status[j] = its, rel, st
                req.cols_left -= 1
                if req.cols_left == 0:
                    done.append(req)
            self.host_copy_s += time.perf_counter() - t
        return done

    def poll(self, wait=False):
        """Finish earlier retirements whose copies are done and, if the last
        step finished, retire its converged columns: their slots are free at
        once, their solutions arrive asynchronously (an event after the copies;
        the host does not wait for the GPU).  Returns the requests completed,
        or None if nothing happened."""
        import torch
        done = self._drain()
        if not self.inflight:
            return done or None
        ready = C.c_int(0)
        self._chk(self.lib.nnmg_batch_poll(self.H.h, int(wait), C.byref(ready),
                                           self._active.ctypes.data, self._iters.ctypes.data,
                                           self._rel.ctypes.data, self._status.ctypes.data),
                  "poll")
        if not ready.value:
            return done or None
        self.inflight = False
        cols = []
        for slot, o in enumerate(self.owner):
            if o is None or self._active[slot]:
                continue
            if self.staged[slot]:                     # an earlier copy into this buffer
                done += self._drain(block=True)
            self._chk(self.lib.nnmg_batch_retire(self.H.h, slot, self.x_stage[slot].data_ptr(), 1,
                                                 self.sptr), "retire")
            req, j = o
            cols.append((slot, req, j, int(self._iters[slot]), float(self._rel[slot]),
                         int(self._status[slot])))
            self.staged[slot] = True
            self.owner[slot] = None
        if cols:
            ev = torch.cuda.Event()
            ev.record(self.stream)
            self.pending.append((ev, cols))
        return done

    def close(self):
        self._drain(block=True)
        self.H.close()


class Server:
    """Admits requests by device-memory budget and runs all families' engines."""

    def __init__(self, families: dict, budget_bytes: int, nslots=16, mode=_abi.FP32_MG_FP64_CG,
                 rtol=1e-8, maxit=200, engine_factory=None, poll_pause_s=0.0):
        self.families = families
        # pause between polls while steps are in flight (0: poll continuously)
        self.poll_pause_s = poll_pause_s
        self.budget = budget_bytes
        self.kw = dict(nslots=nslots, mode=mode, rtol=rtol, maxit=maxit)
        self.engines: dict[str, FamilyEngine] = {}
        self.evictions = 0
        self.builds = 0
        self._sizes: dict[str, int] = {}
        # builds a family's engine: FamilyEngine unless a caller substitutes
        # its own (same constructor arguments, estimate_bytes(), bytes(),
        # busy(), close(), last_used)
        self._make = engine_factory or FamilyEngine

    def used_bytes(self):
        return sum(e.bytes() for e in self.engines.values())

    def family_bytes(self, name):
        """Device bytes of a family's engine, known before it is built (cached)."""
        if name not in self._sizes:
            self._sizes[name] = self._make.estimate_bytes(name, self.families[name], **self.kw)
        return self._sizes[name]

    def engine(self, name):
        """The family's engine, building it if the budget allows (evicting idle
        ones first); None if it has to wait for a busy engine to become idle.
        Nothing is allocated for a family that waits."""
        if name in self.engines:
            return self.engines[name]
        need = self.family_bytes(name)
        if need > self.budget:
            raise MemoryError(f"family {name} needs {need} bytes, budget {self.budget}")
        while self.used_bytes() + need > self.budget:
            idle = [e for e in self.engines.values() if not e.busy()]
            if not idle:
                return None       # wait until an engine becomes idle
            victim = min(idle, key=lambda e: e.last_used)
            victim.close()
            del self.engines[victim.name]
            self.evictions += 1
        eng = self._make(name, self.families[name], **self.kw)
        self.builds += 1
        self.engines[name] = eng
        return eng

    def prepare(self, names):
        for n in names:
            self.engine(n)

    def run(self, requests, time_scale=1.0):
        """Serve requests (sorted by arrival, seconds); returns finished requests."""
        import torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()          # arrived, family not admitted yet
        finished = []
        t0 = time.perf_counter()
        total = len(pending)
        while len(finished) < total:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival * time_scale <= now:
                waiting.append(pending.popleft())
            still = collections.deque()
            for req in waiting:
                eng = self.engine(req.family)
                if eng is None:
                    still.append(req)
                else:
                    eng.queue.append(req)
            waiting = still
            progressed = False
            for eng in list(self.engines.values()):
                done = eng.poll(wait=False)
                if done is not None:
                    progressed = True
                    t = time.perf_counter() - t0
                    for r in done:
                        r.t_done = t
                        finished.append(r)
                if not eng.inflight:
                    eng.admit(time.perf_counter() - t0)
                    eng.step()
            if not progressed:
                # wait for the next event: a step finishing on the GPU (polled
                # without sleeping while steps are in flight) or, with nothing
                # in flight, the next arrival
                inflight = [e for e in self.engines.values() if e.inflight]
                if inflight and not pending and not waiting:
                    inflight[0].stream.synchronize()
                elif inflight and self.poll_pause_s > 0:
                    time.sleep(self.poll_pause_s)
                elif not inflight and pending and not waiting and \
                        not any(e.busy() for e in self.engines.values()):
                    dt = pending[0].arrival * time_scale - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
        torch.cuda.synchronize()
        return finished

    def close(self):
        for e in self.engines.values():
            e.close()
        self.engines.clear()


def latency_stats(finished):
    lat = np.array([r.t_done - r.arrival for r in finished])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}
