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
import ctypes as C
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


class FamilyEngine:
    """One mesh family: cached hierarchy, own stream, 16-slot PCG.

    Right-hand sides and solutions pass through pinned per-slot staging
    buffers, so admission and retirement copies are asynchronous; the host
    waits once per poll.  When nothing is queued for the family, a step runs
    up to `iters_per_step` iterations before the next host round trip."""

    def __init__(self, name, spec, nslots=16, mode=_abi.FP32_MG_FP64_CG, rtol=1e-8, maxit=200,
                 iters_per_step=4):
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
        self.b_stage = torch.empty(nslots, self.rows, dtype=torch.float64, pin_memory=True)
        self.x_stage = torch.empty(nslots, self.rows, dtype=torch.float64, pin_memory=True)
        self._chk(self.lib.nnmg_batch_reset(self.H.h, mode, nslots, rtol, maxit, self.sptr), "reset")
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
        return self.inflight or any(o is not None for o in self.owner) or bool(self.queue)

    def admit(self, now):
        """Move queued requests into free slots while whole requests fit."""
        while self.queue and self.queue[0].nrhs <= self.free_slots():
            req = self.queue.popleft()
            req.t_admit = now
            req.x = np.zeros((self.rows, req.nrhs))
            req.iters = [0] * req.nrhs
            req.relres = [0.0] * req.nrhs
            req.status = [0] * req.nrhs
            req.cols_left = req.nrhs
            for j in range(req.nrhs):
                slot = self.owner.index(None)
                self.owner[slot] = (req, j)
                self.b_stage[slot].numpy()[:] = req.b[:, j]
                self._chk(self.lib.nnmg_batch_admit(self.H.h, slot, self.b_stage[slot].data_ptr(), 1,
                                                    self.sptr), "admit")

    def step(self):
        if any(o is not None for o in self.owner) and not self.inflight:
            n = 1 if self.queue else self.iters_per_step
            self._chk(self.lib.nnmg_batch_step(self.H.h, n, self.sptr), "step")
            self.inflight = True
            self.last_used = time.perf_counter()

    def poll(self, wait=False):
        """If the last step finished: retire finished columns; returns finished requests."""
        if not self.inflight:
            return None
        ready = C.c_int(0)
        self._chk(self.lib.nnmg_batch_poll(self.H.h, int(wait), C.byref(ready),
                                           self._active.ctypes.data, self._iters.ctypes.data,
                                           self._rel.ctypes.data, self._status.ctypes.data),
                  "poll")
        if not ready.value:
            return None
        self.inflight = False
        done = []
        retired = []
        for slot, o in enumerate(self.owner):
            if o is None or self._active[slot]:
                continue
            self._chk(self.lib.nnmg_batch_retire(self.H.h, slot, self.x_stage[slot].data_ptr(), 1,
                                                 self.sptr), "retire")
            retired.append(slot)
        if retired:
            self.stream.synchronize()                 # the retire copies
        for slot in retired:
            req, j = self.owner[slot]
            req.x[:, j] = self.x_stage[slot].numpy()
            req.iters[j] = int(self._iters[slot])
            req.relres[j] = float(self._rel[slot])
            req.status[j] = int(self._status[slot])
            self.owner[slot] = None
            req.cols_left -= 1
            if req.cols_left == 0:
                done.append(req)
        return done

    def close(self):
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
