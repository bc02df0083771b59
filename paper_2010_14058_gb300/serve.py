"""Continuous-batching request server for typed-graphlet counting.

Requests (typed graphs with an arrival time) are admitted while the
device-memory budget allows; requests of the same number of types L whose
size is below `small_edges` are grouped into one batch handle (one build,
one kernel sequence for the whole group); larger requests run alone.  Each
admitted group runs on a worker thread with its own CUDA stream, so the
groups' copies and kernels overlap on the GPU while the scheduler keeps
admitting.  A request's latency is its completion time minus its arrival
time.  Results are the global typed-graphlet totals of each request
(Problem 2), identical to a standalone tg_count of the same graph.

Requests that name their graph (`key`) and are larger than `small_edges`
leave their built handle -- the typed CSR and the counting state -- on the
device after they finish, in LRU order within `resident_bytes`; a later
request for the same graph is counted on that handle without uploading or
building anything.  Resident handles count against the memory budget and
idle ones are released, oldest first, when admission needs the room.

All counting runs in libtg through the binding; this module only moves
host arrays, streams and bookkeeping.
"""
from __future__ import annotations

import queue
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass

import numpy as np

from . import tg

# device bytes a request needs while it is counted, per edge and per node
# (handle arrays plus per-edge intermediates of the 4-node stage, L = 8 bound)
BYTES_PER_EDGE = 40 * 64 + 96
BYTES_PER_NODE = 2 * 8 * 64 + 64


@dataclass
class Request:
    rid: int
    L: int
    row_ptr: np.ndarray
    col: np.ndarray
    types: np.ndarray
    arrival: float = 0.0                  # seconds after the start of the run
    key: object = None                    # identity of the graph (None: never kept resident)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0]) - 1

    @property
    def m(self) -> int:
        return int(self.col.shape[0]) // 2

    def bytes_needed(self) -> int:
        return BYTES_PER_EDGE * self.m + BYTES_PER_NODE * self.n + (1 << 20)


@dataclass
class Result:
    rid: int
    totals: np.ndarray
    arrival: float
    started: float
    done: float
    status: int
    group_size: int
    resident: bool = False                # counted on a handle kept from an earlier request

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Group:
    reqs: list
    nbytes: int
    started: float = 0.0
    handle: object = None                 # resident handle to count on (single request)


@dataclass
class _Resident:
    handle: object
    nbytes: int
    busy: bool = False


def _union(reqs: list):
    """Block-diagonal union of the requests' CSRs: node_off, row_ptr, col, types."""
    n_off = np.zeros(len(reqs) + 1, dtype=np.int64)
    z_off = np.zeros(len(reqs) + 1, dtype=np.int64)
    for k, r in enumerate(reqs):
        n_off[k + 1] = n_off[k] + r.n
        z_off[k + 1] = z_off[k] + int(r.row_ptr[-1])
    rp = np.empty(int(n_off[-1]) + 1, dtype=np.int64)
    col = np.empty(int(z_off[-1]), dtype=np.int32)
    ty = np.empty(int(n_off[-1]), dtype=np.uint8)
    for k, r in enumerate(reqs):
        a, b = int(n_off[k]), int(n_off[k + 1])
        rp[a:b] = r.row_ptr[:-1] + z_off[k]
        col[z_off[k]:z_off[k + 1]] = r.col + a
        ty[a:b] = r.types
    rp[-1] = z_off[-1]
    return n_off, rp, col, ty


class Server:
    """Admission by device-memory budget, micro-batching, overlapped workers."""

    def __init__(self, budget_bytes: int = 40 << 30, workers: int = 4, small_edges: int = 100_000,
                 batch_edges: int = 4_000_000, batch_graphs: int = 512, batching: bool = True, device: int = 0,
                 resident_bytes: int = 0):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.resident_budget = int(resident_bytes)
        self._resident: OrderedDict = OrderedDict()       # key -> _Resident, oldest first
        self._resident_total = 0
        self.workers = max(1, int(workers))
        self.small_edges = small_edges
        self.batch_edges = batch_edges
        self.batch_graphs = batch_graphs
        self.batching = batching
        self.device = device
        self._in_use = 0
        self._lock = threading.Lock()
        self._freed = threading.Condition(self._lock)

    # ------------------------------------------------------------ groups
    def _evict_for(self, need: int) -> None:
        """Releases idle resident handles, oldest first, until `need` more
        bytes fit the budget (caller holds the lock)."""
        for key in list(self._resident):
            if self._in_use + self._resident_total + need <= self.budget:
                return
            r = self._resident[key]
            if not r.busy:
                del self._resident[key]
                self._resident_total -= r.nbytes
                r.handle.free()

    def _take_group(self, pending: list) -> _Group | None:
        """Next admissible group from the arrived requests (FIFO by arrival)."""
        if not pending:
            return None
        head = pending[0]
        need = head.bytes_needed()
        if need > self.budget:
            raise ValueError(f"request {head.rid} needs {need} bytes, more than the budget")
        with self._lock:
            res = self._resident.get(head.key) if head.key is not None else None
            if res is not None and not res.busy:               # counted on its resident handle
                res.busy = True
                self._resident.move_to_end(head.key)
                pending.pop(0)
                return _Group([head], 0, handle=res.handle)
            self._evict_for(need)
            if self._in_use + self._resident_total + need > self.budget:
                return None
            group = [pending.pop(0)]
            total_m, total_b = head.m, need
            if self.batching and head.m <= self.small_edges:
                k = 0
                while k < len(pending) and len(group) < self.batch_graphs:
                    r = pending[k]
                    nb = r.bytes_needed()
                    if (r.L == head.L and r.m <= self.small_edges and total_m + r.m <= self.batch_edges
                            and self._in_use + self._resident_total + total_b + nb <= self.budget):
                        group.append(pending.pop(k))
                        total_m += r.m
                        total_b += nb
                    else:
                        k += 1
            self._in_use += total_b
        return _Group(group, total_b)

    def _finish(self, grp: _Group, h) -> None:
        """After a group: its handle becomes resident (large keyed single
        requests, while resident_bytes allows) or is freed; its reservation
        is returned."""
        r = grp.reqs[0]
        with self._lock:
            if grp.handle is not None:                         # resident hit: stays resident
                self._resident[r.key].busy = False
            elif (h is not None and len(grp.reqs) == 1 and r.key is not None and r.m > self.small_edges
                  and r.key not in self._resident and self.resident_budget > 0):
                nb = max(h.device_bytes, grp.nbytes)
                if nb <= self.resident_budget:
                    while self._resident_total + nb > self.resident_budget:
                        idle = [k for k, v in self._resident.items() if not v.busy]
                        if not idle:
                            break
                        old = self._resident.pop(idle[0])
                        self._resident_total -= old.nbytes
                        old.handle.free()
                    if self._resident_total + nb <= self.resident_budget:
                        self._resident[r.key] = _Resident(h, nb)
                        self._resident_total += nb
                        h = None
            self._in_use -= grp.nbytes
            self._freed.notify_all()
        if h is not None and grp.handle is None:
            h.free()

    def close(self) -> None:
        """Releases every resident handle."""
        with self._lock:
            for r in self._resident.values():
                r.handle.free()
            self._resident.clear()
            self._resident_total = 0

    # ------------------------------------------------------------ worker
    def _run_group(self, grp: _Group, stream, t0: float) -> list:
        torch = self.torch
        reqs = grp.reqs
        L = reqs[0].L
        lay = tg.tg_layout(L, 4)
        G = lay["global_slots"]
        with torch.cuda.stream(stream):
            if grp.handle is not None:
                h = grp.handle
            elif len(reqs) == 1:
                r = reqs[0]
                h = tg.tg_build(torch.from_numpy(r.row_ptr).to("cuda", non_blocking=False),
                                torch.from_numpy(r.col).to("cuda"), torch.from_numpy(r.types).to("cuda"), L,
                                stream=stream)
            else:
                n_off, rp, col, ty = _union(reqs)
                h = tg.tg_build_batch(n_off, torch.from_numpy(rp).to("cuda"), torch.from_numpy(col).to("cuda"),
                                      torch.from_numpy(ty).to("cuda"), L, stream=stream)
            out = torch.empty((len(reqs), G), dtype=torch.int64, device="cuda")
            tg.tg_count(h, 4, None, out, stream=stream)
            host = out.to("cpu", non_blocking=False)
            status = tg.tg_query_status(h)
        done = time.perf_counter() - t0
        res = [Result(r.rid, host[k].numpy().copy(), r.arrival, grp.started, done, status, len(reqs),
                      grp.handle is not None) for k, r in enumerate(reqs)]
        return res, h

    # ------------------------------------------------------------ run
    def run(self, requests: list, realtime: bool = True) -> list:
        """Serves `requests` (sorted by arrival).  realtime: requests become
        visible at their arrival times (open loop); otherwise all at once."""
        torch = self.torch
        torch.cuda.set_device(self.device)
        reqs = sorted(requests, key=lambda r: r.arrival)
        work: queue.Queue = queue.Queue(maxsize=self.workers)
        results: list = []
        res_lock = threading.Lock()
        errors: list = []
        t0 = time.perf_counter()

        def worker():
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream()
            while True:
                grp = work.get()
                if grp is None:
                    return
                h = None
                try:
                    out, h = self._run_group(grp, stream, t0)
                    with res_lock:
                        results.extend(out)
                except Exception as exc:  # reported after the run
                    errors.append(exc)
                finally:
                    self._finish(grp, h)

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.workers)]
        for th in threads:
            th.start()
        pending: list = []
        nxt = 0
        while nxt < len(reqs) or pending:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival <= now):
                pending.append(reqs[nxt])
                nxt += 1
            grp = self._take_group(pending)
            if grp is not None:
                grp.started = time.perf_counter() - t0
                work.put(grp)                          # blocks while every worker is busy
                continue
            if pending:
                with self._lock:
                    self._freed.wait(timeout=0.002)    # wait for memory to free up
            elif nxt < len(reqs):
                time.sleep(min(0.001, max(0.0, reqs[nxt].arrival - now)))
        for _ in threads:
            work.put(None)
        for th in threads:
            th.join()
        if errors:
            raise errors[0]
        return sorted(results, key=lambda r: r.rid)


def summarize(results: list, requests: list, window_start: float = 0.0) -> dict:
    """Latency percentiles and throughput of a served trace, over the
    requests that arrived at or after `window_start` seconds (the ones
    before it warm the server up): edges of those requests / (last
    completion - window_start)."""
    m_of = {r.rid: r.m for r in requests}
    results = [r for r in results if r.arrival >= window_start]
    lat = np.array([r.latency for r in results])
    edges = sum(m_of[r.rid] for r in results)
    span = max(r.done for r in results) - max(window_start, min(r.arrival for r in results))
    return {"requests": len(results), "edges": int(edges), "span_s": round(float(span), 3),
            "edges_per_s": round(edges / span, 1), "p50_ms": round(float(np.percentile(lat, 50) * 1e3), 3),
            "p99_ms": round(float(np.percentile(lat, 99) * 1e3), 3), "mean_ms": round(float(lat.mean() * 1e3), 3),
            "mean_group": round(float(np.mean([r.group_size for r in results])), 2),
            "resident_hits": int(sum(r.resident for r in results))}


def request_pool(count: int, seed: int, m_min: int = 100, m_max: int = 1_000_000, gamma: float = 2.2,
                 L_range=(3, 8)) -> list:
    """Seeded pool of request graphs: Chung-Lu, edges log-uniform in
    [m_min, m_max], n = max(10, ceil(m / 5)), L uniform in L_range, uniform
    types (the request mix of the serving workload)."""
    import graphgen
    rng = np.random.default_rng(seed)
    pool = []
    for k in range(count):
        m = int(round(m_min * (m_max / m_min) ** rng.random()))
        n = max(10, -(-m // 5))
        m = min(m, n * (n - 1) // 2 // 2)
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        wmax = max(2.0, min(0.5 * n, 2.0 * m / n * 40))
        g = graphgen.chung_lu(n, m, gamma, wmax, L, seed * 1000 + k)
        pool.append(g)
    return pool


def poisson_trace(pool: list, rate_per_s: float, duration_s: float, seed: int) -> list:
    """Open-loop Poisson arrivals over `duration_s`, each request a seeded
    draw from the pool."""
    rng = np.random.default_rng(seed)
    t, rid, out = 0.0, 0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > duration_s:
            break
        k = int(rng.integers(len(pool)))
        g = pool[k]
        out.append(Request(rid, g["L"], g["row_ptr"], g["col"], g["types"], t, key=k))
        rid += 1
    return out
