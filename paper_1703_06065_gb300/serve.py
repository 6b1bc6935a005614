"""Serving loop: continuous batching of Block CUR requests on one GPU.

Requests arrive over time (each a matrix to decompose).  The loop

* admits a request when its HBM footprint (its matrix and its share of a
  batch workspace) fits under the budget, and draws its matrix on the
  device at admission (the matrix stays resident until the request is done);
* runs requests on several lanes (CUDA streams) at once: requests are grouped
  into a batched decomposition (every stage one launch over the whole group,
  :class:`Batch`) as soon as a lane is free, so requests that arrive while
  others are on the GPU join the next group.  Heavy requests (l = k + p > 64,
  which need 128-row panels) run on lanes of their own, so that they neither
  widen the panels of the light groups nor hold them up.  By default they
  are grouped into batches of their own (up to ``max_heavy_batch``: a
  group's per-matrix factorisations run side by side, so a 16384^2 request
  costs about 3.3 ms in a group of eight against 13 ms alone); with
  ``heavy_plan=True`` each heavy lane instead keeps one single-matrix plan
  (:class:`Plan`) and runs its heavy requests one after another (about
  9.4 ms each for 16384^2, k = 64);
* retires a group when its completion event has fired, returning its memory
  to the budget.

Latency of a request = completion on the GPU clock - arrival, both measured
from the start of the run (the GPU clock is tied to the host clock by an event
recorded on an idle device at the start).  A decomposition's results do not
depend on the other requests it ran beside: every kernel forms each
per-matrix sum in a fixed order by the same units of work.
"""
from __future__ import annotations

import collections
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import Batch, Plan, _lib

LIGHT_L = 64   # requests with l = k + p above this are heavy (128-row panels)


def _torch():
    import torch

    return torch


def _item(p) -> dict:
    return dict(m=p.m, n=p.n, k=p.k, p=p.p, block=int(p.col_off[1] - p.col_off[0]),
                g_col=p.g_col, g_row=p.g_row)


class _Arena:
    """First-fit sub-allocation of one device buffer (256-byte aligned
    blocks, neighbouring free blocks merged).  Serving allocates every matrix
    and every batch workspace here, so the run never calls cudaMalloc or
    cudaFree (which would synchronise the device and stall the other lanes)."""

    def __init__(self, nbytes: int, device):
        torch = _torch()
        self.size = int(nbytes) // 256 * 256
        self.buf = torch.empty(self.size, dtype=torch.uint8, device=device)
        self.free = [(0, self.size)]   # sorted (offset, size)

    def alloc(self, nbytes: int) -> Optional[int]:
        n = (int(nbytes) + 255) // 256 * 256
        for i, (o, sz) in enumerate(self.free):
            if sz >= n:
                if sz == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, sz - n)
                return o
        return None

    def release(self, off: int, nbytes: int):
        n = (int(nbytes) + 255) // 256 * 256
        import bisect

        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        # merge with the right and left neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (off, n + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)

    def view(self, off: int, nbytes: int):
        return self.buf[off:off + int(nbytes)]


class _Req:
    __slots__ = ("r", "A", "omega", "u_col", "u_row", "bytes", "ready", "t_done", "result",
                 "a_off")

    def __init__(self, r):
        self.r = r
        self.A = self.omega = self.u_col = self.u_row = None
        self.a_off = None
        self.bytes = 0
        self.ready = None
        self.t_done = None
        self.result = None


class Server:
    """Continuous batching over `lanes` CUDA streams with an HBM budget.

    `draw(problem, device, out)` returns the request's inputs on the device:
    the matrix A (FP32, row-major, written into ``out``, an m x n view of the
    arena), the test matrix as an l x n panel and the two vectors of
    uniforms.  The caller supplies it (the benchmark and the tests draw every
    input on the device from the request's seed).  `fit_prec`: "bf16x3a" (the
    adaptive split-BF16 fit, the default) or "bf16x3" for every request.
    """

    def __init__(self, hbm_budget: float = 160e9, lanes: int = 3, max_batch: int = 128,
                 heavy_lanes: int = 2, max_heavy_batch: int = 8, heavy_share: float = 0.6,
                 builders: int = 4, keep_u: bool = False,
                 keep_inputs: Callable = None, draw: Callable = None, device=None,
                 heavy_plan: bool = False, fit_prec: str = "bf16x3a"):
        torch = _torch()
        if draw is None:
            raise ValueError("Server needs draw(problem, device, out) for the requests' inputs")
        self.torch = torch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.budget = float(hbm_budget)
        self.max_batch = max_batch
        self.max_heavy_batch = max_heavy_batch
        self.keep_u = keep_u
        self.keep_inputs = keep_inputs or (lambda r: False)
        self.draw = draw
        self.heavy_plan = heavy_plan
        self.fit_prec = fit_prec  # "bf16x3a": adaptive split-BF16 fit, "bf16x3": all split
        self.gen_stream = torch.cuda.Stream(device=self.device)
        self.light = [{"stream": torch.cuda.Stream(device=self.device), "job": None}
                      for _ in range(lanes)]
        self.heavy = [{"stream": torch.cuda.Stream(device=self.device), "job": None}
                      for _ in range(heavy_lanes)]
        # one arena for matrices and workspaces: the budget plus room for
        # fragmentation
        self.arena = _Arena(min(self.budget * 1.25, _free_bytes(self.device) * 0.9), self.device)
        self.in_use = 0.0
        self.in_heavy = 0.0
        self.heavy_share = heavy_share
        self._ws_cache: Dict[tuple, int] = {}
        self.jobs: List[tuple] = []   # (kind, requests, GPU start s, GPU end s) per group
        from concurrent.futures import ThreadPoolExecutor

        self.pool = ThreadPoolExecutor(max_workers=builders)
        self.building = {False: collections.deque(), True: collections.deque()}

    def _footprint(self, q) -> float:
        """Matrix + panels + this request's share of a workspace."""
        p = q.r.problem
        key = (q.r.heavy, p.m, p.n, p.k, p.p, int(p.col_off[1]), p.g_col, p.g_row)
        ws = self._ws_cache.get(key)
        if ws is None:
            ws = _batch_workspace(_item(p), p.q)
            self._ws_cache[key] = ws
        return 4.0 * p.m * p.n + 4.0 * p.l * (p.m + p.n) + ws

    def _admit(self, q) -> bool:
        """Draw the request's inputs into the arena; False if it has no room."""
        torch = self.torch
        p = q.r.problem
        nbytes = 4 * p.m * p.n
        off = self.arena.alloc(nbytes)
        if off is None:
            return False
        q.a_off = off
        A = self.arena.view(off, nbytes).view(torch.float32).view(p.m, p.n)
        with torch.cuda.stream(self.gen_stream):
            q.A, q.omega, q.u_col, q.u_row = self.draw(p, self.device, A)
            q.ready = torch.cuda.Event()
            q.ready.record(self.gen_stream)
        return True

    # -- jobs -----------------------------------------------------------------
    def _prepare(self, reqs):
        """Reserve a group's workspace in the arena and build its plan (the
        host-side table encoding) on a worker thread; None if the arena has
        no room yet."""
        items = [_item(q.r.problem) for q in reqs]
        ws_bytes = _batch_workspace_many(items, reqs[0].r.problem.q)
        ws_off = self.arena.alloc(ws_bytes)
        if ws_off is None:
            return None
        view = self.arena.view(ws_off, ws_bytes)
        fut = self.pool.submit(Batch, items, reqs[0].r.problem.q, self.device, view, self.fit_prec)
        return dict(reqs=reqs, ws=(ws_off, ws_bytes), fut=fut)

    def _start_light(self, lane, prep):
        """Run a prepared group on `lane`."""
        torch = self.torch
        s = lane["stream"]
        reqs = prep["reqs"]
        ws_off, ws_bytes = prep["ws"]
        b = prep["fut"].result()
        b.set_stream(s)
        with torch.cuda.stream(s):
            for q in reqs:
                s.wait_event(q.ready)
            start = torch.cuda.Event(enable_timing=True)
            start.record(s)
            out = b.run([q.A for q in reqs], [q.omega for q in reqs], [q.u_col for q in reqs],
                        [q.u_row for q in reqs], want_u=self.keep_u)
            # one copy per kind of output into pinned host memory
            host = {}
            for k in ("err", "col_idx", "row_idx", "U"):
                if k not in out["flat"]:
                    host[k] = [None] * len(reqs)
                    continue
                flat, sizes = out["flat"][k]
                h = torch.empty(flat.shape, dtype=flat.dtype, pin_memory=True)
                h.copy_(flat, non_blocking=True)
                views, at = [], 0
                for sz in sizes:
                    views.append(h[at:at + sz])
                    at += sz
                host[k] = views
            done = torch.cuda.Event(enable_timing=True)
            done.record(s)
        lane["job"] = dict(kind="heavy" if reqs[0].r.heavy else "light", reqs=reqs, batch=b,
                           host=host, start=start, done=done, ws=(ws_off, ws_bytes))

    def _heavy_lane_plan(self, lane, p):
        """The lane's single-matrix plan for this heavy shape (built on first
        use with its workspace and outputs in the arena, kept for the run)."""
        torch = self.torch
        key = (p.m, p.n, p.k, p.p, p.q, int(p.col_off[1]), p.g_col, p.g_row)
        pl = lane.get("plan")
        if pl is not None and pl["key"] == key:
            return pl
        if pl is not None:  # another heavy shape: the idle lane's plan is replaced
            self.arena.release(*pl["ws"])
            self.budget += pl["ws"][1]
            lane["plan"] = None
        with torch.cuda.stream(lane["stream"]):
            need = _plan_workspace(p)
            off = self.arena.alloc(need)
            if off is None:
                return None
            plan = Plan(p.m, p.n, p.k, p.p, p.q, p.col_off, p.row_off, p.g_col, p.g_row,
                        dtype="f32", sketch_prec="bf16", fit_prec=self.fit_prec, device=self.device,
                        workspace=self.arena.view(off, need))
        dev = self.device
        outs = dict(cs=torch.empty(plan.G_col, dtype=torch.float64, device=dev),
                    rs=torch.empty(plan.G_row, dtype=torch.float64, device=dev),
                    ci=torch.empty(plan.g_col, dtype=torch.int32, device=dev),
                    ri=torch.empty(plan.g_row, dtype=torch.int32, device=dev),
                    cp=torch.empty(plan.g_col, dtype=torch.float64, device=dev),
                    rp=torch.empty(plan.g_row, dtype=torch.float64, device=dev),
                    U=torch.empty(plan.c_max, plan.r_max, device=dev),
                    err=torch.empty(3, dtype=torch.float64, device=dev))
        self.budget -= need   # held by the lane for the rest of the run
        lane["plan"] = dict(key=key, plan=plan, outs=outs, ws=(off, need))
        return lane["plan"]

    def _start_heavy(self, lane, q, pl):
        """Run one heavy request on `lane` with the lane's plan."""
        torch = self.torch
        s = lane["stream"]
        plan, o = pl["plan"], pl["outs"]
        with torch.cuda.stream(s):
            s.wait_event(q.ready)
            start = torch.cuda.Event(enable_timing=True)
            start.record(s)
            plan.scores(q.A, q.omega, out=(o["cs"], o["rs"]))
            plan.sample(o["cs"], o["rs"], q.u_col, q.u_row, out=(o["ci"], o["ri"], o["cp"], o["rp"]))
            plan.fit(q.A, o["ci"], o["ri"], U=o["U"])
            plan.error(q.A, out=o["err"])
            host = {}
            for k, src in (("err", o["err"]), ("col_idx", o["ci"]), ("row_idx", o["ri"]),
                           ("U", o["U"] if self.keep_u else None)):
                if src is None:
                    host[k] = [None]
                    continue
                h = torch.empty(src.shape, dtype=src.dtype, pin_memory=True)
                h.copy_(src, non_blocking=True)
                host[k] = [h]
            done = torch.cuda.Event(enable_timing=True)
            done.record(s)
        lane["job"] = dict(kind="heavy", reqs=[q], batch=None, plan=plan, host=host,
                           start=start, done=done, ws=None)

    def _retire(self, lane, t_start_ev):
        job = lane["job"]
        t_done = t_start_ev.elapsed_time(job["done"]) / 1000.0
        self.jobs.append((job["kind"], len(job["reqs"]),
                          t_start_ev.elapsed_time(job["start"]) / 1000.0, t_done))
        if job["batch"] is not None:
            job["batch"].sync_status()
        else:
            job["plan"].sync_status()
        for i, q in enumerate(job["reqs"]):
            h = job["host"]
            q.t_done = t_done
            q.result = {k: (h[k][i].numpy().copy() if h[k][i] is not None else None) for k in h}
            if q.result["U"] is not None:
                c = q.r.problem.g_col * int(q.r.problem.col_off[1])
                q.result["U"] = q.result["U"].reshape(c, -1)
            if self.keep_inputs(q.r):
                q.result["inputs"] = tuple(t.cpu().numpy() for t in (q.A, q.omega, q.u_col, q.u_row))
            self.in_use -= q.bytes
            if q.r.heavy:
                self.in_heavy -= q.bytes
            self.arena.release(q.a_off, 4 * q.r.problem.m * q.r.problem.n)
            q.A = q.omega = q.u_col = q.u_row = None
        if job["ws"] is not None:
            self.arena.release(*job["ws"])
        job["batch"] = None
        lane["job"] = None
        return job["reqs"]

    # -- the loop -------------------------------------------------------------
    def run(self, requests, realtime: bool = True, timeout: float = 600.0) -> List[_Req]:
        """Serve `requests` (sorted by arrival).  realtime=False admits every
        request at once (arrival times are then ignored for admission but
        still used for the latencies)."""
        torch = self.torch
        reqs = [_Req(r) for r in requests]
        n = len(reqs)
        waiting = {False: collections.deque(), True: collections.deque()}  # arrived, by class
        light = collections.deque()     # admitted
        heavy = collections.deque()
        done: List[_Req] = []
        torch.cuda.synchronize(self.device)
        t_start_ev = torch.cuda.Event(enable_timing=True)
        t_start_ev.record(self.gen_stream)
        t0 = time.perf_counter()
        i = 0
        while len(done) < n:
            now = time.perf_counter() - t0
            if now > timeout:
                raise RuntimeError(f"serving run exceeded {timeout} s ({len(done)}/{n} done)")
            progressed = False
            # arrivals
            while i < n and (not realtime or reqs[i].r.arrival <= now):
                waiting[reqs[i].r.heavy].append(reqs[i])
                i += 1
                progressed = True
            # completions
            for lane in self.light + self.heavy:
                if lane["job"] is not None and lane["job"]["done"].query():
                    done.extend(self._retire(lane, t_start_ev))
                    progressed = True
            # admission by footprint, first come first served within each class;
            # heavy requests may hold at most `heavy_share` of the budget so that
            # light ones are never starved behind them
            for cls in (False, True):
                wq = waiting[cls]
                while wq:
                    q = wq[0]
                    q.bytes = self._footprint(q)
                    cap = self.budget * (self.heavy_share if cls else 1.0)
                    used = self.in_heavy if cls else self.in_use
                    if (self.in_use + q.bytes > self.budget or used + q.bytes > cap) \
                            and self.in_use > 0:
                        break
                    if not self._admit(q):
                        break
                    wq.popleft()
                    self.in_use += q.bytes
                    if cls:
                        self.in_heavy += q.bytes
                    (heavy if cls else light).append(q)
                    progressed = True
            # heavy requests one at a time on each free heavy lane's plan
            if self.heavy_plan:
                for lane in self.heavy:
                    if lane["job"] is None and heavy:
                        pl = self._heavy_lane_plan(lane, heavy[0].r.problem)
                        if pl is not None:
                            self._start_heavy(lane, heavy.popleft(), pl)
                            progressed = True
            # dispatch groups on free lanes
            for cls, lanes_, queue, cap in ((True, self.heavy, heavy, self.max_heavy_batch),
                                            (False, self.light, light, self.max_batch)):
                if cls and self.heavy_plan:
                    continue
                # keep one group per lane being planned ahead of time
                bq = self.building[cls]
                while queue and len(bq) < len(lanes_):
                    group = [queue[j] for j in range(min(cap, len(queue)))]
                    prep = self._prepare(group)
                    if prep is None:
                        break
                    for _ in group:
                        queue.popleft()
                    bq.append(prep)
                    progressed = True
                for lane in lanes_:
                    if lane["job"] is None and bq and bq[0]["fut"].done():
                        self._start_light(lane, bq.popleft())
                        progressed = True
            if not progressed:
                if i < n and realtime:
                    time.sleep(max(0.0, min(2e-4, reqs[i].r.arrival - now)))
                else:
                    time.sleep(5e-5)
        return done


def _plan_workspace(p) -> int:
    """Workspace bytes of a single-matrix plan (BF16 sketch, split-BF16 fit)."""
    import ctypes

    L = _lib.load()
    col_off = np.ascontiguousarray(np.asarray(p.col_off, dtype=np.int64))
    row_off = np.ascontiguousarray(np.asarray(p.row_off, dtype=np.int64))
    d = _lib.Desc()
    d.m, d.n, d.lda = p.m, p.n, p.n
    d.a_dtype = _lib.BCUR_F32
    d.k, d.p, d.q = p.k, p.p, p.q
    d.G_col = len(col_off) - 1
    d.col_off = col_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.G_row = len(row_off) - 1
    d.row_off = row_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.g_col, d.g_row = p.g_col, p.g_row
    d.replacement = 0
    d.sketch_prec, d.fit_prec = _lib.BCUR_BF16, _lib.BCUR_BF16X3
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _lib.check(L.bcur_plan(ctypes.byref(d), None, ctypes.byref(h), ctypes.byref(ws)), "bcur_plan")
    L.bcur_destroy(h)
    return int(ws.value)


def _batch_workspace(item: dict, q: int) -> int:
    """Workspace bytes of a batched plan holding this one item (host only)."""
    import ctypes

    L = _lib.load()
    arr = (_lib.BatchItem * 1)()
    a = arr[0]
    a.m, a.n, a.lda = item["m"], item["n"], item.get("lda", item["n"])
    a.k, a.p, a.block = item["k"], item["p"], item["block"]
    a.g_col, a.g_row = item["g_col"], item["g_row"]
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _lib.check(L.bcur_batch_plan(arr, 1, q, None, ctypes.byref(h), ctypes.byref(ws)),
               "bcur_batch_plan")
    L.bcur_batch_destroy(h)
    return int(ws.value)


def _batch_workspace_many(items, q: int) -> int:
    """Workspace bytes of a batched plan of these items (host only)."""
    import ctypes

    L = _lib.load()
    arr = (_lib.BatchItem * len(items))()
    for a, item in zip(arr, items):
        a.m, a.n, a.lda = item["m"], item["n"], item.get("lda", item["n"])
        a.k, a.p, a.block = item["k"], item["p"], item["block"]
        a.g_col, a.g_row = item["g_col"], item["g_row"]
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    _lib.check(L.bcur_batch_plan(arr, len(items), q, None, ctypes.byref(h), ctypes.byref(ws)),
               "bcur_batch_plan")
    L.bcur_batch_destroy(h)
    return int(ws.value)


def _free_bytes(device) -> float:
    torch = _torch()
    free, _ = torch.cuda.mem_get_info(device)
    return float(free)


def latency_stats(done: List[_Req]) -> Dict[str, float]:
    lat = np.array([q.t_done - q.r.arrival for q in done])
    t_end = max(q.t_done for q in done)
    t_first = min(q.r.arrival for q in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "max_ms": float(lat.max() * 1e3),
            "decomps_per_s": len(done) / max(t_end - t_first, 1e-9)}
