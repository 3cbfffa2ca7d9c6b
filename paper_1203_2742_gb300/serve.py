"""Request serving on one GPU: resident factors, admission by device-memory
footprint, continuous batching.

Requests (factor, gradient, Hessian with m right-hand sides, inverse Hessian,
completion) name one of the registered patterns.  Every pattern is analysed
once; its factor object, its completion object and their cached blocks stay
resident on the device, so later calls reuse them.  Worker threads each own a
CUDA stream and take requests as they arrive: requests that arrive while
others run are admitted as soon as a worker and enough device memory (the
footprint of the request's inputs, outputs and workspace, against a budget)
are free, and their kernels overlap on the device with the running ones.
A worker that takes a Hessian or inverse-Hessian request also takes the
waiting requests of the same kind for the same pattern and runs them as one
call with m = the sum of their right-hand sides (continuous batching).
Calls on one pattern are serialised by a per-pattern lock (a factor object
has one workspace); different patterns run concurrently.

With ``rhs_block`` set, a batch of Hessian-type requests runs in calls of
exactly ``rhs_block`` right-hand sides (the last one zero-padded) through
device and pinned host buffers that each pattern keeps, the gradient writes
a kept buffer, and the workspaces stay allocated: every call of a kind on a
pattern then has the same arguments, so from its third call on the library
replays it from a CUDA graph (one launch of the graph instead of the call's
kernel launches from the host); these factor objects capture sequences of up
to ``graph_limit`` launches.  This suits pools of small and medium patterns;
with very large ones (millions of nonzeros, hundreds of thousands of
launches per call) the padding, the captures and the kept workspaces cost
more than they save, and the plain path (the default) is faster.

The server computes through the C ABI only (the ``binding`` objects of the
registered patterns); it holds no numerical code of its own.  The trace
generator and the admission rule need no library (they are host logic).
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

OPS = ("factor", "gradient", "hessian", "inv_hessian", "completion")


@dataclass
class Request:
    op: str
    pattern: int
    arrival: float                      # seconds on the server clock
    data: object = None                 # host array (m, nnz) for hessian / inv_hessian
    m: int = 1
    rid: int = 0
    # filled by the server
    start: float = 0.0
    done: float = 0.0
    result: object = None
    batched_with: int = 1


@dataclass
class PatternState:
    sym: object
    x: object          # device values of X (fixed per pattern)
    s: object          # device values of S (fixed per pattern)
    fac: object = None
    cfac: object = None
    # kept buffers of the fixed-shape calls (rhs_block): device input and
    # output, pinned host staging, the gradient's output
    buf_in: object = None
    buf_out: object = None
    host_in: object = None
    host_out: object = None
    g_out: object = None
    lock: threading.Lock = field(default_factory=threading.Lock)
    busy: bool = False  # a worker runs a call on this pattern (guarded by Server.cv)
    ws_bytes_per_rhs: int = 0


class Server:
    """Continuous-batching server over resident factors.

    patterns: list of (Symbolic, x_host, s_host) -- values already on the
    analysed pattern.  workers: concurrent streams.  budget_bytes: device
    memory the in-flight requests may hold (inputs, outputs, workspace).
    batching: merge waiting same-pattern Hessian / inverse-Hessian requests.
    """

    def __init__(self, patterns, workers=8, budget_bytes=None, batching=True, max_batch_rhs=64,
                 keep_workspace_bytes=1 << 30, rhs_block=None, graph_limit=1 << 20):
        import torch
        self.torch = torch
        self.batching = batching
        self.max_batch_rhs = max_batch_rhs
        self.rhs_block = rhs_block
        self.graph_limit = graph_limit
        self.states = []
        for sym, x, s in patterns:
            d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
            st = PatternState(sym=sym, x=d(x), s=d(s))
            sp, par, rp, rows = sym.supernodes()
            nn, J = np.diff(sp), np.diff(rp)
            st.ws_bytes_per_rhs = int(8 * np.sum(J * J + 2 * J * nn))
            self.states.append(st)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(0.5 * free)
        self.budget = budget_bytes
        # per-request workspace cap: a worker's share of the budget; with kept
        # workspaces (rhs_block) every pattern keeps its own, so each gets a
        # pattern's share (the library then runs a call's right-hand sides in
        # chunks that fit)
        share = len(self.states) if rhs_block else workers
        self.ws_limit = max(1, budget_bytes // max(1, share))
        self.keep_ws = keep_workspace_bytes
        self.in_use = 0
        self.nworkers = workers
        self.cv = threading.Condition()
        self.queue = collections.deque()
        self.closed = False
        self.completed = []
        self.t0 = None
        self.threads = []

    # -- resident state -------------------------------------------------------
    def warm(self):
        """Factor every pattern once (resident factors) and cache S for Hessians."""
        torch = self.torch
        for st in self.states:
            st.fac = st.sym.factor(st.x)
            st.fac.set_workspace_limit(self.ws_limit)
            st.fac.gradient()
            st.cfac, _ = st.sym.complete(st.s)
            st.cfac.set_workspace_limit(self.ws_limit)
            if self.rhs_block:
                # fixed arguments per call kind: even the longest launch
                # sequences are captured once and replayed
                st.fac.set_graph_limit(self.graph_limit)
                st.cfac.set_graph_limit(self.graph_limit)
                b, nnz = self.rhs_block, st.sym.nnz
                st.buf_in = torch.zeros((b, nnz), dtype=torch.float64, device="cuda")
                st.buf_out = torch.empty((b, nnz), dtype=torch.float64, device="cuda")
                st.host_in = torch.zeros((b, nnz), dtype=torch.float64).pin_memory()
                st.host_out = torch.empty((b, nnz), dtype=torch.float64).pin_memory()
                st.g_out = torch.empty(nnz, dtype=torch.float64, device="cuda")
            else:
                for f in (st.fac, st.cfac):
                    if f.workspace_bytes() > self.keep_ws:
                        f.release_workspace()
        self.torch.cuda.synchronize()

    def footprint(self, req):
        """Device bytes a request may hold: its inputs and outputs and the
        workspace of the right-hand sides the library processes at once
        (it works in chunks of at most 48 GiB of workspace).  With kept
        buffers and workspaces (rhs_block) the request allocates nothing."""
        st = self.states[req.pattern]
        if self.rhs_block:
            return 0
        nnz = st.sym.nnz
        per = max(st.ws_bytes_per_rhs, 1)
        chunk = max(1, self.ws_limit // per)
        if req.op in ("hessian", "inv_hessian"):
            return 8 * 2 * req.m * nnz + min(req.m, chunk) * per
        return 8 * 2 * nnz + per

    # -- request flow ---------------------------------------------------------
    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, req):
        with self.cv:
            self.queue.append(req)
            self.cv.notify()

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()

    def _take(self):
        """Next admissible request plus its batch (see ``pick``); waits while
        nothing can be admitted."""
        with self.cv:
            while True:
                got = pick(self.queue, lambda p: self.states[p].busy, self.footprint, self.in_use, self.budget,
                           self.batching, self.max_batch_rhs)
                if got is not None:
                    group, need, self.queue = got
                    self.in_use += need
                    self.states[group[0].pattern].busy = True
                    return group, need
                if self.closed and not self.queue:
                    return None, 0
                self.cv.wait(timeout=0.05)

    def _release(self, need, pattern):
        with self.cv:
            self.in_use -= need
            self.states[pattern].busy = False
            self.cv.notify_all()

    def run(self, req, stream=None):
        """Serve one request now, on `stream` (default: the current stream),
        outside the queue: the same code path a worker takes for a batch of
        one.  Fills req.start, req.done and req.result and returns the result."""
        if self.t0 is None:
            self.t0 = time.perf_counter()
        self._run_group([req], stream if stream is not None else self.torch.cuda.current_stream())
        return req.result

    def _run_group(self, group, stream):
        torch = self.torch
        req = group[0]
        st = self.states[req.pattern]
        nnz = st.sym.nnz
        with st.lock, torch.cuda.stream(stream):
            start = self.now()
            if req.op == "factor":
                st.fac.refactor(st.x, stream=stream)
                res = [st.fac.logdet()]
            elif req.op == "gradient":
                g = st.g_out if st.g_out is not None else torch.empty(nnz, dtype=torch.float64, device="cuda")
                st.fac.gradient(out=g, stream=stream)
                res = [g.cpu().numpy()]
            elif req.op == "completion":
                res = [st.cfac.recomplete(st.s, stream=stream)]
            elif self.rhs_block:
                res = self._run_blocks(st, group, req.op, stream)
            else:
                host = np.concatenate([r.data.reshape(r.m, nnz) for r in group], axis=0)
                inp = torch.as_tensor(host, dtype=torch.float64).pin_memory().to("cuda", non_blocking=True)
                out = torch.empty_like(inp)
                if req.op == "hessian":
                    st.fac.hessian(inp, out=out, stream=stream)
                else:
                    st.fac.inv_hessian(inp, out=out, stream=stream)
                allr = out.cpu().numpy()
                res, o = [], 0
                for r in group:
                    res.append(allr[o:o + r.m])
                    o += r.m
            stream.synchronize()
            # keep the resident memory of idle patterns small (kept buffers:
            # the workspaces stay, so that the next call replays its graph)
            if not self.rhs_block:
                for f in (st.fac, st.cfac):
                    if f.workspace_bytes() > self.keep_ws:
                        f.release_workspace()
            done = self.now()
        for r, v in zip(group, res if len(res) == len(group) else res * len(group)):
            r.start, r.done, r.result, r.batched_with = start, done, v, len(group)

    def _run_blocks(self, st, group, op, stream):
        """The group's right-hand sides in calls of exactly rhs_block through
        the pattern's kept buffers (zero rows pad the last call)."""
        b, nnz = self.rhs_block, st.sym.nnz
        host = np.concatenate([r.data.reshape(r.m, nnz) for r in group], axis=0)
        out = np.empty_like(host)
        hin, hout = st.host_in.numpy(), st.host_out.numpy()
        call = st.fac.hessian if op == "hessian" else st.fac.inv_hessian
        for r0 in range(0, host.shape[0], b):
            mc = min(b, host.shape[0] - r0)
            hin[:mc] = host[r0:r0 + mc]
            if mc < b:
                hin[mc:] = 0.0
            st.buf_in.copy_(st.host_in, non_blocking=True)
            call(st.buf_in, out=st.buf_out, stream=stream)
            st.host_out.copy_(st.buf_out, non_blocking=True)
            stream.synchronize()
            out[r0:r0 + mc] = hout[:mc]
        res, o = [], 0
        for r in group:
            res.append(out[o:o + r.m])
            o += r.m
        return res

    def _worker(self):
        torch = self.torch
        stream = torch.cuda.Stream()
        while True:
            group, need = self._take()
            if group is None:
                return
            try:
                self._run_group(group, stream)
            except Exception as e:  # a failed request must not stop the worker
                t = self.now()
                for r in group:
                    r.start, r.done, r.result, r.batched_with = t, t, e, len(group)
            finally:
                self._release(need, group[0].pattern)
                with self.cv:
                    self.completed.extend(group)

    def start(self):
        self.t0 = time.perf_counter()
        for _ in range(self.nworkers):
            t = threading.Thread(target=self._worker, daemon=True)
            t.start()
            self.threads.append(t)

    def join(self):
        self.close()
        for t in self.threads:
            t.join()

    def free(self):
        """Drop the resident factors and kept buffers (the worker threads
        must have finished)."""
        self.threads = []
        for st in self.states:
            st.fac = st.cfac = None
            st.buf_in = st.buf_out = st.host_in = st.host_out = st.g_out = None
        self.states = []


def pick(queue, busy, footprint, in_use, budget, batching, max_batch_rhs):
    """Admission and batching decision of the server (host logic only).

    The first request in FIFO order whose pattern is idle (``busy(pattern)``
    false) and whose footprint fits the budget (or that comes when nothing is
    in flight) is taken; when batching, the waiting Hessian or
    inverse-Hessian requests of the same kind on the same pattern join it
    while their right-hand sides total at most ``max_batch_rhs``.  Returns
    (group, bytes, remaining queue), or None when nothing can be admitted.
    A request on a busy pattern stays queued, so a worker never waits for a
    pattern another worker is running.
    """
    for i, req in enumerate(queue):
        if busy(req.pattern):
            continue
        need = footprint(req)
        if in_use + need > budget and in_use != 0:
            continue
        rest = collections.deque(r for j, r in enumerate(queue) if j != i)
        group = [req]
        if batching and req.op in ("hessian", "inv_hessian"):
            rhs = req.m
            keep = collections.deque()
            while rest:
                r2 = rest.popleft()
                if r2.op == req.op and r2.pattern == req.pattern and rhs + r2.m <= max_batch_rhs:
                    group.append(r2)
                    rhs += r2.m
                    need += footprint(r2)
                else:
                    keep.append(r2)
            rest = keep
        return group, need, rest
    return None


def poisson_trace(npatterns, rate, duration, mix, rng, nnz_of, max_m=16):
    """Requests with exponential inter-arrival times (rate per second) over
    `duration` seconds; op drawn from `mix` (dict op -> probability), pattern
    uniform; Hessian-type requests carry m ~ U{1..max_m} right-hand sides
    uniform[-1, 1] on the pattern."""
    ops = list(mix)
    p = np.array([mix[o] for o in ops], dtype=np.float64)
    p /= p.sum()
    t, out, rid = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        op = ops[rng.choice(len(ops), p=p)]
        pat = int(rng.integers(npatterns))
        m = int(rng.integers(1, max_m + 1)) if op in ("hessian", "inv_hessian") else 1
        data = rng.uniform(-1.0, 1.0, size=(m, nnz_of(pat))) if op in ("hessian", "inv_hessian") else None
        out.append(Request(op=op, pattern=pat, arrival=t, data=data, m=m, rid=rid))
        rid += 1
    return out


def replay(server, trace):
    """Feed the trace at its arrival times, wait for every request, and return
    latency statistics (seconds) and served throughput."""
    server.start()
    for req in trace:
        delay = req.arrival - server.now()
        if delay > 0:
            time.sleep(delay)
        server.submit(req)
    server.join()
    done = sorted(server.completed, key=lambda r: r.rid)
    failed = [r for r in done if isinstance(r.result, Exception)]
    lat = np.array([r.done - r.arrival for r in done])
    wall = max(r.done for r in done) - min(r.arrival for r in done)
    hess = sum(r.m for r in done if r.op == "hessian")
    evals = sum(r.m for r in done)
    return {"requests": len(done), "wall_s": wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "hessian_evals_per_s": hess / wall,
            "evals_per_s": evals / wall, "requests_per_s": len(done) / wall,
            "mean_batch": float(np.mean([r.batched_with for r in done])), "failed": len(failed)}, done
