"""Continuous-batching likelihood server.

Requests for a log-likelihood, or a log-likelihood and its branch-length
gradient, arrive from many MCMC chains at any time. Each chain's data (tip
states, pattern weights, rate categories, its tree topology) lives in a
device-resident instance; a request brings a tree proposal (branch lengths)
and the substitution-model parameters to use (the device model is rebuilt
only when they differ from the chain's last ones). One scheduling
step:

1. completion: launch groups whose CUDA event has fired hand their results
   to the requests' futures and release their chains;
2. admission: queued requests are taken in arrival order, at most one per
   chain (a chain's buffers hold one evaluation at a time). A chain without
   a device instance is admitted when its partials memory fits the budget,
   or, once its request has waited a while, by evicting idle chains least
   recently used first; once a request is blocked on memory, no other
   chain is newly admitted ahead of it. A chain whose whole-tree buffers
   could never fit is served with subtree checkpointing (``checkpoint``:
   post-order partials kept at every few depths, recomputed in the
   pre-order pass; each request its own launch group on the chain's
   stream) when that form fits, and rejected otherwise;
3. launch: per request the model (when it changed) and the transition
   matrices; then every four-state request of the step goes through the
   batched calls (one launch per pass for all of them), and codon requests
   through their tensor-core passes on their chains' streams, so both
   kinds run on the GPU at once. Each group's results come back with one device-to-host
   copy.

The loop never waits for the GPU: a step is queued while earlier ones run,
so requests that arrive meanwhile join the next step. A reduced-precision
result that comes back non-finite (a pattern whose likelihood underflowed)
is evaluated again in FP64 before it is returned.
"""
from __future__ import annotations

import collections
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import TreeLikelihood
from ._lib import Batch
from .checkpoint import CheckpointedLikelihood, best_band

R_CATEGORIES = 4


def footprint(n_tips: int, n_patterns: int, n_states: int, precision: str,
              n_buffers: int | None = None) -> int:
    """Device bytes of a chain's instance (partials of 2(N-1) buffers, or
    ``n_buffers`` with checkpointing, their scale exponents, tip states and
    2(2N-1) matrix slots), with a 2% margin for scratch that grows with use."""
    N, R = n_tips, R_CATEGORIES
    if n_states == 4:
        ppad, spad = -(-n_patterns // 32) * 32, 4
    else:
        ppad, spad = -(-n_patterns // 128) * 128, 64
    elt = 8 if precision == "f64" else 4
    nb = 2 * (N - 1) if n_buffers is None else n_buffers
    partials = nb * R * ppad * spad * elt + nb * ppad * 4
    copies = 4 if precision in ("tf32x2", "tf32x3") else 2   # working copies per matrix slot
    mats = 2 * (2 * N - 1) * R * spad * spad * (8 + copies * elt)
    return int(1.02 * (partials + mats + N * ppad)) + (1 << 20)


@dataclass
class Result:
    logl: float
    gradient: np.ndarray | None
    latency: float       # seconds from arrival to the result on the host
    group_size: int      # requests launched together with this one


@dataclass
class _Chain:
    data: object                      # a synth.Workload-like dataset
    precision: str
    tl: TreeLikelihood | None = None
    bytes: int = 0
    busy: bool = False
    last_used: float = 0.0
    params: np.ndarray | None = None  # parameters currently on the device
    stream: object = None
    queued: int = 0
    band: int = 0                     # > 0: served with subtree checkpointing
    n_buffers: int | None = None


@dataclass
class _Pending:
    req: object
    future: Future
    arrival: float
    chain: int


@dataclass
class _Group:
    event: object
    items: list
    host: object
    arena: object
    offsets: list = field(default_factory=list)   # (logl index, grad index or -1, n_grad)


class Server:
    """Continuous-batching server over device-resident chains.

    ``memory_budget`` bounds the chains' instance bytes (default 80% of the
    device memory free at start). Four-state chains run in ``nuc_precision``
    (FP32 or FP64) through the batched calls; codon chains in
    ``codon_precision``, each on its own stream. A request whose chain is
    not resident evicts idle chains once it has waited ``evict_after``
    seconds (free memory is taken at once)."""

    def __init__(self, memory_budget: int | None = None, max_batch: int = 512,
                 nuc_precision: str = "f32", codon_precision: str = "tf32x3",
                 evict_after: float = 0.0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", torch.cuda.current_device())
        if memory_budget is None:
            memory_budget = int(0.8 * torch.cuda.mem_get_info()[0])
        self.budget = int(memory_budget)
        self.used = 0
        self.max_batch = max_batch
        self.evict_after = evict_after
        self.nuc_precision, self.codon_precision = nuc_precision, codon_precision
        self.stream = torch.cuda.Stream()
        self.batch = Batch(self.stream.cuda_stream)
        self.chains: list[_Chain] = []
        self.queue: collections.deque[_Pending] = collections.deque()
        self.inflight: list[_Group] = []
        self.stats = collections.Counter()
        self.group_sizes: list[int] = []
        # FP64 re-evaluations run on a worker thread (the library calls
        # release the interpreter lock) on a stream of their own, so the
        # scheduling loop keeps serving while one runs
        self._fb_pool = None
        self._fb_stream = None
        self._fallbacks: list = []   # (pending, group size, worker future, bytes, start)

    # chains ---------------------------------------------------------------
    def add_chain(self, data) -> int:
        prec = self.nuc_precision if data.n_states == 4 else self.codon_precision
        c = _Chain(data, prec)
        # every chain has its own stream: its uploads, matrices and (codon)
        # passes queue there, so admitting a chain never waits for other
        # chains' work; batched launches order themselves after each
        # chain's stream and each chain's stream after them (events)
        c.stream = self.torch.cuda.Stream()
        self.chains.append(c)
        return len(self.chains) - 1

    def need(self, k: int) -> int:
        c = self.chains[k]
        d = c.data
        return footprint(d.tree.n_tips, d.n_patterns, d.n_states, c.precision, c.n_buffers)

    def _create(self, k: int) -> None:
        c = self.chains[k]
        d = c.data
        if c.band:
            tl = CheckpointedLikelihood(d.tree.n_tips, d.n_patterns, d.tree.children, d.n_states,
                                        R_CATEGORIES, c.precision, band=c.band,
                                        stream=c.stream.cuda_stream)
            tl.set_data(d.tips, d.model, d.params, d.freqs, d.rates, d.cat_weights,
                        d.pattern_weights)
            c.tl, c.params = tl, np.asarray(d.params, dtype=float).copy()
            c.bytes = max(tl.inst.device_bytes(), self.need(k))
            self.used += c.bytes
            self.stats["admitted"] += 1
            return
        tl = TreeLikelihood(d.tree.n_tips, d.n_patterns, d.n_states, R_CATEGORIES, c.precision,
                            stream=c.stream.cuda_stream)
        tl.inst.set_tip_states_all(d.tips)
        tl.inst.set_model_async(0, d.model, d.params, d.freqs)
        tl.set_rates(d.rates, d.cat_weights)
        tl.set_pattern_weights(d.pattern_weights)
        tl.set_tree(d.tree.children, d.tree.edge_len)
        c.tl, c.params = tl, np.asarray(d.params, dtype=float).copy()
        c.bytes = max(tl.inst.device_bytes(), self.need(k))
        self.used += c.bytes
        self.stats["admitted"] += 1

    def _try_create(self, p: _Pending):
        """Create p's chain; on a device allocation failure evict every idle
        chain and retry once. True when created, False to wait, None when the
        request was failed (nothing else is resident to make room)."""
        from ._lib import TreelikError
        try:
            self._create(p.chain)
            return True
        except TreelikError:
            idle = [k for k, c in enumerate(self.chains) if c.tl is not None and not c.busy]
            for k in idle:
                self._evict(k)
            try:
                self._create(p.chain)
                return True
            except TreelikError as exc:
                if any(c.tl is not None for c in self.chains):
                    return False
                self.chains[p.chain].queued -= 1
                self.stats["rejected"] += 1
                p.future.set_exception(MemoryError(str(exc)))
                return None

    def _evict(self, k: int) -> None:
        c = self.chains[k]
        c.tl.close()
        c.tl = None
        self.used -= c.bytes
        c.bytes = 0
        self.stats["evicted"] += 1

    def _make_room(self, need: int) -> bool:
        """Evict idle chains (no request queued first, then least recently
        used) until ``need`` bytes fit; False if they cannot."""
        if self.used + need <= self.budget:
            return True
        idle = [k for k, c in enumerate(self.chains) if c.tl is not None and not c.busy]
        idle.sort(key=lambda k: (self.chains[k].queued > 0, self.chains[k].last_used))
        free = self.budget - self.used + sum(self.chains[k].bytes for k in idle)
        if free < need:
            return False
        for k in idle:
            if self.used + need <= self.budget:
                break
            self._evict(k)
        return self.used + need <= self.budget

    def preload(self) -> int:
        """Admit chains in order while they fit (a warm start); returns how
        many are resident."""
        for k in range(len(self.chains)):
            if self.chains[k].tl is None and self.used + self.need(k) <= self.budget:
                self._create(k)
        self.torch.cuda.synchronize()
        return sum(c.tl is not None for c in self.chains)

    # requests -------------------------------------------------------------
    def submit(self, req, arrival: float | None = None) -> Future:
        f: Future = Future()
        p = _Pending(req, f, time.perf_counter() if arrival is None else arrival, req.chain)
        c = self.chains[req.chain]
        if self.need(req.chain) > self.budget and not c.band:
            d = c.data
            band, nbuf = best_band(d.tree.children, d.tree.n_tips)
            if footprint(d.tree.n_tips, d.n_patterns, d.n_states, c.precision, nbuf) <= self.budget:
                c.band, c.n_buffers = band, nbuf
        if self.need(req.chain) > self.budget:
            self.stats["rejected"] += 1
            f.set_exception(MemoryError(
                f"chain {req.chain} needs {self.need(req.chain)} bytes, budget {self.budget}"))
            return f
        self.chains[req.chain].queued += 1
        self.queue.append(p)
        return f

    def pending(self) -> int:
        return (len(self.queue) + sum(len(g.items) for g in self.inflight) +
                len(self._fallbacks))

    def _complete(self) -> int:
        done = 0
        keep = []
        for g in self.inflight:
            if not g.event.query():
                keep.append(g)
                continue
            now = time.perf_counter()
            host = g.host.numpy()
            for p, off in zip(g.items, g.offsets):
                li, gi, ng = off[:3]
                nb = off[3] if len(off) > 3 else 1   # checkpointed: one vector per band
                c = self.chains[p.chain]
                c.busy = False
                c.last_used = now
                logl = float(host[li])
                grad = host[gi:gi + ng * nb].reshape(nb, ng).sum(axis=0) if gi >= 0 else None
                bad = not np.isfinite(logl) or (grad is not None and
                                                 not np.all(np.isfinite(grad)))
                if bad and c.precision != "f64":
                    # Reduced precision can lose a pattern entirely: one
                    # exponent per pattern spans all categories, so categories
                    # whose likelihoods differ by more than FP32's range at a
                    # node underflow, and two children may keep disjoint ones;
                    # and a gradient ratio's denominator (the pattern
                    # likelihood up to the scales of its factors) leaves the
                    # FP32 range when the pre-order partial and the subtree
                    # favour codons several changes apart. The request is
                    # evaluated again in FP64 on the worker (its latency
                    # includes that evaluation).
                    kind = "codon" if c.data.n_states > 4 else "nuc"
                    why = "logl" if not np.isfinite(logl) else "gradient"
                    self.stats[f"fp64_fallback_{kind}_{why}"] += 1
                    self._start_fallback(p, len(g.items))
                    done += 1
                    continue
                if not np.isfinite(logl):
                    p.future.set_exception(FloatingPointError("non-finite log-likelihood"))
                else:
                    p.future.set_result(Result(logl, grad, now - p.arrival, len(g.items)))
                done += 1
        self.inflight = keep
        # finished FP64 re-evaluations
        still = []
        for p, gsize, fut, extra, t0 in self._fallbacks:
            if not fut.done():
                still.append((p, gsize, fut, extra, t0))
                continue
            self.used -= extra
            now = time.perf_counter()
            self.stats["fp64_fallback_s"] += now - t0
            try:
                logl, grad = fut.result()
            except Exception:   # reported to the request as a failure below
                logl, grad = float("nan"), None
            if not np.isfinite(logl):
                p.future.set_exception(FloatingPointError("non-finite log-likelihood"))
            else:
                p.future.set_result(Result(logl, grad, now - p.arrival, gsize))
            done += 1
        self._fallbacks = still
        return done

    def _start_fallback(self, p: _Pending, gsize: int) -> None:
        """Queue the FP64 re-evaluation of p on the worker; its temporary
        instance counts against the memory budget from now until it is done
        (idle chains, p's own included, make room first; if even that is not
        enough the device allocation decides)."""
        import concurrent.futures as cf
        c = self.chains[p.chain]
        d = c.data
        self.stats["fp64_fallback"] += 1
        nbuf = c.n_buffers if c.band else None
        extra = footprint(d.tree.n_tips, d.n_patterns, d.n_states, "f64", nbuf)
        self._make_room(extra)
        self.used += extra
        if self._fb_pool is None:
            self._fb_pool = cf.ThreadPoolExecutor(max_workers=1)
            self._fb_stream = self.torch.cuda.Stream()
        dev, stream = self.dev, self._fb_stream

        def work():
            self.torch.cuda.set_device(dev)
            return self._fp64_eval(c, d, p.req, stream.cuda_stream)

        self._fallbacks.append((p, gsize, self._fb_pool.submit(work), extra,
                                time.perf_counter()))

    def _admit(self) -> list[_Pending]:
        picked, seen, rest = [], set(), collections.deque()
        blocked = False
        now = time.perf_counter()
        while self.queue:
            p = self.queue.popleft()
            c = self.chains[p.chain]
            ok = len(picked) < self.max_batch and not c.busy and p.chain not in seen
            if ok and c.tl is None:
                # a new chain takes free memory at once, but evicts others only
                # once its request has waited evict_after seconds, so that
                # resident chains keep their places while their requests flow
                need = self.need(p.chain)
                ok = not blocked and (self.used + need <= self.budget or
                                      (now - p.arrival >= self.evict_after and
                                       self._make_room(need)))
                if ok:
                    ok = self._try_create(p)
                    if ok is None:      # cannot be created even on an empty device
                        continue
                if not ok:
                    blocked = True   # keep memory for the oldest blocked chain
            if ok:
                picked.append(p)
                seen.add(p.chain)
                c.busy = True
                c.queued -= 1
            else:
                rest.append(p)
        self.queue = rest
        return picked

    def _prepare(self, p: _Pending) -> None:
        c = self.chains[p.chain]
        tl, d, r = c.tl, c.data, p.req
        if not np.array_equal(r.params, c.params):
            tl.inst.set_model_async(0, d.model, r.params, d.freqs)
            c.params = np.asarray(r.params, dtype=float).copy()
        tl.set_tree(d.tree.children, r.edge_len)
        tl.update_matrices(r.gradient)

    def _group(self, items, stream, launch) -> None:
        torch = self.torch
        n_grad = [self.chains[p.chain].tl.nn if p.req.gradient else 0 for p in items]
        offsets, pos = [], len(items)
        for i, ng in enumerate(n_grad):
            offsets.append((i, pos if ng else -1, ng))
            pos += ng
        with torch.cuda.stream(stream):
            arena = torch.empty(pos, dtype=torch.float64, device=self.dev)
        launch(arena, offsets)
        host = torch.empty(pos, dtype=torch.float64, pin_memory=True)
        with torch.cuda.stream(stream):
            host.copy_(arena, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.inflight.append(_Group(ev, items, host, arena, offsets))
        self.group_sizes.append(len(items))

    def _launch_nuc(self, items) -> None:
        tls = [self.chains[p.chain].tl for p in items]

        def launch(arena, offsets):
            base = arena.data_ptr()
            insts = [t.inst for t in tls]
            self.batch.update_partials(insts, [t._post for t in tls])
            self.batch.root_loglik_dev(insts, [t.nn - 1 for t in tls], [0] * len(tls), base)
            g = [(t, o) for t, o in zip(tls, offsets) if o[1] >= 0]
            if g:
                self.batch.pre_order_gradient_dev(
                    [t.inst for t, _ in g], [t._pre for t, _ in g], [0] * len(g),
                    [base + 8 * o[1] for _, o in g], [o[2] for _, o in g])

        self._group(items, self.stream, launch)

    def _launch_codon(self, items, stream) -> None:
        def launch(arena, offsets):
            base = arena.data_ptr()
            for p, o in zip(items, offsets):
                t = self.chains[p.chain].tl
                t.inst.update_partials(t._post)
                t.inst.root_loglik_dev(t.nn - 1, 0, base + 8 * o[0])
                if o[1] >= 0:
                    t.inst.pre_order_gradient_dev(t._pre, o[2], 0, base + 8 * o[1])

        self._group(items, stream, launch)

    def _fp64_eval(self, c, d, r, stream: int):
        """(logL, gradient or None) of request r of chain c on a temporary
        FP64 instance on ``stream`` (the calling thread waits); (nan, None)
        if that fails too."""
        from ._lib import TreelikError
        try:
            if c.band:   # a chain served with checkpointing keeps that form in FP64
                tl = CheckpointedLikelihood(d.tree.n_tips, d.n_patterns, d.tree.children,
                                            d.n_states, R_CATEGORIES, "f64", band=c.band,
                                            stream=stream)
            else:
                tl = TreeLikelihood(d.tree.n_tips, d.n_patterns, d.n_states, R_CATEGORIES,
                                    "f64", stream=stream)
        except TreelikError:
            return float("nan"), None
        try:
            if c.band:
                tl.set_data(d.tips, d.model, r.params, d.freqs, d.rates, d.cat_weights,
                            d.pattern_weights)
                if r.gradient:
                    return tl.gradient(r.edge_len)
                return tl.loglik(r.edge_len), None
            tl.inst.set_tip_states_all(d.tips)
            tl.set_model(d.model, r.params, d.freqs)
            tl.set_rates(d.rates, d.cat_weights)
            tl.set_pattern_weights(d.pattern_weights)
            tl.set_tree(d.tree.children, r.edge_len)
            if r.gradient:
                return tl.gradient()
            return tl.loglik(), None
        except TreelikError:
            return float("nan"), None
        finally:
            tl.close()

    def _launch_checkpointed(self, p: _Pending) -> None:
        """A checkpointed chain's request as its own launch group on the
        chain's stream: logL, then (gradient) one vector per band, summed on
        the host when the group completes."""
        c = self.chains[p.chain]
        d, r = c.data, p.req
        if not np.array_equal(r.params, c.params):
            c.tl.inst.set_model_async(0, d.model, r.params, d.freqs)
            c.params = np.asarray(r.params, dtype=float).copy()
        torch = self.torch
        nb = c.tl.n_bands() if r.gradient else 0
        n = 1 + nb * c.tl.nn
        with torch.cuda.stream(c.stream):
            arena = torch.empty(n, dtype=torch.float64, device=self.dev)
        c.tl.launch(r.edge_len, r.gradient, arena.data_ptr())
        host = torch.empty(n, dtype=torch.float64, pin_memory=True)
        with torch.cuda.stream(c.stream):
            host.copy_(arena, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(c.stream)
        self.inflight.append(_Group(ev, [p], host, arena,
                                    [(0, 1 if r.gradient else -1, c.tl.nn, nb)]))
        self.group_sizes.append(1)
        self.stats["checkpointed"] += 1

    def step(self) -> bool:
        """One scheduling step; True if anything completed or launched."""
        done = self._complete()
        picked = self._admit()
        if not picked:
            return done > 0
        for p in [q for q in picked if self.chains[q.chain].band]:
            self._launch_checkpointed(p)
        picked = [p for p in picked if not self.chains[p.chain].band]
        if not picked:
            return True
        for p in picked:
            self._prepare(p)
        nuc = [p for p in picked if self.chains[p.chain].data.n_states == 4]
        if nuc:
            self._launch_nuc(nuc)
        for p in picked:
            c = self.chains[p.chain]
            if c.data.n_states != 4:
                self._launch_codon([p], c.stream)
        self.stats["steps"] += 1
        return True

    def drain(self) -> None:
        while self.pending():
            if not self.step():
                time.sleep(20e-6)

    def close(self) -> None:
        if self._fb_pool is not None:
            self._fb_pool.shutdown(wait=True)
        self.torch.cuda.synchronize()
        for c in self.chains:
            if c.tl is not None:
                c.tl.close()
                c.tl = None
        self.batch.close()


def run_open_loop(server: Server, requests, arrivals) -> tuple[list, float]:
    """Submit request i at time arrivals[i] (seconds from the start, a
    Poisson process) while stepping the server; returns the futures and the
    makespan. Latency counts from the scheduled arrival, so host delays in
    the loop are charged to the requests."""
    n = len(requests)
    futs = [None] * n
    t0 = time.perf_counter()
    i = 0
    while i < n or server.pending():
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            futs[i] = server.submit(requests[i], arrival=t0 + arrivals[i])
            i += 1
        if not server.step():
            time.sleep(20e-6)
    return futs, time.perf_counter() - t0
