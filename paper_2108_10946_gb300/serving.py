"""Continuous-batching shot server over resident meshes.

Shot requests (a source position and wavelet on one of several resident meshes; forward
only, or forward + adjoint + gradient against observed records) arrive at any time. Worker
threads, each with its own CUDA stream, repeatedly take the oldest pending request's mesh,
pack up to ``max_batch`` of its pending requests into one batch (one launch sequence for
all of them: the shots are lanes of the same kernels), and run it. A batch is admitted only
if its device memory (``fwi_batch_bytes``) fits the remaining HBM budget; resident batches
are reused across requests (``fwi_batch_set_sources``), so memory is allocated once per
(mesh, batch size). Requests that arrive while other batches are on the GPU are admitted as
soon as a worker and memory are free, and their work overlaps on the device with the
batches already running (distinct streams, the GIL released during library calls).

The shots of a batch are independent lanes of the same kernels, so a request's result does
not depend on which other requests share its batch (up to the summation order of
floating-point atomics).

Everything numerical runs in the CUDA library; this module only schedules.
"""
import collections
import threading
import time

import numpy as np


class Request:
    __slots__ = ("rid", "mesh", "src", "wavelet", "observed", "arrival", "start", "done",
                 "records", "gradient", "misfit", "error", "event")

    def __init__(self, rid, mesh, src, wavelet, observed=None, arrival=None):
        self.rid = rid
        self.mesh = mesh
        self.src = np.asarray(src, dtype=np.float64)
        self.wavelet = np.asarray(wavelet, dtype=np.float32)
        self.observed = None if observed is None else np.asarray(observed, dtype=np.float32)
        self.arrival = time.perf_counter() if arrival is None else arrival
        self.start = None
        self.done = None
        self.records = None
        self.gradient = None
        self.misfit = None
        self.error = None
        self.event = threading.Event()

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class ShotServer:
    """meshes: {name: (paper_2108_10946_gb300.Mesh, receivers [R][dim])}."""

    def __init__(self, meshes, hbm_budget_bytes, max_batch=4, workers=2, torch_streams=True):
        import torch
        self.torch = torch
        self.meshes = meshes
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.max_batch = max_batch
        self.pending = collections.OrderedDict((name, collections.deque()) for name in meshes)
        self.cv = threading.Condition()
        self.pool = {}            # (mesh, S) -> list of idle Batch objects
        self.nbytes = {}          # (mesh, S) -> device bytes of one such batch
        self.stop = False
        self.completed = []
        self.streams = [torch.cuda.Stream() for _ in range(workers)] if torch_streams else [None] * workers
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                        for i in range(workers)]
        self.device = torch.cuda.current_device()
        for t in self.threads:
            t.start()

    # -- client side ------------------------------------------------------------------
    def submit(self, req):
        with self.cv:
            self.pending[req.mesh].append(req)
            self.cv.notify_all()
        return req

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()
        for batches in self.pool.values():
            for b in batches:
                b.close()

    # -- scheduling ---------------------------------------------------------------------
    def _take(self):
        """Oldest pending request's mesh, up to max_batch of its requests, and a resident
        batch: an idle one of the largest size that the pending requests need, else a new
        one if the HBM budget allows, else the next smaller size. Idle batches of other
        (mesh, size) pairs are closed to make room when nothing else fits. Returns None when
        every candidate must wait for a running batch. Called with the lock held."""
        oldest = None
        for name, q in self.pending.items():
            if q and (oldest is None or q[0].arrival < self.pending[oldest][0].arrival):
                oldest = name
        if oldest is None:
            return None
        q = self.pending[oldest]
        n = min(len(q), self.max_batch)
        S = 1
        while S < n:
            S *= 2
        mesh, recs = self.meshes[oldest]
        batch, key = None, None
        sizes = []
        while S >= 1:
            sizes.append(S)
            S //= 2
        for s2 in sizes:  # an idle resident batch first (no allocation)
            if self.pool.get((oldest, s2)):
                key = (oldest, s2)
                batch = self.pool[key].pop()
                break
        if batch is None:
            for s2 in sizes:  # else a new one that fits, evicting idle batches if needed
                need = mesh.batch_bytes(s2, len(recs))
                if need > self.budget:
                    continue
                self._evict_until(need, keep=(oldest, s2))
                if self.used + need <= self.budget:
                    self.used += need
                    self.nbytes[(oldest, s2)] = need
                    key = (oldest, s2)
                    break
            if key is None:
                if mesh.batch_bytes(1, len(recs)) > self.budget:
                    r = q.popleft()  # can never run: report instead of waiting forever
                    r.error = MemoryError("a one-shot batch of this mesh exceeds the HBM budget")
                    r.done = time.perf_counter()
                    r.event.set()
                    self.completed.append(r)
                return None
        n = min(n, key[1])
        # at most one gradient request per batch (the batch gradient sums over its shots)
        reqs, keep, have_grad = [], collections.deque(), False
        while q and len(reqs) < n:
            r = q.popleft()
            if r.observed is not None and have_grad:
                keep.append(r)
                continue
            have_grad |= r.observed is not None
            reqs.append(r)
        while keep:
            q.appendleft(keep.pop())
        return oldest, key[1], key, batch, reqs

    def _evict_until(self, need, keep):
        """Close idle resident batches (not of ``keep``) until ``need`` bytes fit."""
        for k in list(self.pool):
            if k == keep:
                continue
            while self.pool[k] and self.used + need > self.budget:
                self.pool[k].pop().close()
                self.used -= self.nbytes[k]

    def _worker(self, wi):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = self.streams[wi]
        import paper_2108_10946_gb300 as pkg
        while True:
            with self.cv:
                job = None
                while not self.stop:
                    job = self._take()
                    if job is not None:
                        break
                    self.cv.wait(timeout=0.05)
                if job is None:
                    return
            name, S, key, batch, reqs = job
            mesh, recs = self.meshes[name]
            try:
                self._run(pkg, mesh, recs, S, key, batch, reqs, stream)
            except Exception as e:  # report per request, keep serving
                for r in reqs:
                    r.error = e
                    r.done = time.perf_counter()
                    r.event.set()
                with self.cv:
                    self.completed.extend(reqs)
                    self.cv.notify_all()

    def _run(self, pkg, mesh, recs, S, key, batch, reqs, stream):
        src = np.stack([r.src for r in reqs] + [reqs[0].src] * (S - len(reqs)))
        if batch is None:
            try:
                batch = pkg.Batch(mesh, src, recs)
            except Exception:
                with self.cv:
                    self.used -= self.nbytes[key]
                raise
        try:
            batch.set_sources(src)
            self._run_batch(mesh, recs, S, batch, reqs, stream)
        finally:
            with self.cv:  # the batch stays resident for the next requests
                self.pool.setdefault(key, []).append(batch)
                self.cv.notify_all()

    def _run_batch(self, mesh, recs, S, batch, reqs, stream):
        torch = self.torch
        n = len(reqs)
        nt = mesh.nsteps
        R = len(recs)
        now = time.perf_counter()
        for r in reqs:
            r.start = now
        wav = np.zeros((S, nt), dtype=np.float32)
        for i, r in enumerate(reqs):
            wav[i] = r.wavelet[:nt]
        ctx = torch.cuda.stream(stream) if stream is not None else _null()
        with ctx:
            rec_d = torch.empty((S, nt + 1, R), device="cuda")
            wav_d = torch.from_numpy(wav).cuda(non_blocking=False)
            batch.forward(wav_d, rec_d, stream=stream)
            grad_reqs = [i for i, r in enumerate(reqs) if r.observed is not None]
            if grad_reqs:
                obs = rec_d.clone()  # lanes without observed data get a zero residual
                for i in grad_reqs:
                    obs[i] = torch.from_numpy(reqs[i].observed).cuda()
                for i in range(n, S):
                    obs[i] = rec_d[i]
                for i in range(n):
                    if reqs[i].observed is None:
                        obs[i] = rec_d[i]
                batch.adjoint_misfit(obs, stream=stream)
                G = torch.empty(mesh.N, dtype=torch.float64, device="cuda")
                J = batch.gradient(G, stream=stream)
                Gh = G.cpu().numpy()
            recs_h = rec_d.cpu().numpy()
        done = time.perf_counter()
        for i, r in enumerate(reqs):
            r.records = recs_h[i]
            if r.observed is not None:
                # the batch gradient is summed over its shots; with one gradient request per
                # batch it is that request's own (the scheduler keeps them apart below)
                r.gradient = Gh
                r.misfit = J
            r.done = done
            r.event.set()
        with self.cv:
            self.completed.extend(reqs)
            self.cv.notify_all()

    # -- reporting ---------------------------------------------------------------------
    def stats(self):
        lat = np.array([r.latency for r in self.completed if r.latency is not None and r.error is None])
        if len(lat) == 0:
            return {}
        t0 = min(r.arrival for r in self.completed)
        t1 = max(r.done for r in self.completed)
        return {"shots": int(len(lat)), "shots_per_s": float(len(lat) / (t1 - t0)),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean())}


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
