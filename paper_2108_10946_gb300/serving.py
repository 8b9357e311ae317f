"""Continuous-batching shot server over resident meshes.

Shot requests (a source position and wavelet on one of several resident meshes; forward
only, or forward + adjoint + gradient against observed records) arrive at any time. Worker
threads, each with its own CUDA stream, serve them from resident batches (the shots of a
batch are lanes of the same kernels, Section 4.5); a batch is created only if its device
memory (``fwi_batch_bytes``) fits the remaining HBM budget, and it stays resident for later
requests (``fwi_batch_set_sources``), so memory is allocated once per (mesh, batch size).

Two kinds of job:

* rolling forward batches. Forward-only requests of a mesh share one batch whose lanes
  advance together in segments of ``segment`` time steps (``fwi_forward_segment``; by default
  the mesh's checkpoint stride or a 16th of the record, whichever is longer), sized for the
  waiting requests. At every segment boundary the lanes whose shots have reached
  the end of their record are handed back, and pending requests start in the free lanes
  (their state reset in the same call), so a request joins a batch that is part way through
  other shots' records instead of waiting for them to finish.
* gradient batches. Requests with observed records are packed, up to ``max_batch`` of one
  mesh, into one forward + adjoint launch sequence; ``fwi_gradient_lanes`` returns each
  shot's own gradient and misfit, so any number of gradient requests share a batch.

A lane's arithmetic does not depend on the other lanes, so a request's result is the same
alone and in the mix (up to the summation order of floating-point atomics). Requests that
arrive while other work is on the GPU are admitted as soon as a lane, a worker and memory
are free; work of different workers overlaps on the device (distinct streams, the GIL
released during library calls).

Everything numerical runs in the CUDA library; this module only schedules.
"""
import collections
import threading
import time

import numpy as np


class Request:
    __slots__ = ("rid", "mesh", "src", "wavelet", "observed", "arrival", "start", "done",
                 "records", "gradient", "misfit", "error", "event", "mid_record")

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
        self.mid_record = False  # started in a lane while other lanes were part way through

    @property
    def wants_gradient(self):
        return self.observed is not None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class ShotServer:
    """meshes: {name: (paper_2108_10946_gb300.Mesh, receivers [R][dim])}. rolling=False serves
    forward requests in whole-record batches as well (one launch sequence per batch)."""

    def __init__(self, meshes, hbm_budget_bytes, max_batch=4, workers=2, torch_streams=True,
                 rolling=True, segment=None):
        import torch
        self.torch = torch
        self.meshes = meshes
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.max_batch = max_batch
        self.rolling = rolling
        self.segment = segment
        self.pending = collections.OrderedDict((name, collections.deque()) for name in meshes)
        self.cv = threading.Condition()
        self.pool = {}            # (mesh, S) -> list of idle Batch objects
        self.nbytes = {}          # (mesh, S) -> device bytes of one such batch
        self.rolling_free = collections.Counter()  # mesh -> free lanes of its rolling batches
        self.idle = 0             # workers waiting for work
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

    def submit_many(self, reqs):
        """Submit several requests at once (a worker sees all of them or none)."""
        with self.cv:
            for r in reqs:
                self.pending[r.mesh].append(r)
            self.cv.notify_all()
        return reqs

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()
        for batches in self.pool.values():
            for b in batches:
                b.close()

    # -- scheduling (called with the lock held) -------------------------------------------
    def _oldest(self, exclude_mesh=None):
        """The oldest request that a new job must serve. A mesh's first F pending forward
        requests, F the free lanes of its running rolling batches, wait for those batches'
        next segment boundary instead (rolling mode)."""
        best = None
        for name, q in self.pending.items():
            skip = self.rolling_free[name] if self.rolling else 0
            for r in q:
                if self.rolling and not r.wants_gradient:
                    if name == exclude_mesh:
                        continue
                    if skip > 0:
                        skip -= 1
                        continue
                if best is None or r.arrival < best.arrival:
                    best = r
                break  # queues are in arrival order
        return best

    def _demand(self, name):
        """Lanes for a new rolling batch of mesh `name`: the forward requests it would fill
        now, at most max_batch (rounded up to a power of two by the caller; the lanes that
        leaves free take requests arriving during the record). A spare lane on top was
        measured slower: an idle lane costs about as much as a busy one."""
        n = sum(1 for r in self.pending[name] if not r.wants_gradient)
        return max(1, min(self.max_batch, n - self.rolling_free[name]))

    def _acquire(self, name, S):
        """A resident batch of mesh `name` with S lanes or fewer: an idle one of the largest
        size first, else a new one that fits the budget (idle batches of other sizes closed to
        make room). Returns (key, batch or None to create) or None if nothing fits now."""
        mesh, recs = self.meshes[name]
        sizes = []
        while S >= 1:
            sizes.append(S)
            S //= 2
        for s2 in sizes:
            if self.pool.get((name, s2)):
                return (name, s2), self.pool[(name, s2)].pop()
        for s2 in sizes:
            need = mesh.batch_bytes(s2, len(recs))
            if need > self.budget:
                continue
            self._evict_until(need, keep=(name, s2))
            if self.used + need <= self.budget:
                self.used += need
                self.nbytes[(name, s2)] = need
                return (name, s2), None
        return None

    def _fail_unfittable(self, name, q):
        mesh, recs = self.meshes[name]
        if mesh.batch_bytes(1, len(recs)) > self.budget:
            r = q.popleft()  # can never run: report instead of waiting forever
            r.error = MemoryError("a one-shot batch of this mesh exceeds the HBM budget")
            r.done = time.perf_counter()
            r.event.set()
            self.completed.append(r)

    def _take(self):
        """The next job for an idle worker: for the oldest eligible request, a rolling forward
        batch of its mesh or a gradient batch of up to max_batch of its mesh's gradient
        requests. Returns None when every candidate must wait."""
        r0 = self._oldest()
        if r0 is None:
            return None
        name, q = r0.mesh, self.pending[r0.mesh]
        roll = self.rolling and not r0.wants_gradient
        if roll:  # sized by the demand now: idle lanes would cost as much as busy ones
            n = self._demand(name)
        else:
            n = min(self.max_batch, sum(1 for r in q if r.wants_gradient or not self.rolling))
        S = 1
        while S < n:
            S *= 2
        got = self._acquire(name, S)
        if got is None:
            self._fail_unfittable(name, q)
            return None
        key, batch = got
        if roll:
            self.rolling_free[name] += key[1]
            return "roll", name, key, batch, [], r0.src
        reqs, keep = [], collections.deque()
        while q and len(reqs) < key[1]:
            r = q.popleft()
            if self.rolling and not r.wants_gradient:
                keep.append(r)
                continue
            reqs.append(r)
        while keep:
            q.appendleft(keep.pop())
        return "batch", name, key, batch, reqs, reqs[0].src

    def _admit(self, name, free):
        """Pending forward requests of mesh `name` for `free` lanes of its rolling batch, in
        arrival order. A request older than all of them elsewhere keeps them waiting unless a
        worker is idle to serve it, so that one mesh's stream cannot starve the others."""
        q = self.pending[name]
        out, keep = [], collections.deque()
        while q and len(out) < free:
            r = q.popleft()
            if r.wants_gradient:
                keep.append(r)
                continue
            other = self._oldest(exclude_mesh=name)
            if other is not None and other.arrival < r.arrival and self.idle == 0:
                keep.append(r)
                break
            out.append(r)
        while keep:
            q.appendleft(keep.pop())
        return out

    def _evict_until(self, need, keep):
        """Close idle resident batches (not of ``keep``) until ``need`` bytes fit."""
        for k in list(self.pool):
            if k == keep:
                continue
            while self.pool[k] and self.used + need > self.budget:
                self.pool[k].pop().close()
                self.used -= self.nbytes[k]

    def _release(self, key, batch):
        with self.cv:  # the batch stays resident for the next requests
            if batch is not None:
                self.pool.setdefault(key, []).append(batch)
            else:
                self.used -= self.nbytes[key]
            self.cv.notify_all()

    def _finish(self, reqs):
        with self.cv:
            self.completed.extend(reqs)
            self.cv.notify_all()

    # -- workers --------------------------------------------------------------------------
    def _worker(self, wi):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = self.streams[wi]
        import paper_2108_10946_gb300 as pkg
        while True:
            with self.cv:
                job = None
                self.idle += 1
                while not self.stop:
                    job = self._take()
                    if job is not None:
                        break
                    self.cv.wait(timeout=0.05)
                self.idle -= 1
                if job is None:
                    return
            kind, name, key, batch, reqs, src = job
            mesh, recs = self.meshes[name]
            try:
                if batch is None:
                    batch = pkg.Batch(mesh, np.tile(src, (key[1], 1)), recs)
            except Exception as e:
                self._release(key, None)
                if kind == "roll":
                    with self.cv:
                        self.rolling_free[name] -= key[1]
                self._fail(reqs, e)
                continue
            if kind == "roll":
                self._run_rolling(name, mesh, recs, key, batch, src, stream)
            else:
                try:
                    self._run_batch(mesh, recs, key[1], batch, reqs, stream)
                except Exception as e:  # report per request, keep serving
                    self._fail(reqs, e)
                self._release(key, batch)

    def _fail(self, reqs, e):
        for r in reqs:
            r.error = e
            r.done = time.perf_counter()
            r.event.set()
        self._finish(reqs)

    def _run_rolling(self, name, mesh, recs, key, batch, src0, stream):
        S = key[1]
        nt, R = mesh.nsteps, len(recs)
        # default segment: the checkpoint stride, or a 16th of the record if that is longer
        # (every boundary costs a host round trip; a 16th keeps admission waits short)
        nseg = self.segment or max(getattr(mesh.params, "ckpt_stride", 0) or 50, -(-nt // 16))
        nseg = max(1, min(int(nseg), nt))
        lanes = [None] * S  # [request, own time step t] per lane
        srcs = np.tile(np.asarray(src0, dtype=np.float64), (S, 1))  # idle lanes: any point inside
        wav = np.zeros((S, nseg), dtype=np.float32)
        rec = np.zeros((S, nseg + 1, R), dtype=np.float32)
        while True:
            with self.cv:
                free = [i for i in range(S) if lanes[i] is None]
                new = self._admit(name, len(free)) if not self.stop else []
                self.rolling_free[name] -= len(new)
                if not new and len(free) == S:
                    self.rolling_free[name] -= S
                    self.cv.notify_all()
                    break
            reset = 0
            now = time.perf_counter()
            busy = any(ln is not None and ln[1] > 0 for ln in lanes)
            for i, r in zip(free, new):
                r.start = now
                r.mid_record = busy
                r.records = np.zeros((nt + 1, R), dtype=np.float32)
                lanes[i] = [r, 0]
                srcs[i] = r.src
                reset |= 1 << i
            try:
                if reset:  # idle lanes keep their last source position (zero wavelet)
                    batch.set_sources(srcs)
                for i in range(S):
                    wav[i] = 0.0
                    if lanes[i] is not None:
                        r, t = lanes[i]
                        w = r.wavelet[t:min(t + nseg, nt)]
                        wav[i, :len(w)] = w
                batch.forward_segment(nseg, reset, wav, rec, stream=stream)
            except Exception as e:
                failed = [ln[0] for ln in lanes if ln is not None]
                with self.cv:
                    self.rolling_free[name] += len(failed)
                self._fail(failed, e)
                lanes = [None] * S
                continue
            done = []
            t_done = time.perf_counter()
            for i in range(S):
                if lanes[i] is None:
                    continue
                r, t = lanes[i]
                m = min(nseg, nt - t)
                r.records[t:t + m + 1] = rec[i, :m + 1]
                t += nseg
                if t >= nt:
                    r.done = t_done
                    r.event.set()
                    done.append(r)
                    lanes[i] = None
                else:
                    lanes[i][1] = t
            if done:
                with self.cv:
                    self.rolling_free[name] += len(done)
                self._finish(done)
        self._release(key, batch)

    def _run_batch(self, mesh, recs, S, batch, reqs, stream):
        torch = self.torch
        n = len(reqs)
        nt = mesh.nsteps
        R = len(recs)
        now = time.perf_counter()
        for r in reqs:
            r.start = now
        src = np.stack([r.src for r in reqs] + [reqs[0].src] * (S - n))
        batch.set_sources(src)
        wav = np.zeros((S, nt), dtype=np.float32)
        for i, r in enumerate(reqs):
            wav[i] = r.wavelet[:nt]
        ctx = torch.cuda.stream(stream) if stream is not None else _null()
        with ctx:
            rec_d = torch.empty((S, nt + 1, R), device="cuda")
            wav_d = torch.from_numpy(wav).cuda(non_blocking=False)
            batch.forward(wav_d, rec_d, stream=stream)
            grad_reqs = [i for i, r in enumerate(reqs) if r.wants_gradient]
            if grad_reqs:
                obs = rec_d.clone()  # lanes without observed data get a zero residual
                for i in grad_reqs:
                    obs[i] = torch.from_numpy(reqs[i].observed).cuda()
                batch.set_gradient_lanes(True)
                batch.adjoint_misfit(obs, stream=stream)
                G = torch.empty((S, mesh.N), dtype=torch.float64, device="cuda")
                J = batch.gradient_lanes(G, stream=stream)
                Gh = G.cpu().numpy()
            recs_h = rec_d.cpu().numpy()
        done = time.perf_counter()
        for i, r in enumerate(reqs):
            r.records = recs_h[i]
            if r.wants_gradient:
                r.gradient = Gh[i]  # this shot's own gradient and misfit
                r.misfit = float(J[i])
            r.done = done
            r.event.set()
        self._finish(reqs)

    # -- reporting ---------------------------------------------------------------------
    def stats(self):
        ok = [r for r in self.completed if r.latency is not None and r.error is None]
        if not ok:
            return {}
        lat = np.array([r.latency for r in ok])
        t0 = min(r.arrival for r in self.completed)
        t1 = max(r.done for r in self.completed)
        out = {"shots": int(len(lat)), "shots_per_s": float(len(lat) / (t1 - t0)),
               "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
               "mean_s": float(lat.mean()),
               "admitted_mid_record": int(sum(r.mid_record for r in ok))}
        for kind, sel in (("forward", False), ("gradient", True)):
            l2 = np.array([r.latency for r in ok if r.wants_gradient == sel])
            if len(l2):
                out[kind] = {"shots": int(len(l2)), "p50_s": float(np.percentile(l2, 50)),
                             "p99_s": float(np.percentile(l2, 99))}
        return out


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False
