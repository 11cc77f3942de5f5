"""Serving form of the hot path: a continuous-batching request server.

Requests ask for chi0(G,G',i omega) or for Sigma_nn(i omega) (the whole chain:
chi0 -> W~ -> inverse CT -> Sigma_nn with its Thiele continuation) of systems
of different grid sizes, band counts and time grids.  Systems are registered
once: their orbitals, eigenvalues, time/frequency grids and transform matrices
stay resident on the device.

Scheduling: FIFO.  A request is admitted as soon as a slot (a worker thread
with its own libgw context and CUDA stream) is idle and the HBM footprint of
everything in flight -- each worker's scratch arena (sized by
gw_workspace_size) plus the request's output buffers -- stays within the
budget.  Requests that arrive while others run are admitted the moment a slot
and memory free up, and their kernels overlap with the running ones on the
device (one stream per slot; the C calls release the Python GIL).  Every
request records arrival, start and completion times, from which the server
reports requests/s and p50/p99 latency.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import gw


@dataclass
class System:
    """A registered system, resident on the device."""

    name: str
    grid: object
    psi: object                 # torch tensor [N_b][N_r] on the device
    eps: np.ndarray
    n_occ: int
    mu: float
    tau: np.ndarray
    omega: np.ndarray
    mats: dict                  # C, S, Cinv
    gvec: np.ndarray
    fidx: np.ndarray
    bands: np.ndarray
    n_r: int
    n_chi: int
    prec: str
    r_block: int = 0
    w_real: np.ndarray = field(default_factory=lambda: np.linspace(-1.0, 1.0, 16))
    # frequency-independent part of the QP equation per band of `bands`
    # (<T + V_ne + V_H> + bare exchange); None: the Kohn-Sham energies
    vstat: np.ndarray = None

    @property
    def n_b(self) -> int:
        return int(self.psi.shape[0])

    def scratch_bytes(self) -> int:
        """Arena bytes a context needs to serve this system (largest call)."""
        return max(gw.workspace_size(self.grid, self.n_b, self.n_occ, len(self.tau), self.n_chi, len(self.bands),
                                     self.prec, self.r_block))

    def input_bytes(self) -> int:
        return int(self.psi.numel() * self.psi.element_size())

    def output_bytes(self, kind: str) -> int:
        es = 16 if self.prec == "fp64" else 8
        per = len(self.tau) * self.n_chi * self.n_chi * es
        return per if kind == "chi0" else 2 * per


def register(problem, prec, device=0, r_block=0, n_chi=None) -> System:
    """Upload a problem (inputs.Problem) and its host setup; keep it resident."""
    import torch
    grid = gw.make_grid(problem.n, problem.lattice)
    nchi = int(n_chi or problem.n_chi)
    gvec, fidx = gw.g_set(grid, nchi)
    mats = gw.fit_transform(problem.tau, problem.omega, problem.x_min, problem.x_max, problem.n_x, problem.ridge)
    psi = torch.from_numpy(np.ascontiguousarray(problem.psi)).to(device=f"cuda:{device}", dtype=gw.cdtype(prec))
    return System(problem.name, grid, psi, np.asarray(problem.eps), problem.n_occ, problem.mu,
                  np.asarray(problem.tau), np.asarray(problem.omega), mats, gvec, fidx, np.asarray(problem.bands),
                  problem.n_r, nchi, prec, r_block)


@dataclass
class Request:
    system: System
    kind: str                   # "chi0" or "sigma"
    rid: int = 0
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    result: object = None
    error: str = ""
    reserved: int = 0

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def run_request(ctx, req: Request, stream, keep_chi=False):
    """Run one request on `stream` through the C ABI; returns its result
    (chi0 tensor on the device for "chi0" when keep_chi, else its Frobenius norm;
    for "sigma", the sigma_diag dict with the QP energies, Z and spectral
    functions on w_real + mu under "qp")."""
    import torch
    s = req.system
    n = len(s.tau)
    with torch.cuda.stream(stream):
        chi = torch.empty((n, s.n_chi, s.n_chi), dtype=gw.cdtype(s.prec), device=s.psi.device)
        gw.chi0_omega(ctx, s.grid, s.psi, s.eps, s.n_occ, s.mu, s.tau, s.mats["C"], s.fidx, s.prec, chi,
                      r_block=s.r_block)
        if req.kind == "chi0":
            out = chi if keep_chi else float(torch.linalg.vector_norm(chi).item())
            stream.synchronize()
            return out
        gw.screen_W(ctx, s.grid, s.gvec, s.prec, chi, chi, resid=False)
        w_tau = torch.empty_like(chi)
        gw.tau_to_omega(ctx, gw.CT, s.mats["Cinv"], chi, w_tau, s.prec)
        del chi
        out = gw.sigma_diag(ctx, s.grid, s.psi, s.eps, s.n_occ, s.mu, s.bands, s.tau, s.omega, s.mats["C"],
                            s.mats["S"], w_tau, s.fidx, s.prec, w_real=s.w_real)
        eps_n = s.eps[s.bands]
        out["qp"] = gw.qp_energies(ctx, s.omega, out["sigma_iw"], eps_n, s.mu,
                                   eps_n if s.vstat is None else s.vstat, w=s.w_real + s.mu)
        stream.synchronize()
        return out


class GpuSlot:
    """The device side of one slot: its own libgw context and CUDA stream."""

    def __init__(self, device=0, keep_chi=False):
        import torch
        self.ctx = gw.Context(device)
        self.stream = torch.cuda.Stream(device=device)
        self.keep_chi = keep_chi

    def run(self, req):
        return run_request(self.ctx, req, self.stream, keep_chi=self.keep_chi)

    def arena_bytes(self):
        return self.ctx.scratch_bytes

    def reserve(self, nbytes):
        self.ctx.reserve(nbytes)

    def close(self):
        self.ctx.close()


class _Worker:
    """One slot: a thread that runs the requests the server hands it."""

    def __init__(self, server, index, slot):
        self.server = server
        self.index = index
        self.slot = slot
        self.arena = 0               # scratch bytes this slot's arena holds (grow-only)
        self.job = None
        self.alive = True
        self.cv = threading.Condition()
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def _loop(self):
        while True:
            with self.cv:
                while self.job is None and self.alive:
                    self.cv.wait()
                if self.job is None:
                    return
                req = self.job
            req.t_start = time.perf_counter()
            try:
                req.result = self.slot.run(req)
            except Exception as e:            # reported per request; the server keeps going
                req.error = repr(e)
            req.t_done = time.perf_counter()
            self.server._finished(self, req)

    def give(self, req):
        with self.cv:
            self.job = req
            self.cv.notify()

    def stop(self):
        with self.cv:
            self.alive = False
            self.cv.notify()
        self.thread.join()
        self.slot.close()


class Server:
    """n_slots workers, FIFO admission by device-memory footprint under budget_bytes.

    make_slot(i) builds slot i (an object with run(req), arena_bytes() and
    close()); the default is a GpuSlot on `device`."""

    def __init__(self, n_slots=4, budget_bytes=150 << 30, device=0, keep_chi=False, make_slot=None):
        if n_slots < 1:
            raise ValueError("n_slots must be >= 1")
        self.budget = int(budget_bytes)
        self.lock = threading.Condition()
        self.pending = collections.deque()
        self.done = []
        self.inflight_bytes = 0       # output buffers of running requests
        self.resident = {}            # id(system) -> resident input bytes
        self.running = 0
        self.max_concurrent = 0
        self.next_id = 0
        make_slot = make_slot or (lambda i: GpuSlot(device, keep_chi))
        self.workers = [_Worker(self, i, make_slot(i)) for i in range(n_slots)]

    @staticmethod
    def footprint(worker_arena, scratch, outputs):
        """Device bytes a request adds when run on a slot whose arena holds worker_arena."""
        return max(0, scratch - worker_arena) + outputs

    def held_bytes(self):
        """Device bytes held now: slot arenas, outputs in flight, resident inputs."""
        return sum(w.arena for w in self.workers) + self.inflight_bytes + sum(self.resident.values())

    def prepare(self, systems):
        """Size every idle slot's arena for the largest of `systems` up front,
        as far as the budget allows, so that no arena grows (a device-wide
        synchronisation) while requests are in flight."""
        need = max(s.scratch_bytes() for s in systems)
        with self.lock:
            for w in self.workers:
                if w.job is None and w.arena < need and self.held_bytes() - w.arena + need <= self.budget:
                    w.slot.reserve(need)
                    w.arena = max(need, w.slot.arena_bytes())

    def submit(self, system, kind):
        if kind not in ("chi0", "sigma"):
            raise ValueError("kind must be 'chi0' or 'sigma'")
        with self.lock:
            req = Request(system, kind, rid=self.next_id, t_arrival=time.perf_counter())
            self.next_id += 1
            if system.scratch_bytes() + system.output_bytes(kind) + system.input_bytes() > self.budget:
                req.error = "request needs more device memory than the server budget"
                req.t_start = req.t_done = req.t_arrival
                self.done.append(req)
                return req
            self.pending.append(req)
            self._admit()
            return req

    def _admit(self):
        # FIFO: the head waits for a slot and memory rather than being overtaken
        while self.pending:
            idle = [w for w in self.workers if w.job is None and w.alive]
            if not idle:
                return
            head = self.pending[0]
            scratch = head.system.scratch_bytes()
            outs = head.system.output_bytes(head.kind)
            res = 0 if id(head.system) in self.resident else head.system.input_bytes()
            w = min(idle, key=lambda x: (self.footprint(x.arena, scratch, outs), x.index))
            grow = self.footprint(w.arena, scratch, outs) + res
            if self.running and self.held_bytes() + grow > self.budget:
                return
            self.pending.popleft()
            w.arena = max(w.arena, scratch)
            self.resident[id(head.system)] = head.system.input_bytes()
            head.reserved = outs
            self.inflight_bytes += outs
            self.running += 1
            self.max_concurrent = max(self.max_concurrent, self.running)
            w.give(head)

    def _finished(self, worker, req):
        with self.lock:
            worker.arena = max(worker.arena, worker.slot.arena_bytes())
            with worker.cv:
                worker.job = None
            self.inflight_bytes -= req.reserved
            self.running -= 1
            self.done.append(req)
            self._admit()
            self.lock.notify_all()

    def drain(self, timeout=None):
        """Wait until every submitted request has finished."""
        t0 = time.perf_counter()
        with self.lock:
            while self.pending or self.running:
                left = None if timeout is None else timeout - (time.perf_counter() - t0)
                if left is not None and left <= 0:
                    raise TimeoutError("requests still pending")
                self.lock.wait(left)

    def stats(self, reqs=None):
        """requests/s over the span from first arrival to last completion, and latency percentiles."""
        reqs = [r for r in (self.done if reqs is None else reqs) if not r.error]
        if not reqs:
            return {"requests": 0}
        lat = np.array([r.latency for r in reqs])
        span = max(r.t_done for r in reqs) - min(r.t_arrival for r in reqs)
        return {"requests": len(reqs), "req_per_s": len(reqs) / span if span > 0 else float("nan"),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "max_concurrent": self.max_concurrent}

    def close(self):
        for w in self.workers:
            w.stop()


def poisson_run(server, systems, rate, n_requests, kinds=("chi0", "sigma"), seed=5):
    """Submit n_requests at Poisson arrival times (rate req/s), each on a system
    and kind drawn uniformly (seeded); wait for all of them; return them."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_requests)
    picks = rng.integers(0, len(systems), n_requests)
    kind_picks = rng.integers(0, len(kinds), n_requests)
    reqs = []
    t0 = time.perf_counter()
    t_next = t0
    for i in range(n_requests):
        t_next += gaps[i]
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        reqs.append(server.submit(systems[picks[i]], kinds[kind_picks[i]]))
    server.drain()
    return reqs


def _burst(server, systems, picks):
    """All requests at once: saturation throughput."""
    reqs = [server.submit(systems[i], k) for (i, k) in picks]
    server.drain()
    return reqs


def _warm(server, systems):
    server.prepare(systems)
    for s in systems:                       # one untimed request per system
        server.submit(s, "sigma")
    big = max(systems, key=lambda s: s.output_bytes("sigma"))
    for _ in server.workers:                # and the largest outputs once on every slot's stream
        server.submit(big, "sigma")
    server.drain()
    server.done.clear()
    server.max_concurrent = 0


def main(argv=None):
    """Serving runs over a mix of systems; prints JSON lines."""
    import argparse
    import json
    from . import inputs
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--prec", default="f16x3", choices=["fp64", "fp32", "f16x3", "bf16x3"])
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--rates", default="8", help="comma-separated mean arrival rates (req/s) for Poisson runs")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--systems", default="mix", help="'mix' or comma-separated workload names")
    ap.add_argument("--mix-count", type=int, default=6)
    ap.add_argument("--compare-fp64", type=int, default=0, metavar="N",
                    help="also serve N burst requests through the plain FP64 path and compare Sigma")
    args = ap.parse_args(argv)
    problems = (inputs.serve_mix(args.mix_count) if args.systems == "mix"
                else [getattr(inputs, name)() for name in args.systems.split(",")])
    systems = [register(p, args.prec) for p in problems]
    names = [s.name for s in systems]
    budget = int(args.budget_gb * (1 << 30))
    server = Server(args.slots, budget)
    rng = np.random.default_rng(7)
    n_cmp = args.compare_fp64 or 16
    picks = [(int(rng.integers(0, len(systems))), ("chi0", "sigma")[int(rng.integers(0, 2))]) for _ in range(n_cmp)]
    try:
        _warm(server, systems)
        first = [server.submit(s, "sigma") for s in systems]
        server.drain()
        mixed_sigma = {i: r.result["sigma_iw"] for i, r in enumerate(first) if not r.error}
        server.done.clear()
        reqs = _burst(server, systems, picks)
        st = server.stats(reqs)
        st.update({"run": "burst", "prec": args.prec, "slots": args.slots, "systems": names})
        print(json.dumps(st), flush=True)
        for rate in [float(x) for x in args.rates.split(",") if x]:
            server.done.clear()
            server.max_concurrent = 0
            reqs = poisson_run(server, systems, rate, args.requests)
            st = server.stats(reqs)
            st.update({"run": "poisson", "rate": rate, "prec": args.prec, "slots": args.slots,
                       "errors": [r.error for r in reqs if r.error][:3],
                       "held_gb": server.held_bytes() / (1 << 30)})
            print(json.dumps(st), flush=True)
    finally:
        server.close()
    if not args.compare_fp64:
        return
    import torch
    del systems
    torch.cuda.empty_cache()
    ref = [register(p, "fp64") for p in problems]
    server = Server(args.slots, budget)
    try:
        _warm(server, ref)
        reqs = _burst(server, ref, picks)
        st = server.stats(reqs)
        fp64_sigma = {}
        for (i, k), r in zip(picks, reqs):
            if k == "sigma" and not r.error:
                fp64_sigma[i] = r.result["sigma_iw"]
        for i, s in enumerate(ref):
            if i not in fp64_sigma:
                r = server.submit(s, "sigma")
                server.drain()
                fp64_sigma[i] = r.result["sigma_iw"]
        dev = {names[i]: float(np.max(np.abs(mixed_sigma[i] - fp64_sigma[i])) / 3.674932e-5) for i in mixed_sigma}
        st.update({"run": "burst", "prec": "fp64", "slots": args.slots,
                   "sigma_max_dev_mev_%s_vs_fp64" % args.prec: dev})
        print(json.dumps(st), flush=True)
    finally:
        server.close()


if __name__ == "__main__":
    main()
