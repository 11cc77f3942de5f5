"""Host logic of the request server: FIFO admission, slot concurrency, the
device-memory budget, per-request errors and latency statistics.  The slots
are fakes that sleep instead of launching kernels."""
import threading
import time

import numpy as np
import pytest

from paper_1607_02859_gb300.serve import Request, Server

GB = 1 << 30


class FakeSystem:
    def __init__(self, name, scratch, out, inp=0, t=0.05):
        self.name, self.scratch, self.out, self.inp, self.t = name, scratch, out, inp, t

    def scratch_bytes(self):
        return self.scratch

    def output_bytes(self, kind):
        return self.out if kind == "chi0" else 2 * self.out

    def input_bytes(self):
        return self.inp


class FakeSlot:
    def __init__(self, log, server_ref, fail_on=None):
        self.log, self.server_ref, self.fail_on, self.arena = log, server_ref, fail_on, 0

    def run(self, req):
        srv = self.server_ref[0]
        with srv.lock:
            self.log.append(("start", req.rid, srv.running, srv.held_bytes()))
        self.arena = max(self.arena, req.system.scratch_bytes())
        time.sleep(req.system.t)
        if self.fail_on is not None and req.system.name == self.fail_on:
            raise RuntimeError("slot failure")
        return req.rid

    def arena_bytes(self):
        return self.arena

    def reserve(self, nbytes):
        self.arena = max(self.arena, nbytes)

    def close(self):
        pass


def make(n_slots, budget, fail_on=None):
    log, ref = [], [None]
    srv = Server(n_slots, budget, make_slot=lambda i: FakeSlot(log, ref, fail_on))
    ref[0] = srv
    return srv, log


def test_single_slot_is_fifo():
    srv, log = make(1, 100 * GB)
    try:
        sys_ = FakeSystem("a", GB, GB, t=0.01)
        reqs = [srv.submit(sys_, "chi0") for _ in range(6)]
        srv.drain(timeout=10)
        starts = [e[1] for e in log if e[0] == "start"]
        assert starts == [r.rid for r in reqs]
        assert all(r.result == r.rid for r in reqs)
        assert srv.max_concurrent == 1
    finally:
        srv.close()


def test_concurrency_reaches_slot_count():
    srv, log = make(4, 1000 * GB)
    try:
        sys_ = FakeSystem("a", GB, GB, t=0.2)
        reqs = [srv.submit(sys_, "sigma") for _ in range(8)]
        srv.drain(timeout=10)
        assert srv.max_concurrent == 4
        assert max(e[2] for e in log) == 4
        # the second wave starts only once the first frees its slots
        t_first = sorted(r.t_done for r in reqs)[0]
        assert sorted(r.t_start for r in reqs)[4] >= t_first - 1e-3
    finally:
        srv.close()


def test_budget_bounds_held_memory():
    # each request: 10 GB scratch + 2*5 GB outputs; budget 45 GB fits two slots' worth
    budget = 45 * GB
    srv, log = make(4, budget)
    try:
        sys_ = FakeSystem("a", 10 * GB, 5 * GB, inp=2 * GB, t=0.05)
        reqs = [srv.submit(sys_, "sigma") for _ in range(10)]
        srv.drain(timeout=20)
        assert all(r.error == "" for r in reqs)
        assert srv.max_concurrent == 2
        assert max(e[3] for e in log) <= budget
    finally:
        srv.close()


def test_arenas_are_reused_before_growing_another():
    # after one slot has grown to 30 GB, a 30 GB request goes to it (no growth)
    budget = 60 * GB
    srv, log = make(3, budget)
    try:
        big = FakeSystem("big", 30 * GB, GB, t=0.02)
        for _ in range(4):
            srv.submit(big, "chi0")
            srv.drain(timeout=10)
        assert sorted(w.arena for w in srv.workers) == [0, 0, 30 * GB]
    finally:
        srv.close()


def test_head_of_line_is_not_overtaken():
    # a request that does not fit yet holds back the smaller ones behind it
    budget = 40 * GB
    srv, log = make(3, budget)
    try:
        small = FakeSystem("small", 5 * GB, GB, t=0.3)
        big = FakeSystem("big", 30 * GB, GB, t=0.01)
        r0 = srv.submit(small, "chi0")
        r1 = srv.submit(big, "chi0")           # 5+1 held, big needs 31 more: 37 <= 40, admitted
        r2 = srv.submit(big, "chi0")           # would need another 31: waits
        r3 = srv.submit(small, "chi0")         # fits by itself but is behind r2
        srv.drain(timeout=10)
        order = [e[1] for e in log if e[0] == "start"]
        assert order.index(r2.rid) < order.index(r3.rid)
        assert all(r.error == "" for r in (r0, r1, r2, r3))
    finally:
        srv.close()


def test_oversize_request_is_rejected_and_errors_are_per_request():
    srv, log = make(2, 20 * GB, fail_on="bad")
    try:
        huge = FakeSystem("huge", 30 * GB, GB)
        bad = FakeSystem("bad", GB, GB, t=0.01)
        ok = FakeSystem("ok", GB, GB, t=0.01)
        rh = srv.submit(huge, "chi0")
        rb = srv.submit(bad, "chi0")
        ro = srv.submit(ok, "sigma")
        srv.drain(timeout=10)
        assert "budget" in rh.error
        assert "slot failure" in rb.error
        assert ro.error == "" and ro.result == ro.rid
        assert srv.stats()["requests"] == 1
        with pytest.raises(ValueError):
            srv.submit(ok, "other")
    finally:
        srv.close()


def test_stats_percentiles():
    srv, _ = make(1, GB)
    try:
        reqs = []
        for i in range(100):
            r = Request(None, "chi0", rid=i, t_arrival=float(i), t_start=float(i), t_done=float(i) + (i + 1) * 1e-3)
            reqs.append(r)
        st = srv.stats(reqs)
        lat = np.arange(1, 101) * 1e-3
        assert st["requests"] == 100
        assert abs(st["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-9
        assert abs(st["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-9
        assert abs(st["req_per_s"] - 100 / (99 + 0.1)) < 1e-9
    finally:
        srv.close()


def test_submit_from_many_threads():
    srv, log = make(3, 1000 * GB)
    try:
        sys_ = FakeSystem("a", GB, GB, t=0.005)
        got = []
        lk = threading.Lock()

        def client():
            for _ in range(10):
                r = srv.submit(sys_, "chi0")
                with lk:
                    got.append(r)

        th = [threading.Thread(target=client) for _ in range(5)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        srv.drain(timeout=20)
        assert len(got) == 50 and len({r.rid for r in got}) == 50
        assert all(r.result == r.rid for r in got)
        assert srv.running == 0 and srv.inflight_bytes == 0
    finally:
        srv.close()


def test_autotune_candidates_and_cache(tmp_path):
    import os
    from paper_1607_02859_gb300 import autotune, gw
    if not os.path.exists(gw.LIB_PATH):
        pytest.skip("libgw not built")
    grid = gw.make_grid((12, 12, 12), np.diag([10.0, 10.0, 10.0]))
    all_ = autotune.feasible(grid, 128, 16, 8, 400, "fp32")
    assert all_ == [256, 512, 1024, 1728]          # clipped to N_r = 1728
    need = [gw.workspace_size(grid, 128, 16, 8, 400, 1, "fp32", rb)[0] for rb in all_]
    assert need == sorted(need)                    # the arena grows with the block
    assert autotune.feasible(grid, 128, 16, 8, 400, "fp32", budget_bytes=need[1]) == all_[:2]
    p = str(tmp_path / "rb.json")
    k = autotune.key((12, 12, 12), 128, 16, 8, 400, "fp32", "dev")
    autotune.store(p, {k: {"r_block": 512, "ms": {"512": 1.0}}})
    assert autotune.load(p)[k]["r_block"] == 512
    assert autotune.load(str(tmp_path / "none.json")) == {}


def test_prepare_sizes_arenas_within_budget():
    srv, log = make(3, 50 * GB)
    try:
        a = FakeSystem("a", 10 * GB, GB)
        b = FakeSystem("b", 20 * GB, GB)
        srv.prepare([a, b])
        assert sorted(w.arena for w in srv.workers) == [0, 20 * GB, 20 * GB]   # a third would pass 50 GB
        r = srv.submit(b, "chi0")
        srv.drain(timeout=10)
        assert r.error == "" and sorted(w.arena for w in srv.workers) == [0, 20 * GB, 20 * GB]
    finally:
        srv.close()
