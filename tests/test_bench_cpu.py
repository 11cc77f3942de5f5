"""Host logic of bench.py that needs no GPU: the recorded ncu traffic is
reported only while the profiled kernel source is unchanged."""
import copy

import bench


def test_measured_traffic_is_tied_to_the_kernel_source(monkeypatch):
    import hashlib
    import os
    root = os.path.dirname(os.path.abspath(bench.__file__))
    path = "paper_1607_02859_gb300/csrc/gw_tc.cu"
    with open(os.path.join(root, path), "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    # every recorded entry names a committed profile summary
    for k, r in bench.MEASURED_TRAFFIC.items():
        assert os.path.exists(os.path.join(root, r["profile"])), k
    key = ("w", "f16x3", "green_tc")
    rec = {key: {"bytes_per_launch": 1.0e9, "sources": {path: sha}, "profile": "profiles/x.md"}}
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", rec)
    assert bench.measured_traffic(*key) == 1.0e9
    assert bench.measured_traffic("w", "f16x3", "cgemm_tc") is None
    changed = copy.deepcopy(rec)
    changed[key]["sources"][path] = "0" * 40
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", changed)
    assert bench.measured_traffic(*key) is None


def test_flop_model_at_the_bench_size():
    # G formation 2 * 8 N_r^2 N_b per tau, screening 4 N_chi^3 per omega (si8)
    fl = bench.flop_model(13824, 1024, 16, 13824, 8)
    assert abs(fl["green"] - 2 * 8 * 13824 ** 2 * 1024 * 16) < 1
    assert abs(fl["dyson"] - 4 * 13824 ** 3 * 16) < 1


def _rank(rank, world, port, out_dir):
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [2.0, 5.0][rank]                       # the slowest rank decides the job's time
    t = bench.max_over_ranks(seconds, dist, device="cpu")
    v = bench.job_value(world, 1e12, 3, t)
    with open(os.path.join(out_dir, "r%d" % rank), "w") as f:
        f.write("%r %r" % (t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_timing_over_two_gloo_ranks(tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        t, v = (float(x) for x in (tmp_path / ("r%d" % r)).read_text().split())
        assert t == 5.0
        assert abs(v - 2 * 1e12 * 3 / 5.0 / 1e12) < 1e-12      # all ranks' work over the slowest time
    assert bench.max_over_ranks(7.0) == 7.0


def test_reference_arm_runs_on_rank_zero_only():
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "gamma_toy", "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_batch_mix_and_flops():
    from paper_1607_02859_gb300 import batch, inputs
    ps = inputs.batch_mix(4, seed=9)
    for p in ps:
        assert p.n[0] in (12, 16, 20, 24) and 128 <= p.n_b <= 1024 and p.n_b % 8 == 0
        assert p.n_occ == p.n_b // 8 and 8 <= len(p.tau) <= 16 and p.n_chi <= 2048
    # G formation dominates: 8 N_r^2 N_b per tau, once for chi0 and once for Sigma; agrees with the bench's model
    import bench
    f = batch.chain_flops(1728, 128, 8, 1728, 4)
    assert f > 2 * 8 * 8.0 * 1728 ** 2 * 128
    assert abs(f - bench.flop_model(1728, 128, 8, 1728, 4)["total"]) < 1e-9 * f
