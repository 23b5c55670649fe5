"""The benchmark's output contract, checked on the CPU: the reference arm (the FP64 oracle on a
bounded sample) prints exactly one JSON line with every field the contract asks for, and its
config is the one the GPU line builds for the same workload with the default launch options."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_json_line(monkeypatch):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # the GPU line's config for the same workload, default launch options
    sys.path.insert(0, ROOT)
    import bench
    from paper_2603_04070_gb300 import inputs
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    args.tile_z_used, args.two_step_used, args.persistent_used, args.groups_used = 32, 0, 0, 2
    wl = inputs.make_workload(args.workload, seed=0, nt=args.nt, n_tx=args.n_tx)
    assert d["config"] == json.loads(json.dumps(bench.workload_config(wl, args)))
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    """Launched as the multi-GPU bench is (torchrun, two ranks), the reference arm runs on rank 0
    alone: one JSON line with n_gpus = 2, and every rank exits 0."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_bench_counts_the_shot_groups_the_library_uses():
    """The benchmark's roofline divides a sweep's time by its steps through the number of shot
    groups a call uses: the option's value capped by the shots, and one group for the forms that
    walk every shot in one launch."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2603_04070_gb300 import dufwi
    opts = (dufwi.OPT_SHOT_GROUPS, dufwi.OPT_TWO_STEP, dufwi.OPT_PERSISTENT, dufwi.OPT_MULTI_TILE)
    saved = [dufwi.get_option(o) for o in opts]
    try:
        dufwi.set_option(dufwi.OPT_SHOT_GROUPS, 2)
        assert bench.effective_groups(dufwi, 16) == 2 and bench.effective_groups(dufwi, 1) == 1
        dufwi.set_option(dufwi.OPT_SHOT_GROUPS, 4)
        assert bench.effective_groups(dufwi, 3) == 3
        for o in opts[1:]:
            dufwi.set_option(o, 1)
            assert bench.effective_groups(dufwi, 16) == 1
            dufwi.set_option(o, 0)
    finally:
        for o, v in zip(opts, saved):
            dufwi.set_option(o, v)


def test_committed_traffic_records_match_the_kernel_source():
    """The committed per-launch DRAM traffic records were taken on the current one-step kernel
    source (their hash matches), and the benchmark scales them from the captured shots per launch
    to a step of all shots."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    with open(os.path.join(ROOT, "profiles", "ncu_traffic_scale.json")) as f:
        rs = json.load(f)
    sha = bench.step_kernel_source_sha256()
    assert rec["step_kernel_source_sha256"] == sha and rs["step_kernel_source_sha256"] == sha
    for kind in ("forward", "recompute", "adjoint"):
        per = rec["per_launch_dram_bytes_full_size"][kind]
        assert bench.kernel_traffic(kind, shots=16) == per * 16 / rec["shots_per_launch"]
        assert bench.scale_traffic(64)[kind] == rs["per_launch_dram_bytes_full_size"][kind] * 64 / rs["shots_per_launch"]
        # below the algorithmic bytes with warm L2: nothing is re-read from DRAM
        assert rec["per_launch_dram_bytes_warm_l2"][kind] < rec["algorithmic_bytes_per_launch"][kind]
