#!/usr/bin/env python
"""Benchmark of the Poseidon-12 / Goldilocks Merkle build on GB300.

One step = one whole Merkle tree (Sec. 4.2) over 2^22 synthetic leaf rows of
8 Goldilocks words: leaf sponge hashing in one persistent launch, then every
level up to the root (one launch per level of more than 64 nodes, one cluster
launch for the rest) -- 8,388,607 permutations.  The rows (256 MiB) stay
resident in HBM; they are larger than the 129 MB L2, so no flush is needed
between steps (smaller trees, --log-n, get a 512 MiB write between steps,
outside the timed brackets).

Printed (rank 0, one JSON line): throughput in permutations/s over the
whole job, the build time in ms, the roofline of the kernel against the
integer-multiply pipe, an end-to-end figure through the C ABI with the rows
copied from pinned host memory every step, GPU clocks sampled during the
timed region, and the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poseidon-12 perms/s and 2^22-leaf Merkle build ms; % of IMAD roofline"
# 32-bit multiply results of one permutation in the optimised form with the
# dense 12x12 MDS: S-boxes 118*(2*6+2*8) + full-round MDS 8*144*8 +
# partial-round sparse layers 22*23*8.
MUL_RESULTS_PER_PERM = 118 * (2 * 6 + 2 * 8) + 8 * 144 * 8 + 22 * 23 * 8
# pg12_small: the seven full rounds with the 8-bit matrix take two 32x8-bit
# IMAD.WIDE per term (4 results); round 3's transition matrix stays full width.
MUL_RESULTS_PER_PERM_SMALL = 118 * (2 * 6 + 2 * 8) + 7 * 144 * 4 + 144 * 8 + 22 * 23 * 8
# In the one-thread-per-state kernels a permutation whose capacity cells enter
# as zero (node compressions, the first chunk of a sponge) skips 4 S-boxes and
# 48 products of round 0, and one whose result is a digest (nodes, the last
# chunk of a sponge) computes 4 of the 12 rows of the last dense layer (96
# products fewer): the results such launches execute are fewer than the
# algorithmic count above, which the roofline keeps as its unit of work.
ZCAP_SAVED = 4 * (2 * 6 + 2 * 8) + 48 * 8
ZCAP_SAVED_SMALL = 4 * (2 * 6 + 2 * 8) + 48 * 4
DIGEST_SAVED = 96 * 8
DIGEST_SAVED_SMALL = 96 * 4
ZCAP_KERNELS = ("k_merkle", "k_merkle_level", "k_hash_rows", "k_tc_sponge:leaves", "k_tc_sponge:level",
                "k_tc_sponge:rows")
LEVEL_KERNELS = ("k_merkle_level", "k_tc_sponge:level")
LEAF_KERNELS = ("k_merkle", "k_merkle_top_leaf", "k_tc_sponge:leaves")
IMAD_RESULTS_PER_CLK_SM = 64  # 32-bit multiply results per clock per SM
L2_BYTES = 129 * 10**6  # GB300 L2
def algorithmic_bytes(kernel, perms_per_launch, width):
    """Bytes a launch must move: rows read and digests written (leaves), or two
    child digests read and one written per node (levels)."""
    if kernel in LEAF_KERNELS:
        leaves = perms_per_launch // max(1, (width + 7) // 8)
        return leaves * (8 * width + 32)
    return perms_per_launch * 96


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log-n", type=int, default=22)
    ap.add_argument("--width", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", choices=["merkle", "permute", "batch", "serve", "lde"], default="merkle",
                    help="merkle (default): one 2^log_n-leaf tree per step; permute: 2^24 raw "
                         "permutations; batch: 64 mixed trees, one graph launch vs one launch per "
                         "tree; serve: Poisson stream of tree-build requests; lde: low-degree "
                         "extension of a trace, then its Merkle commitment")
    ap.add_argument("--lde-log-n", type=int, default=21)
    ap.add_argument("--permute-log-n", type=int, default=24, help="log2 of the states of the permute workload")
    ap.add_argument("--log-blowup", type=int, default=1)
    ap.add_argument("--trees", type=int, default=64)
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--max-log-n", type=int, default=22)
    ap.add_argument("--server-order", type=int, default=0, help="tree order inside a served batch: 0 arrival, 1 most work first")
    ap.add_argument("--params", default=None, help="built-in parameter set: pg12_v1 (default) or pg12_small")
    ap.add_argument("--engine", choices=["tensor", "int"], default="tensor",
                    help="permutation engine: tensor-core dense layers (default) or integer pipes only")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the other workloads (permute, width-64 tree, batch, serve, LDE) of the default run")
    ap.add_argument("--serve-low-rate", type=float, default=50.0)
    ap.add_argument("--serve-low-requests", type=int, default=500)
    return ap.parse_args()


def workload(log_n, width):
    n = 1 << log_n
    chunks = max(1, (width + 7) // 8)
    perms = n * chunks + (n - 1)
    name = f"merkle 2^{log_n} leaves x width {width}: leaf sponge + all levels to the root"
    return n, perms, name


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------ measured kernel metrics
METRICS = os.path.join(ROOT, "profiles", "kernel_metrics.json")


def kernel_metrics() -> dict:
    """ncu figures of the current kernels (profiles/kernel_metrics.json): pipe
    utilisation, instructions per permutation and DRAM bytes per launch.  Empty
    when the kernel sources changed since they were captured (stale counters
    are not reported)."""
    import hashlib
    try:
        with open(METRICS) as f:
            m = json.load(f)
        h = hashlib.sha256()
        for rel in m["source_files"]:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        return m if h.hexdigest() == m["source_sha256"] else {}
    except Exception:
        return {}


def metrics_kernel(name: str) -> str:
    return name.split(":")[0]


# ------------------------------------------------------------ stored oracle results
GOLDEN = os.path.join(ROOT, "tests", "golden", "full_size.json")


def goldens() -> dict:
    try:
        with open(GOLDEN) as f:
            return json.load(f)
    except Exception:
        return {}


def sha256_words(t) -> str:
    import hashlib
    import numpy as np
    a = t.detach().cpu().numpy() if not isinstance(t, np.ndarray) else t
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint64).astype("<u8").tobytes()).hexdigest()


def golden_tree(log_n, width, params=None):
    """Stored oracle result of the single-tree workload of this shape, if any."""
    if params not in (None, "pg12_v1"):
        return None
    return goldens().get(f"merkle_2e{log_n}_w{width}")


def tree_matches(nodes, entry) -> bool:
    import numpy as np
    root = [int(v) for v in nodes[-1].cpu().numpy().view(np.uint64)]
    return root == [int(v, 16) for v in entry["root"]] and sha256_words(nodes) == entry["nodes_sha256"]


# ------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.lines = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ oracle timing
def host_cpu_model() -> str:
    """lscpu's model name of the host (or /proc/cpuinfo's), for the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_permute_rates(seconds=4.0):
    """Single-thread and all-core permutations/s of the CPU oracle on random states."""
    import oracle
    import pg_synth
    cores = os.cpu_count() or 1
    out = {}
    for label, threads in (("single_thread", 1), ("all_core", cores)):
        n = 256 * threads
        while True:
            st = pg_synth.matrix(0x5EED0002, n, 12)
            t0 = time.perf_counter()
            oracle.permute(st, nthreads=threads)
            dt = time.perf_counter() - t0
            if dt >= seconds / 4 or n >= (1 << 22):
                out[label] = {"perms_per_s": n / dt, "threads": threads, "sample_states": n, "seconds": dt}
                break
            n *= 4
    return out

def oracle_rate(width, seconds, seed=0x5EED0003):
    """Permutations/s of the CPU oracle (all host cores) on a bounded tree."""
    import numpy as np  # noqa: F401
    import oracle
    import pg_synth
    cores = os.cpu_count() or 1
    log_n = 8
    while True:
        n = 1 << log_n
        rows = pg_synth.matrix(seed, n, width)
        t0 = time.perf_counter()
        oracle.merkle_build(rows, nthreads=cores)
        dt = time.perf_counter() - t0
        perms = workload(log_n, width)[1]
        if dt >= seconds / 4 or log_n >= 22:
            return perms / dt, cores, log_n, dt, perms
        grow = max(1, min(4, int((seconds / max(dt, 1e-3)) ** 0.5).bit_length() - 1))
        log_n = min(22, log_n + grow)


def oracle_step_size(width, target_s):
    """Largest 2^k-leaf tree the oracle builds in about target_s seconds."""
    rate, cores, log_n, dt, perms = oracle_rate(width, min(target_s, 4.0))
    while log_n < 22 and workload(log_n + 1, width)[1] / rate <= target_s:
        log_n += 1
    while log_n > 4 and workload(log_n, width)[1] / rate > 1.5 * target_s:
        log_n -= 1
    return log_n, cores


# ------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import pg_synth
    n, perms_full, name = workload(args.log_n, args.width)
    log_s, cores = oracle_step_size(args.width, target_s=4.0)
    ns, perms, _ = workload(log_s, args.width)
    rows = pg_synth.matrix(0x5EED0003, ns, args.width)
    for _ in range(args.warmup):
        oracle.merkle_build(rows, nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.merkle_build(rows, nthreads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = perms * args.steps / tot
    sample = f"2^{log_s}-leaf subtree of the same workload (width {args.width}), {perms} permutations per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "perms/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": name, "leaves": n, "width": args.width,
                   "parallelism": "cpu oracle, level-parallel threads"},
        "cpu_baseline": {"value": value, "unit": "perms/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "host_cpu": host_cpu_model(),
                         "ms_per_step_std": 1e3 * statistics.pstdev(times) if len(times) > 1 else 0.0},
        "e2e": {"value": value, "unit": "perms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch

    import paper_2506_09505_gb300 as pg
    import pg_synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    pg.load(build_if_missing=True)
    pg.init(local, args.params)
    pg.set_engine(pg.ENGINE_TENSOR if args.engine == "tensor" else pg.ENGINE_INT)
    mul_per_perm = MUL_RESULTS_PER_PERM_SMALL if args.params == "pg12_small" else MUL_RESULTS_PER_PERM

    n, perms, name = workload(args.log_n, args.width)
    # every rank builds the same tree (replicas), from the seed whose oracle
    # root and node-array hash are stored
    rows_np = pg_synth.matrix(pg_synth.tree_rows_seed(args.log_n, args.width), n, args.width)
    rows = torch.from_numpy(rows_np.view(np.int64)).cuda()
    nodes = torch.empty((2 * n - 1, 4), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 0)):
        pg.merkle_build(rows, nodes)
    props = torch.cuda.get_device_properties(local)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(props.uuid) if not str(props.uuid).startswith("GPU-") else str(props.uuid)
    except Exception:
        gpu_id = None
    # Rows smaller than twice the L2 would stay cached from one step to the
    # next: then a 512 MiB write evicts them between steps, outside the timed
    # step brackets.
    flush = rows_np.nbytes < 2 * L2_BYTES
    scratch = torch.empty(512 << 20, dtype=torch.uint8, device="cuda") if flush else None

    def timed_steps(kernel_events):
        """Per-step device times (ms) of args.steps builds; with kernel_events the
        library also brackets each of its launches with CUDA events."""
        ea = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        eb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        pg.profile_enable(kernel_events)
        for k in range(args.steps):
            if flush:
                scratch.zero_()
            ea[k].record(stream)
            pg.merkle_build(rows, nodes)
            eb[k].record(stream)
        barrier()
        kern = pg.profile_read() if kernel_events else None
        pg.profile_enable(False)
        return [a.elapsed_time(b) for a, b in zip(ea, eb)], kern

    barrier()
    sampler = ClockSampler(gpu_id)
    time.sleep(0.4)
    # the timed region: K builds, each bracketed by CUDA events on the stream
    plain_ms, _ = timed_steps(False)
    # the same K builds with the library also recording CUDA events around each
    # of its launches (they cost a little per launch and keep consecutive
    # launches from overlapping): the per-kernel durations of the roofline
    step_ms, kernels = timed_steps(True)
    clocks = sampler.stop()
    total_ms = sum(plain_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms = total_ms / args.steps
    value = perms * world * args.steps / (total_ms / 1e3)

    # end to end through the public call with host rows (pg_merkle_build_host:
    # pinned host rows copied to the device in chunks overlapped with the
    # leaf hashing, the build, the root read back), every step
    host_rows = torch.from_numpy(rows_np.view(np.int64)).pin_memory()
    dev_rows = torch.empty_like(rows)
    for _ in range(2):
        pg.merkle_build_host(host_rows, dev_rows, nodes, want_root=True)
    barrier()
    e_steps = max(3, min(args.steps, 10))
    e_sampler = ClockSampler(gpu_id)
    time.sleep(0.4)
    t0 = time.perf_counter()
    for _ in range(e_steps):
        pg.merkle_build_host(host_rows, dev_rows, nodes, want_root=True)
    e_s = time.perf_counter() - t0
    e_clocks = e_sampler.stop()
    # the same rows as one plain pinned copy: the host link's bandwidth on this machine, which
    # bounds the end-to-end step when the copy outlasts the leaf hashing it overlaps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        dev_rows.copy_(host_rows, non_blocking=True)
    torch.cuda.synchronize()
    h2d_gbs = 3 * rows_np.nbytes / (time.perf_counter() - t0) / 1e9
    if dist is not None:
        t = torch.tensor([e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e_s = float(t.item())
    e2e = {"value": perms * world * e_steps / e_s, "unit": "perms/s",
           "h2d_bytes_per_step": int(rows_np.nbytes), "d2h_bytes_per_step": 32,
           "ms_per_step": 1e3 * e_s / e_steps, "clocks": e_clocks,
           "h2d_copy_gbs": h2d_gbs, "h2d_copy_ms": rows_np.nbytes / h2d_gbs / 1e6}

    peaks = measured_peaks()
    sms = props.multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = IMAD_RESULTS_PER_CLK_SM * sms * max_mhz * 1e6 / 1e12  # T results/s
    dropped = kernels.pop("_dropped", 0)
    tot_kernel_ms = sum(v["total_ms"] for v in kernels.values())

    small = args.params == "pg12_small"
    saved = (ZCAP_SAVED_SMALL + DIGEST_SAVED_SMALL) if small else (ZCAP_SAVED + DIGEST_SAVED)
    chunks = max(1, (args.width + 7) // 8)

    def executed_per_perm(name):
        # node launches: every permutation starts from a zero capacity and ends
        # in a digest; leaf launches: the first and the last of each leaf's chunks
        if name not in ZCAP_KERNELS:
            return mul_per_perm
        share = 1.0 if name in LEVEL_KERNELS else 1.0 / chunks
        return mul_per_perm - share * saved

    km = kernel_metrics()
    traffic_table = km.get("traffic_bytes_per_launch", {}).get(f"merkle_2e{args.log_n}_w{args.width}", {}) \
        if args.params in (None, "pg12_v1") else {}

    def kernel_roofline(name):
        v = kernels[name]
        launch_ms = v["total_ms"] / v["launches"]      # average launch, event-timed
        per_launch = v["perms"] // v["launches"]       # permutations per launch
        ach = per_launch * mul_per_perm / (launch_ms / 1e3) / 1e12
        ach_x = per_launch * executed_per_perm(name) / (launch_ms / 1e3) / 1e12
        return {"achieved": ach, "frac": ach / peak, "launch_ms": launch_ms, "perms_per_launch": per_launch,
                "frac_executed": ach_x / peak, "executed_mul32_results_per_perm": executed_per_perm(name),
                "mul32_results_per_launch": per_launch * mul_per_perm,
                "algorithmic_bytes_per_launch": algorithmic_bytes(name, per_launch, args.width),
                "traffic": traffic_table.get(name)}

    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])   # the kernel with the largest share
    rk = kernel_roofline(dom)
    # which pipe binds, and the issue-slot ceiling, from the kernel's ncu capture
    kmet = km.get("kernels", {}).get(metrics_kernel(dom))
    if kmet:
        busiest = max(kmet["pipes_pct"], key=kmet["pipes_pct"].get)
        bound = "alu" if busiest in ("alu", "fmaheavy") else busiest
        issue_ceiling = 128 * sms * max_mhz * 1e6 / kmet["thread_inst_per_perm"]  # perms/s at 4 warp-issues/clk/SM
        issue = {"thread_inst_per_perm": kmet["thread_inst_per_perm"], "ceiling_perms_per_s": issue_ceiling,
                 "frac": rk["perms_per_launch"] / (rk["launch_ms"] / 1e3) / issue_ceiling,
                 "issue_active_pct_ncu": kmet["issue_active_pct"]}
        bound_basis = (f"ncu on {metrics_kernel(dom)}: pipes busy {kmet['pipes_pct']} (% of peak); the busiest, "
                       f"'{busiest}', carries the carry arithmetic of the field products")
    else:
        bound, issue, bound_basis = "alu", None, "no ncu capture of the current kernel sources"
    roofline = {
        "bound": bound, "bound_basis": bound_basis, "issue": issue, "kernel": dom,
        "achieved": rk["achieved"], "peak": peak, "unit": "T mul32-results/s",
        "frac": rk["frac"],
        "frac_executed": rk["frac_executed"],
        "executed_mul32_results_per_perm": rk["executed_mul32_results_per_perm"],
        "peak_basis": f"{IMAD_RESULTS_PER_CLK_SM} x {sms} SMs x {max_mhz:.0f} MHz (sm_max_mhz)",
        "traffic": rk["traffic"],
        "launch_ms": rk["launch_ms"], "perms_per_launch": rk["perms_per_launch"],
        "mul32_results_per_launch": rk["mul32_results_per_launch"],
        "algorithmic_bytes_per_launch": rk["algorithmic_bytes_per_launch"],
        "step_frac": perms * mul_per_perm / (ms / 1e3) / 1e12 / peak,
        "per_kernel": {k: {"frac": r["frac"], "frac_executed": r["frac_executed"], "launch_ms": r["launch_ms"],
                           "traffic": r["traffic"],
                           "algorithmic_bytes_per_launch": r["algorithmic_bytes_per_launch"]}
                       for k, r in ((k, kernel_roofline(k)) for k in kernels)},
    }
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = rk["achieved"] / (IMAD_RESULTS_PER_CLK_SM * sms * clocks["sm_mhz"] * 1e6 / 1e12)

    line = {
        "metric": METRIC, "value": value, "unit": "perms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": name, "leaves": n, "width": args.width, "perms_per_tree": perms,
                   "trees_per_gpu": 1, "parallelism": f"replicas x{world} (independent trees)",
                   "l2": (f"rows {rows_np.nbytes / 2**20:.3g} MiB/step, under twice the L2: 512 MiB write "
                          "between steps, outside the timed brackets" if flush else
                          f"inputs larger than L2 (rows {rows_np.nbytes / 2**20:.3g} MiB/step), no flush"),
                   "params": args.params or "pg12_v1"},
        "build_ms": ms, "build_ms_min": min(plain_ms),
        "ms_per_step_with_kernel_events": sum(step_ms) / len(step_ms),
        "roofline": roofline, "e2e": e2e,
        "gpu_launches": sum(v["launches"] for v in kernels.values()) + dropped,
        "kernels": {k: {"launches": v["launches"], "ms_per_launch": v["total_ms"] / v["launches"],
                        "share": v["total_ms"] / tot_kernel_ms} for k, v in kernels.items()},
        "clocks": clocks,
    }
    # the timed tree against the oracle's stored result (when one is stored for this shape)
    gold = golden_tree(args.log_n, args.width, args.params)
    if gold is not None:
        ok = tree_matches(nodes, gold)
        if dist is not None:
            t = torch.tensor([1 if ok else 0], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MIN)
            ok = bool(t.item())
        line["bit_exact"] = ok
        line["bit_exact_basis"] = "root and SHA-256 of all 2N-1 nodes of the timed tree vs the stored oracle build"
    else:
        line["bit_exact"] = None
    line["engine"] = "tensor" if pg.get_engine() == pg.ENGINE_TENSOR else "int"
    if world == 1 and not args.headline_only:
        line["workloads"] = run_sub_workloads(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, log_s, dt, sp = oracle_rate(args.width, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "perms/s", "cores": cores, "kind": "oracle",
                                "sample": f"2^{log_s}-leaf tree of width {args.width} "
                                          f"({sp} permutations, {dt:.1f} s), level-parallel threads",
                                "host_cpu": host_cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------ other workloads
# Each returns one dict: run alone with --workload, or embedded under
# "workloads" in the default run's line.  Every one reports the device time,
# permutations/s, the fraction of the IMAD roofline (algorithmic multiply
# results at 64 per clock per SM), the clocks sampled while it ran, and
# whether its outputs equal the oracle's stored results ("bit_exact").
_ARGS = None


def _device_setup():
    import torch
    import paper_2506_09505_gb300 as pg
    torch.cuda.set_device(0)
    pg.load(build_if_missing=True)
    pg.init(0, _ARGS.params if _ARGS is not None else None)
    if _ARGS is not None:
        pg.set_engine(pg.ENGINE_TENSOR if _ARGS.engine == "tensor" else pg.ENGINE_INT)
    return torch, pg


def _peak_results_per_s():
    import torch
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return IMAD_RESULTS_PER_CLK_SM * sms * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6


def _mul_per_perm(args):
    return MUL_RESULTS_PER_PERM_SMALL if args.params == "pg12_small" else MUL_RESULTS_PER_PERM


def _imad_frac(args, perms, seconds):
    return perms * _mul_per_perm(args) / seconds / _peak_results_per_s()


def _gpu_id():
    import torch
    try:
        u = str(torch.cuda.get_device_properties(0).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def _timed(fn, steps, warmup):
    """Device ms per call of fn() (CUDA events on the current stream, after warm-up),
    with the GPU clocks sampled during the timed calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    sampler = ClockSampler(_gpu_id())
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    return e0.elapsed_time(e1) / steps, clocks


def measure_permute(args):
    """Workload 2: 2^24 independent states permuted in place (raw permutation throughput)."""
    torch, pg = _device_setup()
    import pg_synth
    n = 1 << args.permute_log_n
    seed = pg_synth.config_seed(2)
    st = pg_synth.matrix_torch(seed, n, 12, device="cuda")
    # one permutation of the seeded states, checked against the stored oracle output
    pg.permute_batch(st)
    torch.cuda.synchronize()
    g = goldens().get("permute_2e24") if n == 1 << 24 else None
    exact = (sha256_words(st) == g["states_sha256"]) if g and args.params in (None, "pg12_v1") else None
    ms, clocks = _timed(lambda: pg.permute_batch(st), args.steps, args.warmup)
    rate = n / (ms / 1e3)
    out = {"workload": f"permute 2^{args.permute_log_n} states in place", "params": args.params or "pg12_v1",
           "ms": ms, "perms_per_s": rate, "imad_frac": _imad_frac(args, n, ms / 1e3),
           "kernel": "k_tc_permute" if pg.get_engine() == pg.ENGINE_TENSOR else "k_permute",
           "bit_exact": exact, "bit_exact_basis": "SHA-256 of the 2^24 states after one permutation vs the oracle's",
           "clocks": clocks}
    del st
    torch.cuda.empty_cache()
    return out


def measure_tree(args, log_n, width):
    """Workload 3: one tree of 2^log_n leaves of `width` words (rows resident in HBM)."""
    torch, pg = _device_setup()
    import pg_synth
    n, perms, name = workload(log_n, width)
    rows = pg_synth.matrix_torch(pg_synth.tree_rows_seed(log_n, width), n, width, device="cuda")
    nodes = torch.empty((2 * n - 1, 4), dtype=torch.int64, device="cuda")
    ms, clocks = _timed(lambda: pg.merkle_build(rows, nodes), args.steps, args.warmup)
    g = golden_tree(log_n, width, args.params)
    out = {"workload": name, "ms": ms, "perms_per_s": perms / (ms / 1e3),
           "imad_frac": _imad_frac(args, perms, ms / 1e3),
           "bit_exact": tree_matches(nodes, g) if g else None, "clocks": clocks}
    del rows, nodes
    torch.cuda.empty_cache()
    return out


def measure_batch(args):
    """Workload 4: 64 trees of mixed sizes and widths in one captured persistent launch
    (autotuned schedule) against one pg_merkle_build per tree, same GPU, same inputs."""
    torch, pg = _device_setup()
    import pg_synth
    sizes = pg_synth.batch_sizes(args.trees, args.max_log_n)
    rows = [pg_synth.matrix_torch(pg_synth.batch_tree_seed(k), 1 << lg, w, device="cuda")
            for k, (lg, w) in enumerate(sizes)]
    perms = sum((1 << lg) * ((w + 7) // 8) + (1 << lg) - 1 for lg, w in sizes)
    nodes = pg.alloc_nodes(rows)
    t0 = time.perf_counter()
    best, tune_ms = pg.batch_autotune(rows, nodes)
    tune_s = time.perf_counter() - t0
    g = pg.BatchGraph(rows, nodes, schedule=best)
    ms_batch, clocks = _timed(g.launch, args.steps, args.warmup)
    gold = goldens()
    exact = None
    if args.trees == 64 and args.max_log_n >= 20 and args.params in (None, "pg12_v1"):
        exact = all(sha256_words(nd) == gold[f"batch_{k:02d}"]["nodes_sha256"] for k, nd in enumerate(nodes)) \
            if all(f"batch_{k:02d}" in gold for k in range(64)) else None
    batch_out = [t.clone() for t in nodes]
    g.close()
    single = [torch.empty_like(t) for t in nodes]

    def one_per_tree():
        for r, nd in zip(rows, single):
            pg.merkle_build(r, nd)
    ms_single, clocks_single = _timed(one_per_tree, args.steps, args.warmup)
    same = all(torch.equal(a, b) for a, b in zip(batch_out, single))
    out = {
        "workload": f"batch of {len(sizes)} trees, 2^k leaves k in [12,20], widths in {{8..128}}",
        "perms_per_step": perms, "trees": [[lg, w] for lg, w in sizes],
        "batched_graph": {"ms": ms_batch, "perms_per_s": perms / (ms_batch / 1e3),
                          "imad_frac": _imad_frac(args, perms, ms_batch / 1e3),
                          "schedule": best, "autotune_best_ms": tune_ms, "autotune_s": tune_s, "clocks": clocks},
        "one_launch_per_tree": {"ms": ms_single, "perms_per_s": perms / (ms_single / 1e3),
                                "imad_frac": _imad_frac(args, perms, ms_single / 1e3), "clocks": clocks_single},
        "speedup": ms_single / ms_batch, "bit_identical_to_single": same, "bit_exact": exact,
        "bit_exact_basis": "SHA-256 of every tree's 2N-1 nodes from the captured launch vs the stored oracle builds",
    }
    del rows, nodes, single, batch_out
    torch.cuda.empty_cache()
    return out


def _serve_stream(args, requests, rate):
    import pg_synth
    arrivals, ks, ws = pg_synth.served_stream(requests, rate, 10, args.max_log_n)
    perms = [(1 << k) * ((w + 7) // 8) + (1 << k) - 1 for k, w in zip(ks, ws)]
    return arrivals, ks, ws, perms


def _serve_rows(torch, shapes):
    import pg_synth
    # payloads are materialised on the device ahead of their arrival (not timed);
    # every request of one (k, w) shape reuses that shape's rows
    return {key: pg_synth.matrix_torch(pg_synth.served_rows_seed(*key), 1 << key[0], key[1], device="cuda")
            for key in sorted(set(shapes))}


def _serve_server(torch, pg, args, arrivals, ks, ws, cache, keep_shapes=()):
    """The serving runtime on an arrival trace: per-request latency (arrival -> root
    stored), makespan, and copies of the first result of each shape in keep_shapes."""
    import numpy as np
    pool = int(min(torch.cuda.mem_get_info()[0] * 0.5, 64 << 30))
    srv = pg.Server(pool_bytes=pool, max_batch=256, max_inflight=2, schedule={"order": args.server_order})
    lat, pending, kept = {}, [], {}
    keep = {k: torch.empty((2 * (1 << k[0]) - 1, 4), dtype=torch.int64, device="cuda") for k in keep_shapes}
    shape_of = {}

    def reap():
        rest = []
        for rid in pending:
            info = srv.query(rid)
            if info["state"] in (pg.REQ_DONE, pg.REQ_FAILED):
                if info["state"] != pg.REQ_DONE:
                    raise RuntimeError(f"request {rid} failed")
                lat[rid] = info["done_s"] - info["submit_s"]
                key = shape_of[rid]
                if key in keep and key not in kept:
                    keep[key].copy_(srv.nodes(rid, 1 << key[0]))
                    kept[key] = True
                srv.release(rid)
            else:
                rest.append(rid)
        pending[:] = rest

    t_start = time.perf_counter()
    for i in range(len(arrivals)):
        while True:
            now = time.perf_counter() - t_start
            if arrivals[i] <= now:
                break
            reap()
            now = time.perf_counter() - t_start
            if arrivals[i] > now:
                time.sleep(min(arrivals[i] - now, 0.002))
        key = (ks[i], ws[i])
        rid = srv.submit(cache[key])
        shape_of[rid] = key
        pending.append(rid)
    while pending:
        reap()
        time.sleep(0.001)
        if time.perf_counter() - t_start > 900:
            raise RuntimeError("serving run did not finish")
    t_end = time.perf_counter() - t_start
    srv.close()
    torch.cuda.synchronize()
    return np.array(list(lat.values())), t_end, keep


def _serve_sequential(torch, pg, arrivals, ks, ws, cache):
    """Measured baseline: one pg_merkle_build per request, launched in arrival order on
    one stream as each request arrives; latency = arrival -> the build's completion
    event (times on the device's clock, from an event recorded at the trace's start)."""
    import numpy as np
    nodes = {key: torch.empty((2 * r.shape[0] - 1, 4), dtype=torch.int64, device="cuda") for key, r in cache.items()}
    done = [torch.cuda.Event(enable_timing=True) for _ in range(len(arrivals))]
    start = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record()
    t_start = time.perf_counter()
    for i in range(len(arrivals)):
        while time.perf_counter() - t_start < arrivals[i]:
            time.sleep(0.0002)
        key = (ks[i], ws[i])
        pg.merkle_build(cache[key], nodes[key])
        done[i].record()
    torch.cuda.synchronize()
    fin = np.array([start.elapsed_time(e) / 1e3 for e in done])
    return fin - np.asarray(arrivals), float(fin.max())


def measure_serve(args):
    """Workload 5: Poisson stream of tree builds through the serving runtime against
    sequential single-tree builds on the same trace, at the workload's rate (over the
    GPU's capacity) and at a rate under it."""
    torch, pg = _device_setup()
    import numpy as np
    gold = goldens()
    peak = _peak_results_per_s()
    out = {}
    for label, nreq, rate in (("rate_200", args.requests, args.rate),
                              ("rate_low", args.serve_low_requests, args.serve_low_rate)):
        arrivals, ks, ws, perms = _serve_stream(args, nreq, rate)
        cache = _serve_rows(torch, list(zip(ks, ws)))
        torch.cuda.synchronize()
        keep_shapes = [s for s in ((22, 8), (22, 32)) if s in cache] if label == "rate_200" else []
        sampler = ClockSampler(_gpu_id())
        lat, makespan, kept = _serve_server(torch, pg, args, arrivals, ks, ws, cache, keep_shapes)
        clocks = sampler.stop()
        seq_lat, seq_makespan = _serve_sequential(torch, pg, arrivals, ks, ws, cache)
        total = int(sum(perms))
        exact = None
        if keep_shapes and args.params in (None, "pg12_v1"):
            exact = all(tree_matches(kept[s], gold[f"serve_2e22_w{s[1]}"]) for s in keep_shapes
                        if f"serve_2e22_w{s[1]}" in gold)
        out[label] = {
            "requests": nreq, "rate_per_s": rate, "total_perms": total,
            "offered_perms_per_s": total / float(arrivals[-1]),
            "server": {"makespan_s": makespan, "perms_per_s": total / makespan,
                       "imad_frac": total * _mul_per_perm(args) / makespan / peak,
                       "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                       "clocks": clocks},
            "sequential_builds": {"makespan_s": seq_makespan, "perms_per_s": total / seq_makespan,
                                  "imad_frac": total * _mul_per_perm(args) / seq_makespan / peak,
                                  "p50_latency_s": float(np.percentile(seq_lat, 50)),
                                  "p99_latency_s": float(np.percentile(seq_lat, 99))},
            "bit_exact": exact,
        }
        if keep_shapes:
            out[label]["bit_exact_basis"] = ("first served 2^22-leaf result of widths " +
                                             ", ".join(str(s[1]) for s in keep_shapes) +
                                             ": root and SHA-256 of all nodes vs the stored oracle builds")
        del cache, kept
        torch.cuda.empty_cache()
    out["workload"] = (f"serve Poisson requests, 2^k leaves k in [10,{args.max_log_n}], widths {{8,32,128,256}}: "
                       f"{args.requests} at {args.rate}/s and {args.serve_low_requests} at {args.serve_low_rate}/s")
    return out


def run_sub_workloads(args):
    """The other configurations, each measured in this run (workloads 2, 3b, 4, 5, and the
    low-degree extension feeding a commitment)."""
    out = {}
    steps = max(3, min(args.steps, 10))
    sub = argparse.Namespace(**vars(args))
    sub.steps = steps
    out["permute"] = measure_permute(sub)
    out["merkle_w64"] = measure_tree(sub, 22, 64)
    out["batch"] = measure_batch(sub)
    out["serve"] = measure_serve(sub)
    lde = argparse.Namespace(**vars(sub))
    lde.width = 8
    out["lde"] = measure_lde(lde)
    return out


def run_permute(args):
    line = measure_permute(args)
    if not args.no_cpu_baseline and not args.params:
        rates = oracle_permute_rates()
        line["cpu_baseline"] = {"value": rates["all_core"]["perms_per_s"], "unit": "perms/s",
                                "cores": rates["all_core"]["threads"], "kind": "oracle",
                                "sample": f"{rates['all_core']['sample_states']} random states, plain round form",
                                "single_thread_perms_per_s": rates["single_thread"]["perms_per_s"],
                                "host_cpu": host_cpu_model()}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    print(json.dumps(measure_batch(args)), flush=True)
    return 0


def run_serve(args):
    print(json.dumps(measure_serve(args)), flush=True)
    return 0


def measure_lde(args):
    """Low-degree extension of a 2^21-row, 8-column trace with blowup 2 (the NTT
    hotspot), committed as the 2^22 x 8 Merkle tree, every step."""
    torch, pg = _device_setup()
    import pg_synth
    log_n, cols, log_b = args.lde_log_n, args.width, args.log_blowup
    n, big = 1 << log_n, 1 << (log_n + log_b)
    evals = pg_synth.matrix_torch(pg_synth.config_seed(6), n, cols, device="cuda")
    scratch = torch.empty_like(evals)
    out = torch.empty((big, cols), dtype=torch.int64, device="cuda")
    nodes = torch.empty((2 * big - 1, 4), dtype=torch.int64, device="cuda")
    for _ in range(args.warmup):
        pg.lde(evals, log_b, out=out, scratch=scratch)
        pg.merkle_build(out, nodes)
    torch.cuda.synchronize()
    pg.profile_enable(True)
    sampler = ClockSampler(_gpu_id())
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pg.lde(evals, log_b, out=out, scratch=scratch)
        pg.merkle_build(out, nodes)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    kern = pg.profile_read()
    pg.profile_enable(False)
    kern.pop("_dropped", None)
    ms = e0.elapsed_time(e1) / args.steps
    lde_ms = kern["k_ntt_pass"]["total_ms"] / args.steps
    # the last step's extension and commitment against the oracle's stored outputs
    g = goldens().get("lde_2e21x8_b1")
    bit_exact = None
    if g and (g["log_n"], g["cols"], g["log_blowup"]) == (log_n, cols, log_b):
        bit_exact = sha256_words(out) == g["out_sha256"] and sha256_words(nodes) == g["nodes_sha256"]
    # one product per butterfly (8 results) and four per input coefficient for the coset factor
    butterflies = (n // 2) * log_n * cols + (big // 2) * log_n * cols
    mul_results = 8 * (butterflies + 4 * n * cols)
    alg_bytes = 8 * cols * (n + big)
    perms = big * ((cols + 7) // 8) + big - 1
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    del evals, scratch, out, nodes
    torch.cuda.empty_cache()
    return {
        "workload": f"LDE of 2^{log_n} x {cols} evaluations, blowup 2^{log_b}, then the 2^{log_n + log_b} x {cols} Merkle tree",
        "ms_per_step": ms, "steps": args.steps, "bit_exact": bit_exact,
        "bit_exact_basis": "SHA-256 of the whole extension and of its tree's nodes vs the stored oracle outputs",
        "lde": {"ms": lde_ms, "launches_per_step": kern["k_ntt_pass"]["launches"] // args.steps,
                "roofline_alu": {"achieved": mul_results / (lde_ms / 1e3) / 1e12, "peak": _peak_results_per_s() / 1e12,
                                 "unit": "T mul32-results/s",
                                 "frac": mul_results / (lde_ms / 1e3) / _peak_results_per_s()},
                "roofline_hbm": {"achieved": alg_bytes / (lde_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                                 "frac": alg_bytes / (lde_ms / 1e3) / 1e9 / hbm,
                                 "algorithmic_bytes": alg_bytes}},
        "commit": {"ms": ms - lde_ms, "perms": perms, "perms_per_s": perms / ((ms - lde_ms) / 1e3)},
        "kernels": {k: {"launches": v["launches"], "ms_per_step": v["total_ms"] / args.steps} for k, v in kern.items()},
        "clocks": clocks,
    }


def run_lde(args):
    print(json.dumps(measure_lde(args)), flush=True)
    return 0


def main():
    global _ARGS
    args = parse_args()
    _ARGS = args
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "permute":
        return run_permute(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "lde":
        return run_lde(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
