#!/usr/bin/env python
"""Benchmark: energy + forces of the 23,558-atom periodic box (8-member ensemble) on B300.

One step = rebuild the neighbour list (cell lists) + AEVs + the per-element networks
(forward and input gradient) + float64 energy/virial reductions + the AEV adjoint (forces),
all through the C ABI on inputs already resident in HBM.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|bf16|fp8]
    python bench.py --impl reference ...   # the float64 CPU oracle on host cores

Multi-GPU (torchrun, one rank per GPU): every rank evaluates its own replica of the box
(replicas only, no data-path collective); value = atoms of all ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "energy+force atom-evals/s (23.6k-atom box, FP32 vs BF16); serve p50/p99 ms"
UNIT = "atom-evals/s"
WORKLOAD = ("mix23558: 23,558-atom periodic box, 62.2 A cube, H/C/N/O/S = .50/.30/.08/.10/.02, d_min 0.95 A, "
            "seed 3; 8-member random-init ensemble (seeded Xavier); neighbour list rebuilt every step (skin 0)")
PRECISION_NOTE = {
    "fp32x3": "FP32-accurate networks on tcgen05: operands split into bf16 hi + lo, hi*hi + hi*lo + lo*hi "
              "accumulated in FP32; AEV, reductions and adjoint in FP32/FP64",
    "fp32": "networks on SIMT FP32 FFMA",
    "bf16": "networks in BF16 on tcgen05 with FP32 accumulation",
    "bf16_fused": "the BF16 form with the AEV and the first layer in one kernel (64-row AEV tiles built in shared "
                  "memory as the tcgen05 A operand)",
    "fp8": "networks in FP8 e4m3 on tcgen05 (kind::f8f6f4) with FP32 accumulation; per-layer scales "
           "(weights amax/448 per block, activations 2 amax/448 from an FP32 calibration evaluation)",
}
FFMA_LANES_PER_SM = 128          # FP32 FMA lanes per SM
N_SM = 148
L2_FLUSH_BYTES = 256 << 20       # larger than the 126 MB L2


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                "sm_max_mhz": d.get("sm_max_mhz", 2032.0), "src": "measured"}
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0,
            "src": "fallback"}


def kernel_work(name: str, n_atoms: int, nnz: int, M: int):
    """Algorithmic work of one launch of a kernel: (bound, amount, unit, executed) or None.  For the network
    products the amount is the method's own work, one FP32 product of 2 in out FLOP per row and member;
    `executed` is what the tensor pipe runs (three bf16 products for the FP32X3 split), else None."""
    if name == "aev_forward":       # positions once, list entries (index + shift), the AEV row written
        return "hbm", n_atoms * (16 + 4032) + nnz * 8, "B", None
    if name in ("aev_forward_bf16", "aev_forward_x3"):  # bf16 AEV row (x3: hi and lo rows)
        return "hbm", n_atoms * (16 + (4032 if name.endswith("x3") else 2016)) + nnz * 8, "B", None
    if name == "aev_forward_fp8":   # e4m3 AEV row
        return "hbm", n_atoms * (16 + 1008) + nnz * 8, "B", None
    if name == "aev_l1_bf16":       # fused AEV + first layer: the first layer's product (bf16 operands)
        return "tensor", 2.0 * 1008 * 256 * M * n_atoms, "FLOP", None
    if name == "aev_adjoint":       # positions, list, dE/dAEV row read, forces written
        return "hbm", n_atoms * (16 + 4032 + 12) + nnz * 8, "B", None
    gemm = {"l1": 1008 * 256, "l2": 256 * 192, "l3": 192 * 160}
    m = re.match(r"(f32|bf16|fp8|x3)_(l[123])_(fwd|bwd|pair)", name)
    if m:   # "_pair": the fused third layer, forward and backward products
        flops = 2.0 * gemm[m.group(2)] * M * n_atoms * (2 if m.group(3) == "pair" else 1)
        return (("alu" if m.group(1) == "f32" else "tensor"), flops, "FLOP",
                3 * flops if m.group(1) == "x3" else None)
    if name in ("pairs_count", "pairs_fill", "pairs_stage"):
        return "hbm", n_atoms * 16 + (nnz * 8 if name != "pairs_count" else 0), "B", None
    if name == "pairs_compact":     # staged entries read, list entries written
        return "hbm", nnz * 16, "B", None
    return None


KERNEL_SOURCES = [  # kernel-name prefix -> the files that define it (with the shared internal header)
    (("x3_l3_pair", "bf16_l3_pair"), ("tc_gemm.cuh", "tc_fused.cuh", "mlp_tc.cu")),
    (("x3_", "bf16_", "fp8_", "tr16_"), ("tc_gemm.cuh", "tc_pair.cuh", "mlp_tc.cu")),
    (("f32_", "energy_reduce"), ("mlp_simt.cu",)),
    (("aev_l1",), ("aev.cu", "tc_gemm.cuh")),
    (("aev_",), ("aev.cu",)),
    (("pairs_", "scan", "mol_setup", "atom_setup", "mol_grid", "check_", "bin", "scatter", "sort_cells", "elem_"),
     ("nlist.cu",)),
]


def source_digest(kernel: str | None = None) -> str:
    """Digest of the sources a kernel is built from (all of csrc when kernel is None or unknown)."""
    d = os.path.join(ROOT, "paper_2405_01491_b300", "csrc")
    files = sorted(os.listdir(d))
    if kernel:
        for prefixes, srcs in KERNEL_SOURCES:
            if kernel.startswith(prefixes):
                files = ["fnn_internal.cuh", *srcs]
                break
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel: str, digest: str):
    """DRAM bytes per launch from the committed ncu summary, when it was taken on the current sources."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.md")
    if not os.path.exists(p):
        return None
    for line in open(p):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == kernel and cells[3] == digest:
            try:
                return float(cells[2])
            except ValueError:
                return None
    return None


class Ranks:
    """Replicas on one node, one process per GPU (torchrun sets RANK / WORLD_SIZE / MASTER_*): a barrier
    and the max over ranks.  A single process when WORLD_SIZE is unset.  backend "nccl" on GPUs, "gloo"
    for the CPU tests of this logic."""

    def __init__(self, backend: str = "nccl", device: str = "cuda"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            kw = {"device_id": torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x: float) -> float:
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        if self.dist:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def whole_job_rate(units_per_rank: float, seconds_per_rank: float, ranks: Ranks) -> float:
    """Units of every rank over the slowest rank's time (weak scaling: each rank holds its own replica)."""
    return ranks.world * units_per_rank / ranks.max(seconds_per_rank)


class _NvmlLib:
    """The driver's NVML through ctypes (read-only queries: SM clock, its maximum, event reasons, power)."""

    def __init__(self, torch_index: int):
        import ctypes
        self.c = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(torch_index).uuid)
        except Exception:
            pass
        ok = False
        if uuid:
            key = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            ok = lib.nvmlDeviceGetHandleByUUID(key.encode(), ctypes.byref(h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(torch_index, ctypes.byref(h)) != 0:
            raise OSError("no NVML handle for the device")
        self.lib, self.h = lib, h
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        m = ctypes.c_uint()
        self.max_mhz = float(m.value) if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(m)) == 0 else None

    def sample(self):
        c = self.c
        mhz, pw, rs = c.c_uint(), c.c_uint(), c.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, c.byref(mhz)) != 0:
            return None
        self.reasons_fn(self.h, c.byref(rs))
        self.lib.nvmlDeviceGetPowerUsage(self.h, c.byref(pw))
        return float(mhz.value), int(rs.value), pw.value / 1000.0


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region: NVML (the driver library through
    ctypes) from a background thread every 1 ms (the timed regions are milliseconds long), nvidia-smi at
    200 ms if NVML cannot be opened."""
    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40, "sw_power_cap": 0x4}

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.max_mhz = None
        self._stop = None
        self.proc = None
        self.mode = None

    def _nvml_loop(self, nv):
        while not self._stop.is_set():
            try:
                r = nv.sample()
                if r:
                    self.rows.append(r)
            except Exception:
                pass
            self._stop.wait(0.001)

    def __enter__(self):
        import threading
        try:
            nv = _NvmlLib(self.index)
            self.max_mhz = nv.max_mhz
            r = nv.sample()          # one sample at the start of the region
            if r:
                self.rows.append(r)
            self._stop = threading.Event()
            self.thread = threading.Thread(target=self._nvml_loop, args=(nv,), daemon=True)
            self.thread.start()
            self._nv = nv
            self.mode = "nvml"
        except Exception:
            self.mode = "nvidia-smi"
            q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap")
            try:
                self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                              "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                             stderr=subprocess.DEVNULL, text=True)
            except OSError:
                self.proc = None
        return self

    def __exit__(self, *exc):
        if self.mode == "nvml":
            self._stop.set()
            self.thread.join(timeout=2)
            try:
                r = self._nv.sample()     # and one at its end
                if r:
                    self.rows.append(r)
            except Exception:
                pass
            return
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) == 7 and c[0].replace(".", "").isdigit():
                bits = sum(self.REASONS[names[k]] for k in range(4) if c[3 + k].lower() == "active")
                self.max_mhz = float(c[1])
                self.rows.append((float(c[0]), bits, float(c[2]) if c[2].replace(".", "").isdigit() else 0.0))

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unsampled"], "source": self.mode}
        reasons = sorted({n for _, bits, _ in self.rows for n, b in self.REASONS.items() if bits & b})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows), "sm_max_mhz": self.max_mhz,
                "power_w_max": max(r[2] for r in self.rows), "samples": len(self.rows), "reasons": reasons,
                "source": self.mode}


def oracle_full(M: int = 8, min_seconds: float = 10.0, max_reps: int = 3):
    """The float64 oracle, as it stands, on the whole benchmark box (host cores); repeated until about
    min_seconds of CPU work has been timed.  Returns (cpu_baseline entry, oracle result)."""
    import oracle
    from paper_2405_01491_b300 import synth
    s = synth.mix23558()
    w = synth.xavier_weights(M)
    times, res = [], None
    while not times or (len(times) < max_reps and sum(times) < min_seconds):
        t = time.perf_counter()
        res = oracle.energy_forces(s, w)
        times.append(time.perf_counter() - t)
    dt = statistics.mean(times)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    entry = {"value": s.n_atoms / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"{len(times)} full energy+force evaluation(s) of the same 23,558-atom box, M={M}, float64 "
                       f"(all-pairs neighbour search), {dt:.1f} s each"}
    return entry, res


# The oracle timed per configuration in a child process (so its thread count can be pinned): every
# workload of the measurement plan, each a bounded sample, reported in atom-evals/s.
_PLAN_CHILD = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle
from paper_2405_01491_b300 import synth
one_core = sys.argv[2] == "1"
out = {}
def timed(f, min_s=1.0):
    n, t0 = 0, time.perf_counter()
    while True:
        f(); n += 1
        if time.perf_counter() - t0 >= min_s: return (time.perf_counter() - t0) / n, n
s = synth.gas24(); w1 = synth.xavier_weights(1)
dt, n = timed(lambda: oracle.energy_forces(s, w1))
out["gas24"] = {"atom_evals_per_s": s.n_atoms / dt, "sample": f"{n} evaluations, M=1"}
s = synth.water216(); w8 = synth.xavier_weights(8); v = synth.maxwell_boltzmann(s.Z, 300.0, seed=2)
t0 = time.perf_counter(); oracle.velocity_verlet(s, w8, v, 20, 0.5); dt = (time.perf_counter() - t0) / 20
out["water216"] = {"atom_evals_per_s": s.n_atoms / dt, "ms_per_step": 1e3 * dt,
                   "s_per_1000_steps": 1e3 * dt, "sample": "20 velocity-Verlet steps, M=8, extrapolated to 1000"}
if one_core:   # a 1/8-volume box of the same density and composition (2,944 atoms): per-atom cost
    s = synth.mix_box(2944, 62.2 / 2, seed=3)
    sample = "2,944-atom periodic box (31.1 A, same density and composition), M=8, per atom"
else:
    s = synth.mix23558(); sample = "the 23,558-atom box, M=8"
t0 = time.perf_counter(); oracle.energy_forces(s, w8); dt = time.perf_counter() - t0
out["mix23558"] = {"atom_evals_per_s": s.n_atoms / dt, "sample": sample}
b = synth.ragged_batch(); sub = synth.concat([b.molecule(m) for m in range(256)]); E, F = synth.batch_targets(sub)
t0 = time.perf_counter(); oracle.loss_and_weight_grads(sub, w1, E, F); dt = time.perf_counter() - t0
out["batch4096"] = {"atom_evals_per_s": sub.n_atoms / dt, "sample": f"256-molecule subset ({sub.n_atoms} atoms): "
                    "energies, forces, loss and weight gradients, M=1, per atom"}
pool = synth.request_pool(12, seed=5); reqs = [p for p in pool if p.n_atoms <= 4000][:6]
t0 = time.perf_counter()
for p in reqs: oracle.velocity_verlet(p, w1, np.zeros((p.n_atoms, 3)), 10, 0.5)
dt = time.perf_counter() - t0
out["serve"] = {"atom_evals_per_s": 10 * sum(p.n_atoms for p in reqs) / dt,
                "sample": f"the first {len(reqs)} pool requests of at most 4000 atoms "
                          f"({sum(p.n_atoms for p in reqs)} atoms), 10 velocity-Verlet steps each, M=1"}
print(json.dumps(out))
"""


def cpu_model() -> str:
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_plan(timeout_s: float = 240.0) -> dict:
    """The oracle on every configuration of the measurement plan, on all host cores and on one core."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    res = {"cpu_model": cpu_model(), "cores_all": cores}
    for label, one in (("all_cores", False), ("one_core", True)):
        env = dict(os.environ)
        if one:
            for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
                env[k] = "1"
        try:
            r = subprocess.run([sys.executable, "-c", _PLAN_CHILD, ROOT, "1" if one else "0"], env=env,
                               capture_output=True, text=True, timeout=timeout_s)
            res[label] = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else \
                {"error": (r.stderr or "")[-300:]}
        except Exception as e:   # a slow host: the plan is context, not the measurement
            res[label] = {"error": str(e)[:300]}
    return res


def arm_config(precision: str, list_entries, world: int = 1) -> dict:
    """The workload description both arms print."""
    return {"workload": WORKLOAD, "n_atoms": 23558, "members": 8, "precision": precision,
            "precision_note": PRECISION_NOTE.get(precision, ""), "list_entries": list_entries,
            "parallelism": f"replicas x{world}",
            "l2": "flushed before every timed step (256 MB write outside the step's CUDA events)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    times = []
    entry = None
    for k in range(args.warmup + args.steps):
        e, _ = oracle_full(min_seconds=0.0, max_reps=1)
        if k >= args.warmup:
            times.append(23558 / e["value"])
        entry = e
    v = 23558 / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config("float64 oracle (all-pairs neighbour search), host cores", None),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": entry["cores"], "kind": "oracle",
                             "sample": "each step: one float64 energy+force evaluation of the whole 23,558-atom box"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _fifo_latencies(arrivals, services):
    """Completion - arrival of a single first-in first-out server: c_k = max(a_k, c_{k-1}) + s_k."""
    import numpy as np
    c, out = 0.0, []
    for a, sv in zip(arrivals, services):
        c = max(a, c) + sv
        out.append(c - a)
    return np.array(out)


def _served_stream(fnn, srv, pool, vels, stream, n_steps, dt):
    """Submit an open-loop arrival stream (busy-waiting on each arrival time) while draining finished
    tickets, then wait for the rest.  Returns (latencies ms, wall s)."""
    import collections
    import numpy as np
    t0 = time.perf_counter()
    outstanding = collections.deque()
    lat = []
    for t_arr, k in stream:
        while time.perf_counter() - t0 < t_arr:
            if outstanding:
                r = srv.poll(outstanding[0], timeout_s=0.0, arrays=False)
                if r is not None:
                    lat.append(r["latency_ms"])
                    outstanding.popleft()
        outstanding.append(srv.submit(pool[k], vels[k], n_steps, dt))
    while outstanding:
        r = srv.poll(outstanding.popleft(), timeout_s=600, arrays=False)
        lat.append(r["latency_ms"])
    return np.array(lat), time.perf_counter() - t0


def _batch_of_one(fnn, torch, pool, vels, stream, n_steps, dt, budget_s, w1):
    """Each request alone on the GPU (FP32X3, fnn_md_run_ex), in arrival order: service time = host copy of the
    request in, the 10 steps, the result copied out; latencies of a first-in first-out server over the same
    arrivals follow from the measured service times.  Stops after budget_s seconds of service."""
    import numpy as np
    ctx = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx, w1)
    nl = fnn.NeighborList(ctx)
    side = torch.cuda.Stream()
    arr, svc, evals = [], [], 0
    for idx, (t_arr, k) in enumerate(stream):
        s = pool[k]
        torch.cuda.synchronize()
        ta = time.perf_counter()
        with torch.cuda.stream(side):
            ds = fnn.DeviceSystem.from_structures(s)
            vel = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
            vel[:, :3] = torch.from_numpy(vels[k])
            vel = vel.cuda()
            E, _, F, _ = fnn.md_run_ex(ctx, ds, vel, nl, "fp32x3", n_steps, dt, 10, stream=side)
            res = (E.cpu(), ds.pos.cpu(), vel.cpu(), F.cpu())
        fnn.check(ctx, "batch-of-one", stream=side)
        sv = time.perf_counter() - ta
        if idx > 0:   # the first call carries one-time set-up
            arr.append(t_arr)
            svc.append(sv)
            evals += s.n_atoms * n_steps
        if sum(svc) >= budget_s:
            break
    del res
    return np.array(arr), np.array(svc), evals


def serve_bench(fnn, torch, synth, duration_s=60.0, rate_hz=2000.0, pool_n=4096, budget=120 << 30, n_steps=10,
                dt=0.5, one_budget_s=20.0, matched_s=20.0):
    """Serving stream: Poisson arrivals at rate_hz for duration_s of structures drawn from a pool of pool_n
    (log-uniform sizes 8..20000 atoms, periodic above 500), each 10 velocity-Verlet steps, one ensemble member;
    BF16 served form with continuous batching under an HBM budget.  Against it, the FP32-accurate form run
    batch-of-one under the same arrivals (a first-in first-out queue in front of one request at a time), and
    both forms at a matched load that batch-of-one sustains."""
    import numpy as np
    w1 = synth.xavier_weights(1)
    workers = max(1, min(32, (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 4)))
    t_pool = time.perf_counter()
    pool = synth.request_pool(pool_n, seed=5, workers=workers)
    vels = [synth.maxwell_boltzmann(p.Z, 300.0, seed=k) for k, p in enumerate(pool)]
    t_pool = time.perf_counter() - t_pool
    rng = np.random.Generator(np.random.PCG64([5, 2]))

    def poisson(rate, T):
        out, t = [], 0.0
        while True:
            t += rng.exponential(1.0 / rate)
            if t >= T:
                return out
            out.append((t, int(rng.integers(pool_n))))

    stream = poisson(rate_hz, duration_s)
    ctx = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx, w1)
    srv = fnn.Server(ctx, budget, "bf16", rebuild_every=10)
    for k in range(4):                                   # warm-up (allocations, first launches)
        srv.poll(srv.submit(pool[k], vels[k], n_steps, dt), timeout_s=300, arrays=False)
    st0 = srv.stats()
    lat, wall = _served_stream(fnn, srv, pool, vels, stream, n_steps, dt)
    st = srv.stats()
    evals = sum(pool[k].n_atoms * n_steps for _, k in stream)
    out = {"requests": len(stream), "completed": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "atom_evals_per_s": evals / wall,
           "offered_atom_evals_per_s": evals / duration_s, "arrival_window_s": duration_s, "wall_s": wall,
           "rate_hz": rate_hz, "members": 1, "precision": "bf16", "max_batch_atoms": st["max_batch_atoms"],
           "batch_steps": st["batch_steps"] - st0["batch_steps"],
           "mean_atoms": float(np.mean([pool[k].n_atoms for _, k in stream])),
           "pool": f"{pool_n} structures, n = round(exp(U(ln 8, ln 20000))), periodic above 500 atoms, seed 5 "
                   f"(built in {t_pool:.0f} s by {workers} processes)",
           "budget_bytes": budget, "status": st["status"], "scheduler_host_ms": st["host_ms"] - st0["host_ms"],
           "scheduler_step_ms": st["step_ms"] - st0["step_ms"], "rebuilds": st["rebuilds"] - st0["rebuilds"],
           "guard_rebuilds": st["guard_rebuilds"] - st0["guard_rebuilds"]}
    # batch-of-one FP32X3 under the same arrivals (the first one_budget_s seconds of service)
    arr, svc, ev1 = _batch_of_one(fnn, torch, pool, vels, stream, n_steps, dt, one_budget_s, w1)
    l1 = 1e3 * _fifo_latencies(arr, svc)
    cap_hz = len(svc) / svc.sum()
    out["batch_of_one"] = {
        "precision": "fp32x3", "requests": int(len(svc)), "arrival_window_s": float(arr[-1]),
        "p50_ms": float(np.percentile(l1, 50)), "p99_ms": float(np.percentile(l1, 99)),
        "service_p50_ms": float(1e3 * np.percentile(svc, 50)), "saturation_rate_hz": cap_hz,
        "saturation_atom_evals_per_s": ev1 / svc.sum(),
        "note": "same arrivals, one request at a time (first in, first out; host copies in the service time); the "
                f"offered {rate_hz:.0f} req/s exceeds what it completes ({cap_hz:.0f} req/s), so its queue grows "
                "for as long as the stream lasts: latencies are over the first arrival_window_s seconds"}
    # matched load: both forms at half of batch-of-one's saturation rate
    r_m = 0.5 * cap_hz
    mstream = poisson(r_m, matched_s)
    lat_m, wall_m = _served_stream(fnn, srv, pool, vels, mstream, n_steps, dt)
    arr_m, svc_m, ev_m = _batch_of_one(fnn, torch, pool, vels, mstream, n_steps, dt, 1e9, w1)
    l1m = 1e3 * _fifo_latencies(arr_m, svc_m)
    ev_served = sum(pool[k].n_atoms * n_steps for _, k in mstream)
    out["matched_load"] = {"rate_hz": r_m, "arrival_window_s": matched_s, "requests": len(mstream),
                           "served_bf16": {"p50_ms": float(np.percentile(lat_m, 50)),
                                           "p99_ms": float(np.percentile(lat_m, 99)),
                                           "atom_evals_per_s": ev_served / wall_m},
                           "batch_of_one_fp32x3": {"p50_ms": float(np.percentile(l1m, 50)),
                                                   "p99_ms": float(np.percentile(l1m, 99)),
                                                   "atom_evals_per_s": ev_m / max(arr_m[-1] if len(arr_m) else 1,
                                                                                 svc_m.sum())}}
    srv.close()
    return out


def train_bench(fnn, torch, synth, steps, warmup, M=1, precision="bf16"):
    """One training step of the 4096-molecule ragged batch (8..64 atoms each): energies and forces through
    the autograd function, the loss 0.99 mean (F - F*)^2 + 0.01 mean ((E - E*)/n)^2, and its parameter
    gradients (fnn_param_grads) by backward.  Device-resident inputs; CUDA events around each step."""
    import numpy as np
    s = synth.ragged_batch()
    w = synth.xavier_weights(M)
    ctx = fnn.Context(M)
    fnn.load_weights(ctx, w)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    params = [torch.tensor(np.asarray(getattr(w, k), np.float32), device="cuda", requires_grad=True)
              for k in fnn.PARAM_NAMES]
    E_ref, F_ref = synth.batch_targets(s)
    Et = torch.tensor(E_ref, device="cuda")
    Ft = torch.tensor(F_ref, dtype=torch.float32, device="cuda")
    n = torch.tensor(np.maximum(np.diff(s.mol_offsets), 1), dtype=torch.float64, device="cuda")

    def step():
        fnn.build_neighbors(ctx, ds, nl)
        for p in params:
            p.grad = None
        E, F = fnn.energy_forces_autograd(ctx, ds, nl, params, precision=precision)
        L = 0.99 * torch.mean((F - Ft) ** 2) + 0.01 * torch.mean(((E - Et) / n) ** 2)
        L.backward()
        return L

    for _ in range(warmup):
        step()
    fnn.check(ctx, "training warm-up")
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    fnn.profile_read(ctx)
    fnn.profile_enable(ctx, True)
    l0 = fnn.launch_count(ctx)
    torch.cuda.synchronize()
    for k in range(steps):
        ev[k][0].record(stream)
        L = step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = fnn.launch_count(ctx) - l0
    fnn.profile_enable(ctx, False)
    prof = fnn.profile_read(ctx)
    fnn.check(ctx, "training steps")
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    total = sum(v[0] for v in prof.values())
    top = sorted(prof.items(), key=lambda kv: -kv[1][0])[:8]
    return {"workload": f"ragged batch: 4096 molecules, 8-64 atoms, {s.n_atoms} atoms (gas phase)",
            "members": M, "precision": precision, "ms_per_step": ms, "atoms_per_s": s.n_atoms / (ms * 1e-3),
            "loss": float(L.detach()), "gpu_launches_per_step": launches / steps,
            "kernel_ms_per_step": total / steps,
            "kernel_share": {k: round(v[0] / total, 3) for k, v in top},
            "note": "forward (E, F) + loss + parameter gradients; the optimizer update is not timed"}


def latency_bench(fnn, torch, synth, reps: int = 200):
    """The 24-atom gas-phase cluster, one member: microseconds per energy+force evaluation (list rebuild
    included) as CUDA-graph replays back to back and as eager calls, for the FP32 and FP32X3 forms."""
    s = synth.gas24()
    out = {"workload": "gas24: 24-atom gas-phase cluster (10 H, 8 C, 3 N, 3 O), 6 A cube, seed 1", "members": 1}
    ctx = fnn.Context(1)
    fnn.load_weights(ctx, synth.xavier_weights(1))
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    for form in ("fp32", "fp32x3"):
        g = fnn.Graph(ctx, ds, nl, form)
        st = g.stream
        with torch.cuda.stream(st):
            for _ in range(10):
                g.launch()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                g.launch()
            b.record(st)
            torch.cuda.synchronize()
            graph_us = 1e3 * a.elapsed_time(b) / reps
            for _ in range(10):
                fnn.build_neighbors(ctx, ds, nl, stream=st)
                fnn.energy_forces(ctx, ds, nl, form, out=(g.E, g.F, g.W), stream=st)
            a.record(st)
            for _ in range(reps):
                fnn.build_neighbors(ctx, ds, nl, stream=st)
                fnn.energy_forces(ctx, ds, nl, form, out=(g.E, g.F, g.W), stream=st)
            b.record(st)
            torch.cuda.synchronize()
            eager_us = 1e3 * a.elapsed_time(b) / reps
        fnn.check(ctx, "latency", stream=st)
        out[form] = {"graph_us_per_eval": graph_us, "eager_us_per_eval": eager_us, "kernels_per_eval": g.kernels}
        g.close()
    return out


def md_bench(fnn, torch, synth, n_steps: int = 1000, M: int = 8, check: bool = True):
    """The periodic water box (216 H2O, 648 atoms) under NVE velocity Verlet: n_steps force evaluations at
    0.5 fs, 8-member ensemble, FP32X3 networks, list skin 1 A rebuilt every 10 steps and by the skin/2 guard,
    Maxwell-Boltzmann velocities at 300 K; fnn_md_run_ex on a side stream (10-step blocks as CUDA-graph
    replays with conditional rebuilds).  Then the same run in ten continued pieces of 100 steps, the oracle
    evaluated at the GPU positions after each (energy per atom, forces)."""
    import numpy as np
    s = synth.water216()
    ctx = fnn.Context(M, skin=1.0)
    w = synth.xavier_weights(M)
    fnn.load_weights(ctx, w)
    v0 = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
    v0[:, :3] = torch.from_numpy(synth.maxwell_boltzmann(s.Z, 300.0, seed=2))
    nl = fnn.NeighborList(ctx)
    stream = torch.cuda.Stream()

    def fresh():
        return fnn.DeviceSystem.from_structures(s), v0.clone().cuda()

    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ds, vel = fresh()
        fnn.md_run_ex(ctx, ds, vel, nl, "fp32x3", 20, 0.5, 10, stream=stream)   # warm-up (sizes, graphs)
        fnn.check(ctx, "md warm-up", stream=stream)
        ds, vel = fresh()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = fnn.launch_count(ctx)
        a.record(stream)
        E, K, F, cnt = fnn.md_run_ex(ctx, ds, vel, nl, "fp32x3", n_steps, 0.5, 10, kinetic=True, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        fnn.check(ctx, "md", stream=stream)
    ms = a.elapsed_time(b)
    launches = fnn.launch_count(ctx) - l0
    Ep, Kk = E.cpu().numpy()[:, 0], K.cpu().numpy()[:, 0]
    Et = Ep + Kk
    out = {"workload": "water216: 216 rigid H2O (648 atoms), 18.64 A periodic cube, seed 2", "members": M,
           "precision": "fp32x3", "steps": n_steps, "dt_fs": 0.5, "rebuild_every": 10, "skin_A": 1.0,
           "skin_guard": True, "ms_total": ms, "ms_per_step": ms / n_steps,
           "atom_evals_per_s": s.n_atoms * n_steps / (ms * 1e-3), "gpu_launches_per_step": launches / n_steps,
           "potential_first_last": [float(Ep[0]), float(Ep[-1])], "kinetic_first_last": [float(Kk[0]), float(Kk[-1])],
           "total_first_last": [float(Et[0]), float(Et[-1])],
           "total_drift_per_atom": float((Et[-1] - Et[0]) / s.n_atoms)}
    if check:
        import oracle
        ds, vel = fresh()
        worst_e = worst_f = 0.0
        guard = rebuilds = 0
        for chunk in range(n_steps // 100):
            with torch.cuda.stream(stream):
                Ec, _, Fc, c = fnn.md_run_ex(ctx, ds, vel, nl, "fp32x3", 101, 0.5, 10, counters=True, stream=stream)
            fnn.check(ctx, "md snapshot run", stream=stream)
            guard += c["guard_rebuilds"]
            rebuilds += c["rebuilds"]
            st = synth.Structures(s.Z, ds.pos[:, :3].cpu().numpy(), s.mol_offsets, s.cell, s.pbc)
            r = oracle.energy_forces(st, w)
            worst_e = max(worst_e, abs(float(Ec[-1, 0]) - r.energy[0]) / s.n_atoms)
            worst_f = max(worst_f, float(np.abs(Fc.cpu().numpy() - r.forces).max()))
        out["oracle_snapshots"] = {"every_steps": 100, "count": n_steps // 100, "max_dE_per_atom": worst_e,
                                   "max_dF": worst_f, "rebuilds": rebuilds, "guard_rebuilds": guard,
                                   "note": "the run in ten continued pieces of 100 steps; the oracle evaluated at "
                                           "the GPU positions after each"}
    return out


def drift_bench(fnn, torch, synth, forms=("fp32", "fp32x3", "bf16", "fp8"), n_steps=4000, dt=0.1, M=1):
    """Energy conservation by precision form (section V.E: FP32 conserves the total energy in NVE, BF16 and
    TF32 matmuls do not): the water box under NVE at 0.1 fs for n_steps, one member (the paper's ANI-2x
    member 0), skin 1 A with the guard; total energy = potential + kinetic per step.  Reported per form: the
    linear drift (kcal/mol per ps per atom), the spread about it and the largest excursion from the start
    (kcal/mol per atom).  Then a Langevin (BAOAB) run at 300 K: its mean kinetic temperature."""
    import numpy as np
    s = synth.water216()
    w = synth.xavier_weights(M)
    v0 = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
    v0[:, :3] = torch.from_numpy(synth.maxwell_boltzmann(s.Z, 300.0, seed=2))
    stream = torch.cuda.Stream()
    out = {"workload": "water216, NVE velocity Verlet", "dt_fs": dt, "steps": n_steps, "members": M, "forms": {}}
    t_ps = np.arange(n_steps) * dt * 1e-3
    for form in forms:
        ctx = fnn.Context(M, skin=1.0)
        fnn.load_weights(ctx, w)
        nl = fnn.NeighborList(ctx)
        ds = fnn.DeviceSystem.from_structures(s)
        vel = v0.clone().cuda()
        with torch.cuda.stream(stream):
            E, K, _, cnt = fnn.md_run_ex(ctx, ds, vel, nl, form, n_steps, dt, 10, kinetic=True, counters=True,
                                         stream=stream)
        fnn.check(ctx, f"drift {form}", stream=stream)
        Et = (E.cpu().numpy()[:, 0] + K.cpu().numpy()[:, 0]) / s.n_atoms
        slope, icpt = np.polyfit(t_ps, Et, 1)
        out["forms"][form] = {"drift_per_atom_per_ps": float(slope), "spread_per_atom": float(np.std(Et - (slope * t_ps + icpt))),
                              "max_excursion_per_atom": float(np.abs(Et - Et[0]).max()),
                              "kinetic_per_atom_mean": float(K.cpu().numpy()[:, 0].mean() / s.n_atoms),
                              "rebuilds": cnt["rebuilds"], "guard_rebuilds": cnt["guard_rebuilds"]}
    M8 = 8   # the Langevin run uses the 8-member ensemble of the NVE water run (smoother random-weight surface)
    ctx = fnn.Context(M8, skin=1.0)
    fnn.load_weights(ctx, synth.xavier_weights(M8))
    nl = fnn.NeighborList(ctx)
    ds = fnn.DeviceSystem.from_structures(s)
    vel = v0.clone().cuda()
    n_l, dt_l, gamma = 1000, 0.5, 0.01
    with torch.cuda.stream(stream):
        E, K, _, cnt = fnn.md_run_ex(ctx, ds, vel, nl, "fp32x3", n_l, dt_l, 10, integrator="langevin",
                                     temperature_K=300.0, friction_per_fs=gamma, seed=2405, kinetic=True,
                                     counters=True, stream=stream)
    fnn.check(ctx, "langevin", stream=stream)
    Kk = K.cpu().numpy()[:, 0]
    kb = 0.0019872041
    out["langevin"] = {"integrator": "BAOAB", "members": M8, "T_bath_K": 300.0, "friction_per_fs": gamma, "dt_fs": dt_l,
                       "steps": n_l, "T_kinetic_mean_K_second_half": float(2 * Kk[n_l // 2:].mean() / (3 * s.n_atoms * kb)),
                       "rebuilds": cnt["rebuilds"], "guard_rebuilds": cnt["guard_rebuilds"]}
    return out


def variants_bench(fnn, torch, synth, steps=10, warmup=3):
    """The descriptor variants on the 23,558-atom box: the CRATE angular resource (Appendix A) and its
    vector-Jacobian product (random V and dL/dg, seeded), and one energy + force step of the FP32X3 form with
    each switching function (section II.A), M = 8; CUDA events around each call, L2 flushed before each."""
    import numpy as np
    pk = peaks()
    s = synth.mix23558()
    ds = fnn.DeviceSystem.from_structures(s)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    out = {"workload": "mix23558 (23,558 atoms, 62.2 A periodic box)"}
    rng = np.random.default_rng(17)
    V = torch.from_numpy((rng.standard_normal((7, 8, 32)) / 4).astype(np.float32)).cuda()
    G = torch.from_numpy(rng.standard_normal((s.n_atoms, 4, 32)).astype(np.float32)).cuda()
    ctx = fnn.Context(1)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    nnz = fnn.nlist_nnz(nl)
    g = torch.empty((s.n_atoms, 4, 32), dtype=torch.float32, device="cuda")
    ms_f = timed(lambda: fnn.crate_angular(ctx, ds, nl, V, out=g))
    ms_v = timed(lambda: fnn.crate_angular_vjp(ctx, ds, nl, V, G))
    fnn.check(ctx, "crate")
    # algorithmic bytes: positions, the list (index + shift per entry), the resource row (and dL/dg, gradient)
    b_f = s.n_atoms * (16 + 512) + nnz * 8
    b_v = s.n_atoms * (16 + 512 + 12) + nnz * 8
    out["crate_angular"] = {"ms": ms_f, "atoms_per_s": s.n_atoms / (ms_f * 1e-3),
                            "achieved_gbs": b_f / (ms_f * 1e-3) / 1e9, "hbm_frac": b_f / (ms_f * 1e-3) / 1e9 / pk["hbm_gbs"]}
    out["crate_angular_vjp"] = {"ms": ms_v, "atoms_per_s": s.n_atoms / (ms_v * 1e-3),
                                "achieved_gbs": b_v / (ms_v * 1e-3) / 1e9,
                                "hbm_frac": b_v / (ms_v * 1e-3) / 1e9 / pk["hbm_gbs"]}
    w = synth.xavier_weights(8)
    for sw in ("cosine", "polynomial", "exponential"):
        c = fnn.Context(8, switch=sw)
        fnn.load_weights(c, w)
        n2 = fnn.NeighborList(c)
        fnn.build_neighbors(c, ds, n2, checked=True)
        E = torch.empty(s.n_mol, dtype=torch.float64, device="cuda")
        F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device="cuda")
        Wv = torch.empty((s.n_mol, 3, 3), dtype=torch.float64, device="cuda")

        def step():
            fnn.build_neighbors(c, ds, n2)
            fnn.energy_forces(c, ds, n2, "fp32x3", out=(E, F, Wv))
        ms = timed(step)
        fnn.check(c, f"switch {sw}")
        out[f"step_fp32x3_{sw}"] = {"ms": ms, "atom_evals_per_s": s.n_atoms / (ms * 1e-3), "members": 8,
                                    "note": "eager step (list + energies + forces + virials)"}
    return out


def rpmd_bench(fnn, torch, synth, P=32, n_steps=200, dt=0.25, T=300.0):
    """Ring-polymer MD of the water box (section V.D): P beads of 648 atoms as one batch of P structures,
    one member, FP32X3, skin 1 A rebuilt every 10 steps and by the guard; exact normal-mode free steps.
    Reports bead-atom evaluations per second and the ring-polymer Hamiltonian's drift."""
    import numpy as np
    s = synth.water216()
    rng = np.random.default_rng(7)
    x0 = (np.asarray(s.pos, np.float64)[None] + 0.02 * rng.standard_normal((P, s.n_atoms, 3))).astype(np.float32)
    v0 = np.stack([synth.maxwell_boltzmann(s.Z, T, seed=100 + b) for b in range(P)]).astype(np.float32)
    ctx = fnn.Context(1, skin=1.0)
    fnn.load_weights(ctx, synth.xavier_weights(1))
    nl = fnn.NeighborList(ctx)
    stream = torch.cuda.Stream()

    def fresh():
        ds = fnn.bead_system(s, x0)
        vel = torch.zeros((P * s.n_atoms, 4), dtype=torch.float32)
        vel[:, :3] = torch.from_numpy(v0.reshape(-1, 3))
        return ds, vel.cuda()

    with torch.cuda.stream(stream):
        ds, vel = fresh()
        fnn.rpmd_run(ctx, ds, vel, nl, "fp32x3", P, 20, dt, T, 10, stream=stream)   # warm-up (sizes, graphs)
        fnn.check(ctx, "rpmd warm-up", stream=stream)
        ds, vel = fresh()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        E, H, F, cnt = fnn.rpmd_run(ctx, ds, vel, nl, "fp32x3", P, n_steps, dt, T, 10, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        fnn.check(ctx, "rpmd", stream=stream)
    ms = a.elapsed_time(b)
    Hh = H.cpu().numpy()
    n = P * s.n_atoms
    return {"workload": f"water216 ring polymer, {P} beads ({n} bead atoms per evaluation)", "members": 1,
            "precision": "fp32x3", "beads": P, "steps": n_steps, "dt_fs": dt, "T_K": T, "ms_total": ms,
            "ms_per_step": ms / n_steps, "bead_atom_evals_per_s": n * n_steps / (ms * 1e-3),
            "hamiltonian_first_last": [float(Hh[0]), float(Hh[-1])],
            "hamiltonian_drift_per_bead_atom": float((Hh[-1] - Hh[0]) / n)}


def time_form(fnn, torch, ctx, ds, nl, E, F, Wv, flush, form, steps, warmup, barrier):
    """K timed steps of one form, each a replay of the step's CUDA graph (list rebuild + energies +
    forces + virials) on its own stream, CUDA events around every replay (L2 flushed outside them);
    then the same steps launched eagerly with per-kernel events for the kernel table."""
    g = fnn.Graph(ctx, ds, nl, form, virial=True, rebuild=True)
    stream = g.stream
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g.launch()
        fnn.check(ctx, f"warm-up {form}", stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        launches0 = fnn.launch_count(ctx)
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(stream)
                g.launch()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        barrier()
        launches = fnn.launch_count(ctx) - launches0
        fnn.check(ctx, f"timed steps {form}", stream=stream)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        E.copy_(g.E)
        F.copy_(g.F)
        Wv.copy_(g.W)
    torch.cuda.synchronize()
    g.close()

    # per-kernel times: the same steps eagerly, an event pair around every launch (outside the timing above)
    def step():
        fnn.build_neighbors(ctx, ds, nl)
        fnn.energy_forces(ctx, ds, nl, form, out=(E, F, Wv))

    fnn.profile_read(ctx)
    fnn.profile_enable(ctx, True)
    for k in range(steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    fnn.profile_enable(ctx, False)
    prof = fnn.profile_read(ctx)
    fnn.check(ctx, f"profiled steps {form}")
    return ms, prof, launches, clk.summary()


def kernel_table(prof, steps, n_atoms, nnz, M, form, pk):
    """Per kernel: time per launch, share, and the roofline of its algorithmic work.  Kernel times are
    CUDA events around single launches inside a millisecond-long step, so tensor-bound kernels are held
    against the measured burst bf16 rate (fp8: twice it, the nominal ratio)."""
    ffma_peak = N_SM * FFMA_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12   # TFLOP/s
    tensor_peak = pk["bf16_tflops"] * (2 if form == "fp8" else 1)
    kernels = {}
    total = sum(v[0] for v in prof.values())
    for name, (tot_ms, n) in prof.items():
        entry = {"ms_per_launch": tot_ms / n, "launches_per_step": n / steps, "share": tot_ms / total if total else None}
        wk = kernel_work(name, n_atoms, nnz, M)
        if wk:
            bound, amount, u, executed = wk
            t = tot_ms / n * 1e-3
            if u == "B":
                entry.update(bound=bound, achieved=amount / t / 1e9, unit="GB/s", peak=pk["hbm_gbs"])
            else:
                entry.update(bound=bound, achieved=amount / t / 1e12, unit="TFLOP/s",
                             peak=ffma_peak if bound == "alu" else tensor_peak)
                if executed:   # the split products the tensor pipe runs, as a fraction of the same peak
                    entry["executed_frac"] = executed / t / 1e12 / entry["peak"]
            entry["frac"] = entry["achieved"] / entry["peak"]
        kernels[name] = entry
    dom = max((k for k in kernels if "bound" in kernels[k]), key=lambda k: prof[k][0])
    d = kernels[dom]
    roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
            "frac": d["frac"],
            "peak_src": (f"FP32 FFMA: {N_SM} SMs x {FFMA_LANES_PER_SM} lanes x 2 x {pk['sm_max_mhz']:.0f} MHz"
                         if d["bound"] == "alu" else
                         f"{pk['src']} {'HBM copy' if d['bound'] == 'hbm' else 'bf16 burst'}"),
            "work": ("algorithmic: one FP32 product per layer (2 in out FLOP per row and member); the FP32X3 "
                     "split runs three bf16 products, reported as executed_frac" if d["unit"] == "TFLOP/s"
                     else "algorithmic bytes per launch")}
    if "executed_frac" in d:
        roof["executed_frac"] = d["executed_frac"]
    return kernels, roof


def network_summary(kernels, steps, n_atoms, M, form, pk):
    """Every network product of one form's step together: their algorithmic FLOPs (one product of 2 in out
    FLOP per row and member and layer, forward and input gradient) over their summed kernel time, against
    the tensor peak the kernel table uses (the FP32 form against the FFMA rate)."""
    ms, flops = 0.0, 0.0
    for name, v in kernels.items():
        wk = kernel_work(name, n_atoms, 0, M)
        if wk and wk[2] == "FLOP":
            t = v["ms_per_launch"] * v["launches_per_step"]
            ms += t
            flops += wk[1] * v["launches_per_step"]
    if ms <= 0:
        return None
    tf = flops / (ms * 1e-3) / 1e12
    if form == "fp32":
        peak = N_SM * FFMA_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
    else:
        peak = pk["bf16_tflops"] * (2 if form == "fp8" else 1)
    return {"ms": round(ms, 4), "gflop": round(flops / 1e9, 2), "achieved_tflops": round(tf, 1),
            "peak_tflops": round(peak, 1), "frac": round(tf / peak, 4)}


def section(name, fn, *a, **kw):
    """An optional measurement: its result, or the error it raised (the JSON line is printed either way)."""
    try:
        return fn(*a, **kw)
    except Exception as e:   # noqa: BLE001 - reported, not hidden
        print(f"bench: section {name} failed: {e!r}", file=sys.stderr, flush=True)
        return {"error": f"{type(e).__name__}: {e}"[:500]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fnn", choices=["fnn", "reference"])
    ap.add_argument("--precision", default="fp32x3", choices=["fp32", "fp32x3", "bf16", "bf16_fused", "fp8"],
                    help="form whose throughput is the headline value")
    ap.add_argument("--forms", default="fp32x3,fp32,bf16,bf16_fused,fp8", help="forms timed and reported (comma separated)")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--no-md", action="store_true", help="skip the water-box MD measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-stream measurement")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-pool", type=int, default=4096)
    ap.add_argument("--no-drift", action="store_true", help="skip the energy-drift study")
    ap.add_argument("--no-cpu-plan", action="store_true", help="skip the oracle timings of every configuration")
    ap.add_argument("--no-variants", action="store_true", help="skip the CRATE / switch measurements")
    ap.add_argument("--no-rpmd", action="store_true", help="skip the ring-polymer measurement")
    ap.add_argument("--only", default=None, choices=["variants", "rpmd", "md", "drift", "latency", "serve"],
                    help="run one measurement section alone and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    from paper_2405_01491_b300 import fnn, synth

    if args.only:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        fn = {"variants": lambda: variants_bench(fnn, torch, synth, args.steps, args.warmup),
              "rpmd": lambda: rpmd_bench(fnn, torch, synth),
              "md": lambda: md_bench(fnn, torch, synth, check=False),
              "drift": lambda: drift_bench(fnn, torch, synth),
              "latency": lambda: latency_bench(fnn, torch, synth),
              "serve": lambda: serve_bench(fnn, torch, synth, duration_s=args.serve_seconds,
                                           pool_n=args.serve_pool)}[args.only]
        print(json.dumps({"section": args.only, "result": fn()}), flush=True)
        return 0

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ranks = Ranks("nccl", "cuda")
    world, rank = ranks.world, ranks.rank
    barrier, max_over_ranks = ranks.barrier, ranks.max

    M = 8
    s = synth.mix23558()
    w = synth.xavier_weights(M)
    ctx = fnn.Context(M)
    fnn.load_weights(ctx, w)
    ds = fnn.DeviceSystem.from_structures(s)
    nl = fnn.NeighborList(ctx)
    fnn.build_neighbors(ctx, ds, nl, checked=True)
    nnz = fnn.nlist_nnz(nl)
    E = torch.empty(s.n_mol, dtype=torch.float64, device="cuda")
    F = torch.empty((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    Wv = torch.empty((s.n_mol, 3, 3), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    pk = peaks()
    forms = [f for f in args.forms.split(",") if f]
    if args.precision not in forms:
        forms.insert(0, args.precision)

    results = {}
    for form in forms:
        ms, prof, launches, clocks = time_form(fnn, torch, ctx, ds, nl, E, F, Wv, flush, form, args.steps,
                                               args.warmup, barrier)
        fnn.energy_forces(ctx, ds, nl, form, out=(E, F, Wv))   # the reported errors: an eager evaluation
        fnn.check(ctx, form)
        results[form] = dict(ms=max_over_ranks(ms), prof=prof, launches=launches, clocks=clocks,
                             E=E.cpu().numpy().copy(), F=F.cpu().numpy().copy())

    # end to end through the C ABI with host buffers (copies inside the timed region), headline form
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hs = synth.Structures(pin(s.Z), pin(s.pos), pin(s.mol_offsets), pin(s.cell), pin(s.pbc), s.name)
    hout = (pin(np.zeros(s.n_mol)), pin(np.zeros((s.n_atoms, 3), np.float32)), pin(np.zeros((s.n_mol, 3, 3))))
    for _ in range(max(1, args.warmup)):
        fnn.energy_forces_host(ctx, hs, args.precision, out=hout)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fnn.energy_forces_host(ctx, hs, args.precision, out=hout)
    t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps)
    h2d = s.n_atoms * (4 + 12) + (s.n_mol + 1) * 4 + s.n_mol * (36 + 1)
    d2h = s.n_mol * 8 + s.n_atoms * 12 + s.n_mol * 72

    base, ref = (None, None)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, ref = oracle_full(M)
    plan = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.no_cpu_plan:
        plan = section("cpu_plan", cpu_plan)
    serve = None
    if world == 1 and not args.no_serve:
        serve = section("serve", serve_bench, fnn, torch, synth, duration_s=args.serve_seconds, pool_n=args.serve_pool)
    md = latency = drift = None
    if world == 1 and not args.no_md:
        md = section("md", md_bench, fnn, torch, synth)
        latency = section("latency", latency_bench, fnn, torch, synth)
    if world == 1 and not args.no_drift:
        drift = section("drift", drift_bench, fnn, torch, synth)
    variants = rpmd = None
    if world == 1 and not args.no_variants:
        variants = section("variants", variants_bench, fnn, torch, synth)
    if world == 1 and not args.no_rpmd:
        rpmd = section("rpmd", rpmd_bench, fnn, torch, synth)
    train = None
    if world == 1 and not args.no_train:
        train = {p: section(f"train_{p}", train_bench, fnn, torch, synth, args.steps, max(3, args.warmup), precision=p)
                 for p in ("bf16", "fp32")}

    head = results[args.precision]
    kernels, roof = kernel_table(head["prof"], args.steps, s.n_atoms, nnz, M, args.precision, pk)
    roof["traffic"] = recorded_traffic(roof["kernel"], source_digest(roof["kernel"]))
    form_report = {}
    for form, r in results.items():
        ks, rf = kernel_table(r["prof"], args.steps, s.n_atoms, nnz, M, form, pk)
        entry = {"value": world * s.n_atoms / (r["ms"] * 1e-3), "ms_per_step": r["ms"], "gpu_launches": r["launches"],
                 "dominant": rf, "kernel_ms": {k: round(v["ms_per_launch"] * v["launches_per_step"], 4)
                                               for k, v in ks.items()},
                 "kernel_frac": {k: round(v["frac"], 4) for k, v in ks.items() if "frac" in v},
                 "networks": network_summary(ks, args.steps, s.n_atoms, M, form, pk)}
        if ref is not None:
            entry["max_dE_per_atom"] = float(np.abs(r["E"] - ref.energy).max() / s.n_atoms)
            entry["max_dF"] = float(np.abs(r["F"] - ref.forces).max())
            entry["rms_rel_dF"] = float(np.sqrt(np.mean((r["F"] - ref.forces) ** 2) / np.mean(ref.forces ** 2)))
        form_report[form] = entry

    line = {"metric": METRIC, "value": world * s.n_atoms / (head["ms"] * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp32x3": "f32", "bf16": "bf16", "bf16_fused": "bf16", "fp8": "e4m3"}[args.precision], "data": "synthetic",
            "config": arm_config(args.precision, nnz, world),
            "roofline": roof, "gpu_launches": int(head["launches"]),
            "e2e": {"value": world * s.n_atoms / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": head["clocks"], "forms": form_report, "kernels": kernels, "source_digest": source_digest()}
    if base is not None:
        line["cpu_baseline"] = base
        if plan is not None:
            line["cpu_baseline"]["plan"] = plan
    if serve is not None:
        line["serve"] = serve
    if train is not None:
        line["train"] = train
    if md is not None:
        line["md"] = md
    if latency is not None:
        line["latency"] = latency
    if drift is not None:
        line["drift"] = drift
    if variants is not None:
        line["variants"] = variants
    if rpmd is not None:
        line["rpmd"] = rpmd
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
