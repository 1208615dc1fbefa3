"""Benchmark of the GB300 state-vector path (one JSON line on rank 0).

Workload (the configuration the headline metric is quoted on): the
layered sparse-gate circuit at n = 30 qubits in complex128 (a 16 GiB state,
larger than L2): H on every qubit, then 20 layers of [CNOT ladder; CZ on a
random perfect matching; T or S on a random half; RZ(theta) on every
qubit], then the readouts norm^2 and <Z_0>.  One step = reset to |0...0>,
apply the whole circuit, read out.  Metric: amplitude updates per second
(one amplitude rewritten by one gate, counted algorithmically), with the
fused tile kernel's HBM bandwidth against the measured peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fused|per_gate]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

With N > 1 (torchrun) every rank runs an independent replica of the
workload on its own GPU (the path does not shard); value = all ranks'
updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitude-updates/s"
FALLBACK_HBM_GBS = 6800.0


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mera", choices=["mera", "reference"])
    p.add_argument("--mode", default="fused", choices=["fused", "per_gate"])
    p.add_argument("--workload", default="layered", choices=["layered", "grover"])
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--layers", type=int, default=20)
    p.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-qnn", action="store_true")
    p.add_argument("--qnn-requests", type=int, default=512)
    return p.parse_args()


def _workload(args):
    from paper_2411_15332_gb300 import inputs
    if args.workload == "grover":
        ops, _m = inputs.grover_circuit(args.n, 8, seed=3)
        return ops
    return inputs.layered_circuit(args.n, args.layers, seed=2)


def _workload_name(args):
    n, dt = args.n, ("complex128" if args.dtype == "c128" else "complex64")
    if args.workload == "grover":
        return (f"grover_n{n}: n={n} {dt}, |0..0>, H on all, then 8 x [sign flip of a seeded index, H on all, "
                f"sign flip of |0..0>, H on all], readout norm^2 and <Z_0>")
    return (f"layered_n{n}: n={n} {dt}, |0..0>, H on all, "
            f"then {args.layers} x [CNOT ladder q->q+1, CZ on a seeded perfect matching, T/S on a seeded half, "
            f"RZ(theta~U[0,2pi)) on all], readout norm^2 and <Z_0>")


# ----------------------------------------------------------- clocks --------
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- helpers -------
def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks of the default process group (the
    slowest replica's time); the value itself without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, slowest_ms: float) -> float:
    """Whole-job rate: every replica's units over the slowest replica's time."""
    return units_per_rank * world / (slowest_ms / 1e3)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _tile_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_15332_gb300", "csrc")
    for f in ("tile.cuh", "fused.cu", "kernels.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """Per-launch DRAM bytes of the tile kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "tile_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") == _tile_source_hash():
            return d
    except Exception:
        pass
    return None


def _cpu_baseline(sample_seconds=15.0):
    """The FP64 oracle on the host cores, single-threaded, on a bounded
    sample of the same circuit family (reduced n; amplitude updates are
    counted on the sample itself)."""
    code = r"""
import json, os, sys, time
sys.path.insert(0, %r)
from paper_2411_15332_gb300 import inputs
from oracle import statevector as sv
n = 22
ops = inputs.layered_circuit(n, 20, seed=2)
N = 1 << n
def upd(o):
    name, t, c, p, cv = o
    frac = {"X": 1.0, "H": 1.0, "RZ": 1.0, "Z": 0.5, "S": 0.5, "T": 0.5}[name]
    return N * frac / (1 << len(c))
psi = sv.zero_state(n)
t0 = time.perf_counter(); done = 0.0; g = 0
while g < len(ops) and time.perf_counter() - t0 < %f:
    sv.apply_op(psi, n, ops[g]); done += upd(ops[g]); g += 1
dt = time.perf_counter() - t0
print(json.dumps({"value": done / dt, "gates": g, "seconds": dt, "n": n}))
""" % (ROOT, sample_seconds)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": (f"oracle (numpy FP64, 1 thread) applying the first {d['gates']} gates of the same "
                       f"layered circuit family at n={d['n']} for {d['seconds']:.1f} s")}


def _qnn_section(args):
    """Secondary QNN measurements: the serving workload (a bounded prefix of
    the 4096 seeded requests, n ~ U{8..20}, L ~ U{4..12}, complex64) served
    with continuous batching vs one circuit at a time through the plain
    single-state path, and adjoint training gradients (1024 circuits,
    n = 16, 10 layers, 320 angles)."""
    import numpy as np
    import torch
    import paper_2411_15332_gb300 as mera
    from paper_2411_15332_gb300 import inputs
    from paper_2411_15332_gb300.serve import Server, requests_from_workload
    out = {}
    reqs = inputs.qnn_requests(4096, seed=4)[: args.qnn_requests]
    # plain: one circuit at a time (fused single-state path), a sample
    sample = reqs[:64]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat = []
    for r in sample:
        t1 = time.perf_counter()
        st = mera.State(r["n"], "c64")
        st.apply_circuit(inputs.ansatz_ops(r["n"], r["theta"]), mode="fused")
        st.observables(0)
        st.close()
        lat.append(time.perf_counter() - t1)
    plain_s = time.perf_counter() - t0
    plain_rate = len(sample) / plain_s
    out["plain"] = {"circuits_per_s": plain_rate, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                    "p99_ms": float(np.percentile(lat, 99) * 1e3), "sample": len(sample)}
    # serving: saturation (all requests at t=0) and Poisson arrivals at 0.8x plain capacity... of the server
    srv = Server(dtype="c64", mem_budget=64 << 30, slots_per_n=512)
    srv.run(requests_from_workload(reqs))
    sat = srv.stats()
    rate = 0.8 * sat["circuits_per_s"]
    srv2 = Server(dtype="c64", mem_budget=64 << 30, slots_per_n=512)
    srv2.run(requests_from_workload(reqs, rate=rate))
    poi = srv2.stats()
    out["serving"] = {"requests": len(reqs), "saturation": sat,
                      "poisson": dict(poi, rate_per_s=rate)}
    # training: adjoint gradients of the 1024-circuit batch
    theta = inputs.qnn_batch(1024, 16, 10, seed=5)
    b = mera.Batch(16, 1024, "c64")
    b.adjoint_grad(theta[:8])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.adjoint_grad(theta)
    tr = time.perf_counter() - t0
    out["training"] = {"circuits": 1024, "params_per_circuit": 320, "seconds": tr,
                       "circuit_gradients_per_s": 1024 / tr, "dtype": "c64"}
    b.close()
    return out


# ----------------------------------------------------------- arms ----------
def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = []
    for _ in range(args.warmup):
        pass
    per = max(5.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    last = None
    for _ in range(args.steps):
        last = _cpu_baseline(sample_seconds=min(per, 20.0))
        if last["value"] is not None:
            vals.append(last["value"])
    value = statistics.median(vals) if vals else None
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(args), "n": args.n,
                       "note": "CPU oracle timed on a bounded sample at n=22 of the same circuit family"},
            "cpu_baseline": dict(last or {}, value=value),
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _arith_dtype(args):
    """What the timed kernels compute in: complex128 fused passes keep the
    state as int64 fixed point; the per-gate kernels use float64."""
    if args.dtype == "c64":
        return "f32"
    return "i64" if args.mode == "fused" else "f64"


def _arith_note(args):
    if args.dtype == "c64":
        return "float32 state and arithmetic, float64 reductions"
    if args.mode == "fused":
        note = ("complex128 state held as int64 fixed point across the circuit's tile passes "
                "(global scale from a norm bound; exact butterflies and moves; 31-bit-limb integer "
                "products for phases, rounding to nearest); float64 at the circuit's ends and in reductions")
        if args.workload == "grover":
            note = note.replace("rounding to nearest", "roundings dithered by a hash of the amplitude index, "
                                "since Hadamard layers follow the sign flips; an odd level's sqrt(2) carried "
                                "to the next pass")
        return note
    return "float64 per-gate kernels"


def run_mera(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2411_15332_gb300.build import build
    build()
    import paper_2411_15332_gb300 as mera
    from paper_2411_15332_gb300.workload import amplitude_updates

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    n = args.n
    ops = _workload(args)
    upd = amplitude_updates(ops, n)
    st = mera.State(n, args.dtype)
    stream = torch.cuda.current_stream()

    def step():
        st.set_basis(0)
        st.apply_circuit(ops, mode=args.mode)
        return st.observables(0)

    for _ in range(max(args.warmup, 0)):
        obs = step()

    # timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clock = ClockSampler(local_rank)
    clock.start()
    mera.profile_enable(True)
    l0 = mera.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        obs = step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = mera.launch_count() - l0
    prof = mera.profile_read()
    mera.profile_enable(False)
    clocks = clock.stop()
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), device="cuda")
    ms_per_step = total_ms / args.steps
    value = job_throughput(upd, world, ms_per_step)

    # roofline of the dominant kernel (the fused tile pass)
    peak, peak_kind = _peaks()
    kcls = "tile" if args.mode == "fused" else "gate"
    nl, kms, kbytes = prof[kcls]
    achieved = (kbytes / nl) / (kms / nl / 1e3) / 1e9 if nl else None
    # DRAM traffic per launch from the committed ncu capture: only for the
    # kernels and workload it was taken on (the layered circuit's tile
    # passes), scaled from n = 28 by the state size
    tr = _ncu_traffic() if (kcls == "tile" and args.workload == "layered") else None
    traffic = tr["dram_bytes_per_launch_n28"] * 2.0 ** (args.n - 28) if tr else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": traffic,
                "kernel": "k_hpass / k_dpass / k_tile (fused tile passes)" if kcls == "tile" else "per-gate kernels",
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "kernel_launches": nl, "kernel_ms": kms,
                "kernel_share": kms / total_ms if total_ms else None,
                "algorithmic_bytes_per_launch": (kbytes / nl) if nl else None}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        try:
            eb = 16 if args.dtype == "c128" else 8
            host = torch.zeros((1 << n) * 2, dtype=torch.float64 if eb == 16 else torch.float32).pin_memory()
            host[0] = 1.0
            hp = host.numpy().view(np.complex128 if eb == 16 else np.complex64)
            for _ in range(1):
                st.from_numpy(hp)
                st.apply_circuit(ops, mode=args.mode)
                st.observables(0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                st.from_numpy(hp)                       # H2D of the input state
                st.apply_circuit(ops, mode=args.mode)   # ops table is copied per launch
                res = st.observables(0)                 # D2H of the result
            e2e_s = (time.perf_counter() - t0) / args.steps
            ops_bytes = 80 * len(ops)
            e2e = {"value": upd * world / e2e_s, "unit": METRIC,
                   "h2d_bytes_per_step": (1 << n) * eb + ops_bytes, "d2h_bytes_per_step": 24,
                   "seconds_per_step": e2e_s}
            del host
        except Exception as ex:  # pinned allocation can fail on small hosts
            e2e = {"value": None, "unit": METRIC, "error": str(ex)[:200]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = _cpu_baseline()
    qnn = None
    if rank == 0 and world == 1 and not args.no_qnn and args.workload == "layered":
        st.close()
        st.tensor = None            # release the 16 GiB state before the QNN runs
        torch.cuda.empty_cache()
        try:
            qnn = _qnn_section(args)
        except Exception as ex:
            qnn = {"error": str(ex)[:300]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": _arith_dtype(args),
                "data": "synthetic",
                "config": {"workload": _workload_name(args), "n": n, "state": "complex128" if args.dtype == "c128" else "complex64",
                           "arithmetic": _arith_note(args),
                           "amplitude_updates_per_step": upd, "mode": args.mode,
                           "parallelism": f"replicas x{world}",
                           "l2": "state (%d GiB) larger than L2 (129 MB); no flush needed" % (((1 << n) * (16 if args.dtype == 'c128' else 8)) >> 30),
                           "readout": {"norm2": obs[0], "z0": obs[1]}},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks, "kernel_classes": prof, "qnn": qnn}
        print(json.dumps(line), flush=True)
    st.close()


def main():
    args = _args()
    if args.n is None:
        args.n = 33 if args.workload == "grover" else 30
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "mera" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_mera(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
