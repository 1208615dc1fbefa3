"""Benchmark of the GB300 state-vector path (one JSON line on rank 0).

Headline workload (the configuration the metric is quoted on): the layered
sparse-gate circuit at n = 30 qubits in complex128 (a 16 GiB state, larger
than L2): H on every qubit, then 20 layers of [CNOT ladder; CZ on a random
perfect matching; T or S on a random half; RZ(theta) on every qubit], then
the readouts norm^2 and <Z_0>.  One step = reset to |0...0>, apply the
whole circuit (fused tile passes), read out.  Metric: amplitude updates
per second (one amplitude rewritten by one gate, counted algorithmically),
with the dominant kernel's HBM bandwidth against the measured peak.

Sections on the same line (one GPU, rank 0):
  grover_n33    Grover-style circuit, n = 33 complex128 (128 GiB), fused;
                error of all 2^33 amplitudes against the closed form
  per_gate_n30  the headline circuit through the per-gate kernels
  random_n30    a random circuit with the 13-gate mix of the n = 10
                workload, at n = 30 (general fused engines)
  capacity_n34  Grover and the layered circuit at n = 34 complex128
                (256 GiB, in place: no room for a second buffer)
  dax_sweep     materialised DAX / DAS MTP and MVM of m identical gates
  rh_methods    the paper's four RH sign methods for H^(x)n, n = 12..16
  qnn           serving 4096 requests (continuous batching vs one circuit
                at a time through the per-gate path), adjoint training
                gradients of 1024 circuits in complex64 and complex128
and the FP64 oracle on the host cores (one thread; all cores as
independent replicas).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fused|per_gate]
                  [--workload layered|grover] [--sections a,b,...|none]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

With N > 1 (torchrun) every rank runs an independent replica of the
headline workload on its own GPU (the path does not shard); value = all
ranks' updates / the slowest rank's time.  Sections run at N = 1 only.
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
ALL_SECTIONS = ("grover", "per_gate", "random", "capacity", "dax", "rh", "qnn")


def _args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mera", choices=["mera", "reference"])
    p.add_argument("--mode", default="fused", choices=["fused", "per_gate"])
    p.add_argument("--workload", default="layered", choices=["layered", "grover", "random"])
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--layers", type=int, default=20)
    p.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    p.add_argument("--sections", default="all",
                   help="comma list of " + ",".join(ALL_SECTIONS) + ", 'all' or 'none'")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--qnn-requests", type=int, default=4096)
    return p.parse_args(argv)


def _sections(args):
    if args.sections in ("", "none"):
        return ()
    if args.sections == "all":
        return ALL_SECTIONS
    out = tuple(s.strip() for s in args.sections.split(",") if s.strip())
    for s in out:
        if s not in ALL_SECTIONS:
            raise SystemExit(f"unknown section {s!r}")
    return out


RANDOM_GATES_N30 = 200


def _workload(name, n, layers=20):
    from paper_2411_15332_gb300 import inputs
    if name == "grover":
        ops, _m = inputs.grover_circuit(n, 8, seed=3)
        return ops
    if name == "random":
        return inputs.random_circuit(n, RANDOM_GATES_N30, seed=1)
    return inputs.layered_circuit(n, layers, seed=2)


def _workload_name(name, n, dtype="c128", layers=20):
    dt = "complex128" if dtype == "c128" else "complex64"
    if name == "grover":
        return (f"grover_n{n}: n={n} {dt}, |0..0>, H on all, then 8 x [sign flip of a seeded index, H on all, "
                f"sign flip of |0..0>, H on all], readout norm^2 and <Z_0>")
    if name == "random":
        return (f"random_n{n}: n={n} {dt}, |0..0>, {RANDOM_GATES_N30} gates drawn uniformly from "
                f"{{X,Y,Z,S,T,CNOT,CZ,SWAP,Toffoli,RZ,H,RX,RY}} on random distinct qubits (seed 1), "
                f"readout norm^2 and <Z_0>")
    return (f"layered_n{n}: n={n} {dt}, |0..0>, H on all, "
            f"then {layers} x [CNOT ladder q->q+1, CZ on a seeded perfect matching, T/S on a seeded half, "
            f"RZ(theta~U[0,2pi)) on all], readout norm^2 and <Z_0>")


# ----------------------------------------------------------- clocks --------
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""

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


def _kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_15332_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kclass, workload, n):
    """DRAM bytes per launch of kernel class ``kclass`` from the committed ncu
    summary, if it was captured on the current kernel sources and on this
    workload (scaled from the captured size by 2^(n - n_captured): every
    pass reads and writes the whole state once)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") != _kernel_source_hash():
            return None
        e = d["kernels"][workload][kclass]
        return e["dram_bytes_per_launch"] * 2.0 ** (n - e["n"])
    except Exception:
        return None


def _kernel_table(prof, window_ms, peak, classes=None):
    """Per kernel class in ``prof``: launches, device ms, share of the timed
    window, algorithmic GB/s and its fraction of the peak."""
    out = {}
    for name, (nl, ms, by) in prof.items():
        if classes is not None and name not in classes:
            continue
        if nl == 0:
            continue
        gbs = (by / (ms / 1e3) / 1e9) if ms > 0 else None
        out[name] = {"launches": nl, "ms": ms, "share": (ms / window_ms) if window_ms else None,
                     "algorithmic_bytes_per_launch": by / nl, "achieved_gbs": gbs,
                     "frac": (gbs / peak) if gbs else None}
    return out


def _dominant(table):
    return max(table, key=lambda k: table[k]["ms"]) if table else None


KERNEL_NAMES = {"amp": "k_amp (monomial run pass: affine permutation gather, diagonal tables)",
                "dpass": "k_dpass (streaming single-phase table pass)",
                "hpass": "k_hpass (Hadamard pass: butterflies, sign terms)",
                "tile": "k_tile (general tile pass)",
                "gate_diag": "k_diag / k_phase (per-gate diagonal)",
                "gate_1q": "k_dense1_* (per-gate one-target)",
                "gate": "k_mono / k_dense_k (per-gate two- and three-target)",
                "reduce": "reductions", "dax": "DAX / DAS kernels", "qnn": "QNN kernels",
                "rh": "RH sign-method MVM kernels"}


def _roofline(table, peak, peak_kind, workload, n):
    dom = _dominant(table)
    if dom is None:
        return None
    e = table[dom]
    tr = _ncu_traffic(dom, workload, n)
    return {"bound": "hbm", "achieved": e["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": e["frac"],
            "traffic": tr, "kernel": KERNEL_NAMES.get(dom, dom), "kclass": dom,
            "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "kernel_launches": e["launches"], "kernel_ms": e["ms"], "kernel_share": e["share"],
            "algorithmic_bytes_per_launch": e["algorithmic_bytes_per_launch"]}


def _chunks(N, chunk=1 << 27):
    for c0 in range(0, N, chunk):
        yield c0, min(N, c0 + chunk)


def _magnitude_dev(t, target):
    """max_i | |amp_i| - target | of a device state tensor, in chunks."""
    import torch
    worst = 0.0
    for c0, c1 in _chunks(t.shape[0]):
        v = t[c0:c1]
        worst = max(worst, float(torch.max(torch.abs(torch.hypot(v[:, 0], v[:, 1]) - target)).item()))
    return worst


def _grover_closed_form(n, k):
    """Amplitudes after H on all and k iterations of [flip m; H all; flip 0;
    H all]: each iteration is minus the textbook Grover iterate, so the
    marked amplitude is (-1)^k sin((2k+1) theta) and every other one
    (-1)^k cos((2k+1) theta) / sqrt(N - 1), sin(theta) = N^(-1/2)."""
    N = float(1 << n)
    th = math.asin(1.0 / math.sqrt(N))
    sg = -1.0 if k % 2 else 1.0
    return sg * math.sin((2 * k + 1) * th), sg * math.cos((2 * k + 1) * th) / math.sqrt(N - 1.0)


def _grover_error(t, n, m, iters=8):
    """Max absolute and relative error over all 2^n amplitudes of a Grover
    state tensor against the closed form (device reductions in chunks)."""
    import torch
    a_m, a_o = _grover_closed_form(n, iters)
    worst = 0.0
    for c0, c1 in _chunks(1 << n):
        v = t[c0:c1]
        err = torch.hypot(v[:, 0] - a_o, v[:, 1])
        if c0 <= m < c1:
            err[m - c0] = 0.0
        worst = max(worst, float(torch.max(err).item()))
    vm = t[m].cpu().tolist()
    em = abs(complex(vm[0], vm[1]) - a_m)
    return {"max_abs": max(worst, em), "max_rel": max(worst / abs(a_o), em / abs(a_m)),
            "amplitudes_checked": 1 << n, "against": "closed form"}


# ----------------------------------------------------------- CPU oracle ----
_CPU_CODE = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
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
while g < len(ops) and time.perf_counter() - t0 < %(secs)f:
    sv.apply_op(psi, n, ops[g]); done += upd(ops[g]); g += 1
dt = time.perf_counter() - t0
print(json.dumps({"value": done / dt, "gates": g, "seconds": dt, "n": n}))
"""


def _oracle_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def _cpu_baseline(sample_seconds=15.0, procs=1):
    """The FP64 oracle (numpy, one thread per process) on a bounded sample of
    the headline circuit family at reduced n, in ``procs`` independent
    processes at once (replicas: the host's cores each run the oracle as it
    stands); value = the processes' summed amplitude updates per second."""
    code = _CPU_CODE % {"root": ROOT, "secs": sample_seconds}
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=_oracle_env()) for _ in range(procs)]
    vals, last, err = [], None, ""
    for p in ps:
        out, e = p.communicate(timeout=900)
        if p.returncode == 0:
            last = json.loads(out.strip().splitlines()[-1])
            vals.append(last["value"])
        else:
            err = e[-300:]
    if not vals:
        return {"value": None, "unit": METRIC, "cores": procs, "kind": "oracle", "sample": "failed: " + err}
    what = "1 thread" if procs == 1 else f"{len(vals)} single-thread processes at once, rates summed"
    return {"value": float(sum(vals)), "unit": METRIC, "cores": len(vals), "kind": "oracle",
            "sample": (f"oracle (numpy FP64, {what}) applying the first {last['gates']} gates of the layered "
                       f"circuit family at n={last['n']} for {last['seconds']:.1f} s")}


_QNN_ORACLE_CODE = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from paper_2411_15332_gb300 import inputs
from oracle import statevector as sv
reqs = inputs.qnn_requests(%(count)d, seed=4)[:%(k)d]
t0 = time.perf_counter(); z = []
for r in reqs:
    psi = sv.simulate(r["n"], inputs.ansatz_ops(r["n"], r["theta"]))
    z.append(sv.expect_z(psi, r["n"], 0))
dt = time.perf_counter() - t0
print(json.dumps({"circuits_per_s": len(reqs) / dt, "seconds": dt, "z0": z}))
"""


def _qnn_oracle(count, k):
    """The oracle on the first k serving requests (one thread): its
    circuits/s and <Z_0> of each (the served results' accuracy figure)."""
    code = _QNN_ORACLE_CODE % {"root": ROOT, "count": count, "k": k}
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=_oracle_env(),
                       timeout=900)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------- timing --------
def _time_steps(step, steps, warmup, stream):
    """W untimed steps, then K steps between CUDA events on ``stream``;
    returns (ms per step, per-kernel profile of the timed steps, launches)."""
    import torch
    import paper_2411_15332_gb300 as mera
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    mera.profile_enable(True)
    l0 = mera.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(steps):
        out = step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = mera.launch_count() - l0
    prof = mera.profile_read()
    mera.profile_enable(False)
    return e0.elapsed_time(e1) / steps, prof, launches, out


def _free_cuda():
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


# ----------------------------------------------------------- sections ------
def _section_statevector(name, n, mode, steps, warmup, peak, peak_kind, check):
    import torch
    import paper_2411_15332_gb300 as mera
    from paper_2411_15332_gb300.workload import amplitude_updates
    ops = _workload(name, n)
    upd = amplitude_updates(ops, n)
    st = mera.State(n, "c128")
    stream = torch.cuda.current_stream()

    def step():
        st.set_basis(0)
        return st.apply_circuit_observe(ops, 0, mode=mode)

    ms, prof, launches, obs = _time_steps(step, steps, warmup, stream)
    table = _kernel_table(prof, ms * steps, peak)
    sec = {"workload": _workload_name(name, n), "mode": mode, "steps": steps, "warmup": warmup,
           "ms_per_step": ms, "amplitude_updates_per_step": upd, "value": upd / (ms / 1e3), "unit": METRIC,
           "gpu_launches": int(launches), "roofline": _roofline(table, peak, peak_kind, name, n),
           "kernels": table, "readout": {"norm2": obs[0], "z0": obs[1]}}
    try:
        st.close()
        sec["error"] = check(st.tensor, ops)
    except Exception as ex:
        sec["error"] = {"failed": str(ex)[:200]}
    st.tensor = None
    del st
    _free_cuda()
    return sec


def _section_grover(peak, peak_kind):
    from paper_2411_15332_gb300 import inputs
    n = 33
    m = inputs.grover_marked(n, seed=3)
    return _section_statevector("grover", n, "fused", 3, 3, peak, peak_kind,
                                lambda t, ops: _grover_error(t, n, m))


def _layered_check(n):
    def check(t, ops):
        # after the H layer every gate is a phase times a permutation: every
        # amplitude keeps magnitude 2^(-n/2)
        return {"max_abs_dev_of_magnitude": _magnitude_dev(t, 2.0 ** (-n / 2)), "amplitudes_checked": 1 << n,
                "against": "closed form |amp| = 2^(-n/2)"}
    return check


def _section_per_gate(peak, peak_kind):
    # one 8 s step of continuous per-gate launches warms the device up
    return _section_statevector("layered", 30, "per_gate", 2, 1, peak, peak_kind, _layered_check(30))


def _section_random(peak, peak_kind):
    def check(t, ops):
        import torch
        nrm = 0.0
        for c0, c1 in _chunks(t.shape[0]):
            nrm += float(torch.sum(t[c0:c1].double() ** 2).item())
        return {"norm2_minus_1": nrm - 1.0, "against": "unitarity (norm preserved)"}
    return _section_statevector("random", 30, "fused", 3, 3, peak, peak_kind, check)


def _section_capacity(peak, peak_kind):
    """n = 34 complex128 (2^34 amplitudes, 256 GiB): the largest state the
    GPU holds; every pass runs in place."""
    import torch
    from paper_2411_15332_gb300 import inputs
    n = 34
    free, total = torch.cuda.mem_get_info()
    if free < (16 << n) + (4 << 30):
        return {"skipped": f"{free >> 30} GiB free, {(16 << n) >> 30} GiB needed"}
    m = inputs.grover_marked(n, seed=3)
    out = {"grover_n34": _section_statevector("grover", n, "fused", 1, 1, peak, peak_kind,
                                              lambda t, ops: _grover_error(t, n, m)),
           "layered_n34": _section_statevector("layered", n, "fused", 1, 1, peak, peak_kind, _layered_check(n))}
    return out


def _section_dax(peak):
    """m identical gates filling n qubits (the paper's MTP / MVM sweeps):
    the layer operator built by m - 1 device Kronecker products (MTP), then
    one materialised MVM out of place."""
    import numpy as np
    import torch
    import paper_2411_15332_gb300 as mera
    from paper_2411_15332_gb300.core import gate_matrix
    from paper_2411_15332_gb300 import inputs
    gates = {"X": gate_matrix("X"), "Y": gate_matrix("Y"), "H": gate_matrix("H"), "SWAP": gate_matrix("SWAP"),
             "CNOT": None, "TOFFOLI": None}
    cx = np.eye(4, dtype=complex)[[0, 1, 3, 2]]       # |c t>: control the high bit
    ccx = np.eye(8, dtype=complex)[[0, 1, 2, 3, 4, 5, 7, 6]]
    gates["CNOT"], gates["TOFFOLI"] = cx, ccx
    sizes = {"X": (6, 12, 18, 24, 30), "Y": (6, 12, 18, 24, 30), "SWAP": (6, 12, 18, 24, 30),
             "CNOT": (6, 12, 18, 24, 30), "TOFFOLI": (6, 12, 18, 24, 30), "H": (6, 12, 14)}
    rows = []
    stream = torch.cuda.current_stream()
    for g, G in gates.items():
        k = int(round(math.log2(G.shape[0])))
        for n in sizes[g]:
            for cls in (mera.DAX, mera.DAS):
                m = n // k
                base = cls.from_dense(G)
                torch.cuda.synchronize()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                acc, mid = base, []
                for _ in range(m - 1):
                    nxt = acc.kron(base)
                    if acc is not base:
                        mid.append(acc)
                    acc = nxt
                e1.record(stream)
                torch.cuda.synchronize()
                for x in mid:
                    x.close()
                nnz = acc.nnz
                src = mera.State(n, "c128")
                src.from_numpy(inputs.random_state(n, seed=n)) if n <= 24 else src.hadamard_layer((1 << n) - 1)
                dst = mera.State(n, "c128")
                acc.mvm(src, dst)               # warm
                torch.cuda.synchronize()
                e1b = torch.cuda.Event(enable_timing=True)
                e1b.record(stream)
                acc.mvm(src, dst)
                e2.record(stream)
                torch.cuda.synchronize()
                mtp_ms = e0.elapsed_time(e1)
                mvm_ms = e1b.elapsed_time(e2)
                mvm_bytes = 24.0 * nnz + (2 * 16 + 8) * (1 << n)
                rows.append({"gate": g, "kind": cls._kind, "n": n, "m": m, "nnz": nnz,
                             "bytes": 24 * nnz, "mtp_ms": mtp_ms,
                             "mtp_write_gbs": 24.0 * nnz / (mtp_ms / 1e3) / 1e9 if mtp_ms > 0 else None,
                             "mvm_ms": mvm_ms, "mvm_gbs": mvm_bytes / (mvm_ms / 1e3) / 1e9 if mvm_ms > 0 else None,
                             "mvm_frac": (mvm_bytes / (mvm_ms / 1e3) / 1e9 / peak) if mvm_ms > 0 else None})
                for x in (src, dst):
                    x.close()
                    x.tensor = None
                acc.close()
                base.close()
                _free_cuda()
    return {"rows": rows,
            "note": "MTP time covers the m - 1 device Kronecker products that build the layer (24 B written per "
                    "entry of each product); MVM bytes = 24 B per entry + 16 B gathered + 16 B written + 8 B row "
                    "pointer per row"}


def _section_rh(peak):
    import torch
    import paper_2411_15332_gb300 as mera
    from paper_2411_15332_gb300 import inputs
    rows = []
    stream = torch.cuda.current_stream()
    for n in (12, 14, 16):
        src = mera.State(n, "c128")
        src.from_numpy(inputs.random_state(n, seed=n))
        dst = mera.State(n, "c128")
        for method in mera.RH_METHODS:
            mera.rh_mvm(src, dst, method)          # warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            signs = mera.rh_mvm(src, dst, method)
            e1.record(stream)
            torch.cuda.synchronize()
            rows.append({"n": n, "method": method, "ms": e0.elapsed_time(e1), "sign_computations": signs})
        src.close()
        dst.close()
    _free_cuda()
    return {"rows": rows, "note": "H^(x)n MVM (Alg. 1 and the three other sign methods of Sec. III-B), "
                                  "one thread per output row, complex128"}


def _section_qnn(args):
    """Serving: all requests of the seeded workload (n ~ U{8..20}, L ~
    U{4..12}, complex64 states, FP64 <Z_0>), served with continuous batching
    (all at once, then Poisson arrivals at 0.8x the saturation throughput)
    and one circuit at a time through the per-gate path on states allocated
    before timing.  Training: adjoint gradients of 1024 circuits (n = 16, 10
    layers, 320 angles) in complex64 and complex128."""
    import numpy as np
    import torch
    import paper_2411_15332_gb300 as mera
    from paper_2411_15332_gb300 import inputs
    from paper_2411_15332_gb300.serve import Server, requests_from_workload
    out = {}
    reqs = inputs.qnn_requests(4096, seed=4)[: args.qnn_requests]
    # plain: one circuit at a time, per-gate kernels, one preallocated state per n
    states = {n: mera.State(n, "c64") for n in sorted({r["n"] for r in reqs})}
    opsl = [inputs.ansatz_ops(r["n"], r["theta"]) for r in reqs]
    for r, ops in list(zip(reqs, opsl))[:16]:             # warm
        st = states[r["n"]]
        st.set_basis(0)
        st.apply_circuit(ops, mode="per_gate")
        st.observables(0)
    torch.cuda.synchronize()
    lat, plain_z = [], []
    t0 = time.perf_counter()
    for r, ops in zip(reqs, opsl):
        t1 = time.perf_counter()
        st = states[r["n"]]
        st.set_basis(0)
        st.apply_circuit(ops, mode="per_gate")
        plain_z.append(st.observables(0)[1])
        lat.append(time.perf_counter() - t1)
    plain_s = time.perf_counter() - t0
    for st in states.values():
        st.close()
        st.tensor = None
    states = None
    _free_cuda()
    out["plain"] = {"circuits": len(reqs), "seconds": plain_s, "circuits_per_s": len(reqs) / plain_s,
                    "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                    "path": "per-gate kernels, one circuit at a time, states allocated before timing"}
    # serving
    warm = Server(dtype="c64", mem_budget=64 << 30, slots_per_n=512)
    warm.run(requests_from_workload(reqs[:64]))
    srv = Server(dtype="c64", mem_budget=64 << 30, slots_per_n=512)
    done = srv.run(requests_from_workload(reqs))
    sat = srv.stats()
    served = {r.rid: r.result for r in done}
    rate = 0.8 * sat["circuits_per_s"]
    srv2 = Server(dtype="c64", mem_budget=64 << 30, slots_per_n=512)
    arr = requests_from_workload(reqs, rate=rate)
    done2 = srv2.run(arr)
    poi = srv2.stats()
    served2 = {r.rid: r.result for r in done2}
    diff_plain = max(abs(served[r["id"]] - z) for r, z in zip(reqs, plain_z))
    out["serving"] = {"requests": len(reqs), "saturation": sat,
                      "poisson": dict(poi, offered_rate_per_s=rate, arrival_window_s=max(a.arrival for a in arr)),
                      "max_abs_diff_served_vs_plain_z0": diff_plain,
                      "poisson_equals_saturation_results": all(served2[k] == served[k] for k in served)}
    out["speedup_vs_plain"] = sat["circuits_per_s"] / out["plain"]["circuits_per_s"]
    out["_served_z0"] = [served[r["id"]] for r in reqs[:64]]
    out["_plain_z0"] = plain_z[:64]
    # training
    for dt in ("c64", "c128"):
        theta = inputs.qnn_batch(1024, 16, 10, seed=5)
        b = mera.Batch(16, 1024, dt)
        b.adjoint_grad(theta[:8])
        b.adjoint_grad(theta[:8])
        b.adjoint_grad(theta[:8])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.adjoint_grad(theta)
        tr = time.perf_counter() - t0
        out[f"training_{dt}"] = {"circuits": 1024, "params_per_circuit": 320, "seconds": tr,
                                 "circuit_gradients_per_s": 1024 / tr}
        b.close()
        _free_cuda()
    return out


# ----------------------------------------------------------- arms ----------
def run_reference(args, rank, world):
    """The FP64 oracle on the host cores (all cores, one process each), each
    step a bounded sample of the headline circuit family at reduced n."""
    if rank != 0:
        return
    procs = max(1, os.cpu_count() or 1)
    per = max(2.0, min(20.0, 90.0 / max(1, args.steps + args.warmup)))
    vals = []
    last = None
    for _ in range(args.warmup):
        _cpu_baseline(sample_seconds=min(per, 2.0), procs=procs)
    for _ in range(args.steps):
        last = _cpu_baseline(sample_seconds=per, procs=procs)
        if last["value"] is not None:
            vals.append(last["value"])
    value = statistics.median(vals) if vals else None
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(args.workload, args.n), "n": args.n,
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
        return ("complex128 state held as int64 fixed point across the circuit's tile passes "
                "(global scale from a norm bound; exact butterflies and moves; 31-bit-limb integer "
                "products for phases, rounding to nearest); float64 at the circuit's ends and in reductions")
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
    ops = _workload(args.workload, n, args.layers)
    upd = amplitude_updates(ops, n)
    st = mera.State(n, args.dtype)
    stream = torch.cuda.current_stream()

    def step():
        st.set_basis(0)
        # the circuit and its readout (norm^2, <Z_0>) in one call: the last
        # pass sums the readout while it writes the state where it can
        return st.apply_circuit_observe(ops, 0, mode=args.mode)

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
    own_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(own_ms, device="cuda")
    ms_per_step = total_ms / args.steps
    value = job_throughput(upd, world, ms_per_step)

    peak, peak_kind = _peaks()
    table = _kernel_table(prof, own_ms, peak)
    roofline = _roofline(table, peak, peak_kind, args.workload, n)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        try:
            eb = 16 if args.dtype == "c128" else 8
            host = torch.zeros((1 << n) * 2, dtype=torch.float64 if eb == 16 else torch.float32).pin_memory()
            host[0] = 1.0
            hp = host.numpy().view(np.complex128 if eb == 16 else np.complex64)
            st.from_numpy(hp)
            st.apply_circuit_observe(ops, 0, mode=args.mode)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                st.from_numpy(hp)                                # H2D of the input state
                st.apply_circuit_observe(ops, 0, mode=args.mode)  # ops table copied; D2H of the result
            seq_s = (time.perf_counter() - t0) / args.steps
            ops_bytes = 80 * len(ops)
            # pipelined: two states on two streams, the next step's input
            # upload (asynchronous, pinned) overlapping this step's circuit;
            # every step still uploads its input and reads its result
            e2e_s = None
            sts = [st]
            try:
                sts.append(mera.State(n, args.dtype, stream=torch.cuda.Stream()))
                st.set_stream(torch.cuda.Stream())
                for s2 in sts:   # warm both plans
                    s2.from_host_async(hp)
                    s2.apply_circuit_observe(ops, 0, mode=args.mode)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sts[0].from_host_async(hp)
                for k in range(args.steps):
                    cur, nxt = sts[k % 2], sts[(k + 1) % 2]
                    # enqueue the next step's upload first: the readout's
                    # synchronisation then waits only for this state's stream
                    if k + 1 < args.steps:
                        nxt.from_host_async(hp)
                    cur.apply_circuit_observe(ops, 0, mode=args.mode)
                e2e_s = (time.perf_counter() - t0) / args.steps
            except Exception:   # no room for a second state: sequential only
                e2e_s = None
            finally:
                if len(sts) > 1:   # release the second state and its memory
                    sts[1].close()
                    sts[1].tensor = None
                del sts
                _free_cuda()
            e2e = {"value": upd * world / (e2e_s or seq_s), "unit": METRIC,
                   "h2d_bytes_per_step": (1 << n) * eb + ops_bytes, "d2h_bytes_per_step": 24,
                   "seconds_per_step": e2e_s or seq_s,
                   "pipelined": e2e_s is not None,
                   "sequential": {"value": upd * world / seq_s, "seconds_per_step": seq_s}}
            del host
        except Exception as ex:  # pinned allocation can fail on small hosts
            e2e = {"value": None, "unit": METRIC, "error": str(ex)[:200]}

    # error of the headline result (closed-form properties of the circuit)
    err = None
    if args.workload == "layered" and args.dtype == "c128":
        st.set_basis(0)
        st.apply_circuit(ops, mode=args.mode)
        err = _layered_check(n)(st.tensor, ops)
    elif args.workload == "grover" and args.dtype == "c128":
        from paper_2411_15332_gb300 import inputs
        st.set_basis(0)
        st.apply_circuit(ops, mode=args.mode)
        st.close()
        err = _grover_error(st.tensor, n, inputs.grover_marked(n, seed=3))
    st.close()
    st.tensor = None
    del st
    _free_cuda()

    sections = {}
    headline_default = args.workload == "layered" and args.mode == "fused" and args.dtype == "c128" and n == 30
    if rank == 0 and world == 1:
        todo = _sections(args)
        if not headline_default:
            todo = tuple(s for s in todo if s in ("dax", "rh"))
        fns = {"grover": lambda: _section_grover(peak, peak_kind),
               "per_gate": lambda: _section_per_gate(peak, peak_kind),
               "random": lambda: _section_random(peak, peak_kind),
               "capacity": lambda: _section_capacity(peak, peak_kind),
               "dax": lambda: _section_dax(peak),
               "rh": lambda: _section_rh(peak),
               "qnn": lambda: _section_qnn(args)}
        keys = {"grover": "grover_n33", "per_gate": "per_gate_n30", "random": "random_n30",
                "capacity": "capacity_n34", "dax": "dax_sweep",
                "rh": "rh_methods", "qnn": "qnn"}
        for s in todo:
            try:
                sections[keys[s]] = fns[s]()
            except Exception as ex:
                sections[keys[s]] = {"error": str(ex)[:300]}
                _free_cuda()

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = _cpu_baseline()
        cpu_all = _cpu_baseline(procs=max(1, os.cpu_count() or 1))
        q = sections.get("qnn")
        if isinstance(q, dict) and "_served_z0" in q:
            o = _qnn_oracle(args.qnn_requests, len(q["_served_z0"]))
            if o is not None:
                q["accuracy_vs_oracle"] = {
                    "requests": len(o["z0"]),
                    "max_abs_err_served_z0": max(abs(a - b) for a, b in zip(q["_served_z0"], o["z0"])),
                    "max_abs_err_plain_z0": max(abs(a - b) for a, b in zip(q["_plain_z0"], o["z0"]))}
                q["oracle_circuits_per_s_1_thread"] = o["circuits_per_s"]
    for q in (sections.get("qnn"),):
        if isinstance(q, dict):
            q.pop("_served_z0", None)
            q.pop("_plain_z0", None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": _arith_dtype(args),
                "data": "synthetic",
                "config": {"workload": _workload_name(args.workload, n, args.dtype, args.layers), "n": n,
                           "state": "complex128" if args.dtype == "c128" else "complex64",
                           "arithmetic": _arith_note(args),
                           "amplitude_updates_per_step": upd, "mode": args.mode,
                           "parallelism": f"replicas x{world}",
                           "l2": "state (%d GiB) larger than L2 (129 MB); no flush needed" % (
                               ((1 << n) * (16 if args.dtype == 'c128' else 8)) >> 30),
                           "readout": {"norm2": obs[0], "z0": obs[1]}},
                "roofline": roofline, "kernels": table, "error": err, "cpu_baseline": cpu,
                "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks}
        line.update(sections)
        print(json.dumps(line), flush=True)


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
