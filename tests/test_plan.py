"""Host-side planning of the fused tile passes (no GPU): which engine each
pass runs, that CNOT/X/SWAP runs become exchange index maps instead of
register ops, the per-pass Hadamard cap, and when the complex128 state is
kept as fixed point across passes.  CPU only."""
import re

import numpy as np
import pytest

from paper_2411_15332_gb300 import inputs
from paper_2411_15332_gb300.inputs import op


@pytest.fixture(scope="module")
def core():
    from paper_2411_15332_gb300.build import build
    build()
    from paper_2411_15332_gb300 import core as c
    return c


def parse(summary):
    head = summary.splitlines()[0]
    info = dict(re.findall(r"(\w+)=(\d+)", head))
    passes = []
    for line in summary.splitlines()[1:]:
        if "per-gate" in line:
            passes.append({"single": True})
            continue
        d = dict(re.findall(r"(\w+)=([\w\d]+)", line.split("tile=")[0]))
        d.update(re.findall(r"\b(qend|qexit|qgi)=(\d+)", line))
        d["phase_ops"] = re.search(r"phase_ops=\[([^\]]*)\]", line).group(1)
        passes.append(d)
    return {k: int(v) for k, v in info.items()}, passes


def test_layered_n30_plan(core):
    """Three Hadamard passes, then one pass per layer: each layer (CNOT
    ladder, CZ matching, T/S, RZ on all) is one monomial operator applied
    by a single streaming pass."""
    summary = core.plan_summary(30, inputs.layered_circuit(30, 20, seed=2))
    head, passes = parse(summary)
    lines = summary.splitlines()[1:]
    assert head["resident"] == 1 and head["passes"] == 23
    assert all(p["eng"] == "q" for p in passes)
    assert all("pipelined" in l for l in lines[:3])
    amp = [l for l in lines if " amp " in l]
    assert len(amp) == 20 and all("ops=89 " in l and "mono=29 " in l and "diag=60 " in l for l in amp)
    # the resident run converts from doubles once and back once
    assert passes[0]["q_in"] == "0" and passes[-1]["q_out"] == "0"
    assert all(p["q_in"] == "1" for p in passes[1:]) and all(p["q_out"] == "1" for p in passes[:-1])


def test_layered_n30_plan_without_monomial_runs(core):
    """The tile planner alone (MERA_AMP=0 is read per plan): three passes per
    layer, the CNOT ladders riding on exchanges."""
    import subprocess
    import sys
    code = ("from paper_2411_15332_gb300 import core, inputs\n"
            "print(core.plan_summary(30, inputs.layered_circuit(30, 20, seed=2)))\n")
    out = subprocess.run([sys.executable, "-c", code], env={**__import__("os").environ, "MERA_AMP": "0"},
                         capture_output=True, text=True, check=True, timeout=300).stdout.strip()
    head, passes = parse(out)
    assert head["resident"] == 1 and head["passes"] == 60
    assert " amp " not in out
    assert all(p["mono"] == "0" for p in passes)
    assert all(int(p["dsep"]) <= 2 for p in passes)


def test_hadamard_levels_per_pass_are_capped(core):
    ops, _ = inputs.grover_circuit(12, 8, seed=3)
    head, passes = parse(core.plan_summary(12, ops))
    assert all(int(p["nh"]) <= 16 for p in passes)
    assert sum(int(p["nh"]) for p in passes) == 12 * 17


def test_non_unitary_gate_disables_resident_format(core):
    n = 12
    m = np.diag([2.0, 0.5]).astype(np.complex128)
    ops = inputs.hadamard_all(n) + [(m, (3,), (), (), 0)]   # an explicit (non-unitary) matrix
    head, passes = parse(core.plan_summary(n, ops))
    assert head["resident"] == 0
    assert all(p.get("eng") != "q" for p in passes if not p.get("single"))


def test_exact_only_circuit_stays_in_float64(core):
    """Permutations and unit phases only: exact moves in float64, no
    fixed-point round trip."""
    n = 20
    ops = [op("X", (q + 1,), (q,)) for q in range(n - 1)] + [op("S", (q,)) for q in range(n)]
    head, passes = parse(core.plan_summary(n, ops))
    assert head["resident"] == 0
    assert all(p["eng"] == "fp" for p in passes)


def test_complex64_plans_use_the_float_engine(core):
    head, passes = parse(core.plan_summary(24, inputs.layered_circuit(24, 3, seed=2), dtype="c64"))
    assert head["resident"] == 0
    assert all(p["eng"] == "fp" for p in passes)


def test_mixing_gates_after_the_body_keep_doubles(core):
    """Grover: Hadamard layers after phase flips.  With one global scale a
    small amplitude keeps fewer bits and a later Hadamard layer adds up the
    errors of many amplitudes, so the state keeps float64 storage; every
    tile pass runs the Hadamard-pass kernel in its per-tile int64 engine
    (exponent from the tile maximum), loads staged through shared memory."""
    ops, _ = inputs.grover_circuit(24, 4, seed=3)
    summary = core.plan_summary(24, ops)
    head, passes = parse(summary)
    assert head["resident"] == 0
    assert all(p["eng"] == "i64" for p in passes)
    lines = summary.splitlines()[1:]
    assert all("pipelined" in l for l in lines)
    assert all(p["load_smem"] == "1" for p in passes)


def test_hadamard_runs_keep_per_amplitude_exponents(core):
    """Consecutive int64 Hadamard passes of a unitary circuit pass the state
    on in the per-amplitude exponent format: only the run's first pass reads
    doubles and only its last writes doubles."""
    ops, _ = inputs.grover_circuit(24, 4, seed=3)
    head, passes = parse(core.plan_summary(24, ops))
    assert head["efmt"] == 1
    assert passes[0]["q_in"] == "0" and passes[-1]["q_out"] == "0"
    assert all(p["q_in"] == "1" for p in passes[1:]) and all(p["q_out"] == "1" for p in passes[:-1])


def test_non_unitary_circuit_keeps_doubles_between_hadamard_passes(core):
    n = 14
    m = np.diag([2.0, 0.5]).astype(np.complex128)
    ops = inputs.hadamard_all(n) + [inputs.flip_index(n, 5)] + inputs.hadamard_all(n) + [(m, (3,), (), (), 0)]
    head, passes = parse(core.plan_summary(n, ops))
    assert head["efmt"] == 0 and head["resident"] == 0
    assert all(p.get("q_in", "0") == "0" and p.get("q_out", "0") == "0" for p in passes if not p.get("single"))


def test_mixing_gates_after_the_body_without_the_kernel_keep_doubles(core):
    """A table pass (RZ on every qubit) between Hadamard layers does not run
    the Hadamard-pass kernel, so that circuit keeps double storage (per-tile
    int64 for the butterflies)."""
    n = 20
    rng = np.random.default_rng(5)
    ops = inputs.hadamard_all(n)
    ops += [op("Z", (q,)) for q in range(0, n, 3)]
    ops += [op("RZ", (q,), (), (float(t),)) for q, t in enumerate(rng.uniform(0, 6.28, n))]
    ops += inputs.hadamard_all(n)
    head, passes = parse(core.plan_summary(n, ops))
    assert head["resident"] == 0
    assert all(p["eng"] in ("i64", "fp") for p in passes if not p.get("single"))

def test_hadamard_passes_around_a_per_gate_op(core):
    """A three-target gate between Hadamard layers and sign flips: per-tile
    int64 Hadamard-pass kernels on both sides of the per-gate op."""
    n = 17
    m = inputs.grover_marked(n, seed=7)
    perm8 = np.roll(np.eye(8, dtype=np.complex128), 1, axis=0)
    ops = (inputs.hadamard_all(n) + [inputs.flip_index(n, m)] + [op("H", (q,)) for q in range(0, n, 2)]
           + [(perm8, (n - 1, 3, 6), (), (), 0)] + [inputs.flip_index(n, 0)] + inputs.hadamard_all(n))
    summary = core.plan_summary(n, ops)
    head, passes = parse(summary)
    assert head["resident"] == 0
    assert sum(1 for p in passes if p.get("single")) == 1
    tile = [l for l in summary.splitlines()[1:] if "per-gate" not in l]
    assert tile and all("pipelined" in l and "eng=i64" in l for l in tile)


def _phase_levels(p):
    return [int(x.rstrip("p")) for x in p["phase_ops"].split(",")]


@pytest.mark.parametrize("n,iters", [(33, 8), (20, 3), (13, 2)])
def test_int64_hadamard_passes_scale_at_phase_exits(core, n, iters):
    """Per-tile int64 Hadamard passes take part of the 2^(-nh/2) scale at
    every phase exit (a shift by half the pending levels): every level of
    the circuit is scaled once, and the headroom over the tile
    maximum is the smaller of the max-norm and 2-norm growth bounds between
    two exits, plus one bit -- at most 9 bits for a K = 12 tile, where a
    whole 12-level pass unscaled would need 13."""
    ops, _ = inputs.grover_circuit(n, iters, seed=3)
    head, passes = parse(core.plan_summary(n, ops))
    K = head["K"]
    assert head["resident"] == 0
    carry = 0
    for k, p in enumerate(passes):
        nh, qexit, qend = int(p["nh"]), int(p["qexit"]), int(p["qend"])
        # an odd level count leaves one level (sqrt(2) on the stored state)
        # to the next pass; only the last pass may scale an odd count
        cout = nh + carry - qexit - qend
        assert cout in (0, 1) and (k + 1 < len(passes) or cout == 0)
        assert qend % 2 == 0 or k + 1 == len(passes)
        carry = cout
        levels = _phase_levels(p)       # sign-term ops are in the counts too, butterflies dominate
        if len(levels) > 1 and nh >= 4:
            assert qexit > 0
        assert int(p["guard"]) <= min(nh, (nh + K + 1) // 2) + 1
        if K == 12 and nh >= 9:
            assert int(p["guard"]) <= 9
    assert sum(int(p["qexit"]) + int(p["qend"]) for p in passes) == n * (2 * iters + 1)


def test_resident_scaling_uses_exits(core):
    """The layered circuit (resident) scales at phase exits once 8 levels are
    pending and the rest at its end; every level once."""
    head, passes = parse(core.plan_summary(30, inputs.layered_circuit(30, 20, seed=2)))
    assert head["resident"] == 1
    assert sum(int(p["qend"]) + int(p["qexit"]) for p in passes) == sum(int(p["nh"]) for p in passes) == 30
    assert any(int(p["qexit"]) > 0 for p in passes)


def test_hadamard_kernel_eligibility(core):
    """Which passes the Hadamard-pass kernel runs: butterflies and exact
    sign terms only (no tables), a closing permutation run on the stores
    allowed; in a circuit that keeps double storage its per-tile int64
    engine takes the Hadamard passes."""
    n = 20
    rng = np.random.default_rng(5)
    ops = inputs.hadamard_all(n)
    ops += [op("Z", (q,)) for q in range(0, n, 3)]
    ops += [op("RZ", (q,), (), (float(t),)) for q, t in enumerate(rng.uniform(0, 6.28, n))]
    ops += inputs.hadamard_all(n)
    summary = core.plan_summary(n, ops)
    head, passes = parse(summary)
    lines = summary.splitlines()[1:]
    assert head["resident"] == 0
    for p, line in zip(passes, lines):
        has_table = int(re.search(r"dsep=(\d+)", line).group(1)) > 0
        if "pipelined" in line:
            assert p["eng"] == "i64" and not has_table and p["load_smem"] == "1"
        if has_table:
            assert "pipelined" not in line
    assert any("pipelined" in l for l in lines)
    # the layered circuit: its three Hadamard passes run in the kernel (the
    # CNOT ladder after them starts the first monomial run pass)
    summary = core.plan_summary(30, inputs.layered_circuit(30, 20, seed=2)).splitlines()[1:]
    hp = [l for l in summary if "pipelined" in l]
    assert len(hp) == 3 and all("gather" not in l for l in hp)


def test_bulk_staging_eligibility(core):
    """Hadamard passes stage their tiles with bulk copies of 128-byte chunks
    when the tile holds the state's low three bits and phase 0 reads the
    natural layout without bank conflicts (no register bit among local bits
    0..2); only the pipelined kernel does."""
    ops, _ = inputs.grover_circuit(33, 8, seed=3)
    passes = core.plan_summary(33, ops).splitlines()[1:]
    bulk = [p for p in passes if " bulk" in p]
    assert len(bulk) >= 30
    for p in bulk:
        assert "pipelined" in p and "tile={0,1,2," in p
    # pass 0 starts with H on qubits 0..3: phase 0 has register bits 0..2
    assert " bulk" not in passes[0]
    for p in core.plan_summary(30, inputs.layered_circuit(30, 20, seed=2)).splitlines()[1:]:
        assert " bulk" not in p or "pipelined" in p


def test_monomial_runs_respect_table_limits_at_n34(core):
    """With 22 tile qubits the per-qubit phases of a layer may not all fit
    table A's selection and table T: runs are cut so that T keeps at most 16
    qubits and A selects at most 8 (the plan as described assumes room for
    the second buffer)."""
    summary = core.plan_summary(34, inputs.layered_circuit(34, 20, seed=2))
    amp = [l for l in summary.splitlines()[1:] if " amp " in l]
    assert len(amp) >= 20
    for l in amp:
        assert int(re.search(r"tile_tab=(\d+)", l).group(1)) <= 16
        assert int(re.search(r"sel_a=(\d+)", l).group(1)) <= 8
