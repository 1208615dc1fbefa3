"""The Hadamard-pass kernel (butterflies and sign terms; persistent, the
next tile copied asynchronously under the last phase) against the oracle:
whole-state tiles of a few threads (n < 12), and the per-tile int64 engine
it also runs for circuits that keep double storage."""
import numpy as np
import pytest

from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from paper_2411_15332_gb300.inputs import op
from tests.gpu_helpers import lib_ready, max_err, new_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


def _pipelined(n, ops):
    from paper_2411_15332_gb300 import core
    lines = core.plan_summary(n, ops).splitlines()
    return lines[0], [l for l in lines[1:] if "per-gate" not in l]


@pytest.mark.parametrize("n", [5, 6, 8, 11])
def test_small_states(n):
    """n < 12: one tile of 2^(n-4) threads (fewer than a warp for n < 9)."""
    ops, m = inputs.grover_circuit(n, 3, seed=3)
    head, tile = _pipelined(n, ops)
    assert "resident=0" in head and all("pipelined" in l and "eng=i64" in l for l in tile)
    s = new_state(n)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    assert max_err(got, sv.simulate(n, ops)) <= 1e-13


@pytest.mark.parametrize("n", [7, 20])
def test_per_tile_engine(n):
    """Hadamard layers around a table pass (RZ on every qubit) keep double
    storage: the Hadamard passes run the kernel's per-tile int64 engine
    (block exponent from a tile max, conversions in and out)."""
    rng = np.random.default_rng(50 + n)
    ops = inputs.hadamard_all(n)
    ops += [op("Z", (q,)) for q in range(0, n, 3)]
    ops += [op("RZ", (q,), (), (float(t),)) for q, t in enumerate(rng.uniform(0, 6.28, n))]
    ops += inputs.hadamard_all(n)
    ops += [inputs.flip_index(n, int(rng.integers(0, 1 << n)))]
    ops += [op("H", (q,)) for q in range(1, n, 2)]
    head, tile = _pipelined(n, ops)
    assert "resident=0" in head
    assert any("eng=i64" in l and "pipelined" in l for l in tile)
    s = new_state(n)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    assert max_err(got, sv.simulate(n, ops)) <= 1e-13


def test_small_then_full_tiles():
    """The same kernel variant with a whole-state tile of a few hundred
    bytes, then a full 64 KiB tile, then small again: a kernel's dynamic
    shared-memory limit may only grow between launches."""
    for n in (6, 14, 7, 14):
        ops, _ = inputs.grover_circuit(n, 1, seed=3)
        s = new_state(n)
        s.apply_circuit(ops, mode="fused")
        got = s.to_numpy()
        s.close()
        assert max_err(got, sv.simulate(n, ops)) <= 1e-13


def test_bulk_staging_matches_element_copies(tmp_path):
    """Tiles staged by bulk copies of whole 128-byte chunks (natural order in
    shared memory) give the same bits as 16-byte asynchronous copies into a
    swizzled layout (a process with MERA_BULK=0), and both match the oracle."""
    import os
    import subprocess
    import sys
    n = 20
    ops, _ = inputs.grover_circuit(n, 2, seed=3)
    head, tile = _pipelined(n, ops)
    assert sum(" bulk" in l for l in tile) >= len(tile) // 2
    s = new_state(n)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    out = tmp_path / "elementwise.npy"
    code = ("import numpy as np\n"
            "from paper_2411_15332_gb300 import inputs, core\n"
            f"ops, _ = inputs.grover_circuit({n}, 2, seed=3)\n"
            f"assert ' bulk' not in core.plan_summary({n}, ops)\n"
            f"s = core.State({n})\n"
            "s.apply_circuit(ops, mode='fused')\n"
            f"np.save({str(out)!r}, s.to_numpy())\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code], cwd=root, env={**os.environ, "MERA_BULK": "0"}, check=True,
                   timeout=600)
    ref = np.load(out)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    assert max_err(got, sv.simulate(n, ops)) <= 1e-13


def test_bulk_wait_runs_out_and_is_reported():
    """Failure detection of the bulk staging: with a test hook every tile
    expects 16 bytes more than its copies deliver, so each CTA's bounded
    wait runs out (about a second), sets the status flag and returns.  The
    next synchronising call reports MERA_ETIMEOUT once; the context and the
    state stay usable and a normal run afterwards matches the oracle."""
    from paper_2411_15332_gb300 import _lib as L
    n = 16
    ops = [op("H", (q,)) for q in list(range(4, 12)) + [0]]
    head, tile = _pipelined(n, ops)
    assert len(tile) == 1 and " bulk" in tile[0]
    s = new_state(n)
    L.check(L.lib().mera_test_bulk_shortfall(16))
    try:
        s.apply_circuit(ops, mode="fused")
        with pytest.raises(L.MeraError) as e:
            s.synchronize()
        assert e.value.code == L.MERA_ETIMEOUT
    finally:
        L.check(L.lib().mera_test_bulk_shortfall(0))
    s.synchronize()   # reported once
    s.set_basis(0)
    s.apply_circuit(ops, mode="fused")
    got = s.to_numpy()
    s.close()
    assert max_err(got, sv.simulate(n, ops)) <= 1e-13


def test_bulk_shortfall_hook_validates():
    from paper_2411_15332_gb300 import _lib as L
    assert L.lib().mera_test_bulk_shortfall(8) == L.MERA_EINVAL
    assert L.lib().mera_test_bulk_shortfall(8192) == L.MERA_EINVAL
    assert L.lib().mera_test_bulk_shortfall(0) == L.MERA_OK


def test_thirteen_bit_tiles(tmp_path):
    """MERA_TILE_BITS=13 (another process): 2^13-amplitude tiles, the
    512-thread variant of the kernel, one CTA per SM; same result as the
    oracle."""
    import os
    import subprocess
    import sys
    n = 17
    ops, _ = inputs.grover_circuit(n, 2, seed=3)
    out = tmp_path / "k13.npy"
    code = ("import numpy as np\n"
            "from paper_2411_15332_gb300 import inputs, core\n"
            f"ops, _ = inputs.grover_circuit({n}, 2, seed=3)\n"
            f"assert core.plan_summary({n}, ops).startswith('K=13')\n"
            f"s = core.State({n})\n"
            "s.apply_circuit(ops, mode='fused')\n"
            f"np.save({str(out)!r}, s.to_numpy())\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code], cwd=root, env={**os.environ, "MERA_TILE_BITS": "13"}, check=True,
                   timeout=600)
    assert max_err(np.load(out), sv.simulate(n, ops)) <= 1e-13
