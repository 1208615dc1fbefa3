"""GPU parity of the batched QNN ansatz (forward, expectations) and of the
adjoint gradients, against the FP64 oracle (full simulation, parameter
shift, central differences)."""
import numpy as np
import pytest

from oracle import circuits as oc
from oracle import statevector as sv
from paper_2411_15332_gb300 import inputs
from tests.gpu_helpers import TOL, lib_ready, max_err, obs_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _ready():
    lib_ready()


def _batch(n, cap, dtype):
    from paper_2411_15332_gb300 import Batch
    return Batch(n, cap, dtype)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,L,B", [(6, 3, 5), (9, 4, 3), (14, 2, 4), (16, 2, 2)])
def test_batch_forward_matches_oracle(dtype, n, L, B):
    theta = inputs.qnn_batch(B, n, L, seed=n + L)
    b = _batch(n, B + 2, dtype)
    b.forward(theta)
    got = b.states(range(B))
    obs = b.observables(range(B), q=0)
    for j in range(B):
        ref = sv.simulate(n, inputs.ansatz_ops(n, theta[j]))
        assert max_err(got[j], ref) <= TOL[dtype]
        assert abs(obs[j, 0] - 1.0) <= TOL[dtype]
        assert abs(obs[j, 1] - sv.expect_z(ref, n, 0)) <= obs_tol(dtype, 1)
        assert abs(obs[j, 2] - sv.expect_z_sum(ref, n)) <= obs_tol(dtype, n)


def test_slot_results_do_not_depend_on_the_mix():
    """Continuous-batching invariant: a circuit's state and expectations are
    bit-identical run alone or among other circuits at other layers."""
    n, L = 10, 5
    th = inputs.qnn_batch(4, n, L, seed=3)
    alone = _batch(n, 1, "c64")
    alone.forward(th[:1])
    ref_state = alone.states([0])[0]
    ref_obs = alone.observables([0], 0)[0]
    mix = _batch(n, 8, "c64")
    mix.reset(range(8))
    # slot 5 runs circuit 0; the other slots start at different times
    for step in range(L + 3):
        slots, rows = [], []
        if step < L:
            slots.append(5)
            rows.append(th[0, step])
        for k, s in enumerate((1, 2, 6)):
            if step >= k:
                slots.append(s)
                rows.append(th[1 + k, min(step - k, L - 1)])
        mix.layer(slots, np.stack(rows))
    assert np.array_equal(mix.states([5])[0], ref_state)
    assert np.array_equal(mix.observables([5], 0)[0], ref_obs)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adjoint_matches_parameter_shift_and_fd(dtype):
    n, L, B = 6, 2, 3
    tol = obs_tol(dtype, n)          # loss = sum_q <Z_q>: observable norm n
    theta = inputs.qnn_batch(B, n, L, seed=11)
    b = _batch(n, B, dtype)
    loss, grad = b.adjoint_grad(theta)
    for j in range(B):
        f = oc.qnn_value(n, theta[j], inputs.ansatz_ops, "zsum")
        assert abs(loss[j] - f) <= tol
        ps = oc.param_shift_grad(n, theta[j], inputs.ansatz_ops, "zsum")
        np.testing.assert_allclose(grad[j], ps, atol=tol, rtol=0)
    # central differences carry O(h^2) ~ 1e-12 truncation and ~1e-10
    # cancellation error of their own
    fd = oc.finite_diff_grad(n, theta[0], inputs.ansatz_ops, "zsum")
    np.testing.assert_allclose(grad[0], fd, atol=max(tol, 1e-8), rtol=0)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_adjoint_training_full_shape(dtype):
    """The training workload at its full shape (1024 circuits, n = 16, 10
    layers, 320 angles each) in one call; every one of the 320 derivatives
    and the loss of three circuits (first, middle, last row) against the
    oracle's reverse sweep, and 8 derivatives of circuit 0 against the
    parameter-shift rule."""
    n, L, B = 16, 10, 1024
    tol = obs_tol(dtype, n)
    theta = inputs.qnn_batch(B, n, L, seed=5)
    b = _batch(n, B, dtype)
    loss, grad = b.adjoint_grad(theta)
    b.close()
    ops_fn = inputs.ansatz_ops
    worst_g, worst_f = 0.0, 0.0
    for j in (0, B // 2, B - 1):
        f, g = oc.adjoint_grad(n, theta[j], ops_fn, "zsum")
        worst_g = max(worst_g, float(np.max(np.abs(grad[j] - g))))
        worst_f = max(worst_f, abs(loss[j] - f))
    rng = np.random.default_rng(0)
    flat = theta[0].reshape(-1)
    for p in rng.choice(flat.size, size=8, replace=False):
        tp = flat.copy()
        tp[p] += np.pi / 2
        fp = oc.qnn_value(n, tp.reshape(theta[0].shape), ops_fn, "zsum")
        tp[p] -= np.pi
        fm = oc.qnn_value(n, tp.reshape(theta[0].shape), ops_fn, "zsum")
        worst_g = max(worst_g, abs(grad[0].reshape(-1)[p] - 0.5 * (fp - fm)))
    print(f"adjoint n=16 L=10 B=1024 {dtype}: max |d grad| = {worst_g:.3e}, max |d loss| = {worst_f:.3e} "
          f"(bound {tol:.1e})")
    assert worst_g <= tol
    assert worst_f <= tol


def test_autograd_function():
    import torch
    from paper_2411_15332_gb300 import AdjointExpectation
    n, L, B = 6, 2, 2
    theta = torch.tensor(inputs.qnn_batch(B, n, L, seed=2), dtype=torch.float64, requires_grad=True)
    b = _batch(n, B, "c128")
    loss = AdjointExpectation.apply(theta, b)
    loss.backward()
    ref = np.mean([oc.qnn_value(n, theta.detach().numpy()[j], inputs.ansatz_ops, "zsum") for j in range(B)])
    assert abs(loss.item() - ref) <= obs_tol("c128", n)
    ps = np.stack([oc.param_shift_grad(n, theta.detach().numpy()[j], inputs.ansatz_ops, "zsum") for j in range(B)])
    np.testing.assert_allclose(theta.grad.numpy(), ps / B, atol=obs_tol("c128", n), rtol=0)


def test_server_mix_equals_alone_and_oracle():
    """Continuous batching on the GPU: every request's <Z_0> equals its
    result served alone (bit for bit) and the oracle (complex64 tolerance)."""
    from paper_2411_15332_gb300.serve import Server, requests_from_workload
    reqs = requests_from_workload(inputs.qnn_requests(40, seed=4, n_lo=8, n_hi=12, l_lo=2, l_hi=6))
    srv = Server(dtype="c64", mem_budget=1 << 27, slots_per_n=6)
    done = {r.rid: r for r in srv.run(reqs)}
    assert len(done) == 40 and all(r.error is None for r in done.values())
    st = srv.stats()
    assert st["launches"] < sum(r.layers for r in done.values())   # layers shared launches
    for rid in list(done)[:8]:
        r = done[rid]
        solo = Server(dtype="c64", mem_budget=1 << 27, slots_per_n=1)
        (alone,) = solo.run([type(r)(rid=r.rid, n=r.n, theta=r.theta)])
        assert alone.result == r.result
        ref = sv.expect_z(sv.simulate(r.n, inputs.ansatz_ops(r.n, r.theta)), r.n, 0)
        assert abs(r.result - ref) <= 2e-5
