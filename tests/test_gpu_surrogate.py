"""Lens-surrogate MLP on the tensor cores: gradients against the float64 oracle,
training with exact-solver fallback, and the delay error it leaves (<= lambda/50)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402
from oracle import mlp_oracle as mo  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def tiny_plan():
    p = synth.config_tiny()
    psi = synth.simulate(p, 2000, seed=20261202)
    dev = torch.device("cuda")
    plan = af.Plan(p)
    iq = torch.from_numpy(psi).to(dev)
    s = torch.from_numpy(p.initial_slowness()).to(dev)
    loss = torch.zeros(4, device=dev)
    plan.af_forward(iq, s, loss)
    torch.cuda.synchronize()
    return p, plan, iq, s


def test_mlp_gradient_matches_float64_oracle(tiny_plan):
    p, plan, iq, s = tiny_plan
    dev = torch.device("cuda")
    rng = np.random.default_rng(4)
    params = mo.init(5)
    params = params + 0.05 * rng.standard_normal(params.shape)     # non-zero biases too
    plan.set_surrogate_params(torch.from_numpy(params.astype(np.float32)).to(dev))
    X = rng.uniform(-1, 1, (512, 4)).astype(np.float32)
    Y = rng.uniform(-1, 1, (512, 2)).astype(np.float32)
    g, L = plan.surrogate_grad(torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev))
    g = g.cpu().numpy().astype(np.float64)
    p32 = params.astype(np.float32).astype(np.float64)
    L_or, g_or = mo.forward_backward(p32, X, Y, round_bf16=True)
    assert L == pytest.approx(L_or, rel=2e-3)
    o = 0
    for name, shape in mo.SIZES:
        n = int(np.prod(shape))
        e = rel_l2(g[o:o + n], g_or[o:o + n])
        print(f"{name}: rel L2 {e:.2e}")
        assert e < 1e-2, name
        o += n


def test_surrogate_training_fallback_and_delay_error(tiny_plan):
    p, plan, iq, s = tiny_plan
    rep = plan.surrogate_train(n_samples=1_000_000, epochs=3, tiles_per_step=32, lr=2e-3, seed=7)
    print(rep)
    assert rep["train_loss"] < 1e-2
    assert rep["fallback_fraction"] < 0.2
    dev = torch.device("cuda")
    loss = torch.zeros(4, device=dev)
    plan.surrogate_enable(False)
    plan.af_forward(iq, s, loss)
    T0, a0 = plan.delays()
    plan.surrogate_enable(True)
    plan.af_forward(iq, s, loss)
    T1, a1 = plan.delays()
    plan.surrogate_enable(False)
    on = (a0 == 1).cpu().numpy()
    err = np.abs((T1 - T0).cpu().numpy())[on]
    print(f"surrogate delay error: max {err.max() * 1e9:.4f} ns, tolerance {rep['tolerance'] * 1e9:.3f} ns")
    assert err.max() <= rep["tolerance"]


def test_surrogate_gain_over_the_exact_solver_full_size():
    """What the trained network gains over the method without it, on the 128-element
    workload: the same plan with the surrogate off and on, timed (CUDA events on the
    plan's stream) for whole iterations (exit solve warm-started from the previous
    iteration) and for cold starts (exit angles of moved pixels, as at each speed of the
    dynamic sweep).  The gain or loss is printed, not asserted; the delay error the
    surrogate leaves after fallback must stay within lambda/50."""
    p = synth.config_full()
    dev = torch.device("cuda")
    iq = synth.simulate_gpu(p, 150_000, seed=20261203)
    plan = af.Plan(p)
    s = torch.from_numpy(p.initial_slowness()).to(dev)
    g, m, v = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
    loss = torch.zeros(4, device=dev)
    plan.af_forward(iq, s, loss)
    rep = plan.surrogate_train(n_samples=10_000_000, epochs=4, tiles_per_step=32, lr=2e-3, seed=1)

    def timed(fn, n):
        st = plan.stream
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(n):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    def iterate():
        plan.af_iterate(iq, s, g, m, v, 1, loss)

    def cold_forward():
        plan.af_set_pixels(p.pix_x, p.pix_z)           # drops the warm start
        plan.af_forward(iq, s, loss)

    out = {}
    for on in (False, True):
        plan.surrogate_enable(on)
        s.fill_(1.0 / 1540.0)
        out[on] = (timed(iterate, 10), timed(cold_forward, 5))
    plan.surrogate_enable(False)
    plan.af_forward(iq, s, loss)
    T0, a0 = plan.delays()
    plan.surrogate_enable(True)
    plan.af_forward(iq, s, loss)
    T1, _ = plan.delays()
    plan.surrogate_enable(False)
    on = (a0 == 1).cpu().numpy()
    err = float(np.abs((T1 - T0).cpu().numpy())[on].max())
    print(f"surrogate gain, 128-element workload: iteration {out[False][0]:.3f} -> {out[True][0]:.3f} ms "
          f"({1e3 / out[False][0]:.0f} -> {1e3 / out[True][0]:.0f} it/s); cold-start forward "
          f"{out[False][1]:.3f} -> {out[True][1]:.3f} ms; max delay error {err * 1e9:.3f} ns "
          f"(lambda/50 = {rep['tolerance'] * 1e9:.2f} ns); fallback {rep['fallback_fraction']:.4f}")
    assert err <= rep["tolerance"]
    assert all(np.isfinite(x) and x > 0 for x in out[False] + out[True])
    plan.close()
