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
