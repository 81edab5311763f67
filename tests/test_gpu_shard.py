"""The patch-sharded iteration through the library on one GPU: two plans, each on
half of the patches (regularisers on the first), whose CMPE totals and gradients
are added as an all-reduce would add them (plain device sums, no collective: the
two plans' kernels never wait on each other).  The result must be the single
plan's loss, dL/ds and Adam update."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402
from paper_2608_06853_b300.shard import shard_problem  # noqa: E402


@pytest.mark.parametrize("maker,n_scat", [(synth.config_tiny, 2000), (synth.config_full, 150_000)])
def test_two_patch_shards_equal_one_plan(maker, n_scat):
    p = maker()
    dev = torch.device("cuda")
    iq = synth.simulate_gpu(p, n_scat, seed=20261207)
    rng = np.random.default_rng(4)
    s0 = torch.from_numpy((1.0 / (1530.0 + 15.0 * rng.standard_normal((p.nz, p.nx)))).astype(np.float32)).to(dev)

    def fresh():
        return s0.clone(), torch.zeros_like(s0), torch.zeros_like(s0), torch.zeros_like(s0)

    # one plan over every patch
    one = af.Plan(p)
    s1, g1, m1, v1 = fresh()
    L1 = torch.zeros(4, device=dev)
    one.af_iterate(iq, s1, g1, m1, v1, 1, L1)
    # two shards, their exchanges done as sums on the device
    shards = [af.Plan(shard_problem(p, r, 2)) for r in range(2)]
    losses = [torch.zeros(4, device=dev) for _ in shards]
    grads = [torch.zeros_like(s0) for _ in shards]
    for pl, L in zip(shards, losses):
        pl.af_forward(iq, s0, L)
    tot = shards[0].cmpe_totals() + shards[1].cmpe_totals()
    for pl, L, g in zip(shards, losses, grads):
        pl.set_cmpe_totals(tot, L)
        pl.af_adjoint(g)
    g2 = grads[0] + grads[1]
    s2, _, m2, v2 = fresh()
    shards[0].af_step(g2, s2, m2, v2, 1)
    torch.cuda.synchronize()
    assert int(round(float(tot[1]))) == one.counters()["n_active"] > 0
    # loss of the whole problem on the shard holding the regularisers
    np.testing.assert_allclose(losses[0].cpu().numpy(), L1.cpu().numpy(), rtol=2e-6)
    # the ray adjoint sums in fixed point scaled by each plan's own max |dL/dT| (about
    # 1e-5 relative; the tolerance of the ray-adjoint parity tests), and the DAS
    # adjoint's float atomics add in any order
    assert float((g2 - g1).norm() / g1.norm()) <= 1e-4
    # Adam normalises per node: nodes with a rounding-level gradient may move differently
    step = p.lr * p.c_unit / 1540.0 ** 2
    d = (s2 - s1).abs()
    assert d.max().item() <= 2 * step and d.median().item() <= 0.01 * step
    for pl in shards + [one]:
        assert pl.af_sync_status() == af.AF_OK
        pl.close()
