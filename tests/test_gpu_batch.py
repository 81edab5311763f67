"""Batched acquisitions of uneven size as one CUDA graph: the graph replay gives
the same speed maps as issuing the same calls stream by stream."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from paper_2608_06853_b300.batch import BatchRunner  # noqa: E402


def test_graph_replay_matches_eager_for_uneven_batch():
    dev = torch.device("cuda")
    problems, iqs = [], []
    for k in range(3):
        p = synth.config_batch_member(k, n_ang=4, n_rad=4, nx=32, nz=32)
        psi = synth.simulate(p, 3000, seed=50 + k)
        problems.append(p)
        iqs.append(torch.from_numpy(psi).to(dev))
    sizes = {(p.ne, p.ns, p.nx) for p in problems}
    assert len(sizes) == 3                                    # uneven
    br = BatchRunner(problems, iqs)

    def run(n, graph):
        br.reset()
        if graph:
            br.capture(n)
            br.reset()
            br.replay()
        else:
            br.run_eager(n)
        torch.cuda.synchronize()
        return ([x.cpu().numpy().copy() for x in br.s], [x.cpu().numpy().copy() for x in br.g],
                [x.cpu().numpy().copy() for x in br.loss])

    # one iteration: the forward is deterministic, the adjoint differs only by the
    # order of float atomic additions
    s1e, g1e, l1e = run(1, False)
    s1g, g1g, l1g = run(1, True)
    for k in range(len(problems)):
        np.testing.assert_allclose(l1g[k], l1e[k], rtol=1e-6)
        assert np.linalg.norm(g1g[k] - g1e[k]) <= 1e-4 * np.linalg.norm(g1e[k])
    # five iterations: Adam's per-node normalisation can turn rounding-level gradient
    # differences on near-zero gradients into a fraction of a step; bound the divergence
    s5e, _, l5e = run(5, False)
    s5g, _, l5g = run(5, True)
    for k in range(len(problems)):
        step = problems[k].lr * problems[k].c_unit / 1540.0 ** 2    # one Adam step in slowness
        d = np.abs(s5g[k] - s5e[k])
        assert np.isfinite(s5g[k]).all()
        assert d.max() <= 2.0 * step and np.median(d) <= 0.01 * step
        np.testing.assert_allclose(l5g[k], l5e[k], rtol=1e-2)


def _uneven(n=3, n_scat=3000, seed=50):
    dev = torch.device("cuda")
    problems, iqs = [], []
    for k in range(n):
        p = synth.config_batch_member(k, n_ang=4, n_rad=4, nx=32, nz=32)
        problems.append(p)
        iqs.append(torch.from_numpy(synth.simulate(p, n_scat, seed=seed + k)).to(dev))
    return problems, iqs


@pytest.mark.parametrize("legacy_stream", [False, True])
def test_batch_members_match_single_plans(legacy_stream):
    """af_batch_iterate gives every member what af_iterate gives the same problem
    on a plan of its own (the caller's stream may be the legacy default stream)."""
    import paper_2608_06853_b300 as af
    problems, iqs = _uneven()
    stream = torch.cuda.default_stream() if legacy_stream else torch.cuda.Stream()
    assert (stream.cuda_stream == 0) == legacy_stream
    br = BatchRunner(problems, iqs, stream=stream)
    br.reset()
    br.run_eager(2)
    torch.cuda.synchronize()
    for k, p in enumerate(problems):
        plan = af.Plan(p)
        s = torch.from_numpy(p.initial_slowness()).cuda()
        g, m, v = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
        loss = torch.zeros(4, device="cuda")
        for it in (1, 2):
            plan.af_iterate(iqs[k], s, g, m, v, it, loss)
        torch.cuda.synchronize()
        np.testing.assert_allclose(br.loss[k].cpu().numpy(), loss.cpu().numpy(), rtol=1e-5)
        assert torch.linalg.norm(br.g[k] - g) <= 1e-4 * torch.linalg.norm(g)
        # float atomics in the DAS adjoint: near-zero gradients may flip an Adam step
        step = p.lr * p.c_unit / 1540.0 ** 2
        d = (br.s[k] - s).abs()
        assert d.max().item() <= 4.0 * step and d.median().item() <= 0.01 * step
        # the member getters reach the batch's plan
        b_batch, _ = br.plans[k].bmode()
        b_single, _ = plan.bmode()
        assert b_batch.shape == b_single.shape
        assert br.plans[k].af_sync_status() == af.AF_OK
        plan.close()
    br.close()


def test_batch_state_errors():
    import ctypes

    import paper_2608_06853_b300 as af
    problems, iqs = _uneven(n=2)
    br = BatchRunner(problems, iqs)
    lib = br.lib
    assert lib.af_batch_launch(br.handle) == af.AF_ERR_STATE            # nothing captured yet
    h = ctypes.c_void_p()
    assert lib.af_batch_plan_of(br.handle, 2, ctypes.byref(h)) == af.AF_ERR_ARG
    assert lib.af_batch_plan_of(br.handle, -1, ctypes.byref(h)) == af.AF_ERR_ARG
    iq, sc, s, g, m, v, loss = br._ptrs
    holes = (ctypes.c_void_p * 2)(s[0], None)                          # member 1 has no buffer
    assert lib.af_batch_iterate(br.handle, iq, sc, holes, g, m, v, 1, loss) == af.AF_ERR_ARG
    assert lib.af_batch_capture(br.handle, iq, sc, s, g, m, v, loss, 0, 1) == af.AF_ERR_ARG
    br.plans[1].set_timing(True)
    assert lib.af_batch_capture(br.handle, iq, sc, s, g, m, v, loss, 1, 1) == af.AF_ERR_STATE
    br.plans[1].set_timing(False)
    br.capture(2)
    br.reset()
    br.replay()
    torch.cuda.synchronize()
    assert all(np.isfinite(x.cpu().numpy()).all() for x in br.s)
    br.close()
