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
    br.reset()
    br.run_eager(5)
    torch.cuda.synchronize()
    eager = [x.cpu().numpy().copy() for x in br.s]
    br.capture(5)
    br.reset()
    br.replay()
    torch.cuda.synchronize()
    graph = [x.cpu().numpy() for x in br.s]
    for a, b in zip(eager, graph):
        # float atomics in the adjoint may reorder: compare to float32 rounding scale
        np.testing.assert_allclose(b, a, rtol=1e-4)
        assert np.isfinite(b).all()
