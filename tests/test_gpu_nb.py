"""Best-so-far sharing ablation (nb-ParIS+ keeps a BSF per worker, ParIS+ shares one, Sec. 3.3.2
and 3.3.3): with per-warp private thresholds the answers stay exact (each private threshold still
bounds the k-th distance from above), and refinement reads at least about as many rows, on noisy copies of dataset rows and on independent random
walks (the hard queries)."""
import numpy as np
import pytest

from gpu_common import require_gpu, small_dataset, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k", [1, 10])
def test_private_bsf_exact_and_reads_more(mode, k):
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = small_dataset()
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    src = synth.sigma_query_sources(x.shape[0], 10)
    q = np.concatenate([synth.noisy_queries(x[src], 0.3, [7, 1]), synth.random_walk(10, 256, seed=31)])
    Q = torch.from_numpy(q).to(dev)
    wi, wd = oknn.knn(x, q, k)
    out = {}
    for priv in (False, True):
        gi, gd, st = P.paris_exact_knn_ex(idx, Q, k, mode=mode, want_stats=True, private_bsf=priv)
        torch.cuda.synchronize()
        assert np.array_equal(gi.cpu().numpy(), wi)
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0)
        out[priv] = st
    assert out[True]["refined"] >= 0.95 * out[False]["refined"]
    assert out[False]["bsf_updates"] > 0
    idx.free()
