"""Collections kept in host memory (series_on_host): the build streams the series through two
device staging buffers (1.1M x 256 = three 512 MB chunks, so both buffers are reused) and the
searches read raw rows from host memory; answers equal the device-built index's and the
oracle's, for pinned and for pageable host memory (registered by the library for the index's
lifetime), with and without the BF16 copy."""
import numpy as np
import pytest

from gpu_common import require_gpu, rw, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("where", ["pinned", "pageable"])
@pytest.mark.parametrize("shadow", [False, True])
def test_series_on_host(where, shadow):
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    n = 1_100_003
    x = rw(n, 256, 23)
    host = torch.from_numpy(x)
    if where == "pinned":
        host = host.pin_memory()
    idx = P.paris_build_ex(host, bf16_shadow=shadow, series_on_host=True)
    view = P.paris_index_describe(idx)
    ref = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    assert np.array_equal(P.paris_export_sax(idx).cpu().numpy(), P.paris_export_sax(ref).cpu().numpy())
    for a, b in zip(P.paris_export_order(idx), P.paris_export_order(ref)):
        assert np.array_equal(a, b)
    q, _, _ = synth.mixed_sigma_queries(x, n, 256, 16, 0.01, 2.0, seed=19)
    Q = torch.from_numpy(q).to(dev)
    wi, wd = oknn.knn(x, q, 3)
    for mode, prec in ((P.PARIS_MODE_PLAIN, P.PARIS_REFINE_FP32), (P.PARIS_MODE_BATCHED, P.PARIS_REFINE_FP32),
                       (P.PARIS_MODE_BATCHED, P.PARIS_REFINE_MIXED)):
        gi, gd = P.paris_exact_knn_ex(idx, Q, 3, mode=mode, precision=prec)
        torch.cuda.synchronize()
        assert np.array_equal(gi.cpu().numpy(), wi)
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0)
    assert view["n"] == n
    idx.free()
    ref.free()
    del host
