"""GPU parity of the index build (PAA, iSAX symbols, keys, index order) against the oracle.
Bit-exact: symbols, keys, sorted order, and the FP64 PAA values themselves."""
import numpy as np
import pytest

import planted
from gpu_common import require_gpu, rw, small_dataset, torch
from oracle import index as oindex
from oracle import isax

pytestmark = pytest.mark.gpu


def encode_gpu(x, w, card):
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    sax, key, paa = P.paris_encode(torch.from_numpy(np.ascontiguousarray(x)).to(dev), w, card, want_paa=True)
    torch.cuda.synchronize()
    return sax.cpu().numpy(), key.cpu().numpy().view(np.uint64), paa.cpu().numpy()


def encode_gpu_symbols(x, w, card):
    """paris_encode without the PAA output: the symbols may then be decided from an fp32 sum
    with a proven error bound (the exact sum only near a breakpoint), as in the index build."""
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    sax, key = P.paris_encode(torch.from_numpy(np.ascontiguousarray(x)).to(dev), w, card)
    torch.cuda.synchronize()
    return sax.cpu().numpy(), key.cpu().numpy().view(np.uint64)


def check_encode(x, w, card):
    sax, key, paa = encode_gpu(x, w, card)
    want_paa = isax.paa(x, w)
    assert paa.tobytes() == want_paa.tobytes(), "PAA differs from the exactly rounded segment sums"
    want_sax = isax.symbols(want_paa, card)
    assert np.array_equal(sax, want_sax)
    assert np.array_equal(key, isax.key64(want_sax, card))
    sax2, key2 = encode_gpu_symbols(x, w, card)
    assert np.array_equal(sax2, want_sax)
    assert np.array_equal(key2, key)


def test_encode_random_walk_100k():
    check_encode(small_dataset(), 16, 256)


@pytest.mark.parametrize("n,length,w,card", [
    (1000, 128, 16, 256), (777, 1024, 16, 256), (513, 256, 4, 4), (300, 96, 8, 256),
    (257, 200, 10, 16), (33, 64, 16, 256), (5, 16, 16, 2), (1, 256, 16, 256), (100, 2048, 16, 256),
    (64, 4096, 16, 256), (100, 48, 16, 64)])
def test_encode_shapes(n, length, w, card):
    check_encode(rw(n, length, 7 + length), w, card)


def test_encode_tiny_and_exact_values():
    x = rw(200, 256, 5)
    x[3, 5] = np.float32(1e-30)            # far below the fast path's fixed-point step
    x[4, 17] = np.float32(-3e-40)          # subnormal
    x[5, :16] = np.float32([2.0 ** 60, 1.0, -(2.0 ** 60), 2.0 ** -20] + [0.0] * 12)
    x[6, :16] = np.float32([1.0, -1.0] * 8)  # PAA exactly 0 = the middle breakpoint
    x[7, 16:32] = 0.0
    x[8, :] = -0.0
    x[9, 32:48] = np.float32(3.0e38)        # large but finite
    x[9, 48:64] = np.float32(-3.0e38)
    check_encode(x, 16, 256)


@pytest.mark.parametrize("length", [256, 512, 1024, 2048, 4096])
def test_encode_planted_exactness(length):
    """Segments built to break a summation that drops low bits (w = 16, so s = len / 16 values
    per segment): the wide-span pattern 1.9999999 / 2^-15+2^-18-2^-38 in four orders and signs,
    random segments at exponent spans around every span limit a TwoSum argument could use, and
    segments whose exact mean lies less than 2^-38/s below the breakpoints 64, 128, 160, 192.
    The PAA bytes must equal the correctly rounded segment sums / s, and the symbols must be
    the lower region's."""
    s = length // 16
    lg = s.bit_length() - 1
    rng = np.random.default_rng(length)
    x = rw(96, length, 40 + length)
    r = 0
    for variant in range(4):
        for seg in (0, 7, 15):
            x[r, seg * s:(seg + 1) * s] = planted.wide_span(s, rng, variant)
            r += 1
    for span in sorted({24 - 2 * lg - 1, 24 - 2 * lg, 24 - 2 * lg + 1, 10, 12, 15, 16}):
        for _ in range(3):
            seg = int(rng.integers(16))
            x[r, seg * s:(seg + 1) * s] = planted.gate(s, span, rng)
            r += 1
    beta = isax.breakpoints(256)
    near = []
    for j in (64, 128, 160, 192):
        for order in ("plain", "reversed", "shuffled"):
            seg = int(rng.integers(16))
            x[r, seg * s:(seg + 1) * s] = planted.below_breakpoint(beta[j - 1], s, order, seed=j)
            near.append((r, seg, j - 1))
            r += 1
    assert r <= x.shape[0]
    check_encode(x, 16, 256)
    sax, _, _ = encode_gpu(x, 16, 256)
    sax2, _ = encode_gpu_symbols(x, 16, 256)
    for row, seg, sym in near:
        assert sax[row, seg] == sym and sax2[row, seg] == sym


@pytest.mark.parametrize("length", [64, 128, 256])
def test_encode_symbols_at_breakpoints(length):
    """Segments whose every value is the fp32 value nearest to a breakpoint, or the fp32 value
    just above or just below it (the mean is then that value exactly): the segment mean lies
    within one fp32 step of the breakpoint, inside any error interval of an fp32 sum, so the
    symbol must come from the exact comparison (upper region on a tie)."""
    s = length // 16
    beta = isax.breakpoints(256)
    x = rw(3 * 255 // 16 + 3, length, 70 + length)
    f32 = np.float32
    k = 0
    for j in range(255):
        c = f32(beta[j])
        for v in (c, np.nextafter(c, f32(np.inf), dtype=f32), np.nextafter(c, f32(-np.inf), dtype=f32)):
            r, seg = divmod(k, 16)
            x[r, seg * s:(seg + 1) * s] = v
            k += 1
    check_encode(x, 16, 256)


def test_encode_rejects_nonfinite():
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = rw(64, 256, 3)
    x[10, 100] = np.inf
    with pytest.raises(P.ParisError) as e:
        P.paris_encode(torch.from_numpy(x).to(dev), 16, 256)
    assert e.value.status == 1
    x[10, 100] = np.nan
    with pytest.raises(P.ParisError):
        P.paris_build(torch.from_numpy(x).to(dev), 16, 256)


@pytest.mark.parametrize("n", [100_000, 4096 * 3 + 17, 1, 2])
def test_build_index_order(n):
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = small_dataset()[:n] if n <= 100_000 else rw(n, 256, 1)
    idx = P.paris_build(torch.from_numpy(np.ascontiguousarray(x)).to(dev), 16, 256)
    view = P.paris_index_describe(idx)
    assert view["n"] == n and view["leaf_capacity"] == 2048
    sax = P.paris_export_sax(idx).cpu().numpy()
    want_sax = isax.isax_words(x, 16, 256)
    assert np.array_equal(sax, want_sax)
    got_keys, got_rows = P.paris_export_order(idx)
    want_rows, want_keys = oindex.sort_order(isax.key64(want_sax, 256))
    assert np.array_equal(got_keys, want_keys)
    assert np.array_equal(got_rows, want_rows)
    idx.free()


@pytest.mark.parametrize("where", ["pinned", "pageable"])
@pytest.mark.parametrize("shadow", [False, True])
def test_build_from_host_series(where, shadow):
    """A host series is copied in 512 MB chunks on two copy streams while the encode pass works
    through the chunks already copied (1.1 GB here: three chunks, the last one partial). Pinned
    or pageable, the index equals the device-built one and the answers are exact."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    n = 1_100_003
    x = rw(n, 256, 21)
    host = torch.from_numpy(x)
    if where == "pinned":
        host = host.pin_memory()
    idx = P.paris_build_ex(host, bf16_shadow=shadow)
    ref = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    assert np.array_equal(P.paris_export_sax(idx).cpu().numpy(), P.paris_export_sax(ref).cpu().numpy())
    for a, b in zip(P.paris_export_order(idx), P.paris_export_order(ref)):
        assert np.array_equal(a, b)
    q, _, _ = synth.mixed_sigma_queries(x, n, 256, 12, 0.01, 2.0, seed=9)
    wi, wd = oindex_knn(x, q)
    for prec in (P.PARIS_REFINE_FP32, P.PARIS_REFINE_MIXED):
        gi, gd = P.paris_exact_knn_ex(idx, torch.from_numpy(q).to(dev), 3, mode=P.PARIS_MODE_BATCHED, precision=prec)
        assert np.array_equal(gi.cpu().numpy(), wi)
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0)
    idx.free()
    ref.free()


def oindex_knn(x, q):
    from oracle import knn as oknn
    return oknn.knn(x, q, 3)
