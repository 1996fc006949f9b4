"""The learned best-so-far proposal on the GPU: forward pass and gradients against the FP64
oracle (same BF16-representable weights; the GPU rounds GEMM operands to BF16 and accumulates
in FP32), the uniform-logit closed form, training, and what the trained network gains over the
plain approximate search (a tighter seed, never a looser one) at unchanged exact answers."""
import math

import numpy as np
import pytest

import mlp_bounds
from gpu_common import require_gpu, small_dataset, torch
from oracle import isax
from oracle import knn as oknn
from oracle import mlp

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even) and back to float32."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def bf16_params(seed, scale, bias=None):
    """BF16-representable weights ~ N(0, scale^2 / fan_in); biases ~ N(0, bias^2) when given."""
    rng = np.random.default_rng(seed)
    out = {k: bf16_round(rng.standard_normal(s) * scale / math.sqrt(s[-1])) for k, s in mlp.SHAPES.items()}
    if bias is not None:
        for k in ("b1", "b2", "b3"):
            out[k] = bf16_round(rng.standard_normal(mlp.SHAPES[k]) * bias)
    return out


def sparse_params(seed, nnz=6, scale=0.5, bias=0.5):
    """BF16-representable weights with `nnz` nonzeros ~ N(0, scale^2) at random inputs of every
    output, biases ~ N(0, bias^2). Few terms per output keep the worst-case error bounds
    tight through three layers, and every output depends on specific rows and columns, so an
    indexing mistake moves it far outside its bound."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, s in mlp.SHAPES.items():
        if len(s) == 2:
            w = np.zeros(s, np.float32)
            for o in range(s[0]):
                cols = rng.choice(s[1], nnz, replace=False)
                w[o, cols] = rng.standard_normal(nnz) * scale
            out[k] = bf16_round(w)
        else:
            out[k] = bf16_round(rng.standard_normal(s) * bias)
    return out


def f64(p):
    return {k: v.astype(np.float64) for k, v in p.items()}


def paa_inputs(m, seed):
    return np.random.default_rng(seed).standard_normal((m, 16)) * 0.8


def test_forward_elementwise():
    """Every logit within its element-wise bound (BF16 operand rounding, FP32 accumulation and
    the FP32 GELU, carried through the layers) of the FP64 oracle; a bias shifted by one bucket
    in the oracle is far outside those bounds."""
    import paper_2009_00166_gb300 as P
    require_gpu()
    p = sparse_params(1)
    x = paa_inputs(200, 2)
    md = P.SeedModel(0)
    md.set_weights(p)
    got = md.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    want, bound, _ = mlp_bounds.forward_bounds(f64(p), x)
    err = np.abs(got - want)
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert np.all(err <= bound), (worst, err[worst], bound[worst])
    assert np.median(bound) < 0.1 * np.std(want)           # the bound is far tighter than the data
    wrong = f64(p)
    wrong["b3"] = np.roll(wrong["b3"], 1)
    bad, _, _ = mlp_bounds.forward_bounds(wrong, x)
    assert np.mean(np.abs(got - bad) > bound) > 0.5
    md.free()


def test_gradients_elementwise():
    """Loss and every gradient element within its bound of the FP64 oracle (the softmax, GELU'
    and column sums in FP32, every GEMM with BF16 operands); labels shifted by one bucket or
    input features shifted by one segment in the oracle land far outside those bounds."""
    import paper_2009_00166_gb300 as P
    require_gpu()
    p = sparse_params(3)
    B = 16
    x = paa_inputs(B, 4)
    y = np.random.default_rng(5).integers(0, 4096, B).astype(np.int32)
    md = P.SeedModel(0)
    md.set_weights(p)
    loss, g = md.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    wl, wg, bound = mlp_bounds.gradient_bounds(f64(p), x, y)
    assert abs(loss - wl) < 1e-3 * wl
    for k in mlp.ORDER:
        a, b, e = g[k].astype(np.float64), wg[k], bound[k]
        err = np.abs(a - b)
        with np.errstate(invalid="ignore", divide="ignore"):
            i = np.unravel_index(np.argmax(err / e), err.shape)
        assert np.all(err <= e), (k, i, err[i], e[i], b[i])
        assert np.median(e) < 0.25 * np.std(b), k             # the bound is tighter than the data
    _, wrong_y, _ = mlp_bounds.gradient_bounds(f64(p), x, (y + 1) % 4096)
    assert np.mean(np.abs(g["b3"] - wrong_y["b3"]) > bound["b3"]) > 0.9 * 2 * B / 4096
    _, wrong_x, _ = mlp_bounds.gradient_bounds(f64(p), np.roll(x, 1, axis=1), y)
    assert np.mean(np.abs(g["W1"] - wrong_x["W1"]) > bound["W1"]) > 0.3
    md.free()


def test_topr_matches_oracle_with_ties():
    """The top-r selection on the GPU's own logits equals the oracle's ordering (score
    descending, bucket ascending) exactly, with planted exact ties: duplicated output rows and
    biases make buckets 100 and 3000 tie for first place and 7, 2000 and 4000 tie below them."""
    import paper_2009_00166_gb300 as P
    require_gpu()
    p = sparse_params(8)
    for j in (3000,):
        p["W3"][j] = p["W3"][100]
    p["b3"][[100, 3000]] = 20.0
    for j in (2000, 4000):
        p["W3"][j] = p["W3"][7]
    p["b3"][[7, 2000, 4000]] = 16.0
    x = paa_inputs(300, 9)
    md = P.SeedModel(0)
    md.set_weights(p)
    X = torch.from_numpy(x).cuda()
    logits = md.forward(X).cpu().numpy()
    for r in (1, 3, 5, 8):
        got = md.topr(X, r).cpu().numpy()
        want = mlp.topr_of_logits(logits, r)
        assert np.array_equal(got, want), r
    top = md.topr(X, 5).cpu().numpy()
    assert np.mean(np.all(top[:, :2] == [100, 3000], axis=1)) > 0.9
    # where the exact FP64 scores are separated by more than twice their bounds, the GPU picks
    # the oracle's buckets
    want64, bound, _ = mlp_bounds.forward_bounds(f64(p), x)
    ranked = np.sort(want64, axis=1)[:, ::-1]
    sep = np.all(ranked[:, :8] - ranked[:, 1:9] > 2 * bound.max(axis=1, keepdims=True), axis=1)
    if sep.any():
        assert np.array_equal(md.topr(X, 8).cpu().numpy()[sep], mlp.topr_of_logits(want64, 8)[sep])
    with pytest.raises(P.ParisError):
        md.topr(X, 9)
    md.free()


def test_uniform_logits_closed_form():
    import paper_2009_00166_gb300 as P
    require_gpu()
    md = P.SeedModel(0)
    md.set_weights({k: np.zeros(s, np.float32) for k, s in mlp.SHAPES.items()})
    y = np.array([0, 5, 4095, 77], np.int32)
    loss, g = md.gradients(torch.from_numpy(paa_inputs(4, 6)).cuda(), torch.from_numpy(y).cuda())
    assert abs(loss - math.log(4096)) < 1e-5
    assert np.all(g["W1"] == 0) and np.all(g["W3"] == 0)
    assert abs(g["b3"][0] - (4 / 4096 - 1) / 4) < 1e-7
    md.free()


def test_row_buckets_match_oracle_keys():
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = small_dataset()[:5000]
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    rows = np.array([0, 1, 17, 4999, 2500])
    got = P.paris_row_buckets(idx, rows)
    want = (isax.key64(isax.isax_words(x[rows], 16, 256), 256) >> np.uint64(52)).astype(np.int32)
    assert np.array_equal(got, want)
    with pytest.raises(P.ParisError):
        P.paris_row_buckets(idx, np.array([5000]))
    idx.free()


def test_learned_seed_gains_over_plain_descent():
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = small_dataset()
    n = x.shape[0]
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)

    def make(seed, m, sigma):
        src = np.random.default_rng([seed, 0]).choice(n, m, replace=False)
        return synth.noisy_queries(x[src], sigma, [seed, 1])

    train_q = np.concatenate([make(40, 6000, 0.1), make(41, 6000, 1.0)])
    tq = torch.from_numpy(train_q).to(dev)
    nn_rows, _ = P.paris_exact_knn_ex(idx, tq, 1, precision=P.PARIS_REFINE_MIXED)
    labels = P.paris_row_buckets(idx, nn_rows.cpu().numpy()[:, 0])
    _, _, paa = P.paris_encode(tq, 16, 256, want_paa=True)
    md = P.SeedModel(7)
    losses = md.train(paa, torch.from_numpy(labels).to(dev), batch=256, epochs=30, lr=3e-3, order_seed=3)
    assert losses[-1] < losses[0] * 0.8

    held_np = make(50, 400, 1.0)
    held = torch.from_numpy(held_np).to(dev)
    true_sq = oknn.knn(x, held_np, 1)[1][:, 0] ** 2
    _, plain = P.paris_approx_search(idx, held, 1, P.PARIS_SEED_DESCENT)
    plain = plain.cpu().numpy()
    untrained = P.SeedModel(7)                            # same initial weights, no training
    P.paris_attach_seed_model(idx, untrained, 3)
    _, rnd = P.paris_approx_search(idx, held, 1, P.PARIS_SEED_LEARNED)
    P.paris_attach_seed_model(idx, md, 3)
    _, learned = P.paris_approx_search(idx, held, 1, P.PARIS_SEED_LEARNED)
    rnd, learned = rnd.cpu().numpy(), learned.cpu().numpy()
    assert np.all(learned <= plain) and np.all(rnd <= plain)   # extra leaves only tighten the seed
    # seed looseness (seed / true squared distance, >= 1): the trained network beats both the
    # plain descent and an untrained network that adds the same number of leaves
    loose_plain = float(np.mean(plain / true_sq))
    loose_rnd = float(np.mean(rnd / true_sq))
    loose_learned = float(np.mean(learned / true_sq))
    assert loose_learned < loose_rnd < loose_plain + 1e-6, (loose_learned, loose_rnd, loose_plain)
    exact_plain = np.mean(plain <= true_sq * (1 + 1e-5))
    exact_learned = np.mean(learned <= true_sq * (1 + 1e-5))
    assert exact_learned > exact_plain
    untrained.free()
    # answers stay exact with the learned seed
    gi, gd = P.paris_exact_knn_ex(idx, held[:40], 1, seed=P.PARIS_SEED_LEARNED)[:2]
    wi, wd = oknn.knn(x, held[:40].cpu().numpy(), 1)
    assert np.array_equal(gi.cpu().numpy(), wi)
    md.free()
    idx.free()
