"""The learned best-so-far proposal on the GPU: forward pass and gradients against the FP64
oracle (same BF16-representable weights; the GPU rounds GEMM operands to BF16 and accumulates
in FP32), the uniform-logit closed form, training, and what the trained network gains over the
plain approximate search (a tighter seed, never a looser one) at unchanged exact answers."""
import math

import numpy as np
import pytest

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


def bf16_params(seed, scale):
    rng = np.random.default_rng(seed)
    return {k: bf16_round(rng.standard_normal(s) * scale / math.sqrt(s[-1])) for k, s in mlp.SHAPES.items()}


def paa_inputs(m, seed):
    return np.random.default_rng(seed).standard_normal((m, 16)) * 0.8


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_matches_oracle():
    import paper_2009_00166_gb300 as P
    require_gpu()
    p = bf16_params(1, 1.0)
    x = paa_inputs(200, 2)
    md = P.SeedModel(0)
    md.set_weights(p)
    got = md.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = mlp.forward({k: v.astype(np.float64) for k, v in p.items()}, x.astype(np.float32).astype(np.float64))
    assert rel(got, want) < 1.5e-2
    md.free()


def test_gradients_match_oracle():
    import paper_2009_00166_gb300 as P
    require_gpu()
    p = bf16_params(3, 1.5)
    x = paa_inputs(96, 4)
    y = np.random.default_rng(5).integers(0, 4096, 96).astype(np.int32)
    md = P.SeedModel(0)
    md.set_weights(p)
    loss, g = md.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    wl, wg = mlp.loss_and_grads({k: v.astype(np.float64) for k, v in p.items()}, x.astype(np.float32), y)
    assert abs(loss - wl) < 1e-3 * wl
    for k in mlp.ORDER:
        a, b = g[k].ravel().astype(np.float64), wg[k].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert cos > 0.999, (k, cos)
        assert rel(a, b) < 3e-2, (k, rel(a, b))
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
