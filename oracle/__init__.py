"""CPU oracle for the ParIS+ hot path — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct restatements of what the GPU library computes, written from
the paper (Peng, Fatourou, Palpanas, "ParIS+: Data Series Indexing on Multi-Core
Architectures"). Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import this package; the library never does, and this package never imports the
library. Shared with the GPU side: nothing but the seeded input generator (``synth``).

Modules
  isax   -- breakpoints, PAA, iSAX symbols, the interleaved key, MINDIST (Sec. 2.2, 3.3.1)
  knn    -- exact k-NN by brute force with exact integer re-ranking of near ties (Sec. 2.1)
  index  -- sorted-key order, approximate-search leaf and seed (Sec. 3.3), LB candidate set
            (Alg. 8), page envelopes and their box MINDIST (leaf pruning), the full exact
            search driver (Alg. 7)
  mlp    -- the learned best-so-far proposal network (forward, backward, AdamW), FP64

Parity pinning: every function is checked by ``tests/test_oracle_*.py`` against values fixed by
the paper or by mathematics (hand-computed words, closed forms, invariants such as
MINDIST <= ED, brute force on tiny inputs, finite differences).
"""
