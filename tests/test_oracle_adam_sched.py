"""Pins of the oracle's Adam step (against torch.optim.Adam in float64) and of the
adaptive keyframe scheduler, Eqs. 5-8 (invariants, a worked example and brute-force
enumeration on small pools).  CPU only."""
import itertools

import numpy as np
import pytest
import torch

from oracle import oracle as O


def test_adam_matches_torch_float64():
    rng = np.random.default_rng(0)
    n, deg = 7, 1
    lr6 = (1e-3, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 1.25e-4)
    lr = O.lr_per_element(n, deg, lr6)
    theta = rng.normal(size=lr.size)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    sizes = [3 * n, 3 * n, 4 * n, n, 3 * n, 9 * n]
    chunks = np.split(torch.tensor(theta.copy()), np.cumsum(sizes)[:-1])
    tparams = [torch.nn.Parameter(c.clone()) for c in chunks]
    opt = torch.optim.Adam([{"params": [p], "lr": l} for p, l in zip(tparams, lr6)],
                           betas=(0.9, 0.999), eps=1e-15)
    for step in range(1, 6):
        g = rng.normal(size=theta.size)
        g[::5] = 0.0                      # zero-grad elements still move by momentum
        theta, m, v = O.adam(theta, g, m, v, step, lr)
        for p, gc in zip(tparams, np.split(g, np.cumsum(sizes)[:-1])):
            p.grad = torch.tensor(gc)
        opt.step()
        ref = torch.cat([p.detach() for p in tparams]).numpy()
        np.testing.assert_allclose(theta, ref, rtol=1e-12, atol=1e-15)


def test_scheduler_worked_refill():
    # pool of 4, d = 4 -> d_k = max(1, 4 // 4) = 1: the largest loss gets r = 2
    s = O.Scheduler(d=4)
    for k in range(4):
        s.add(k, 1)
    for loss_i, i in zip([0.3, 0.9, 0.1, 0.5], range(4)):
        j = s.draw(0)            # draws the lowest eligible index each time
        assert j == i
        s.report(j, loss_i)
    assert s.R == [0, 0, 0, 0]
    s.draw(0)
    assert s.R == [0, 2, 1, 1]   # refilled [1, 2, 1, 1], then index 0 drawn


def test_scheduler_refill_ties_and_dk():
    s = O.Scheduler(d=4)
    for k in range(9):
        s.add(k, 1)
        s.L[k] = [5, 1, 5, 2, 5, 0, 3, 3, 1][k]
    s.R = [0] * 9
    s._refill()
    # d_k = max(1, floor(9/4)) = 2: top-2 losses are the 5s at indices 0 and 2 (lower index wins)
    assert s.R == [2, 1, 2, 1, 1, 1, 1, 1, 1]
    assert sum(s.R) == 9 + 2


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_scheduler_brute_force_cycles(k):
    # every sequence of draw choices: within one refill cycle each keyframe is drawn
    # exactly r_i times, and the r = 2 set is the top-d_k losses
    losses = [0.7, 0.2, 0.9, 0.4][:k]
    for d in (1, 2, 4):
        dk = max(1, k // d)
        for rand in itertools.product(range(k), repeat=min(2 * k + 1, 7)):
            s = O.Scheduler(d=d)
            for i in range(k):
                s.add(i, 1)
            counts = [0] * k
            for i in range(k):                    # initial r0 = 1 each
                j = s.draw(rand[i % len(rand)])
                s.report(j, losses[j])
                counts[j] += 1
            assert counts == [1] * k
            cyc = [0] * k
            total = k + dk
            for t in range(total):
                j = s.draw(rand[t % len(rand)])
                cyc[j] += 1
            top = sorted(range(k), key=lambda i: (-losses[i], i))[:dk]
            assert cyc == [2 if i in top else 1 for i in range(k)]
            assert sum(s.R) == 0


def test_scheduler_new_keyframe_trained_before_refill():
    s = O.Scheduler(d=4)
    s.add(0, 2)
    s.draw(0)
    s.report(0, 1.0)
    s.add(1, 8)                               # Replica-like r0 = 8
    drawn = [s.draw(r) for r in range(9)]
    assert drawn.count(1) == 8 and drawn.count(0) == 1
