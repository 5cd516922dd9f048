"""The combining policy (Section 3.1 adaptive rule, Section 4.3 static
baseline) on scripted arrival traces with a fake clock, and the occupancy
arithmetic of Section 4.3.  Host-only: the library loads without a GPU."""
import json
import os

import pytest

from paper_2008_05712_gb300 import gcharm as g

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "combining_occupancy.json")


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2008_05712_gb300 import build
    build.build()
    g.load()


def test_occupancy_golden():
    d = json.load(open(GOLDEN))
    for c in d["cases"]:
        assert g.combine_size_from_occupancy(c["occupancy"], d["max_blocks_per_sm"],
                                             d["n_sm"]) == c["max_size"]


def test_adaptive_interval_rule_boundaries():
    c = g.Combiner(g.GC_COMBINE_ADAPTIVE, max_size=4)
    for t in (0, 10, 30):                 # intervals 10, 20 -> maxInterval 20
        c.arrive(t)
    assert c.max_interval() == 20
    assert c.poll(60, 3) == 0             # idle 30 <= 40
    assert c.poll(70, 3) == 0             # idle 40 == 2 x maxInterval: not greater
    assert c.poll(71, 3) == 3             # idle 41 > 40: combine all pending


def test_adaptive_occupancy_rule():
    c = g.Combiner(g.GC_COMBINE_ADAPTIVE, max_size=4)
    for t in range(6):
        c.arrive(t)
    assert c.poll(5, 4) == 4              # count == maxSize: combine now
    assert c.poll(5, 6) == 4              # more than maxSize: maxSize, rest stays
    assert c.poll(5, 2) == 0              # fewer, no idle gap yet
    assert c.poll(5, 0) == 0


def test_running_max_never_decays_window_does():
    a = g.Combiner(g.GC_COMBINE_ADAPTIVE, max_size=100)
    w = g.Combiner(g.GC_COMBINE_ADAPTIVE_WINDOW, max_size=100, window=3)
    t = 0
    a.arrive(t)
    w.arrive(t)
    for gap in [1000] + [5] * 10:
        t += gap
        a.arrive(t)
        w.arrive(t)
    assert a.max_interval() == 1000       # one long gap inflates the timeout for good
    assert w.max_interval() == 5          # the window has forgotten it
    assert a.poll(t + 11, 1) == 0
    assert w.poll(t + 11, 1) == 1


def test_first_arrival_and_simultaneous_arrivals():
    c = g.Combiner(g.GC_COMBINE_ADAPTIVE, max_size=10)
    c.arrive(100, count=3)                # three at once: intervals 0
    assert c.max_interval() == 0
    assert c.poll(100, 3) == 0            # no time has passed
    assert c.poll(101, 3) == 3


def test_static_every_n():
    d = json.load(open(GOLDEN))
    n = d["static_n"]
    c = g.Combiner(g.GC_COMBINE_STATIC, static_n=n)
    for i in range(n - 1):
        c.arrive(i)
    assert c.poll(10 ** 9, n - 1) == 0    # no timeout in the static rule
    c.arrive(n)
    assert c.poll(n, n) == n
    c.arrive(n + 1)
    assert c.poll(n + 1, 1) == 0          # counter restarted


def test_per_task_and_bad_arguments():
    c = g.Combiner(g.GC_COMBINE_PER_TASK)
    assert c.poll(0, 5) == 1 and c.poll(0, 0) == 0
    for args in [(g.GC_COMBINE_ADAPTIVE, 0, 0, 0), (g.GC_COMBINE_STATIC, 4, 0, 0),
                 (g.GC_COMBINE_ADAPTIVE_WINDOW, 4, 0, 0), (7, 1, 1, 1)]:
        with pytest.raises(g.GcError):
            g.Combiner(*args)


def test_greedy_takes_everything_pending():
    c = g.Combiner(g.GC_COMBINE_GREEDY, max_size=5)
    assert c.poll(0, 0) == 0
    assert c.poll(0, 3) == 3              # no waiting: all pending
    assert c.poll(0, 12) == 12            # not capped: batches grow with the queue
    assert g.Combiner(g.GC_COMBINE_GREEDY, max_size=0).poll(0, 7) == 7


def test_windowed_max_is_the_max_of_the_last_gaps():
    """The windowed rule's maxInterval equals the largest of the last
    `window` arrival gaps (checked against a direct maximum on a random
    arrival stream)."""
    import numpy as np
    rng = np.random.default_rng(5)
    t = np.cumsum(rng.integers(1, 1000, 3000)).astype(np.uint64)
    for window in (1, 3, 64):
        c = g.Combiner(g.GC_COMBINE_ADAPTIVE_WINDOW, max_size=10, window=window)
        for k, tk in enumerate(t):
            c.arrive(int(tk))
            if k >= 1:
                gaps = np.diff(t[:k + 1].astype(np.int64))
                assert c.max_interval() == int(gaps[-window:].max()), (window, k)


def test_adaptive_rule_under_poisson_arrivals_waits_for_max_size():
    """With Poisson arrivals the idle timeout 2 x maxInterval (running max of
    the gaps) almost never expires between arrivals, so the adaptive rule
    combines at maxSize; the greedy rule combines at every poll."""
    import numpy as np
    from paper_2008_05712_gb300 import inputs
    arr = inputs.poisson_arrivals(4000, 1e4, 3)
    for policy, window in [(g.GC_COMBINE_ADAPTIVE, 0), (g.GC_COMBINE_ADAPTIVE_WINDOW, 256)]:
        c = g.Combiner(policy, max_size=64, window=window)
        queued, sizes = 0, []
        for k, t in enumerate(arr):
            c.arrive(int(t))
            queued += 1
            # poll just before the next arrival (the longest the queue can idle)
            t_poll = int(arr[k + 1]) - 1 if k + 1 < len(arr) else int(t) + 10 ** 9
            take = c.poll(t_poll, queued)
            if take:
                sizes.append(take)
                queued -= take
        sizes = np.array(sizes)
        assert (sizes[:-1] == 64).mean() > 0.95, np.bincount(sizes)
