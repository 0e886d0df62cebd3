"""Bookkeeping of the class-split filter's pass 1, modelled for one warp: per
column step every lane may append one key to its class; before the step,
every class with more than 16 staged entries moves its first 16 to the
class list (the rest move down); at the end every class is drained, its
last entries padded to 16 with an impossible key.  The model checks the
invariants the kernel's indexing relies on -- a staged slot is always below
the 48-entry buffer, a flush moves at most 32 entries down, every key
reaches its class list exactly once, and every list grows by whole groups
of 16 -- for random classes and for the worst cases (all 32 lanes on one
class for many steps, all classes at once, ragged last words).
"""
import numpy as np

BUF, GROUP, NONE = 48, 16, -1


def _run_warp(classes):
    """classes: steps x 32 array of class ids (0..15), -1 for no key."""
    staged = [[] for _ in range(16)]
    lists = [[] for _ in range(16)]
    expected = [[] for _ in range(16)]
    key = 0
    for step in classes:
        # room for this step's appends: no class above 16 staged
        while True:
            full = [q for q in range(16) if len(staged[q]) > GROUP]
            if not full:
                break
            for q in full:
                cnt = len(staged[q])
                assert cnt - GROUP <= 32              # entries moved down by the 32 lanes
                lists[q].extend(staged[q][:GROUP])
                staged[q] = staged[q][GROUP:]
        for q in step:
            if q < 0:
                continue
            slot = len(staged[q])
            assert slot < BUF                         # the staged slot stays inside the buffer
            staged[q].append(key)
            expected[q].append(key)
            key += 1
    for q in range(16):
        while len(staged[q]) >= GROUP:
            lists[q].extend(staged[q][:GROUP])
            staged[q] = staged[q][GROUP:]
        if staged[q]:
            pad = GROUP - len(staged[q])
            assert 0 < pad < GROUP
            lists[q].extend(staged[q] + [NONE] * pad)
            staged[q] = []
    for q in range(16):
        assert len(lists[q]) % GROUP == 0
        got = [k for k in lists[q] if k != NONE]
        assert got == expected[q]                     # every key once, in order
    return lists


def test_staging_random_classes():
    rng = np.random.default_rng(1)
    for steps in (1, 7, 40):
        for _ in range(20):
            cls = rng.integers(0, 16, size=(steps * 32, 32))
            cls[rng.random(cls.shape) < 0.05] = -1    # ragged words: lanes without a key
            _run_warp(cls)


def test_staging_worst_cases():
    # every lane on one class, step after step (the buffer fills to 48)
    _run_warp(np.full((200, 32), 3))
    # classes cycling so that all 16 fill at once
    _run_warp(np.tile(np.arange(32) % 16, (300, 1)))
    # two lanes per class except one class taking half the warp
    row = np.concatenate([np.arange(16), np.full(16, 9)])
    _run_warp(np.tile(row, (150, 1)))
    # nothing at all, and a single key
    _run_warp(np.full((5, 32), -1))
    one = np.full((1, 32), -1)
    one[0, 7] = 12
    lists = _run_warp(one)
    assert lists[12] == [0] + [NONE] * 15
