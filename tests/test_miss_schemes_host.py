"""Host check of the two miss-update schemes of the filtered walk (Sec. III-C
phase one, the clamped log-odds update of Eq. 2 with the clamp of Sec. II-B).

Within one integrate call every miss of a voxel adds the same increment
delta < 0, and readers take max(stored, l_min).  The walk kernels apply the
misses of concurrent threads as atomics in any order:

- waited CAS (single-map walk): a thread that loaded an unknown (NaN) voxel
  swaps NaN for fl(0 + delta); if the swap lost, it adds delta to the value it
  found when that is above l_min;
- unchecked CAS + add (multi-map batch walk): a thread that loaded NaN swaps
  NaN for the prior 0 without looking at the result, then adds delta;

and in both, a thread that loaded a known value adds delta when the value is
above l_min and does nothing otherwise.  Loads may be stale: they happen at
any point before the thread's own atomics.

These tests replay random interleavings of such threads in float32 (IEEE
round to nearest, as the device's float atomics) and require the value read
back to equal, bit for bit, k sequential clamped updates from the voxel's
state at the start of the call (0 for an unknown voxel).
"""
import numpy as np
import pytest

F32 = np.float32
NAN_BITS = np.uint32(0xFFFFFFFF)


def _f(bits):
    return np.array([bits], dtype=np.uint32).view(np.float32)[0]


def _bits(x):
    return np.array([x], dtype=np.float32).view(np.uint32)[0]


def sequential(start, k, delta, l_min, l_max):
    """k one-at-a-time clamped updates l <- min(max(l + delta, l_min), l_max)."""
    l = F32(0.0) if np.isnan(start) else max(F32(start), l_min)
    for _ in range(k):
        l = min(max(F32(l + delta), l_min), l_max)
    return l


def replay(start_bits, k, delta, l_min, scheme, rng):
    """One voxel, k threads each with one miss, in a random interleaving.

    Each thread loads the word at a random point before its own atomics;
    the atomics of all threads interleave at random, each thread's in
    program order.  Returns the stored word at the end."""
    word = start_bits
    # per thread: a list of pending steps; step 0 is the load
    pending = [["load"] for _ in range(k)]
    loaded = [None] * k
    cas_result = [None] * k
    active = list(range(k))
    miss0 = _bits(F32(F32(0.0) + delta))
    while active:
        t = active[rng.integers(len(active))]
        step = pending[t].pop(0)
        if step == "load":
            loaded[t] = word
            l = _f(word)
            if np.isnan(l):
                pending[t] = ["cas_init"] if scheme == "unchecked" else ["cas_wait"]
                if scheme == "unchecked":
                    pending[t].append("add")
            elif l > l_min:
                pending[t] = ["add"]
            else:
                pending[t] = []
        elif step == "cas_init":  # NaN -> prior 0, result not looked at
            if word == loaded[t]:
                word = _bits(F32(0.0))
        elif step == "cas_wait":  # NaN -> fl(0 + delta); a loser adds to what it found
            prev = word
            if word == loaded[t]:
                word = miss0
            cas_result[t] = prev
            if prev != loaded[t] and _f(prev) > l_min:
                pending[t] = ["add"]
        elif step == "add":
            word = _bits(F32(_f(word) + delta))
        if not pending[t]:
            active.remove(t)
    return word


@pytest.mark.parametrize("scheme", ["waited", "unchecked"])
def test_any_interleaving_gives_the_sequential_clamped_updates(scheme):
    rng = np.random.default_rng(0x0A1B)
    for case in range(3000):
        delta = F32(-rng.uniform(0.05, 1.0))
        l_min = F32(-rng.uniform(0.5, 4.0))
        l_max = F32(rng.uniform(0.5, 4.0))
        kind = rng.integers(4)
        if kind == 0:
            start = F32(np.nan)
        elif kind == 1:  # known, above the lower clamp
            start = F32(rng.uniform(float(l_min), float(l_max)))
        elif kind == 2:  # stored at or below l_min (earlier adds went past it)
            start = F32(l_min - F32(rng.uniform(0.0, 3.0)))
        else:  # just above l_min: the first miss crosses it
            start = F32(l_min + F32(rng.uniform(0.0, 1.0)) * (-delta))
        start_bits = NAN_BITS if np.isnan(start) else _bits(start)
        k = int(rng.integers(1, 12))
        got = replay(start_bits, k, delta, l_min, scheme, rng)
        read = _f(got)
        assert not np.isnan(read), (case, scheme)
        read = max(read, l_min)
        want = sequential(start, k, delta, l_min, l_max)
        assert _bits(read) == _bits(want), (case, scheme, float(start), k, float(delta), float(l_min))


def test_unchecked_scheme_stores_the_prior_sequence_for_unknown_voxels():
    """An unknown voxel missed k times, with every thread's load before any
    atomic (the case where each of them sees NaN): the stored value is the
    k-th float of 0, fl(0 + delta), ... whichever thread's swap lands first."""
    rng = np.random.default_rng(7)
    delta, l_min = F32(-0.4054651), F32(-2.0)
    for k in range(1, 9):
        want = F32(0.0)
        for _ in range(k):
            want = F32(want + delta)
        # all loads first, then a random order of the swaps and adds
        word = NAN_BITS
        ops = [(t, s) for t in range(k) for s in ("cas", "add")]
        order = rng.permutation(len(ops))
        done_cas = set()
        queue = [ops[i] for i in order]
        while queue:
            for idx, (t, s) in enumerate(queue):
                if s == "add" and t not in done_cas:
                    continue  # a thread's add follows its own swap
                queue.pop(idx)
                if s == "cas":
                    if word == NAN_BITS:
                        word = _bits(F32(0.0))
                    done_cas.add(t)
                else:
                    word = _bits(F32(_f(word) + delta))
                break
        assert _bits(_f(word)) == _bits(want), k
        assert _bits(max(_f(word), l_min)) == _bits(sequential(F32(np.nan), k, delta, l_min, F32(3.5)))
