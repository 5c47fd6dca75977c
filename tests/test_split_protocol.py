"""The split kernel's barrier protocol, replayed on the host under random
schedules (tests/split_protocol.py): no deadlock, no phase aliasing and no
reuse race for random unit sequences (one or many exact windows per unit,
mixed leaf sizes), in both kernel configurations, and for the kernel of
one-pair C leaves; each planted protocol mistake is caught."""

from __future__ import annotations

import random

import pytest

from tests import split_protocol as sp


def _units(seed: int, sizes, windows):
    rng = random.Random(seed)
    out = []
    for _ in range(rng.randint(1, 9)):
        b = rng.choice(sizes)
        w = windows[b]
        out.append((b, rng.choice([1, 2, w - 1, w, w + 1, 2 * w, 3 * w + 1,
                                   rng.randint(1, 3 * w + 2)])))
    return out


CASES = {
    "kernel64_b64": (sp.KERNEL_64, (64,)),
    "kernel64_mixed": (sp.KERNEL_64, (64, 32)),
    "kernel32": (sp.KERNEL_32, (32,)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_protocol_holds_under_random_schedules(case):
    cfg, sizes = CASES[case]
    for seed in range(60):
        sp.run(cfg, _units(seed, sizes, cfg.windows), seed)


def test_protocol_with_no_units_and_one_pair():
    for cfg, sizes in CASES.values():
        sp.run(cfg, [], 0)
        sp.run(cfg, [(sizes[0], 1)], 1)


MISTAKES = {
    # the MMA restarts the exact regions without the epilogue's release
    "mma_skips_window_wait": ("kernel64_b64", 8),
    # the MMA starts a unit while the previous unit's data is unread
    "mma_skips_unit_wait": ("kernel64_b64", 8),
    # the epilogue releases TMEM before it has read the low region
    "epi_releases_before_low_read": ("kernel64_b64", 8),
    # a single exchange buffer without the barrier after the reads
    "no_second_exchange_barrier": ("kernel64_b64", 8),
    # the producer refills a stage the MMAs may still read
    "producer_skips_empty_wait": ("kernel32", 32),
    # the epilogue reads one accumulator set while the MMA alternates two
    "epi_single_accumulator_set": ("kernel32", 32),
}


@pytest.mark.parametrize("mistake", list(MISTAKES))
def test_planted_protocol_mistakes_are_caught(mistake):
    case, w = MISTAKES[mistake]
    cfg, sizes = CASES[case]
    units = [(sizes[0], n) for n in (1, 2 * w + 3, 1, w, 3, 1, 2 * w, 1)]
    caught = 0
    for seed in range(300):
        try:
            sp.run(cfg, units, seed, mistakes=frozenset([mistake]))
        except sp.ProtocolError:
            caught += 1
    assert caught > 0, mistake


@pytest.mark.parametrize("case", list(CASES))
def test_timeouts_end_cleanly(case):
    # one role's wait runs out of time at a random point: the abort reaches
    # every role, the status word records it, and no copy or MMA is left in
    # flight when the roles end
    cfg, sizes = CASES[case]
    rng = random.Random(11)
    aborted = 0
    for seed in range(80):
        units = _units(seed, sizes, cfg.windows)
        role = rng.choice(["producer", "mma", "epi0", "epi5"])
        st = sp.run(cfg, units, seed, timeout=(role, rng.randint(0, 12)))
        if st.abort:
            aborted += 1
            assert st.status_timeout
    assert aborted >= 20


@pytest.mark.parametrize("mistake", ["producer_no_drain", "mma_no_drain"])
def test_missing_drain_is_caught(mistake):
    cfg, sizes = CASES["kernel64_b64"]
    units = [(64, n) for n in (20, 3, 17, 1, 9)]
    caught = 0
    for seed in range(200):
        role = ("mma", "producer", "epi2")[seed % 3]
        try:
            sp.run(cfg, units, seed, mistakes=frozenset([mistake]), timeout=(role, seed % 7))
        except sp.ProtocolError:
            caught += 1
    assert caught > 0


# ---------------------------------------------- the one-pair C leaf kernel --

def _groups(seed: int):
    rng = random.Random(seed)
    return [rng.randint(1, 4) for _ in range(rng.randint(0, 11))]


def test_one_pair_protocol_holds_under_random_schedules():
    for seed in range(120):
        sp.run(sp.ONE_PAIR, _groups(seed), seed)


@pytest.mark.parametrize("mistake", ["mma_skips_unit_wait", "epi_releases_before_last_region",
                                     "producer_skips_empty_wait", "epi_skips_slot_release",
                                     "epi_single_accumulator_set", "producer_one_lane_short",
                                     "producer_single_end_slot"])
def test_one_pair_planted_mistakes_are_caught(mistake):
    groups = [4, 1, 3, 4, 2, 4, 4, 1, 4]
    caught = 0
    for seed in range(300):
        try:
            sp.run(sp.ONE_PAIR, groups, seed, mistakes=frozenset([mistake]))
        except sp.ProtocolError:
            caught += 1
    assert caught > 0, mistake


def test_one_pair_timeouts_end_cleanly():
    rng = random.Random(12)
    aborted = 0
    for seed in range(80):
        role = rng.choice(["producer", "mma", "epi0", "epi6"])
        st = sp.run(sp.ONE_PAIR, _groups(seed) + [4, 4, 4], seed,
                    timeout=(role, rng.randint(0, 10)))
        if st.abort:
            aborted += 1
            assert st.status_timeout
    assert aborted >= 20


@pytest.mark.parametrize("mistake", ["producer_no_drain", "mma_no_drain"])
def test_one_pair_missing_drain_is_caught(mistake):
    caught = 0
    for seed in range(200):
        role = ("mma", "producer", "epi2")[seed % 3]
        try:
            sp.run(sp.ONE_PAIR, [4, 3, 4, 4, 2, 4], seed, mistakes=frozenset([mistake]),
                   timeout=(role, seed % 7))
        except sp.ProtocolError:
            caught += 1
    assert caught > 0
