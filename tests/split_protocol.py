"""Host-side model of the split kernel's synchronisation protocol (test
infrastructure; no GPU).

One CTA of ``k_split_gemm`` runs three roles that talk only through
mbarriers: the producer warp (unit queue slots and operand stages), the MMA
thread (slice MMAs into TMEM accumulator regions) and eight epilogue warps
(exact-window reads, the final read, the exchange buffer).  This module
replays that protocol with every wait, arrival, copy completion and MMA
completion as a separate step under a random scheduler, and checks:

- no deadlock: until every role has finished, some step can run;
- no phase aliasing: when a parity wait passes, the barrier has completed
  exactly the phase the waiter meant (a waiter a full phase behind would
  pass or block on the wrong phase);
- no reuse race: an operand stage is not refilled while MMAs still read it;
  a TMEM region is not restarted while an epilogue warp has still to read
  its previous data, nor read while MMAs on it are in flight; a queue slot
  is not rewritten while a role still uses it; an exchange buffer is not
  rewritten while a warp still reads it;
- a clean exit: when the roles end (the CTA then frees TMEM and its shared
  memory) no copy and no MMA is in flight, also after a wait ran out of time.

``kernel_roles`` mirrors the kernel's producer loop, ``mma_unit``,
``epi_unit`` and their exits: the same barriers, arrival counts, parities and
hand-off order (exact regions 0 and 1 restart every window of 8 [32] pairs;
the low region 2 accumulates over the unit and is read once; from the second
window of a unit on, the first pair's region-2 MMAs go out before the wait
for the epilogue's release).  A wait that gives up (its budget ran out, or
another role set the abort flag) returns False, as ``wait_or_abort`` does;
the producer then waits for its copies in flight and the MMA thread for its
MMAs (bounded drain waits that ignore the flag).  ``mistakes`` plants one
protocol error at a time so that the tests can show the checks catch it.
"""

from __future__ import annotations

import random
from dataclasses import dataclass, field

QUEUE = 4        # unit queue slots
EPI_WARPS = 8    # epilogue warps of the general kernel
EPI_WARPS_ONE_PAIR = 16  # epilogue warps of the one-pair kernel (four per lane quarter)
LANES = 32       # producer lanes (one cp.async arrival each per stage fill)
REGIONS = 3      # TMEM regions per accumulator set


class ProtocolError(AssertionError):
    pass


class Barrier:
    """An mbarrier: expected arrivals per phase, a transaction byte count and
    the number of completed phases (whose low bit is the phase parity)."""

    def __init__(self, name: str, count: int):
        self.name, self.count = name, count
        self.pending, self.tx, self.completed = count, 0, 0

    def arrive(self, expect_tx: int = 0):
        self.tx += expect_tx
        self.pending -= 1
        if self.pending < 0:
            raise ProtocolError(f"{self.name}: more arrivals than expected in one phase")
        self._maybe_complete()

    def complete_tx(self, nbytes: int):
        self.tx -= nbytes
        self._maybe_complete()

    def _maybe_complete(self):
        if self.pending == 0 and self.tx == 0:
            self.completed += 1
            self.pending = self.count

    def passes(self, phase: int) -> bool:
        """try_wait.parity(phase & 1)."""
        return (self.completed & 1) != (phase & 1)


@dataclass
class Config:
    nb: int        # TMEM accumulator sets (2 in the 32-leaf kernel)
    nxb: int       # exchange buffers (2 in the 32-leaf kernel)
    stages: int    # operand stages
    windows: dict  # pairs per exact window, by leaf size
    kind: str = "general"  # "one_pair": the kernel of one-pair C leaves
    teams: int = 1  # one-pair kernel: epilogue teams taking alternate groups


# the kernel taking 64-leaves (and 32-leaf units of mixed batches), and the
# 32-leaf-only kernel
KERNEL_64 = Config(nb=1, nxb=1, stages=2, windows={64: 8, 32: 32})
KERNEL_32 = Config(nb=2, nxb=2, stages=4, windows={32: 32})
# k_split_single32: groups of up to 4 one-pair C leaves sharing a B leaf; two
# accumulator sets of 6 regions (group n uses set n % 2), each read whole and
# released by every epilogue warp before it stores; no exchange buffer
ONE_PAIR = Config(nb=2, nxb=0, stages=3, windows={}, kind="one_pair", teams=2)
ONE_PAIR_REGIONS = 6


@dataclass
class State:
    cfg: Config
    bars: dict = field(default_factory=dict)
    stage_busy: dict = field(default_factory=dict)     # stage -> pair still read by MMAs
    readers: dict = field(default_factory=dict)        # (set, region) -> (tag, warps to read)
    slot_readers: dict = field(default_factory=dict)   # slot -> roles still using it
    xb_use: dict = field(default_factory=dict)         # buffer -> (unit, warps still reading)
    inflight: list = field(default_factory=list)       # issued MMAs and commits, in order
    copies: list = field(default_factory=list)         # (barrier, bytes) in flight
    abort: bool = False                                # the kernel's abort flag
    status_timeout: bool = False                       # the device status word


def kernel_roles(st: State, units, mistakes=frozenset()):
    """Generators for the producer, the MMA thread and the eight epilogue
    warps.  ``units`` is the list of (leaf size, pairs) this CTA takes.  A
    generator yields ("wait", barrier, phase, abortable) and receives True
    (the phase completed) or False (it gave up), or yields None (one plain
    step)."""
    cfg = st.cfg
    S = cfg.stages
    bars = st.bars
    for i in range(S):
        bars[f"full{i}"] = Barrier(f"full{i}", 1)
        bars[f"empty{i}"] = Barrier(f"empty{i}", 1)
    for i in range(QUEUE):
        bars[f"qfull{i}"] = Barrier(f"qfull{i}", 1)
        bars[f"qempty{i}"] = Barrier(f"qempty{i}", 1 + EPI_WARPS)
    for i in range(cfg.nb):
        bars[f"acc_full{i}"] = Barrier(f"acc_full{i}", 1)
        bars[f"acc_empty{i}"] = Barrier(f"acc_empty{i}", EPI_WARPS)
    bars["ep_bar"] = Barrier("ep_bar", EPI_WARPS)
    bars["drain"] = Barrier("drain", 1)
    everyone = frozenset(["mma"] + [f"epi{w}" for w in range(EPI_WARPS)])
    warps = frozenset(f"epi{w}" for w in range(EPI_WARPS))
    slots = {}

    def wait(name, phase, abortable=True):
        return ("wait", bars[name], phase, abortable)

    def fail():
        st.status_timeout = True
        st.abort = True

    def producer():
        k = 0
        ok = True
        for n in range(len(units) + 1):
            qs = n % QUEUE
            if not (yield wait(f"qempty{qs}", n // QUEUE - 1)):
                fail()
                break
            if st.slot_readers.get(qs):
                raise ProtocolError(f"slot {qs} rewritten for unit {n} while "
                                    f"{sorted(st.slot_readers[qs])} still use it")
            b, np_ = units[n] if n < len(units) else (0, 0)
            slots[qs] = (b, np_, n)
            st.slot_readers[qs] = set(everyone)
            bars[f"qfull{qs}"].arrive()
            if b == 0:
                break
            yield None
            for _ in range(np_):
                s = k % S
                if "producer_skips_empty_wait" not in mistakes:
                    ok = yield wait(f"empty{s}", k // S - 1)
                    if not ok:
                        fail()
                        break
                if s in st.stage_busy:
                    raise ProtocolError(f"stage {s} refilled for pair {k} while MMAs of "
                                        f"pair {st.stage_busy[s]} still read it")
                st.stage_busy[s] = k
                bars[f"full{s}"].arrive(expect_tx=2)
                st.copies.extend([(bars[f"full{s}"], 1), (bars[f"full{s}"], 1)])
                k += 1
                yield None
            if not ok:
                break
        # copies in flight land before shared memory goes away
        if "producer_no_drain" not in mistakes:
            for j in range(max(0, k - S), k):
                yield wait(f"full{j % S}", j // S, abortable=False)

    def issue(bf, region, tag, fresh):
        key = (bf, region)
        if fresh:
            old = st.readers.get(key)
            if old and old[1]:
                raise ProtocolError(f"TMEM set {bf} region {region} restarted for {tag} while "
                                    f"{sorted(old[1])} have not read {old[0]}")
            st.readers[key] = (tag, set(warps))
        st.inflight.append(("mma", key))

    def mma_unit(n, np_, W, bf, win, k):
        """One unit; returns (ok, pairs consumed)."""
        fresh = [True] * REGIONS
        for w0 in range(0, np_, W):
            ahead = w0 != 0
            if not ahead and "mma_skips_unit_wait" not in mistakes:
                if not (yield wait(f"acc_empty{bf}", win[bf] - 1)):
                    return False, k
            for i in range(w0, min(np_, w0 + W)):
                s = k % S
                if not (yield wait(f"full{s}", k // S)):
                    return False, k
                exact_tag, low_tag = (n, win[bf]), (n, "low")
                if i == w0 and ahead:
                    issue(bf, 2, low_tag, fresh[2])
                    fresh[2] = False
                    if "mma_skips_window_wait" not in mistakes:
                        if not (yield wait(f"acc_empty{bf}", win[bf] - 1)):
                            return False, k
                if i == w0:
                    fresh[0] = fresh[1] = True
                for r in range(REGIONS):
                    if r == 2 and i == w0 and ahead:
                        continue
                    issue(bf, r, exact_tag if r < 2 else low_tag, fresh[r])
                    fresh[r] = False
                st.inflight.append(("commit", bars[f"empty{s}"], k))
                k += 1
                yield None
            st.inflight.append(("commit", bars[f"acc_full{bf}"], None))
            win[bf] += 1
            yield None
        return True, k

    def mma():
        k = 0
        win = [0] * cfg.nb
        for n in range(len(units) + 1):
            qs = n % QUEUE
            if not (yield wait(f"qfull{qs}", n // QUEUE)):
                fail()
                break
            b, np_, _ = slots[qs]
            st.slot_readers[qs].discard("mma")
            if b == 0:
                break
            bars[f"qempty{qs}"].arrive()
            ok, k = yield from mma_unit(n, np_, cfg.windows[b], n % cfg.nb, win, k)
            if not ok:
                fail()
                break
        # in-flight MMAs finish before TMEM is released
        if "mma_no_drain" not in mistakes:
            st.inflight.append(("commit", bars["drain"], None))
            yield wait("drain", 0, abortable=False)

    def read(me, bf, region, tag):
        key = (bf, region)
        if any(op[0] == "mma" and op[1] == key for op in st.inflight):
            raise ProtocolError(f"{me} reads TMEM set {bf} region {region} ({tag}) while "
                                f"MMAs on it are in flight")
        cur = st.readers.get(key)
        if cur is None or cur[0] != tag or me not in cur[1]:
            raise ProtocolError(f"{me} expected {tag} in TMEM set {bf} region {region}, "
                                f"found {cur and cur[0]}")
        cur[1].discard(me)

    def epi_unit(me, n, qs, np_, W, bf, win, epb):
        """One unit; returns (ok, exchange barrier uses)."""
        for w0 in range(0, np_, W):
            last = w0 + W >= np_
            if not (yield wait(f"acc_full{bf}", win[bf])):
                return False, epb
            for r in (0, 1):
                read(me, bf, r, (n, win[bf]))
            if not last:
                bars[f"acc_empty{bf}"].arrive()
                win[bf] += 1
                yield None
                continue
            early = "epi_releases_before_low_read" in mistakes
            if early:
                bars[f"acc_empty{bf}"].arrive()
                yield None
            read(me, bf, 2, (n, "low"))
            if not early:
                bars[f"acc_empty{bf}"].arrive()
            win[bf] += 1
            yield None
        # the final conversion uses the slot's exponents and C pointer
        if slots[qs][2] != n:
            raise ProtocolError(f"{me}: slot {qs} of unit {n} was rewritten for unit "
                                f"{slots[qs][2]} while still in use")
        # exchange: write this warp's values, meet, read the others'
        xb = n % cfg.nxb
        use = st.xb_use.get(xb)
        if use and use[0] != n and use[1]:
            raise ProtocolError(f"exchange buffer {xb} rewritten by {me} for unit {n} "
                                f"while {sorted(use[1])} still read unit {use[0]}")
        if not use or use[0] != n:
            st.xb_use[xb] = (n, set(warps))
        bars["ep_bar"].arrive()
        if not (yield wait("ep_bar", epb)):
            return False, epb
        epb += 1
        yield None  # reads
        st.xb_use[xb][1].discard(me)
        return True, epb

    def epilogue(wid):
        me = f"epi{wid}"
        win = [0] * cfg.nb
        epb = 0
        for n in range(len(units) + 1):
            qs = n % QUEUE
            if not (yield wait(f"qfull{qs}", n // QUEUE)):
                fail()
                break
            b, np_, _ = slots[qs]
            if b == 0:
                st.slot_readers[qs].discard(me)
                break
            bf = 0 if "epi_single_accumulator_set" in mistakes else n % cfg.nb
            ok, epb = yield from epi_unit(me, n, qs, np_, cfg.windows[b], bf, win, epb)
            if not ok:
                fail()
                break
            if cfg.nxb == 1 and "no_second_exchange_barrier" not in mistakes:
                # one exchange buffer: every warp has read it before the next unit
                bars["ep_bar"].arrive()
                if not (yield wait("ep_bar", epb)):
                    fail()
                    break
                epb += 1
            st.slot_readers[qs].discard(me)
            bars[f"qempty{qs}"].arrive()
            yield None

    roles = {"producer": producer(), "mma": mma()}
    for wid in range(EPI_WARPS):
        roles[f"epi{wid}"] = epilogue(wid)
    return roles


def one_pair_roles(st: State, groups, mistakes=frozenset()):
    """Generators for the roles of k_split_single32 (same conventions as
    kernel_roles).  ``groups`` lists the units of each group this CTA takes
    (1..4); the protocol does not depend on them.  The 16 epilogue warps form
    ``cfg.teams`` teams (of 8 with two teams); team t takes the groups n with
    n % teams == t, and accumulator set n % 2 (with two teams: its own set).
    Per group: the producer stages the slot and one operand stage; the MMA
    thread waits for the release of the group before last (the previous user
    of the same accumulator set), then for the stage, and restarts that set's
    six regions; every warp of the group's team reads all six regions,
    releases the set, then stores (reading the slot) and frees the slot.
    After the last group the producer publishes one end slot per team, so
    that every team meets one."""
    cfg = st.cfg
    S = cfg.stages
    T = cfg.teams
    W = EPI_WARPS_ONE_PAIR // T  # warps per team
    bars = st.bars
    for i in range(S):
        # the B copy's expect_tx arrival and one cp.async arrival per lane
        bars[f"full{i}"] = Barrier(f"full{i}", 1 + LANES)
        bars[f"empty{i}"] = Barrier(f"empty{i}", 1)
    for i in range(QUEUE):
        bars[f"qfull{i}"] = Barrier(f"qfull{i}", 1)
        bars[f"qempty{i}"] = Barrier(f"qempty{i}", 1 + W)
    for bf in range(cfg.nb):
        bars[f"acc_full{bf}"] = Barrier(f"acc_full{bf}", 1)
        bars[f"acc_empty{bf}"] = Barrier(f"acc_empty{bf}", W)
    bars["drain"] = Barrier("drain", 1)
    team_of = {f"epi{w}": w // W for w in range(EPI_WARPS_ONE_PAIR)}
    team_warps = [frozenset(f"epi{w}" for w in range(t * W, (t + 1) * W)) for t in range(T)]
    slots = {}
    ngroups = len(groups)
    nb = cfg.nb
    ends = 1 if "producer_single_end_slot" in mistakes else T

    def wait(name, phase, abortable=True):
        return ("wait", bars[name], phase, abortable)

    def fail():
        st.status_timeout = True
        st.abort = True

    def producer():
        n = 0
        staged = 0
        for n in range(ngroups + ends):
            qs = n % QUEUE
            if not (yield wait(f"qempty{qs}", n // QUEUE - 1)):
                fail()
                break
            if st.slot_readers.get(qs):
                raise ProtocolError(f"slot {qs} rewritten for group {n} while "
                                    f"{sorted(st.slot_readers[qs])} still use it")
            count = groups[n] if n < ngroups else 0
            slots[qs] = (count, n)
            readers = set(team_warps[n % T])
            if n <= ngroups:
                readers.add("mma")  # the MMA thread stops at the first end slot
            st.slot_readers[qs] = readers
            bars[f"qfull{qs}"].arrive()
            if count == 0:
                continue
            yield None
            s = n % S
            if "producer_skips_empty_wait" not in mistakes:
                if not (yield wait(f"empty{s}", n // S - 1)):
                    fail()
                    break
            if s in st.stage_busy:
                raise ProtocolError(f"stage {s} refilled for group {n} while MMAs of "
                                    f"group {st.stage_busy[s]} still read it")
            st.stage_busy[s] = n
            # lane 0: the B leaf's bulk copy (expect_tx); every lane: its
            # 16-byte A copies, then an arrival that fires once they land
            bars[f"full{s}"].arrive(expect_tx=1)
            st.copies.append((bars[f"full{s}"], 1))
            lanes = LANES - 1 if "producer_one_lane_short" in mistakes else LANES
            st.copies.extend([(bars[f"full{s}"], None)] * lanes)
            staged = n + 1
            yield None
        if "producer_no_drain" not in mistakes:
            for j in range(max(0, staged - S), staged):
                yield wait(f"full{j % S}", j // S, abortable=False)

    def mma():
        for n in range(ngroups + 1):
            qs = n % QUEUE
            if not (yield wait(f"qfull{qs}", n // QUEUE)):
                fail()
                break
            count, _ = slots[qs]
            st.slot_readers[qs].discard("mma")
            if count == 0:
                break
            bars[f"qempty{qs}"].arrive()
            bf = n % nb
            if "mma_skips_unit_wait" not in mistakes:
                if not (yield wait(f"acc_empty{bf}", n // nb - 1)):
                    fail()
                    break
            s = n % S
            if not (yield wait(f"full{s}", n // S)):
                fail()
                break
            for r in range(ONE_PAIR_REGIONS):
                key = (bf, r)
                old = st.readers.get(key)
                if old and old[1]:
                    raise ProtocolError(f"region {r} restarted for group {n} while "
                                        f"{sorted(old[1])} have not read group {old[0]}")
                st.readers[key] = (n, set(team_warps[n % T]))
                st.inflight.append(("mma", key))
            st.inflight.append(("commit", bars[f"empty{s}"], n))
            st.inflight.append(("commit", bars[f"acc_full{bf}"], None))
            yield None
        if "mma_no_drain" not in mistakes:
            st.inflight.append(("commit", bars["drain"], None))
            yield wait("drain", 0, abortable=False)

    def epilogue(wid):
        me = f"epi{wid}"
        t = team_of[me]
        n = t
        while True:
            qs = n % QUEUE
            if not (yield wait(f"qfull{qs}", n // QUEUE)):
                fail()
                break
            count, _ = slots[qs]
            if count == 0:
                st.slot_readers[qs].discard(me)
                break
            bf = 0 if "epi_single_accumulator_set" in mistakes else n % nb
            if not (yield wait(f"acc_full{bf}", n // nb)):
                fail()
                break
            regions = range(ONE_PAIR_REGIONS)
            if "epi_releases_before_last_region" in mistakes:
                for r in range(ONE_PAIR_REGIONS - 1):
                    _read(st, me, (bf, r), n)
                bars[f"acc_empty{bf}"].arrive()
                yield None
                _read(st, me, (bf, ONE_PAIR_REGIONS - 1), n)
            else:
                for r in regions:
                    _read(st, me, (bf, r), n)
                bars[f"acc_empty{bf}"].arrive()
            yield None  # assemble and store, with the slot's pointers
            if slots[qs][1] != n:
                raise ProtocolError(f"{me}: slot {qs} of group {n} was rewritten for group "
                                    f"{slots[qs][1]} while still in use")
            st.slot_readers[qs].discard(me)
            if "epi_skips_slot_release" not in mistakes or wid != 3:
                bars[f"qempty{qs}"].arrive()
            yield None
            n += T

    roles = {"producer": producer(), "mma": mma()}
    for wid in range(EPI_WARPS_ONE_PAIR):
        roles[f"epi{wid}"] = epilogue(wid)
    return roles


def _read(st: State, me: str, key, tag):
    if any(op[0] == "mma" and op[1] == key for op in st.inflight):
        raise ProtocolError(f"{me} reads TMEM region {key} ({tag}) while MMAs on it are in "
                            f"flight")
    cur = st.readers.get(key)
    if cur is None or cur[0] != tag or me not in cur[1]:
        raise ProtocolError(f"{me} expected {tag} in TMEM region {key}, found {cur and cur[0]}")
    cur[1].discard(me)


def run(cfg: Config, units, seed: int, mistakes=frozenset(), timeout=None,
        max_steps: int = 2_000_000) -> State:
    """Replay the protocol under one random schedule and return the final
    state; raises ProtocolError on a deadlock, a phase aliasing, a reuse race
    or an unclean exit.  ``timeout`` = (role, i): from the role's i-th
    abortable wait on, its first wait that would block runs out of time."""
    rng = random.Random(seed)
    st = State(cfg)
    make = one_pair_roles if cfg.kind == "one_pair" else kernel_roles
    roles = make(st, units, mistakes)
    waiting, done = {}, set()
    nwaits = {name: 0 for name in roles}

    def advance(name, value=None):
        try:
            req = next(roles[name]) if value is None else roles[name].send(value)
        except StopIteration:
            done.add(name)
            waiting.pop(name, None)
            return
        if req is not None and req[3]:
            nwaits[name] += 1
        waiting[name] = req

    def gives_up(name, req):
        if not req[3]:
            return False
        return st.abort or (timeout is not None and name == timeout[0]
                            and nwaits[name] > timeout[1])

    for name in list(roles):
        advance(name)
    for _ in range(max_steps):
        if len(done) == len(roles):
            if st.inflight or st.copies:
                raise ProtocolError(f"the roles ended with {len(st.inflight)} MMA operations "
                                    f"and {len(st.copies)} copies in flight")
            return st
        choices = [("role", name) for name, req in waiting.items()
                   if req is None or req[1].passes(req[2]) or gives_up(name, req)]
        if st.copies:
            choices.append(("copy", None))
        if st.inflight:
            choices.append(("tensor", None))
        if not choices:
            blocked = {n: (r[1].name, r[2]) for n, r in waiting.items() if r is not None}
            raise ProtocolError(f"deadlock: {blocked}")
        kind, name = rng.choice(choices)
        if kind == "copy":
            bar, nbytes = st.copies.pop(rng.randrange(len(st.copies)))
            if nbytes is None:
                bar.arrive()  # a cp.async arrival: this lane's copies landed
            else:
                bar.complete_tx(nbytes)
        elif kind == "tensor":
            op = st.inflight.pop(0)  # MMAs and commits complete in issue order
            if op[0] == "commit":
                _, bar, pair = op
                if pair is not None and st.stage_busy.get(pair % cfg.stages) == pair:
                    del st.stage_busy[pair % cfg.stages]
                bar.arrive()
        else:
            req = waiting[name]
            if req is None:
                advance(name)
            elif req[1].passes(req[2]):
                if req[1].completed != req[2] + 1:
                    raise ProtocolError(f"{name}: waited for phase {req[2]} of {req[1].name}, "
                                        f"which has completed {req[1].completed} phases")
                advance(name, True)
            else:
                advance(name, False)  # budget expired, or the abort flag is set
    raise ProtocolError("step limit reached")
