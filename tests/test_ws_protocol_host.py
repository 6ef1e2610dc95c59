"""The FIR/FFT hand-off of the warp-specialised F-stage kernels (ppf_ws_kernel,
ppf_correct_ws_kernel, ppf_correct_ws256_kernel), checked on the host.

Both roles are modelled as agents on counting barriers with the semantics of
bar.sync / bar.arrive (an instance completes when all participants arrived;
sync waits for completion, arrive does not). The FIR role writes round b into
row buffer b % 2 (after waiting on EMPTY[b % 2] from round 2 on) and arrives
on FULL[b % 2]; the FFT role syncs on FULL[b % 2], reads the buffer, and
arrives on EMPTY[b % 2] while b + 2 < rounds. Random interleavings must finish
(no deadlock), every FFT read must see its own round's data, and no barrier
may be left with a partial instance.

The 256-channel kernel splits its FFT threads into two groups: group g takes
the rounds b with b % 2 == g, so FULL[g] and EMPTY[g] are shared by the FIR
role and group g only (a barrier instance = the FIR threads + one group).
That protocol is checked the same way, with three agents."""
import random

import pytest


class Barrier:
    def __init__(self, parties):
        self.parties, self.count, self.generation = parties, 0, 0

    def arrive(self):
        self.count += 1
        if self.count == self.parties:
            self.count, self.generation = 0, self.generation + 1


def fir_program(rounds):
    for b in range(rounds):
        q = b & 1
        if b >= 2:
            yield ("sync", ("EMPTY", q))
        yield ("write", (q, b))
        yield ("arrive", ("FULL", q))


def fft_program(rounds):
    for b in range(rounds):
        q = b & 1
        yield ("sync", ("FULL", q))
        yield ("read", (q, b))
        if b + 2 < rounds:
            yield ("arrive", ("EMPTY", q))


def fft_group_program(g):
    def prog(rounds):
        for b in range(g, rounds, 2):
            q = b & 1
            yield ("sync", ("FULL", q))
            yield ("read", (q, b))
            if b + 2 < rounds:
                yield ("arrive", ("EMPTY", q))
    return prog


def simulate(rounds, seed, fir=fir_program, fft=fft_program, ffts=None):
    rng = random.Random(seed)
    bars = {(k, q): Barrier(2) for k in ("FULL", "EMPTY") for q in (0, 1)}
    buf = {0: None, 1: None}
    agents = {"fir": fir(rounds)}
    if ffts is None:
        agents["fft"] = fft(rounds)
    else:
        for g, prog in enumerate(ffts):
            agents[f"fft{g}"] = prog(rounds)
    pending = {a: next(g, None) for a, g in agents.items()}
    waiting = {}                     # agent -> (barrier key, generation to reach)
    while any(v is not None for v in pending.values()):
        runnable = [a for a, op in pending.items() if op is not None and
                    (a not in waiting or bars[waiting[a][0]].generation >= waiting[a][1])]
        if not runnable:
            return "deadlock", None
        a = rng.choice(runnable)
        if a in waiting:             # its sync completed
            del waiting[a]
            pending[a] = next(agents[a], None)
            continue
        kind, arg = pending[a]
        if kind == "write":
            buf[arg[0]] = arg[1]
        elif kind == "read":
            if buf[arg[0]] != arg[1]:
                return "stale", (arg, buf[arg[0]])
        elif kind == "arrive":
            bars[arg].arrive()
        elif kind == "sync":
            target = bars[arg].generation + 1
            bars[arg].arrive()
            if bars[arg].generation < target:
                waiting[a] = (arg, target)
                continue
        pending[a] = next(agents[a], None)
    if any(b.count for b in bars.values()):
        return "partial", {k: b.count for k, b in bars.items() if b.count}
    return "ok", None


@pytest.mark.parametrize("rounds", [1, 2, 3, 4, 5, 16, 48, 64])
def test_handoff_completes_and_reads_fresh_rows(rounds):
    for seed in range(200):
        res, info = simulate(rounds, seed)
        assert res == "ok", (rounds, seed, res, info)


def test_missing_empty_wait_is_caught():
    """Planting the mistake (the FIR role does not wait for EMPTY) must make
    some interleaving read a buffer that the next-but-one round overwrote."""
    def fir_no_wait(rounds):
        for b in range(rounds):
            yield ("write", (b & 1, b))
            yield ("arrive", ("FULL", b & 1))

    def fft_no_arrive(rounds):
        for b in range(rounds):
            yield ("sync", ("FULL", b & 1))
            yield ("read", (b & 1, b))

    results = {simulate(8, seed, fir_no_wait, fft_no_arrive)[0] for seed in range(200)}
    assert results - {"ok"}, results


@pytest.mark.parametrize("rounds", [1, 2, 3, 4, 5, 16, 48, 64])
def test_two_fft_groups_handoff_completes_and_reads_fresh_rows(rounds):
    groups = [fft_group_program(0), fft_group_program(1)]
    for seed in range(200):
        res, info = simulate(rounds, seed, ffts=groups)
        assert res == "ok", (rounds, seed, res, info)


def test_two_fft_groups_wrong_parity_is_caught():
    """A group that takes the wrong rounds (both groups on buffer 0's rounds)
    must deadlock or read stale rows."""
    def wrong(rounds):
        for b in range(0, rounds, 2):
            yield ("sync", ("FULL", 0))
            yield ("read", (0, b))
            if b + 2 < rounds:
                yield ("arrive", ("EMPTY", 0))
    results = {simulate(8, seed, ffts=[fft_group_program(0), wrong])[0] for seed in range(200)}
    assert results - {"ok"}, results
