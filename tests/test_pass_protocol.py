"""The ordering protocol of the coordinate passes (sweeps.cu), modelled and checked under
random interleavings on the CPU.

The persistent pass kernel orders its roles by counters and flags instead of grid barriers:
CTA 0 holds the serial chain (phase B), a feeder lane (bulk copies of each batch's step
constants and coefficient panels into shared-memory buffers, and publication of each
batch's steps) and the correction warps (the part carried from the previous batch); CTAs
1.. run phase C of batch k (the cache update of their band) and phase A of batch k + 2.
This model restates, step by step, what each role waits for and what it reads and writes,
and a random scheduler interleaves the roles and the asynchronous copies.  Every schedule
must finish (no deadlock), and every read must see exactly the data the sequential pass
would: phase A of batch j sees the cache with batches 0 .. j-2 applied on every band and
nothing else; the chain reads batch k's constants, panels and carried corrections; the
carried corrections read X(k, k-1) and the steps of batch k-1; phase C of batch k reads batch
k's steps; no buffer is overwritten while a reader still needs it.  A planted mistake (a
feeder that does not wait for a panel buffer to be released, phase C that does not wait for
every phase A, corrections formed before the previous batch's steps are all in) must be
caught.  This model is the race check of the protocol (no memory
checker runs the kernels); the kernels' outputs are checked against the oracle by the GPU
tests.
"""
import random

import pytest


class Deadlock(Exception):
    pass


class Violation(Exception):
    pass


def simulate(nA, nbatch, NS, NBUF, last_panels, seed, mistake=None, max_steps=200000):
    rnd = random.Random(seed)
    npan = [NS] * nbatch
    npan[-1] = last_panels
    st = {
        "mu_ready": 0, "a_done": 0, "c_done": 0, "prog": 0, "corr_prog": 0,
        "applied": [set() for _ in range(nA)],      # batches applied to each band
        "A_active": {},                               # cta -> batch being read by phase A
        "C_active": {},                               # cta -> batch being written
        "X": [None, None],                            # cross coefficients (batch parity)
        "pre_g": [None, None], "coef_g": [None, None],  # phase A outputs in device memory
        "mu_g": [None, None],                         # steps in device memory
        "mu_s": [None, None],                         # steps in shared memory (CTA 0)
        "corr": [None] * NS,                          # carried corrections per panel
        "pre_s": [None, None], "pre_landed": [0, 0],  # step-constant buffers, copies landed
        "buf": [None] * NBUF, "buf_landed": [0] * NBUF,
        "inflight": [],                               # (kind, index, content)
        "C_done_batches": [0] * nbatch,               # CTAs that finished phase C of a batch
    }

    def check(cond, what):
        if not cond:
            raise Violation(what)

    def phase_a(cta, j):
        """Phase A of batch j on one CTA: reads every band (the rows of a batch cross all
        bands) and writes its share of batch j's constants, coefficients and X(j, j-1),
        destroying what the buffers of that parity held (batch j - 2's)."""
        want = set(range(j - 1))
        for b in range(nA):
            check(st["applied"][b] == want, f"A({j}) on {cta} sees band {b} at {st['applied'][b]}")
        for c2, k in st["C_active"].items():
            check(False, f"A({j}) on {cta} while C({k}) runs on {c2}")
        for kind, _, content in st["inflight"]:
            check(content[0] != j - 2, f"A({j}) overwrites the source of a copy of batch {j - 2}")
        st["pre_g"][j & 1] = st["coef_g"][j & 1] = st["X"][j & 1] = ("writing", j)
        st["A_active"][cta] = j
        yield
        for b in range(nA):
            check(st["applied"][b] == want, f"A({j}) on {cta}: band {b} changed under it")
        del st["A_active"][cta]
        if not any(v == j for v in st["A_active"].values()):
            st["pre_g"][j & 1] = st["coef_g"][j & 1] = st["X"][j & 1] = j

    # ---- CTAs 1..: the band owners ----
    def other(cta):
        if nbatch > 1:
            yield from phase_a(cta, 1)
            st["a_done"] += 1
        for k in range(nbatch):
            nbn = nbatch > k + 1
            while not (st["mu_ready"] >= k + 1 and (not nbn or mistake == "c_no_wait_a"
                                                   or st["a_done"] >= (k + 1) * nA)):
                yield "wait"
            check(st["mu_g"][k & 1] == ("done", k), f"C({k}) reads steps {st['mu_g'][k & 1]}")
            for c2, j in st["A_active"].items():
                check(False, f"C({k}) on {cta} while A({j}) reads on {c2}")
            st["C_active"][cta] = k
            yield
            st["applied"][cta].add(k)
            del st["C_active"][cta]
            st["C_done_batches"][k] += 1
            st["c_done"] += 1
            while st["c_done"] < (k + 1) * nA:
                yield "wait"
            if k + 2 < nbatch:
                yield from phase_a(cta, k + 2)
                st["a_done"] += 1

    # ---- CTA 0: the chain ----
    def chain():
        for k in range(nbatch):
            pb = k & 1
            while st["pre_landed"][pb] < k // 2 + 1:
                yield "wait"
            check(st["pre_s"][pb] == k, f"chain reads constants of {st['pre_s'][pb]} for {k}")
            if k >= 2:
                check(st["C_done_batches"][k - 2] == nA, f"B({k}) overwrites steps before C({k-2})")
            st["mu_g"][pb] = ("partial", k)
            for s in range(npan[k]):
                bi = s % NBUF
                need = (k * NS + s) // NBUF + 1 if NBUF != NS else k + 1
                while st["buf_landed"][bi] < need:
                    yield "wait"
                check(st["buf"][bi] == (k, s), f"chain reads panel {st['buf'][bi]} for {(k, s)}")
                if k > 0:
                    while st["corr_prog"] < k * NS + s + 1:
                        yield "wait"
                    check(st["corr"][s] == k, f"chain reads corrections {st['corr'][s]} for {(k, s)}")
                yield
                st["mu_s"][pb] = ("partial", k)
                st["prog"] = k * NS + s + 1
            st["mu_g"][pb] = ("done", k)
            st["mu_s"][pb] = ("done", k)

    # ---- CTA 0: the feeder ----
    def feeder():
        published = 0

        def publish():
            nonlocal published
            done = st["prog"] // NS
            if st["prog"] == (nbatch - 1) * NS + npan[-1]:
                done = nbatch
            if done > published:
                for j in range(published, done):
                    check(st["mu_g"][j & 1] == ("done", j), f"publishes batch {j} before it is done")
                st["mu_ready"] += done - published
                published = done

        for k in range(nbatch):
            pb = k & 1
            if k > 0:
                while st["a_done"] < k * nA:
                    publish()
                    yield "wait"
            check(st["pre_g"][pb] == k and st["coef_g"][pb] == k, f"copies of {k} before phase A")
            if k >= 2:
                while st["prog"] < (k - 1) * NS:
                    yield "wait"
                publish()
            st["inflight"].append(("pre", pb, (k,)))
            for s in range(npan[k]):
                prev = k * NS + s - NBUF
                if prev >= 0 and mistake != "feeder_no_wait":
                    while st["prog"] < prev + 1:
                        yield "wait"
                    publish()
                st["inflight"].append(("panel", s % NBUF, (k, s)))
                yield
            if k >= 1:
                while st["prog"] < k * NS:
                    yield "wait"
                publish()
        while st["prog"] < (nbatch - 1) * NS + npan[-1]:
            yield "wait"
        publish()

    # ---- CTA 0: the correction warps ----
    def corrections():
        for k in range(1, nbatch):
            while st["a_done"] < k * nA:
                yield "wait"
            check(st["X"][k & 1] == k, f"corrections of {k} read X of {st['X'][k & 1]}")
            while st["prog"] < k * NS and mistake != "corr_no_wait":
                yield "wait"
            check(st["mu_s"][(k - 1) & 1] == ("done", k - 1), f"corrections of {k} read steps {st['mu_s'][(k-1) & 1]}")
            for s in range(npan[k]):
                yield
                check(st["X"][k & 1] == k, f"X of {k} overwritten while its corrections run")
                st["corr"][s] = k
                st["corr_prog"] = k * NS + s + 1

    # prologue: phase A of batch 0 on every CTA, then a grid barrier
    st["pre_g"][0] = st["coef_g"][0] = 0
    st["X"][0] = 0
    roles = {f"other{c}": other(c) for c in range(nA)}
    roles.update(chain=chain(), feeder=feeder(), corrections=corrections())
    def signature():
        return (st["mu_ready"], st["a_done"], st["c_done"], st["prog"], st["corr_prog"],
                len(st["inflight"]))

    for step in range(max_steps):
        live = [n for n in roles]
        if not live and not st["inflight"]:
            return step
        choices = live + (["copy"] if st["inflight"] else [])
        rnd.shuffle(choices)
        progressed = False
        for n in choices:
            if n == "copy":
                kind, idx, content = st["inflight"].pop(rnd.randrange(len(st["inflight"])))
                if kind == "pre":
                    st["pre_s"][idx] = content[0]
                    st["pre_landed"][idx] += 1
                else:
                    st["buf"][idx] = content
                    st["buf_landed"][idx] += 1
                progressed = True
                break
            before = signature()
            try:
                r = next(roles[n])
            except StopIteration:
                del roles[n]
                progressed = True
                break
            if r != "wait" or signature() != before:  # a wait that changed state moved too
                progressed = True
                break
        if not progressed:
            raise Deadlock(f"no role can move: {sorted(roles)}; counters mu {st['mu_ready']} "
                           f"a {st['a_done']} c {st['c_done']} prog {st['prog']}")
    raise Deadlock("step limit")


CASES = [
    # nA, nbatch, NS, NBUF, last batch's panels
    (3, 6, 3, 3, 3),
    (3, 7, 3, 3, 1),
    (1, 5, 2, 2, 2),
    (4, 1, 3, 3, 2),
    (2, 2, 4, 4, 4),
    (3, 6, 4, 2, 3),   # two panel buffers taking turns (B > 256)
    (2, 9, 8, 8, 5),
]


@pytest.mark.parametrize("case", CASES)
def test_every_interleaving_finishes_and_reads_the_sequential_data(case):
    nA, nbatch, NS, NBUF, last = case
    for seed in range(60):
        simulate(nA, nbatch, NS, NBUF, last, seed)


@pytest.mark.parametrize("mistake", ["feeder_no_wait", "c_no_wait_a", "corr_no_wait"])
def test_planted_ordering_mistakes_are_caught(mistake):
    caught = 0
    for seed in range(60):
        try:
            simulate(3, 6, 3, 3, 3, seed, mistake=mistake)
        except (Violation, Deadlock):
            caught += 1
    assert caught > 0
