"""The order of the pipelined moment-record backward (adjoint.WidthGradient._backward_pipelined),
checked on the host with stand-ins for the CUDA streams, events and library calls: every
adjoint chain must read the records of its own segment (recorded by the forward or by a
recompute that completed before it), a recompute must not refill a record set before the
adjoint that last read it has finished, and a stream must never wait on an event that has not
been recorded yet (CUDA would not wait at all).  The streams run in order, in two extreme
interleavings (the adjoint stream ahead whenever it can run, or the recompute stream ahead).
"""
import pytest


@pytest.fixture(scope="module")
def adjoint():
    from paper_1405_1253_b300 import build
    build.build()                    # the module loads the library on import
    from paper_1405_1253_b300 import adjoint as m
    return m


class Event:
    def __init__(self):
        self.issued = False      # its record has been enqueued (host order)
        self.done = False        # the stream has reached that record

    def record(self, stream):
        self.issued = True
        stream.ops.append(("event", self))


class Stream:
    def __init__(self, name):
        self.name = name
        self.ops = []

    def wait_event(self, ev):
        assert ev.issued, f"{self.name} waits on an event that is not recorded yet"
        self.ops.append(("wait", ev))

    def wait_stream(self, other):
        ev = Event()
        ev.record(other)
        self.wait_event(ev)


class Torch:
    class cuda:
        Event = Event


class RecordSet:
    def __init__(self, i):
        self.i = i

    def __getitem__(self, j):
        return (self.i, j)


class Context:
    def __init__(self, stream, kind, drv):
        self.stream, self.kind, self.drv = stream, kind, drv

    def record_moments(self, f0, wa, wb, moms):
        self.stream.ops.append(("record", (moms[0][0], self.drv.ckpts.index(f0))))

    def adjoint_chain_moments(self, moms, a, b):
        self.stream.ops.append(("adjoint", moms[0][0]))
        self.drv._adj_order.append(moms[0][0])
        return 0


def driver(adjoint, S, nset, K=5):
    d = object.__new__(adjoint.WidthGradient)
    d.torch = Torch
    d.N, d.K = S * K, K
    d.ckpts = [object() for _ in range(S)]
    d.work = [object(), object()]
    d.moms_sets = [RecordSet(i) for i in range(nset)]
    d.n_taped = min(nset, S)
    d.stats = adjoint.AdjointStats()
    d.rec_stream = Stream("recompute")
    d.L = Context(Stream("adjoint"), "main", d)
    d.Lrec = Context(d.rec_stream, "rec", d)
    d._adj_order = []
    return d


def simulate(d, S, nset, main_first):
    """Run both streams in order, one operation at a time, the preferred stream whenever it
    can move; returns (record set, segment it held) for each adjoint chain in run order."""
    holds = {s % nset: s for s in range(S - d.n_taped, S)}     # written by the forward
    streams = [d.L.stream, d.rec_stream] if main_first else [d.rec_stream, d.L.stream]
    pos = {id(st): 0 for st in streams}
    seen = []

    def step(st):
        if pos[id(st)] >= len(st.ops):
            return False
        kind, arg = st.ops[pos[id(st)]]
        if kind == "wait" and not arg.done:
            return False
        if kind == "event":
            arg.done = True
        elif kind == "record":
            holds[arg[0]] = arg[1]
        elif kind == "adjoint":
            seen.append((arg, holds.get(arg)))
        pos[id(st)] += 1
        return True

    while any(step(st) for st in streams):
        pass
    assert all(pos[id(st)] == len(st.ops) for st in streams), "the streams deadlock"
    return seen


@pytest.mark.parametrize("S,nset", [(20, 2), (20, 3), (20, 4), (7, 3), (5, 4), (3, 4), (2, 2), (4, 2)])
@pytest.mark.parametrize("main_first", [True, False])
def test_pipelined_backward_order(adjoint, S, nset, main_first):
    d = driver(adjoint, S, nset)
    d._backward_pipelined("lam_a", "lam_b")
    seen = simulate(d, S, nset, main_first)
    # the adjoint chains run from the last segment down, each on its own segment's records
    assert [a for a, _ in seen] == [s % nset for s in range(S - 1, -1, -1)]
    order = list(range(S - 1, -1, -1))
    for s, (set_read, held) in zip(order, seen):
        assert held == s, f"adjoint of segment {s} read the records of segment {held}"
    assert d.stats.recompute_steps == d.K * max(0, S - d.n_taped)
    assert d.stats.adjoint_steps == d.K * S
