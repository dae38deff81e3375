"""The bench's wave scheduling on CPU with fake streams and events: every batch of a wave has
its inputs queued before any environment build of the wave, each stream waits for all of the
wave's input events before its build, contexts are used round-robin, and the timing marks are
recorded on the right streams."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class Log:
    def __init__(self):
        self.items = []


class Event:
    count = 0

    def __init__(self, log):
        Event.count += 1
        self.name, self.log = "e%d" % Event.count, log

    def record(self, stream):
        self.log.items.append(("record", self.name, stream.i))


class Stream:
    def __init__(self, i, log):
        self.i, self.log = i, log

    def wait_event(self, e):
        self.log.items.append(("wait", self.i, e.name))


def test_waves_queue_inputs_first_and_wait_for_all_of_them():
    bench = _bench()
    log = Log()
    S = 3
    streams = [Stream(i, log) for i in range(S)]
    marks = [[Event(log) for _ in range(4)] for _ in range(7)]

    def inputs(k, i):
        log.items.append(("inputs", k, i))

    def work(i, m):
        log.items.append(("work", i, m is not None))

    bench.run_waves(range(10, 17), S, streams, lambda: Event(log), inputs, work, marks)
    items = log.items
    inp_pos = [n for n, x in enumerate(items) if x[0] == "inputs"]
    wk_pos = [n for n, x in enumerate(items) if x[0] == "work"]
    inp = [items[n] for n in inp_pos]
    wk = [items[n] for n in wk_pos]
    assert [k for _, k, _ in inp] == list(range(10, 17))
    assert [i for _, _, i in inp] == [j % S for j in range(7)]
    assert [i for _, i, _ in wk] == [j % S for j in range(7)] and all(m for _, _, m in wk)
    # waves of S: all inputs of a wave come before the wave's first work item
    for w0 in range(0, 7, S):
        wave_inputs = inp_pos[w0:w0 + S]
        wave_work = wk_pos[w0:w0 + S]
        assert max(wave_inputs) < min(wave_work)
        # each stream of the wave waits for every input event of the wave before its work
        ready = [items[p + 1][1] for p in wave_inputs]          # the event recorded after inputs
        for x, p in zip(wk[w0:w0 + S], wave_work):
            i = x[1]
            waited = {it[2] for it in items[:p] if it[0] == "wait" and it[1] == i}
            assert set(ready) <= waited
    # the first timing mark of batch j is recorded on its stream before its inputs
    for j in range(7):
        rec = [n for n, it in enumerate(items) if it == ("record", marks[j][0].name, j % S)]
        assert rec and rec[0] < inp_pos[j]


def test_warmup_without_marks():
    bench = _bench()
    log = Log()
    streams = [Stream(i, log) for i in range(2)]
    seen = []
    bench.run_waves(range(3), 2, streams, lambda: Event(log), lambda k, i: seen.append((k, i)),
                    lambda i, m: seen.append(("w", i, m)))
    assert seen == [(0, 0), (1, 1), ("w", 0, None), ("w", 1, None), (2, 0), ("w", 0, None)]
