"""Ordering contract of `pipeline.contract_batches`, on the host.

The GPU tests check the pipeline's amplitudes against the oracle; this test
checks the order of its operations with a stand-in for torch's CUDA
streams, events and buffers and for the library's plan.  Device work runs
eagerly at launch and every bind, contraction, event wait and error check
is logged, so the test sees:

* with several workspaces, a batch binds into a workspace only after the
  batch that used it last has been waited for, and batch i + 1 is launched
  before batch i's result is read (the overlap the pipeline exists for);
* with one workspace, a batch binds only after the previous one was read;
* every result is read after its batch's event, in input order, and holds
  that batch's values although the next batch was launched before it was
  read (two amplitude buffers in turn).
"""

import sys
import threading
import types

import numpy as np
import pytest

from paper_2212_04749_gb300 import pipeline


class _Log:
    def __init__(self):
        self.items = []
        self.lock = threading.Lock()
        self.last_contract = None

    def add(self, *item):
        with self.lock:
            self.items.append(item + (threading.get_ident(),))

    def index(self, *item):
        # first entry matching item (any thread)
        return next(n for n, x in enumerate(self.items) if x[:len(item)] == item)

    def waited_before(self, batch, pos, thread):
        # the given thread waited for batch's event before log position pos
        return any(x[:2] == ("sync", batch) and x[-1] == thread for x in self.items[:pos])


class _Tensor:
    def __init__(self, n):
        self.a = np.zeros(n)

    def numel(self):
        return self.a.size

    def __getitem__(self, sl):
        t = _Tensor(0)
        t.a = self.a[sl]
        return t

    def zero_(self):
        self.a[:] = 0

    def copy_(self, other, non_blocking=False):
        self.a[:] = other.a

    def numpy(self):
        return self.a


def _fake_torch(log):
    class Stream:
        def __init__(self, device=None):
            self.device = "cuda:0"

        def synchronize(self):
            pass

    class Event:
        def record(self, stream):
            self.batch = log.last_contract

        def synchronize(self):
            log.add("sync", self.batch)

    class _StreamCtx:
        def __init__(self, s):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False

    main = Stream()
    cuda = types.SimpleNamespace(Stream=Stream, Event=Event, stream=_StreamCtx, current_stream=lambda: main)
    return types.SimpleNamespace(cuda=cuda, float64="float64", zeros=lambda n, **kw: _Tensor(n),
                                 empty=lambda n, **kw: _Tensor(n))


class _Workspace:
    def __init__(self, wid):
        self.wid = wid

    def numel(self):
        return 1 << 20


def _values(i, m):
    # a batch's amplitudes as float64 pairs: batch index in the real parts
    v = np.zeros(2 * m)
    v[0::2] = i
    v[1::2] = np.arange(m)
    return v


def _fake_tn(log):
    class Plan:
        def __init__(self, circ, bits, ssa, sliced, **opts):
            self.i = int(bits[0, 0])
            self.k = bits.shape[0]
            self.info = {"workspace_bytes": 1024, "amps_per_row": 1}

        def tn_plan_bind(self, ws, stream=None):
            log.add("bind", self.i, ws.wid)

        def tn_plan_set_config(self, s, c):
            pass

        def tn_plan_set_chain(self, c, on):
            pass

        def tn_contract(self, a, precision, stream=None):
            a.a[:] = _values(self.i, self.k)
            log.add("contract", self.i)
            log.last_contract = self.i

        def tn_plan_check(self, stream=None):
            log.add("check", self.i)

    return types.SimpleNamespace(Plan=Plan)


@pytest.mark.parametrize("nws", [1, 2, 3])
def test_pipeline_orders_binds_launches_and_reads(monkeypatch, nws):
    log = _Log()
    monkeypatch.setitem(sys.modules, "torch", _fake_torch(log))
    monkeypatch.setattr(pipeline, "tn", _fake_tn(log))
    sizes = [3, 5, 2, 8, 8, 1, 6]  # rows per batch: the buffers grow and shrink
    batches = [np.full((k, 1), i, np.uint8) for i, k in enumerate(sizes)]
    spaces = [_Workspace(w) for w in range(nws)]
    got = list(pipeline.contract_batches(None, batches, None, (), "bf16x3",
                                         spaces if nws > 1 else spaces[0], configs=[2, 3], chains=[1]))
    # results in input order, each with its own batch's values
    assert [j for j, _ in got] == list(range(len(sizes)))
    for (j, amps), k in zip(got, sizes):
        ref = _values(j, k)
        np.testing.assert_array_equal(amps, ref[0::2] + 1j * ref[1::2])
    n = len(sizes)
    for j in range(n):
        # read only after its batch was waited for, by the reading thread
        chk = log.index("check", j)
        assert log.waited_before(j, chk, log.items[chk][-1])
        bind = log.index("bind", j)
        assert log.items[bind][2] == (j % nws)
        if nws == 1:
            if j > 0:  # the previous batch was read before this one binds
                assert log.index("check", j - 1) < bind
        else:
            if j >= nws:  # the binding thread waited for the workspace's last batch
                assert log.waited_before(j - nws, bind, log.items[bind][-1])
            if j + 1 < n:  # the next batch runs before this one is read
                assert log.index("contract", j + 1) < chk
