"""Streaming (device-resident overlap tail) and batched multi-beam launches:
the concatenation of a stream's outputs equals the direct transform of the
concatenated input, and a batch equals per-stream pushes, bit for bit."""
import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from _gpu import odelays, torch_cuda

pytestmark = pytest.mark.gpu


def _plan(nchans=256, ndm=40, hi=400.0, df=None):
    return dd.Plan(nchans, 64e-6, 1500.0, df if df else -100.0 / nchans,
                   dms=np.linspace(0.0, hi, ndm))


def _push_all(stream, x, sizes, ndm, torch, device=True):
    outs, pos = [], 0
    for n in sizes:
        chunk = x[pos:pos + n]
        pos += n
        if device:
            o = torch.zeros((ndm, max(n, 1)), dtype=torch.int32, device="cuda")
            k = stream.push(torch.from_numpy(np.ascontiguousarray(chunk)).cuda(), n, o)
            torch.cuda.synchronize()
            outs.append(o[:, :k].cpu().numpy().view(np.uint32))
        else:
            o = np.zeros((ndm, max(n, 1)), np.uint32)
            k = stream.push(np.ascontiguousarray(chunk), n, o)
            outs.append(o[:, :k])
    return np.concatenate(outs, axis=1)


@pytest.mark.parametrize("nbits", [2, 8])
def test_stream_concatenation_equals_one_shot(orc, nbits):
    torch = torch_cuda()
    plan = _plan()
    rng = np.random.default_rng(1)
    sizes = list(rng.integers(1, 3000, 12)) + [plan.max_delay + 5, 1, 2999]
    total = int(sum(sizes))
    x = synth.uniform_packed(31, nbits, total, 256, nbits)
    s = dd.Stream(plan, nbits, max_gulp=3000)
    got = _push_all(s, x, sizes, plan.dm_count, torch)
    nout = total - plan.max_delay
    assert got.shape[1] == nout
    assert s.position() == (total, nout)
    ref = orc.direct(x, nbits, 256, nout, odelays(orc, plan))
    assert np.array_equal(got, ref)


def test_stream_host_pointers(orc):
    torch_cuda()
    plan = _plan()
    sizes = [700, 2500, 10, 1800]
    x = synth.uniform_packed(32, 0, sum(sizes), 256, 2)
    s = dd.Stream(plan, 2, max_gulp=2500)
    got = _push_all(s, x, sizes, plan.dm_count, None, device=False)
    nout = sum(sizes) - plan.max_delay
    assert np.array_equal(got, orc.direct(x, 2, 256, nout, odelays(orc, plan)))


def test_stream_snapshot_restore_continues_identically():
    torch = torch_cuda()
    plan = _plan()
    sizes = [1500, 1500, 1500, 1500, 1500]
    x = synth.uniform_packed(33, 0, sum(sizes), 256, 2)
    a = dd.Stream(plan, 2, max_gulp=2000)
    first = _push_all(a, x[:3000], sizes[:2], plan.dm_count, torch)
    snap = a.snapshot()
    rest_a = _push_all(a, x[3000:], sizes[2:], plan.dm_count, torch)
    b = dd.Stream(plan, 2, max_gulp=2000)
    b.restore(snap)
    rest_b = _push_all(b, x[3000:], sizes[2:], plan.dm_count, torch)
    assert np.array_equal(rest_a, rest_b)
    assert b.position() == a.position()
    one = dd.Stream(plan, 2, max_gulp=8000)
    ref = _push_all(one, x, [sum(sizes)], plan.dm_count, torch)
    assert np.array_equal(np.concatenate([first, rest_a], axis=1), ref)


def test_batch_equals_individual_streams(orc):
    """Beams of different channel counts, trial lists and gulp lengths in one
    launch give the same bits as separate pushes (and as the oracle)."""
    torch = torch_cuda()
    plans = [_plan(nchans=256, ndm=40), _plan(nchans=512, ndm=23, hi=700.0),
             _plan(nchans=128, ndm=70, hi=900.0)]
    gulps = [[3000, 2000, 2500], [1000, 3100, 900], [2200, 2200, 2200]]
    xs = [synth.uniform_packed(40 + i, 0, sum(g), p.nchans, 8)
          for i, (p, g) in enumerate(zip(plans, gulps))]
    batch_streams = [dd.Stream(p, 8, max_gulp=4000) for p in plans]
    solo_streams = [dd.Stream(p, 8, max_gulp=4000) for p in plans]
    b = dd.Batch()
    outs_b = [[] for _ in plans]
    outs_s = [[] for _ in plans]
    pos = [0] * len(plans)
    for step in range(3):
        b.clear()
        bufs = []
        for i, p in enumerate(plans):
            n = gulps[i][step]
            chunk = torch.from_numpy(np.ascontiguousarray(xs[i][pos[i]:pos[i] + n])).cuda()
            o = torch.zeros((p.dm_count, n), dtype=torch.int32, device="cuda")
            b.add(batch_streams[i], chunk, n, o)
            bufs.append((chunk, o))
        ks = b.launch()
        torch.cuda.synchronize()
        for i, p in enumerate(plans):
            n = gulps[i][step]
            outs_b[i].append(bufs[i][1][:, :ks[i]].cpu().numpy().view(np.uint32))
            o2 = torch.zeros((p.dm_count, n), dtype=torch.int32, device="cuda")
            k2 = solo_streams[i].push(bufs[i][0], n, o2)
            torch.cuda.synchronize()
            assert k2 == ks[i]
            outs_s[i].append(o2[:, :k2].cpu().numpy().view(np.uint32))
            pos[i] += n
    for i, p in enumerate(plans):
        gb = np.concatenate(outs_b[i], axis=1)
        gs = np.concatenate(outs_s[i], axis=1)
        assert np.array_equal(gb, gs)
        nout = sum(gulps[i]) - p.max_delay
        assert np.array_equal(gb, orc.direct(xs[i], 8, p.nchans, nout, odelays(orc, p)))


@pytest.mark.parametrize("churn", [False, True])
def test_batch_graph_replay_equals_the_oracle(orc, churn):
    """A captured batch launch replayed gulp after gulp (new data written
    into the same input buffers) continues every beam's series exactly.
    With churn, each plan's staging-table cache is refilled past its bound
    (executes under 17 other tilings, then the tiling is put back) between
    capture and replay: the graph holds the tables its kernels read, so the
    replay still reads live tables."""
    torch = torch_cuda()
    plans = [_plan(256, 40, 400.0), _plan(128, 23, 300.0), _plan(256, 17, 250.0)]
    G = 2048
    ngulps = 6
    xs = [synth.uniform_packed(90 + i, 2, G * ngulps, p.nchans, 2) for i, p in enumerate(plans)]
    ins = [torch.zeros((G, p.nchans // 4), dtype=torch.uint8, device="cuda") for p in plans]
    outs = [torch.zeros((p.dm_count, G), dtype=torch.int32, device="cuda") for p in plans]
    streams = [dd.Stream(p, 2, G) for p in plans]
    batch = dd.Batch()
    for i in range(3):
        batch.add(streams[i], ins[i], G, outs[i])
    got = [[] for _ in plans]

    def load(k):
        for i in range(3):
            ins[i].copy_(torch.from_numpy(np.ascontiguousarray(xs[i][k * G:(k + 1) * G])))

    def collect(nouts):
        torch.cuda.synchronize()
        for i in range(3):
            got[i].append(outs[i][:, :nouts[i]].cpu().numpy().view(np.uint32).copy())

    for k in range(2):                 # prime the tails and warm the buffers
        load(k)
        collect(batch.launch())
    graph = batch.capture()
    if churn:
        for p in plans:
            tilings = [(b, cc, kk) for (b, kk) in ((32, 4), (64, 2), (16, 4), (32, 2), (32, 8))
                       for cc in (4, 8, 16)] + [(32, 32, 4), (64, 32, 2)]
            x = torch.zeros((G + p.max_delay, p.nchans // 4), dtype=torch.uint8, device="cuda")
            o = torch.zeros((p.dm_count, G), dtype=torch.int32, device="cuda")
            for t in tilings:
                p.set_tuning(*t)
                p.execute(x, 2, G, o)
            p.set_tuning(32, 32, -1)   # the tiling the graph was captured with
        torch.cuda.synchronize()
    for k in range(2, ngulps):
        load(k)
        collect(graph.launch())
    for i, p in enumerate(plans):
        series = np.concatenate(got[i], axis=1)
        nout = G * ngulps - p.max_delay
        assert series.shape[1] == nout
        assert streams[i].position() == (G * ngulps, nout)
        ref = orc.direct(xs[i], 2, p.nchans, nout, odelays(orc, p))
        assert np.array_equal(series, ref), i


def test_batch_graph_needs_primed_streams():
    torch_cuda()
    import torch
    p = _plan(128, 10, 300.0)
    s = dd.Stream(p, 2, 1000)
    b = dd.Batch()
    x = torch.zeros((1000, 32), dtype=torch.uint8, device="cuda")
    o = torch.zeros((p.dm_count, 1000), dtype=torch.int32, device="cuda")
    b.add(s, x, 1000, o)
    with pytest.raises(dd.DedispError):
        b.capture()                    # tail still empty


def test_batch_of_differently_tuned_plans_equals_the_oracle(orc):
    """Beams whose plans carry different tilings run in one launch per
    tiling, each with its own; every beam's series is still exact."""
    torch = torch_cuda()
    plans = [_plan(256, 40, 400.0), _plan(128, 23, 300.0), _plan(256, 17, 250.0),
             _plan(512, 31, 350.0)]
    plans[0].set_tuning(64, 16, 2)
    plans[1].set_tuning(16, 8, 4)
    plans[3].set_tuning(32, 8, 8)
    G, ngulps = 1500, 4
    xs = [synth.uniform_packed(95 + i, 8, G * ngulps, p.nchans, 8) for i, p in enumerate(plans)]
    streams = [dd.Stream(p, 8, G) for p in plans]
    got = [[] for _ in plans]
    for k in range(ngulps):
        batch = dd.Batch()
        bufs = []
        for i, p in enumerate(plans):
            x = torch.from_numpy(np.ascontiguousarray(xs[i][k * G:(k + 1) * G])).cuda()
            o = torch.zeros((p.dm_count, G), dtype=torch.int32, device="cuda")
            batch.add(streams[i], x, G, o)
            bufs.append((x, o))
        ks = batch.launch()
        torch.cuda.synchronize()
        for i in range(len(plans)):
            got[i].append(bufs[i][1][:, :ks[i]].cpu().numpy().view(np.uint32))
    for i, p in enumerate(plans):
        series = np.concatenate(got[i], axis=1)
        nout = G * ngulps - p.max_delay
        assert series.shape[1] == nout
        assert np.array_equal(series, orc.direct(xs[i], 8, p.nchans, nout, odelays(orc, p))), i
