"""Serving engine (continuous batching of many beams): every request's output
equals the oracle's transform of that beam's series, alone and in the mix,
bit for bit; admission waits for arena memory; device outputs can be copied
out and released."""
import numpy as np
import pytest

import paper_1201_5380_gb300 as dd
import synth
from _gpu import odelays, torch_cuda

pytestmark = pytest.mark.gpu

# two bands (as the serving workload: the same 400 MHz split into 2x channels)
BANDS = [dict(nchans=128, df=-100.0 / 128), dict(nchans=64, df=-100.0 / 64)]


def _beam_plans(nbeams, ndm=(24, 17)):
    plans = []
    for b in range(nbeams):
        band = BANDS[b % 2]
        plans.append(dd.Plan(band["nchans"], 64e-6, 1500.0, band["df"],
                             dms=np.linspace(0.0, 300.0 + 40 * b, ndm[b % 2])))
    return plans


def _series(plans, sizes, nbits=8):
    """Per beam: the whole input series (pinned-free numpy) and gulp sizes."""
    xs = []
    for b, p in enumerate(plans):
        xs.append(synth.uniform_packed(70 + b, nbits, int(sum(sizes[b])), p.nchans, nbits))
    return xs


def _expected(orc, plan, x, nbits):
    nout = x.shape[0] - plan.max_delay
    return orc.direct(x, nbits, plan.nchans, nout, odelays(orc, plan))


def _serve(server, plans, xs, sizes, beams, host_out=True, poll_every=1):
    """Submit every gulp of every beam (interleaved), run to completion and
    return per-beam concatenated outputs plus the completion records."""
    outs = {b: [] for b in beams}
    reqs = {}
    for k in range(max(len(s) for s in sizes)):
        for b in beams:
            if k >= len(sizes[b]):
                continue
            pos = int(sum(sizes[b][:k]))
            n = int(sizes[b][k])
            chunk = np.ascontiguousarray(xs[b][pos:pos + n])
            o = np.zeros((plans[b].dm_count, max(n, 1)), np.uint32) if host_out else None
            r = server.submit(beams[b], chunk, n, o)
            reqs[r] = (b, k, o)
        if k % poll_every == 0:
            server.step()
    done = {}
    for _ in range(10000):
        for info in server.poll():
            done[info["request"]] = info
        if len(done) == len(reqs):
            break
        server.step(wait=True)
    assert len(done) == len(reqs)
    per_beam = {b: {} for b in beams}
    for r, (b, k, o) in reqs.items():
        info = done[r]
        assert info["status"] == 0
        n = info["nsamps_out"]
        if host_out:
            got = o[:, :n]
        else:
            got = np.zeros((plans[b].dm_count, max(n, 1)), np.uint32)
            if n:
                server.copy_out(r, got)
            server.release(r)
            got = got[:, :n]
        per_beam[b][k] = got
    for b in beams:
        outs[b] = np.concatenate([per_beam[b][k] for k in sorted(per_beam[b])], axis=1)
    return outs, done


def test_server_outputs_equal_oracle_in_the_mix(orc):
    torch_cuda()
    plans = _beam_plans(4)
    rng = np.random.default_rng(5)
    sizes = [[int(v) for v in rng.integers(300, 2500, 4)] for _ in plans]
    xs = _series(plans, sizes)
    server = dd.Server(arena_bytes=64 << 20, max_batch=4, max_inflight=2)
    beams = {b: server.add_beam(p, 8, 2500) for b, p in enumerate(plans)}
    outs, done = _serve(server, plans, xs, sizes, beams)
    for b, p in enumerate(plans):
        assert np.array_equal(outs[b], _expected(orc, p, xs[b], 8)), b
    assert all(d["latency_ms"] > 0 for d in done.values())
    st = server.stats()
    assert st["queued"] == 0 and st["inflight"] == 0 and st["arena_used"] == 0


def test_server_beam_alone_equals_beam_in_the_mix():
    torch_cuda()
    plans = _beam_plans(3)
    sizes = [[1200, 900, 1700], [800, 2000, 400], [1500, 1500, 1500]]
    xs = _series(plans, sizes)
    mixed = dd.Server(arena_bytes=64 << 20, max_batch=3, max_inflight=2)
    bm = {b: mixed.add_beam(p, 8, 2000) for b, p in enumerate(plans)}
    out_mix, _ = _serve(mixed, plans, xs, sizes, bm)
    for b in range(3):
        alone = dd.Server(arena_bytes=64 << 20, max_batch=1, max_inflight=1)
        ba = {b: alone.add_beam(plans[b], 8, 2000)}
        out_alone, _ = _serve(alone, plans, xs, sizes, ba)
        assert np.array_equal(out_alone[b], out_mix[b]), b
        alone.close()


def test_server_admission_waits_for_arena_memory(orc):
    torch_cuda()
    plans = _beam_plans(4)
    sizes = [[1000] * 5 for _ in plans]
    xs = _series(plans, sizes)
    # room for about two gulps' buffers at a time: most gulps must wait
    one = max(p.dm_count * 1000 * 4 + 1000 * p.nchans for p in plans)
    server = dd.Server(arena_bytes=int(2.2 * one) + (1 << 12), max_batch=4, max_inflight=3)
    beams = {b: server.add_beam(p, 8, 1000) for b, p in enumerate(plans)}
    outs, done = _serve(server, plans, xs, sizes, beams)
    for b, p in enumerate(plans):
        assert np.array_equal(outs[b], _expected(orc, p, xs[b], 8)), b
    assert server.stats()["arena_used"] == 0


def test_server_device_outputs_copy_out_and_release(orc):
    torch_cuda()
    plans = _beam_plans(2)
    sizes = [[900, 1800, 700], [1600, 300, 1200]]
    xs = _series(plans, sizes)
    server = dd.Server(arena_bytes=64 << 20, max_batch=2, max_inflight=2)
    beams = {b: server.add_beam(p, 8, 1800) for b, p in enumerate(plans)}
    outs, _ = _serve(server, plans, xs, sizes, beams, host_out=False)
    for b, p in enumerate(plans):
        assert np.array_equal(outs[b], _expected(orc, p, xs[b], 8)), b
    assert server.stats()["arena_used"] == 0


def test_server_rejects_a_gulp_larger_than_the_arena():
    torch_cuda()
    plan = _beam_plans(1)[0]
    server = dd.Server(arena_bytes=1 << 20, max_batch=1, max_inflight=1)
    b = server.add_beam(plan, 8, 1 << 16)
    x = np.zeros((1 << 16, plan.nchans), np.uint8)
    with pytest.raises(dd.DedispError) as e:
        server.submit(b, x)
    assert e.value.code == 11


def test_server_wait_deadline_returns_timeout_and_recovers(orc):
    """A launch held back on the host (a 700 ms pause in the compute stream,
    no device work) makes a waiting step reach the server's 100 ms deadline:
    DD_ERR_TIMEOUT (7) comes back, the launch stays in flight, and once the
    pause ends the server retires it and every result is still exact.  The
    outputs stay on the device (a copy into pageable host memory would make
    the launch itself wait on the host)."""
    import time
    torch_cuda()
    plans = _beam_plans(2)
    sizes = [[1500, 1300], [1100, 1700]]
    xs = _series(plans, sizes)
    server = dd.Server(arena_bytes=64 << 20, max_batch=2, max_inflight=2)
    beams = {b: server.add_beam(p, 8, 1700) for b, p in enumerate(plans)}
    server.set_timeout(100.0)
    server.pause_next_launch(700.0)
    reqs = {}
    for b in beams:
        reqs[server.submit(beams[b], np.ascontiguousarray(xs[b][:sizes[b][0]]))] = (b, 0)
    assert server.step() == 2          # both gulps in one launch, held by the pause
    t0 = time.monotonic()
    with pytest.raises(dd.DedispError) as e:
        server.step(wait=True)
    waited = time.monotonic() - t0
    assert e.value.code == 7
    assert 0.05 < waited < 0.6
    assert server.stats()["inflight"] == 2
    with pytest.raises(dd.DedispError) as e:
        server.drain()                 # still inside the pause
    assert e.value.code == 7
    server.set_timeout(5000.0)
    server.drain()
    assert server.stats()["inflight"] == 0
    for b in beams:                     # the server goes on serving
        pos = sizes[b][0]
        reqs[server.submit(beams[b], np.ascontiguousarray(xs[b][pos:pos + sizes[b][1]]))] = (b, 1)
    server.step()
    server.drain()
    done = {i["request"]: i for i in server.poll()}
    assert len(done) == 4
    per = {b: {} for b in beams}
    for r, (b, k) in reqs.items():
        assert done[r]["status"] == 0
        n = done[r]["nsamps_out"]
        o = np.zeros((plans[b].dm_count, max(n, 1)), np.uint32)
        if n:
            server.copy_out(r, o)
        server.release(r)
        per[b][k] = o[:, :n]
    for b, p in enumerate(plans):
        got = np.concatenate([per[b][0], per[b][1]], axis=1)
        assert np.array_equal(got, _expected(orc, p, xs[b], 8)), b
    server.close()
