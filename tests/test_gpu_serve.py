"""GPU tests of the serving layer: every result of the continuous-batching
server and of the one-at-a-time pipeline is checked against the CPU oracle
(served streams decode with the oracle's strict decoder to the request's
elements; decompressed results equal the elements the stream was made from);
each request yields the same bytes alone and in the mix; admission never
reserves more than the cap; timestamps are ordered."""
import numpy as np
import pytest
import torch

from paper_1503_00638_gb300 import synth

pytestmark = pytest.mark.gpu

DT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_00638_gb300 import build
    build.build()
    from paper_1503_00638_gb300 import bsgpu, serve
    return bsgpu, serve


def make_requests(bs, serve, n=60, seed=0, rate=2000.0):
    rng = np.random.default_rng(seed)
    vis = synth.visibilities(synth.CONFIG_SMALL).view(np.uint8).reshape(-1)
    reqs, originals = [], {}
    t = 0.0
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        es = int(rng.choice([2, 4, 8]))
        nbytes = int(np.exp(rng.uniform(np.log(16 << 10), np.log(6 << 20)))) // es * es
        if i % 9 == 0:
            nbytes = int(rng.integers(0, 8)) * es          # tiny: no blocks
        if rng.random() < 0.5:
            a = np.resize(vis, nbytes).copy()
        else:
            a = synth.random_walk(nbytes // es, DT[es], seed=i).view(np.uint8)
        x = torch.from_numpy(a.copy()).cuda()
        B = int(rng.choice([0, 8192 // es, 2048 // es]))
        originals[i] = x
        if rng.random() < 0.7:
            reqs.append(serve.Request(i, "compress", t, x, nbytes // es, es, B))
        else:
            c = bs.compress(x, B, elem_size=es)
            stream = c.buf[:c.nbytes].clone()
            idx = c.offsets.clone() if i % 2 else None       # half carry their index
            reqs.append(serve.Request(i, "decompress", t, stream, nbytes // es, es, B, index=idx))
    torch.cuda.synchronize()
    return reqs, originals


def check(bs, reqs, results, originals):
    """Every served result against the oracle: a compressed stream must decode
    with the oracle's strict decoder to exactly the request's elements, and
    its block index must point at each block's length field; a decompressed
    result must equal the elements the stream was made from."""
    import oracle as orc
    orc.lib()
    for r in reqs:
        assert r.status == 0, r.rid
        assert r.arrival <= r.admitted <= r.done
        out, idx = results[r.rid]
        x = originals[r.rid]
        if r.kind == "compress":
            a = x.cpu().numpy().view(DT[r.elem_size])
            s = out.numpy().tobytes()
            rc, back = orc.decompress(s, r.n_elem, a.dtype, r.block_elems)
            assert rc == 0 and np.array_equal(back.view(np.uint8), a.view(np.uint8)), r.rid
            nb = bs.num_blocks(r.n_elem, r.elem_size, r.block_elems)
            pos = 12
            for b in range(nb):
                assert int(idx[b]) == pos, r.rid
                pos += 4 + int.from_bytes(s[pos:pos + 4], "big")
        else:
            assert torch.equal(out, x.cpu()), r.rid


def collector(results):
    def on_done(server, r):
        out = server.output(r).cpu()
        idx = server.output_index(r).cpu() if r.kind == "compress" else None
        results[r.rid] = (out, idx)
    return on_done


@pytest.mark.parametrize("cap_mb,depth", [(64, 2), (1024, 1), (1024, 3)])
def test_batching_server_matches_alone(mods, cap_mb, depth):
    bs, serve = mods
    reqs, originals = make_requests(bs, serve, seed=cap_mb + depth)
    results = {}
    srv = serve.BatchingServer(cap_bytes=cap_mb << 20, depth=depth, max_chunks=32,
                               on_done=collector(results))
    srv.run(reqs)
    check(bs, reqs, results, originals)
    st = srv.arena.stats()
    assert st["used"] == 0 and st["high_water"] <= srv.cap
    assert len(srv.batches) >= 1
    if cap_mb == 64:
        # the small cap forced requests to wait for earlier ones to finish
        assert len(srv.batches) > 2
    s = serve.latency_summary(reqs)
    assert s["n"] == len(reqs) and s["p50_ms"] <= s["p99_ms"]


def test_serial_server_matches_alone(mods):
    bs, serve = mods
    reqs, originals = make_requests(bs, serve, n=30, seed=5)
    results = {}
    srv = serve.SerialServer(cap_bytes=256 << 20, on_done=collector(results))
    srv.run(reqs)
    check(bs, reqs, results, originals)
    assert srv.arena.stats()["used"] == 0


def test_same_bytes_alone_and_in_the_mix(mods):
    bs, serve = mods
    reqs, originals = make_requests(bs, serve, n=40, seed=9, rate=1e6)   # all at once
    mixed = {}
    serve.BatchingServer(cap_bytes=2 << 30, on_done=collector(mixed)).run(reqs)
    for r in reqs:
        alone = {}
        solo = serve.Request(r.rid, r.kind, 0.0, r.data, r.n_elem, r.elem_size, r.block_elems,
                             index=r.index)
        serve.BatchingServer(cap_bytes=64 << 20, depth=1, on_done=collector(alone)).run([solo])
        assert torch.equal(alone[r.rid][0], mixed[r.rid][0]), r.rid
        if r.kind == "compress" and alone[r.rid][1] is not None:
            assert torch.equal(alone[r.rid][1], mixed[r.rid][1]), r.rid


def test_request_larger_than_cap_is_refused(mods):
    bs, serve = mods
    x = torch.zeros(4 << 20, dtype=torch.uint8, device="cuda")
    r = serve.Request(0, "compress", 0.0, x, x.numel() // 4, 4, 0)
    with pytest.raises(ValueError):
        serve.BatchingServer(cap_bytes=1 << 20).run([r])


def test_expired_and_cancelled_requests_leave_the_queue(mods):
    """Host-side failures of the serving loop: with a small cap, later
    requests wait behind earlier ones; those whose admission deadline passes
    while they wait, and those the client cancels, leave the queue without a
    launch (status EXPIRED / CANCELLED), and every other request completes
    with a result the oracle decodes."""
    bs, serve = mods
    reqs, originals = make_requests(bs, serve, n=40, seed=21, rate=1e6)
    for r in reqs[10::5]:
        r.deadline = r.arrival          # expires unless admitted at once
    for r in reqs[12::7]:
        r.cancelled = True
    results = {}
    srv = serve.BatchingServer(cap_bytes=16 << 20, depth=1, max_chunks=4,
                               on_done=collector(results))
    srv.run(reqs)
    gone = [r for r in reqs if r.status in (serve.EXPIRED, serve.CANCELLED)]
    assert any(r.status == serve.CANCELLED for r in gone)
    assert all(r.cancelled or r.deadline is not None for r in gone)
    assert all(r.rid not in results for r in gone)
    kept = [r for r in reqs if r not in gone]
    check(bs, kept, results, originals)
    assert srv.arena.stats()["used"] == 0
    s = serve.latency_summary(reqs)
    assert s["n"] == len(kept)
