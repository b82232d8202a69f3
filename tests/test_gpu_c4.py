"""GPU parity for C4 (key-value service over UDP, Sec. 7.3): a persistent GPU
kernel receives request batches with recvmmsg and answers with sendmmsg; every
reply's bytes equal the sequential CPU server's (the oracle replays the same
requests in client sequence order), and the table's final values match."""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    import paper_1705_06965_b300 as G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return G


@pytest.fixture(scope="module")
def ctx(G):
    c = G.Context(device=0, service_threads=8, staging_bytes=128 << 20, deadline_ns=10_000_000_000)
    yield c
    c.close()


def _port():
    return 20000 + (os.getpid() * 97) % 30000


@pytest.mark.parametrize("n_sockets,batch,rate", [(8, 64, 100_000.0), (1, 16, 50_000.0), (32, 32, 200_000.0)])
def test_c4_replies_bit_exact(G, ctx, n_sockets, batch, rate):
    p = dict(workloads.C4_SMALL, rate_per_s=rate)
    tr = workloads.kv_trace(p)
    want = oracle.c4_replay(tr)
    reqs, off = workloads.kv_request_bytes(tr)
    port = _port() + n_sockets
    srv = G.KVServer(ctx, tr.keys, tr.vlen0, tr.vseed0, n_sockets=n_sockets, batch=batch, port_base=port)
    try:
        reps, lat, st = G.kv_client(reqs, off, tr.arrival_ns, port, n_sockets)
        # final value of the most popular keys, read back from device memory
        hot = np.bincount(tr.key_idx, minlength=len(tr.keys)).argsort()[::-1][:5]
        final = {int(k): srv.value(int(k)) for k in hot}
    finally:
        served = srv.stop()
    assert st["rc"] == 0 and st["received"] == len(tr), st
    assert st["duplicates"] == 0 and st["malformed"] == 0
    bad = [j for j in range(len(tr)) if reps[j] != want[j]]
    assert not bad, (len(bad), bad[:5])
    assert served == len(tr)
    assert np.all(lat > 0)
    for k, v in final.items():
        sets = np.where((tr.key_idx == k) & (tr.op == workloads.KV_SET))[0]
        expect = (workloads.stream_bytes(int(tr.vseed[sets[-1]]), int(tr.vlen[sets[-1]])) if len(sets)
                  else tr.value0(k))
        assert v == expect


def test_c4_full_table_replies_bit_exact(G, ctx):
    """The benchmark's configuration: the 1 M-key table in HBM, 32 sockets,
    batches of 64, 100 k requests at 200 k/s offered; every reply equals the
    oracle's replay in client sequence order."""
    p = dict(workloads.C4_FULL, n_requests=100_000, rate_per_s=200_000.0)
    tr = workloads.kv_trace(p)
    want = oracle.c4_replay(tr)
    reqs, off = workloads.kv_request_bytes(tr)
    port = _port() + 101
    srv = G.KVServer(ctx, tr.keys, tr.vlen0, tr.vseed0, n_sockets=32, batch=64, port_base=port)
    try:
        reps, lat, st = G.kv_client(reqs, off, tr.arrival_ns, port, 32)
    finally:
        served = srv.stop()
    assert st["rc"] == 0 and st["received"] == len(tr), st
    bad = [j for j in range(len(tr)) if reps[j] != want[j]]
    assert not bad, (len(bad), bad[:5])
    assert served == len(tr)


def test_c4_full_table_at_800k_per_s_every_reply_bit_exact(G, ctx):
    """The benchmark's configuration at 800 k requests/s offered, where the
    server's batches fill and requests of one hot key meet in a batch (they
    are applied in arrival order): the 1 M-key table, 32 sockets, batches of
    64, 1 M requests; every reply equals the oracle's replay in client
    sequence order, and none is missing."""
    p = dict(workloads.C4_FULL, n_requests=1_000_000, rate_per_s=800_000.0)
    tr = workloads.kv_trace(p)
    want = oracle.c4_replay(tr)
    reqs, off = workloads.kv_request_bytes(tr)
    port = _port() + 201
    srv = G.KVServer(ctx, tr.keys, tr.vlen0, tr.vseed0, n_sockets=32, batch=64, port_base=port)
    try:
        reps, lat, st = G.kv_client(reqs, off, tr.arrival_ns, port, 32, timeout_ns=20_000_000_000)
        seen = srv.received(len(tr))
    finally:
        served = srv.stop()
    assert st["rc"] == 0 and st["received"] == len(tr), st
    assert st["duplicates"] == 0 and st["malformed"] == 0
    assert seen.all()  # the server's log of received requests
    bad = [j for j in range(len(tr)) if reps[j] != want[j]]
    assert not bad, (len(bad), bad[:5])
    assert served == len(tr)


def test_c4_lost_requests_are_left_out_of_the_replay(G, ctx):
    """The server logs the requests that reached it; the oracle replays
    exactly those (a lost SET must not change the expected replies of later
    GETs of its key).  The loss is made on the client side: a plain UDP
    client sends the trace in sequence order but skips every 7th request, and
    the received log must say exactly which arrived."""
    import socket
    import time
    p = dict(workloads.C4_SMALL, n_requests=3000)
    tr = workloads.kv_trace(p)
    keep = np.arange(len(tr)) % 7 != 3
    n_sockets = 8
    port = _port() + 301
    srv = G.KVServer(ctx, tr.keys, tr.vlen0, tr.vseed0, n_sockets=n_sockets, batch=32, port_base=port)
    so = socket.socket(socket.AF_INET, socket.SOCK_DGRAM)
    so.setsockopt(socket.SOL_SOCKET, socket.SO_RCVBUF, 16 << 20)
    so.settimeout(5.0)
    reps = {}
    try:
        for j in np.nonzero(keep)[0]:
            d, _ = workloads.kv_request_bytes(tr, [j])
            k0 = int.from_bytes(d[8:12], "little")
            so.sendto(d, ("127.0.0.1", port + k0 % n_sockets))
            if j % 64 == 0:
                time.sleep(0.001)      # a gentle rate: nothing is lost on the way
        while len(reps) < int(keep.sum()):
            r = so.recv(2048)
            reps[int.from_bytes(r[4:8], "little")] = r
        seen = srv.received(len(tr))
    finally:
        so.close()
        srv.stop()
    assert np.array_equal(seen, keep)
    idx = np.nonzero(seen)[0]
    want = oracle.c4_replay(tr, idx)
    bad = [int(j) for i, j in enumerate(idx) if reps[int(j)] != want[i]]
    assert not bad, (len(bad), bad[:5])
