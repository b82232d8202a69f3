"""The oracle's plain UDP servers (Sec. 7.3: an echo server whose packets can
be processed on the CPU, and the key-value service) exercised on the host,
no GPU: the echo server's replies equal the datagrams byte for byte (checked
by the closed-loop client), and the key-value server's replies equal the
sequential replay of the same requests in client sequence order."""
import os

import numpy as np
import pytest

import oracle
import workloads


@pytest.fixture(scope="module")
def G():
    import paper_1705_06965_b300 as G
    G.lib()  # the host-only load generators; no device needed
    return G


def _port(k):
    return 21000 + (os.getpid() * 131 + 977 * k) % 28000


@pytest.mark.parametrize("packet,threads,window", [(8, 1, 1), (100, 2, 4), (1500, 2, 8), (65504, 1, 2)])
def test_oracle_echo_identity(G, packet, threads, window):
    port, n_sockets = _port(packet % 97), 4
    srv = oracle.UdpServer("echo", port, n_sockets, threads=threads, idle_ns=5_000_000_000)
    try:
        st = G.echo_client(port, n_sockets, packet, 2000, window=window, threads=2)
    finally:
        got = srv.join()
    assert st["sent"] == 2000 and st["echoed"] == 2000, st
    assert st["bad"] == 0 and st["lost"] == 0 and st["send_errors"] == 0
    assert st["bytes"] == 2000 * packet
    assert got["answered"] == 2000 and got["bytes"] == 2000 * packet


def test_oracle_echo_catches_a_corrupted_reply(G):
    """The client's byte check is what pins the echo: a server that flips a
    byte of every reply gets every reply counted bad."""
    import socket
    import threading
    port, n = _port(3), 1
    so = socket.socket(socket.AF_INET, socket.SOCK_DGRAM)
    so.bind(("127.0.0.1", port))
    so.settimeout(5.0)

    def bad_server():
        while True:
            data, addr = so.recvfrom(70000)
            if len(data) == 4:
                return
            b = bytearray(data)
            b[-1] ^= 0x01
            so.sendto(bytes(b), addr)

    th = threading.Thread(target=bad_server, daemon=True)
    th.start()
    st = G.echo_client(port, n, 64, 50, window=1, threads=1)
    th.join(10)
    so.close()
    assert st["echoed"] == 0 and st["bad"] == 50, st


@pytest.mark.parametrize("n_sockets", [1, 8])
def test_oracle_kv_server_equals_replay(G, n_sockets):
    p = dict(workloads.C4_SMALL, n_requests=6000, rate_per_s=200_000.0)
    tr = workloads.kv_trace(p)
    want = oracle.c4_replay(tr)
    reqs, off = workloads.kv_request_bytes(tr)
    port = _port(50 + n_sockets)
    srv = oracle.UdpServer("kv", port, n_sockets, trace=tr, idle_ns=5_000_000_000)
    try:
        reps, lat, st = G.kv_client(reqs, off, tr.arrival_ns, port, n_sockets, timeout_ns=10_000_000_000)
    finally:
        got = srv.join()
    assert st["rc"] == 0 and st["received"] == len(tr), st
    bad = [j for j in range(len(tr)) if reps[j] != want[j]]
    assert not bad, (len(bad), bad[:5])
    assert got["answered"] == len(tr)
    assert np.all(lat > 0)


def test_values0_table_matches_stream():
    tr = workloads.kv_trace(dict(workloads.C4_SMALL, n_keys=300, n_requests=10))
    T = tr.values0_table()
    for i in range(300):
        v = tr.value0(i)
        assert T[i, :len(v)].tobytes() == v and not T[i, len(v):].any()


def test_kv_client_refuses_offsets_that_do_not_describe_the_requests():
    """The load generator reads request j at reqs[req_off[j]:req_off[j + 1]]:
    offsets that do not cover n requests of at least a header each are
    refused before anything is sent."""
    import paper_1705_06965_b300 as G
    reqs = bytes(48)
    with pytest.raises(ValueError):
        G.kv_client(reqs, [0, 24], [0, 0], 47999, 1)          # n + 1 offsets needed
    with pytest.raises(ValueError):
        G.kv_client(reqs, [0, 24, 72], [0, 0], 47999, 1)      # runs past the bytes
    with pytest.raises(ValueError):
        G.kv_client(reqs, [0, 8, 48], [0, 0], 47999, 1)       # shorter than a header
