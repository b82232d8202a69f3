"""GPU UDP echo server (Sec. 7.3, Fig. 10): a persistent kernel, one block per
socket, receives datagrams with recvfrom (the paper's work-group, blocking,
weak form) or recvmmsg batches, copies them through the SMs and sends them
back.  Every reply must equal its datagram byte for byte (the closed-loop
client compares them), none may be lost, and the server's own count must
match the client's."""
import os

import pytest

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
    c = G.Context(device=0, service_threads=4, staging_bytes=96 << 20, deadline_ns=10_000_000_000)
    yield c
    c.close()


def _port(k):
    return 22000 + (os.getpid() * 53 + 211 * k) % 27000


# packet sizes: the 8-byte minimum, a ragged size (not a multiple of 16),
# a common MTU-sized one and the largest
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("packet", [8, 1000, 1500, 65504])
def test_echo_bytes_exact(G, ctx, form, packet):
    n_sockets, n = 4, 3000
    port = _port(form * 7 + packet % 13)
    srv = G.EchoServer(ctx, n_sockets=n_sockets, max_packet=packet, form=form, batch=8, threads=256, port_base=port)
    try:
        st = G.echo_client(port, n_sockets, packet, n, window=4, threads=2)
    finally:
        got = srv.stop()
    assert st["sent"] == n and st["echoed"] == n, st
    assert st["bad"] == 0 and st["lost"] == 0 and st["send_errors"] == 0, st
    assert got["packets"] == n and got["bytes"] == n * packet, got
    status = ctx.status()
    assert status[0] == 0 and status[1] == 0, status


def test_echo_stops_when_idle(G, ctx):
    """No traffic at all: genesys_echo_stop ends the idle blocks at once."""
    import time
    srv = G.EchoServer(ctx, n_sockets=2, max_packet=256, form=1, port_base=_port(99))
    t = time.time()
    got = srv.stop(timeout_ns=5_000_000_000)
    assert got == {"packets": 0, "bytes": 0}
    assert time.time() - t < 2.0


def test_echo_rejects_bad_arguments(G, ctx):
    with pytest.raises(G.GenesysError):
        G.EchoServer(ctx, n_sockets=1, max_packet=G.ECHO_PACKET_MAX + 16, port_base=_port(98))
    with pytest.raises(G.GenesysError):
        G.EchoServer(ctx, n_sockets=1, max_packet=4, port_base=_port(97))
    with pytest.raises(G.GenesysError):
        G.EchoServer(ctx, n_sockets=1, form=1, batch=G.ECHO_MAX_BATCH + 1, port_base=_port(96))


def test_a_context_with_a_running_server_is_not_shut_down(G):
    """genesys_shutdown refuses (and frees nothing) while a server kernel runs
    on the context; once the server is stopped the context closes."""
    c = G.Context(device=0, service_threads=2, staging_bytes=8 << 20)
    with G.EchoServer(c, n_sockets=1, max_packet=256, form=0, port_base=_port(95)) as srv:
        with pytest.raises(G.GenesysError):
            c.close()
        st = G.echo_client(srv.port_base, 1, 64, 50, window=2, threads=1)   # still served
        assert st["echoed"] == 50, st
    c.close()
    with pytest.raises(RuntimeError):
        c.handle
