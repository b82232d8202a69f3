"""GPU parity for C6 (block permutation + work-group pwrite, Sec. 6 / Fig. 6):
the written file equals the oracle's for every ordering x blocking mode."""
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
    c = G.Context(device=0, service_threads=4, staging_bytes=64 << 20)
    yield c
    c.close()


@pytest.mark.parametrize("relaxed,nonblocking", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("n_blocks,iters", [(1, 0), (37, 1), (300, 5), (2048, 16)])
def test_c6_permute_matches_oracle(G, ctx, tmp_path, relaxed, nonblocking, n_blocks, iters):
    data, perm = workloads.c6_inputs(n_blocks)
    want_p = str(tmp_path / "want.bin")
    oracle.c6_permute(data, perm, iters, want_p)
    d_in = torch.from_numpy(data).cuda()
    d_perm = torch.from_numpy(perm.view(np.int16)).cuda()
    ctx.staging_reset()
    st = ctx.staging(n_blocks * 8192)
    got_p = str(tmp_path / "got.bin")
    fd = os.open(got_p, os.O_CREAT | os.O_TRUNC | os.O_WRONLY, 0o644)
    try:
        ctx.c6_permute(fd, d_in.data_ptr(), d_perm.data_ptr(), n_blocks, iters, relaxed, nonblocking, st,
                       n_blocks * 8192)
    finally:
        os.close(fd)
    assert open(got_p, "rb").read() == open(want_p, "rb").read()
