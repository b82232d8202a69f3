"""GPU parity for C3 (wordcount over many files, Sec. 7.1): the persistent
pread + scan kernel against the CPU oracle, bit-exact, at small sizes with
tokens cut by every chunk boundary, and at the full configuration (2,000 files,
~2.8 GiB) against the generator's recorded ground truth (which the oracle is
pinned to)."""
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
    c = G.Context(device=0, service_threads=8, staging_bytes=1 << 30, deadline_ns=10_000_000_000)
    yield c
    c.close()


def run_c3(ctx, paths, queries, chunk, ctas, threads, form):
    fds = [os.open(p, os.O_RDONLY) for p in paths]
    sizes = [os.path.getsize(p) for p in paths]
    counts = torch.zeros(len(queries), dtype=torch.int64, device="cuda")
    try:
        ctx.staging_reset()
        need = ctas * (chunk + 64) * 2
        st = ctx.staging(need)
        ctx.c3_wordcount(fds, sizes, queries, counts.data_ptr(), st, need, chunk=chunk, ctas=ctas,
                         threads=threads, form=form)
    finally:
        for fd in fds:
            os.close(fd)
    return counts.cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("chunk,ctas,threads", [(64, 7, 32), (4096, 148, 256), (1 << 20, 296, 512), (4000, 3, 1024)])
def test_c3_small_corpus(ctx, form, chunk, ctas, threads):
    c = workloads.corpus(workloads.C3_SMALL)
    want, _ = oracle.c3_wordcount(c.paths, c.queries, chunk=4096)
    got = run_c3(ctx, c.paths, c.queries, chunk, ctas, threads, form)
    assert np.array_equal(got, want)
    assert ctx.status() == [0] * 8


EDGE_FILES = [
    b"", b" ", b"\n\n  \n", b"cat", b"cat ", b" cat", b"cat\ncat cat\n\ncat", b"catcat cat cat1 ca t",
    b"abcdefghijklmnopqrstuvwxyz cat abcdefghijklmnop cat", b"abcdefghijklmnop",
    b"abcdefghijklmnopq abcdefghijklmnop", b"t " * 100 + b"ca" + b"t" * 3,
]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("chunk", [64, 80, 4096])
def test_c3_edge_files(ctx, tmp_path, form, chunk):
    paths = []
    for i, data in enumerate(EDGE_FILES):
        p = tmp_path / f"e{i}.txt"
        p.write_bytes(data)
        paths.append(str(p))
    queries = [b"cat", b"ca", b"t", b"abcdefghijklmnop", b"dog", b"catcat", b"cat1"]
    want, _ = oracle.c3_wordcount(paths, queries, chunk=7)
    got = run_c3(ctx, paths, queries, chunk, 4, 64, form)
    assert np.array_equal(got, want)


def test_c3_long_tokens_across_boundaries(ctx, tmp_path):
    # tokens of every length 1..40 at every alignment against 64-byte chunks
    rng = np.random.default_rng(11)
    words = [bytes(rng.integers(97, 100, n, dtype=np.uint8)) for n in range(1, 41)]
    data = b" ".join(words[i % 40] for i in range(3000))
    p = tmp_path / "long.txt"
    p.write_bytes(data)
    queries = sorted({w for w in words if len(w) <= 16})[:64]
    want, _ = oracle.c3_wordcount([str(p)], queries, chunk=13)
    for form in (0, 1):
        got = run_c3(ctx, [str(p)], queries, 64, 5, 32, form)
        assert np.array_equal(got, want)


def test_c3_bad_arguments(ctx, G, tmp_path):
    p = tmp_path / "x.txt"
    p.write_bytes(b"a b c")
    with pytest.raises(G.GenesysError) as e:
        run_c3(ctx, [str(p)], [b"a" * 17], 4096, 1, 32, 1)
    assert e.value.code == G.EINVAL
    with pytest.raises(G.GenesysError):
        run_c3(ctx, [str(p)], [b"a"], 100, 1, 32, 1)       # chunk not a multiple of 16


def test_c3_full_config_ground_truth(ctx):
    """2,000 files, lognormal sizes (median 256 KiB, cap 64 MiB), Zipf(1.1) over
    50k words, 64 queries: counts equal the generator's recorded emissions."""
    c = workloads.corpus(workloads.C3_FULL)
    got = run_c3(ctx, c.paths, c.queries, 1 << 20, 296, 512, 1)
    assert np.array_equal(got, c.truth_total())
    # sampled files against the oracle itself
    idx = list(range(0, 2000, 97))
    want, _ = oracle.c3_wordcount([c.paths[i] for i in idx], c.queries, chunk=1 << 20)
    got_s = run_c3(ctx, [c.paths[i] for i in idx], c.queries, 256 << 10, 148, 512, 0)
    assert np.array_equal(got_s, want)
