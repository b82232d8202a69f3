"""genesys_launch from a user's own kernels (tests/c_abi/launch_demo.cu, built
here against include/ and the library):

- GENESYS_LAUNCH_GRAPH: a work-group pwrite kernel relaunched through one
  instantiated graph with new arguments each time (other source bytes, other
  file offsets) writes exactly the bytes each launch names; the same for a
  strongly ordered kernel-grain pwrite (a cooperative graph node);
- relaxed kernel-grain calls at their own sites in one kernel (Sec. 4.1:
  a consumer whose caller is the first block to arrive, a producer whose
  caller is the last) return the right results, launch after launch, also when
  the launch flags declare another grain;
- a relaxed kernel-grain site reached twice by every block is reported (status
  word GENESYS_ST_BAD_ARGS, -EINVAL to the extra arrivals) instead of serving
  stale results silently.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    import paper_1705_06965_b300 as G
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.lib()
    return G


@pytest.fixture(scope="module")
def demo(G, tmp_path_factory):
    from paper_1705_06965_b300 import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir, libname = os.path.split(G.LIB_PATH)
    so = str(tmp_path_factory.mktemp("launch_demo") / "launch_demo.so")
    r = subprocess.run([build.nvcc(), *build.ARCH, "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-shared", "-cudart",
                        "shared", "-I", os.path.join(root, "include"),
                        os.path.join(root, "tests", "c_abi", "launch_demo.cu"), "-o", so, "-L", libdir,
                        f"-l:{libname}", "-Xlinker", f"-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    D = ctypes.CDLL(so)
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    D.launch_demo_pwrite_run.argtypes = [vp, ctypes.c_int, vp, u64, u64, u32, u32, ctypes.c_int, vp, u32]
    D.launch_demo_sites_run.argtypes = [vp, ctypes.c_int, vp, u64, u32, vp, u32]
    D.launch_demo_reuse_run.argtypes = [vp, u32, vp]
    for f in (D.launch_demo_pwrite_run, D.launch_demo_sites_run, D.launch_demo_reuse_run):
        f.restype = ctypes.c_int
    return D


GRAPH = 0x400
GRAN_GROUP = 2


@pytest.mark.parametrize("kernel_grain", [0, 1])
def test_graph_relaunch_with_new_arguments(G, demo, tmp_path, kernel_grain):
    blocks, threads, block_bytes, launches = 8, 128, 4096, 5
    with G.Context(device=0, service_threads=2, staging_bytes=8 << 20) as ctx:
        src = ctx.staging(launches * blocks * block_bytes)
        data = np.frombuffer(workloads.stream_bytes(0x5EED0A01, launches * blocks * block_bytes), np.uint8)
        ctx.host_view(src, data.size)[:] = data
        path = str(tmp_path / "g.bin")
        fd = os.open(path, os.O_CREAT | os.O_TRUNC | os.O_RDWR, 0o644)
        ret = torch.zeros(blocks, dtype=torch.int64, device="cuda")
        before = ctx.graph_launches()
        try:
            # launch i writes source piece i at file piece (launches - 1 - i): new
            # arguments on every relaunch of the one graph
            for i in range(launches):
                piece = blocks * block_bytes
                ret.zero_()
                rc = demo.launch_demo_pwrite_run(ctx.handle, fd, src + i * piece, block_bytes,
                                                 (launches - 1 - i) * piece, blocks, threads, kernel_grain,
                                                 ret.data_ptr(), GRAPH)
                assert rc == 0, G.last_error()
                got = ret.cpu().numpy()
                if kernel_grain:
                    assert np.all(got == piece)          # strong: every block receives the result
                else:
                    assert np.all(got == block_bytes)
        finally:
            os.close(fd)
        assert ctx.graph_launches() - before == launches
        assert ctx.status() == [0] * G.ST_WORDS
    out = np.fromfile(path, np.uint8)
    want = data.reshape(launches, -1)[::-1].reshape(-1)
    assert np.array_equal(out, want)


def test_relaxed_kernel_grain_sites_in_one_kernel(G, demo, tmp_path):
    blocks, n = 12, 3000
    data = np.frombuffer(workloads.stream_bytes(0x5EED0A02, n), np.uint8)
    path = str(tmp_path / "k.bin")
    with G.Context(device=0, service_threads=2, staging_bytes=1 << 20) as ctx:
        buf = ctx.staging(n)
        ret = torch.zeros(2 * blocks, dtype=torch.int64, device="cuda")
        # the first launch declares the kernel grain; the others declare
        # another grain, and GENESYS_LAUNCH_GRAPH: the sites are reset anyway
        for k, flags in enumerate((3 | 0x10, GRAN_GROUP, GRAN_GROUP | GRAPH, GRAN_GROUP | GRAPH)):
            with open(path, "wb") as f:
                f.write(data.tobytes())
            fd = os.open(path, os.O_RDWR)
            try:
                ret.zero_()
                rc = demo.launch_demo_sites_run(ctx.handle, fd, buf, n, blocks, ret.data_ptr(), flags)
                assert rc == 0, (k, G.last_error())
            finally:
                os.close(fd)
            r = ret.cpu().numpy().reshape(blocks, 2)
            assert np.all(r[:, 0] == n), k                  # consumer: every block has the pread's result
            assert sorted(r[:, 1]) == [0] * (blocks - 1) + [n], k   # producer: the last block called
            out = np.fromfile(path, np.uint8)
            assert out.size == 2 * n and np.array_equal(out[n:], data), k
            assert ctx.status() == [0] * G.ST_WORDS


def test_reused_relaxed_kernel_grain_site_is_reported(G, demo):
    blocks = 6
    with G.Context(device=0, service_threads=2, staging_bytes=1 << 20) as ctx:
        ret = torch.zeros(2 * blocks, dtype=torch.int64, device="cuda")
        assert demo.launch_demo_reuse_run(ctx.handle, blocks, ret.data_ptr()) == 0, G.last_error()
        st = ctx.status()
        r = ret.cpu().numpy()
        # 2 * blocks arrivals at a site that serves `blocks`: the extra ones are refused
        assert st[G.ST_BAD_ARGS] == blocks and st[G.ST_FIRST_ERROR] == -22
        assert int((r == -22).sum()) == blocks
        assert int((r == os.getpid()).sum()) == blocks
