"""Full-size workloads in the launch configuration the benchmark times
(captured whole-integration graphs over a batch), checked on sampled outputs
the oracle computes one by one, plus channel sharding over two contexts and
guard bytes around every output buffer."""
import numpy as np
import pytest
import torch

import oracle
from paper_1501_05992_gb300 import corr
from synth import voltgen as vg
from synth.gpu import DeviceGenerator

from _gpu import path_available

pytestmark = pytest.mark.gpu


def _pairs(rng, n, k):
    i = rng.integers(0, n, k)
    j = (rng.random(k) * (i + 1)).astype(np.int64)
    return i, j


def test_full_band_graph_sampled():
    """256 inputs x 3072 channels x 5000 samples (one integration of the
    benchmark's full-band step), replayed from a captured graph: whole
    triangles of four channels and 64 random visibilities elsewhere."""
    N, F, T = 256, 3072, 5000
    volt = DeviceGenerator(vg.gauss3_params(1503, N, F)).make(0, T)
    b = corr.Batch([{"n_inputs": N, "n_chan": F, "n_time_per_int": T}])
    s = torch.cuda.Stream()
    graph, outs = b.capture([volt], stream=s)
    graph.launch(s)
    s.synchronize()
    tri = outs[0]
    chans = [0, 1, 1777, 3071]
    got = tri[chans].cpu().numpy()
    sub = volt[:, chans].cpu().numpy()
    assert np.array_equal(got, oracle.to_int32(oracle.xmac(sub)))
    rng = np.random.default_rng(3)
    fs = rng.integers(0, F, 64)
    i, j = _pairs(rng, N, 64)
    host = tri.cpu().numpy()
    for f, a, c in zip(fs, i, j):
        col = volt[:, int(f):int(f) + 1].cpu().numpy()
        want = oracle.xmac_pair(col, 0, int(a), int(c))
        assert tuple(host[f, a * (a + 1) // 2 + c]) == want, (f, a, c)
    graph.close()
    b.close()


def test_uneven_batch_full_sizes_sampled():
    """The three arrays of the uneven batch at full size in one persistent
    launch (128 x 1536 x 2000, 256 x 3072 x 5000, 1024 x 512 x 10000)."""
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    arrays = [(128, 1536, 2000), (256, 3072, 5000), (1024, 512, 10000)]
    volts = [DeviceGenerator(vg.gauss3_params(1504, n, f, array=a)).make(0, t)
             for a, (n, f, t) in enumerate(arrays)]
    b = corr.Batch([{"n_inputs": n, "n_chan": f, "n_time_per_int": t} for n, f, t in arrays])
    outs = b.integrate(volts)
    b.sync()
    rng = np.random.default_rng(4)
    for a, ((n, f, t), v, o) in enumerate(zip(arrays, volts, outs)):
        host = o.cpu().numpy()
        fs = rng.integers(0, f, 24)
        i, j = _pairs(rng, n, 24)
        for ff, x, y in zip(fs, i, j):
            col = v[:, int(ff):int(ff) + 1].cpu().numpy()
            assert tuple(host[ff, x * (x + 1) // 2 + y]) == oracle.xmac_pair(col, 0, int(x), int(y)), (a, ff, x, y)
    b.close()


def test_channel_sharding_over_two_contexts():
    """Channels are independent (the paper spreads them over hosts): two
    contexts on halves of the channels give the one-context result."""
    N, F, T = 256, 64, 900
    volt = torch.from_numpy(np.random.default_rng(5).integers(0, 256, (T, F, N), dtype=np.uint8)).cuda()
    whole = corr.Correlator(N, F, T).integrate(volt)
    halves = []
    for lo, hi in ((0, 24), (24, 64)):
        c = corr.Correlator(N, hi - lo, T)
        halves.append(c.integrate(volt[:, lo:hi].contiguous()))
        c.sync()
        c.close()
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(halves), whole)


GUARD = 4096


def _guarded(shape, dtype):
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * GUARD,), -77 if dtype == torch.int32 else 0x5A, dtype=dtype, device="cuda")
    return buf, buf[GUARD:GUARD + n].view(shape)


def _guards_intact(buf, dtype):
    fill = -77 if dtype == torch.int32 else 0x5A
    return bool((buf[:GUARD] == fill).all()) and bool((buf[-GUARD:] == fill).all())


@pytest.mark.parametrize("path", ["cudacore", "mma_i8", "tc_fp8"])
def test_outputs_stay_inside_their_buffers(path):
    N, F, T = 144, 5, 333
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    volt = torch.from_numpy(np.random.default_rng(6).integers(0, 256, (T, F, N), dtype=np.uint8)).cuda()
    P = N * (N + 1) // 2
    c = corr.Correlator(N, F, T, path=path)
    b1, o1 = _guarded((F, P, 2), torch.int32)
    c.integrate(volt, o1)
    b2, o2 = _guarded((F, P, 2), torch.int32)
    c.accumulate(volt[:100])
    c.accumulate(volt[100:])
    c.dump(o2)
    c.sync()
    want = oracle.to_int32(oracle.xmac(volt.cpu().numpy()))
    assert np.array_equal(o1.cpu().numpy(), want) and np.array_equal(o2.cpu().numpy(), want)
    assert _guards_intact(b1, torch.int32) and _guards_intact(b2, torch.int32)
    c.close()


def test_mode_outputs_stay_inside_their_buffers():
    N, F, T = 128, 6, 40
    volt = torch.from_numpy(np.random.default_rng(7).integers(0, 256, (T, F, N), dtype=np.uint8)).cuda()
    bb, ob = _guarded((T // 4, F), torch.int32)
    corr.incoherent_beam(volt, 4, out=ob)
    tri = corr.Correlator(N, F, T).integrate(volt)
    S = N // 2
    br, orr = _guarded((F // 2, S * (S + 1) // 2, 2, 2, 2), torch.int32)
    corr.remap([tri, tri], None, 2, out=orr)
    torch.cuda.synchronize()
    assert _guards_intact(bb, torch.int32) and _guards_intact(br, torch.int32)
    assert np.array_equal(ob.cpu().numpy(), oracle.beam(volt.cpu().numpy(), 4))
