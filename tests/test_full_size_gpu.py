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
    launch (128 x 1536 x 2000, 256 x 3072 x 5000, 1024 x 512 x 10000): whole
    triangles of two channels of every array (the 1024-input array at its
    full 10000 samples, i.e. with pair items) and random visibilities
    elsewhere."""
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
        chans = [int(rng.integers(0, f)), f - 1]
        want = oracle.to_int32(oracle.xmac(v[:, chans].cpu().numpy()))
        assert np.array_equal(o[chans].cpu().numpy(), want), (a, chans)
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


def test_fine_pfb_full_band_sampled():
    """The fine filterbank at the benchmark's size (24 coarse channels x 256
    inputs x 5000 frames, 12 taps, codes only, as timed), checked on sampled
    (coarse channel, input) streams over a run of frames each: the codes
    equal the oracle's except within the fp32 bound of a rounding boundary."""
    from synth import coarse
    Q, N, M, taps = 24, 256, 5000, 12
    S = 128 * (M + taps - 1)
    g = torch.Generator(device="cuda")
    g.manual_seed(1505)
    x = torch.empty((Q, N, S, 2), dtype=torch.int8, device="cuda")
    for q in range(Q):
        x[q] = torch.randn((N, S, 2), device="cuda", generator=g).mul_(8.0).round_().clamp_(-127, 127).to(torch.int8)
    h = coarse.kaiser_sinc_window(taps).astype(np.float32)
    scale = coarse.output_scale(h.astype(np.float64), 8.0)
    codes, _ = corr.fine_pfb(x, torch.from_numpy(h).cuda(), scale)
    torch.cuda.synchronize()
    vals = np.array([v if v < 8 else v - 16 for v in range(16)])
    rng = np.random.default_rng(5)
    checked = 0
    for q, i, m0 in [(0, 0, 0), (23, 255, M - 40), (11, 128, 2500)] + \
            [(int(a), int(b), int(c)) for a, b, c in zip(rng.integers(0, Q, 5), rng.integers(0, N, 5),
                                                         rng.integers(0, M - 40, 5))]:
        xs = x[q, i, m0 * 128:(m0 + 40 + taps - 1) * 128].cpu().numpy()[None, None]
        spec, want = oracle.fine_pfb(xs, h.astype(np.float64), scale)      # frames m0 .. m0 + 39
        got = codes[m0:m0 + 40, q * 128:(q + 1) * 128, i].cpu().numpy()
        want = want[:, :, 0]
        spec = spec[:, :, 0] * scale
        a = (np.abs(xs[0, 0, :, 0].astype(np.float64)) + np.abs(xs[0, 0, :, 1])).reshape(-1, 128)
        ah = np.abs(h.astype(np.float64)).reshape(taps, 128)
        bound = np.array([sum(a[m + p] @ ah[p] for p in range(taps)) for m in range(40)]) * 64 * 2.0 ** -24 * scale
        for part, shift, exact in (("real", 4, spec.real), ("imag", 0, spec.imag)):
            gv, wv = vals[(got >> shift) & 15], vals[(want >> shift) & 15]
            near = np.abs(np.abs(exact - np.floor(exact)) - 0.5) <= bound[:, None]
            assert ((gv == wv) | near).all(), (part, q, i, m0)
        checked += got.size
    assert checked == 8 * 40 * 128
