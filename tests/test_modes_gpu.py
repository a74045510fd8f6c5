"""The incoherent beam and the output remap (with channel and dump
averaging) against the oracle, element by element."""
import numpy as np
import pytest
import torch

import oracle
from paper_1501_05992_gb300 import corr
from synth import voltgen as vg
from synth.gpu import DeviceGenerator

pytestmark = pytest.mark.gpu


def _rand(shape, seed):
    return np.random.default_rng(seed).integers(0, 256, shape, dtype=np.uint8)


@pytest.mark.parametrize("shape,n_avg", [((36, 5, 48), 1), ((36, 5, 48), 4), ((20, 3, 13), 5),
                                         ((7, 300, 256), 7), ((1, 1, 1), 1),
                                         # 1, 2, 4, 8 and 32 lanes per row (2 chunks a lane at 1024),
                                         # 13 chunks a row, a block's 128 channels and a ragged rest
                                         ((8, 300, 16), 2), ((6, 50, 96), 3), ((4, 33, 64), 1),
                                         ((9, 130, 128), 3), ((5, 70, 512), 5), ((3, 40, 1024), 1),
                                         ((5, 20, 208), 5)])
@pytest.mark.parametrize("zero_invalid", [False, True])
def test_beam_exact(shape, n_avg, zero_invalid):
    volt = _rand(shape, sum(shape) + n_avg)
    volt.reshape(-1)[::11] = 0x88
    volt.reshape(-1)[5::13] = 0x38
    got = corr.incoherent_beam(torch.from_numpy(volt).cuda(), n_avg, zero_invalid).cpu().numpy()
    want = oracle.beam(volt, n_avg, zero_invalid)
    assert np.array_equal(got, want)


def test_beam_full_band_sampled_channels():
    N, F, T = 256, 3072, 5000
    volt = DeviceGenerator(vg.gauss3_params(1503, N, F)).make(0, T)
    got = corr.incoherent_beam(volt, 1).cpu().numpy()
    torch.cuda.synchronize()
    chans = [0, 1, 1535, 3071]
    sub = volt[:, chans].cpu().numpy()
    want = oracle.beam(sub, 1)
    assert np.array_equal(got[:, chans], want)


def test_beam_arguments():
    v = torch.zeros((10, 2, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        corr.incoherent_beam(v, 3)


def _tri_of(volt_np, path="auto"):
    T, F, N = volt_np.shape
    c = corr.Correlator(N, F, max(T, 1), path=path)
    out = c.integrate(torch.from_numpy(volt_np).cuda())
    c.sync()
    c.close()
    return out


@pytest.mark.parametrize("N,F,T", [(8, 4, 30), (128, 6, 200), (70, 2, 33)])
@pytest.mark.parametrize("f_avg,n_dumps", [(1, 1), (2, 2), (1, 3), (3, 2), (1, 8)])
def test_remap_exact_custom_order(N, F, T, f_avg, n_dumps):
    if F % f_avg:
        pytest.skip("channels not divisible")
    rng = np.random.default_rng(N + F + T + f_avg + n_dumps)
    perm = rng.permutation(N).astype(np.int32)
    volts = [_rand((T, F, N), 7 * d + N) for d in range(n_dumps)]
    tris = [_tri_of(v) for v in volts]
    got = corr.remap(tris, torch.from_numpy(perm).cuda(), f_avg=f_avg).cpu().numpy()
    want = oracle.remap(np.stack([oracle.xmac(v) for v in volts]), perm, f_avg=f_avg)
    assert np.array_equal(got, oracle.to_int32(want))


def test_remap_default_pfb_order_full_channel():
    N, F, T = 256, 4, 300
    volt = _rand((T, F, N), 77)
    tri = _tri_of(volt)
    got = corr.remap(tri).cpu().numpy()
    want = oracle.remap(oracle.xmac(volt), oracle.pfb_order(N))
    assert got.shape == (F, 128 * 129 // 2, 2, 2, 2)
    assert got[0].size // 2 == 33024                      # products per channel (Section 3.4.3)
    assert np.array_equal(got, oracle.to_int32(want))


def test_remap_arguments():
    t = torch.zeros((2, 70 * 71 // 2, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(corr.CorrError):
        corr.remap(t)                                         # default order needs whole PFBs
    with pytest.raises(corr.CorrError):
        corr.remap(t, torch.arange(70, dtype=torch.int32, device="cuda"), f_avg=3)


@pytest.mark.parametrize("path", ["cudacore", "mma_i8", "tc_fp8"])
def test_integrate_beam_exact(path):
    """corr_integrate_beam: the triangle and the incoherent beam of the same
    samples, both equal to the oracle's; on the tensor-core path the beam
    comes from the X-engine's own unpack (pair and single items, a padded
    input count, block averages, the invalid-code reading)."""
    cases = [(256, 6, 4160, 1, False), (256, 3, 700, 5, False), (384, 2, 4096, 64, True),
             (65, 3, 300, 3, False), (128, 4, 1000, 1, True)]
    ran = 0
    for N, F, T, n_avg, zi in cases:
        try:
            c = corr.Correlator(N, F, T, path=path, zero_invalid=zi)
        except corr.CorrError as e:
            if e.status == corr.CORR_E_UNSUPPORTED:
                continue
            raise
        rng = np.random.default_rng(N + F + T + n_avg)
        volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
        d = torch.from_numpy(volt).cuda()
        tri, beam = c.integrate_beam(d, n_avg)
        c.sync()
        c.close()
        assert np.array_equal(tri.cpu().numpy(), oracle.to_int32(oracle.xmac(volt, zero_invalid=zi))), (N, F, T)
        assert np.array_equal(beam.cpu().numpy(), oracle.beam(volt, n_avg, zero_invalid=zi)), (N, F, T, n_avg)
        ran += 1
    assert ran


def test_integrate_beam_long_and_extreme():
    """A 40000-sample integration (two tensor-core launches, the beam's second
    half offset by the first launch's samples) of all -8-8i samples: the
    largest power per sample, 128 per input."""
    N, F, T = 128, 2, 40000
    c = corr.Correlator(N, F, T, path="auto")
    volt = np.full((T, F, N), 0x88, np.uint8)
    volt[::3, 1, ::5] = 0x77
    d = torch.from_numpy(volt).cuda()
    tri, beam = c.integrate_beam(d, 8)
    c.sync()
    c.close()
    assert np.array_equal(beam.cpu().numpy(), oracle.beam(volt, 8))
    assert np.array_equal(tri.cpu().numpy(), oracle.to_int32(oracle.xmac(volt)))
