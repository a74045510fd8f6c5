"""Parity of every X-engine path with the CPU oracle (bit-exact: the method is
exact integer arithmetic, so the tolerance is zero)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from synth import voltgen as vg
from paper_1501_05992_gb300 import corr

from _gpu import ALL_PATHS, correlate, path_available

pytestmark = pytest.mark.gpu


def _paths_for(n_inputs):
    return [p for p in ALL_PATHS if path_available(p, n_inputs)]


@pytest.fixture(scope="module")
def small_volt():
    name = "small"
    recipe, seed, arrays, _ = vg.WORKLOADS[name]
    spec = arrays[0]
    p = vg.make_params(recipe, seed, spec)
    return vg.generate(p, 0, spec.n_time)


@pytest.fixture(scope="module")
def coarse_volt():
    recipe, seed, arrays, _ = vg.WORKLOADS["coarse_channel"]
    spec = arrays[0]
    p = vg.make_params(recipe, seed, spec)
    volt = vg.generate(p, 0, spec.n_time)
    return volt, oracle.to_int32(oracle.xmac(volt))


@pytest.mark.parametrize("path", ALL_PATHS)
def test_small_workload_exact(path, small_volt):
    if not path_available(path, small_volt.shape[2]):
        pytest.skip(f"{path} unsupported for N={small_volt.shape[2]}")
    want = oracle.to_int32(oracle.xmac(small_volt))
    got = correlate(small_volt, path)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("path", ALL_PATHS)
def test_coarse_channel_workload_exact(path, coarse_volt):
    volt, want = coarse_volt
    if not path_available(path, volt.shape[2]):
        pytest.skip(f"{path} unsupported")
    got = correlate(volt, path)
    assert np.array_equal(got, want)


ODD_SHAPES = [(1, 1, 1), (2, 3, 31), (3, 2, 63), (17, 3, 65), (16, 1, 1), (32, 2, 97),
              (64, 2, 100), (65, 2, 129), (128, 1, 255), (130, 1, 257), (144, 2, 300),
              (192, 1, 130), (256, 1, 4097)]


@pytest.mark.parametrize("path", ALL_PATHS)
@pytest.mark.parametrize("shape", ODD_SHAPES, ids=lambda s: "N%d_F%d_T%d" % s)
def test_odd_shapes_exact(path, shape):
    N, F, T = shape
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported for N={N}")
    rng = np.random.default_rng(N * 1000 + F * 10 + T)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)     # every code, including 8
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, path), want)


@pytest.mark.parametrize("path", ALL_PATHS)
def test_extreme_values_exact(path):
    """All samples -8-8i (the largest magnitude), then alternating extremes."""
    N, F, T = 64, 2, 3000
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    volt = np.full((T, F, N), 0x88, np.uint8)
    volt[1::2, :, ::2] = 0x77
    volt[::3, 1, 1::2] = 0x87
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, path), want)


@pytest.mark.parametrize("path", ALL_PATHS)
def test_zero_invalid_exact(path):
    N, F, T = 48, 3, 200
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    rng = np.random.default_rng(5)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt, zero_invalid=True))
    assert np.array_equal(correlate(volt, path, zero_invalid=True), want)


@pytest.mark.parametrize("path", ALL_PATHS)
def test_split_accumulate_and_dump_resets(path):
    N, F, T = 96, 4, 1000
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    rng = np.random.default_rng(7)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt))
    got = correlate(volt, path, chunks=[(0, 300), (300, 301), (301, 333), (333, 1000)])
    assert np.array_equal(got, want)

    c = corr.Correlator(N, F, T, path=path)
    vt = torch.from_numpy(volt).cuda()
    c.accumulate(vt[:500])
    first = c.dump().cpu().numpy()
    assert np.array_equal(first, oracle.to_int32(oracle.xmac(volt[:500])))
    assert c.samples == 0
    empty = c.dump().cpu().numpy()
    assert not empty.any(), "an empty integration must dump zeros"
    c.accumulate(vt[500:])
    second = c.dump().cpu().numpy()
    assert np.array_equal(second, oracle.to_int32(oracle.xmac(volt[500:])))
    c.sync()
    c.close()


@pytest.mark.parametrize("path", ALL_PATHS)
def test_host_buffers_exact(path):
    N, F, T = 64, 5, 1234
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    rng = np.random.default_rng(8)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, path, host=True), want)
    assert np.array_equal(correlate(volt, path, host=True, chunks=[(0, 1), (1, 1234)]), want)


@pytest.mark.parametrize("path", ALL_PATHS)
def test_back_to_back_host_integrations(path):
    """Host dumps run on the context's output stream while the next
    integration is already being correlated: every dump must still hold its
    own integration, including a device dump and a state restore that follow
    a host dump without any synchronisation in between."""
    N, F, T = 128, 6, 1700
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    rng = np.random.default_rng(81)
    volts = [rng.integers(0, 256, (T, F, N), dtype=np.uint8) for _ in range(4)]
    wants = [oracle.to_int32(oracle.xmac(v)) for v in volts]
    hv = [torch.from_numpy(v).pin_memory() for v in volts]
    P = N * (N + 1) // 2
    outs = [torch.full((F, P, 2), -5, dtype=torch.int32).pin_memory() for _ in range(3)]
    d3 = torch.from_numpy(volts[3]).cuda()
    c = corr.Correlator(N, F, T, path=path)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    c.accumulate_host(hv[0], stream=s)
    c.dump_host(outs[0], stream=s)
    c.accumulate_host(hv[1][:900], stream=s)
    c.accumulate_host(hv[1][900:], stream=s)
    c.dump_host(outs[1], stream=s)
    c.accumulate_host(hv[2], stream=s)
    dv = c.dump(stream=s)                        # device dump right after a host dump
    c.accumulate(d3, stream=s)
    c.dump_host(outs[2], stream=s)
    c.sync(s)
    assert np.array_equal(outs[0].numpy(), wants[0])
    assert np.array_equal(outs[1].numpy(), wants[1])
    assert np.array_equal(dv.cpu().numpy(), wants[2])
    assert np.array_equal(outs[2].numpy(), wants[3])
    # a restore right after a host dump must not race the copy out
    c.accumulate_host(hv[0][:1000], stream=s)
    state = c.get_state(stream=s)
    c.dump_host(outs[0], stream=s)
    c.set_state(state, stream=s)
    c.accumulate_host(hv[0][1000:], stream=s)
    c.dump_host(outs[1], stream=s)
    c.sync(s)
    assert np.array_equal(outs[0].numpy(), oracle.to_int32(oracle.xmac(volts[0][:1000])))
    assert np.array_equal(outs[1].numpy(), wants[0])
    c.close()


@pytest.mark.parametrize("path", ALL_PATHS)
def test_empty_host_dump_right_after_a_host_dump(path):
    """A host dump of an empty integration zeroes the accumulators; it must not
    do so while the previous host dump's copy is still reading them."""
    N, F, T = 256, 48, 1500
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    volt = np.random.default_rng(82).integers(0, 256, (T, F, N), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt))
    P = N * (N + 1) // 2
    outs = [torch.full((F, P, 2), -5, dtype=torch.int32).pin_memory() for _ in range(2)]
    c = corr.Correlator(N, F, T, path=path)
    s = torch.cuda.Stream()
    for _ in range(3):
        c.accumulate_host(torch.from_numpy(volt).pin_memory(), stream=s)
        c.dump_host(outs[0], stream=s)
        c.dump_host(outs[1], stream=s)           # nothing accumulated since: all zeros
        c.sync(s)
        assert np.array_equal(outs[0].numpy(), want)
        assert not outs[1].numpy().any()
    c.close()


@pytest.mark.parametrize("path", ALL_PATHS)
def test_integrate_exact_and_leaves_running_integration(path):
    """corr_integrate writes one whole integration straight to the output and
    does not disturb an integration that is being accumulated meanwhile."""
    N, F, T = 128, 5, 1700
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    rng = np.random.default_rng(91)
    a_np = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    b_np = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    a, b = torch.from_numpy(a_np).cuda(), torch.from_numpy(b_np).cuda()
    c = corr.Correlator(N, F, T, path=path)
    c.accumulate(a[:600])
    got_b = c.integrate(b).cpu().numpy()
    assert c.samples == 600
    c.accumulate(a[600:])
    got_a = c.dump().cpu().numpy()
    zeros = c.integrate(b[:0]).cpu().numpy()
    c.sync()
    assert np.array_equal(got_b, oracle.to_int32(oracle.xmac(b_np)))
    assert np.array_equal(got_a, oracle.to_int32(oracle.xmac(a_np)))
    assert not zeros.any()
    with pytest.raises(corr.CorrError) as e:
        c.integrate(torch.zeros((T + 1, F, N), dtype=torch.uint8, device="cuda"))
    assert e.value.status == corr.CORR_E_OVERFLOW
    c.close()


def test_integrate_long_splits_launches():
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    N, F, T = 128, 2, 40000
    volt = np.full((T, F, N), 0x77, np.uint8)
    volt[::7] = 0x99
    c = corr.Correlator(N, F, T, path="tc_fp8")
    got = c.integrate(torch.from_numpy(volt).cuda()).cpu().numpy()
    c.sync()
    c.close()
    assert np.array_equal(got, oracle.to_int32(oracle.xmac(volt)))


def test_overflow_and_state_errors():
    c = corr.Correlator(16, 2, 100, path="cudacore")
    v = torch.zeros((60, 2, 16), dtype=torch.uint8, device="cuda")
    c.accumulate(v)
    with pytest.raises(corr.CorrError) as e:
        c.accumulate(v)
    assert e.value.status == corr.CORR_E_OVERFLOW
    assert c.samples == 60
    with pytest.raises(corr.CorrError) as e:
        c.set_path("mma_i8")
    assert e.value.status == corr.CORR_E_STATE
    with pytest.raises(ValueError):
        c.accumulate(torch.zeros((4, 3, 16), dtype=torch.uint8, device="cuda"))
    c.dump()
    c.set_path("mma_i8")
    c.sync()
    c.close()


@pytest.mark.parametrize("path", ALL_PATHS)
def test_checkpoint_resume(path):
    N, F, T = 64, 3, 800
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    rng = np.random.default_rng(9)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    vt = torch.from_numpy(volt).cuda()
    a = corr.Correlator(N, F, T, path=path)
    a.accumulate(vt[:333])
    state = a.get_state()
    a.close()
    b = corr.Correlator(N, F, T, path=path)
    b.set_state(state)
    assert b.samples == 333
    b.accumulate(vt[333:])
    got = b.dump().cpu().numpy()
    b.close()
    assert np.array_equal(got, oracle.to_int32(oracle.xmac(volt)))
    bad = bytearray(state)
    bad[8] ^= 1                                          # wrong N in the header
    c = corr.Correlator(N, F, T, path=path)
    with pytest.raises(corr.CorrError):
        c.set_state(bytes(bad))
    c.close()


def test_unpack_matches_oracle_decode():
    rng = np.random.default_rng(10)
    volt = rng.integers(0, 256, (77, 3, 37), dtype=np.uint8)
    volt[0, 0, :] = np.arange(37, dtype=np.uint8) * 7
    for zi in (False, True):
        re, im = oracle.decode(volt, zero_invalid=zi)
        got = corr.unpack(torch.from_numpy(volt).cuda(), zero_invalid=zi).cpu().numpy()
        want = np.stack([re, im], axis=-1).transpose(1, 2, 0, 3)   # [F][N][T][2]
        assert np.array_equal(got.astype(np.int32), want)


def test_paths_agree_with_each_other(coarse_volt):
    volt, want = coarse_volt
    sub = volt[:1500, :16]
    outs = {p: correlate(sub, p) for p in _paths_for(256)}
    ref = oracle.to_int32(oracle.xmac(sub))
    for p, o in outs.items():
        assert np.array_equal(o, ref), p


@pytest.mark.parametrize("path", ALL_PATHS)
def test_long_integration_worst_case_magnitude(path):
    """All samples 7+7i for 40000 samples: the largest sums the tensor-core
    encoding produces (its FP32 partials peak at 450 x 32768 < 2^24 per launch),
    across the split into several launches."""
    N, F, T = 128, 2, 40000
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    volt = np.full((T, F, N), 0x77, np.uint8)
    volt[:, 1, ::3] = 0x88                        # -8-8i on every third input of channel 1
    volt[::7, 1, 1::3] = 0x79
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, path), want)
    got = correlate(volt, path, chunks=[(0, 32767), (32767, 32769), (32769, T)])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("path", ALL_PATHS)
def test_many_channels_and_tiles(path):
    """More work items than SMs: 384 inputs (6 tile pairs per channel) x 40 ch."""
    N, F, T = 384, 40, 200
    if not path_available(path, N):
        pytest.skip(f"{path} unsupported")
    rng = np.random.default_rng(12)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, path), want)


# Work-item schemes of the tensor-core kernel: a launch of at least 64 stages
# of 64 samples (4033+ samples) pairs each diagonal tile with the tile below
# it; shorter launches use one item per tile pair.  These shapes cover 2, 3 and
# 4 tiles with a ragged last tile, and each is run as one long fresh launch
# (pairs), as a short fresh launch followed by a long accumulating one (pairs
# adding into the output), and as launches of 1000 samples (single items).
PAIR_SHAPES = [(144, 2, 4097), (256, 7, 4100), (272, 3, 4160), (400, 2, 4160)]


@pytest.mark.parametrize("shape", PAIR_SHAPES, ids=lambda s: "N%d_F%d_T%d" % s)
def test_tc_pair_and_single_items_exact(shape):
    N, F, T = shape
    if not path_available("tc_fp8", N):
        pytest.skip("tc_fp8 unsupported")
    rng = np.random.default_rng(N * 7 + F * 3 + T)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, "tc_fp8"), want)
    assert np.array_equal(correlate(volt, "tc_fp8", chunks=[(0, 64), (64, T)]), want)
    short = [(a, min(a + 1000, T)) for a in range(0, T, 1000)]
    assert np.array_equal(correlate(volt, "tc_fp8", chunks=short), want)


def test_tc_pair_items_many_channels():
    """More pair items than SMs, with a channel count that leaves a ragged last
    round (256 inputs, 2 items per channel, 331 channels)."""
    N, F, T = 256, 331, 4096
    if not path_available("tc_fp8", N):
        pytest.skip("tc_fp8 unsupported")
    rng = np.random.default_rng(331)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    got = correlate(volt, "tc_fp8")
    chans = [0, 1, 151, 152, 153, 303, 304, 330]
    want = oracle.to_int32(oracle.xmac(np.ascontiguousarray(volt[:, chans])))
    assert np.array_equal(got[chans], want)


def test_tc_pair_items_zero_invalid():
    """Pair items (a long fresh launch) with the invalid-code reading on: every
    sample with a nibble of 8 counts as zero, in the diagonal and the off-
    diagonal part of each pair alike."""
    N, F, T = 256, 3, 4160
    if not path_available("tc_fp8", N):
        pytest.skip("tc_fp8 unsupported")
    rng = np.random.default_rng(88)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    volt.reshape(-1)[::7] = 0x88
    volt.reshape(-1)[3::11] = 0x38
    want = oracle.to_int32(oracle.xmac(volt, zero_invalid=True))
    assert np.array_equal(correlate(volt, "tc_fp8", zero_invalid=True), want)
    assert not np.array_equal(correlate(volt, "tc_fp8"), want)      # the reading matters here


def test_tc_any_input_count_and_auto_choice():
    """Input counts that are not a multiple of 16 run on the tensor-core path
    through a padded copy of the rows; AUTO takes that path from 64 inputs."""
    if not path_available("tc_fp8", 64):
        pytest.skip("tc_fp8 unsupported")
    for n, want_path in [(17, "cudacore"), (63, "cudacore"), (65, "tc_fp8"), (130, "tc_fp8"), (250, "tc_fp8")]:
        c = corr.Correlator(n, 2, 100)
        assert c.path == want_path, (n, c.path)
        c.close()
    rng = np.random.default_rng(65)
    volt = rng.integers(0, 256, (333, 3, 250), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, "auto"), want)
    assert np.array_equal(correlate(volt, "tc_fp8", chunks=[(0, 100), (100, 333)]), want)
    assert np.array_equal(correlate(volt, "tc_fp8", zero_invalid=True),
                          oracle.to_int32(oracle.xmac(volt, zero_invalid=True)))


def test_tc_padded_rows_in_chunks():
    """17 inputs x 2048 channels x 5000 samples: the padded copy (32-byte rows)
    holds 4096 samples, so one call is correlated in two padded chunks."""
    if not path_available("tc_fp8", 17):
        pytest.skip("tc_fp8 unsupported")
    N, F, T = 17, 2048, 5000
    rng = np.random.default_rng(17)
    volt = rng.integers(0, 256, (T, F, N), dtype=np.uint8)
    want = oracle.to_int32(oracle.xmac(volt))
    assert np.array_equal(correlate(volt, "tc_fp8"), want)


def test_tc_misaligned_voltages_rejected():
    """The tensor-core path reads rows of a multiple of 16 inputs in place
    through TMA: a voltage pointer off a 16-byte boundary is an argument error
    and enqueues nothing."""
    if not path_available("tc_fp8", 64):
        pytest.skip("tc_fp8 unsupported")
    buf = torch.zeros(64 * 3 * 20 + 8, dtype=torch.uint8, device="cuda")
    c = corr.Correlator(64, 3, 20, path="tc_fp8")
    lib = corr.load()
    assert lib.corr_accumulate(c._ctx, ctypes.c_void_p(buf.data_ptr() + 8), 20, None) == corr.CORR_E_ARG
    assert c.samples == 0
    c.close()
