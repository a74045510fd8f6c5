"""Batched arrays (one persistent tensor-core launch), CUDA-graph replay,
CUDA-core tile shapes and the autotuner, all bit-exact against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1501_05992_gb300 import autotune, corr

from _gpu import path_available

pytestmark = pytest.mark.gpu


def _rand(shape, seed):
    return np.random.default_rng(seed).integers(0, 256, shape, dtype=np.uint8)


def _check_batch(specs, volts_np, chunks=1):
    b = corr.Batch(specs)
    vt = [torch.from_numpy(v).cuda() for v in volts_np]
    T = [v.shape[0] for v in volts_np]
    for k in range(chunks):
        part = [v[(t * k) // chunks:(t * (k + 1)) // chunks].contiguous() for v, t in zip(vt, T)]
        b.accumulate(part)
    outs = b.dump()
    b.sync()
    for a, (v, o) in enumerate(zip(volts_np, outs)):
        assert np.array_equal(o.cpu().numpy(), oracle.to_int32(oracle.xmac(v))), f"array {a}"
    return b


def test_uneven_arrays_in_one_launch():
    """Three arrays shaped like the uneven-batch workload (fewer channels)."""
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    specs = [{"n_inputs": 128, "n_chan": 40, "n_time_per_int": 2000, "path": "tc_fp8"},
             {"n_inputs": 256, "n_chan": 24, "n_time_per_int": 700, "path": "tc_fp8"},
             {"n_inputs": 1024, "n_chan": 3, "n_time_per_int": 300, "path": "tc_fp8"}]
    volts = [_rand((2000, 40, 128), 1), _rand((700, 24, 256), 2), _rand((300, 3, 1024), 3)]
    b = _check_batch(specs, volts)
    assert b.paths == ["tc_fp8"] * 3
    _check_batch(specs, volts, chunks=3)


def test_more_arrays_than_one_launch_holds():
    if not path_available("tc_fp8", 64):
        pytest.skip("tc_fp8 unsupported")
    shapes = [(64, 5, 130), (128, 3, 64), (192, 2, 200), (64, 7, 1), (256, 1, 90), (48, 4, 333)]
    specs = [{"n_inputs": n, "n_chan": f, "n_time_per_int": t, "path": "tc_fp8"} for n, f, t in shapes]
    volts = [_rand((t, f, n), 10 + k) for k, (n, f, t) in enumerate(shapes)]
    _check_batch(specs, volts)


def test_mixed_paths_and_skipped_arrays():
    specs = [{"n_inputs": 64, "n_chan": 6, "n_time_per_int": 500, "path": "cudacore", "tile": 32},
             {"n_inputs": 128, "n_chan": 4, "n_time_per_int": 500, "path": "auto"},
             {"n_inputs": 40, "n_chan": 5, "n_time_per_int": 500, "path": "mma_i8"}]
    volts = [_rand((500, 6, 64), 21), _rand((500, 4, 128), 22), _rand((500, 5, 40), 23)]
    _check_batch(specs, volts)
    b = corr.Batch(specs)
    b.accumulate([torch.from_numpy(volts[0]).cuda(), None, None])
    assert [b.samples(a) for a in range(3)] == [500, 0, 0]
    outs = b.dump([torch.empty((6, 64 * 65 // 2, 2), dtype=torch.int32, device="cuda"), None, None])
    b.sync()
    assert np.array_equal(outs[0].cpu().numpy(), oracle.to_int32(oracle.xmac(volts[0])))


def test_long_batched_integration_splits_launches():
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    specs = [{"n_inputs": 128, "n_chan": 2, "n_time_per_int": 40000, "path": "tc_fp8"},
             {"n_inputs": 256, "n_chan": 1, "n_time_per_int": 33000, "path": "tc_fp8"}]
    volts = [np.full((40000, 2, 128), 0x77, np.uint8), _rand((33000, 1, 256), 31)]
    _check_batch(specs, volts)


def test_batch_accumulate_after_a_member_host_dump():
    """A host dump of one batch member copies out on the member's output
    stream; the next batched tensor-core launch must wait for that copy
    before it overwrites the member's accumulators."""
    if not path_available("tc_fp8", 256):
        pytest.skip("tc_fp8 unsupported")
    specs = [{"n_inputs": 256, "n_chan": 48, "n_time_per_int": 2000, "path": "tc_fp8"},
             {"n_inputs": 128, "n_chan": 20, "n_time_per_int": 2000, "path": "tc_fp8"}]
    rng = np.random.default_rng(91)
    va = [rng.integers(0, 256, (1000, 48, 256), dtype=np.uint8),
          rng.integers(0, 256, (1000, 20, 128), dtype=np.uint8)]
    vb = [rng.integers(0, 256, (1000, 48, 256), dtype=np.uint8),
          rng.integers(0, 256, (1000, 20, 128), dtype=np.uint8)]
    b = corr.Batch(specs)
    da = [torch.from_numpy(v).cuda() for v in va]
    db = [torch.from_numpy(v).cuda() for v in vb]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    host = b.dump_host(0, stream=s)
    for _ in range(3):
        b.accumulate(da, stream=s)
        b.dump_host(0, host, stream=s)
        b.accumulate(db, stream=s)
        outs = b.dump(stream=s)
        b.sync(s)
        assert np.array_equal(host.numpy(), oracle.to_int32(oracle.xmac(va[0])))
        assert np.array_equal(outs[0].cpu().numpy(), oracle.to_int32(oracle.xmac(vb[0])))
        both = np.concatenate([va[1], vb[1]])
        assert np.array_equal(outs[1].cpu().numpy(), oracle.to_int32(oracle.xmac(both)))
    b.close()


def test_overflow_in_one_array_enqueues_nothing():
    specs = [(64, 2, 100), (128, 2, 50)]
    b = corr.Batch(specs)
    v0 = torch.zeros((80, 2, 64), dtype=torch.uint8, device="cuda")
    v1 = torch.zeros((60, 2, 128), dtype=torch.uint8, device="cuda")
    with pytest.raises(corr.CorrError) as e:
        b.accumulate([v0, v1])
    assert e.value.status == corr.CORR_E_OVERFLOW
    assert b.samples(0) == 0 and b.samples(1) == 0
    b.accumulate([v0, v1[:50].contiguous()])
    assert b.samples(0) == 80 and b.samples(1) == 50
    b.dump()
    b.sync()


def test_batch_integrate_mixed_paths():
    specs = [{"n_inputs": 128, "n_chan": 6, "n_time_per_int": 900, "path": "auto"},
             {"n_inputs": 64, "n_chan": 3, "n_time_per_int": 900, "path": "cudacore"},
             {"n_inputs": 256, "n_chan": 2, "n_time_per_int": 900, "path": "tc_fp8"},
             {"n_inputs": 40, "n_chan": 4, "n_time_per_int": 900, "path": "mma_i8"}]
    if not path_available("tc_fp8", 256):
        specs[2]["path"] = "auto"
    shapes = [(900, 6, 128), (700, 3, 64), (333, 2, 256), (900, 4, 40)]
    volts = [_rand(sh, 100 + k) for k, sh in enumerate(shapes)]
    b = corr.Batch(specs)
    b.accumulate([torch.from_numpy(volts[0][:100]).cuda(), None, None, None])
    outs = b.integrate([torch.from_numpy(v).cuda() for v in volts])
    b.sync()
    for a in range(4):
        assert np.array_equal(outs[a].cpu().numpy(), oracle.to_int32(oracle.xmac(volts[a]))), a
    assert b.samples(0) == 100                       # the running integration is kept
    part = b.dump()
    b.sync()
    assert np.array_equal(part[0].cpu().numpy(), oracle.to_int32(oracle.xmac(volts[0][:100])))
    # arrays without an output buffer are skipped
    only1 = torch.full((3, 64 * 65 // 2, 2), -3, dtype=torch.int32, device="cuda")
    b.integrate([torch.from_numpy(v).cuda() for v in volts], [None, only1, None, None])
    b.sync()
    assert np.array_equal(only1.cpu().numpy(), oracle.to_int32(oracle.xmac(volts[1])))
    b.close()


def test_graph_replays_whole_integrations():
    specs = [{"n_inputs": 128, "n_chan": 8, "n_time_per_int": 1000},
             {"n_inputs": 64, "n_chan": 3, "n_time_per_int": 1000, "path": "cudacore"}]
    volts = [_rand((1000, 8, 128), 41), _rand((1000, 3, 64), 42)]
    b = corr.Batch(specs)
    vt = [torch.from_numpy(v).cuda() for v in volts]
    stream = torch.cuda.Stream()
    graph, outs = b.capture(vt, stream=stream)
    assert b.samples(0) == 0 and b.samples(1) == 0
    want = [oracle.to_int32(oracle.xmac(v)) for v in volts]
    for rep in range(3):
        for o in outs:
            o.fill_(-7)
        torch.cuda.synchronize()
        graph.launch(stream)
        stream.synchronize()
        for a in range(2):
            assert np.array_equal(outs[a].cpu().numpy(), want[a]), (rep, a)
    # new data in the captured input buffers is picked up by the next replay
    new0 = _rand((1000, 8, 128), 43)
    vt[0].copy_(torch.from_numpy(new0))
    torch.cuda.synchronize()
    graph.launch(stream)
    stream.synchronize()
    assert np.array_equal(outs[0].cpu().numpy(), oracle.to_int32(oracle.xmac(new0)))
    b.sync(stream)
    graph.close()


@pytest.mark.parametrize("tile", [32, 64])
@pytest.mark.parametrize("shape", [(1, 1, 5), (17, 3, 65), (33, 2, 129), (100, 2, 64)])
def test_cudacore_tiles_exact(tile, shape):
    N, F, T = shape
    volt = _rand((T, F, N), N + F + T + tile)
    c = corr.Correlator(N, F, T, path="cudacore")
    c.set_tile(tile)
    c.accumulate(torch.from_numpy(volt).cuda())
    got = c.dump().cpu().numpy()
    c.sync()
    c.close()
    assert np.array_equal(got, oracle.to_int32(oracle.xmac(volt)))


@pytest.mark.parametrize("tile", [128, 256])
def test_tc_item_shapes_exact(tile):
    """Both tcgen05 work-item shapes forced on launches of every length (single
    tile pairs and pair items, fresh and accumulating, 2, 3 and 5 tiles with
    ragged last tiles), alone and as arrays of one batch with different
    shapes."""
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    for N, F, T in [(256, 5, 300), (272, 3, 1100), (560, 2, 700)]:
        volt = _rand((T, F, N), N + T + tile)
        c = corr.Correlator(N, F, T, path="tc_fp8")
        c.set_tile(tile)
        d = torch.from_numpy(volt).cuda()
        c.accumulate(d[:T // 3])
        c.accumulate(d[T // 3:])
        got = c.dump().cpu().numpy()
        whole = c.integrate(d).cpu().numpy()
        c.sync()
        c.close()
        want = oracle.to_int32(oracle.xmac(volt))
        assert np.array_equal(got, want), (N, F, T)
        assert np.array_equal(whole, want), (N, F, T)
    other = 384 - tile
    specs = [{"n_inputs": 384, "n_chan": 3, "n_time_per_int": 400, "path": "tc_fp8", "tile": tile},
             {"n_inputs": 256, "n_chan": 4, "n_time_per_int": 400, "path": "tc_fp8", "tile": other}]
    _check_batch(specs, [_rand((400, 3, 384), 71), _rand((400, 4, 256), 72)])


def test_set_tile_rejects_other_values():
    c = corr.Correlator(64, 2, 10)
    for bad in (1, 16, 96, 512, -1):
        with pytest.raises(corr.CorrError):
            c.set_tile(bad)
    for good in (0, 32, 64, 128, 256):
        c.set_tile(good)
    c.close()


def test_autotune_picks_and_caches(tmp_path):
    cache = str(tmp_path / "tune.json")
    r = autotune.tune(256, 8, 500, cache_path=cache, reps=1)
    assert r["path"] in ("tc_fp8", "mma_i8", "cudacore") and r["ms"]
    again = autotune.tune(256, 8, 500, cache_path=cache, reps=1)
    assert again == r
    small = autotune.tune(16, 8, 500, cache_path=cache, reps=1)
    plan = autotune.plan([(256, 8, 500), (16, 8, 500)], cache_path=cache)
    assert plan[0]["path"] == r["path"] and plan[1]["path"] == small["path"]
    volts = [_rand((500, 8, 256), 51), _rand((500, 8, 16), 52)]
    _check_batch(plan, volts)


def test_batch_with_padded_tensor_core_arrays():
    """Arrays whose input count is not a multiple of 16 correlate on the
    tensor-core path in launches of their own, beside the shared launch of
    the others; accumulate, dump and whole-integration calls alike."""
    if not path_available("tc_fp8", 65):
        pytest.skip("tc_fp8 unsupported")
    shapes = [(65, 4, 300), (128, 3, 300), (200, 2, 300), (9, 5, 300)]
    specs = [{"n_inputs": n, "n_chan": f, "n_time_per_int": t, "path": "tc_fp8"} for n, f, t in shapes]
    volts = [_rand((t, f, n), 80 + k) for k, (n, f, t) in enumerate(shapes)]
    _check_batch(specs, volts, chunks=2)
    b = corr.Batch(specs)
    outs = b.integrate([torch.from_numpy(v).cuda() for v in volts])
    b.sync()
    for v, o in zip(volts, outs):
        assert np.array_equal(o.cpu().numpy(), oracle.to_int32(oracle.xmac(v)))
    b.close()


def test_tc_last_round_split_exact():
    """Launches whose item count leaves a partial last round on the GPU's SMs,
    where the last channels run as single items instead of pair items (200
    inputs on a padded copy, 384 inputs with three tiles): whole triangles of
    the first, the last paired and the single-item channels, fresh and
    accumulating launches (the same samples twice), and the fused beam of
    every channel."""
    if not path_available("tc_fp8", 128):
        pytest.skip("tc_fp8 unsupported")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # pair items from 64 stages on: 4100 samples; 2 and 4 items per channel
    for N, F in [(200, sms + 8), (384, sms // 4 + 6)]:
        T = 4100
        volt = _rand((T, F, N), N + F)
        c = corr.Correlator(N, F, 2 * T, path="tc_fp8")
        d = torch.from_numpy(volt).cuda()
        tri, beam = c.integrate_beam(d, 4)
        c.accumulate(d)
        c.accumulate(d)
        acc = c.dump()
        c.sync()
        c.close()
        chans = sorted({0, F - 25, F - 9, F - 8, F - 7, F - 1})
        vis = oracle.xmac(volt[:, chans])
        assert np.array_equal(tri[chans].cpu().numpy(), oracle.to_int32(vis)), (N, F)
        assert np.array_equal(acc[chans].cpu().numpy(), oracle.to_int32(2 * vis)), (N, F)
        assert np.array_equal(beam.cpu().numpy(), oracle.beam(volt, 4)), (N, F)
