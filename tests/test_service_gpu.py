"""The streaming service on the GPU: three arrays of different sizes, blocks
arriving as fast as accepted, dumps checked against the oracle on sampled
channels (regenerated from the seeded generator)."""
import numpy as np
import pytest

import oracle
from synth import voltgen as vg
from paper_1501_05992_gb300.service import GpuBackend, Service, StreamSpec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("paced,mode", [(False, "block"), (True, "block"), (False, "dump"), (True, "dump")])
def test_service_dumps_are_exact(paced, mode):
    specs = [StreamSpec("a256", 256, 12, block_samples=500, blocks_per_dump=4, array=0),
             StreamSpec("a128", 128, 20, block_samples=500, blocks_per_dump=4, array=1),
             StreamSpec("a64", 64, 9, block_samples=500, blocks_per_dump=4, array=2)]
    be = GpuBackend(pool_blocks=3, verify_channels=3)
    svc = Service(specs, 1 << 36, be, paced=paced, mode=mode)
    rep = svc.run(8)
    for a in rep["arrays"]:
        assert a["blocks"] == 8 and a["dumps"] == 2 and a["gaps"] == 0, a
        assert a["p99_ms"] is not None
    assert rep["x_real_time_margin"] > 1.0
    checked = 0
    for a, d, rows in be.kept:
        spec = specs[a]
        params = vg.gauss3_params(spec.seed, spec.n_inputs, spec.n_chan, array=spec.array)
        seqs = range(d * spec.blocks_per_dump, (d + 1) * spec.blocks_per_dump)
        for f, got in rows.items():
            want = np.zeros((1, spec.n_inputs * (spec.n_inputs + 1) // 2, 2), np.int64)
            for q in seqs:
                t0 = (q % be.pool_blocks) * spec.block_samples
                oracle.xmac(vg.gauss3(params, t0, spec.block_samples, f, 1), vis=want)
            assert np.array_equal(got.numpy(), oracle.to_int32(want)[0]), (spec.name, d, f)
            checked += 1
    assert checked == sum(2 * len(be.kept_channels[a]) for a in range(3))


def test_service_rejects_what_does_not_fit():
    specs = [StreamSpec("big", 512, 3072, array=0), StreamSpec("small", 64, 8, array=1)]
    svc = Service(specs, 2 << 30, GpuBackend(pool_blocks=1))
    assert [s.name for s in svc.admitted] == ["small"]
    assert svc.rejected[0][0].name == "big"
