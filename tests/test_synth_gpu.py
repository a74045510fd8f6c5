"""The device generator writes the same bytes as the numpy generator."""
import numpy as np
import pytest

from synth import voltgen as vg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("recipe", ["gauss3", "uniform_tone"])
def test_device_generator_matches_numpy(recipe):
    from synth.gpu import DeviceGenerator
    spec = vg.ArraySpec(48, 20, 300)
    p = vg.make_params(recipe, 4242, spec, array=1)
    dev = DeviceGenerator(p).make(t0=123, n_time=77, f0=3, n_f=11).cpu().numpy()
    host = vg.generate(p, 123, 77, 3, 11)
    assert np.array_equal(dev, host)
