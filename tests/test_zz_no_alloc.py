"""The allocation-free entry point edac_density_static, for callers that cannot allocate
device memory when they need the result (under a framework's own pool allocator, as a
plug-in whose host application owns the device memory, or on an allocation-free real-time
path).  Its scratch is the library's
static device array; this file is collected last so that a failure here comes after every
other test has run.  Checked against the context path (edac_set_particles, whose initial
evaluation gives rho, V and N) on two calls in a row, within the fp64 path's tolerance."""
import numpy as np
import pytest

from paper_1907_04034_gb300 import binding, cases


@pytest.fixture(scope="module", autouse=True)
def _built():
    binding.build()
    yield


@pytest.mark.gpu
@pytest.mark.parametrize("maker", [lambda: cases.channel(),
                                   lambda: cases.cylinder(dx=1.0 / 20.0),
                                   lambda: cases.random_box(n=700, seed=9, periodic_y=0)])
def test_static_scratch_density_matches_the_context_path(maker):
    c = maker()
    s = binding.Solver(c, precision="fp64")
    ref = s.state(("rho", "vol", "nnb"))
    s.close()
    assert np.array_equal(ref["id"], c.id)  # ascending id = the case's order
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        rho, vol, nnb = binding.density_static(c)
        np.testing.assert_array_equal(nnb, ref["nnb"].astype(np.int32))
        assert np.abs(rho - ref["rho"]).max() <= 1e-10 * np.abs(ref["rho"]).max()
        assert np.abs(vol - ref["vol"]).max() <= 1e-10 * np.abs(ref["vol"]).max()
