"""JSON presets of the five configurations (synthetic/presets): each builds
exactly the workload of the corresponding synthetic.workload_* recipe (the
same phantom arrays, source, transport, histories and seed)."""
import numpy as np
import pytest

import synthetic as S


def _same_workload(a, b):
    assert a.name == b.name
    assert a.phantom.shape == b.phantom.shape
    assert (a.phantom.dx, a.phantom.dy, a.phantom.dz) == (b.phantom.dx, b.phantom.dy, b.phantom.dz)
    np.testing.assert_array_equal(a.phantom.mat, b.phantom.mat)
    np.testing.assert_array_equal(a.phantom.rho, b.phantom.rho)
    assert [m.name for m in a.phantom.materials] == [m.name for m in b.phantom.materials]
    sa, sb = a.source, b.source
    for f in ("particle", "shape", "x0", "y0", "hx", "hy", "energy"):
        assert getattr(sa, f) == pytest.approx(getattr(sb, f), rel=1e-15, abs=0), f
    for f in ("edges", "weights"):
        x, y = getattr(sa, f), getattr(sb, f)
        assert (x is None) == (y is None), f
        if x is not None:
            np.testing.assert_array_equal(x, y)
    assert a.transport == b.transport
    assert (a.n_hist, a.seed) == (b.n_hist, b.seed)


def test_every_configuration_has_a_preset():
    assert S.preset_names() == ["c1_water20_pencil", "c2_grf128_photon_field", "c3_ct256_electron",
                                "c4_batch64", "c5_differentiable"]


@pytest.mark.parametrize("name, make", [
    ("c1_water20_pencil", lambda: S.workload_water_pencil()),
    ("c2_grf128_photon_field", lambda: S.workload_grf_spectrum()),
    ("c3_ct256_electron", lambda: S.workload_ct_electron()),
])
def test_preset_equals_recipe(name, make):
    _same_workload(S.load_preset(name), make())


def test_batched_preset_equals_recipe():
    """The first jobs of the 64 (the job parameters are drawn in job order)."""
    a = S.load_preset("c4_batch64", n_jobs=3)
    b = S.batched_jobs(3, 4)
    assert len(a) == 3
    for x, y in zip(a, b):
        _same_workload(x, y)


def test_differentiable_preset_equals_recipe():
    (a, ta), (b, tb) = S.load_preset("c5_differentiable"), S.workload_differentiable()
    _same_workload(a, b)
    np.testing.assert_array_equal(ta, tb)
