"""The sensor-family workloads (pad, DIGIT-like dome, 9DTact-like block):
valid positively oriented meshes near the requested size, a fixed bottom, an
indenter that starts dhat above the gel and a pixel grid over the sensor."""
import numpy as np
import pytest

from oracle import mesh as omesh
from synth import indenters, workloads


@pytest.mark.parametrize("sensor,nt", [("pad", 5000), ("dome", 8000), ("block", 10000)])
def test_sensor_env_is_valid(sensor, nt):
    e = workloads.sensor_env(5, sensor, nt, steps=4)
    X, T = e["X"], e["tets"]
    assert abs(len(T) - nt) <= 0.25 * nt
    _, vol = omesh.rest_shape(X, T)  # raises on a non-positive tet
    assert np.all(vol > 0)
    assert len(e["fixed"]) > 0 and np.all(X[e["fixed"], 2] == 0.0)
    V = e["ind_V"] @ e["start_pose"]["R"].T + e["start_pose"]["t"]
    assert V[:, 2].min() == pytest.approx(X[:, 2].max() + e["opts"]["dhat"], abs=1e-12)
    assert e["poses"][-1]["t"][2] < e["start_pose"]["t"][2]
    g = e["grid"]
    assert g["H"] > 0 and g["W"] > 0


def test_dome_geometry():
    X, T = workloads.sensor_mesh("dome", 8000)[0]
    # slab 1.5 mm + cap (radius 30 mm, height 3 mm): the apex region reaches
    # ~4.5 mm; a corner of the 20 x 16 mm base lies 12.8 mm off-axis, where the
    # cap surface is at 1.5 + 3 - 30 + sqrt(30^2 - 12.8^2) mm
    assert 4.4e-3 < X[:, 2].max() <= 4.5e-3 + 1e-12
    corner = (X[:, 0] == 0.0) & (X[:, 1] == 0.0)
    expect = 1.5e-3 + 3e-3 - 30e-3 + np.sqrt(30e-3 ** 2 - (10e-3 ** 2 + 8e-3 ** 2))
    assert X[corner, 2].max() == pytest.approx(expect, rel=1e-9)


def test_mixed_envs_sizes():
    envs = workloads.mixed_envs(1, n_per_family=2, pads=(5000, 6000), domes=(8000, 9000), blocks=(10000, 11000),
                                steps=2)
    fams = [e["sensor"] for e in envs]
    assert fams == ["pad", "pad", "dome", "dome", "block", "block"]
    assert len({e["name"] for e in envs}) == len(envs)
