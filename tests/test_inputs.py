"""Checks of the seeded input generators (no solver arithmetic here)."""
import numpy as np
import pytest

import qcd_inputs as qi


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: first outputs of the published generator
    z = qi.splitmix64(0, 0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_and_normal_moments():
    u = qi.uniforms(5, 0, 200000)
    assert u.min() > 0 and u.max() < 1
    n = qi.normals(6, 200000)
    assert abs(n.mean()) < 0.01 and abs(n.std() - 1) < 0.01


def test_gauge_field_is_su3_and_chunk_invariant():
    dims = (4, 4, 4, 4)
    U = qi.gauge_field(dims, 0.3, seed=1000)
    assert np.abs(U @ U.conj().swapaxes(-1, -2) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    U2 = qi.gauge_field(dims, 0.3, seed=1000, chunk_sites=64)
    assert np.array_equal(U, U2)
    # eps -> 0 gives the unit field
    U0 = qi.gauge_field(dims, 0.0, seed=1000)
    assert np.abs(U0 - np.eye(3)).max() < 1e-15


def test_torch_path_matches_numpy_on_cpu():
    torch = pytest.importorskip("torch")
    dims = (2, 2, 2, 4)
    u_np = qi.uniforms(77, 64, 1000)
    u_t = qi._uniforms_torch(77, 64, 1000, "cpu").numpy()
    assert np.array_equal(u_np, u_t)
    U = qi.gauge_field(dims, 0.3, seed=3)
    Ut = qi._gauge_field_torch(dims, 0.3, 3, "cpu").numpy()
    assert np.abs(U - Ut).max() < 1e-13
    s = qi.gaussian_spinor(dims, seed=9, nrhs=2)
    st = qi.gaussian_spinor_torch(dims, 9, 2, "cpu").numpy()
    assert np.abs(s - st).max() < 1e-13


def test_point_sources():
    b = qi.point_sources((2, 2, 2, 2))
    assert b.shape == (12, 16, 4, 3)
    assert np.array_equal(b.reshape(12, -1)[:, :12], np.eye(12))
    assert b.reshape(12, -1)[:, 12:].sum() == 0
