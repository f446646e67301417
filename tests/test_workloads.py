"""The seeded input generators: the counter-based splitmix64 against its
published outputs, and the torch version (used for the large benchmark
fields, drawn on the device) against the NumPy one (used by the parity
tests), so both sides of every comparison start from the same numbers."""
import numpy as np
import pytest

from paper_1004_0480_gb300 import workloads as W


def test_splitmix64_matches_the_published_sequence():
    # the first outputs of splitmix64 from state 0 (Steele, Lea and Flood's
    # generator as published with its reference implementation)
    got = W.splitmix64(np.array([0, 0x9E3779B97F4A7C15, 2 * 0x9E3779B97F4A7C15 % 2 ** 64],
                                dtype=np.uint64))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                     0x06C45D188009454F]


@pytest.mark.parametrize("seed,species,start", [(0, 0, 0), (1, 1, 5), (3, 2, 1 << 20),
                                                (2 ** 40 + 7, 3, 123)])
def test_torch_draws_equal_numpy_draws(seed, species, start):
    torch = pytest.importorskip("torch")
    a = W.uniform01(seed, species, 4096, start=start)
    b = W.uniform01_torch(seed, species, 4096, "cpu", start=start).numpy()
    assert np.array_equal(a, b)
    assert 0.0 <= a.min() and a.max() < 1.0
    del torch


@pytest.mark.parametrize("make", [
    lambda: W.brusselator(shape=(9, 7, 5)),
    lambda: W.ch_front(shape=(8, 6, 5)),
    lambda: W.air((10, 6, 4), src=(1, 1, 1)),
    lambda: W.turing(shape=(7, 8, 6)),
    lambda: W.ch_table1(shape=(7, 5, 6)),
    lambda: W.plume(shape=(6, 5, 7)),
    lambda: W.with_(W.diffusion_blob(shape=(6, 5, 4)), init="uniform_noise"),
])
def test_initial_fields_on_the_device_path_equal_the_host_path(make):
    pytest.importorskip("torch")
    cfg = make()
    a = W.initial_fields(cfg)
    b = W.initial_fields_torch(cfg, "cpu").numpy()
    assert a.dtype == b.dtype == np.float32
    assert np.array_equal(a, b)


def test_blob_initial_fields_agree_to_rounding():
    pytest.importorskip("torch")
    cfg = W.diffusion_blob(shape=(13, 11, 9))
    a = W.initial_fields(cfg)
    b = W.initial_fields_torch(cfg, "cpu").numpy()
    # exp may differ in the last bit of float64 between libraries
    np.testing.assert_allclose(a, b, rtol=2e-7, atol=0)
