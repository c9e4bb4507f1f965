"""The seeded input generators (paper_2103_06998_gb300/inputs.py; no GPU):
SplitMix64 against its published output sequence, the order independence of
the hashed uniforms, and the head-like material map, dipole, random fields and
batch descriptions against the ranges and classes their definitions state."""
import numpy as np

from paper_2103_06998_gb300 import inputs


def test_splitmix64_reproduces_the_published_sequence():
    # the generator seeded with 0 advances its state by the golden-ratio constant
    # and mixes it: its first outputs are e220a8397b1dcdaf, 6e789e6aa1b965f4, 06c45d188009454f
    G = 0x9E3779B97F4A7C15
    got = [int(inputs.splitmix64(np.uint64((k * G) & 0xFFFFFFFFFFFFFFFF))) for k in range(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniforms_are_in_range_and_independent_of_evaluation_order():
    idx = np.arange(10000, dtype=np.uint64)
    u = inputs.uniform(7, 3, idx)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.005
    perm = np.random.default_rng(0).permutation(idx.size)
    np.testing.assert_array_equal(inputs.uniform(7, 3, idx[perm]), u[perm])
    # other seeds and streams give other values
    assert not np.array_equal(inputs.uniform(8, 3, idx), u)
    assert not np.array_equal(inputs.uniform(7, 4, idx), u)


def test_head_map_classes_and_values():
    n = (24, 20, 28)
    eps, mu, sigma, cls = inputs.head_map(n, 2103)
    assert eps.shape == mu.shape == sigma.shape == cls.shape == (n[2], n[1], n[0])
    assert np.all(mu == 1.0)
    air, skull, tissue = cls == 0, cls == 1, cls == 2
    assert air.any() and skull.any() and tissue.any()
    assert np.all(eps[air] == 1.0) and np.all(sigma[air] == 0.0)
    assert np.all(eps[skull] == 12.0) and np.all(sigma[skull] == 0.05)
    assert eps[tissue].min() >= 45.0 and eps[tissue].max() <= 55.0
    assert sigma[tissue].min() >= 0.63 and sigma[tissue].max() <= 0.77
    # the centre of the cube lies inside the inner ellipsoid, the corners in air
    assert cls[n[2] // 2, n[1] // 2, n[0] // 2] == 2
    assert cls[0, 0, 0] == cls[-1, -1, -1] == 0
    # the same seed gives the same map, another seed another one
    np.testing.assert_array_equal(inputs.head_map(n, 2103)[0], eps)
    assert not np.array_equal(inputs.head_map(n, 2104)[0], eps)


def test_dipole_fields_and_batch_descriptions():
    for seed in range(5):
        d = inputs.dipole(seed)
        assert all(0.2 <= v <= 0.8 for v in d["x0"]) and d["comp"] == 2
        assert d["f0"] == 2.0 and d["s"] == 0.5 and d["t0"] == 1.5 and d["amp"] == 1.0
    f = inputs.random_fields((5, 4, 3), 9, scale=2.0)
    assert f.shape == (6, 5, 4, 3) and np.abs(f).max() <= 2.0
    np.testing.assert_array_equal(inputs.random_fields((5, 4, 3), 9, scale=2.0), f)
    inst = inputs.batch_instances(count=6, seed=11)
    assert len(inst) == 6
    for d in inst:
        assert all(32 <= v <= 128 for v in d["n"]) and d["p"] in (2, 3)
        assert d["eps"].shape == (d["n"][2], d["n"][1], d["n"][0])
    assert [d["n"] for d in inputs.batch_instances(count=6, seed=11)] == [d["n"] for d in inst]
