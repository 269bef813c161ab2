"""The seeded input generators shared by the parity tests and the benchmark:
shapes, box bounds, neutrality, determinism, and the structure each workload
is documented to have (the clustered share of the wire workload, the size and
periodicity mix of the batch)."""
import numpy as np
import pytest

from paper_1712_04732_gb300 import workloads as wl


@pytest.mark.parametrize("name", ["lattice_3p", "free_0p", "slab_2p"])
def test_named_workloads_shapes_bounds_and_charges(name):
    x, q, spec = wl.make(name, seed=3)
    n = spec["N"]
    assert x.shape == (n, 3) and q.shape == (n,)
    assert x.dtype == np.float64 and q.dtype == np.float64
    assert np.all(x >= 0.0) and np.all(x < spec["L"])
    assert abs(q.sum()) <= 1e-9 * np.abs(q).sum()             # neutral
    if spec["charges"] == "alternating":
        assert set(np.unique(q)) == {-1.0, 1.0}
    else:
        assert np.all(np.abs(q) <= 1.0 + 3.0 / np.sqrt(n))       # U(-1, 1) less its sample mean
        assert abs(np.mean(np.abs(q)) - 0.5) < 0.02               # E|q| = 1/2 for U(-1, 1)


def test_same_seed_same_arrays_other_seed_other_arrays():
    x1, q1, _ = wl.make("free_0p", seed=7)
    x2, q2, _ = wl.make("free_0p", seed=7)
    x3, q3, _ = wl.make("free_0p", seed=8)
    assert np.array_equal(x1, x2) and np.array_equal(q1, q2)
    assert not np.array_equal(x1, x3) and not np.array_equal(q1, q3)


def test_wire_workload_has_a_sixth_of_its_particles_in_ten_clouds():
    """1e6 uniform + 2e5 in ten Gaussian clouds (sigma = 0.03), scaled down here to
    N = 60 000: the clustered sixth sits within 4 sigma of ten centres inside
    [0.15, 0.85]^3, far above the share a uniform cloud would put there."""
    n = 60000
    x, q, spec = wl.make("wire_1p", seed=2, N=n)
    assert x.shape == (n, 3) and np.all((x >= 0.0) & (x < 1.0))
    assert abs(q.sum()) <= 1e-9 * np.abs(q).sum()
    blobs = x[n - n // 6:]
    uniform = x[: n - n // 6]
    # the blob points group around ten centres: k-means-free check by a 3D histogram
    H, _ = np.histogramdd(blobs, bins=20, range=[(0, 1)] * 3)
    dense = H > 0.002 * len(blobs)
    assert dense.sum() < 0.02 * H.size                          # concentrated in few cells
    assert np.all(blobs.min(0) > 0.0) and np.all(blobs.max(0) < 1.0)
    Hu, _ = np.histogramdd(uniform, bins=20, range=[(0, 1)] * 3)
    assert Hu.max() < 3 * Hu.mean()                             # the rest is uniform


def test_batch_systems_sizes_and_periodicities():
    sysl = wl.batch_systems(64, seed=1)
    assert len(sysl) == 64
    Ns = np.array([len(q) for _, q, _ in sysl])
    assert Ns.min() >= 1000 and Ns.max() <= 100000
    assert np.all(Ns % 2 == 0)
    # log-uniform: about half the systems below the geometric mean of the range
    assert 20 <= (Ns < 10000).sum() <= 44
    assert [D for _, _, D in sysl] == [3 if i % 2 == 0 else 2 for i in range(64)]
    for x, q, _ in sysl:
        assert np.all((x >= 0.0) & (x < 1.0))
        assert abs(q.sum()) <= 1e-9 * np.abs(q).sum()


def test_nacl_cell_is_the_rock_salt_arrangement():
    x, q = wl.nacl_cell(8)
    assert x.shape == (512, 3) and abs(q.sum()) == 0.0
    # every ion's six nearest neighbours (spacing 1/8, periodic) carry the opposite charge
    for i in (0, 77, 300):
        d = x - x[i]
        d -= np.round(d)
        r = np.sqrt((d ** 2).sum(1))
        nn = np.isclose(r, 1.0 / 8.0)
        assert nn.sum() == 6 and np.all(q[nn] == -q[i])
