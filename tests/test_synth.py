"""The seeded generators produce the shapes they claim (CPU only)."""
import math

import numpy as np
import pytest

import synth


def test_deterministic():
    for d in synth.U32_DISTRIBUTIONS:
        assert np.array_equal(synth.u32(d, 5000, 3), synth.u32(d, 5000, 3))
    for d in synth.U64_DISTRIBUTIONS:
        assert np.array_equal(synth.u64(d, 5000, 3), synth.u64(d, 5000, 3))


def test_shapes_u32():
    n = 1 << 21
    a = synth.normal_u32(n, 1).astype(np.float64)
    assert abs(a.mean() / 2 ** 31 - 1) < 1e-3 and abs(a.std() / 2 ** 28 - 1) < 1e-2
    e = synth.exponential_u32(n, 2).astype(np.float64)
    assert abs(e.mean() / 2 ** 24 - 1) < 1e-2
    assert abs(np.mean(e < 2 ** 24) - (1 - math.exp(-1))) < 2e-3
    z = synth.zipf_u32(n, 3)
    _, counts = np.unique(z, return_counts=True)
    h = sum(k ** -1.1 for k in range(1, (1 << 20) + 1))
    assert abs(counts.max() / n - 1 / h) < 2e-3
    s = synth.sorted_u32(n, 4)
    assert np.all(s[1:] >= s[:-1])
    assert abs(s.astype(np.float64).mean() / 2 ** 31 - 1) < 5e-3
    r = synth.reverse_u32(n, 4)
    assert np.array_equal(r, s[::-1])
    q = synth.equal_u32(n, 5)
    assert np.all(q == q[0])


def test_shapes_u64():
    n = 1 << 20
    u = synth.uniform16_u64(n, 1)
    assert u.max() < 2 ** 16
    d = synth.dup90_u64(n, 2)
    vals, counts = np.unique(d, return_counts=True)
    top = np.sort(counts)[::-1][:1024].sum()
    assert abs(top / n - 0.9) < 5e-3
    w = synth.uniform64_u64(n, 3)
    assert (w >> np.uint64(63)).mean() == pytest.approx(0.5, abs=5e-3)


def test_mix32_is_bijection_on_sample():
    x = np.arange(1 << 20, dtype=np.uint32)
    assert np.unique(synth.mix32(x)).size == x.size


def test_batch_sizes():
    s = synth.batch_sizes(4096, 40)
    assert s.min() >= 256 and s.max() <= 1 << 20
    assert abs(np.log(s).mean() - (math.log(256) + math.log(1 << 20)) / 2) < 0.15


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 seeded with 0, as published with the
    # generator's reference implementation
    z = synth.splitmix64(0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counter-based: any window of the stream can be generated on its own
    assert np.array_equal(synth.splitmix64(12345, 10, start=90), synth.splitmix64(12345, 100)[90:])
    assert np.array_equal(synth.splitmix64_u32(7, 5), (synth.splitmix64(7, 5) >> np.uint64(32)).astype(np.uint32))


def test_served_stream_shape():
    sizes, kv = synth.served_stream(100_000, 50)
    assert sizes.min() >= 1 << 10 and sizes.max() <= 1 << 24
    assert abs(np.log(sizes).mean() - (math.log(1 << 10) + math.log(1 << 24)) / 2) < 0.05
    assert abs(kv.mean() - 0.3) < 0.01
    assert synth.request_seed(50, 3) != synth.request_seed(50, 4)
