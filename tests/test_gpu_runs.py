"""Inputs made of runs of equal digits, for the key-only scatter's run mode
(a tile that follows a tile of at most eight distinct digits takes each
warp's run of one digit with a single atomic): sorted and reverse-sorted
keys, runs of random lengths, sawtooth and organ-pipe orders, runs that
straddle tile boundaries, arrays that start off a 16-byte boundary, and
mixtures where run-like tiles alternate with random ones.  Every result is
compared element by element with the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_sort, need_gpu, sorter

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dfr():
    return need_gpu()


def _runs(n, seed, mean_run):
    """Keys in runs of equal values with geometric run lengths."""
    g = np.random.default_rng(seed)
    lens = g.geometric(1.0 / mean_run, size=2 * (n // mean_run) + 16)
    vals = g.integers(0, 1 << 32, size=lens.size, dtype=np.uint64).astype(np.uint32)
    out = np.repeat(vals, lens)[:n]
    assert out.size == n
    return out


def _check(dfr, a):
    k, _, st = gpu_sort(dfr, a)
    assert st == dfr.DFR_OK
    assert np.array_equal(k, oracle.sort_u32(a))


@pytest.mark.parametrize("n", [70_001, 1_000_003, 3_000_017])
def test_sorted_and_reverse(dfr, n):
    a = np.sort(synth.uniform_u32(n, synth.BASE_SEED + 2000 + n))
    _check(dfr, a)
    _check(dfr, a[::-1].copy())


@pytest.mark.parametrize("mean_run", [7, 100, 4000, 50_000])
def test_random_runs(dfr, mean_run):
    _check(dfr, _runs(2_000_003, 2100 + mean_run, mean_run))


def test_sawtooth_and_organ_pipe(dfr):
    n = 2_500_007
    base = np.sort(synth.uniform_u32(n // 5 + 1, synth.BASE_SEED + 2200))
    saw = np.tile(base, 5)[:n]
    _check(dfr, saw)
    half = np.sort(synth.uniform_u32(n // 2, synth.BASE_SEED + 2201))
    _check(dfr, np.concatenate([half, half[::-1], half[:7]]))


def test_runs_across_tile_edges(dfr):
    # runs whose lengths are near multiples of the tile (512 x 24) and of a
    # warp chunk (32 x 4), so run ends land inside, at and just past chunk
    # and tile boundaries
    g = np.random.default_rng(2300)
    lens = []
    for L in (128, 127, 129, 12288, 12287, 12289, 24576, 4096):
        lens += [L] * 40
    g.shuffle(lens)
    vals = g.integers(0, 1 << 32, size=len(lens), dtype=np.uint64).astype(np.uint32)
    a = np.repeat(vals, lens)
    _check(dfr, a)
    _check(dfr, np.sort(a))


def test_mixed_run_and_random_tiles(dfr):
    # blocks of one repeated key alternate with blocks of random keys, so a
    # CTA's next tile often differs in kind from its last
    g = np.random.default_rng(2400)
    parts = []
    for i in range(60):
        m = int(g.integers(5_000, 60_000))
        if i % 2:
            parts.append(g.integers(0, 1 << 32, size=m, dtype=np.uint64).astype(np.uint32))
        else:
            parts.append(np.full(m, g.integers(0, 1 << 32), dtype=np.uint32))
    _check(dfr, np.concatenate(parts))


def test_sorted_misaligned_view(dfr):
    import torch

    n = 1_500_001
    a = np.sort(synth.uniform_u32(n, synth.BASE_SEED + 2500))
    s = sorter(dfr, dfr.DFR_U32, n + 3)
    for lead in (1, 2, 3):
        base = torch.zeros(n + lead, dtype=torch.int32, device="cuda")
        base[lead:] = torch.from_numpy(a[::-1].copy().view(np.int32)).cuda()
        view = base[lead:]
        assert s.sort_(view) == dfr.DFR_OK
        assert s.device_status() == dfr.DFR_OK
        assert np.array_equal(view.cpu().numpy().view(np.uint32), a), lead


def test_u64_sorted_runs(dfr):
    n = 1_200_007
    a = np.sort(synth.uniform64_u64(n, synth.BASE_SEED + 2600))
    k, _, st = gpu_sort(dfr, a[::-1].copy())
    assert st == dfr.DFR_OK and np.array_equal(k, oracle.sort_u64(a))
    b = np.repeat(synth.uniform64_u64(n // 1000 + 1, synth.BASE_SEED + 2601), 1000)[:n]
    k, _, st = gpu_sort(dfr, b)
    assert st == dfr.DFR_OK and np.array_equal(k, oracle.sort_u64(b))


@pytest.mark.parametrize("share", [0.5, 0.7, 0.95, 0.999])
def test_dominant_digit(dfr, share):
    # one top byte held by a large share of the keys at random positions (the
    # scatter's dominant-digit ranking), the rest uniform; and one heavy value
    # inside that heavy bucket (a dominant digit again at the next level)
    n = 2_000_011
    g = np.random.default_rng(int(share * 1000) + 2700)
    a = g.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    pick = g.random(n) < share
    a[pick] = (a[pick] & np.uint32(0x00FFFFFF)) | np.uint32(0x5A000000)
    _check(dfr, a)
    heavy = g.random(n) < share * share
    b = a.copy()
    b[heavy] = np.uint32(0x5A3C1234)
    _check(dfr, b)


def test_workspace_sized_above_the_geometry_switch(dfr):
    # a workspace sized for more than 2^22 keys (large-tile geometry) serves a
    # call just below 2^22 keys (small-tile geometry)
    import torch

    n_cap = (1 << 22) + 5
    s = dfr.Sorter(dfr.DFR_U32, n_cap)
    for n in ((1 << 22) - 3, (1 << 22) - 100_000, 1 << 22, n_cap):
        a = synth.uniform_u32(n, synth.BASE_SEED + 2800 + n)
        dk = dfr.to_device(a)
        assert s.sort_(dk) == dfr.DFR_OK
        assert s.device_status() == dfr.DFR_OK
        assert np.array_equal(dfr.to_numpy(dk, np.uint32), oracle.sort_u32(a)), n
    del s
    torch.cuda.empty_cache()
