"""Scratch sizing of the chunk table (host arithmetic, CPU only).

A plan reserves work items for the sizes of the calls made on it and grows
the reservation (which allocates) only when a call needs more.  Calls too
small to give every resident warp two items halve their chunk, and a smaller
chunk means more items, so a smaller call can need more items than a larger
one.  The reserve must therefore cover every call up to the sizes reserved
for, whatever chunk it gets: otherwise a smaller call captured in a CUDA
graph after a warm-up with the largest sizes would allocate inside the
capture.  These tests check degrid_schedule_reserve through the C ABI
against a model of the chunk table's item counts.
"""
import ctypes

import numpy as np
import pytest

from paper_2102_12739_gb300 import _native, build

SPARSE_ITEMS = 64       # a list shorter than 64 chunks is sparse: items of 64 visibilities


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def query(lib, sms, plan_chunk, S, n):
    c, k = ctypes.c_int(), ctypes.c_int64()
    rc = lib.degrid_schedule_reserve(sms, plan_chunk, S, n, ctypes.byref(c), ctypes.byref(k))
    assert rc == _native.DG_OK
    return c.value, k.value


def items_needed(counts, chunk):
    """Items of the chunk table of one call (sparse lists in items of 64)."""
    small = 64 if chunk > 64 else 0
    total = 0
    for n in counts:
        size = small if small and n < SPARSE_ITEMS * chunk else chunk
        total += -(-int(n) // size)
    return total


def expected_chunk(sms, plan_chunk, n):
    c = plan_chunk
    while c > 64 and c % 64 == 0 and n // c < 2 * 16 * sms:
        c //= 2
    return c


def test_call_chunk_halves_for_small_calls(lib):
    for sms in (1, 152, 160):
        for plan_chunk in (64, 96, 128, 192, 256, 512, 1024, 4096):
            for n in (0, 1, 20_000, 1_300_000, 2_000_000, 16_000_000):
                assert query(lib, sms, plan_chunk, 1, n)[0] == expected_chunk(sms, plan_chunk, n)


def test_reserve_covers_the_example_of_a_smaller_call_with_more_items(lib):
    # 160 SMs, one subgrid, chunk 256: 2,000,000 visibilities keep chunk 256,
    # 1,300,000 drop to chunk 128 and need more items than the larger call
    c_big, k_big = query(lib, 160, 256, 1, 2_000_000)
    c_small, _ = query(lib, 160, 256, 1, 1_300_000)
    assert (c_big, c_small) == (256, 128)
    assert items_needed([1_300_000], 128) > items_needed([2_000_000], 256)
    assert k_big >= items_needed([1_300_000], 128)


def test_reserve_grows_with_the_sizes(lib):
    rng = np.random.default_rng(3)
    for sms in (152, 160):
        for plan_chunk in (128, 256, 512, 1024):
            ns = np.unique(np.concatenate([
                rng.integers(0, 40_000_000, 300),
                # around every halving boundary n = 4 * warps * c
                [4 * 16 * sms * c + d for c in (64, 128, 256, 512) for d in (-2, -1, 0, 1)]]))
            for S in (1, 7, 64, 512, 5000):
                prev = -1
                for n in ns:
                    k = query(lib, sms, plan_chunk, S, int(n))[1]
                    assert k >= prev, (sms, plan_chunk, S, n)
                    prev = k
            for n in (0, 1000, 3_000_000):
                ks = [query(lib, sms, plan_chunk, S, n)[1] for S in range(0, 300, 7)]
                assert ks == sorted(ks)


def test_reserve_covers_every_smaller_call(lib):
    # random count vectors (dense, sparse and empty lists): the items of any
    # call with at most S subgrids and N visibilities fit the reserve of
    # (S, N), for the chunk that call gets
    rng = np.random.default_rng(11)
    for trial in range(400):
        sms = int(rng.choice([1, 8, 152, 160]))
        plan_chunk = int(rng.choice([128, 256, 512, 1024]))
        S = int(rng.integers(1, 600))
        counts = np.where(rng.random(S) < 0.2, 0,
                          np.round(10 ** rng.uniform(0, rng.uniform(2, 7), S))).astype(np.int64)
        n = int(counts.sum())
        chunk = query(lib, sms, plan_chunk, S, n)[0]
        need = items_needed(counts, chunk)
        S_big = S + int(rng.integers(0, 50))
        n_big = n + int(rng.integers(0, 3 * max(n, 1)))
        _, reserve = query(lib, sms, plan_chunk, S_big, n_big)
        assert need <= reserve, (trial, sms, plan_chunk, S, n, S_big, n_big)


def test_reserve_rejects_bad_arguments(lib):
    k = ctypes.c_int64()
    assert lib.degrid_schedule_reserve(0, 256, 1, 10, None, ctypes.byref(k)) == _native.DG_ERR_ARG
    assert lib.degrid_schedule_reserve(152, 100, 1, 10, None, ctypes.byref(k)) == _native.DG_ERR_ARG
    assert lib.degrid_schedule_reserve(152, 256, -1, 10, None, ctypes.byref(k)) == _native.DG_ERR_ARG
    assert lib.degrid_schedule_reserve(152, 256, 1, -1, None, ctypes.byref(k)) == _native.DG_ERR_ARG
    assert lib.degrid_schedule_reserve(152, 256, 1, 10, None, None) == _native.DG_OK
