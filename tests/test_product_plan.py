"""Host logic of the split-BF16 product's schedule (no GPU): the slice pairs
(s, t) with s + t < S, taken in units of up to 2 x 2 that share their
operand tiles, spread over the CTAs of an output tile, and the tiles of a
symmetric product (on and above the diagonal).  Queried through
pjac_product_plan, which makes the same plan the product kernel runs."""
import math

import pytest

from paper_2607_23187_b300 import pjac

SHAPES = [(4096, 4096, 4096, False), (4096, 4096, 4096, True), (2048, 2048, 2048, True),
          (1024, 1024, 1024, True), (130, 130, 7, True), (300, 200, 4100, False),
          (64, 72, 5000, False), (1, 1, 1, False), (700, 700, 4100, True)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2607_23187_b300 import build_lib
    build_lib.build()
    return pjac.load()


@pytest.mark.parametrize("m,n,k,sym", SHAPES)
def test_plan_covers_every_slice_pair_once(m, n, k, sym):
    info, pairs = pjac.product_plan(m, n, k, symmetric=sym, sms=148)
    # digit width and slice count of the splitting: partial sums of one
    # pair below 2^24 (K (2^b - 1)^2 <= 2^24), b S >= 54
    b = 6 if k * 63 * 63 <= 2 ** 24 else 5
    S = -(-54 // b)
    assert (info["b"], info["S"]) == (b, S)
    want = {(s, t) for s in range(S) for t in range(S) if s + t < S}
    got = [(s, t) for s, t, _, _ in pairs]
    assert info["pairs"] == len(want) == len(got)
    assert len(set(got)) == len(got) and set(got) == want
    # units: at most four pairs, inside one 2 x 2 block at even (s0, t0)
    units = {}
    for s, t, u, z in pairs:
        units.setdefault(u, []).append((s, t, z))
    assert len(units) == info["units"]
    for u, ps in units.items():
        assert 1 <= len(ps) <= 4
        assert len({(s // 2, t // 2) for s, t, _ in ps}) == 1
        assert len({z for _, _, z in ps}) == 1          # a unit is never split
    # splits: contiguous runs of units in launch order, none empty
    zs = [z for _, _, _, z in pairs]
    us = [u for _, _, u, _ in pairs]
    assert zs == sorted(zs) and us == sorted(us)
    assert set(zs) == set(range(info["splits"])) and 1 <= info["splits"] <= 16
    # CTAs: output tiles of 128 x 128 (on and above the diagonal when
    # symmetric) times the splits
    tm, tn = math.ceil(m / 128), math.ceil(n / 128)
    tiles = tn * (tn + 1) // 2 if sym else tm * tn
    assert info["ctas"] == tiles * info["splits"]


def test_units_at_the_benchmark_order():
    """n = 4096: 15 units (ten full 2 x 2 blocks and five single pairs on
    the last diagonal), one CTA per output tile."""
    info, pairs = pjac.product_plan(4096, 4096, 4096, sms=148)
    assert info["units"] == 15 and info["splits"] == 1
    sizes = {}
    for _, _, u, _ in pairs:
        sizes[u] = sizes.get(u, 0) + 1
    assert sorted(sizes.values()) == [1] * 5 + [4] * 10
    singles = sorted((s, t) for s, t, u, _ in pairs if sizes[u] == 1)
    assert singles == [(0, 8), (2, 6), (4, 4), (6, 2), (8, 0)]
    info_s, _ = pjac.product_plan(4096, 4096, 4096, symmetric=True, sms=148)
    assert info_s["ctas"] == 32 * 33 // 2


def test_plan_rejects_bad_queries():
    lib = pjac.load()
    import ctypes
    info = (ctypes.c_int * 6)()
    assert lib.pjac_product_plan(0, 4, 4, 0, 148, info, None, 0) == pjac.PJAC_EINVAL
    assert lib.pjac_product_plan(4, 5, 4, 1, 148, info, None, 0) == pjac.PJAC_EINVAL   # symmetric, m != n
    assert lib.pjac_product_plan(4, 4, 4, 2, 148, info, None, 0) == pjac.PJAC_EINVAL
    assert lib.pjac_product_plan(4, 4, 4, 0, 148, None, None, 0) == pjac.PJAC_EINVAL
    assert lib.pjac_product_plan(4, 4, 20000, 0, 148, info, None, 0) == pjac.PJAC_EINVAL   # k > PJAC_MAX_N
    # the largest k has a plan (5-bit digits, 11 slices)
    assert lib.pjac_product_plan(4, 4, 16384, 0, 148, info, None, 0) == pjac.PJAC_OK
    assert (info[0], info[1]) == (5, 11)
