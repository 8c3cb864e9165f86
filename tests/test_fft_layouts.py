"""Shared-memory layouts of the FFT exchanges (csrc/fft.cuh), checked on the host.

A length-N Stockham transform with E values per thread (TPT = N / E threads)
writes, after a stage of radix R with NS = R_1 ... R_{l-1}, output r of
butterfly j = t + b TPT to position (j / NS) NS R + (j mod NS) + r NS, and the
next stage (radix RN) reads input r of butterfly j at j + r N / RN.  A padded
layout stores position p at F(p); the kernels compute F(base) once per
butterfly and add F(offset), which needs F(base + o) = F(base) + F(o) ("no
carry").  Shared memory serves a warp's 8-byte accesses per half-warp: sixteen
lanes in one wavefront when they reach sixteen distinct bank pairs (slot index
mod 16, after multiplying by the W transforms interleaved in a column layout).

These tests restate the three padding policies and check, for the 512-point
plans of the one-warp-per-row pass and the staged column pass and for the
768- and 384-point row and column tiles of the work queue, that every exchange
is free of carries, injective within the slot, and takes the minimum number of
wavefronts, and that the plain Pad16 layouts collide where the other policies
were introduced to avoid it.
"""

import pytest


def pad16(p):
    return p + p // 16


def pad8(p):
    return p + p // 8


def pad64x8(p):
    return p + 8 * (p // 64)


def _stages(radices):
    ns, out = 1, []
    for r in radices:
        out.append((r, ns))
        ns *= r
    return out


def _wavefronts(addrs):
    total = 0
    for half in (addrs[:16], addrs[16:]):
        banks = {}
        for a in half:
            banks.setdefault(a % 16, set()).add(a)
        total += max(len(v) for v in banks.values())
    return total


def _accesses(n, e, radices, x, layout, lane_map, w, warps):
    """Per warp instruction, the 32 lanes' slot indices of the write and the read of exchange x."""
    tpt = n // e
    st = _stages(radices)
    r_, ns = st[x]
    rn = st[x + 1][0]
    writes, reads = [], []
    for wp in range(warps):
        for b in range(e // r_):
            for r in range(r_):
                a = []
                for lane in range(32):
                    t, c = lane_map(wp, lane)
                    j = t + b * tpt
                    a.append(layout(((j // ns) * ns * r_ + j % ns) + r * ns) * w + c)
                writes.append(a)
        for b in range(e // rn):
            for r in range(rn):
                a = []
                for lane in range(32):
                    t, c = lane_map(wp, lane)
                    a.append(layout(t + b * tpt + r * (n // rn)) * w + c)
                reads.append(a)
    return writes, reads


def _no_carry(n, e, radices, x, f):
    tpt = n // e
    st = _stages(radices)
    r_, ns = st[x]
    rn = st[x + 1][0]
    for t in range(tpt):
        for b in range(e // r_):
            j = t + b * tpt
            base = (j // ns) * ns * r_ + j % ns
            for r in range(r_):
                if f(base + r * ns) != f(base) + f(r * ns):
                    return False
        for b in range(e // rn):
            j = t + b * tpt
            for r in range(rn):
                if f(j + r * (n // rn)) != f(j) + f(r * (n // rn)):
                    return False
    return True


ROW = lambda wp, lane: (32 * wp + lane, 0)          # one transform per row, lanes on consecutive positions
COL4 = lambda wp, lane: (8 * wp + lane // 4, lane % 4)   # four interleaved columns, eight positions per warp

COL8 = lambda wp, lane: (4 * wp + lane // 8, lane % 8)    # eight interleaved columns (768-point queue tiles)
COL16 = lambda wp, lane: (2 * wp + lane // 16, lane % 16)  # sixteen (384-point queue tiles)
ROW16 = lambda wp, lane: (lane % 16, 0)                    # a 16-thread row per half-warp (384-point rows)

CASES = {
    # name: (N, E, radices, lane map, W, warps per transform set, layouts per exchange (the last
    # one serves every later exchange))
    "warp_row_512": (512, 16, (8, 8, 8), ROW, 1, 1, (pad16, pad64x8)),
    "staged_col_512": (512, 8, (8, 8, 8), COL4, 4, 8, (pad8, pad16)),
    "queue_row_768": (768, 24, (8, 8, 4, 3), ROW, 1, 1, (pad16, pad64x8)),
    "queue_col_768": (768, 24, (8, 8, 4, 3), COL8, 8, 8, (pad8, pad16)),
    "queue_row_384": (384, 24, (8, 8, 2, 3), ROW16, 1, 1, (pad16, pad64x8)),
    "queue_col_384": (384, 24, (8, 8, 2, 3), COL16, 16, 8, (pad8, pad16)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_layouts_carry_free_injective_minimal(name):
    n, e, radices, lane_map, w, warps, lays = CASES[name]
    slot = max(f(n - 1) for f in lays) + 1
    assert slot <= n + n // 8               # the slot the kernels allocate: the longer policy's size
    for x in range(len(radices) - 1):
        f = lays[min(x, len(lays) - 1)]
        assert _no_carry(n, e, radices, x, f), (name, x)
        assert len({f(p) for p in range(n)}) == n and max(f(p) for p in range(n)) < slot
        writes, reads = _accesses(n, e, radices, x, f, lane_map, w, warps)
        for a in writes + reads:
            assert _wavefronts(a) == 2, (name, x)


def test_pad16_collides_where_512_layouts_differ():
    # rows: the write after the second stage; columns: the write after the first stage
    writes, _ = _accesses(512, 16, (8, 8, 8), 1, pad16, ROW, 1, 1)
    assert max(_wavefronts(a) for a in writes) == 4
    writes, _ = _accesses(512, 8, (8, 8, 8), 0, pad16, COL4, 4, 8)
    assert max(_wavefronts(a) for a in writes) == 4
    # and Pad16 is minimal for the other exchange of each
    for x, lm, w, wp, e in ((0, ROW, 1, 1, 16), (1, COL4, 4, 8, 8)):
        writes, reads = _accesses(512, e, (8, 8, 8), x, pad16, lm, w, wp)
        assert all(_wavefronts(a) == 2 for a in writes + reads)


PLANS = {
    # N: (E, radices) of fft::Plan<N> and fft::WarpPlan<512>
    64: (8, (8, 8)), 128: (8, (8, 4, 4)), 256: (8, (8, 8, 4)), 512: (8, (8, 8, 8)),
    1024: (8, (8, 8, 4, 4)), 2048: (16, (8, 8, 8, 4)), 4096: (16, (8, 8, 8, 8)),
    384: (24, (8, 8, 2, 3)), 768: (24, (8, 8, 4, 3)), "warp512": (16, (8, 8, 8)),
}
POLICIES = {"Pad16": (pad16, 16), "Pad8": (pad8, 8), "Pad64x8": (pad64x8, 64)}


def _write_ok(ns, r, k):
    # the compile-time condition of write_out (fft.cuh)
    m = ns * r
    return ns % k == 0 or (k % ns == 0 and m % k == 0) or (m <= k and k % m == 0)


def _read_ok(n, rn, k):
    # the compile-time condition of read_in (fft.cuh)
    return (n // rn) % k == 0 or k % (n // rn) == 0


@pytest.mark.parametrize("plan", sorted(PLANS, key=str))
@pytest.mark.parametrize("policy", sorted(POLICIES))
def test_static_carry_conditions_are_sound(plan, policy):
    """Wherever the kernels' static_asserts accept a policy for an exchange,
    the padded addresses really are base plus offset for every butterfly."""
    n = 512 if plan == "warp512" else plan
    e, radices = PLANS[plan]
    f, k = POLICIES[policy]
    st = _stages(radices)
    for x in range(len(radices) - 1):
        r_, ns = st[x]
        rn = st[x + 1][0]
        if _write_ok(ns, r_, k) and _read_ok(n, rn, k):
            assert _no_carry(n, e, radices, x, f), (plan, policy, x)


def test_pad16_accepted_for_every_plan():
    # the layouts every other kernel uses must compile for every plan
    for plan, (e, radices) in PLANS.items():
        n = 512 if plan == "warp512" else plan
        st = _stages(radices)
        for x in range(len(radices) - 1):
            r_, ns = st[x]
            assert _write_ok(ns, r_, 16) and _read_ok(n, st[x + 1][0], 16), (plan, x)
