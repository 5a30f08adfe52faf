"""Host-side checks of the shared-memory index maps the FFT kernels use
(csrc/common.cuh: swz, wstride, stockham_out_index; csrc/render_fwd.cu and
csrc/render_bwd.cu: work-row strides and skews).  The maps are mirrored here
and tied to the source by the text checks in test_mirrors_match_the_source.

Pinned: every map stays inside its row and is one-to-one (no access leaves a
work row, no two elements share a slot); the real row transforms pair rows p
and p + N/2 that the last column pass leaves in one thread, covering each pair
once; and, by a model of the shared-memory banks (32 banks of 4 bytes; an
8-byte access is served per half-warp, a 4-byte one per warp), the chosen maps
make every pass pattern of a 128- or 256-point transform take the minimum
number of wavefronts, which the i + i/8 map does not."""

import math
import os
import re
from collections import defaultdict

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2012_15797_gb300", "csrc")
SIZES = (32, 64, 128, 256)
LAST_RADIX = {32: 4, 64: 8, 128: 2, 256: 4}
# radix schedules per side (Radix<N, V> in common.cuh); the first pass is radix 8
SCHEDULE = {0: {32: (8, 4), 64: (8, 8), 128: (8, 8, 2), 256: (8, 8, 4)},
            1: {32: (8, 2, 2), 64: (8, 4, 2), 128: (8, 4, 4), 256: (8, 4, 8)}}


def swz_xor(n):
    return n >= 128


def swz(n, i):
    return i ^ ((i >> 3) & 15) if swz_xor(n) else i + (i >> 3)


def wstride(n):
    return n if swz_xor(n) else n + n // 8


def stockham_out_index(n, r, j, ns, q, m):
    b = j + q * (n // 8)
    return (b // ns) * ns * r + (b % ns) + m * ns


def wavefronts(word_addrs, width):
    """Shared-memory wavefronts of one warp-wide access of `width` 4-byte
    words per lane (1: a warp at a time; 2: a half-warp at a time)."""
    groups = [range(32)] if width == 1 else [range(0, 16), range(16, 32)]
    total = 0
    for g in groups:
        banks = defaultdict(set)
        for lane in g:
            for w in range(width):
                banks[(word_addrs[lane] + w) % 32].add(word_addrs[lane] + w)
        total += max(len(s) for s in banks.values())
    return total


def test_mirrors_match_the_source():
    common = open(os.path.join(CSRC, "common.cuh")).read()
    assert "constexpr bool swz_xor() { return N >= 128; }" in common
    assert "return swz_xor<N>() ? (i ^ ((i >> 3) & 15)) : i + (i >> 3);" in common
    assert "return swz_xor<N>() ? N : N + N / 8;" in common
    assert "return (b / ns) * ns * R + (b & (ns - 1)) + m * ns;" in common
    fwd = open(os.path.join(CSRC, "render_fwd.cu")).read()
    assert "static constexpr int WS = wstride<N>() + (N == 128 ? 2 : N == 64 ? 16 : 0);" in fwd
    assert "static constexpr int SKEW = N == 64 ? 4 : 0;" in fwd
    assert re.search(r"row\(int r\) \{ return r \* WS \+ SKEW \* \(\(r >> 1\) & 1\); \}", fwd)
    for v, table in SCHEDULE.items():
        for n, r in table.items():
            rr = list(r) + [1] * (3 - len(r))
            spec = f"Radix<{n}>" if v == 0 else f"Radix<{n}, {v}>"
            line = (f"template <> struct {spec} {{ static constexpr int P = {len(r)}; "
                    f"static constexpr int r[3] = {{{rr[0]}, {rr[1]}, {rr[2]}}}; }};")
            assert line in common, line
    bwd = open(os.path.join(CSRC, "render_bwd.cu")).read()
    assert "static constexpr int WSA = N == 64 ? 88 : N == 128 ? 129 : WS;" in bwd
    assert "static constexpr int SKEWA = N == 64 ? 4 : 0;" in bwd


@pytest.mark.parametrize("n", SIZES)
def test_index_map_is_one_to_one_inside_the_row(n):
    slots = [swz(n, i) for i in range(n)]
    assert len(set(slots)) == n
    assert min(slots) >= 0 and max(slots) < wstride(n)


@pytest.mark.parametrize("n", (32, 64, 128))
def test_forward_work_rows_do_not_overlap(n):
    ws = wstride(n) + (2 if n == 128 else 16 if n == 64 else 0)
    skew = 4 if n == 64 else 0
    assert skew <= ws - wstride(n)
    rows = [r * ws + skew * ((r >> 1) & 1) for r in range(n // 2)]
    for a, b in zip(rows, rows[1:]):
        assert b - a >= wstride(n)
    if n == 64:   # rows stay 16-byte aligned for the float4 output reads
        assert all(r % 2 == 0 for r in rows)


def test_schedules_factor_the_sides():
    for table in SCHEDULE.values():
        for n, r in table.items():
            assert r[0] == 8 and all(x in (2, 4, 8) for x in r)
            prod = 1
            for x in r:
                prod *= x
            assert prod == n
            # passes after the first read with a stride N / R that the
            # i + i/8 map needs to be a multiple of 8
            assert all((n // x) % 8 == 0 for x in r[1:])


@pytest.mark.parametrize("v", [0, 1])
@pytest.mark.parametrize("n", SIZES)
def test_row_pairs_meet_in_one_thread(n, v):
    """The last column pass leaves outputs m and m + R/2 of a thread in rows p
    and p + N/2; over all threads those p cover [0, N/2) once (both radix
    schedules)."""
    r = SCHEDULE[v][n][-1]
    assert v != 0 or r == LAST_RADIX[n]
    ns = n // r
    seen = []
    for j in range(n // 8):
        for q in range(8 // r):
            for m in range(r // 2):
                p = stockham_out_index(n, r, j, ns, q, m)
                assert stockham_out_index(n, r, j, ns, q, m + r // 2) == p + n // 2
                seen.append(p)
    assert sorted(seen) == list(range(n // 2))


def _pass_patterns(n, index_map):
    """Word addresses per warp instruction of the five pass access patterns
    of one transform held by 16 (N = 128) or 32 (N = 256) lanes."""
    tpf = n // 8
    lanes = range(tpf) if tpf == 32 else list(range(16)) * 2
    r1, r2 = 8, LAST_RADIX[n]
    pats = []
    for m in range(8):
        pats.append([2 * index_map(8 * j + m) for j in lanes])                             # first-pass store
        pats.append([2 * index_map(j + (n // r1) * m) for j in lanes])                     # pass-2 load
        pats.append([2 * index_map((j // 8) * 64 + j % 8 + 8 * m) for j in lanes])         # pass-2 store
        pats.append([2 * index_map(j + tpf * m) for j in lanes])                           # first-pass load
    for q in range(8 // r2):
        for m in range(r2):
            pats.append([2 * index_map(j + tpf * q + (n // r2) * m) for j in lanes])      # pass-3 load
    return pats


@pytest.mark.parametrize("n", (128, 256))
def test_large_transforms_take_the_minimum_wavefronts(n):
    chosen = _pass_patterns(n, lambda i: swz(n, i))
    assert all(wavefronts(p, 2) == 2 for p in chosen)   # 16 lanes x 8 bytes per half-warp: one wavefront each
    # with i + i/8 a half-warp's 16th lane meets its first lane's banks
    linear = _pass_patterns(n, lambda i: i + (i >> 3))
    assert sum(wavefronts(p, 2) for p in linear) > 2 * len(linear)


def test_adjoint_untangle_writes_spread_over_the_banks():
    """The adjoint's untangle writes column k of 16 rows per half-warp for
    N = 128: an odd row stride gives each lane its own bank pair."""
    n, tpf, wsa = 128, 16, 129
    for w in range(2):
        for i in range(1, n // 2 // tpf):
            addrs = []
            for lane in range(32):
                f, j = divmod(w * 32 + lane, tpf)
                addrs.append(2 * ((j + tpf * i) * wsa + swz(n, f)))
            assert wavefronts(addrs, 2) == 2


def shfl_out_index(j, k):
    return (j & 7) + 8 * ((k & 3) + (4 if j & 8 else 0)) + 64 * (k >> 2)


def _dft(v, sign):
    r = len(v)
    return [sum(v[m] * complex(math.cos(2 * math.pi * m * k / r), sign * math.sin(2 * math.pi * m * k / r))
                for m in range(r)) for k in range(r)]


def test_shuffle_schedule_128_is_the_dft_and_pairs_rows():
    """The third 128-point schedule (8 x 8 x 2, the radix-2 pass across lane
    pairs j, j ^ 8 by shuffles), run as the kernel runs it, lane by lane: its
    outputs, placed by shfl_out_index, are the length-128 inverse DFT; and
    the row pairs p, p + 64 it leaves in one lane (v[i], v[i + 4]) cover
    [0, 64) once."""
    import numpy as np
    common = open(os.path.join(CSRC, "common.cuh")).read()
    assert "return (j & 7) + 8 * ((k & 3) + ((j & 8) ? 4 : 0)) + 64 * (k >> 2);" in common
    assert ("template <> struct Radix<128, 2> { static constexpr int P = 3; "
            "static constexpr int r[3] = {8, 8, 2}; };") in common
    n, tpf = 128, 16
    rng = np.random.default_rng(5)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = lambda e: complex(math.cos(2 * math.pi * e / n), math.sin(2 * math.pi * e / n))   # w_128^e, sign +1
    buf = [0j] * n
    for j in range(tpf):                       # pass 1 (sub-length 1): x[j + 16 m] -> slots 8 j + k
        y = _dft([x[j + tpf * m] for m in range(8)], +1)
        for k in range(8):
            buf[8 * j + k] = y[k]
    v = {}
    for j in range(tpf):                       # pass 2 (radix 8 at sub-length 8), kept in registers
        vals = [buf[j + 16 * m] * (w(m * (j & 7) * 2) if m else 1) for m in range(8)]
        v[j] = _dft(vals, +1)
        for k in range(8):
            assert stockham_out_index(n, 8, j, 8, 0, k) == 64 * (j >> 3) + (j & 7) + 8 * k
    out = {}
    for j in range(tpf):                       # pass 3: lanes j and j ^ 8 exchange four values each
        up = bool(j & 8)
        recv = [v[j ^ 8][i] if (j ^ 8) & 8 else v[j ^ 8][4 + i] for i in range(4)]
        res = [0j] * 8
        for i in range(4):
            x0 = recv[i] if up else v[j][i]
            x1 = v[j][4 + i] if up else recv[i]
            t = w((j & 7) + (32 if up else 0) + 8 * i)
            res[i], res[4 + i] = x0 + t * x1, x0 - t * x1
        for k in range(8):
            out[shfl_out_index(j, k)] = res[k]
    assert sorted(out) == list(range(n))
    ref = np.fft.ifft(x) * n
    got = np.array([out[e] for e in range(n)])
    assert np.max(np.abs(got - ref)) < 1e-9 * np.max(np.abs(ref))
    rows = [shfl_out_index(j, i) for j in range(tpf) for i in range(4)]
    assert all(shfl_out_index(j, i + 4) == shfl_out_index(j, i) + 64 for j in range(tpf) for i in range(4))
    assert sorted(rows) == list(range(64))
