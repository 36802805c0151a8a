"""The plane kernel's shared-memory layout (CPU model): row y of the plane holds position p
at y * N2 + pswz(y, p), pswz(y, p) = (p & ~15) | ((p & 15) ^ (2 (p >> 4) & 15) ^ (9 if y odd)),
the kernel's swizzle restated.  Modelled here with 32 four-byte banks, a float2 access by a
half-warp of 16 threads being one wavefront when the 16 float2 indices differ mod 16:
  - the map is a bijection within each row,
  - the column phase (a warp on 32 consecutive kz at one position) is conflict-free,
  - the two Stockham patterns of the 8-thread row transforms (positions t + 8 i and
    8 t + r, two rows per half-warp) are conflict-free,
  - the real-split mirror reads (position N2 - k) cost 512 extra wavefronts per 128-row
    plane, in line with the 0.13 M conflicts per 128-plane launch that ncu counts.
The separable march's plane kernel (pft_sep.cuh) is modelled the same way: its column and
row exchange maps are bijections, the float view agrees with the float2 view, and the
column phase, the transposed row accesses and both Stockham patterns of the row
transforms are conflict-free at N = 64 and 128.
Every map is read from the kernel source (its return expression, translated to Python), so
the model follows the layout the kernels use."""
import os
import re
from collections import Counter

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1204_5434_gb300", "csrc")
N2 = 64
NY = 128


def _source_map(fname, pattern, consts=None):
    """The return expression of a one-line index function of a kernel header, as a Python
    function of its two arguments (C ternaries and integer division translated)."""
    with open(os.path.join(CSRC, fname)) as f:
        src = f.read()
    m = re.search(pattern, src)
    assert m, (fname, pattern)
    a, b, expr = m.group(1), m.group(2), " ".join(m.group(3).split())
    expr = re.sub(r"\(([^()]+)\) \? (\w+) : (\w+)", r"(\2 if (\1) else \3)", expr)
    expr = expr.replace(" / ", " // ")
    env = dict(consts or {})
    return eval(f"lambda {a}, {b}: {expr}", env)


pswz = _source_map("pft_plane.cuh", r"int pswz\(int (y), int (p)\) \{\s*return ([^;]+);")


def test_source_map_is_the_documented_swizzle():
    for y in range(4):
        for p in range(N2):
            assert pswz(y, p) == (p & ~15) | ((p & 15) ^ (((p >> 4) << 1) & 15) ^ (9 if (y & 1) else 0))


def extra_wavefronts(idx):
    return max(Counter(a % 16 for a in idx).values()) - 1


def test_bijection_within_rows():
    for y in range(4):
        assert sorted(pswz(y, p) for p in range(N2)) == list(range(N2))


def test_column_phase_is_conflict_free():
    total = 0
    for pos in range(NY):
        for kz0 in range(0, N2, 16):
            total += extra_wavefronts([pos * N2 + pswz(pos, kz0 + j) for j in range(16)])
    assert total == 0


def test_row_transform_patterns_are_conflict_free():
    a = b = mirror = 0
    for y0 in range(0, NY, 2):
        rows = (y0, y0 + 1)
        for i in range(8):
            a += extra_wavefronts([y * N2 + pswz(y, t + 8 * i) for y in rows for t in range(8)])
            b += extra_wavefronts([y * N2 + pswz(y, 8 * t + i) for y in rows for t in range(8)])
            mirror += extra_wavefronts([y * N2 + pswz(y, (N2 - (t + 8 * i)) % N2) for y in rows for t in range(8)])
    assert a == 0 and b == 0
    assert mirror == 512


# ------------------------------------------------- separable march plane kernel (pft_sep.cuh)
def _sep_maps(N, RSH):
    c = {"N": N, "RSH": RSH}
    pat = r"static __forceinline__ int {}\(int (\w+), int (\w+)\) \{{ return ([^;]+); \}}"
    return (_source_map("pft_sep.cuh", pat.format("ucol"), c), _source_map("pft_sep.cuh", pat.format("ucol_f"), c),
            _source_map("pft_sep.cuh", pat.format("urow"), c))


# (N, log2 of the first radix, the first radix): Plan<128> = 16 x 8, Plan<64> = 8 x 8
SEP = [(128, 4, 16), (64, 3, 8)]


def test_separable_maps_are_bijections_and_views_agree():
    for N, RSH, _ in SEP:
        ucol, ucol_f, urow = _sep_maps(N, RSH)
        for y in range(8):
            assert sorted(ucol(y, cc) for cc in range(N // 2)) == list(range(y * (N // 2), (y + 1) * (N // 2)))
            assert sorted(ucol_f(y, k) for k in range(N)) == list(range(y * N, (y + 1) * N))
            for cc in range(N // 2):
                for h in range(2):
                    assert ucol_f(y, 2 * cc + h) == 2 * ucol(y, cc) + h
            assert sorted(urow(y, p) for p in range(N)) == list(range(y * N, (y + 1) * N))


def test_separable_column_and_transposed_accesses_are_conflict_free():
    for N, RSH, _ in SEP:
        ucol, ucol_f, _u = _sep_maps(N, RSH)
        col = tr = 0
        for y in range(N):
            for cc0 in range(0, N // 2, 16):  # a half-warp on 16 consecutive column pairs of one row
                col += extra_wavefronts([ucol(y, cc0 + j) for j in range(16)])
        for y0 in range(0, N, 4):  # eight threads on eight consecutive floats of four rows
            for k0 in range(0, N, 8):
                idx = [ucol_f(y0 + r, k0 + t) for r in range(4) for t in range(8)]
                tr += max(Counter(a % 32 for a in idx).values()) - 1
        assert col == 0 and tr == 0, (N, col, tr)


def test_separable_row_transform_patterns_are_conflict_free():
    for N, RSH, R1 in SEP:
        _c, _f, urow = _sep_maps(N, RSH)
        put = get = 0
        for L0 in range(0, N // 2, 2):  # two lines of eight threads per half-warp
            lines = (L0, L0 + 1)
            for r in range(R1):   # first stage: thread t puts position R1 t + r
                put += extra_wavefronts([urow(L, R1 * t + r) for L in lines for t in range(8)])
            for i in range(N // 8):  # second stage: thread t gets position t + 8 i
                get += extra_wavefronts([urow(L, t + 8 * i) for L in lines for t in range(8)])
        assert put == 0 and get == 0, (N, put, get)
