"""The plane kernel's shared-memory layout (CPU model): row y of the plane holds position p
at y * N2 + pswz(y, p), pswz(y, p) = (p & ~15) | ((p & 15) ^ (2 (p >> 4) & 15) ^ (9 if y odd)),
the kernel's swizzle restated.  Modelled here with 32 four-byte banks, a float2 access by a
half-warp of 16 threads being one wavefront when the 16 float2 indices differ mod 16:
  - the map is a bijection within each row,
  - the column phase (a warp on 32 consecutive kz at one position) is conflict-free,
  - the two Stockham patterns of the 8-thread row transforms (positions t + 8 i and
    8 t + r, two rows per half-warp) are conflict-free,
  - the real-split mirror reads (position N2 - k) cost 512 extra wavefronts per 128-row
    plane, in line with the 0.13 M conflicts per 128-plane launch that ncu counts."""
from collections import Counter

N2 = 64
NY = 128


def pswz(y, p):
    return (p & ~15) | ((p & 15) ^ (((p >> 4) << 1) & 15) ^ (9 if (y & 1) else 0))


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
