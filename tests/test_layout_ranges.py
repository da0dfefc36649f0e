"""Bounds of the staged 16-bit step kernel's bulk copies, checked on the CPU
(compute-sanitizer is not available to these tests): for every lattice
width, each copy a task issues must start 16-byte aligned, move whole
16-byte units, fit its shared-memory row buffer, stay inside its padded row
of the population plane (or of the u* plane), and cover every column a real
node of the segment reads; the lanes' shared-memory word reads must stay in
their row buffers.

Layout (as the library creates it for 16-bit storage): xoff = 64 columns
(128 bytes), pitch = round_up(xoff + nx + 8, 64), u* pitch =
round_up(nx + 4, 16) doubles. A task covers columns [x0s, x0s + 128) of one
row; lane l owns nodes x0s + 4 l ... + 3. Copies: q = 0 from x0s - 8 (halo),
q = 2 from x0s, q = 1 and q = 3 (rows y -/+ 1) from x0s, u* from x0s, with
the lengths the kernel computes from rem = min(128, nx - x0s).
"""


def rup(a, b):
    return (a + b - 1) // b * b


SW, HALO = 128, 8
L02, L13 = SW + HALO, SW  # shared row buffers (16-bit elements)


def copies(nx, x0s):
    rem = min(SW, nx - x0s)
    n1 = (rem + 7) & ~7
    n0 = HALO + n1
    n2 = (rem + 8) & ~7
    nu = (rem + 1) & ~1
    return rem, n0, n2, n1, nu


def check_width(nx):
    xoff = 64
    pitch = rup(xoff + nx + 8, 64)
    upitch = rup(nx + 4, 16)
    for seg in range((nx + SW - 1) // SW):
        x0s = seg * SW
        rem, n0, n2, n1, nu = copies(nx, x0s)
        # whole 16-byte units, fitting the shared buffers
        assert n0 <= L02 and n2 <= L02 and n1 <= L13 and nu <= SW
        assert (2 * n0) % 16 == 0 and (2 * n2) % 16 == 0 and (2 * n1) % 16 == 0 and (8 * nu) % 16 == 0
        # 16-byte aligned starts (row starts are: pitch is a multiple of 64 elements)
        assert ((xoff + x0s - HALO) * 2) % 16 == 0 and ((xoff + x0s) * 2) % 16 == 0 and (x0s * 8) % 16 == 0
        # inside the padded row
        assert xoff + x0s - HALO >= 0 and xoff + x0s - HALO + n0 <= pitch
        assert xoff + x0s + n2 <= pitch and xoff + x0s + n1 <= pitch and x0s + nu <= upitch
        # every real node's operands are copied; the shared index of each matches the lane's reads
        for x in range(x0s, x0s + rem):
            assert x0s - HALO <= x - 1 < x0s - HALO + n0      # +x pulls column x - 1
            assert x0s <= x + 1 < x0s + n2                    # -x pulls column x + 1 (ghost nx at most)
            assert x0s <= x < x0s + n1 and x0s <= x < x0s + nu
            l, e = (x - x0s) // 4, (x - x0s) % 4
            assert 4 * l + 7 + e == (x - 1) - (x0s - HALO)
            assert 4 * l + 1 + e == (x + 1) - x0s
    # words each lane reads stay inside the row buffers
    for l in range(32):
        assert 2 * l + 5 < L02 // 2 and 2 * l + 2 < L02 // 2 and 2 * l + 1 < L13 // 2 and 4 * l + 3 < SW


def test_staged_copies_in_bounds_for_every_width():
    for nx in list(range(1, 520)) + [1000, 2896, 4095, 4096, 4097, 8192, 12345]:
        check_width(nx)
