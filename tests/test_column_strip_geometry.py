"""Geometry of the FP32 warp strips with two columns per lane (host-side
arithmetic, no GPU).  A strip owns columns x0 .. x0 + 59; lane l holds
columns X0 + 2l and X0 + 2l + 1 with X0 = x0 - 2; the pulls of a row come
from a 72-float buffer per population starting at B = 4 floor((X0 - 1) / 4),
filled by 18 aligned 16-byte pieces, piece c from lattice column
(B + 4c) mod nx.  Checked for every width that is a multiple of 4 up to
4096 (the GPU tests cover sampled widths bit for bit):
  - every lattice column is owned by exactly one lane of one strip;
  - every pull of every lane (its two columns shifted by -1, 0, +1) lies in
    the buffer, and the aligned 8-byte loads start on even buffer indices;
  - every piece starts on a 16-byte boundary and stays inside its row after
    the periodic wrap, and the buffer's column c holds lattice column
    (B + c) mod nx."""
OWN, BUF = 60, 72


def _strips(nx):
    return range(0, nx, OWN)


def _check(nx):
    owner = [0] * nx
    for x0 in _strips(nx):
        X0 = x0 - 2
        B = (X0 - 1) & ~3
        assert B % 4 == 0 and B <= X0 - 1 and X0 - B <= 4
        # pieces: 16-byte aligned, whole inside the row after the wrap
        for c in range(BUF // 4):
            g = (B + 4 * c) % nx
            assert g % 4 == 0 and g + 3 < nx
        for lane in range(32):
            c0 = X0 + 2 * lane
            assert (c0 - B) % 2 == 0  # the aligned pair of the unshifted pulls
            for half in (0, 1):
                for dx in (-1, 0, 1):
                    j = c0 + half + dx - B
                    assert 0 <= j < BUF, (nx, x0, lane, half, dx)
                    # buffer index j holds column (B + j) mod nx, the pull source
                    assert (B + j) % nx == (c0 + half + dx) % nx
            if 1 <= lane <= OWN // 2 and c0 < nx:
                owner[c0] += 1
                owner[c0 + 1] += 1
    assert owner == [1] * nx, nx


def test_column_pair_strip_geometry():
    for nx in range(4, 4097, 4):
        _check(nx)
