"""Host checks of the 3D steps' work partition (hydro_debug_pieces walks the
same PieceIter the step kernels walk; no GPU needed).

* chunked grid: CTA (tile, chunk) marches exactly planes [chunk Z, chunk Z + Z)
  of its tile, clipped to the column;
* balanced grid: the pieces of all G CTAs cover every (tile, plane) exactly
  once; every CTA marches the same number of planes, give or take one; the
  first pieces of CTA b are the whole chunks b, b + G, ... (chunks ordered row
  by row), as many as there are whole waves of G chunks; the rest is marched
  from the last piece back.
"""

import itertools

import numpy as np
import pytest

from paper_1510_05061_gb300 import hydro


@pytest.fixture(scope="module")
def hy():
    from paper_1510_05061_gb300 import build

    build.build()
    hydro.load()
    return hydro


def test_chunked_grid_one_piece(hy):
    assert hy.hydro_debug_pieces(16, tiles=9, nz=45, tile=4, chunk=2) == [(4, 32, 45)]
    assert hy.hydro_debug_pieces(16, tiles=9, nz=45, tile=0, chunk=0) == [(0, 0, 16)]
    with pytest.raises(hy.HydroError):
        hy.hydro_debug_pieces(16, tiles=9, nz=45, tile=0, chunk=3)   # past the column
    with pytest.raises(hy.HydroError):
        hy.hydro_debug_pieces(-1, tiles=9, nz=45, G=4, b=4)           # no such CTA


CASES = list(itertools.product(
    (1, 9, 64, 256, 257),            # tiles
    (1, 5, 45, 64, 256),             # planes per column
    (-1, -4, -7, -64, -128, -10**6),  # balanced grid settings
    (1, 3, 152, 456),                # CTAs of the grid
))


@pytest.mark.parametrize("tiles,nz,zchunk,G", CASES)
def test_balanced_grid_partition(hy, tiles, nz, zchunk, G):
    W = tiles * nz
    if G > W:
        G = W                       # the launcher never starts more CTAs than plane-tiles
    Z = nz if zchunk >= -1 else min(-zchunk, nz)
    nch = -(-nz // Z)
    I = tiles * nch
    waves = I // G
    seen = np.zeros((tiles, nz), dtype=np.int32)
    planes = []
    for b in range(G):
        pieces = hy.hydro_debug_pieces(zchunk, tiles, nz, G=G, b=b)
        n = 0
        for j, (t, z0, z1) in enumerate(pieces):
            assert 0 <= t < tiles and 0 <= z0 < z1 <= nz, (b, pieces)
            seen[t, z0:z1] += 1
            n += z1 - z0
            if j < waves:
                # whole chunk b + j G, chunks ordered row by row
                i = b + j * G
                c, tt = divmod(i, tiles)
                assert (t, z0, z1) == (tt, c * Z, min(c * Z + Z, nz)), (b, j, pieces)
        # the split part is marched from its last piece back: its pieces'
        # positions in the chunk order decrease
        keys = [((z0 // Z) * tiles + t) * Z + z0 % Z for t, z0, _ in pieces[waves:]]
        assert keys == sorted(keys, reverse=True), (b, pieces)
        planes.append(n)
    assert np.all(seen == 1)
    if nz % Z == 0:
        # equal chunks: every CTA marches the same number of planes, give or take one
        assert max(planes) - min(planes) <= 1, (min(planes), max(planes))


def test_balanced_shares_are_even(hy):
    # RT 256^3 with 16 x 16 tiles on 152 CTAs: one wave of whole columns, the
    # other 104 columns split; 128-plane chunks: three waves, 56 chunks split
    for zchunk in (-1, -128, -64):
        counts = [sum(z1 - z0 for _, z0, z1 in hy.hydro_debug_pieces(zchunk, 256, 256, G=152, b=b))
                  for b in range(152)]
        assert sum(counts) == 256 * 256
        assert max(counts) - min(counts) <= 1, (zchunk, min(counts), max(counts))
