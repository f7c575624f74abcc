"""The stage kernels' tile index arithmetic (csrc/fdlb_tile.cuh, the code the
kernels call), compiled for the host: on odd grid sizes, tiles that do not
divide the grid and both boundaries, every staged position, ghost source,
own cell, march read and interface write lies inside its array, every staged
position and interface slot is covered exactly once, and ghosts take the
adjacent fluid node (outlet) or the periodic image (Sec. IV)."""
import ctypes
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "tile_index_host.cpp")
HDR = os.path.join(os.path.dirname(HERE), "paper_1909_08390_gb300", "csrc", "fdlb_tile.cuh")
LIB = os.path.join(HERE, "host", "_build", "libtileindex.so")

# (dim, TX, TY, SEG, G, NT): the 2-D tile and the five 1-D tile shapes
SHAPES = [(2, 16, 16, 17, 4, 128), (1, 127, 1, 8, 8, 128), (1, 63, 1, 8, 16, 128),
          (1, 255, 1, 16, 8, 128), (1, 15, 1, 4, 16, 64), (1, 31, 1, 8, 16, 64)]


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                              os.path.getmtime(HDR)):
        tmp = LIB + f".{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", SRC, "-o", tmp], check=True)
        os.replace(tmp, LIB)
    L = ctypes.CDLL(LIB)
    L.check_tiles.argtypes = [ctypes.c_int] * 9
    L.check_chunks.argtypes = [ctypes.c_int] * 5
    return L


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", [0, 1])
def test_tile_indices_stay_in_bounds(lib, shape, bc):
    dim = shape[0]
    sizes = [1, 5, 11, 13, 17] + ([] if dim == 2 else [127, 128, 300])
    for nx in sizes:
        for ny in (sizes if dim == 2 else [1]):
            assert lib.check_tiles(*shape, nx, ny, bc) == 0, (shape, nx, ny, bc)


@pytest.mark.parametrize("bc", [0, 1])
def test_chunked_landing_reads_the_right_cells(lib, bc):
    """2-D tiles of grids whose rows hold a multiple of 4 cells land 16-byte
    chunks; on grids narrower than a tile, ragged tiles and both boundaries,
    each staged position reads the cell (or ghost source) it needs."""
    for nx in (4, 8, 12, 16, 20, 36, 64):
        for ny in (1, 5, 16, 17, 33):
            assert lib.check_chunks(16, 16, nx, ny, bc) == 0, (nx, ny, bc)
