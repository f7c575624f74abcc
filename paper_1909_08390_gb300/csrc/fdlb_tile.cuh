// fdlb_tile.cuh -- index arithmetic of a stage kernel's tile, shared by the
// device kernels and a host build (the index checks of the CPU tests): which
// tile position a staged element holds and which grid cell feeds it (5 ghost
// nodes per side by clamp or wrap, Sec. IV), and which tile positions and
// interface slots a march task reads and writes.
#pragma once

#if defined(__CUDACC__)
#define FDLB_HD __host__ __device__ __forceinline__
#else
#define FDLB_HD inline
#endif

namespace fdlb {

constexpr int kGhost = 5;  // ghost nodes per side (Sec. IV)

// Grid index of tile position i (may lie up to kGhost outside [0, n)): the
// adjacent fluid node's index (outlet, bc 0) or the periodic image (bc 1).
FDLB_HD int wrap_or_clamp(int i, int n, int bc) {
  if (bc == 1) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Staged element e of a tile of TX x TY cells (2-D) or TX cells (1-D) with
// its halo, in the compact order that skips the 2-D corner blocks (they feed
// no line): the kGhost rows above the tile (tile columns only), the tile's
// rows with both side halos, the kGhost rows below (tile columns only).
// Returns the element count; (r, c) is e's row and column in the tile
// buffer, whose cell (kGhost, kGhost) is the tile's first cell (1-D: row 0).
FDLB_HD int staged_count(int dim, int TX, int TY) {
  return dim == 2 ? TY * (TX + 2 * kGhost) + 2 * kGhost * TX : TX + 2 * kGhost;
}
FDLB_HD void staged_pos(int e, int dim, int TX, int TY, int& r, int& c) {
  const int SXH = TX + 2 * kGhost;
  if (dim == 1) {
    r = 0;
    c = e;
  } else if (e < kGhost * TX) {
    r = e / TX;
    c = kGhost + e % TX;
  } else if (e < kGhost * TX + TY * SXH) {
    r = kGhost + (e - kGhost * TX) / SXH;
    c = (e - kGhost * TX) % SXH;
  } else {
    r = kGhost + TY + (e - kGhost * TX - TY * SXH) / TX;
    c = kGhost + (e - kGhost * TX - TY * SXH) % TX;
  }
}

// Chunked landing of a 2-D tile (grids whose rows hold a multiple of 4
// cells): the staged region is copied in 16-byte chunks of 4 cells into a
// landing buffer of chunk_count(TX, TY) chunks, chunk q at slots 4q..4q+3:
// first the kGhost rows above the tile (its TX columns, TX/4 chunks a row),
// then the tile's TY rows from column x0 - 8 to x0 + TX + 8 ((TX+16)/4
// chunks, the 5-cell halos rounded out to whole chunks), then the kGhost rows
// below.  chunk_offset gives chunk q's first cell as an offset from the
// population's first cell: rows clamp (outlet) or wrap (periodic) as a
// whole; periodic columns wrap chunk by chunk; an outlet chunk reaching past
// the left or right edge is not copied (-1), and chunk_slot sends the cells
// that would read it to the edge column instead (the ghost value), which the
// row's other chunks hold.  chunk_slot gives the landing slot of staged
// position (r, c) (the tile's first cell at (kGhost, kGhost)).
FDLB_HD int chunk_count(int TX, int TY) { return (2 * kGhost * TX + TY * (TX + 16)) / 4; }
FDLB_HD int chunk_offset(int q, int TX, int TY, int x0, int y0, int nx, int ny, int bc) {
  const int top = kGhost * TX / 4, mid = TY * (TX + 16) / 4;
  int r, col;
  if (q < top) {
    r = q / (TX / 4);
    col = x0 + (q % (TX / 4)) * 4;
  } else if (q < top + mid) {
    r = kGhost + (q - top) / ((TX + 16) / 4);
    col = x0 - 8 + ((q - top) % ((TX + 16) / 4)) * 4;
  } else {
    r = kGhost + TY + (q - top - mid) / (TX / 4);
    col = x0 + ((q - top - mid) % (TX / 4)) * 4;
  }
  const int rr = wrap_or_clamp(y0 - kGhost + r, ny, bc);
  if (bc == 1) return rr * nx + wrap_or_clamp(col, nx, 1);
  return (col >= 0 && col + 4 <= nx) ? rr * nx + col : -1;
}
FDLB_HD int chunk_slot(int r, int c, int TX, int TY, int x0, int nx, int bc) {
  int cc = x0 - kGhost + c;
  if (bc != 1) cc = cc < 0 ? 0 : (cc >= nx ? nx - 1 : cc);
  if (r < kGhost) return r * TX + (cc - x0);
  if (r < kGhost + TY) return kGhost * TX + (r - kGhost) * (TX + 16) + (cc - x0 + 8);
  return kGhost * TX + TY * (TX + 16) + (r - kGhost - TY) * TX + (cc - x0);
}

// March task of thread tid for a group of populations: which population of
// the group (tg), whether it marches an x line (in 2-D, lines 0..TY-1 are
// the tile's rows, TY..TY+TX-1 its columns), and, for velocity sign sgn,
// the tile position of the upwind cell of its first interface (row `br`,
// column `bc_`), the element step from one interface's upwind cell to the
// next (`stride`, in tile-buffer elements of row pitch SX, signed with sgn),
// and the interface slot of its first output (`orow`, `ofirst`: row of hx or
// column of hy, and slot; later outputs step by sgn).  Interface i of a line
// lies between its cells i-1 and i; a line has TX+1 (x) or TY+1 (y)
// interfaces in segments of SEG, marched upwind to downwind; for p < 0 the
// construction is the mirror image (index s+j <-> s+1-j).
struct MarchTask {
  int tg;
  bool xline;
  int br, bc_, stride, orow, ofirst;
};
FDLB_HD MarchTask march_task(int tid, int dim, int TX, int TY, int SEG, int SX, int sgn) {
  const int nline = dim == 2 ? TX + TY : 1;
  const int nseg = (TX + 1) / SEG;
  MarchTask t;
  t.tg = tid / (nline * nseg);
  const int tline = (tid / nseg) % nline;
  const int tseg = tid % nseg;
  t.xline = dim == 1 || tline < TY;
  const int i0 = tseg * SEG;
  t.ofirst = sgn > 0 ? i0 : i0 + SEG - 1;
  const int up = (sgn > 0 ? t.ofirst - 1 : t.ofirst) + kGhost;
  if (t.xline) {
    t.orow = dim == 2 ? tline : 0;
    t.br = dim == 2 ? tline + kGhost : 0;
    t.bc_ = up;
    t.stride = sgn;
  } else {
    t.orow = tline - TY;
    t.br = up;
    t.bc_ = tline - TY + kGhost;
    t.stride = sgn * SX;
  }
  return t;
}

}  // namespace fdlb
