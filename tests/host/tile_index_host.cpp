// Host build of the stage kernels' tile index arithmetic (csrc/fdlb_tile.cuh)
// for the CPU tests: every staged element, ghost source, own cell, march
// read and interface write of every tile of a grid, checked to lie inside
// its array, with staged positions and interface slots each covered once.
// Also the chunked landing of 2-D tiles (16-byte copies of 4 cells).
// Returns the number of violations (0 when all hold); prints the first few.
#include <cstdio>
#include <vector>

#include "../../paper_1909_08390_gb300/csrc/fdlb_tile.cuh"

using namespace fdlb;

static int bad = 0;
#define CHECK(cond, ...)                   \
  do {                                     \
    if (!(cond)) {                         \
      if (bad < 10) {                      \
        std::printf("violated: " #cond " "); \
        std::printf(__VA_ARGS__);          \
        std::printf("\n");                 \
      }                                    \
      ++bad;                               \
    }                                      \
  } while (0)

// One tile shape (dim, TX, TY, SEG, G, NT) on an nx x ny grid with boundary bc.
extern "C" int check_tiles(int dim, int TX, int TY, int SEG, int G, int NT, int nx, int ny,
                           int bc) {
  bad = 0;
  const int H = kGhost;
  const int SXH = TX + 2 * H;
  const int SX = SXH + (dim == 2 ? 1 : 0);
  const int SY = dim == 2 ? TY + 2 * H : 1;
  const int NSC = staged_count(dim, TX, TY);
  const int CELLS = TX * TY;
  const int nline = dim == 2 ? TX + TY : 1;
  const int nseg = (TX + 1) / SEG;
  CHECK(nseg * SEG == TX + 1, "segments");
  CHECK(G * nline * nseg == NT, "one task per thread");
  if (dim == 2) CHECK(TX == TY, "square tiles: y lines use the x segmentation");
  auto corner = [&](int r, int c) {
    return dim == 2 && (r < H || r >= H + TY) && (c < H || c >= H + TX);
  };
  // staged positions: in the buffer, never a corner, each non-corner once
  std::vector<int> seen(SY * SX, 0);
  for (int e = 0; e < NSC; ++e) {
    int r, c;
    staged_pos(e, dim, TX, TY, r, c);
    CHECK(r >= 0 && r < SY && c >= 0 && c < SXH, "e=%d r=%d c=%d", e, r, c);
    if (!(r >= 0 && r < SY && c >= 0 && c < SXH)) continue;
    CHECK(!corner(r, c), "corner e=%d", e);
    ++seen[r * SX + c];
  }
  for (int r = 0; r < SY; ++r)
    for (int c = 0; c < SXH; ++c)
      CHECK(seen[r * SX + c] == (corner(r, c) ? 0 : 1), "coverage r=%d c=%d", r, c);
  // every tile of the grid: ghost sources and own cells
  const int gy_tiles = dim == 2 ? (ny + TY - 1) / TY : 1;
  for (int ty = 0; ty < gy_tiles; ++ty)
    for (int tx = 0; tx < (nx + TX - 1) / TX; ++tx) {
      const int x0 = tx * TX, y0 = ty * TY;
      std::vector<int> own(CELLS, 0);
      for (int e = 0; e < NSC; ++e) {
        int r, c;
        staged_pos(e, dim, TX, TY, r, c);
        const int lx = x0 - H + c, ly = y0 - H + r;
        const int gx = wrap_or_clamp(lx, nx, bc);
        const int gy = dim == 2 ? wrap_or_clamp(ly, ny, bc) : 0;
        CHECK(gx >= 0 && gx < nx && gy >= 0 && gy < (dim == 2 ? ny : 1), "src %d %d", gx, gy);
        if (bc == 0) {
          CHECK(gx == (lx < 0 ? 0 : (lx >= nx ? nx - 1 : lx)), "outlet x");
        } else {
          CHECK(((lx - gx) % nx + nx) % nx == 0, "periodic x");
          if (dim == 2) CHECK(((ly - gy) % ny + ny) % ny == 0, "periodic y");
        }
        const int ox = c - H, oy = dim == 2 ? r - H : 0;
        if (ox >= 0 && ox < TX && oy >= 0 && oy < TY && x0 + ox < nx && y0 + oy < ny) {
          CHECK(oy * TX + ox < CELLS, "own index");
          CHECK(gx == x0 + ox && gy == (dim == 2 ? y0 + oy : 0), "own source");
          ++own[oy * TX + ox];
        }
      }
      for (int o = 0; o < CELLS; ++o) {
        const bool inside = x0 + o % TX < nx && y0 + o / TX < (dim == 2 ? ny : 1);
        CHECK(own[o] == (inside ? 1 : 0), "own cell %d staged %d times", o, own[o]);
      }
    }
  // march tasks: reads inside staged positions, writes inside the interface
  // rows, every interface of every line written once per sign pattern
  for (int sx = -1; sx <= 1; sx += 2)
    for (int sy = -1; sy <= 1; sy += 2) {
      std::vector<int> hx(G * TY * (TX + 1), 0), hy(G * TX * (TY + 1), 0);
      for (int tid = 0; tid < NT; ++tid) {
        MarchTask t0 = march_task(tid, dim, TX, TY, SEG, SX, 1);
        const int sgn = t0.xline ? sx : sy;
        const MarchTask t = march_task(tid, dim, TX, TY, SEG, SX, sgn);
        CHECK(t.tg >= 0 && t.tg < G, "tg");
        const int off0 = t.br * SX + t.bc_;
        auto read_ok = [&](int off) {
          const int r = off / SX, c = off % SX;
          return off >= 0 && r < SY && c < SXH && !corner(r, c);
        };
        for (int j = 0; j < 9; ++j)
          CHECK(read_ok(off0 + (j - 4) * t.stride), "tid=%d window %d", tid, j);
        for (int k = 0; k + 1 < SEG; ++k)
          CHECK(read_ok(off0 + (k + 5) * t.stride), "tid=%d read %d", tid, k);
        for (int k = 0; k < SEG; ++k) {
          const int slot = t.ofirst + k * sgn;
          // the upwind cell of interface `slot` (between line cells slot-1
          // and slot): cell slot-1 for p > 0, slot for p < 0 (Sec. IV and
          // its mirror image), at tile column/row cell + H
          const int up = off0 + k * t.stride, ur = up / SX, uc = up % SX;
          const int ucell = sgn > 0 ? slot - 1 : slot;
          if (t.xline)
            CHECK(uc == ucell + H && ur == (dim == 2 ? t.orow + H : 0), "tid=%d upwind x", tid);
          else
            CHECK(ur == ucell + H && uc == t.orow + H, "tid=%d upwind y", tid);
          if (t.xline) {
            CHECK(slot >= 0 && slot <= TX && t.orow >= 0 && t.orow < TY, "hx write");
            if (slot >= 0 && slot <= TX && t.orow >= 0 && t.orow < TY)
              ++hx[(t.tg * TY + t.orow) * (TX + 1) + slot];
          } else {
            CHECK(slot >= 0 && slot <= TY && t.orow >= 0 && t.orow < TX, "hy write");
            if (slot >= 0 && slot <= TY && t.orow >= 0 && t.orow < TX)
              ++hy[(t.tg * TX + t.orow) * (TY + 1) + slot];
          }
        }
      }
      for (int v : hx) CHECK(v == 1, "hx coverage");
      if (dim == 2)
        for (int v : hy) CHECK(v == 1, "hy coverage");
      // 2-D: one segment per line writes the flux difference of each of its
      // cells, from slot c0 (the first interface's slot, one lower when
      // marching downwards) in steps of sgn
      if (dim == 2) {
        std::vector<int> cx(G * TY * TX, 0), cy(G * TX * TY, 0);
        for (int tid = 0; tid < NT; ++tid) {
          const int sgn = march_task(tid, dim, TX, TY, SEG, SX, 1).xline ? sx : sy;
          const MarchTask t = march_task(tid, dim, TX, TY, SEG, SX, sgn);
          const int c0 = sgn > 0 ? t.ofirst : t.ofirst - 1;
          for (int k = 0; k + 1 < SEG; ++k) {
            const int cell = c0 + k * sgn, n = t.xline ? TX : TY;
            CHECK(cell >= 0 && cell < n, "delta cell %d", cell);
            if (cell >= 0 && cell < n) ++(t.xline ? cx : cy)[(t.tg * (t.xline ? TY : TX) + t.orow) * n + cell];
          }
        }
        for (int v : cx) CHECK(v == 1, "x delta coverage");
        for (int v : cy) CHECK(v == 1, "y delta coverage");
      }
    }
  // pass 1: a thread's own cells and the interface slots they read
  const int cpt = (CELLS + NT - 1) / NT;
  for (int tid = 0; tid < NT; ++tid)
    for (int k = 0; k < cpt; ++k) {
      const int c = tid + k * NT < CELLS ? tid + k * NT : 0;
      const int lx = c % TX, ly = c / TX;
      CHECK(lx + 1 <= TX && ly < TY && ly * TX + lx < CELLS, "own slot");
      if (dim == 2) CHECK(ly + 1 <= TY && lx < TX, "own y slot");
    }
  return bad;
}

// Chunked landing of a 2-D tile (chunk_offset, chunk_slot) on an nx x ny grid
// with nx a multiple of 4: every tile, every copied chunk aligned and inside
// the population, every chunk slot inside the landing buffer, and every
// staged position reading a landed slot that holds the cell it needs (the
// adjacent fluid node past an outlet edge, the periodic image otherwise).
extern "C" int check_chunks(int TX, int TY, int nx, int ny, int bc) {
  bad = 0;
  const int H = kGhost;
  const int NCHK = chunk_count(TX, TY);
  const int NSC = staged_count(2, TX, TY);
  CHECK(nx % 4 == 0 && TX % 4 == 0, "aligned rows");
  for (int y0 = 0; y0 < ny; y0 += TY)
    for (int x0 = 0; x0 < nx; x0 += TX) {
      std::vector<long> land(4 * NCHK, -1);  // cell held by each slot
      for (int q = 0; q < NCHK; ++q) {
        const int o = chunk_offset(q, TX, TY, x0, y0, nx, ny, bc);
        if (o < 0) {
          CHECK(bc == 0, "periodic chunks are always copied");
          continue;
        }
        CHECK(o % 4 == 0 && o + 3 < nx * ny, "chunk q=%d offset %d", q, o);
        CHECK(o % nx + 3 < nx, "chunk within its row");
        for (int k = 0; k < 4; ++k) land[4 * q + k] = o + k;
      }
      for (int e = 0; e < NSC; ++e) {
        int r, c;
        staged_pos(e, 2, TX, TY, r, c);
        const int s = chunk_slot(r, c, TX, TY, x0, nx, bc);
        CHECK(s >= 0 && s < 4 * NCHK, "slot e=%d s=%d", e, s);
        if (!(s >= 0 && s < 4 * NCHK)) continue;
        const long want = (long)wrap_or_clamp(y0 - H + r, ny, bc) * nx + wrap_or_clamp(x0 - H + c, nx, bc);
        CHECK(land[s] == want, "tile (%d,%d) e=%d reads %ld, needs %ld", x0, y0, e, land[s], want);
      }
    }
  return bad;
}
