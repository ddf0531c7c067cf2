// Host-side layout of a masked grid: row-compacted storage, the column / segment partition of
// the rows among the blocks of a team, and the active-cell bitmask.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace cmx {

// Cells are stored per (y, z) row: the span from the row's first magnetic x (xs) rounded down
// to a multiple of ROW_ALIGN to its last magnetic x + 1 (xe) rounded up, at a storage offset
// that is a multiple of ROW_ALIGN as well.  rows[z*ny + y] = (offset of the stored span, xs | xe<<16);
// box cell x of the row is stored at offset + x - (xs rounded down).  Stored cells outside
// [xs, xe) are padding; non-magnetic cells inside it are holes.  Both are inactive.
struct Layout {
    int nx = 0, ny = 0, nz = 0;
    int ncell = 0, ncell_mag = 0;
    bool holes = false;             // some row has a non-magnetic cell inside [xs, xe)
    bool padded = false;            // some stored cell is inactive (holes or padding)
    std::vector<int2> rows;
    std::vector<int> box_of_cell;   // box index of each stored cell
    std::vector<uint8_t> active;    // 1 = magnetic (stored cells)
};

void build_layout(Layout &L, int nx, int ny, int nz, const uint8_t *mask);

// 32-bit words of the active-cell bitmask (bit i of word i/32 = stored cell i is magnetic).
std::vector<uint32_t> active_bits(const Layout &L);

// Columns of ix x iy cells (x0 a multiple of ix, y0 of iy) with the planes that hold magnetic
// cells and a work weight per plane.
struct Column {
    int x0, y0, zlo, zhi;
    std::vector<float> w;
};
std::vector<Column> build_columns(const Layout &L, int ix, int iy);

// Split the columns into segments (x0, y0, z0, z1) and give `blocks` blocks contiguous runs of
// them with balanced work; begin[b] .. begin[b+1] are block b's segments.  Returns false if the
// partition cannot cover every plane of every column within `blocks` blocks of at most
// MAX_BLOCK_SEGMENTS segments each (the caller must reject the problem or the launch shape).
bool build_segments(const std::vector<Column> &cols, int blocks, std::vector<int4> &segs,
                    std::vector<int> &begin);

}  // namespace cmx
