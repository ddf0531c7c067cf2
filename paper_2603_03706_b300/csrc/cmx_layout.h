// Host-side layout of a masked grid: row-compacted storage, the column / segment partition of
// the rows among the blocks of a team, and the active-cell bitmask.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace cmx {

// Cells are stored per (y, z) row between the first and the last magnetic x of the row, the
// span widened to multiples of `align` cells; cells in it that are not magnetic are holes
// (inactive).  rows[z*ny + y] = (offset, xs | xe<<16).  With align = 4 every row starts at a
// multiple of 4 stored cells and ncell is a multiple of 4 (16-byte aligned groups of four).
struct Layout {
    int nx = 0, ny = 0, nz = 0;
    int ncell = 0, ncell_mag = 0;
    bool holes = false;
    std::vector<int2> rows;
    std::vector<int> box_of_cell;   // box index of each stored cell
    std::vector<uint8_t> active;    // 1 = magnetic (stored cells)
};

void build_layout(Layout &L, int nx, int ny, int nz, const uint8_t *mask, int align = 1);

// 32-bit words of the active-cell bitmask (bit i of word i/32 = stored cell i is magnetic).
std::vector<uint32_t> active_bits(const Layout &L);

// Columns of (wx-2) x (wy-2) interior cells of a wx x wy block window, with the planes that
// hold magnetic cells and a work weight per plane.
struct Column {
    int x0, y0, zlo, zhi;
    std::vector<float> w;
};
std::vector<Column> build_columns(const Layout &L, int wx, int wy);

// Split the columns into segments (x0, y0, z0, z1) and give `blocks` blocks contiguous runs of
// them with balanced work; begin[b] .. begin[b+1] are block b's segments.
void build_segments(const std::vector<Column> &cols, int blocks, std::vector<int4> &segs,
                    std::vector<int> &begin);

}  // namespace cmx
