// Host-side layout of a masked grid (see cmx_layout.h).
#include <algorithm>

#include "cmx_internal.cuh"
#include "cmx_layout.h"

namespace cmx {

void build_layout(Layout &L, int nx, int ny, int nz, const uint8_t *mask)
{
    constexpr int align = ROW_ALIGN;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.rows.assign((size_t)ny * nz, make_int2(0, 0));
    L.box_of_cell.clear();
    L.active.clear();
    L.holes = false;
    int off = 0, nmag = 0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++) {
            const size_t rb = ((size_t)z * ny + y) * nx;
            int xs = -1, xe = -1;
            for (int x = 0; x < nx; x++)
                if (mask[rb + x]) {
                    if (xs < 0) xs = x;
                    xe = x + 1;
                }
            if (xs < 0) {
                L.rows[(size_t)z * ny + y] = make_int2(off, 0);
                continue;
            }
            // the stored span starts and ends on multiples of `align` (cells beyond the box are
            // inactive padding), so that aligned groups of `align` cells are aligned in memory
            const int xa = xs - xs % align;
            const int xb = (xe + align - 1) / align * align;
            L.rows[(size_t)z * ny + y] = make_int2(off, xs | (xe << 16));
            for (int x = xa; x < xb; x++) {
                const bool in = x >= xs && x < xe;
                const bool on = in && mask[rb + x];
                if (in && !on) L.holes = true;
                L.box_of_cell.push_back((int)(rb + std::min(x, nx - 1)));
                L.active.push_back(on ? 1 : 0);
                nmag += on ? 1 : 0;
            }
            off += xb - xa;
        }
    L.ncell = off;
    L.ncell_mag = nmag;
    L.padded = nmag != off;
}

std::vector<uint32_t> active_bits(const Layout &L)
{
    std::vector<uint32_t> bits(((size_t)L.ncell + 31) / 32, 0u);
    for (size_t i = 0; i < (size_t)L.ncell; i++)
        if (L.active[i]) bits[i >> 5] |= 1u << (i & 31);
    return bits;
}

// Columns of (wx-2) x (wy-2) interior cells (a wx x wy thread window with its one-cell rim):
// the range of planes [zlo, zhi) that hold magnetic cells of the column, and per plane a work
// weight (1: a plane iteration is latency-bound and costs about the same whatever its cells).
std::vector<Column> build_columns(const Layout &L, int ix, int iy)
{
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int bx = ix, by = iy;
    auto count = [&](int x0, int x1, int y0, int y1, int z) {
        int n = 0;
        if (z < 0 || z >= nz) return 0;
        for (int y = std::max(0, y0); y < std::min(ny, y1); y++) {
            const int2 r = L.rows[(size_t)z * ny + y];
            const int xs = r.y & 0xffff, xe = (int)((unsigned)r.y >> 16);
            const int base = r.x - (xs - xs % ROW_ALIGN);
            for (int x = std::max(xs, x0); x < std::min(xe, x1); x++) n += L.active[base + x];
        }
        return n;
    };
    std::vector<Column> out;
    for (int y0 = 0; y0 < ny; y0 += by)
        for (int x0 = 0; x0 < nx; x0 += bx) {
            Column c{x0, y0, -1, -1, {}};
            std::vector<float> w(nz);
            for (int z = 0; z < nz; z++) {
                const int inner = count(x0, x0 + bx, y0, y0 + by, z);
                if (inner > 0) {
                    if (c.zlo < 0) c.zlo = z;
                    c.zhi = z + 1;
                }
                w[z] = 1.0f;   // a plane iteration costs about the same whatever its cells
            }
            if (c.zlo >= 0) {
                c.w.assign(w.begin() + c.zlo, w.begin() + c.zhi);
                out.push_back(std::move(c));
            }
        }
    return out;
}

// Greedy fill of blocks with capacity `cap` (plane weights plus two halo planes per segment):
// each block takes planes of consecutive columns until the next plane would exceed its
// capacity; columns are cut into segments at block boundaries and every MAX_TILE_PLANES - 2
// planes.  Returns the number of blocks used (segments and block starts in segs / begin).
static int fill_blocks(const std::vector<Column> &cols, double cap, int max_blocks,
                std::vector<int4> &segs, std::vector<int> &begin)
{
    segs.clear();
    begin.assign(1, 0);
    double load = 0.0;
    int nseg_block = 0;
    for (const Column &c : cols) {
        int z = c.zlo;
        while (z < c.zhi) {
            // a new segment costs its two halo planes plus at least one plane
            if (nseg_block > 0 && (load + 2.0 + c.w[z - c.zlo] > cap ||
                                   nseg_block >= MAX_BLOCK_SEGMENTS)) {
                begin.push_back((int)segs.size());
                if ((int)begin.size() - 1 >= max_blocks) return max_blocks + 1;
                load = 0.0;
                nseg_block = 0;
            }
            load += 2.0;
            int len = 0;
            while (z + len < c.zhi && len < MAX_TILE_PLANES - 2 &&
                   (len == 0 || load + c.w[z + len - c.zlo] <= cap)) {
                load += c.w[z + len - c.zlo];
                len++;
            }
            segs.push_back(make_int4(c.x0, c.y0, z, z + len));
            nseg_block++;
            z += len;
        }
    }
    begin.push_back((int)segs.size());
    return (int)begin.size() - 1;
}

// Smallest per-block capacity (binary search) whose greedy fill needs at most `blocks`
// blocks; the partition then has no block above that capacity.  False if even the largest
// capacity cannot place every plane (too many columns for MAX_BLOCK_SEGMENTS per block).
bool build_segments(const std::vector<Column> &cols, int blocks, std::vector<int4> &segs,
                    std::vector<int> &begin)
{
    double total = 0.0, wmax = 0.0;
    long long planes = 0;
    for (const Column &c : cols) {
        for (float v : c.w) {
            total += v;
            wmax = std::max(wmax, (double)v);
        }
        planes += c.zhi - c.zlo;
    }
    double lo = std::max(total / blocks, 2.0 + wmax), hi = total + 2.0 * (total + cols.size());
    if (fill_blocks(cols, hi, blocks, segs, begin) > blocks) return false;
    for (int it = 0; it < 60 && hi - lo > 0.5; it++) {
        const double mid = 0.5 * (lo + hi);
        if (fill_blocks(cols, mid, blocks, segs, begin) <= blocks)
            hi = mid;
        else
            lo = mid;
    }
    if (fill_blocks(cols, hi, blocks, segs, begin) > blocks) return false;
    while ((int)begin.size() < blocks + 1) begin.push_back((int)segs.size());
    // every plane of every column is in exactly one segment
    long long covered = 0;
    for (const int4 &t : segs) covered += t.w - t.z;
    for (size_t b = 0; b + 1 < begin.size(); b++)
        if (begin[b + 1] - begin[b] > MAX_BLOCK_SEGMENTS) return false;
    return covered == planes;
}


}  // namespace cmx
