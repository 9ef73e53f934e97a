// lbm_copy_plan.h -- which bulk copies stage one tile of the TMA-pipelined
// passes into shared memory.  Shared by the kernels (device) and by the
// host self-check (lbm_selfcheck), which proves on the CPU, for many
// lattice shapes, that every copy is 16-byte aligned on both sides, has a
// size that is a multiple of 16, stays inside its lattice's allocation and
// its shared-memory box, and that together the copies cover every value an
// active site reads.
//
// Stage layout (bytes): nine population boxes, then (for the collision
// pass) the psi box.  Box 0 (the rest plane) holds rows y0 - 1 + r
// (r < TY + 2), box i (i >= 1) rows y0 - c_iy + r (r < TY), all with lattice
// columns [x0 - H, x0 + TX + H): the value a site pulls, f*_i(x - c_i,
// y - c_iy), sits in box row y - y0 (box 0: y - y0 + 1) at column
// x - x0 + H - c_ix, and the rest value of its source site, R(x - c_i), in
// box 0, row y - y0 + 1 - c_iy.  The psi box holds rows y0 - 1 + rr
// (rr < TY + 2) and columns [x0 - 4, x0 + TX + 4).
#pragma once
#include "lbm_device.cuh"

namespace pplbm {

__host__ __device__ constexpr int align128(int v) { return (v + 127) / 128 * 128; }

template <int ES, int TX, int TY, bool WITH_PSI>
struct TileGeo {
    static constexpr int H = 16 / ES;                  // halo columns kept per side (16 bytes)
    static constexpr int BW = TX + 2 * H;              // population box width (elements)
    static constexpr int ROWS0 = TY + 2;               // rows of box 0
    static constexpr int BOX0B = align128(ROWS0 * BW * ES);
    static constexpr int BOXB = align128(TY * BW * ES);  // boxes 1..8
    static constexpr int POPB = BOX0B + 8 * BOXB;       // the psi box starts here
    static constexpr int PW = TX + 8;                  // psi box width (floats)
    static constexpr int PSIB = WITH_PSI ? align128((TY + 2) * PW * 4) : 0;
    static constexpr int HDRB = align128((int)sizeof(LatDev) + 16);  // tile + its lattice
    static constexpr int HDR = POPB + PSIB;                          // header offset
    static constexpr int STAGEB = HDR + HDRB;
    static constexpr int NCOPY = ROWS0 + 8 * TY + (WITH_PSI ? TY + 2 : 0);
    // byte offset of box i in the stage
    static __host__ __device__ constexpr int boxoff(int i) {
        return i == 0 ? 0 : BOX0B + (i - 1) * BOXB;
    }
    // element offsets, in the stage, of what site (tx, ty) of the tile pulls
    // from plane i, and of the rest value R(x - c_i) of its source site
    static __host__ __device__ constexpr int pull(int i, int tx, int ty) {
        return i == 0 ? (ty + 1) * BW + tx + H : boxoff(i) / ES + ty * BW + tx + H - plane_cx(i);
    }
    static __host__ __device__ constexpr int rest(int i, int tx, int ty) {
        return (ty + 1 - plane_cy(i)) * BW + tx + H - plane_cx(i);
    }
};

struct CopyOp {
    int64_t src;  // byte offset into the population arena (psi = false) or psi arena
    int32_t dst;  // byte offset inside the stage
    int32_t bytes;
    bool psi;
};

// Copy q of the tile with origin (x0, y0) of lattice L, reading population
// buffer `parity`.  Returns false when the copy is not needed (its rows lie
// beyond what active sites read).
template <int ES, int TX, int TY, bool WITH_PSI>
__host__ __device__ inline bool plan_copy(const LatDev& L, int parity, int x0, int y0, int q,
                                          CopyOp& op) {
    using G = TileGeo<ES, TX, TY, WITH_PSI>;
    if (q < G::ROWS0 + 8 * TY) {
        int i, r, y;  // box, its row, the lattice row it holds
        if (q < G::ROWS0) {
            i = 0;
            r = q;
            y = y0 - 1 + r;
        } else {
            const int k = q - G::ROWS0;
            i = 1 + k / TY;
            r = k - (k / TY) * TY;
            y = y0 - plane_cy(i) + r;
        }
        if (y < -1 || y > L.ny) return false;
        const int avail = L.pitch - (x0 - G::H + L.gx);  // columns left in the row
        const int cols = avail < G::BW ? avail : G::BW;
        op.src = (L.off_f[parity] + (int64_t)i * L.plane + (int64_t)(y + GY) * L.pitch +
                  (x0 - G::H + L.gx)) *
                 ES;
        op.dst = G::boxoff(i) + r * G::BW * ES;
        op.bytes = cols * ES;
        op.psi = false;
        return true;
    }
    const int rr = q - G::ROWS0 - 8 * TY;
    const int y = y0 - 1 + rr;
    if (y > L.ny) return false;
    const int avail = L.pitch_psi - (x0 - 4 + L.gx_psi);
    const int cols = avail < G::PW ? avail : G::PW;
    op.src = (L.off_psi + (int64_t)(y + GY) * L.pitch_psi + (x0 - 4 + L.gx_psi)) * 4;
    op.dst = G::POPB + rr * G::PW * 4;
    op.bytes = cols * 4;
    op.psi = true;
    return true;
}

// ---- single-pass (fused) step --------------------------------------------
// Stage layout (bytes): nine population boxes.  Box i (i >= 1) holds
// ROWS = TY + 2 rows: box row rr is lattice row y0 - 1 - c_iy + rr, so the
// value a cell (x, y) of the tile or of its one-site ring pulls,
// f*_i(x - c_ix, y - c_iy), sits in box row y - y0 + 1 at column
// x - c_ix - x0 + H.  Box 0 (the rest plane) holds ROWS0 = TY + 4 rows,
// lattice rows y0 - 2 .. y0 + TY + 1: a cell's own rest value and the rest
// values R(x - c_i) of all its sources (rows y - c_iy).  Columns
// [x0 - H, x0 + TX + H) of the lattice rows.
template <int ES, int TX, int TY>
struct FusedGeo {
    static constexpr int H = 16 / ES;        // halo columns per side (16 bytes)
    static constexpr int BW = TX + 2 * H;    // box width (elements)
    static constexpr int ROWS = TY + 2;      // rows of boxes 1..8
    static constexpr int ROWS0 = TY + 4;     // rows of box 0
    static constexpr int BOX0B = align128(ROWS0 * BW * ES);
    static constexpr int BOXB = align128(ROWS * BW * ES);
    static constexpr int STAGEB = BOX0B + 8 * BOXB;
    static constexpr int NCOPY = ROWS0 + 8 * ROWS;
    static __host__ __device__ constexpr int boxoff(int i) {
        return i == 0 ? 0 : BOX0B + (i - 1) * BOXB;
    }
    static __host__ __device__ constexpr int rows(int i) { return i == 0 ? ROWS0 : ROWS; }
    // element offsets, in the stage, of what cell (lx, ly) of the tile
    // (-1 .. TX, -1 .. TY) pulls from plane i, and of the rest value of its
    // source site R(x - c_i)
    static __host__ __device__ constexpr int pull(int i, int lx, int ly) {
        return i == 0 ? (ly + 2) * BW + lx + H
                      : boxoff(i) / ES + (ly + 1) * BW + lx + H - plane_cx(i);
    }
    static __host__ __device__ constexpr int rest(int i, int lx, int ly) {
        return (ly + 2 - plane_cy(i)) * BW + lx + H - plane_cx(i);
    }
};

// Copy q of the fused tile with origin (x0, y0) of lattice L, reading
// population buffer `parity`.  Rows outside the lattice allocation (beyond
// the ghost frame of a ragged last tile) are not copied; no active cell
// reads them.
template <int ES, int TX, int TY>
__host__ __device__ inline bool plan_copy_fused(const LatDev& L, int parity, int x0, int y0, int q,
                                                CopyOp& op) {
    using G = FusedGeo<ES, TX, TY>;
    int i, rr, y;  // box, its row, the lattice row it holds
    if (q < G::ROWS0) {
        i = 0;
        rr = q;
        y = y0 - 2 + rr;
    } else {
        const int k = q - G::ROWS0;
        i = 1 + k / G::ROWS;
        rr = k - (k / G::ROWS) * G::ROWS;
        y = y0 - 1 - plane_cy(i) + rr;
    }
    if (y < -GY || y > L.ny + GY - 1) return false;
    const int avail = L.pitch - (x0 - G::H + L.gx);  // columns left in the row
    const int cols = avail < G::BW ? avail : G::BW;
    op.src = (L.off_f[parity] + (int64_t)i * L.plane + (int64_t)(y + GY) * L.pitch +
              (x0 - G::H + L.gx)) *
             ES;
    op.dst = G::boxoff(i) + rr * G::BW * ES;
    op.bytes = cols * ES;
    op.psi = false;
    return true;
}

// Cell r of the one-site ring around a tile with active extent up to
// (xend, yend): (x0-1 .. xend) x {y0-1, yend} and {x0-1, xend} x (y0 .. yend-1),
// r < 2 (TX + TY) + 4.  Returns false for cells beyond the active region of
// a ragged tile; (gx, gy) are then clamped onto a cell of the region.
__host__ __device__ inline bool ring_cell(int r, int TX, int TY, int x0, int y0, int xend,
                                          int yend, int& gx, int& gy) {
    const int W = TX + 2;
    int lx, ly;
    if (r < W) {
        lx = r;
        ly = 0;
    } else if (r < 2 * W) {
        lx = r - W;
        ly = TY + 1;
    } else {
        const int q = r - 2 * W;  // 2 * TY side cells
        lx = (q & 1) ? TX + 1 : 0;
        ly = 1 + (q >> 1);
    }
    gx = x0 - 1 + lx;
    gy = y0 - 1 + ly;
    // the right/bottom ring of a ragged tile sits at the active edge
    if (lx == TX + 1) gx = xend;
    if (ly == TY + 1) gy = yend;
    const bool on = gx <= xend && gy <= yend;
    gx = gx < xend ? gx : xend;
    gy = gy < yend ? gy : yend;
    return on;
}

// Tensor-path coordinates of tile (x0, y0) of lattice L, whose ghost row -GY
// is row `row0` of the row space, reading population buffer `parity`:
//   load box (TX + 2H) x (TY + 4) x 9 at (x0, row0 + y0, 9 parity): element x0
//     of a row is lattice column x0 - H (the row starts with gx = H ghost
//     columns), row row0 + y0 is lattice row y0 - 2;
//   store box TX x TY x 9 at (x0 + gx, row0 + GY + y0, 9 (parity ^ 1)), used
//     only for tiles inside the lattice (store set): the store unit clips a
//     box at 16-byte granularity in x, so a ragged tile would write ghost
//     columns too.
// x coordinates must be multiples of 16 bytes (lbm_selfcheck checks them,
// and that every store box lies inside its lattice).
struct TmaCoords {
    int lx, ly, lz;  // load box origin
    int sx, sy, sz;  // store box origin
    bool store;      // the tile is stored by one tensor store
};
template <int TX, int TY>
__host__ __device__ inline TmaCoords fused_tma_coords(const LatDev& L, int row0, int parity,
                                                      int x0, int y0) {
    TmaCoords c;
    c.lx = x0;
    c.ly = row0 + y0;
    c.lz = 9 * parity;
    c.sx = x0 + L.gx;
    c.sy = row0 + GY + y0;
    c.sz = 9 * (parity ^ 1);
    c.store = x0 + TX <= L.nx && y0 + TY <= L.ny;
    return c;
}

}  // namespace pplbm
