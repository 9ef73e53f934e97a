// lbm_copy_plan.h -- which bulk copies stage one tile of the TMA-pipelined
// passes into shared memory.  Shared by the kernels (device) and by the
// host self-check (lbm_selfcheck), which proves on the CPU, for many
// lattice shapes, that every copy is 16-byte aligned on both sides, has a
// size that is a multiple of 16, stays inside its lattice's allocation and
// its shared-memory box, and that together the copies cover every value an
// active site reads.
//
// Stage layout (bytes): nine population boxes of BOXB bytes, then (for the
// collision pass) the psi box.  Population box i holds rows
// y0 - c_iy + r (r < TY) and lattice columns [x0 - H, x0 + TX + H): the
// value a site pulls, f*_i(x - c_i, y - c_iy), sits in box row y - y0 at
// column x - x0 + H - c_ix.  The psi box holds rows y0 - 1 + rr (rr < TY + 2)
// and columns [x0 - 4, x0 + TX + 4).
#pragma once
#include "lbm_device.cuh"

namespace pplbm {

__host__ __device__ constexpr int align128(int v) { return (v + 127) / 128 * 128; }
__host__ __device__ constexpr int plane_cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int plane_cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}

template <int ES, int TX, int TY, bool WITH_PSI>
struct TileGeo {
    static constexpr int H = 16 / ES;                  // halo columns kept per side (16 bytes)
    static constexpr int BW = TX + 2 * H;              // population box width (elements)
    static constexpr int BOXB = align128(TY * BW * ES);
    static constexpr int BOXE = BOXB / ES;             // box stride in elements
    static constexpr int PW = TX + 8;                  // psi box width (floats)
    static constexpr int PSIB = WITH_PSI ? align128((TY + 2) * PW * 4) : 0;
    static constexpr int HDRB = align128((int)sizeof(LatDev) + 16);  // tile + its lattice
    static constexpr int HDR = 9 * BOXB + PSIB;                       // header offset
    static constexpr int STAGEB = HDR + HDRB;
    static constexpr int NCOPY = 9 * TY + (WITH_PSI ? TY + 2 : 0);
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
    if (q < 9 * TY) {
        const int i = q / TY, r = q - (q / TY) * TY;
        const int y = y0 - plane_cy(i) + r;  // lattice row held by box row r
        if (y < -1 || y > L.ny) return false;
        const int avail = L.pitch - (x0 - G::H + L.gx);  // columns left in the row
        const int cols = avail < G::BW ? avail : G::BW;
        op.src = (L.off_f[parity] + (int64_t)i * L.plane + (int64_t)(y + GY) * L.pitch +
                  (x0 - G::H + L.gx)) *
                 ES;
        op.dst = i * G::BOXB + r * G::BW * ES;
        op.bytes = cols * ES;
        op.psi = false;
        return true;
    }
    const int rr = q - 9 * TY;
    const int y = y0 - 1 + rr;
    if (y > L.ny) return false;
    const int avail = L.pitch_psi - (x0 - 4 + L.gx_psi);
    const int cols = avail < G::PW ? avail : G::PW;
    op.src = (L.off_psi + (int64_t)(y + GY) * L.pitch_psi + (x0 - 4 + L.gx_psi)) * 4;
    op.dst = 9 * G::BOXB + rr * G::PW * 4;
    op.bytes = cols * 4;
    op.psi = true;
    return true;
}

// ---- single-pass (fused) step --------------------------------------------
// Stage layout (bytes): nine population boxes of BOXB bytes.  Box i holds
// ROWS = TY + 2 rows: box row rr is lattice row y0 - 1 - c_iy + rr, so the
// value a cell (x, y) of the tile or of its one-site ring pulls,
// f*_i(x - c_ix, y - c_iy), sits in box row y - y0 + 1 at column
// x - c_ix - x0 + H; columns [x0 - H, x0 + TX + H) of the lattice row.
template <int ES, int TX, int TY>
struct FusedGeo {
    static constexpr int H = 16 / ES;        // halo columns per side (16 bytes)
    static constexpr int BW = TX + 2 * H;    // box width (elements)
    static constexpr int ROWS = TY + 2;      // box rows
    static constexpr int BOXB = align128(ROWS * BW * ES);
    static constexpr int STAGEB = 9 * BOXB;
    static constexpr int NCOPY = 9 * ROWS;
};

// Copy q of the fused tile with origin (x0, y0) of lattice L, reading
// population buffer `parity`.  Rows outside the lattice allocation (beyond
// the ghost frame of a ragged last tile) are not copied; no active cell
// reads them.
template <int ES, int TX, int TY>
__host__ __device__ inline bool plan_copy_fused(const LatDev& L, int parity, int x0, int y0, int q,
                                                CopyOp& op) {
    using G = FusedGeo<ES, TX, TY>;
    const int i = q / G::ROWS, rr = q - (q / G::ROWS) * G::ROWS;
    const int y = y0 - 1 - plane_cy(i) + rr;  // lattice row held by box row rr
    if (y < -GY || y > L.ny + GY - 1) return false;
    const int avail = L.pitch - (x0 - G::H + L.gx);  // columns left in the row
    const int cols = avail < G::BW ? avail : G::BW;
    op.src = (L.off_f[parity] + (int64_t)i * L.plane + (int64_t)(y + GY) * L.pitch +
              (x0 - G::H + L.gx)) *
             ES;
    op.dst = i * G::BOXB + rr * G::BW * ES;
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
