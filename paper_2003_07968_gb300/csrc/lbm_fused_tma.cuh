// lbm_fused_tma.cuh -- the single-pass step with tiles staged by TMA bulk copies.
//
// Kernel and launch templates; the instances are compiled in four units
// (lbm_fused_tma_{f32,f16}_{bgk,mrt}.cu) and dispatched by lbm_fused_tma.cu.
//
// One launch per step, persistent CTAs over the global tile list.  Per CTA,
// one producer warp and eight consumer warps (1, 2 or 4 sites per consumer
// thread, site pairs on the paired FP32 instructions), and for tiles of one
// or two sites per thread a ring warp.
//
// The default path (one lattice, or a batch whose lattices share one row
// space, rows at least a box wide): the producer loads each tile with one
// 3-D tensor copy (cp.async.bulk.tensor over a tensor map of both
// population buffers, passed as a __grid_constant__ parameter: box =
// (TX + 2H) columns x (TY + 4) rows x 9 planes, rows y0 - 2 .. y0 + TY + 1,
// unshifted, parts outside the tensor zero-filled) into a ring of
// shared-memory stages.  The consumers
//   - read from the stage the pulled values of their own sites and the rest
//     values of the sources (make_site, lbm_device.cuh), keep the sites'
//     states in registers and compute rho (Eq. FD) and psi (Eqs. DED,
//     CSEOS);
//   - psi on the tile's one-site ring comes from the ring warp, which
//     computes tile k's ring while the consumers still collide tile k - 1
//     (at four sites per thread the consumers compute it themselves);
//   - consumers and ring warp meet at one named barrier (psi tile complete);
//   - run the force (Eq. IFT) and the collision (Eqs. BGKCO, GFSBGK, or
//     MRTCO), write the nine stored values of a tile inside the lattice back
//     into the stage they have just read, laid out as the store box, and
//     arrive on the stage's mbarrier (edge tiles: plain stores, plus the
//     periodic images of edge sites).
// The producer sends a finished tile out with one 3-D tensor store, waits
// until the store has read the stage and refills it, so loads run up to
// STAGES - 1 tiles ahead of the consumers.  One tensor copy replaces the
// 9 (TY + 2) + 2 row copies of the other form, whose issue cost limits it
// (measured about 32 SM cycles per copy on GB300).
// The other path (batches in a compact layout, lattices narrower than a
// box): bulk row copies per plane and row (lbm_copy_plan.h, FusedGeo), rows
// shifted by -c_iy, the rest plane two rows taller; the stage goes back to
// the producer after the psi phase and the outputs leave by plain stores.
// The stage ring decouples DRAM latency from the arithmetic and the bytes in
// flight cost no registers.  The psi tile is double-buffered, so one barrier
// per tile suffices.
//
// Every mbarrier wait is bounded (lbm_async.cuh).  A consumer warp whose wait
// runs out does not release its stage; the consumers agree on the failure at
// the named barrier (an OR reduction) and all leave together, after raising
// status bit 2 of the tile's lattice; the producer's own waits then run out,
// it drains (bounded) the copies it issued and leaves.  No wait is unbounded
// and no copy lands after its CTA has exited.
#pragma once
#include <cuda.h>

#include <cstring>

#include "lbm_async.cuh"
#include "lbm_copy_plan.h"
#include "lbm_kernels.h"

namespace pplbm {
namespace {

constexpr int kConsumers = 256;             // eight consumer warps
constexpr int kStageBudget = 100 * 1024;    // bytes of stages per CTA (two CTAs per SM)

template <class S, int TX, int TY, bool TMAP>
struct FGeo : FusedGeo<(int)sizeof(typename S::T), TX, TY> {
    using B = FusedGeo<(int)sizeof(typename S::T), TX, TY>;
    static constexpr int ES = (int)sizeof(typename S::T);
    static constexpr int SPT = TX * TY / kConsumers;  // sites per consumer thread
    // tiles of one or two sites per consumer thread get a ring warp, which
    // computes psi on the tile's one-site ring while the consumers collide
    // the tile before; at four sites per thread the consumers keep the ring
    // (the extra warp's registers would make those instances spill)
    static constexpr bool RINGW = SPT <= 2;
    static constexpr int THREADS = kConsumers + (RINGW ? 64 : 32);  // + producer (+ ring warp)
    static constexpr int PSIBAR = kConsumers + (RINGW ? 32 : 0);    // threads at the psi barrier
    static constexpr int RPB = kConsumers / TX;       // tile rows per pass of the block
    static constexpr int PW = TX + 2;                 // psi tile width (with the ring)
    static constexpr int PSIB = align128(PW * (TY + 2) * 4);
    // tensor box: rows y0 - 2 .. y0 + TY + 1 of all nine planes, dense
    static constexpr int TROWS = TY + 4;
    static constexpr int TBYTES = 9 * TROWS * B::BW * ES;
    static constexpr int STAGEB = TMAP ? align128(TBYTES) : B::STAGEB;
    static constexpr int BOXE = TROWS * B::BW;  // plane stride of the tensor box (elements)
    static constexpr int STAGES = kStageBudget / STAGEB >= 4   ? 4
                                  : kStageBudget / STAGEB >= 3 ? 3
                                                               : 2;
    // constants of the tile's lattice, copied in beside each stage (batches
    // on the tensor path)
    static constexpr int LATB = (int)((sizeof(LatDev) + 15) & ~size_t(15));
    static constexpr int LATOFF = STAGES * STAGEB + 2 * PSIB;
    static constexpr int DESCOFF = LATOFF + STAGES * LATB;  // tile descriptor of each stage
    static constexpr int BAR = DESCOFF + STAGES * 16;  // mbarriers after stages, psi, constants
    // element offsets, inside a stage, of the value that cell (lx, ly) of the
    // tile (lx, ly in -1 .. TX, -1 .. TY) pulls from plane i, and of the rest
    // value R(x - c_i) of its source (both layouts hold the rest plane's rows
    // y0 - 2 .. y0 + TY + 1 first)
    static __host__ __device__ constexpr int pull(int i, int lx, int ly) {
        return TMAP ? i * BOXE + (ly + 2 - plane_cy(i)) * B::BW + lx + B::H - plane_cx(i)
                    : B::pull(i, lx, ly);
    }
    static __host__ __device__ constexpr int rest(int i, int lx, int ly) {
        return (ly + 2 - plane_cy(i)) * B::BW + lx + B::H - plane_cx(i);
    }
    static constexpr int SMEM = BAR + 2 * STAGES * 8 + 16;
    static_assert(SPT == 1 || SPT == 2 || SPT == 4, "a tile holds 256, 512 or 1024 sites");
    static_assert(TX % 32 == 0 && kConsumers % TX == 0, "tile width: 32, 64, 128 or 256");
    static_assert(!TMAP || (B::BW <= 256 && TROWS <= 256), "tensor box dimensions");
};

// 3-D tensor copy global -> shared completing on *bar: box at element
// coordinates (x, y, z) of the tensor map (x a multiple of 16 bytes).
__device__ __forceinline__ void tensor_g2s(void* dst, const CUtensorMap* map, int x, int y, int z,
                                           uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// 3-D tensor store shared -> global of a box at (x, y, z) (x a multiple of 16
// bytes, all coordinates >= 0); parts outside the tensor are not written.
__device__ __forceinline__ void tensor_s2g(const CUtensorMap* map, const void* src, int x, int y,
                                           int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ bool tile_skipped(const StepArgs& a, int t) {
    return a.quota && a.step >= __ldg(&a.quota[__ldg(&a.tiles[t]).x]);
}

static_assert(sizeof(LatDev) % 16 == 0, "LatDev rows are bulk-copied (16-byte granules)");

// Copies of one tile into `stage`, issued by the 32 lanes of the producer warp.
template <class S, int TX, int TY>
__device__ __forceinline__ void issue_fused(const StepArgs& a, int4 tl, unsigned char* stage,
                                            uint64_t* bar) {
    using G = FGeo<S, TX, TY, false>;
    constexpr int ES = (int)sizeof(typename S::T);
    constexpr int PER = (G::NCOPY + 31) / 32;
    const int lane = threadIdx.x & 31;
    const LatDev& L = a.lats[tl.x];
    CopyOp op[PER];
    bool on[PER];
    uint32_t bytes = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = lane + 32 * k;
        on[k] = q < G::NCOPY && plan_copy_fused<ES, TX, TY>(L, a.parity, tl.y, tl.z, q, op[k]);
        // the plan is proven on the host (lbm_selfcheck); a copy that still broke
        // the bulk-copy rules would be skipped and flagged, never issued
        if (on[k] && ((op[k].src | op[k].dst | op[k].bytes) & 15)) {
            atomicOr(&a.status[tl.x], 4u);
            on[k] = false;
        }
        if (on[k]) bytes += (uint32_t)op[k].bytes;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    const char* pop = reinterpret_cast<const char*>(a.pop);
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (on[k]) bulk_g2s(stage + op[k].dst, pop + op[k].src, (uint32_t)op[k].bytes, bar);
}

// psi on the one-site ring of tile (x0, y0) of lattice L, from the tile's
// stage st into the psi tile ps: ring cells r and r + nhalf in the two lanes
// of a float2, for r = first, first + stride, ... below nhalf.
template <class S, int EOSP, int TX, int TY, bool TMAP>
__device__ __forceinline__ void ring_psi(const StepArgs& a, const LatDev& L,
                                         const typename S::T* st, float* ps, int x0, int y0,
                                         int first, int stride) {
    using G = FGeo<S, TX, TY, TMAP>;
    using T = typename S::T;
    constexpr int nhalf = TX + TY + 2;  // half of the 2 (TX + TY) + 4 ring cells
    const int xend = min(x0 + TX, L.nx), yend = min(y0 + TY, L.ny);
    for (int r = first; r < nhalf; r += stride) {
        int gx[2], gy[2];
        unsigned live = 0;
        float2 R[9], Gs[9];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            live |= (unsigned)ring_cell(r + l * nhalf, TX, TY, x0, y0, xend, yend, gx[l], gy[l])
                    << l;
            const T* b = st + G::pull(0, gx[l] - x0, gy[l] - y0);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                Lanes<float2>::put(R[i], l, S::lds(b + (G::rest(i, 0, 0) - G::pull(0, 0, 0))));
                Lanes<float2>::put(Gs[i], l,
                                   i ? S::lds(b + (G::pull(i, 0, 0) - G::pull(0, 0, 0))) : 0.f);
            }
        }
        const float2 psi = Eos<EOSP>::psi(L, site_rho(make_site(R, Gs), L.rho0), a.status, live);
        if (live & 1u) ps[(gy[0] - y0 + 1) * G::PW + (gx[0] - x0 + 1)] = psi.x;
        if (live & 2u) ps[(gy[1] - y0 + 1) * G::PW + (gx[1] - x0 + 1)] = psi.y;
    }
}

// MODE 0: row copies, lattice constants from a.lats; 1: tensor copies, one
// lattice whose constants are the parameter lat0; 2: tensor copies, a batch
// in one row space, constants from a.lats.
template <class S, int EOSP, int TX, int TY, bool MRT, int MODE>
__global__ void __launch_bounds__((FGeo<S, TX, TY, MODE != 0>::THREADS), 2)
    k_fused_tma(StepArgs a, const __grid_constant__ CUtensorMap tmap,
                const __grid_constant__ CUtensorMap smap, const __grid_constant__ LatDev lat0) {
    constexpr bool TMAP = MODE != 0;
    using G = FGeo<S, TX, TY, TMAP>;
    using T = typename S::T;
    using V = typename LaneOf<G::SPT>::V;
    using Ln = Lanes<V>;
    constexpr int NV = G::SPT / Ln::n;
    constexpr int PW = G::PW;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::BAR);
    uint64_t* empty = full + G::STAGES;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + G::STAGES);
    float* psi_buf = reinterpret_cast<float*>(smem + G::STAGES * G::STAGEB);
    // the tile each stage holds, written by the producer before its arrival
    // on the stage's barrier, so a consumer reads it from shared memory
    int4* desc = reinterpret_cast<int4*>(smem + G::DESCOFF);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < G::STAGES; ++s) {
            mbar_init(&full[s], 1);
            // row copies: each consumer warp releases a stage after reading it;
            // tensor path: every consumer arrives once the tile's f* is in the
            // stage (the producer stores it, then refills the stage)
            mbar_init(&empty[s], TMAP ? kConsumers : kConsumers / 32 + (G::RINGW ? 1 : 0));
        }
        *abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == kConsumers / 32) {
        // ------------------------------------------------------------ producer
        // Tensor path: a stage comes back when its tile is done; the producer
        // then sends the tile's f* out with one tensor store (tiles inside the
        // lattice; edge tiles were stored by the consumers), waits until the
        // store has read the stage and refills it at once, so loads run up to
        // STAGES - 1 tiles ahead of the consumers.
        int k = 0;
        int tq[G::STAGES] = {};  // tile held by each stage (tensor path)
        int2 sq[G::STAGES] = {};  // its store box origin (x, row), row -1: stored by the consumers
        bool alive = true;
        const int sz = 9 * (a.parity ^ 1);
        // store of the finished tile in stage s (lane 0), at the coordinates
        // computed when the tile was loaded
        auto store_tile = [&](int s) {
            if (sq[s].y >= 0) {
                tensor_s2g(&smap, smem + s * G::STAGEB, sq[s].x, sq[s].y, sz);
                bulk_commit();
                bulk_wait_read<0>();
            }
        };
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            if (tile_skipped(a, t)) continue;
            if (*abort_flag) {
                alive = false;
                break;
            }
            const int s = k % G::STAGES;
            // failure-detection test: no copy and no arrival for this tile
            const bool starved = a.starve == t + 1;
            // the tile and its box coordinates (lane 0), read before the wait
            // for the stage so that the loads overlap it (2 % faster on an
            // 8192^2 lattice; 5 % on 512 uneven lattices, where reading them
            // after the wait had measured faster on earlier forms of the kernel)
            int4 tl = make_int4(0, 0, 0, 0);
            TmaCoords c{};
            auto locate = [&] {
                tl = __ldg(&a.tiles[t]);
                const LatDev& Lt = MODE == 1 ? lat0 : a.lats[tl.x];
                c = fused_tma_coords<TX, TY>(Lt, Lt.row0, a.parity, tl.y, tl.z);
            };
            if (TMAP && lane == 0) locate();
            if (k >= G::STAGES) {
                const bool ok =
                    mbar_wait_bounded(&empty[s], (uint32_t)(k / G::STAGES - 1) & 1u, a.wait_cycles);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) atomicOr(&a.status[__ldg(&a.tiles[t]).x], 2u);
                    alive = false;
                    break;
                }
                if (TMAP) {
                    if (lane == 0) store_tile(s);
                    __syncwarp();
                }
                // the consumers' generic-proxy reads of the stage come before the refill
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            if (TMAP) {
                // one tensor copy: columns from x0 - H (element x0 of the row, a
                // multiple of 32), rows from y0 - 2 (row row0 + y0 of the row
                // space), planes of the current buffer
                if (lane == 0 && !starved) {
                    desc[s] = tl;
                    mbar_expect_tx(&full[s], (uint32_t)G::TBYTES +
                                                 (MODE == 2 ? (uint32_t)sizeof(LatDev) : 0u));
                    tensor_g2s(smem + s * G::STAGEB, &tmap, c.lx, c.ly, c.lz, &full[s]);
                    if (MODE == 2)
                        bulk_g2s(smem + G::LATOFF + s * G::LATB, a.lats + tl.x,
                                 (uint32_t)sizeof(LatDev), &full[s]);
                }
                tq[s] = t;
                sq[s] = make_int2(c.sx, c.store ? c.sy : -1);
                __syncwarp();
            } else {
                const int4 tl = __ldg(&a.tiles[t]);
                if (lane == 0) desc[s] = tl;
                __syncwarp();
                if (!starved) issue_fused<S, TX, TY>(a, tl, smem + s * G::STAGEB, &full[s]);
            }
            ++k;
        }
        // tensor path: store the tiles still held by the stages
        if (TMAP && alive) {
            for (int j = (k > G::STAGES ? k - G::STAGES : 0); j < k; ++j) {
                const int s = j % G::STAGES;
                const bool ok =
                    mbar_wait_bounded(&empty[s], (uint32_t)(j / G::STAGES) & 1u, a.wait_cycles);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) atomicOr(&a.status[__ldg(&a.tiles[tq[s]]).x], 2u);
                    break;
                }
                if (lane == 0) store_tile(s);
                __syncwarp();
            }
        }
        // drain: the last issue into each stage must have landed, and every
        // tile store must be complete, before exit
        for (int j = (k > G::STAGES ? k - G::STAGES : 0); j < k; ++j)
            mbar_wait_bounded(&full[j % G::STAGES], (uint32_t)(j / G::STAGES) & 1u,
                              a.wait_cycles);
        if (TMAP && lane == 0) bulk_wait_all();
        return;
    }

    if (G::RINGW && warp == kConsumers / 32 + 1) {
        // ------------------------------------------------------------ ring warp
        // psi on the tile's one-site ring.  Tile k's ring is computed while
        // the consumers still run the collision of tile k - 1 (the psi tile
        // is double buffered): only the consumers' own psi stands before the
        // barrier.
        int k = 0;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            if (tile_skipped(a, t)) continue;
            const int s = k % G::STAGES;
            float* ps = psi_buf + (k & 1) * (G::PSIB / 4);
            const bool ok = __all_sync(
                0xffffffffu,
                mbar_wait_bounded(&full[s], (uint32_t)(k / G::STAGES) & 1u, a.wait_cycles));
            if (ok) {
                const int4 tl = desc[s];
                const LatDev& L =
                    MODE == 1   ? lat0
                    : MODE == 2 ? *reinterpret_cast<const LatDev*>(smem + G::LATOFF + s * G::LATB)
                                : a.lats[tl.x];
                ring_psi<S, EOSP, TX, TY, TMAP>(
                    a, L, reinterpret_cast<const T*>(smem + s * G::STAGEB), ps, tl.y, tl.z, lane, 32);
                // row copies: this warp's reads of the stage are done
                if (!TMAP) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);
                }
            }
            uint32_t failed;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.eq.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                : "=r"(failed)
                : "r"((uint32_t)ok), "n"(G::PSIBAR)
                : "memory");
            if (failed) return;
            ++k;
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int tid = threadIdx.x;  // 0 .. kConsumers-1
    // a thread's SPT sites are consecutive rows of one column, ly0 .. ly0 +
    // SPT - 1, so that their 3 x 3 windows of rest values and of psi overlap:
    // (SPT + 2) x 3 loads each instead of 9 SPT
    const int tx = tid % TX, ly0 = (tid / TX) * G::SPT;
    int k = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        if (tile_skipped(a, t)) continue;
        const int s = k % G::STAGES;
        float* ps = psi_buf + (k & 1) * (G::PSIB / 4);
        const bool ok = __all_sync(
            0xffffffffu, mbar_wait_bounded(&full[s], (uint32_t)(k / G::STAGES) & 1u, a.wait_cycles));
        // the tile, from the stage's descriptor (from global memory only if
        // the wait ran out, to name the lattice in the status word)
        const int4 tl = ok ? desc[s] : __ldg(&a.tiles[t]);
        // one lattice: its constants are kernel parameters (constant-bank
        // operands); a batch on the tensor path: they arrived with the tile
        // and stay until the stage goes back; row copies: global (the stage
        // goes back before the collision)
        const LatDev& L =
            MODE == 1   ? lat0
            : MODE == 2 ? *reinterpret_cast<const LatDev*>(smem + G::LATOFF + s * G::LATB)
                        : a.lats[tl.x];
        const int nx = L.nx, ny = L.ny, x0 = tl.y, y0 = tl.z;
        const int xend = min(x0 + TX, nx), yend = min(y0 + TY, ny);
        const int x = x0 + tx;
        Site<V> sv[NV];
        if (ok) {
            const T* st = reinterpret_cast<const T*>(smem + s * G::STAGEB);
            // own sites: pulled states into registers, rho, psi
            // rest values of the (SPT + 2) x 3 window: rows ly0 - 1 .. ly0 + SPT,
            // columns tx - 1 .. tx + 1 (the rest plane's value at (lx, ly) is
            // G::rest(0, lx, ly))
            float Rw[G::SPT + 2][3];
#pragma unroll
            for (int r = 0; r < G::SPT + 2; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    Rw[r][c] = S::lds(st + G::rest(0, tx + c - 1, ly0 + r - 1));
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                V R[9], Gs[9];
#pragma unroll
                for (int l = 0; l < Ln::n; ++l) {
                    const int kk = j * Ln::n + l;  // row ly0 + kk
                    // the other planes at constant offsets from the site's own value
                    const T* b = st + G::pull(0, tx, ly0 + kk);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        // R(x - c_i): row kk - c_iy, column -c_ix of the window
                        Ln::put(R[i], l, Rw[kk + 1 - plane_cy(i)][1 - plane_cx(i)]);
                        Ln::put(Gs[i], l,
                                i ? S::lds(b + (G::pull(i, 0, 0) - G::pull(0, 0, 0))) : 0.f);
                    }
                }
                sv[j] = make_site(R, Gs);
            }
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                unsigned live = 0;
#pragma unroll
                for (int l = 0; l < Ln::n; ++l)
                    live |= (unsigned)(x < nx && y0 + ly0 + j * Ln::n + l < ny) << l;
                const V psi = Eos<EOSP>::psi(L, site_rho(sv[j], L.rho0), a.status, live);
#pragma unroll
                for (int l = 0; l < Ln::n; ++l)
                    if ((live >> l) & 1u)
                        ps[(ly0 + j * Ln::n + l + 1) * PW + tx + 1] = Ln::get(psi, l);
            }
            if (!G::RINGW)
                ring_psi<S, EOSP, TX, TY, TMAP>(a, L, st, ps, x0, y0, tid, kConsumers);
            // row copies: every read of the stage is done, hand it back
            if (!TMAP) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
        }
        // psi tile complete (own sites here, the ring from the ring warp); a
        // warp whose wait ran out makes every consumer and the ring warp leave
        uint32_t failed;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.eq.u32 p, %1, 0;\n\t"
            "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(failed)
            : "r"((uint32_t)ok), "n"(G::PSIBAR)
            : "memory");
        if (failed) {
            if (tid == 0) {
                *abort_flag = 1;
                atomicOr(&a.status[tl.x], 2u);
            }
            return;
        }
        ++k;
        if (!TMAP && x >= nx) continue;
        // force, collision, stores
        const SiteConsts C = site_consts(L);
        T* o = reinterpret_cast<T*>(a.pop) + L.off_f[a.parity ^ 1];
        const bool tile_in = x0 >= GW && y0 >= GW && x0 + TX <= nx - GW && y0 + TY <= ny - GW;
        // tensor path, tiles inside the lattice: f* of the tile goes to the
        // stage just consumed, laid out as the store box [plane][TY][TX], and
        // leaves in one tensor store issued by the producer.  A ragged edge
        // tile uses plain stores:
        // the store unit clips a box at 16-byte granularity in x (measured), so
        // a partial box would also write the ghost columns just past nx.
        const bool bulk_out = TMAP && fused_tma_coords<TX, TY>(L, 0, 0, x0, y0).store;
        T* out = reinterpret_cast<T*>(smem + s * G::STAGEB);
        // psi of the (SPT + 2) x 3 window around the thread's column: rows
        // ly0 - 1 .. ly0 + SPT, columns tx - 1 .. tx + 1
        float Pw[G::SPT + 2][3];
#pragma unroll
        for (int r = 0; r < G::SPT + 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Pw[r][c] = ps[(ly0 + r) * PW + tx + c];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            V p[9], v[9];
#pragma unroll
            for (int l = 0; l < Ln::n; ++l) {
                const int kk = j * Ln::n + l;
#pragma unroll
                for (int i = 0; i < 9; ++i)  // psi(x + c_i)
                    Ln::put(p[i], l, Pw[kk + 1 + plane_cy(i)][1 + plane_cx(i)]);
            }
            collide<S, MRT>(C, L.mrt_s, sv[j], p, v);
#pragma unroll
            for (int l = 0; l < Ln::n; ++l) {
                const int ly = ly0 + j * Ln::n + l;
                const int y = y0 + ly;
                if (bulk_out) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) out[(i * TY + ly) * TX + tx] = S::cv(Ln::get(v[i], l));
                    // sites within GW of an edge: their periodic images too
                    if (!tile_in && ((x < GW) | (x >= nx - GW) | (y < GW) | (y >= ny - GW)))
#pragma unroll
                        for (int i = 0; i < 9; ++i)
                            store_images(o + i * L.plane, MODE == 2 ? i : 0, L.pitch, L.gx, x,
                                         y, nx, ny, S::cv(Ln::get(v[i], l)));
                } else {
                    if (x >= nx || y >= ny) continue;
                    float vs[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) vs[i] = Ln::get(v[i], l);
                    if (MODE == 2)
                        store_site_read<S>(o, L.plane, L.pitch, L.gx, x, y, nx, ny, vs, tile_in);
                    else
                        store_site<S>(o, L.plane, L.pitch, L.gx, x, y, nx, ny, vs, tile_in);
                }
            }
        }
        if (TMAP) {
            // the tile's f* is in the stage (or, for an edge tile, stored):
            // hand the stage to the producer, which stores and refills it
            if (bulk_out) fence_proxy_async_smem();
            mbar_arrive(&empty[s]);
        }
    }
}

// ---------------------------------------------------------------- launchers
template <class S, int EOSP, int TX, int TY, bool MRT, int MODE>
cudaError_t fused_inst(const StepArgs& a, const CUtensorMap* map, const LatDev* lat0, int grid,
                       cudaStream_t st, bool query, int* occ) {
    // map[0]: load map, map[1]: store map (tensor path)
    using G = FGeo<S, TX, TY, MODE != 0>;
    const void* fn = (const void*)k_fused_tma<S, EOSP, TX, TY, MRT, MODE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, G::THREADS, G::SMEM);
    CUtensorMap none;
    std::memset(&none, 0, sizeof none);
    const LatDev nolat{};
    k_fused_tma<S, EOSP, TX, TY, MRT, MODE><<<grid, dim3(G::THREADS), G::SMEM, st>>>(
        a, map ? map[0] : none, map ? map[1] : none, lat0 ? *lat0 : nolat);
    return cudaGetLastError();
}

template <class S, bool MRT, int TX, int TY, int MODE>
cudaError_t fused_eos(int eos, const StepArgs& a, const CUtensorMap* map, const LatDev* lat0,
                      int grid, cudaStream_t st, bool q, int* occ) {
    switch (eos) {
        case EOS_F64: return fused_inst<S, EOS_F64, TX, TY, MRT, MODE>(a, map, lat0, grid, st, q, occ);
        case EOS_DF: return fused_inst<S, EOS_DF, TX, TY, MRT, MODE>(a, map, lat0, grid, st, q, occ);
        default: return fused_inst<S, EOS_F32, TX, TY, MRT, MODE>(a, map, lat0, grid, st, q, occ);
    }
}

template <class S, bool MRT, int TX, int TY>
cudaError_t fused_map(int eos, const StepArgs& a, const CUtensorMap* map, const LatDev* lat0,
                      int grid, cudaStream_t st, bool q, int* occ) {
    // tensor maps with lat0: one lattice; tensor maps alone: a batch in one row space
    return !map ? fused_eos<S, MRT, TX, TY, 0>(eos, a, nullptr, nullptr, grid, st, q, occ)
           : lat0 ? fused_eos<S, MRT, TX, TY, 1>(eos, a, map, lat0, grid, st, q, occ)
                  : fused_eos<S, MRT, TX, TY, 2>(eos, a, map, nullptr, grid, st, q, occ);
}

}  // namespace

// One storage type and collision: every tile shape, EOS arithmetic and
// staging form (the body of the four instance units).
template <class S, bool MRT>
cudaError_t fused_tma_any(int tx, int ty, int eos, const StepArgs& a, const CUtensorMap* map,
                          const LatDev* lat0, int grid, cudaStream_t st, bool q, int* occ) {
    if (tx == 64 && ty == 8) return fused_map<S, MRT, 64, 8>(eos, a, map, lat0, grid, st, q, occ);
    if (tx == 32 && ty == 16) return fused_map<S, MRT, 32, 16>(eos, a, map, lat0, grid, st, q, occ);
    if (tx == 64 && ty == 16) return fused_map<S, MRT, 64, 16>(eos, a, map, lat0, grid, st, q, occ);
    if (tx == 128 && ty == 8) return fused_map<S, MRT, 128, 8>(eos, a, map, lat0, grid, st, q, occ);
    return cudaErrorInvalidValue;
}

}  // namespace pplbm
