// lbm_tma.cu -- TMA-pipelined versions of the two passes of the step.
//
// Each CTA walks its share of the global tile list.  For every tile the
// first warp issues bulk asynchronous copies (cp.async.bulk, executed by the
// TMA unit) of whole row segments into shared memory: for each population
// plane the TY rows the tile pulls from (already shifted by -c_iy, with 16
// bytes of halo columns on each side; the rest plane also the row above and
// the row below, which hold the rest values of the sources), plus the psi
// rows of the tile and its one-site halo for the collision pass
// (lbm_copy_plan.h).  The warps are
// specialised: one producer warp only issues copies, eight consumer warps
// only compute.  Each stage has a "full" mbarrier (completed by the copies'
// byte count) and an "empty" mbarrier (one arrival per consumer warp once it
// has read the stage), so no CTA-wide barrier sits in the loop and the
// producer runs up to kStages tiles ahead; the bytes in flight cost no
// registers.
// Outputs leave through plain coalesced stores (the periodic images of edge
// sites go to the ghost frame at the same time).
//
// Every mbarrier wait is bounded by a clock budget: on expiry the CTA sets
// bit 1 of the lattice status word, waits (again bounded) for the copies it
// still has in flight, and returns.
#include "lbm_async.cuh"
#include "lbm_copy_plan.h"
#include "lbm_kernels.h"

namespace pplbm {
namespace {

constexpr int kStages = 4;
constexpr int kThreads = 256;              // consumer threads (eight warps)
constexpr int kBlock = kThreads + 32;      // plus one producer warp
struct StageHeader {
    int4 tile;
    LatDev lat;
};

template <class S, int TX, int TY, bool WITH_PSI>
struct Geo : TileGeo<(int)sizeof(typename S::T), TX, TY, WITH_PSI> {
    using B = TileGeo<(int)sizeof(typename S::T), TX, TY, WITH_PSI>;
    static constexpr int SMEM = kStages * B::STAGEB + 2 * kStages * 8 + 16;  // + mbarriers, flag
    static constexpr int RP = kThreads / TX;               // rows per pass of the block
    static_assert(TY % RP == 0, "tile height must be a multiple of the block's rows");
};

// Issue the copies of tile `t` into `stage`; called by all 32 lanes of warp 0.
template <class S, int TX, int TY, bool WITH_PSI>
__device__ __forceinline__ void issue_tile(const StepArgs& a, int t, unsigned char* stage,
                                           uint64_t* bar) {
    using G = Geo<S, TX, TY, WITH_PSI>;
    constexpr int ES = (int)sizeof(typename S::T);
    constexpr int PER = (G::NCOPY + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int4 tl = __ldg(&a.tiles[t]);
    const LatDev& L = a.lats[tl.x];
    // stage header: the tile and its lattice's constants, so consumers read
    // them from shared memory; written before the arrive (release) below
    if (lane == 0) {
        StageHeader* h = reinterpret_cast<StageHeader*>(stage + G::HDR);
        h->tile = tl;
        h->lat = L;
    }
    CopyOp op[PER];
    bool on[PER];
    uint32_t bytes = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = lane + 32 * k;
        on[k] = q < G::NCOPY && plan_copy<ES, TX, TY, WITH_PSI>(L, a.parity, tl.y, tl.z, q, op[k]);
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
    if (lane == 0) mbar_expect_tx(bar, bytes);  // arrive: releases the header writes
    __syncwarp();
    const char* pop = reinterpret_cast<const char*>(a.pop);
    const char* psi = reinterpret_cast<const char*>(a.psi);
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (on[k])
            bulk_g2s(stage + op[k].dst, (op[k].psi ? psi : pop) + op[k].src, (uint32_t)op[k].bytes,
                     bar);
}

// Warp-specialised pipeline: the producer warp (the last one) fills stages,
// the consumer warps call body(tile, stage) for each tile of this CTA.
// Waits are bounded; a consumer that gives up raises the CTA's abort flag,
// the producer then stops issuing and, before it exits, waits (bounded) for
// every copy it has issued, so no copy lands after the CTA is gone.
template <class S, int TX, int TY, bool WITH_PSI, class Body>
__device__ __forceinline__ void run_pipeline(const StepArgs& a, Body&& body) {
    using G = Geo<S, TX, TY, WITH_PSI>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * G::STAGEB);
    uint64_t* empty = full + kStages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kConsumerWarps = kThreads / 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        *abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == kConsumerWarps) {
        // ---------------- producer
        int k = 0;
        for (;; ++k) {
            const int t = blockIdx.x + k * gridDim.x;
            if (t >= a.ntiles || *abort_flag) break;
            const int s = k % kStages;
            if (k >= kStages) {
                const bool ok = mbar_wait_bounded(&empty[s], (uint32_t)(k / kStages - 1) & 1u);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) atomicOr(&a.status[__ldg(&a.tiles[t]).x], 2u);
                    break;
                }
                // order the consumers' generic-proxy reads before the async refill
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            issue_tile<S, TX, TY, WITH_PSI>(a, t, smem + s * G::STAGEB, &full[s]);
        }
        // drain: the last issue into each stage must have landed before exit
        for (int j = (k > kStages ? k - kStages : 0); j < k; ++j)
            mbar_wait_bounded(&full[j % kStages], (uint32_t)(j / kStages) & 1u);
        return;
    }
    // ---------------- consumers
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= a.ntiles) break;
        const int s = k % kStages;
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)(k / kStages) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                *abort_flag = 1;
                atomicOr(&a.status[__ldg(&a.tiles[t]).x], 2u);
            }
            return;
        }
        body(t, smem + s * G::STAGEB);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// The pulled state of site (tx, ty) of the staged tile (make_site).
template <class S, class G>
__device__ __forceinline__ Site<float> stage_site(const typename S::T* P, int tx, int ty) {
    float R[9], Gs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R[i] = S::lds(P + G::rest(i, tx, ty));
        Gs[i] = i ? S::lds(P + G::pull(i, tx, ty)) : 0.f;
    }
    return make_site(R, Gs);
}

}  // namespace

// ---------------------------------------------------------------- pass 1: psi
template <class S, int EOSP, int TX, int TY>
__global__ void __launch_bounds__(kBlock, 2) k_psi_tma(StepArgs a) {
    using G = Geo<S, TX, TY, false>;
    using T = typename S::T;
    const int tx = threadIdx.x % TX, ty0 = threadIdx.x / TX;
    run_pipeline<S, TX, TY, false>(a, [&](int, unsigned char* stage) {
        const StageHeader& hd = *reinterpret_cast<const StageHeader*>(stage + G::HDR);
        const int4 tl = hd.tile;
        const LatDev& L = hd.lat;
        const int nx = L.nx, ny = L.ny;
        const T* P = reinterpret_cast<const T*>(stage);
        const int x = tl.y + tx;
        if (x >= nx) return;
#pragma unroll
        for (int ty = ty0; ty < TY; ty += G::RP) {
            const int y = tl.z + ty;
            if (y >= ny) break;
            const Site<float> st = stage_site<S, G>(P, tx, ty);
            const float psi = Eos<EOSP>::psi(L, site_rho(st, L.rho0), a.status);
            store_img(a.psi + L.off_psi, L.pitch_psi, L.gx_psi, x, y, nx, ny, psi);
        }
    });
}

// --------------------------------------------- pass 2: force + collide + store
template <class S, int TX, int TY>
__global__ void __launch_bounds__(kBlock, 2) k_collide_tma(StepArgs a) {
    using G = Geo<S, TX, TY, true>;
    using T = typename S::T;
    const int tx = threadIdx.x % TX, ty0 = threadIdx.x / TX;
    run_pipeline<S, TX, TY, true>(a, [&](int, unsigned char* stage) {
        const StageHeader& hd = *reinterpret_cast<const StageHeader*>(stage + G::HDR);
        const int4 tl = hd.tile;
        const LatDev& L = hd.lat;
        const int nx = L.nx, ny = L.ny;
        const int x = tl.y + tx;
        if (x >= nx) return;
        const SiteConsts C = site_consts(L);
        const int pitch = L.pitch, gx = L.gx;
        const int64_t plane = L.plane;
        T* o = reinterpret_cast<T*>(a.pop) + L.off_f[a.parity ^ 1];
        const T* P = reinterpret_cast<const T*>(stage);
        const float* PS = reinterpret_cast<const float*>(stage + G::POPB);
#pragma unroll 1
        for (int ty = ty0; ty < TY; ty += G::RP) {
            const int y = tl.z + ty;
            if (y >= ny) break;
            const Site<float> st = stage_site<S, G>(P, tx, ty);
            float p[9], v[9];
            constexpr int W = G::PW;
            const float* c = PS + (ty + 1) * W + tx + 4;
            p[0] = c[0];
            p[1] = c[1];
            p[2] = c[W];
            p[3] = c[-1];
            p[4] = c[-W];
            p[5] = c[W + 1];
            p[6] = c[W - 1];
            p[7] = c[-W - 1];
            p[8] = c[-W + 1];
            collide<S, false>(C, nullptr, st, p, v);
            store_site<S>(o, plane, pitch, gx, x, y, nx, ny, v);
        }
    });
}

// ================================================================ launchers
namespace {

template <class S, int TX, int TY>
cudaError_t psi_shape(int eos, const StepArgs& a, int grid, cudaStream_t st, bool query,
                      int* occ) {
    using G = Geo<S, TX, TY, false>;
    const void* fn = eos == EOS_F64 ? (const void*)k_psi_tma<S, EOS_F64, TX, TY>
                   : eos == EOS_DF  ? (const void*)k_psi_tma<S, EOS_DF, TX, TY>
                                    : (const void*)k_psi_tma<S, EOS_F32, TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, kBlock, G::SMEM);
    const dim3 b(kBlock);
    switch (eos) {
        case EOS_F64: k_psi_tma<S, EOS_F64, TX, TY><<<grid, b, G::SMEM, st>>>(a); break;
        case EOS_DF: k_psi_tma<S, EOS_DF, TX, TY><<<grid, b, G::SMEM, st>>>(a); break;
        default: k_psi_tma<S, EOS_F32, TX, TY><<<grid, b, G::SMEM, st>>>(a); break;
    }
    return cudaGetLastError();
}

template <class S, int TX, int TY>
cudaError_t collide_shape(const StepArgs& a, int grid, cudaStream_t st, bool query, int* occ) {
    using G = Geo<S, TX, TY, true>;
    const void* fn = (const void*)k_collide_tma<S, TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, kBlock, G::SMEM);
    k_collide_tma<S, TX, TY><<<grid, dim3(kBlock), G::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <class S>
cudaError_t psi_any(int tx, int ty, int eos, const StepArgs& a, int grid, cudaStream_t st,
                    bool q, int* occ) {
    if (tx == 64 && ty == 8) return psi_shape<S, 64, 8>(eos, a, grid, st, q, occ);
    if (tx == 64 && ty == 16) return psi_shape<S, 64, 16>(eos, a, grid, st, q, occ);
    if (tx == 128 && ty == 4) return psi_shape<S, 128, 4>(eos, a, grid, st, q, occ);
    if (tx == 128 && ty == 8) return psi_shape<S, 128, 8>(eos, a, grid, st, q, occ);
    if (tx == 32 && ty == 16) return psi_shape<S, 32, 16>(eos, a, grid, st, q, occ);
    return cudaErrorInvalidValue;
}
template <class S>
cudaError_t collide_any(int tx, int ty, const StepArgs& a, int grid, cudaStream_t st, bool q,
                        int* occ) {
    if (tx == 64 && ty == 8) return collide_shape<S, 64, 8>(a, grid, st, q, occ);
    if (tx == 64 && ty == 16) return collide_shape<S, 64, 16>(a, grid, st, q, occ);
    if (tx == 128 && ty == 4) return collide_shape<S, 128, 4>(a, grid, st, q, occ);
    if (tx == 128 && ty == 8) return collide_shape<S, 128, 8>(a, grid, st, q, occ);
    if (tx == 32 && ty == 16) return collide_shape<S, 32, 16>(a, grid, st, q, occ);
    return cudaErrorInvalidValue;
}

}  // namespace

bool tma_shape_supported(int tx, int ty) {
    return (tx == 64 && (ty == 8 || ty == 16)) || (tx == 128 && (ty == 4 || ty == 8)) ||
           (tx == 32 && ty == 16);
}

cudaError_t launch_psi_tma(int f16, int eos, int tx, int ty, const StepArgs& a, int grid,
                           cudaStream_t st) {
    int occ = 0;
    return f16 ? psi_any<StoreF16>(tx, ty, eos, a, grid, st, false, &occ)
               : psi_any<StoreF32>(tx, ty, eos, a, grid, st, false, &occ);
}

cudaError_t launch_collide_tma(int f16, int tx, int ty, const StepArgs& a, int grid,
                               cudaStream_t st) {
    int occ = 0;
    return f16 ? collide_any<StoreF16>(tx, ty, a, grid, st, false, &occ)
               : collide_any<StoreF32>(tx, ty, a, grid, st, false, &occ);
}

int occupancy_psi_tma(int f16, int eos, int tx, int ty) {
    int occ = 0;
    StepArgs a{};
    cudaError_t e = f16 ? psi_any<StoreF16>(tx, ty, eos, a, 0, nullptr, true, &occ)
                        : psi_any<StoreF32>(tx, ty, eos, a, 0, nullptr, true, &occ);
    return (e == cudaSuccess && occ > 0) ? occ : 1;
}

int occupancy_collide_tma(int f16, int tx, int ty) {
    int occ = 0;
    StepArgs a{};
    cudaError_t e = f16 ? collide_any<StoreF16>(tx, ty, a, 0, nullptr, true, &occ)
                        : collide_any<StoreF32>(tx, ty, a, 0, nullptr, true, &occ);
    return (e == cudaSuccess && occ > 0) ? occ : 1;
}

}  // namespace pplbm
