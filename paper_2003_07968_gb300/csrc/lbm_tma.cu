// lbm_tma.cu -- TMA-pipelined versions of the two passes of the step.
//
// Each CTA walks its share of the global tile list.  For every tile the
// first warp issues bulk asynchronous copies (cp.async.bulk, executed by the
// TMA unit) of whole row segments into shared memory: for each population
// plane the TY rows the tile pulls from (already shifted by -c_iy, with 16
// bytes of halo columns on each side), plus the psi rows of the tile and its
// one-site halo for the collision pass (lbm_copy_plan.h).  The copies
// complete on an mbarrier per stage; three stages keep two tiles in flight
// while the third is computed, so the bytes in flight cost no registers.
// Outputs leave through plain coalesced stores (the periodic images of edge
// sites go to the ghost frame at the same time).
//
// Every mbarrier wait is bounded by a clock budget: on expiry the CTA sets
// bit 1 of the lattice status word, waits (again bounded) for the copies it
// still has in flight, and returns.
#include "lbm_copy_plan.h"
#include "lbm_kernels.h"

namespace pplbm {
namespace {

constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr long long kWaitBudgetCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of *bar; false if the clock budget ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (long long it = 0; it < (1LL << 40); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > kWaitBudgetCycles) return false;
    }
    return false;
}
// Bulk copy global -> shared completing on *bar (both addresses 16-byte
// aligned, size a multiple of 16: guaranteed by the copy plan).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <class S, int TX, int TY, bool WITH_PSI>
struct Geo : TileGeo<(int)sizeof(typename S::T), TX, TY, WITH_PSI> {
    using B = TileGeo<(int)sizeof(typename S::T), TX, TY, WITH_PSI>;
    static constexpr int SMEM = kStages * B::STAGEB + 64;  // + mbarriers
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
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    const char* pop = reinterpret_cast<const char*>(a.pop);
    const char* psi = reinterpret_cast<const char*>(a.psi);
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (on[k])
            bulk_g2s(stage + op[k].dst, (op[k].psi ? psi : pop) + op[k].src, (uint32_t)op[k].bytes,
                     bar);
}

// Shared pipeline driver: calls body(tile, stage) for each tile of this CTA.
template <class S, int TX, int TY, bool WITH_PSI, class Body>
__device__ __forceinline__ void run_pipeline(const StepArgs& a, Body&& body) {
    using G = Geo<S, TX, TY, WITH_PSI>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * G::STAGEB);
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncwarp();
    if (tid < 32) {
        for (int s = 0; s < kStages; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < a.ntiles) issue_tile<S, TX, TY, WITH_PSI>(a, t, smem + s * G::STAGEB, &bars[s]);
        }
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= a.ntiles) break;
        const int s = k % kStages;
        const uint32_t par = (uint32_t)(k / kStages) & 1u;
        const bool ok = mbar_wait_bounded(&bars[s], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                // drain the copies still in flight (this tile's and later ones), then flag
                for (int j = 0; j < kStages; ++j) {
                    const int tj = blockIdx.x + (k + j) * gridDim.x;
                    if (tj < a.ntiles)
                        mbar_wait_bounded(&bars[(k + j) % kStages], (uint32_t)((k + j) / kStages) & 1u);
                }
                atomicOr(&a.status[__ldg(&a.tiles[t]).x], 2u);
            }
            return;
        }
        body(t, smem + s * G::STAGEB);
        __syncthreads();  // every thread is done reading this stage
        if (tid < 32) {
            const int tn = t + kStages * gridDim.x;
            if (tn < a.ntiles) {
                // order the generic-proxy reads of this stage before the async-proxy refill
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_tile<S, TX, TY, WITH_PSI>(a, tn, smem + s * G::STAGEB, &bars[s]);
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- pass 1: psi
template <class S, int EOSP, int TX, int TY>
__global__ void __launch_bounds__(kThreads, 2) k_psi_tma(StepArgs a) {
    using G = Geo<S, TX, TY, false>;
    using T = typename S::T;
    run_pipeline<S, TX, TY, false>(a, [&](int t, unsigned char* stage) {
        const int4 tl = __ldg(&a.tiles[t]);
        const LatDev& L = a.lats[tl.x];
        const int nx = L.nx, ny = L.ny;
        const T* P = reinterpret_cast<const T*>(stage);
        const int x = tl.y + threadIdx.x;
        if (x >= nx) return;
#pragma unroll
        for (int ty = threadIdx.y; ty < TY; ty += G::RP) {
            const int y = tl.z + ty;
            if (y >= ny) break;
            const T* b = P + ty * G::BW + threadIdx.x + G::H;
            float d = S::lds(b);
            d += S::lds(b + 1 * G::BOXE - 1);
            d += S::lds(b + 2 * G::BOXE);
            d += S::lds(b + 3 * G::BOXE + 1);
            d += S::lds(b + 4 * G::BOXE);
            d += S::lds(b + 5 * G::BOXE - 1);
            d += S::lds(b + 6 * G::BOXE + 1);
            d += S::lds(b + 7 * G::BOXE + 1);
            d += S::lds(b + 8 * G::BOXE - 1);
            const float rho = d + L.rho0;
            bool ok;
            float psi = eval_psi<EOSP>(L, rho, ok);
            if (!ok) {
                atomicOr(&a.status[L.lattice], 1u);
                psi = __int_as_float(0x7fc00000);
            }
            store_img(a.psi + L.off_psi, L.pitch_psi, L.gx_psi, x, y, nx, ny, psi);
        }
    });
}

// --------------------------------------------- pass 2: force + collide + store
template <class S, int TX, int TY>
__global__ void __launch_bounds__(kThreads, 2) k_collide_tma(StepArgs a) {
    using G = Geo<S, TX, TY, true>;
    using T = typename S::T;
    run_pipeline<S, TX, TY, true>(a, [&](int t, unsigned char* stage) {
        const int4 tl = __ldg(&a.tiles[t]);
        const LatDev& L = a.lats[tl.x];
        const int nx = L.nx, ny = L.ny;
        const T* P = reinterpret_cast<const T*>(stage);
        const float* PS = reinterpret_cast<const float*>(stage + 9 * G::BOXB);
        const int x = tl.y + threadIdx.x;
        if (x >= nx) return;
        const int pitch = L.pitch, gx = L.gx;
        const int64_t plane = L.plane;
        T* o = reinterpret_cast<T*>(a.pop) + L.off_f[a.parity ^ 1];
        const float om = L.omega, gu = L.guo, rho0 = L.rho0;
#pragma unroll 1
        for (int ty = threadIdx.y; ty < TY; ty += G::RP) {
            const int y = tl.z + ty;
            if (y >= ny) break;
            const T* b = P + ty * G::BW + threadIdx.x + G::H;
            const float g0 = S::lds(b);
            const float g1 = S::lds(b + 1 * G::BOXE - 1);
            const float g2 = S::lds(b + 2 * G::BOXE);
            const float g3 = S::lds(b + 3 * G::BOXE + 1);
            const float g4 = S::lds(b + 4 * G::BOXE);
            const float g5 = S::lds(b + 5 * G::BOXE - 1);
            const float g6 = S::lds(b + 6 * G::BOXE + 1);
            const float g7 = S::lds(b + 7 * G::BOXE + 1);
            const float g8 = S::lds(b + 8 * G::BOXE - 1);
            const float drho = ((g0 + g1) + (g2 + g3)) + ((g4 + g5) + (g6 + g7)) + g8;
            const float rho = drho + rho0;
            const float jx = (g1 - g3) + (g5 - g6) + (g8 - g7);
            const float jy = (g2 - g4) + (g5 + g6) - (g7 + g8);
            const float* c = PS + (ty + 1) * G::PW + threadIdx.x + 4;
            constexpr int W = G::PW;
            const Force F = site_force(L, c[0], c[1], c[W], c[-1], c[-W], c[W + 1], c[W - 1],
                                       c[-W - 1], c[-W + 1]);
            const float inv = 1.f / rho;
            const float ux = (jx + 0.5f * F.x) * inv;  // Eq. (FMD)
            const float uy = (jy + 0.5f * F.y) * inv;
            const float usq = ux * ux + uy * uy;
            const float Fu = F.x * ux + F.y * uy;
            // Directions 1..8 by Eqs. (BGKCO), (SEDF), (GFS); the rest population
            // from mass conservation (see k_collide).
#define PPLBM_OUT(I, GV)                                                                  \
    const float o##I = bgk_guo<I>(GV, drho, rho, ux, uy, usq, F.x, F.y, Fu, om, gu);      \
    store_img(o + I * plane, pitch, gx, x, y, nx, ny, S::cv(o##I))
            PPLBM_OUT(1, g1);
            PPLBM_OUT(2, g2);
            PPLBM_OUT(3, g3);
            PPLBM_OUT(4, g4);
            PPLBM_OUT(5, g5);
            PPLBM_OUT(6, g6);
            PPLBM_OUT(7, g7);
            PPLBM_OUT(8, g8);
#undef PPLBM_OUT
            const float o0 = drho - (((o1 + o2) + (o3 + o4)) + ((o5 + o6) + (o7 + o8)));
            store_img(o, pitch, gx, x, y, nx, ny, S::cv(o0));
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
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, kThreads, G::SMEM);
    const dim3 b(TX, kThreads / TX);
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
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, kThreads, G::SMEM);
    k_collide_tma<S, TX, TY><<<grid, dim3(TX, kThreads / TX), G::SMEM, st>>>(a);
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
