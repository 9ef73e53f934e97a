// lbm_tma.cu -- TMA-pipelined versions of the two passes of the step.
//
// Each CTA walks its share of the global tile list.  For every tile one
// elected thread issues nine tiled bulk-tensor copies (cp.async.bulk.tensor,
// one box per population plane, already shifted by -c_i so that the box row
// holding site y carries f*_i(x - c_i)), plus the psi tile with its one-site
// halo for the collision pass.  Copies complete on an mbarrier per stage;
// three stages keep two tiles in flight while the third is computed, so the
// bytes in flight cost no registers.  Outputs leave through plain coalesced
// stores (the periodic images of edge sites go to the ghost frame at the
// same time).  Box x-coordinates are the tile origin x0, a multiple of 32,
// and boxes are (TX + 2H) wide with H = 16 bytes of halo, so every copy
// starts on a 16-byte boundary; rows and columns past the allocation read
// as zero and only feed inactive lanes.
//
// Every mbarrier wait is bounded by a clock budget: on expiry the CTA sets
// bit 1 of the lattice status word, waits (again bounded) for the copies it
// still has in flight, and returns.
#include <cudaTypedefs.h>

#include "lbm_kernels.h"

namespace pplbm {
namespace {

constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr long long kWaitBudgetCycles = 4000000000LL;  // about 2 s at 2 GHz

__host__ __device__ constexpr int align128(int v) { return (v + 127) / 128 * 128; }

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
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

template <class S, int TX, int TY, bool WITH_PSI>
struct Geo {
    using T = typename S::T;
    static constexpr int H = S::kGx;                      // halo columns per side in a box
    static constexpr int BW = TX + 2 * H;                 // population box width
    static constexpr int BOXB = align128(TY * BW * (int)sizeof(T));
    static constexpr int BOXE = BOXB / (int)sizeof(T);   // box stride in elements
    static constexpr int PW = TX + 8;                     // psi box width (4 floats each side)
    static constexpr int PSIB = WITH_PSI ? align128((TY + 2) * PW * 4) : 0;
    static constexpr int STAGEB = 9 * BOXB + PSIB;
    static constexpr int SMEM = kStages * STAGEB + 64;   // + mbarriers
    static constexpr uint32_t TXB = 9u * TY * BW * sizeof(T) + (WITH_PSI ? (TY + 2) * PW * 4 : 0);
    static constexpr int RP = kThreads / TX;              // rows per pass of the block
    static_assert(TY % RP == 0, "tile height must be a multiple of the block's rows");
    static_assert(BW <= 256 && TY + 2 <= 256, "TMA box too large");
};

// Issue the copies of tile `t` into `stage` (called by one thread).
template <class S, int TX, int TY, bool WITH_PSI>
__device__ __forceinline__ void issue_tile(const StepArgs& a, int t, unsigned char* stage,
                                           uint64_t* bar) {
    using G = Geo<S, TX, TY, WITH_PSI>;
    const int4 tl = __ldg(&a.tiles[t]);
    const CUtensorMap* pm = a.pop_maps + tl.x;
    mbar_expect_tx(bar, G::TXB);
    const int x0 = tl.y, y0 = tl.z + GY, p9 = 9 * a.parity;
    // box column 0 is lattice x0 - H (ghost offset gx == H), box row 0 is y0 - c_iy
    tma_load_3d(stage + 0 * G::BOXB, pm, bar, x0, y0, p9 + 0);
    tma_load_3d(stage + 1 * G::BOXB, pm, bar, x0, y0, p9 + 1);
    tma_load_3d(stage + 2 * G::BOXB, pm, bar, x0, y0 - 1, p9 + 2);
    tma_load_3d(stage + 3 * G::BOXB, pm, bar, x0, y0, p9 + 3);
    tma_load_3d(stage + 4 * G::BOXB, pm, bar, x0, y0 + 1, p9 + 4);
    tma_load_3d(stage + 5 * G::BOXB, pm, bar, x0, y0 - 1, p9 + 5);
    tma_load_3d(stage + 6 * G::BOXB, pm, bar, x0, y0 - 1, p9 + 6);
    tma_load_3d(stage + 7 * G::BOXB, pm, bar, x0, y0 + 1, p9 + 7);
    tma_load_3d(stage + 8 * G::BOXB, pm, bar, x0, y0 + 1, p9 + 8);
    if (WITH_PSI) tma_load_2d(stage + 9 * G::BOXB, a.psi_maps + tl.x, bar, x0, y0 - 1);
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
        if (tid == 0) {
            // order the generic-proxy reads of this stage before the async-proxy refill
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int tn = t + kStages * gridDim.x;
            if (tn < a.ntiles) issue_tile<S, TX, TY, WITH_PSI>(a, tn, smem + s * G::STAGEB, &bars[s]);
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

// Tensor maps of one lattice: populations as a 3-D tensor [18 planes][rows][pitch]
// (buffers A and B are adjacent with one plane stride), psi as [rows][pitch_psi].
int encode_tensor_maps(int f16, int tx, int ty, const LatDev& L, void* pop, float* psi,
                       CUtensorMap* pop_map, CUtensorMap* psi_map) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const int es = f16 ? 2 : 4;
    const int H = 16 / es;
    const int rows = L.ny + 2 * GY;
    char* base = reinterpret_cast<char*>(pop) + L.off_f[0] * es;
    cuuint64_t gdim[3] = {(cuuint64_t)L.pitch, (cuuint64_t)rows, 18};
    cuuint64_t gstr[2] = {(cuuint64_t)L.pitch * es, (cuuint64_t)L.plane * es};
    cuuint32_t box[3] = {(cuuint32_t)(tx + 2 * H), (cuuint32_t)ty, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(pop_map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        3, base, gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -2;
    cuuint64_t pdim[2] = {(cuuint64_t)L.pitch_psi, (cuuint64_t)rows};
    cuuint64_t pstr[1] = {(cuuint64_t)L.pitch_psi * 4};
    cuuint32_t pbox[2] = {(cuuint32_t)(tx + 8), (cuuint32_t)(ty + 2)};
    cuuint32_t pes[2] = {1, 1};
    r = encode(psi_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, psi + L.off_psi, pdim, pstr, pbox,
               pes, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

}  // namespace pplbm
