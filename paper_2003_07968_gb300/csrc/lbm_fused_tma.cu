// lbm_fused_tma.cu -- host side of the single-pass TMA step: tensor maps and
// dispatch to the instance units (lbm_fused_tma_{f32,f16}_{bgk,mrt}.cu; the
// kernel itself is in lbm_fused_tma.cuh).
#include <cuda.h>

#include <cstring>

#include "lbm_kernels.h"

namespace pplbm {

cudaError_t fused_tma_f32_bgk(int, int, int, const StepArgs&, const CUtensorMap*, const LatDev*,
                              int, cudaStream_t, bool, int*);
cudaError_t fused_tma_f32_mrt(int, int, int, const StepArgs&, const CUtensorMap*, const LatDev*,
                              int, cudaStream_t, bool, int*);
cudaError_t fused_tma_f16_bgk(int, int, int, const StepArgs&, const CUtensorMap*, const LatDev*,
                              int, cudaStream_t, bool, int*);
cudaError_t fused_tma_f16_mrt(int, int, int, const StepArgs&, const CUtensorMap*, const LatDev*,
                              int, cudaStream_t, bool, int*);

namespace {

cudaError_t fused_any(int f16, int mrt, int tx, int ty, int eos, const StepArgs& a,
                      const CUtensorMap* map, const LatDev* lat0, int grid, cudaStream_t st,
                      bool q, int* occ) {
    if (f16)
        return mrt ? fused_tma_f16_mrt(tx, ty, eos, a, map, lat0, grid, st, q, occ)
                   : fused_tma_f16_bgk(tx, ty, eos, a, map, lat0, grid, st, q, occ);
    return mrt ? fused_tma_f32_mrt(tx, ty, eos, a, map, lat0, grid, st, q, occ)
               : fused_tma_f32_bgk(tx, ty, eos, a, map, lat0, grid, st, q, occ);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

}  // namespace

bool fused_tma_shape_supported(int tx, int ty) {
    return (tx == 64 && (ty == 8 || ty == 16)) || (tx == 32 && ty == 16) ||
           (tx == 128 && ty == 8);
}

namespace {

// Load and store maps over a row space: `rows` rows of `pitch` elements in
// each of 18 planes `plane` elements apart, starting at `base`; stores
// clipped to (store_x, store_y).
bool encode_maps(int f16, int tx, int ty, int64_t pitch, int64_t plane, int64_t rows,
                 int64_t store_x, int64_t store_y, void* base, CUtensorMap map[2]) {
    const int es = f16 ? 2 : 4, h = 16 / es, bw = tx + 2 * h;
    // every box must lie inside its tensor: rows at least a box wide and
    // enough rows; the row and plane strides are multiples of 16 bytes
    if (!fused_tma_shape_supported(tx, ty) || pitch < bw || rows < ty + 4 || store_x < tx ||
        store_y < ty)
        return false;
    if ((pitch * es) % 16 || (plane * es) % 16 || pitch * rows > plane) return false;
    if (reinterpret_cast<uintptr_t>(base) % 16) return false;
    EncodeTiled enc = encode_fn();
    if (!enc) return false;
    const CUtensorMapDataType dt = f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)plane * es};
    const cuuint32_t estr[3] = {1, 1, 1};
    // loads: both population buffers as 18 planes of whole rows, ghost frames
    // included: x (row elements), y (rows of the row space), z (plane)
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)rows, 18};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)(ty + 4), 9};
    if (enc(&map[0], dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    // stores: boxes of one tile
    const cuuint64_t sdims[3] = {(cuuint64_t)store_x, (cuuint64_t)store_y, 18};
    const cuuint32_t sbox[3] = {(cuuint32_t)tx, (cuuint32_t)ty, 9};
    return enc(&map[1], dt, 3, base, sdims, strides, sbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool fused_tma_make_map(int f16, int tx, int ty, const LatDev* lats, int n, void* pop,
                        CUtensorMap map[2]) {
    if (n < 1) return false;
    const LatDev& L = lats[0];
    // one lattice, or a batch in one row space (common pitch and planes,
    // off_f[0] = row0 * pitch, buffer B nine planes after A)
    int64_t rows = 0;
    for (int i = 0; i < n; ++i) {
        const LatDev& M = lats[i];
        if (M.row0 != (int32_t)rows || M.pitch != L.pitch || M.plane != L.plane ||
            M.off_f[0] != (int64_t)M.row0 * M.pitch || M.off_f[1] != M.off_f[0] + 9 * M.plane)
            return false;
        rows += M.ny + 2 * GY;
    }
    // stores: one lattice, clipped after its last interior column and row
    // (x < gx + nx, y < GY + ny); a batch, the whole row space (only tiles
    // inside their lattice are stored this way)
    return encode_maps(f16, tx, ty, L.pitch, L.plane, rows, n == 1 ? L.gx + L.nx : L.pitch,
                       n == 1 ? GY + L.ny : rows, pop, map);
}

bool fused_tma_make_space_map(int f16, int tx, int ty, int64_t pitch, int64_t plane,
                              int64_t rows, void* pop, CUtensorMap map[2]) {
    return encode_maps(f16, tx, ty, pitch, plane, rows, pitch, rows, pop, map);
}

cudaError_t launch_fused_tma(int f16, int mrt, int eos, int tx, int ty, const StepArgs& a,
                             const CUtensorMap* map, const LatDev* lat0, int grid,
                             cudaStream_t st) {
    int occ = 0;
    // a batch on the tensor path bulk-copies LatDev rows: 16-byte aligned array
    if (map && !lat0 && (reinterpret_cast<uintptr_t>(a.lats) & 15u)) return cudaErrorInvalidValue;
    return fused_any(f16, mrt, tx, ty, eos, a, map, lat0, grid, st, false, &occ);
}

int occupancy_fused_tma(int f16, int mrt, int eos, int tx, int ty, bool with_map, bool single) {
    int occ = 0;
    StepArgs a{};
    CUtensorMap m[2];
    std::memset(m, 0, sizeof m);
    const CUtensorMap* mp = with_map ? m : nullptr;
    const LatDev lat{};
    cudaError_t e =
        fused_any(f16, mrt, tx, ty, eos, a, mp, single ? &lat : nullptr, 0, nullptr, true, &occ);
    return (e == cudaSuccess && occ > 0) ? occ : 1;
}

}  // namespace pplbm
