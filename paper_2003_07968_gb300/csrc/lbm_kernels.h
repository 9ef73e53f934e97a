// lbm_kernels.h -- host launchers of the kernels in lbm_kernels.cu.
#pragma once
#include <cuda.h>

#include "lbm_device.cuh"

namespace pplbm {

// Plain-load passes: block (tile_x, tile_y / spt), spt sites per thread.
bool plain_spt_supported(int spt);
cudaError_t launch_psi(int storage_f16, int eos, int spt, const StepArgs& a, dim3 g, dim3 b,
                       cudaStream_t st);
cudaError_t launch_collide(int storage_f16, int mrt, int spt, const StepArgs& a, dim3 g,
                           dim3 b, size_t smem, cudaStream_t st);
// rho32: the field rounded to FP32 (launch_scan writes it), used for the
// neighbours' densities when ux and uy are NULL.
cudaError_t launch_init(int storage_f16, const LatDev& L, void* pop, int parity,
                        const double* rho, const float* rho32, const double* ux, const double* uy,
                        cudaStream_t st);
// rho, u of rows y0 .. y1 - 1 into [ny][nx] fields (any may be NULL).
cudaError_t launch_moments(int storage_f16, const LatDev& L, const void* pop, int parity,
                           const float* psi, double* rho, double* ux, double* uy, int y0, int y1,
                           cudaStream_t st);
// The smallest of n device values into *out, or NaN if any is not finite
// (partials: at least n_partials doubles of scratch); the values rounded to
// FP32 into v32.
cudaError_t launch_scan(const double* v, int64_t n, double* partials, int n_partials, double* out,
                        float* v32, cudaStream_t st);
// v rounded to FP32 into v32 (n values).
cudaError_t launch_to_f32(const double* v, int64_t n, float* v32, cudaStream_t st);
// The step's psi of n device densities with lattice L's constants, the
// float-float radicand (FP64; NaN for other arithmetics), lane check in flags[0]
// (flags: 2 words, zeroed by the caller).
cudaError_t launch_eos_check(int eos, const LatDev& L, const float* rho, int64_t n, float* psi,
                             double* rad, uint32_t* flags, cudaStream_t st);
cudaError_t launch_arith_check(const float* x, int64_t n, float* rcp, float* sq,
                               uint32_t* mismatch, cudaStream_t st);
cudaError_t launch_mass(int storage_f16, const LatDev& L, const void* pop, int parity,
                        double* partials, int n_partials, double* out, cudaStream_t st);
int occupancy_psi(int storage_f16, int eos, int spt, int threads);
// TMA-pipelined passes (lbm_tma.cu); tile shapes are compile-time instances.
bool tma_shape_supported(int tx, int ty);
cudaError_t launch_psi_tma(int f16, int eos, int tx, int ty, const StepArgs& a, int grid,
                           cudaStream_t st);
cudaError_t launch_collide_tma(int f16, int tx, int ty, const StepArgs& a, int grid,
                               cudaStream_t st);
int occupancy_psi_tma(int f16, int eos, int tx, int ty);
int occupancy_collide_tma(int f16, int tx, int ty);
int occupancy_collide(int storage_f16, int mrt, int spt, int threads, size_t smem);
// Single-pass step (psi rebuilt on the tile's halo): same block and shared
// memory shape as the plain collision pass.
cudaError_t launch_fused(int storage_f16, int mrt, int eos, int spt, const StepArgs& a, dim3 g,
                         dim3 b, size_t smem, cudaStream_t st);
int occupancy_fused(int storage_f16, int mrt, int eos, int spt, int threads, size_t smem);
// Single-pass step with TMA-staged tiles (lbm_fused_tma.cu): eight consumer
// warps, a producer warp and, at one or two sites per consumer thread, a
// ring warp (288 or 320 threads), persistent over the tile list.
// With tensor maps (fused_tma_make_map: one lattice, or a batch in one row
// space (row_space_layout), rows at least a box wide; map[0] loads, map[1]
// stores) each tile is one 3-D tensor copy in and, inside its lattice, one
// out; one lattice's constants travel by value (lat0), a batch's come from
// a.lats (lat0 null).  Without maps: bulk row copies in, plain stores out.
bool fused_tma_shape_supported(int tx, int ty);
bool fused_tma_make_map(int f16, int tx, int ty, const LatDev* lats, int n, void* pop,
                        CUtensorMap map[2]);
// Maps over a whole row space of `rows` rows (the server's arena, whose
// lattices come and go): stores unclipped.
bool fused_tma_make_space_map(int f16, int tx, int ty, int64_t pitch, int64_t plane,
                              int64_t rows, void* pop, CUtensorMap map[2]);
cudaError_t launch_fused_tma(int f16, int mrt, int eos, int tx, int ty, const StepArgs& a,
                             const CUtensorMap* map, const LatDev* lat0, int grid,
                             cudaStream_t st);
int occupancy_fused_tma(int f16, int mrt, int eos, int tx, int ty, bool with_map, bool single);

}  // namespace pplbm
