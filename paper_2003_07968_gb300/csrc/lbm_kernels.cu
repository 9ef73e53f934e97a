// lbm_kernels.cu -- CUDA kernels of the D2Q9 pseudopotential step
// (arXiv 2003.07968) for sm_103a, and their host launchers.
//
//   k_psi      pass 1: pull f, rho (Eq. FD), psi (Eqs. DED, CSEOS) -> psi plane
//   k_collide  pass 2: psi tile + halo in shared memory, force (Eq. IFT),
//              velocity (Eq. FMD), BGK + Guo (Eqs. BGKCO, SEDF, GFS), store f*
//   k_init     f* such that the next pull yields f^eq(rho, u)
//   k_moments  rho, force-shifted u of the current state (FP64 out)
//   k_mass_*   FP64 sum of the stored populations (two-level reduction; site
//              sums as float-float pairs on the FP32 pipe)
//
// Both passes walk a global tile list with a persistent grid, so one launch
// covers one lattice or a batch of uneven lattices alike.
#include <climits>

#include "lbm_copy_plan.h"
#include "lbm_kernels.h"

namespace pplbm {

// Each plain pass gives a thread SPT sites of one column (rows
// threadIdx.y + k blockDim.y): all SPT x 9 loads are issued before any of
// them is used, which keeps more bytes in flight per thread.  With SPT even,
// sites k and k+1 share the lanes of one float2 and go through the EOS and
// the collision together on the paired FP32 instructions.

// The pulled state of site (x, y) (make_site): `f` points at (x, y) of
// plane 0 of the buffer; plane i of the source site x - c_i and its rest
// value R(x - c_i) are read.
template <class S>
__device__ __forceinline__ Site<float> pulled_site(const typename S::T* f, int64_t plane,
                                                   int pitch) {
    float R[9], Gs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int64_t src = -(int64_t)plane_cy(i) * pitch - plane_cx(i);
        R[i] = S::ld(f + src);
        Gs[i] = i ? S::ld(f + i * plane + src) : 0.f;
    }
    return make_site(R, Gs);
}

// The pulled states of SPT sites of one column (rows y0 + k by, clamped to
// the last row), in the lanes of V.
template <class S, int SPT, class V>
__device__ __forceinline__ void load_sites(const typename S::T* base, int64_t plane, int pitch,
                                           int y0, int by, int ny, Site<V>* sv) {
    using Ln = Lanes<V>;
#pragma unroll
    for (int j = 0; j < SPT / Ln::n; ++j) {
        V R[9], Gs[9];
#pragma unroll
        for (int l = 0; l < Ln::n; ++l) {
            const int y = min(y0 + (j * Ln::n + l) * by, ny - 1);
            const typename S::T* f = base + (int64_t)(y + GY) * pitch;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int64_t src = -(int64_t)plane_cy(i) * pitch - plane_cx(i);
                Ln::put(R[i], l, S::ld(f + src));
                Ln::put(Gs[i], l, i ? S::ld(f + i * plane + src) : 0.f);
            }
        }
        sv[j] = make_site(R, Gs);
    }
}

// ---------------------------------------------------------------- pass 1: psi
template <class S, int EOSP, int SPT>
__global__ void __launch_bounds__(512) k_psi(StepArgs a) {
    using T = typename S::T;
    using V = typename LaneOf<SPT>::V;
    using Ln = Lanes<V>;
    constexpr int NV = SPT / Ln::n;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = __ldg(&a.tiles[t]);
        if (a.quota && a.step >= __ldg(&a.quota[tl.x])) continue;
        const LatDev& L = a.lats[tl.x];
        const int nx = L.nx, ny = L.ny;
        const int x = tl.y + threadIdx.x;
        if (x >= nx) continue;
        const int pitch = L.pitch;
        const int64_t plane = L.plane;
        const T* base = reinterpret_cast<const T*>(a.pop) + L.off_f[a.parity] + (x + L.gx);
        Site<V> sv[NV];
        load_sites<S, SPT>(base, plane, pitch, tl.z + (int)threadIdx.y, (int)blockDim.y, ny, sv);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const V psi = Eos<EOSP>::psi(L, site_rho(sv[j], L.rho0), a.status);
#pragma unroll
            for (int l = 0; l < Ln::n; ++l) {
                const int y = tl.z + (int)threadIdx.y + (j * Ln::n + l) * (int)blockDim.y;
                if (y < ny)
                    store_img(a.psi + L.off_psi, L.pitch_psi, L.gx_psi, x, y, nx, ny,
                              Ln::get(psi, l));
            }
        }
    }
}

// Whether every site of the tile at (x0, y0) lies at least GW from each edge
// (then no site of it has periodic images to write).
__device__ __forceinline__ bool tile_interior(int x0, int y0, int TX, int TY, int nx, int ny) {
    return x0 >= GW && y0 >= GW && x0 + TX <= nx - GW && y0 + TY <= ny - GW;
}

// Collision of the SPT sites of a thread from the psi tile in shared memory
// (row stride W, the thread's column at offset tx + 1) and their stores.
template <class S, int SPT, bool MRT, class V>
__device__ __forceinline__ void collide_store(const LatDev& L, const float* sps, int W, int tx,
                                              int ly0, int by, int x, int y0, const Site<V>* sv,
                                              typename S::T* o, bool tile_in) {
    using Ln = Lanes<V>;
    constexpr int NV = SPT / Ln::n;
    const SiteConsts C = site_consts(L);
    const int nx = L.nx, ny = L.ny;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        V p[9], v[9];
#pragma unroll
        for (int l = 0; l < Ln::n; ++l) {
            const float* c = sps + (ly0 + (j * Ln::n + l) * by + 1) * W + (tx + 1);
            Ln::put(p[0], l, c[0]);
            Ln::put(p[1], l, c[1]);
            Ln::put(p[2], l, c[W]);
            Ln::put(p[3], l, c[-1]);
            Ln::put(p[4], l, c[-W]);
            Ln::put(p[5], l, c[W + 1]);
            Ln::put(p[6], l, c[W - 1]);
            Ln::put(p[7], l, c[-W - 1]);
            Ln::put(p[8], l, c[-W + 1]);
        }
        collide<S, MRT>(C, L.mrt_s, sv[j], p, v);
#pragma unroll
        for (int l = 0; l < Ln::n; ++l) {
            const int y = y0 + (j * Ln::n + l) * by;
            if (y >= ny) break;
            float vs[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) vs[i] = Ln::get(v[i], l);
            store_site<S>(o, L.plane, L.pitch, L.gx, x, y, nx, ny, vs, tile_in);
        }
    }
}

// --------------------------------------------- pass 2: force + collide + store
template <class S, int SPT, bool MRT>
__global__ void __launch_bounds__(512) k_collide(StepArgs a) {
    using T = typename S::T;
    using V = typename LaneOf<SPT>::V;
    constexpr int NV = SPT / Lanes<V>::n;
    extern __shared__ float sps[];
    const int TX = blockDim.x, BY = blockDim.y, TY = BY * SPT;
    const int W = TX + 2;
    const int nthr = TX * BY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = __ldg(&a.tiles[t]);
        if (a.quota && a.step >= __ldg(&a.quota[tl.x])) continue;  // uniform per block
        const LatDev& L = a.lats[tl.x];
        const int nx = L.nx, ny = L.ny;
        const int xend = min(tl.y + TX, nx);  // one past the last active column
        const int yend = min(tl.z + TY, ny);
        __syncthreads();  // the previous tile is done with sps
        {
            const float* ps = a.psi + L.off_psi;
            const int pp = L.pitch_psi, gxp = L.gx_psi;
            const int n = W * (TY + 2);
            for (int k = tid; k < n; k += nthr) {
                const int ly = k / W, lx = k - ly * W;
                const int gx = tl.y - 1 + lx, gy = tl.z - 1 + ly;
                if (gx <= xend && gy <= yend) sps[k] = ps[(int64_t)(gy + GY) * pp + (gx + gxp)];
            }
        }
        const int x = tl.y + threadIdx.x;
        const T* base = reinterpret_cast<const T*>(a.pop) + L.off_f[a.parity] + (x + L.gx);
        Site<V> sv[NV];
        if (x < nx) load_sites<S, SPT>(base, L.plane, L.pitch, tl.z + (int)threadIdx.y, BY, ny, sv);
        __syncthreads();  // psi tile complete
        if (x >= nx) continue;
        collide_store<S, SPT, MRT>(L, sps, W, threadIdx.x, threadIdx.y, BY, x,
                                   tl.z + (int)threadIdx.y, sv,
                                   reinterpret_cast<T*>(a.pop) + L.off_f[a.parity ^ 1],
                                   tile_interior(tl.y, tl.z, TX, TY, nx, ny));
    }
}

// ------------------------------------------- single pass: psi rebuilt in the tile
// One launch per step.  Each thread pulls the populations of its own sites
// (kept in registers for the collision), computes rho (Eq. FD) and psi
// (Eqs. DED, CSEOS) from them and writes psi to shared memory; the first
// threads of the block also compute psi on the one-site ring around the
// tile, two ring cells per thread (pulling from up to two sites out, which
// the ghost frame holds).  After one barrier the collision runs as in
// k_collide.  Every psi is the same function of the same loaded values in
// the same order as in the psi pass, so both schedules give the same
// numbers; DRAM sees each population read once and written once.

template <class S, int EOSP, int SPT, bool MRT>
__global__ void __launch_bounds__(512) k_fused(StepArgs a) {
    using T = typename S::T;
    using V = typename LaneOf<SPT>::V;
    using Ln = Lanes<V>;
    constexpr int NV = SPT / Ln::n;
    extern __shared__ float sps[];
    const int TX = blockDim.x, BY = blockDim.y, TY = BY * SPT;
    const int W = TX + 2;
    const int nthr = TX * BY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int nhalf = TX + TY + 2;  // half of the 2 (TX + TY) + 4 ring cells
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int4 tl = __ldg(&a.tiles[t]);
        if (a.quota && a.step >= __ldg(&a.quota[tl.x])) continue;  // uniform per block
        const LatDev& L = a.lats[tl.x];
        const int nx = L.nx, ny = L.ny;
        const int pitch = L.pitch;
        const int64_t plane = L.plane;
        const T* base = reinterpret_cast<const T*>(a.pop) + L.off_f[a.parity] + L.gx;
        const int xend = min(tl.y + TX, nx);  // one past the last active column
        const int yend = min(tl.z + TY, ny);
        __syncthreads();  // the previous tile is done with sps
        const int x = tl.y + threadIdx.x;
        Site<V> sv[NV];
        if (x < nx) load_sites<S, SPT>(base + x, plane, pitch, tl.z + (int)threadIdx.y, BY, ny, sv);
        // the ring, cells r and r + nhalf in the two lanes of a float2
        for (int r = tid; r < nhalf; r += nthr) {
            int cx0, cy0, cx1, cy1;
            const bool on0 = ring_cell(r, TX, TY, tl.y, tl.z, xend, yend, cx0, cy0);
            const bool on1 = ring_cell(r + nhalf, TX, TY, tl.y, tl.z, xend, yend, cx1, cy1);
            const Site<float> s0 = pulled_site<S>(base + (int64_t)(cy0 + GY) * pitch + cx0, plane, pitch);
            const Site<float> s1 = pulled_site<S>(base + (int64_t)(cy1 + GY) * pitch + cx1, plane, pitch);
            const float2 rho = make_float2(site_rho(s0, L.rho0), site_rho(s1, L.rho0));
            const float2 psi = Eos<EOSP>::psi(L, rho, a.status);
            if (on0) sps[(cy0 - tl.z + 1) * W + (cx0 - tl.y + 1)] = psi.x;
            if (on1) sps[(cy1 - tl.z + 1) * W + (cx1 - tl.y + 1)] = psi.y;
        }
        if (x < nx) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const V psi = Eos<EOSP>::psi(L, site_rho(sv[j], L.rho0), a.status);
#pragma unroll
                for (int l = 0; l < Ln::n; ++l) {
                    const int ly = (int)threadIdx.y + (j * Ln::n + l) * BY;
                    if (tl.z + ly < ny) sps[(ly + 1) * W + (threadIdx.x + 1)] = Ln::get(psi, l);
                }
            }
        }
        __syncthreads();  // psi tile complete
        if (x >= nx) continue;
        collide_store<S, SPT, MRT>(L, sps, W, threadIdx.x, threadIdx.y, BY, x,
                                   tl.z + (int)threadIdx.y, sv,
                                   reinterpret_cast<T*>(a.pop) + L.off_f[a.parity ^ 1],
                                   tile_interior(tl.y, tl.z, TX, TY, nx, ny));
    }
}

// ------------------------------------------------------------------ init
// f*_i(y) = f^eq_i(y + c_i) (FP64), so that the next pull
// f_i(x) = f*_i(x - c_i) yields f^eq_i(x), written in the stored form
// (lbm_device.cuh, rest_finish): R(y) = f*_0(y) - w_0 rho0 rounded to the
// storage type, G_i(y) = (f*_i(y) - w_i rho0) - c'_i (f*_0(y) - w_0 rho0)
// + E/8 with E = 9/4 (exact R - stored R) = -9/4 e0.  Each thread writes
// its own site, gathering the densities of its eight neighbours.  With
// u = 0 (no velocity given) f^eq_i = w_i rho and
// G_i(y) = w_i (rho(y + c_i) - rho(y)) - 9/32 e0: a subtraction and an FMA
// per direction on the FP64 pipe (the slow one on GB300).
template <class S>
__global__ void k_init(LatDev L, void* pop, int parity, const double* rho, const float* rho32,
                       const double* ux, const double* uy) {
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int nx = L.nx, ny = L.ny;
    if (x >= nx || y >= ny) return;
    T* o = reinterpret_cast<T*>(pop) + L.off_f[parity];
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                         1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const bool still = !ux && !uy;
    const double r0 = (double)L.rho0;
    // f^eq_i - w_i rho0 at site (sx, sy), Eq. (SEDF)
    auto geq = [&](int i, int sx, int sy) {
        const int64_t q = (int64_t)sy * nx + sx;
        const double r = rho[q];
        if (still) return w[i] * (r - r0);
        const double vx = ux ? ux[q] : 0.0, vy = uy ? uy[q] : 0.0;
        const double cu = kCx[i] * vx + kCy[i] * vy;
        return w[i] * (r + r * (3.0 * cu + 4.5 * cu * cu - 1.5 * (vx * vx + vy * vy))) - w[i] * r0;
    };
    const double g0 = geq(0, x, y);
    const T R = S::cv((float)g0);
    const double e0 = (double)S::rt((float)g0) - g0;
    store_img(o, L.pitch, L.gx, x, y, nx, ny, R);
    const float rc = rho32 ? rho32[(int64_t)y * nx + x] : 0.f;
    const float e0f = (float)e0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int sx = x + kCx[i], sy = y + kCy[i];
        sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
        sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
        // u = 0: w_i (rho(y + c_i) - rho(y)) from the FP32 copy of the field
        // (the differences of the rounded values sum to zero over the lattice,
        // so the stored mass stays that of the FP64 field), e0 in FP32
        const float G =
            still && rho32
                ? fmaf(-0.28125f, e0f, (float)w[i] * (rho32[(int64_t)sy * nx + sx] - rc))
                : (float)((geq(i, sx, sy) - (double)cref(i) * g0) - 0.28125 * e0);
        store_img(o + i * L.plane, L.pitch, L.gx, x, y, nx, ny, S::cv(G));
    }
}

// ------------------------------------------------------------------ field scan
// The smallest value of a device field and whether every value is finite
// (lbm_init's check of the densities it was handed, on the staged copy):
// each block writes its minimum, or NaN if it met a value that is not
// finite; k_scan_final reduces the partials the same way into *out.  The
// values are also written rounded to FP32 into v32 (k_init's copy).
// The minimum and the finiteness test work on the 64-bit patterns, on the
// integer pipe (GB300's FP64 pipe is slow): a finite double has an exponent
// field below 0x7ff, and flipping the other 63 bits of a negative double
// gives a signed integer key whose order is the order of the values.
__device__ __forceinline__ long long order_key(long long b) {
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool finite_bits(long long b) {
    return (b & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

__global__ void __launch_bounds__(256) k_scan_partial(const double* v, int64_t n, double* partials,
                                                      float* v32) {
    long long m = LLONG_MAX;  // order key of the smallest value so far
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // four independent loads in flight per thread
    for (; i + 3 * stride < n; i += 4 * stride) {
        double x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = v[i + k * stride];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long b = __double_as_longlong(x[k]);
            bad |= !finite_bits(b);
            m = min(m, order_key(b));
            v32[i + k * stride] = (float)x[k];
        }
    }
    for (; i < n; i += stride) {
        const double x = v[i];
        const long long b = __double_as_longlong(x);
        bad |= !finite_bits(b);
        m = min(m, order_key(b));
        v32[i] = (float)x;
    }
    bad = __syncthreads_or(bad);
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ long long red[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long k = red[0];
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j) k = min(k, red[j]);
        // the key of a value is its own inverse
        partials[blockIdx.x] =
            bad ? __longlong_as_double(0x7ff8000000000000LL) : __longlong_as_double(order_key(k));
    }
}

// v rounded to FP32 (the copy k_init reads the neighbours' densities from,
// for fields that are not scanned on the device).
__global__ void k_to_f32(const double* v, int64_t n, float* v32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v32[i] = (float)v[i];
}

// One warp: lane l takes partials l, l + 32, ...; then a shuffle tree.
__global__ void k_scan_final(const double* partials, int n, double* out) {
    const int lane = threadIdx.x & 31;
    long long m = LLONG_MAX;
    bool bad = false;
    for (int i = lane; i < n; i += 32) {
        const long long b = __double_as_longlong(partials[i]);
        bad |= !finite_bits(b);
        m = min(m, order_key(b));
    }
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_down_sync(0xffffffffu, m, o));
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0)
        *out = bad ? __longlong_as_double(0x7ff8000000000000LL) : __longlong_as_double(order_key(m));
}

// ------------------------------------------------------------------ moments
// rho (FP64 sum of the pulled populations) and u = (j + F/2)/rho, with F from
// the psi plane of the current state (computed by k_psi just before).
// Knuth's TwoSum on the FP32 pipe: returns s = fl(a + b) and sets e with
// s + e = a + b exactly (explicit .rn steps the compiler cannot fold).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = vadd(a, b);
    const float bb = vsub(s, a);
    e = vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
    return s;
}

// sum_i w_i v_i for weights w_i in {-1, 0, 1} as an unevaluated pair
// hi + lo: hi by error-free steps, their rounding errors (each at most u
// times a partial sum) gathered in lo with FP32 roundings of their own, so
// that hi + lo is within N^2 u^2 of the largest partial sum of the exact sum
// (u = 2^-24).
// This keeps the per-site sums off the FP64 pipe, which is slow on GB300.
template <int N>
__device__ __forceinline__ void signed_sum(const float v[N], const int w[N], float& hi,
                                           float& lo) {
    hi = 0.f;
    lo = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (w[i] == 0) continue;
        float e;
        hi = two_sum(hi, w[i] > 0 ? v[i] : -v[i], e);
        lo = vadd(lo, e);
    }
}

// Rows y0 .. y1 - 1; the output pointers point at row y0 of their fields.
template <class S>
__global__ void k_moments(LatDev L, const void* pop, int parity, const float* psi_arena,
                          double* rho_out, double* ux_out, double* uy_out, int y0, int y1) {
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const int nx = L.nx;
    if (x >= nx || y >= y1) return;
    const int pitch = L.pitch;
    const int64_t plane = L.plane;
    const T* f = reinterpret_cast<const T*>(pop) + L.off_f[parity] + (int64_t)(y + GY) * pitch +
                 (x + L.gx);
    // the pulled deviations g_i = G_i(x - c_i) + c'_i R(x - c_i) as 17 exact
    // terms: v[i] = G_i, v[8 + i] = c'_i R(x - c_i) (i = 1..8), v[0] = R(x)
    float v[17];
    int ones[17], wx[17], wy[17];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int64_t src = -(int64_t)plane_cy(i) * pitch - plane_cx(i);
        const float R = S::ld(f + src);
        if (i == 0) {
            v[0] = R;
            ones[0] = 1;
            wx[0] = wy[0] = 0;
        } else {
            v[i] = S::ld(f + i * plane + src);
            v[8 + i] = cref(i) * R;
            ones[i] = ones[8 + i] = 1;
            wx[i] = wx[8 + i] = kCx[i];
            wy[i] = wy[8 + i] = kCy[i];
        }
    }
    float hi, lo;
    signed_sum<17>(v, ones, hi, lo);
    // rho = sum_i f_i (Eq. FD) plus the deviation reference, in FP64
    const double rho = ((double)hi + (double)lo) + (double)L.rho0;
    const int64_t s = (int64_t)(y - y0) * nx + x;
    if (rho_out) rho_out[s] = rho;
    if (!ux_out && !uy_out) return;  // density only: no force, psi not read
    float jxh, jxl, jyh, jyl;
    signed_sum<17>(v, wx, jxh, jxl);
    signed_sum<17>(v, wy, jyh, jyl);
    const float* c = psi_arena + L.off_psi + (int64_t)(y + GY) * L.pitch_psi + (x + L.gx_psi);
    const int W = L.pitch_psi;
    const float p[9] = {c[0], c[1], c[W], c[-1], c[-W], c[W + 1], c[W - 1], c[-W - 1], c[-W + 1]};
    float Fx, Fy;
    site_force(site_consts(L), p, Fx, Fy);
    // force-shifted velocity, Eq. FMD
    const double inv = 1.0 / rho;
    if (ux_out) ux_out[s] = (((double)jxh + (double)jxl) + 0.5 * (double)Fx) * inv;
    if (uy_out) uy_out[s] = (((double)jyh + (double)jyl) + 0.5 * (double)Fy) * inv;
}

// ------------------------------------------------------------------ mass
// Each block sums whole rows of all nine planes and writes one FP64
// partial; k_mass_final adds the partials in a fixed order (deterministic).
// A site's stored mass rho0 + 9/4 R + sum_i G_i (lbm_device.cuh) is summed
// as a float-float pair over the exact terms R, R, R/4, G_1 .. G_8
// (signed_sum); the pairs' leading parts accumulate in FP64, their small
// trailing parts in FP32, and the sites' rho0 is added once per thread.
template <class S>
__global__ void __launch_bounds__(256) k_mass_partial(LatDev L, const void* pop, int parity,
                                                      double* partials) {
    using T = typename S::T;
    const T* f = reinterpret_cast<const T*>(pop) + L.off_f[parity];
    const int nx = L.nx, ny = L.ny;
    constexpr int kOne[11] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    double acc = 0.0;
    float acc_lo = 0.f;
    int64_t sites = 0;
    for (int y = blockIdx.x; y < ny; y += gridDim.x) {
        const T* row = f + (int64_t)(y + GY) * L.pitch + L.gx;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            float v[11];
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = S::ld(row + i * L.plane + x);
            v[9] = v[0];
            v[10] = 0.25f * v[0];
            float hi, lo;
            signed_sum<11>(v, kOne, hi, lo);
            acc += (double)hi;
            acc_lo = vadd(acc_lo, lo);
            ++sites;
        }
    }
    acc += (double)acc_lo + (double)sites * (double)L.rho0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) partials[blockIdx.x] = acc;
    }
}

__global__ void k_mass_final(const double* partials, int n, double* out) {
    // one warp: lane l adds partials l, l + 32, ... in order, then a fixed
    // shuffle tree (deterministic)
    const int lane = threadIdx.x & 31;
    double m = 0.0;
    for (int i = lane; i < n; i += 32) m += partials[i];
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if (lane == 0) *out = m;
}

// ------------------------------------------------------------------ arithmetic check
// The step's reciprocal and square root on n values: paired lanes (two
// values per thread, as the kernels run them) to the outputs, and the scalar
// lane on each value, compared bitwise (a mismatch sets *mismatch).
__global__ void k_arith_check(const float* x, int64_t n, float* rcp, float* sq,
                              uint32_t* mismatch) {
    const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const bool two = i + 1 < n;
    const float2 v = make_float2(x[i], two ? x[i + 1] : 1.f);
    const float2 r2 = vrcp(v), s2 = vsqrt(v);
    bool same = __float_as_uint(vrcp(v.x)) == __float_as_uint(r2.x) &&
                __float_as_uint(vsqrt(v.x)) == __float_as_uint(s2.x);
    if (two)
        same = same && __float_as_uint(vrcp(v.y)) == __float_as_uint(r2.y) &&
               __float_as_uint(vsqrt(v.y)) == __float_as_uint(s2.y);
    if (!same) atomicOr(mismatch, 1u);
    rcp[i] = r2.x;
    sq[i] = s2.x;
    if (two) {
        rcp[i + 1] = r2.y;
        sq[i + 1] = s2.y;
    }
}

// ------------------------------------------------------------------ EOS check
// The step's psi (Eqs. DED and CSEOS, or van der Waals) of n given densities
// with the constants of lattice L: paired lanes (two values per thread, as
// the kernels run them) to psi, the scalar lane on each value compared
// bitwise (a mismatch sets bit 0 of *flags); for the float-float arithmetic
// also the radicand rho (hh + hl) before its rounding to FP32, in FP64
// (NaN for the other arithmetics).
template <int EOSP>
__global__ void k_eos_check(LatDev L, const float* rho, int64_t n, float* psi, double* rad,
                            uint32_t* flags) {
    const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const bool two = i + 1 < n;
    const float2 r2 = make_float2(rho[i], two ? rho[i + 1] : rho[i]);
    uint32_t* st = flags + 1;  // numeric fault bits land here, not in a handle
    const float2 p2 = Eos<EOSP>::psi(L, r2, st);
    const float p0 = Eos<EOSP>::psi(L, r2.x, st), p1 = Eos<EOSP>::psi(L, r2.y, st);
    if (__float_as_uint(p0) != __float_as_uint(p2.x) || (two && __float_as_uint(p1) != __float_as_uint(p2.y)))
        atomicOr(flags, 1u);
    psi[i] = p2.x;
    if (two) psi[i + 1] = p2.y;
    double r0 = __longlong_as_double(0x7ff8000000000000LL), r1 = r0;
    if (EOSP == EOS_DF) {
        float2 sh, hh, hl;
        Eos<EOS_DF>::radicand(L, r2, sh, hh, hl);
        r0 = (double)r2.x * (double)hh.x + (double)r2.x * (double)hl.x;
        r1 = (double)r2.y * (double)hh.y + (double)r2.y * (double)hl.y;
    }
    rad[i] = r0;
    if (two) rad[i + 1] = r1;
}

cudaError_t launch_eos_check(int eos, const LatDev& L, const float* rho, int64_t n, float* psi,
                             double* rad, uint32_t* flags, cudaStream_t st) {
    const int64_t pairs = (n + 1) / 2;
    const unsigned g = (unsigned)((pairs + 255) / 256);
    switch (eos) {
        case EOS_F64: k_eos_check<EOS_F64><<<g, 256, 0, st>>>(L, rho, n, psi, rad, flags); break;
        case EOS_DF: k_eos_check<EOS_DF><<<g, 256, 0, st>>>(L, rho, n, psi, rad, flags); break;
        case EOS_F32: k_eos_check<EOS_F32><<<g, 256, 0, st>>>(L, rho, n, psi, rad, flags); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ================================================================ launchers
namespace {
template <class S, int SPT>
cudaError_t psi_dispatch(int eos, const StepArgs& a, dim3 g, dim3 b, cudaStream_t st) {
    switch (eos) {
        case EOS_F64: k_psi<S, EOS_F64, SPT><<<g, b, 0, st>>>(a); break;
        case EOS_DF: k_psi<S, EOS_DF, SPT><<<g, b, 0, st>>>(a); break;
        case EOS_F32: k_psi<S, EOS_F32, SPT><<<g, b, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template <class S>
cudaError_t psi_spt(int spt, int eos, const StepArgs& a, dim3 g, dim3 b, cudaStream_t st) {
    switch (spt) {
        case 1: return psi_dispatch<S, 1>(eos, a, g, b, st);
        case 2: return psi_dispatch<S, 2>(eos, a, g, b, st);
        case 4: return psi_dispatch<S, 4>(eos, a, g, b, st);
        default: return cudaErrorInvalidValue;
    }
}
template <class S, bool MRT>
cudaError_t collide_spt(int spt, const StepArgs& a, dim3 g, dim3 b, size_t smem,
                        cudaStream_t st) {
    switch (spt) {
        case 1: k_collide<S, 1, MRT><<<g, b, smem, st>>>(a); break;
        case 2: k_collide<S, 2, MRT><<<g, b, smem, st>>>(a); break;
        case 4: k_collide<S, 4, MRT><<<g, b, smem, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template <class S>
const void* psi_fn(int spt, int eos) {
#define PPLBM_F(N)                                                                  \
    if (spt == N)                                                                   \
        return eos == EOS_F64 ? (const void*)k_psi<S, EOS_F64, N>                   \
             : eos == EOS_DF  ? (const void*)k_psi<S, EOS_DF, N>                    \
                              : (const void*)k_psi<S, EOS_F32, N>;
    PPLBM_F(1)
    PPLBM_F(2)
    PPLBM_F(4)
#undef PPLBM_F
    return nullptr;
}
template <class S, bool MRT>
const void* collide_fn(int spt) {
    return spt == 1 ? (const void*)k_collide<S, 1, MRT>
         : spt == 2 ? (const void*)k_collide<S, 2, MRT>
         : spt == 4 ? (const void*)k_collide<S, 4, MRT> : nullptr;
}
}  // namespace

bool plain_spt_supported(int spt) { return spt == 1 || spt == 2 || spt == 4; }

namespace {
template <class S, int SPT, bool MRT>
cudaError_t fused_eos(int eos, const StepArgs& a, dim3 g, dim3 b, size_t smem, cudaStream_t st) {
    switch (eos) {
        case EOS_F64: k_fused<S, EOS_F64, SPT, MRT><<<g, b, smem, st>>>(a); break;
        case EOS_DF: k_fused<S, EOS_DF, SPT, MRT><<<g, b, smem, st>>>(a); break;
        case EOS_F32: k_fused<S, EOS_F32, SPT, MRT><<<g, b, smem, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
template <class S, bool MRT>
cudaError_t fused_spt(int spt, int eos, const StepArgs& a, dim3 g, dim3 b, size_t smem,
                      cudaStream_t st) {
    switch (spt) {
        case 1: return fused_eos<S, 1, MRT>(eos, a, g, b, smem, st);
        case 2: return fused_eos<S, 2, MRT>(eos, a, g, b, smem, st);
        case 4: return fused_eos<S, 4, MRT>(eos, a, g, b, smem, st);
        default: return cudaErrorInvalidValue;
    }
}
template <class S, bool MRT>
const void* fused_fn(int spt, int eos) {
#define PPLBM_F(N)                                                                  \
    if (spt == N)                                                                   \
        return eos == EOS_F64 ? (const void*)k_fused<S, EOS_F64, N, MRT>            \
             : eos == EOS_DF  ? (const void*)k_fused<S, EOS_DF, N, MRT>             \
                              : (const void*)k_fused<S, EOS_F32, N, MRT>;
    PPLBM_F(1)
    PPLBM_F(2)
    PPLBM_F(4)
#undef PPLBM_F
    return nullptr;
}
}  // namespace

cudaError_t launch_fused(int storage_f16, int mrt, int eos, int spt, const StepArgs& a, dim3 g,
                         dim3 b, size_t smem, cudaStream_t st) {
    if (mrt)
        return storage_f16 ? fused_spt<StoreF16, true>(spt, eos, a, g, b, smem, st)
                           : fused_spt<StoreF32, true>(spt, eos, a, g, b, smem, st);
    return storage_f16 ? fused_spt<StoreF16, false>(spt, eos, a, g, b, smem, st)
                       : fused_spt<StoreF32, false>(spt, eos, a, g, b, smem, st);
}

int occupancy_fused(int storage_f16, int mrt, int eos, int spt, int threads, size_t smem) {
    int n = 0;
    const void* fn = mrt ? (storage_f16 ? fused_fn<StoreF16, true>(spt, eos)
                                        : fused_fn<StoreF32, true>(spt, eos))
                         : (storage_f16 ? fused_fn<StoreF16, false>(spt, eos)
                                        : fused_fn<StoreF32, false>(spt, eos));
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_psi(int storage_f16, int eos, int spt, const StepArgs& a, dim3 g, dim3 b,
                       cudaStream_t st) {
    return storage_f16 ? psi_spt<StoreF16>(spt, eos, a, g, b, st)
                       : psi_spt<StoreF32>(spt, eos, a, g, b, st);
}

cudaError_t launch_collide(int storage_f16, int mrt, int spt, const StepArgs& a, dim3 g,
                           dim3 b, size_t smem, cudaStream_t st) {
    if (mrt)
        return storage_f16 ? collide_spt<StoreF16, true>(spt, a, g, b, smem, st)
                           : collide_spt<StoreF32, true>(spt, a, g, b, smem, st);
    return storage_f16 ? collide_spt<StoreF16, false>(spt, a, g, b, smem, st)
                       : collide_spt<StoreF32, false>(spt, a, g, b, smem, st);
}

cudaError_t launch_init(int storage_f16, const LatDev& L, void* pop, int parity,
                        const double* rho, const float* rho32, const double* ux, const double* uy,
                        cudaStream_t st) {
    dim3 b(32, 8), g((L.nx + 31) / 32, (L.ny + 7) / 8);
    if (storage_f16)
        k_init<StoreF16><<<g, b, 0, st>>>(L, pop, parity, rho, rho32, ux, uy);
    else
        k_init<StoreF32><<<g, b, 0, st>>>(L, pop, parity, rho, rho32, ux, uy);
    return cudaGetLastError();
}

cudaError_t launch_moments(int storage_f16, const LatDev& L, const void* pop, int parity,
                           const float* psi, double* rho, double* ux, double* uy, int y0, int y1,
                           cudaStream_t st) {
    if (y1 <= y0) return cudaSuccess;
    // rows y0 .. y1 - 1: the outputs' rows start at row y0 of the [ny][nx] fields
    dim3 b(32, 8), g((L.nx + 31) / 32, (y1 - y0 + 7) / 8);
    const int64_t off = (int64_t)y0 * L.nx;
    double* r = rho ? rho + off : nullptr;
    double* u = ux ? ux + off : nullptr;
    double* v = uy ? uy + off : nullptr;
    if (storage_f16)
        k_moments<StoreF16><<<g, b, 0, st>>>(L, pop, parity, psi, r, u, v, y0, y1);
    else
        k_moments<StoreF32><<<g, b, 0, st>>>(L, pop, parity, psi, r, u, v, y0, y1);
    return cudaGetLastError();
}

cudaError_t launch_mass(int storage_f16, const LatDev& L, const void* pop, int parity,
                        double* partials, int n_partials, double* out, cudaStream_t st) {
    const int nb = n_partials < L.ny ? n_partials : L.ny;
    if (storage_f16)
        k_mass_partial<StoreF16><<<nb, 256, 0, st>>>(L, pop, parity, partials);
    else
        k_mass_partial<StoreF32><<<nb, 256, 0, st>>>(L, pop, parity, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, 32, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_scan(const double* v, int64_t n, double* partials, int n_partials, double* out,
                        float* v32, cudaStream_t st) {
    const int64_t want = (n + 255) / 256;
    const int nb = (int)(want < n_partials ? want : n_partials);
    k_scan_partial<<<nb, 256, 0, st>>>(v, n, partials, v32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_final<<<1, 32, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* v, int64_t n, float* v32, cudaStream_t st) {
    const int64_t want = (n + 255) / 256;
    k_to_f32<<<(unsigned)(want < 4096 ? want : 4096), 256, 0, st>>>(v, n, v32);
    return cudaGetLastError();
}

cudaError_t launch_arith_check(const float* x, int64_t n, float* rcp, float* sq,
                               uint32_t* mismatch, cudaStream_t st) {
    const int64_t pairs = (n + 1) / 2;
    k_arith_check<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(x, n, rcp, sq, mismatch);
    return cudaGetLastError();
}

int occupancy_psi(int storage_f16, int eos, int spt, int threads) {
    int n = 0;
    const void* fn = storage_f16 ? psi_fn<StoreF16>(spt, eos) : psi_fn<StoreF32>(spt, eos);
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

int occupancy_collide(int storage_f16, int mrt, int spt, int threads, size_t smem) {
    int n = 0;
    const void* fn = mrt ? (storage_f16 ? collide_fn<StoreF16, true>(spt)
                                        : collide_fn<StoreF32, true>(spt))
                         : (storage_f16 ? collide_fn<StoreF16, false>(spt)
                                        : collide_fn<StoreF32, false>(spt));
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace pplbm
