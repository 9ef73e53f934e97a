// lbm_runtime.cu -- the C ABI of include/pplbm.h: handles, device memory
// layout, step scheduling (direct launches or captured CUDA graphs),
// measurement hooks and the tile-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pplbm.h"
#include "lbm_async.cuh"
#include "lbm_copy_plan.h"
#include "lbm_kernels.h"
#include "lbm_host_scan.h"
#include "lbm_layout.h"

using namespace pplbm;

namespace {

constexpr int kMassPartials = 1024;

struct ProfRec {
    std::string name;
    int64_t launches = 0;
    double total_ms = 0.0;
    double bytes = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

struct TuneKey {
    int device, storage, eos, schedule;
    int64_t sites_class, nlat_class;
    bool operator<(const TuneKey& o) const {
        return std::tie(device, storage, eos, schedule, sites_class, nlat_class) <
               std::tie(o.device, o.storage, o.eos, o.schedule, o.sites_class, o.nlat_class);
    }
};
struct PassCfg {
    int variant, tx, ty, grid, spt;
};
struct TuneVal {
    PassCfg pass[2];
};

// One pass of the step (0: psi, 1: force + collision + stream): its kernel
// variant, tile shape, tile list and persistent grid.
struct Pass {
    int variant = LBM_KERNEL_TMA;
    int tx = 64, ty = 8, grid = 1, ntiles = 0;
    int spt = 1;  // sites per thread of the plain kernels (the block is tx x ty/spt)
    int4* tiles = nullptr;
    size_t cap = 0;
    std::vector<int> begin, count;  // per-lattice tile ranges
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

}  // namespace

struct lbm_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lbm_runtime_opts opts{};
    std::vector<lbm_lattice_desc> desc;
    std::vector<LatDev> lat;
    int storage = LBM_STORE_F32_DEV;
    int f16 = 0;
    int eos = LBM_EOS_F64;
    int collision = LBM_COLL_BGK;
    int schedule = LBM_SCHED_FUSED;
    // device memory
    void* pop = nullptr;
    size_t pop_bytes = 0;
    float* psi = nullptr;
    size_t psi_bytes = 0;
    LatDev* lat_dev = nullptr;
    uint32_t* status = nullptr;
    Pass pass[2];
    double* partials = nullptr;  // mass partials + one result slot
    double* staging = nullptr;   // FP64 field staging (rho, ux, uy), then rho in FP32
    size_t staging_elems = 0;
    cudaStream_t side = nullptr;  // copies of lbm_moments results, beside the kernels
    cudaEvent_t chunk_ev[5] = {};
    int64_t device_bytes = 0;
    // host side
    uint32_t* status_host = nullptr;  // pinned
    double* scan_host = nullptr;      // pinned: lbm_init's field scan result
    cudaEvent_t status_ev = nullptr;
    bool status_pending = false;
    int32_t starve = 0;        // armed failure-detection test (tile + 1), for one launch
    int numeric_lattice = -1;  // first lattice with a device fault bit
    uint32_t fault_bits = 0;   // OR of the device fault bits seen
    int sm_count = 0;
    int parity = 0;
    int64_t sites = 0;
    int64_t launches = 0;
    // graphs
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // by starting parity
    int graph_steps = 32;
    int tune_variant = LBM_KERNEL_AUTO;  // the kernel_variant the handle was created with
    // tensor maps (loads, stores) of the population arena for the single-pass
    // TMA kernel (one lattice, or a batch in one row space; rows at least a box
    // wide); else that kernel uses row copies
    CUtensorMap tmap[2]{};  // loads, stores
    bool has_tmap = false;
    // profiling
    bool prof = false;
    ProfRec rec[2];
    std::vector<cudaEvent_t> ev_pool;
    std::string err;
};

// ------------------------------------------------------------------ helpers
namespace {

int cuda_fail(lbm_handle* h, cudaError_t e, const char* what) {
    if (h) {
        h->err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    }
    return LBM_ERR_CUDA;
}

#define CK(h, call)                                        \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

void* dev_alloc(lbm_handle* h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (h->opts.alloc) {
        p = h->opts.alloc(bytes, h->opts.alloc_ctx);
        if (p && (reinterpret_cast<uintptr_t>(p) & 255u)) {
            h->opts.free(p, bytes, h->opts.alloc_ctx);
            h->err = "allocator returned memory not aligned to 256 bytes";
            return nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) h->device_bytes += (int64_t)bytes;
    return p;
}

void dev_free(lbm_handle* h, void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (h->opts.alloc)
        h->opts.free(p, bytes, h->opts.alloc_ctx);
    else
        cudaFree(p);
    h->device_bytes -= (int64_t)bytes;
}

LatDev make_lat(const lbm_lattice_desc& d, int index, int64_t& pop_cursor,
                int64_t& psi_cursor) {
    LatDev L = lat_layout(d, index);
    L.off_f[0] = pop_cursor;
    L.off_f[1] = pop_cursor + 9 * L.plane;
    pop_cursor += lat_pop_elems(L);
    L.off_psi = psi_cursor;
    psi_cursor += lat_psi_elems(L);
    return L;
}

void drop_graph(lbm_handle* h);

int build_tiles(lbm_handle* h, int k, int tx, int ty) {
    drop_graph(h);  // captured launches embed the tile lists, grids and tensor map
    Pass& P = h->pass[k];
    if (k == 1)
        h->has_tmap = h->schedule == LBM_SCHED_FUSED && P.variant == LBM_KERNEL_TMA &&
                      fused_tma_make_map(h->f16, tx, ty, h->lat.data(), (int)h->lat.size(),
                                         h->pop, h->tmap);
    std::vector<int4> t;
    P.begin.assign(h->lat.size(), 0);
    P.count.assign(h->lat.size(), 0);
    for (size_t l = 0; l < h->lat.size(); ++l) {
        const LatDev& L = h->lat[l];
        P.begin[l] = (int)t.size();
        for (int y0 = 0; y0 < L.ny; y0 += ty)
            for (int x0 = 0; x0 < L.nx; x0 += tx) t.push_back(make_int4((int)l, x0, y0, 0));
        P.count[l] = (int)t.size() - P.begin[l];
    }
    const size_t bytes = t.size() * sizeof(int4);
    if (bytes > P.cap) {
        dev_free(h, P.tiles, P.cap);
        P.tiles = (int4*)dev_alloc(h, bytes);
        if (!P.tiles) {
            P.cap = 0;
            return LBM_ERR_OOM;
        }
        P.cap = bytes;
    }
    CK(h, cudaMemcpyAsync(P.tiles, t.data(), bytes, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    P.tx = tx;
    P.ty = ty;
    P.ntiles = (int)t.size();
    return LBM_OK;
}

bool shape_ok(int variant, int tx, int ty, int spt, bool fused = false) {
    if (variant == LBM_KERNEL_TMA)
        return fused ? fused_tma_shape_supported(tx, ty) : tma_shape_supported(tx, ty);
    return tx > 0 && ty > 0 && (tx % 32) == 0 && plain_spt_supported(spt) && ty % spt == 0 &&
           tx * (ty / spt) <= 512;
}

size_t collide_smem(int tx, int ty) { return (size_t)(tx + 2) * (ty + 2) * sizeof(float); }

// Persistent grid of pass k: SMs x resident CTAs, capped by the tile count.
void default_grid(lbm_handle* h, int k) {
    Pass& P = h->pass[k];
    int occ;
    if (P.variant == LBM_KERNEL_TMA && k == 1 && h->schedule == LBM_SCHED_FUSED)
        occ = occupancy_fused_tma(h->f16, h->collision == LBM_COLL_MRT, h->eos, P.tx, P.ty,
                                  h->has_tmap, h->lat.size() == 1);
    else if (P.variant == LBM_KERNEL_TMA)
        occ = k == 0 ? occupancy_psi_tma(h->f16, h->eos, P.tx, P.ty)
                     : occupancy_collide_tma(h->f16, P.tx, P.ty);
    else if (k == 1 && h->schedule == LBM_SCHED_FUSED)
        occ = occupancy_fused(h->f16, h->collision == LBM_COLL_MRT, h->eos, P.spt, P.tx * (P.ty / P.spt),
                              collide_smem(P.tx, P.ty));
    else
        occ = k == 0 ? occupancy_psi(h->f16, h->eos, P.spt, P.tx * (P.ty / P.spt))
                     : occupancy_collide(h->f16, h->collision == LBM_COLL_MRT, P.spt, P.tx * (P.ty / P.spt),
                                         collide_smem(P.tx, P.ty));
    P.grid = std::max(1, std::min(P.ntiles, h->sm_count * occ));
}

void drop_graph(lbm_handle* h) {
    for (auto& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

StepArgs step_args(lbm_handle* h, int parity, int k) {
    StepArgs a{};
    a.lats = h->lat_dev;
    a.tiles = h->pass[k].tiles;
    a.ntiles = h->pass[k].ntiles;
    a.pop = h->pop;
    a.psi = h->psi;
    a.status = h->status;
    a.parity = parity;
    a.quota = nullptr;
    a.step = 0;
    return a;
}

cudaError_t launch_pass(lbm_handle* h, int k, const StepArgs& a, int grid) {
    const Pass& P = h->pass[k];
    const dim3 block(P.tx, P.ty / P.spt);
    if (k == 0)
        return P.variant == LBM_KERNEL_TMA
                   ? launch_psi_tma(h->f16, h->eos, P.tx, P.ty, a, grid, h->stream)
                   : launch_psi(h->f16, h->eos, P.spt, a, dim3(grid), block, h->stream);
    if (h->schedule == LBM_SCHED_FUSED && P.variant == LBM_KERNEL_TMA)
        return launch_fused_tma(h->f16, h->collision == LBM_COLL_MRT, h->eos, P.tx, P.ty, a,
                                h->has_tmap ? h->tmap : nullptr,
                                h->lat.size() == 1 ? &h->lat[0] : nullptr, grid, h->stream);
    if (h->schedule == LBM_SCHED_FUSED)
        return launch_fused(h->f16, h->collision == LBM_COLL_MRT, h->eos, P.spt, a, dim3(grid), block, collide_smem(P.tx, P.ty),
                            h->stream);
    return P.variant == LBM_KERNEL_TMA
               ? launch_collide_tma(h->f16, P.tx, P.ty, a, grid, h->stream)
               : launch_collide(h->f16, h->collision == LBM_COLL_MRT, P.spt, a, dim3(grid), block, collide_smem(P.tx, P.ty),
                                h->stream);
}

cudaEvent_t take_event(lbm_handle* h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch the two passes of one step on parity p (state in buffer p, result
// in buffer p^1).  Records events around each launch when profiling.
int launch_step(lbm_handle* h, int p) {
    const bool fused = h->schedule == LBM_SCHED_FUSED;
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (h->prof) {
        e1 = take_event(h);
        e2 = take_event(h);
        if (!fused) {
            e0 = take_event(h);
            CK(h, cudaEventRecord(e0, h->stream));
        }
    }
    if (!fused) CK(h, launch_pass(h, 0, step_args(h, p, 0), h->pass[0].grid));
    if (h->prof) CK(h, cudaEventRecord(e1, h->stream));
    StepArgs a1 = step_args(h, p, 1);
    a1.starve = h->starve;  // an armed failure-detection test goes into this launch only
    if (h->starve) a1.wait_cycles = kTestWaitBudgetCycles;
    h->starve = 0;
    CK(h, launch_pass(h, 1, a1, h->pass[1].grid));
    if (h->prof) {
        CK(h, cudaEventRecord(e2, h->stream));
        // the psi pair owns e0, the step pair owns e1 and e2
        if (!fused) h->rec[0].pending.emplace_back(e0, e1);
        h->rec[1].pending.emplace_back(e1, e2);
    }
    h->launches += fused ? 1 : 2;
    return LBM_OK;
}

int capture_graph(lbm_handle* h) {
    cudaGraphExec_t& slot = h->graph[h->parity];
    if (slot) {
        cudaGraphExecDestroy(slot);
        slot = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int p = h->parity;
    const int64_t before = h->launches;
    int rc = LBM_OK;
    for (int s = 0; s < h->graph_steps && rc == LBM_OK; ++s) {
        rc = launch_step(h, p);
        p ^= 1;
    }
    h->launches = before;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&slot, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        slot = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    return LBM_OK;
}

int fault_code(lbm_handle* h) {
    if (h->fault_bits & 2u) return LBM_ERR_TIMEOUT;
    if (h->fault_bits & 4u) {
        h->err = "a staging copy broke the bulk-copy alignment rules and was skipped";
        return LBM_ERR_STATE;
    }
    return h->numeric_lattice >= 0 ? LBM_ERR_NUMERIC : LBM_OK;
}

void absorb_status(lbm_handle* h) {
    for (size_t l = 0; l < h->lat.size(); ++l)
        if (h->status_host[l]) {
            h->fault_bits |= h->status_host[l];
            if (h->numeric_lattice < 0) h->numeric_lattice = (int)l;
        }
}

int check_status_async(lbm_handle* h) {
    if (h->status_pending && cudaEventQuery(h->status_ev) == cudaSuccess) {
        h->status_pending = false;
        absorb_status(h);
    }
    return fault_code(h);
}

int sync_status(lbm_handle* h) {
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->status_host, h->status, h->lat.size() * sizeof(uint32_t),
                     cudaMemcpyDeviceToHost));
    h->status_pending = false;
    absorb_status(h);
    return fault_code(h);
}

// Bytes of the staging buffer for fields of `elems` sites: three FP64 fields
// and one FP32 copy of the density.
size_t staging_bytes(size_t elems) { return elems * (3 * sizeof(double) + sizeof(float)); }
float* staging32(lbm_handle* h) { return reinterpret_cast<float*>(h->staging + 3 * h->staging_elems); }

int ensure_staging(lbm_handle* h, size_t elems) {
    if (elems <= h->staging_elems) return LBM_OK;
    dev_free(h, h->staging, staging_bytes(h->staging_elems));
    h->staging = (double*)dev_alloc(h, staging_bytes(elems));
    if (!h->staging) {
        h->staging_elems = 0;
        return LBM_ERR_OOM;
    }
    h->staging_elems = elems;
    return LBM_OK;
}

void release(lbm_handle* h) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    // psi pairs own e0; step pairs own (e1, e2)
    for (auto& pr : h->rec[0].pending) cudaEventDestroy(pr.first);
    for (auto& pr : h->rec[1].pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    h->rec[0].pending.clear();
    h->rec[1].pending.clear();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    if (h->status_ev) cudaEventDestroy(h->status_ev);
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->scan_host) cudaFreeHost(h->scan_host);
    dev_free(h, h->staging, staging_bytes(h->staging_elems));
    dev_free(h, h->partials, (kMassPartials + 1) * sizeof(double));
    for (cudaEvent_t& e : h->chunk_ev)
        if (e) cudaEventDestroy(e);
    if (h->side) cudaStreamDestroy(h->side);
    for (auto& P : h->pass) dev_free(h, P.tiles, P.cap);
    dev_free(h, h->status, h->lat.size() * sizeof(uint32_t));
    dev_free(h, h->lat_dev, h->lat.size() * sizeof(LatDev));
    dev_free(h, h->psi, h->psi_bytes);
    dev_free(h, h->pop, h->pop_bytes);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Host proof of one tile's copy plan (see lbm_copy_plan.h).
template <int ES, int TX, int TY, bool P>
std::string check_plan_t(const LatDev& L, int par, int x0, int y0, int64_t lo, int64_t hi,
                         int64_t plo, int64_t phi) {
    using G = TileGeo<ES, TX, TY, P>;
    char buf[256];
    // bytes of the stage written by some copy
    std::vector<char> cov(G::STAGEB, 0);
    int64_t total = 0;
    for (int q = 0; q < G::NCOPY; ++q) {
        CopyOp op;
        if (!plan_copy<ES, TX, TY, P>(L, par, x0, y0, q, op)) continue;
        const int64_t a = op.psi ? plo : lo, b = op.psi ? phi : hi;
        if (op.src % 16 || op.dst % 16 || op.bytes % 16 || op.bytes <= 0 || op.src < a ||
            op.src + op.bytes > b || op.dst < 0 || op.dst + op.bytes > G::STAGEB) {
            std::snprintf(buf, sizeof buf,
                          "bad copy: es=%d tile=%dx%d psi=%d lattice %dx%d x0=%d y0=%d q=%d src=%lld "
                          "dst=%d bytes=%d range=[%lld,%lld)",
                          ES, TX, TY, (int)P, L.nx, L.ny, x0, y0, q, (long long)op.src, op.dst,
                          op.bytes, (long long)a, (long long)b);
            return buf;
        }
        // a population copy must stay inside its own box
        if (!op.psi) {
            const int box = op.dst < G::BOX0B ? 0 : 1 + (op.dst - G::BOX0B) / G::BOXB;
            if (box > 8 || op.dst + op.bytes > G::boxoff(box) + (box ? TY : G::ROWS0) * G::BW * ES)
                return "copy crosses its box";
        }
        for (int k = 0; k < op.bytes; ++k) cov[op.dst + k] = 1;
        total += op.bytes;
    }
    if (total >= (1 << 20)) return "transaction count too large";
    // every value an active site reads is covered
    for (int ty = 0; ty < TY; ++ty)
        for (int tx = 0; tx < TX; ++tx) {
            const int x = x0 + tx, y = y0 + ty;
            if (x >= L.nx || y >= L.ny) continue;
            // the pulled value of every plane and the rest value of its source
            for (int i = 0; i < 18; ++i) {
                const int off = (i < 9 ? G::pull(i, tx, ty) : G::rest(i - 9, tx, ty)) * ES;
                const int b = i < 9 ? i : 0;  // the box the value must lie in
                const int lo_b = G::boxoff(b), hi_b = lo_b + (b ? TY : G::ROWS0) * G::BW * ES;
                for (int k = 0; k < ES; ++k)
                    if (off < lo_b || off + k >= hi_b || !cov[off + k]) {
                        std::snprintf(buf, sizeof buf, "uncovered read: %s %d site (%d,%d)",
                                      i < 9 ? "plane" : "rest of", i % 9, x, y);
                        return buf;
                    }
            }
            if (P)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int off = G::POPB + ((ty + 1 + dy) * G::PW + tx + 4 + dx) * 4;
                        for (int k = 0; k < 4; ++k)
                            if (!cov[off + k]) return "uncovered psi read";
                    }
        }
    return "";
}

// Host proof of one fused tile's copy plan (FusedGeo): every copy aligned,
// inside the lattice allocation and inside its own box, and every pulled
// value that an active site or a ring cell (clamped or not) reads covered.
template <int ES, int TX, int TY>
std::string check_fused_t(const LatDev& L, int par, int x0, int y0, int64_t lo, int64_t hi) {
    using G = FusedGeo<ES, TX, TY>;
    char buf[256];
    std::vector<char> cov(G::STAGEB, 0);
    for (int q = 0; q < G::NCOPY; ++q) {
        CopyOp op;
        if (!plan_copy_fused<ES, TX, TY>(L, par, x0, y0, q, op)) continue;
        const int box = op.dst < G::BOX0B ? 0 : 1 + (op.dst - G::BOX0B) / G::BOXB;
        if (op.src % 16 || op.dst % 16 || op.bytes % 16 || op.bytes <= 0 || op.src < lo ||
            op.src + op.bytes > hi || op.dst < 0 || box > 8 ||
            op.dst + op.bytes > G::boxoff(box) + G::rows(box) * G::BW * ES) {
            std::snprintf(buf, sizeof buf,
                          "bad fused copy: es=%d tile=%dx%d lattice %dx%d x0=%d y0=%d q=%d src=%lld "
                          "dst=%d bytes=%d range=[%lld,%lld)",
                          ES, TX, TY, L.nx, L.ny, x0, y0, q, (long long)op.src, op.dst, op.bytes,
                          (long long)lo, (long long)hi);
            return buf;
        }
        for (int k = 0; k < op.bytes; ++k) cov[op.dst + k] = 1;
    }
    const int xend = std::min(x0 + TX, L.nx), yend = std::min(y0 + TY, L.ny);
    // the pulled value of every plane and the rest value of its source
    auto covered = [&](int gx, int gy) {
        for (int i = 0; i < 18; ++i) {
            const int off = (i < 9 ? G::pull(i, gx - x0, gy - y0) : G::rest(i - 9, gx - x0, gy - y0)) * ES;
            const int b = i < 9 ? i : 0;  // the box the value must lie in
            if (off < G::boxoff(b) || off + ES > G::boxoff(b) + G::rows(b) * G::BW * ES)
                return false;
            for (int k = 0; k < ES; ++k)
                if (!cov[off + k]) return false;
        }
        return true;
    };
    for (int y = y0; y < yend; ++y)
        for (int x = x0; x < xend; ++x)
            if (!covered(x, y)) {
                std::snprintf(buf, sizeof buf, "uncovered fused read: site (%d,%d) of %dx%d", x, y,
                              L.nx, L.ny);
                return buf;
            }
    for (int r = 0; r < 2 * (TX + TY) + 4; ++r) {
        int gx, gy;
        ring_cell(r, TX, TY, x0, y0, xend, yend, gx, gy);
        if (!covered(gx, gy)) {
            std::snprintf(buf, sizeof buf, "uncovered fused read: ring cell %d (%d,%d) of %dx%d", r,
                          gx, gy, L.nx, L.ny);
            return buf;
        }
    }
    return "";
}

// Tensor-path coordinates (fused_tma_coords) of every tile of the lattices
// in `lats`, as the single pass uses them with one tensor map over a row
// space of `rows` rows of `pitch` elements whose stores are clipped at
// (store_x, store_y): 16-byte aligned x, rows and planes in range, and every
// store box inside its own lattice and inside the clip.  Layouts the runtime
// gives no tensor map (rows narrower than a load box, too few rows) are
// skipped, as the runtime falls back to row copies there.
template <int TX, int TY>
std::string check_tma_coords(const std::vector<LatDev>& lats, int es, int64_t pitch, int64_t rows,
                             int64_t store_x, int64_t store_y, int64_t& checked) {
    const int bw = TX + 2 * (16 / es);
    if (pitch < bw || rows < TY + 4) return "";
    for (const LatDev& L : lats)
        for (int y0 = 0; y0 < L.ny; y0 += TY)
            for (int x0 = 0; x0 < L.nx; x0 += TX)
                for (int par = 0; par < 2; ++par) {
                    const TmaCoords c = fused_tma_coords<TX, TY>(L, L.row0, par, x0, y0);
                    ++checked;
                    char buf[200];
                    std::snprintf(buf, sizeof buf,
                                  "tensor tile %dx%d of %dx%d at (%d,%d), row0 %d, es %d: ", TX, TY,
                                  L.nx, L.ny, x0, y0, L.row0, es);
                    if ((int64_t)c.lx * es % 16 || c.ly < 0 || (c.lz != 0 && c.lz != 9))
                        return std::string(buf) + "load box origin";
                    if (!c.store) continue;
                    if ((int64_t)c.sx * es % 16 || c.sy < 0 || (c.sz != 0 && c.sz != 9))
                        return std::string(buf) + "store box origin";
                    if (c.sx < L.gx || c.sx + TX > L.gx + L.nx || c.sy < L.row0 + GY ||
                        c.sy + TY > L.row0 + GY + L.ny)
                        return std::string(buf) + "store box outside the lattice";
                    if (c.sx + TX > store_x || c.sy + TY > store_y)
                        return std::string(buf) + "store box outside the clip";
                }
    return "";
}

template <int TX, int TY>
std::string check_tma_layouts(const int (*shapes)[2], int nshapes, int64_t& checked) {
    for (int f16 = 0; f16 < 2; ++f16) {
        const int es = f16 ? 2 : 4;
        std::vector<LatDev> all;
        for (int i = 0; i < nshapes; ++i) {
            lbm_lattice_desc d;
            lbm_desc_default(&d, shapes[i][0], shapes[i][1]);
            d.storage = f16 ? LBM_STORE_F16_DEV : LBM_STORE_F32_DEV;
            int64_t pc = 0, qc = 0;
            LatDev L = make_lat(d, i, pc, qc);
            all.push_back(L);
            // one lattice alone: row 0 of its own buffers, stores clipped
            // after its last interior column and row
            L.row0 = 0;
            const std::vector<LatDev> one{L};
            std::string e = check_tma_coords<TX, TY>(one, es, L.pitch, L.ny + 2 * GY,
                                                     L.gx + L.nx, GY + L.ny, checked);
            if (!e.empty()) return e;
        }
        // all of them stacked in one row space (a batch, or the server's arena)
        if (row_space_layout(all, es, 1e30) < 0) return "row space refused";
        int64_t rows = 0;
        for (const LatDev& L : all) rows += L.ny + 2 * GY;
        std::string e =
            check_tma_coords<TX, TY>(all, es, all[0].pitch, rows, all[0].pitch, rows, checked);
        if (!e.empty()) return e;
    }
    return "";
}

template <int ES>
std::string check_fused_shape(int tx, int ty, const LatDev& L, int par, int x0, int y0,
                              int64_t lo, int64_t hi) {
    if (tx == 64 && ty == 8) return check_fused_t<ES, 64, 8>(L, par, x0, y0, lo, hi);
    if (tx == 32 && ty == 16) return check_fused_t<ES, 32, 16>(L, par, x0, y0, lo, hi);
    if (tx == 64 && ty == 16) return check_fused_t<ES, 64, 16>(L, par, x0, y0, lo, hi);
    if (tx == 128 && ty == 8) return check_fused_t<ES, 128, 8>(L, par, x0, y0, lo, hi);
    return "unknown fused tile shape";
}

template <int ES, bool P>
std::string check_shape(int tx, int ty, const LatDev& L, int par, int x0, int y0, int64_t lo,
                        int64_t hi, int64_t plo, int64_t phi) {
    if (tx == 64 && ty == 8) return check_plan_t<ES, 64, 8, P>(L, par, x0, y0, lo, hi, plo, phi);
    if (tx == 64 && ty == 16) return check_plan_t<ES, 64, 16, P>(L, par, x0, y0, lo, hi, plo, phi);
    if (tx == 128 && ty == 4) return check_plan_t<ES, 128, 4, P>(L, par, x0, y0, lo, hi, plo, phi);
    if (tx == 128 && ty == 8) return check_plan_t<ES, 128, 8, P>(L, par, x0, y0, lo, hi, plo, phi);
    if (tx == 32 && ty == 16) return check_plan_t<ES, 32, 16, P>(L, par, x0, y0, lo, hi, plo, phi);
    return "unknown tile shape";
}

std::string check_tile_plan(int f16, int tx, int ty, bool with_psi, const LatDev& L, int par,
                            int x0, int y0, int64_t lo, int64_t hi, int64_t plo, int64_t phi) {
    if (f16)
        return with_psi ? check_shape<2, true>(tx, ty, L, par, x0, y0, lo, hi, plo, phi)
                        : check_shape<2, false>(tx, ty, L, par, x0, y0, lo, hi, plo, phi);
    return with_psi ? check_shape<4, true>(tx, ty, L, par, x0, y0, lo, hi, plo, phi)
                    : check_shape<4, false>(tx, ty, L, par, x0, y0, lo, hi, plo, phi);
}

// No exception crosses the C ABI: an allocation failure inside an entry point
// returns LBM_ERR_OOM, anything else LBM_ERR_STATE.
template <class F>
int guarded(F&& f) noexcept {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return LBM_ERR_OOM;
    } catch (...) {
        return LBM_ERR_STATE;
    }
}

}  // namespace

// ================================================================== C ABI
extern "C" {

void lbm_desc_default(lbm_lattice_desc* d, int32_t nx, int32_t ny) {
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->nx = nx;
    d->ny = ny;
    d->tau = 1.0;
    d->G = -1.0;
    d->eps = 1.73;
    d->sigma = 1.0;
    d->T = 0.8;
    d->eos_a = 3.852462257;
    d->eos_b = 0.1304438842;
    d->eos_c = 2.785855166;
    d->eos_k = 0.01;
    d->rho0 = -1.0;  // automatic: the smallest density handed to lbm_init
    d->storage = LBM_STORE_F32_DEV;
    d->eos_precision = LBM_EOS_DF;
    d->m2_trace_variant = 0;
    d->collision = LBM_COLL_BGK;
    for (int i = 0; i < 9; ++i) d->mrt_rates[i] = i < 7 ? 1.0 : 1.0 / d->tau;
}

const char* lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_PENDING: return "pending";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_OOM: return "out of memory";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_NUMERIC: return "psi undefined (rho <= 0, b rho >= 1 or negative radicand)";
        case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
        case LBM_ERR_STATE: return "call not valid in this state";
        case LBM_ERR_UNKNOWN_TICKET: return "unknown ticket";
        case LBM_ERR_CAPACITY: return "request exceeds server capacity";
        default: return "unknown status";
    }
}

const char* lbm_last_error(lbm_handle* h) { return h ? h->err.c_str() : ""; }

static int lbm_create_body(const lbm_lattice_desc* descs, int32_t n, const lbm_runtime_opts* opts,
               lbm_handle** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!descs || n < 1) return LBM_ERR_ARG;
    std::string why;
    for (int i = 0; i < n; ++i) {
        int rc = validate_desc(descs[i], why);
        if (rc) return rc;
        if (descs[i].storage != descs[0].storage || descs[i].eos_precision != descs[0].eos_precision ||
            descs[i].collision != descs[0].collision ||
            descs[i].m2_trace_variant != descs[0].m2_trace_variant)
            return LBM_ERR_ARG;
    }
    if (opts && (opts->alloc == nullptr) != (opts->free == nullptr)) return LBM_ERR_ARG;
    if (opts && (opts->tile_x < 0 || opts->tile_y < 0 || opts->grid_ctas < 0)) return LBM_ERR_ARG;
    const int variant = opts ? opts->kernel_variant : LBM_KERNEL_AUTO;
    if (variant != LBM_KERNEL_AUTO && variant != LBM_KERNEL_TMA && variant != LBM_KERNEL_PLAIN)
        return LBM_ERR_ARG;
    // per-pass defaults (measured on GB300): psi pass with plain loads, the
    // collision pass through the TMA pipeline with 128 x 4 tiles
    PassCfg cfg[2];
    for (int q = 0; q < 2; ++q)
        cfg[q] = PassCfg{kPassDefaults[q].variant, kPassDefaults[q].tx, kPassDefaults[q].ty, 0,
                         kPassDefaults[q].spt};
    if (opts && opts->schedule != LBM_SCHED_AUTO && opts->schedule != LBM_SCHED_TWO_PASS &&
        opts->schedule != LBM_SCHED_FUSED)
        return LBM_ERR_ARG;
    // LBM_SCHED_AUTO: the single pass, unless TMA tiles were asked for in a
    // shape that only the two-pass kernels have
    int schedule = (opts && opts->schedule != LBM_SCHED_AUTO) ? opts->schedule : LBM_SCHED_FUSED;
    if (!(opts && opts->schedule != LBM_SCHED_AUTO) && variant == LBM_KERNEL_TMA && opts &&
        (opts->tile_x || opts->tile_y) &&
        !fused_tma_shape_supported(opts->tile_x ? opts->tile_x : 64, opts->tile_y ? opts->tile_y : 8))
        schedule = LBM_SCHED_TWO_PASS;
    const bool fused = schedule == LBM_SCHED_FUSED;
    if (variant == LBM_KERNEL_TMA)
        for (auto& c : cfg) c = PassCfg{variant, 64, 8, 0, 1};
    if (opts && (opts->tile_x || opts->tile_y)) {
        for (int q = 0; q < 2; ++q) {
            PassCfg& c = cfg[q];
            c.tx = opts->tile_x ? opts->tile_x : 64;
            c.ty = opts->tile_y ? opts->tile_y : 8;
            c.spt = opts->sites_per_thread ? opts->sites_per_thread : 1;
            if (!shape_ok(c.variant, c.tx, c.ty, c.spt, fused && q == 1)) return LBM_ERR_ARG;
        }
    }
    if (!fused && descs[0].collision == LBM_COLL_MRT && variant == LBM_KERNEL_TMA)
        return LBM_ERR_ARG;  // the two-pass MRT collision exists as a plain-load kernel only

    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ERR_OOM;
    if (opts) h->opts = *opts;
    h->desc.assign(descs, descs + n);
    h->storage = descs[0].storage;
    h->f16 = h->storage == LBM_STORE_F16_DEV;
    h->schedule = schedule;
    h->eos = descs[0].eos_precision;
    h->collision = descs[0].collision;
    h->graph_steps = (opts && opts->graph_steps != 0) ? opts->graph_steps : 32;
    if (h->graph_steps > 0 && (h->graph_steps & 1)) h->graph_steps += 1;

    auto fail = [&](int rc) {
        release(h);
        delete h;
        return rc;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(LBM_ERR_CUDA);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) !=
        cudaSuccess)
        return fail(LBM_ERR_CUDA);
    if (opts && opts->stream) {
        h->stream = (cudaStream_t)opts->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(LBM_ERR_CUDA);
        h->own_stream = true;
    }
    int64_t pc = 0, qc = 0;
    for (int i = 0; i < n; ++i) {
        h->lat.push_back(make_lat(descs[i], i, pc, qc));
        h->sites += (int64_t)descs[i].nx * descs[i].ny;
    }
    const size_t es = h->f16 ? 2 : 4;
    if (n == 1) {
        h->lat[0].row0 = 0;  // the lattice is the whole row space
    } else {
        // a batch in one row space (one tensor map for all lattices) unless the
        // common pitch costs more than 2.5x the memory of the compact layout
        const int64_t rs = row_space_layout(h->lat, (int)es, 2.5);
        if (rs > 0) pc = rs;
    }
    h->pop_bytes = (size_t)pc * es;
    h->psi_bytes = (size_t)qc * sizeof(float);
    h->pop = dev_alloc(h, h->pop_bytes);
    h->psi = (float*)dev_alloc(h, h->psi_bytes);
    h->lat_dev = (LatDev*)dev_alloc(h, n * sizeof(LatDev));
    h->status = (uint32_t*)dev_alloc(h, n * sizeof(uint32_t));
    h->partials = (double*)dev_alloc(h, (kMassPartials + 1) * sizeof(double));
    if (!h->pop || !h->psi || !h->lat_dev || !h->status || !h->partials)
        return fail(LBM_ERR_OOM);
    if (cudaMallocHost(&h->status_host, n * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&h->scan_host, sizeof(double)) != cudaSuccess)
        return fail(LBM_ERR_OOM);
    if (cudaEventCreateWithFlags(&h->status_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess)
        return fail(LBM_ERR_CUDA);
    for (cudaEvent_t& e : h->chunk_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(LBM_ERR_CUDA);
    if (cudaMemsetAsync(h->pop, 0, h->pop_bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->psi, 0, h->psi_bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->status, 0, n * sizeof(uint32_t), h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->lat_dev, h->lat.data(), n * sizeof(LatDev), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
        return fail(LBM_ERR_CUDA);
    // LBM_KERNEL_AUTO, single pass: the TMA kernel with 32 x 16 tiles wherever
    // the population arena can be one tensor (one lattice, or a batch in one
    // row space, rows at least a box wide); measured fastest on GB300
    if (fused && variant == LBM_KERNEL_AUTO && !(opts && (opts->tile_x || opts->tile_y))) {
        CUtensorMap probe[2];
        if (fused_tma_make_map(h->f16, 32, 16, h->lat.data(), n, h->pop, probe))
            cfg[1] = PassCfg{LBM_KERNEL_TMA, 32, 16, 0, 2};
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        TuneKey k{h->device, h->storage, h->eos, variant * 4 + h->schedule,
                  (int64_t)std::log2((double)h->sites), (int64_t)std::log2((double)n)};
        auto it = g_tune_cache.find(k);
        if (it != g_tune_cache.end() && !(opts && (opts->tile_x || opts->tile_y)))
            for (int q = 0; q < 2; ++q) cfg[q] = it->second.pass[q];
    }
    if (cfg[1].variant == LBM_KERNEL_TMA &&
        !shape_ok(LBM_KERNEL_TMA, cfg[1].tx, cfg[1].ty, 1, fused))
        cfg[1] = PassCfg{LBM_KERNEL_PLAIN, kPassDefaults[1].tx, kPassDefaults[1].ty, 0,
                         kPassDefaults[1].spt};
    if (!fused && h->collision == LBM_COLL_MRT && cfg[1].variant == LBM_KERNEL_TMA)
        cfg[1] = PassCfg{LBM_KERNEL_PLAIN, kPassDefaults[1].tx, kPassDefaults[1].ty, 0,
                         kPassDefaults[1].spt};
    for (int q = 0; q < 2; ++q) {
        h->pass[q].variant = cfg[q].variant;
        h->pass[q].spt = cfg[q].variant != LBM_KERNEL_TMA ? cfg[q].spt
                         : (fused && q == 1)              ? cfg[q].tx * cfg[q].ty / 256
                                                          : 1;
        int rc = build_tiles(h, q, cfg[q].tx, cfg[q].ty);
        if (rc) return fail(rc);
        default_grid(h, q);
        if (cfg[q].grid > 0) h->pass[q].grid = std::min(cfg[q].grid, h->pass[q].ntiles);
        if (opts && opts->grid_ctas) h->pass[q].grid = std::min(opts->grid_ctas, h->pass[q].ntiles);
    }
    h->tune_variant = variant;
    h->rec[0].name = "psi_pass";
    h->rec[1].name = h->schedule == LBM_SCHED_FUSED ? "fused_step" : "collide_stream";
    h->rec[0].bytes = (double)h->sites * (9.0 * es + 4.0);
    h->rec[1].bytes = (double)h->sites * (h->schedule == LBM_SCHED_FUSED ? 18.0 * es
                                                                        : 18.0 * es + 4.0);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(LBM_ERR_CUDA);
    *out = h;
    return LBM_OK;
}

int lbm_create(const lbm_lattice_desc* descs, int32_t n, const lbm_runtime_opts* opts,
               lbm_handle** out) {
    return guarded([&] { return lbm_create_body(descs, n, opts, out); });
}

static int lbm_init_body(lbm_handle* h, int32_t lattice, const double* rho, const double* ux,
             const double* uy) {
    if (!h || !rho || lattice < 0 || lattice >= (int)h->lat.size()) return LBM_ERR_ARG;
    LatDev& L = h->lat[lattice];
    const size_t n = (size_t)L.nx * L.ny;
    int rc = ensure_staging(h, n);
    if (rc) return rc;
    double* dr = h->staging;
    double* dx = h->staging + h->staging_elems;
    double* dy = h->staging + 2 * h->staging_elems;
    // the staged densities are scanned on the GPU (every one finite, and the
    // smallest); the staging buffers hold nothing else, and nothing reads
    // them unless the scan passes
    CK(h, cudaMemcpyAsync(dr, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (ux) CK(h, cudaMemcpyAsync(dx, ux, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (uy) CK(h, cudaMemcpyAsync(dy, uy, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, launch_scan(dr, (int64_t)n, h->partials, kMassPartials, h->partials + kMassPartials,
                      staging32(h), h->stream));
    h->launches += 2;
    CK(h, cudaMemcpyAsync(h->scan_host, h->partials + kMassPartials, sizeof(double),
                          cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const double mn = *h->scan_host;
    if (std::isnan(mn)) return LBM_ERR_ARG;  // a density that is not finite
    if (h->desc[lattice].storage != LBM_STORE_F32 && h->desc[lattice].rho0 < 0.0) {
        // automatic reference: the smallest density keeps the vapour deviations
        // small (best relative precision where rho is smallest) and the liquid
        // ones no larger than plain storage would hold
        const float r0 = auto_rho0_of_min(mn);
        if (r0 != L.rho0) drop_graph(h);  // captured launches may carry the lattice by value
        L.rho0 = r0;
        CK(h, cudaMemcpyAsync(h->lat_dev + lattice, &L, sizeof(LatDev), cudaMemcpyHostToDevice,
                              h->stream));
    }
    CK(h, launch_init(h->f16, L, h->pop, h->parity, dr, staging32(h), ux ? dx : nullptr,
                      uy ? dy : nullptr,
                      h->stream));
    h->launches += 1;
    CK(h, cudaMemsetAsync(h->status + lattice, 0, sizeof(uint32_t), h->stream));
    if (h->numeric_lattice == lattice) {
        h->numeric_lattice = -1;
        h->fault_bits = 0;
    }
    return LBM_OK;
}

int lbm_init(lbm_handle* h, int32_t lattice, const double* rho, const double* ux,
             const double* uy) {
    return guarded([&] { return lbm_init_body(h, lattice, rho, ux, uy); });
}

static int lbm_step_body(lbm_handle* h, int64_t nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_ARG;
    int rc = check_status_async(h);
    if (rc) return rc;
    int64_t left = nsteps;
    if (!h->prof && !h->starve && h->graph_steps > 0 && left >= h->graph_steps) {
        if (!h->graph[h->parity]) {
            rc = capture_graph(h);
            if (rc) return rc;
        }
        while (left >= h->graph_steps) {
            CK(h, cudaGraphLaunch(h->graph[h->parity], h->stream));
            h->launches += (h->schedule == LBM_SCHED_FUSED ? 1 : 2) * (int64_t)h->graph_steps;
            left -= h->graph_steps;  // graph_steps is even: parity unchanged
        }
    }
    for (; left > 0; --left) {
        rc = launch_step(h, h->parity);
        if (rc) return rc;
        h->parity ^= 1;
    }
    if (!h->status_pending) {
        CK(h, cudaMemcpyAsync(h->status_host, h->status, h->lat.size() * sizeof(uint32_t),
                              cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaEventRecord(h->status_ev, h->stream));
        h->status_pending = true;
    }
    return LBM_OK;
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
    return guarded([&] { return lbm_step_body(h, nsteps); });
}

static int lbm_sync_body(lbm_handle* h) {
    if (!h) return LBM_ERR_ARG;
    return sync_status(h);
}

int lbm_sync(lbm_handle* h) {
    return guarded([&] { return lbm_sync_body(h); });
}

static int lbm_status_detail_body(lbm_handle* h, int32_t* lattice) {
    if (!h || !lattice) return LBM_ERR_ARG;
    *lattice = h->numeric_lattice;
    return LBM_OK;
}

int lbm_status_detail(lbm_handle* h, int32_t* lattice) {
    return guarded([&] { return lbm_status_detail_body(h, lattice); });
}

static int lbm_moments_body(lbm_handle* h, int32_t lattice, double* rho, double* ux, double* uy,
                double* mass) {
    if (!h || lattice < 0 || lattice >= (int)h->lat.size()) return LBM_ERR_ARG;
    const LatDev& L = h->lat[lattice];
    const size_t n = (size_t)L.nx * L.ny;
    if (rho || ux || uy) {
        int rc = ensure_staging(h, n);
        if (rc) return rc;
        // velocities: psi of the current state for this lattice's tiles (the
        // force-shifted u needs the force); density alone needs neither
        if (ux || uy) {
            StepArgs a = step_args(h, h->parity, 0);
            a.tiles = h->pass[0].tiles + h->pass[0].begin[lattice];
            a.ntiles = h->pass[0].count[lattice];
            CK(h, launch_pass(h, 0, a, std::min(h->pass[0].grid, a.ntiles)));
            h->launches += 1;
        }
    }
    // The fields are computed in row chunks on the handle's stream; the side
    // stream copies each finished chunk to the caller while the next chunk
    // and the mass reduction run.  The handle's stream then waits for the
    // copies, so nothing later reuses the staging buffer before they are done.
    const int nchunk = (rho || ux || uy) ? (n >= ((size_t)1 << 22) ? 4 : 1) : 0;
    for (int c = 0; c < nchunk; ++c) {
        const int y0 = (int)((int64_t)L.ny * c / nchunk), y1 = (int)((int64_t)L.ny * (c + 1) / nchunk);
        const size_t off = (size_t)y0 * L.nx, cnt = (size_t)(y1 - y0) * L.nx;
        double* dr = h->staging;
        double* dx = h->staging + h->staging_elems;
        double* dy = h->staging + 2 * h->staging_elems;
        CK(h, launch_moments(h->f16, L, h->pop, h->parity, h->psi, dr, (ux || uy) ? dx : nullptr,
                             (ux || uy) ? dy : nullptr, y0, y1, h->stream));
        h->launches += 1;
        CK(h, cudaEventRecord(h->chunk_ev[c], h->stream));
        CK(h, cudaStreamWaitEvent(h->side, h->chunk_ev[c], 0));
        const size_t b = cnt * sizeof(double);
        if (rho) CK(h, cudaMemcpyAsync(rho + off, dr + off, b, cudaMemcpyDeviceToHost, h->side));
        if (ux) CK(h, cudaMemcpyAsync(ux + off, dx + off, b, cudaMemcpyDeviceToHost, h->side));
        if (uy) CK(h, cudaMemcpyAsync(uy + off, dy + off, b, cudaMemcpyDeviceToHost, h->side));
    }
    if (mass) {
        CK(h, launch_mass(h->f16, L, h->pop, h->parity, h->partials, kMassPartials,
                          h->partials + kMassPartials, h->stream));
        h->launches += 2;
        CK(h, cudaMemcpyAsync(mass, h->partials + kMassPartials, sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
    }
    if (nchunk) {
        CK(h, cudaEventRecord(h->chunk_ev[4], h->side));
        CK(h, cudaStreamWaitEvent(h->stream, h->chunk_ev[4], 0));
    }
    return sync_status(h);
}

int lbm_moments(lbm_handle* h, int32_t lattice, double* rho, double* ux, double* uy,
                double* mass) {
    return guarded([&] { return lbm_moments_body(h, lattice, rho, ux, uy, mass); });
}

static int lbm_mass_body(lbm_handle* h, int32_t lattice, double* mass) {
    if (!mass) return LBM_ERR_ARG;
    return lbm_moments(h, lattice, nullptr, nullptr, nullptr, mass);
}

int lbm_mass(lbm_handle* h, int32_t lattice, double* mass) {
    return guarded([&] { return lbm_mass_body(h, lattice, mass); });
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    release(h);
    delete h;
}

static int lbm_profile_body(lbm_handle* h, int32_t on) {
    if (!h) return LBM_ERR_ARG;
    h->prof = on != 0;
    return LBM_OK;
}

int lbm_profile(lbm_handle* h, int32_t on) {
    return guarded([&] { return lbm_profile_body(h, on); });
}

static int lbm_profile_read_body(lbm_handle* h, lbm_kernel_stat* out, int32_t max, int32_t* n) {
    if (!h || !n) return LBM_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 2; ++k) {
        ProfRec& r = h->rec[k];
        for (auto& pr : r.pending) {
            float ms = 0.f;
            CK(h, cudaEventElapsedTime(&ms, pr.first, pr.second));
            r.total_ms += ms;
            r.launches += 1;
        }
    }
    // return events to the pool: psi pairs own e0, step pairs own (e1, e2)
    for (auto& pr : h->rec[0].pending) h->ev_pool.push_back(pr.first);
    for (auto& pr : h->rec[1].pending) {
        h->ev_pool.push_back(pr.first);
        h->ev_pool.push_back(pr.second);
    }
    h->rec[0].pending.clear();
    h->rec[1].pending.clear();
    const int cnt = 2;
    for (int k = 0; k < cnt && k < max && out; ++k) {
        std::memset(&out[k], 0, sizeof(lbm_kernel_stat));
        std::snprintf(out[k].name, sizeof(out[k].name), "%s", h->rec[k].name.c_str());
        out[k].launches = h->rec[k].launches;
        out[k].total_ms = h->rec[k].total_ms;
        out[k].bytes_per_launch = h->rec[k].bytes;
    }
    *n = cnt;
    return LBM_OK;
}

int lbm_profile_read(lbm_handle* h, lbm_kernel_stat* out, int32_t max, int32_t* n) {
    return guarded([&] { return lbm_profile_read_body(h, out, max, n); });
}

int64_t lbm_launch_count(lbm_handle* h) { return h ? h->launches : 0; }

static int lbm_info_body(lbm_handle* h, lbm_info_t* out) {
    if (!h || !out) return LBM_ERR_ARG;
    out->sites = h->sites;
    out->device_bytes = h->device_bytes;
    out->tile_x = h->pass[1].tx;
    out->tile_y = h->pass[1].ty;
    out->n_tiles = h->pass[1].ntiles;
    out->grid_ctas = h->pass[1].grid;
    out->psi_tile_x = h->pass[0].tx;
    out->psi_tile_y = h->pass[0].ty;
    out->psi_n_tiles = h->pass[0].ntiles;
    out->psi_grid_ctas = h->pass[0].grid;
    out->psi_variant = h->pass[0].variant;
    out->collide_variant = h->pass[1].variant;
    out->schedule = h->schedule;
    out->n_lattices = (int32_t)h->lat.size();
    out->spt = h->pass[1].spt;
    out->psi_spt = h->pass[0].spt;
    out->tensor_map = h->has_tmap ? 1 : 0;
    return LBM_OK;
}

int lbm_info(lbm_handle* h, lbm_info_t* out) {
    return guarded([&] { return lbm_info_body(h, out); });
}

static int lbm_autotune_body(lbm_handle* h, int32_t repeats) {
    if (!h || repeats < 1) return LBM_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    static const int shapes_tma[][2] = {{64, 8}, {64, 16}, {128, 4}, {128, 8}, {32, 16}};
    static const int shapes_fused_tma[][2] = {{64, 8}, {32, 16}, {64, 16}, {128, 8}};
    // plain: tile width, tile height, sites per thread
    static const int shapes_plain[][3] = {{32, 4, 1}, {32, 8, 1}, {64, 2, 1}, {64, 4, 1},
                                          {128, 2, 1}, {32, 8, 2}, {32, 16, 2}, {64, 4, 2},
                                          {64, 8, 2}, {128, 4, 2}, {32, 16, 4}, {64, 8, 4},
                                          {32, 32, 4}};
    cudaEvent_t ea = nullptr, eb = nullptr;
    CK(h, cudaEventCreate(&ea));
    CK(h, cudaEventCreate(&eb));
    const bool was_prof = h->prof;
    h->prof = false;
    const int64_t launches0 = h->launches;
    int rc = LBM_OK;
    TuneVal best_cfg{};
    // Each pass is tuned on its own.  Trial launches read population buffer
    // `parity` and write psi or the other buffer only, so repeating them
    // leaves the state unchanged; the collision trials run on the psi of
    // the current state, computed first.
    for (int k = 0; k < 2 && rc == LBM_OK; ++k) {
        std::vector<PassCfg> cand;
        const bool fused = k == 1 && h->schedule == LBM_SCHED_FUSED;
        const bool allow_tma = h->tune_variant != LBM_KERNEL_PLAIN &&
                               !(k == 1 && !fused && h->collision == LBM_COLL_MRT);
        const bool allow_plain = h->tune_variant != LBM_KERNEL_TMA;
        if (allow_tma && fused)
            for (const auto& c : shapes_fused_tma)
                cand.push_back({LBM_KERNEL_TMA, c[0], c[1], 0, c[0] * c[1] / 256});
        else if (allow_tma)
            for (const auto& c : shapes_tma) cand.push_back({LBM_KERNEL_TMA, c[0], c[1], 0, 1});
        if (allow_plain)
            for (const auto& c : shapes_plain)
                cand.push_back({LBM_KERNEL_PLAIN, c[0], c[1], 0, c[2]});
        float best = 1e30f;
        PassCfg bc{h->pass[k].variant, h->pass[k].tx, h->pass[k].ty, h->pass[k].grid,
                   h->pass[k].spt};
        for (const auto& c : cand) {
            h->pass[k].variant = c.variant;
            h->pass[k].spt = c.spt;
            rc = build_tiles(h, k, c.tx, c.ty);
            if (rc) break;
            default_grid(h, k);
            const int g0 = h->pass[k].grid;
            for (int mode = 0; mode < 2 && rc == LBM_OK; ++mode) {
                const int grid = mode == 0 ? g0 : h->pass[k].ntiles;  // persistent vs one CTA per tile
                const StepArgs a = step_args(h, h->parity, k);
                if (k == 1 && h->schedule != LBM_SCHED_FUSED) {
                    cudaError_t e = launch_pass(h, 0, step_args(h, h->parity, 0), h->pass[0].grid);
                    if (e != cudaSuccess) { rc = cuda_fail(h, e, "autotune psi"); break; }
                }
                cudaError_t e = launch_pass(h, k, a, grid);  // warm-up
                if (e != cudaSuccess) { rc = cuda_fail(h, e, "autotune"); break; }
                cudaEventRecord(ea, h->stream);
                for (int r = 0; r < repeats && e == cudaSuccess; ++r) e = launch_pass(h, k, a, grid);
                cudaEventRecord(eb, h->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(eb);
                if (e != cudaSuccess) { rc = cuda_fail(h, e, "autotune"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ea, eb);
                if (ms < best) {
                    best = ms;
                    bc = PassCfg{c.variant, c.tx, c.ty, grid, c.spt};
                }
            }
        }
        if (rc) break;
        h->pass[k].variant = bc.variant;
        h->pass[k].spt = bc.spt;
        rc = build_tiles(h, k, bc.tx, bc.ty);
        h->pass[k].grid = bc.grid;
        best_cfg.pass[k] = bc;
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    h->launches = launches0;
    h->prof = was_prof;
    if (rc) return rc;
    rc = sync_status(h);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneKey key{h->device, h->storage, h->eos, h->tune_variant * 4 + h->schedule,
                (int64_t)std::log2((double)h->sites), (int64_t)std::log2((double)h->lat.size())};
    g_tune_cache[key] = best_cfg;
    return LBM_OK;
}

int lbm_autotune(lbm_handle* h, int32_t repeats) {
    return guarded([&] { return lbm_autotune_body(h, repeats); });
}

static int lbm_inject_copy_timeout_body(lbm_handle* h, int32_t tile) {
    if (!h) return LBM_ERR_ARG;
    const Pass& P = h->pass[1];
    if (h->schedule != LBM_SCHED_FUSED || P.variant != LBM_KERNEL_TMA || tile < 0 ||
        tile >= P.ntiles)
        return LBM_ERR_ARG;
    h->starve = tile + 1;  // the next launch of the single pass; no graph replays it
    return LBM_OK;
}

int lbm_inject_copy_timeout(lbm_handle* h, int32_t tile) {
    return guarded([&] { return lbm_inject_copy_timeout_body(h, tile); });
}

static int lbm_selfcheck_arith_body(const float* x, int64_t n, float* rcp, float* sq) {
    if (!x || !rcp || !sq || n < 1 || n > ((int64_t)1 << 24)) return LBM_ERR_ARG;
    float* d = nullptr;
    uint32_t* flag = nullptr;
    const size_t bytes = (size_t)n * sizeof(float);
    if (cudaMalloc(&d, 3 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    if (cudaMalloc(&flag, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d);
        return LBM_ERR_OOM;
    }
    uint32_t mismatch = 0;
    cudaError_t e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(flag, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = launch_arith_check(d, n, d + n, d + 2 * n, flag, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(rcp, d + n, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(sq, d + 2 * n, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&mismatch, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    cudaFree(flag);
    cudaFree(d);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    return mismatch ? LBM_ERR_STATE : LBM_OK;
}

int lbm_selfcheck_arith(const float* x, int64_t n, float* rcp, float* sq) {
    return guarded([&] { return lbm_selfcheck_arith_body(x, n, rcp, sq); });
}

static int lbm_selfcheck_psi_body(const lbm_lattice_desc* d, const float* rho, int64_t n,
                                  float* psi, double* radicand) {
    if (!d || !rho || !psi || !radicand || n < 1 || n > ((int64_t)1 << 24)) return LBM_ERR_ARG;
    std::string why;
    if (validate_desc(*d, why) != LBM_OK) return LBM_ERR_ARG;
    const LatDev L = lat_layout(*d, 0);
    const size_t fb = (size_t)n * sizeof(float), db = (size_t)n * sizeof(double);
    char* buf = nullptr;
    if (cudaMalloc(&buf, 2 * fb + db + 2 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    float* dr = reinterpret_cast<float*>(buf);
    float* dp = dr + n;
    double* dq = reinterpret_cast<double*>(buf + 2 * fb);  // 2 fb is a multiple of 8
    uint32_t* flags = reinterpret_cast<uint32_t*>(buf + 2 * fb + db);
    uint32_t fl[2] = {0, 0};
    cudaError_t e = cudaMemcpy(dr, rho, fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(flags, 0, 2 * sizeof(uint32_t));
    if (e == cudaSuccess) e = launch_eos_check(d->eos_precision, L, dr, n, dp, dq, flags, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(psi, dp, fb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(radicand, dq, db, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(fl, flags, sizeof fl, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    return fl[0] ? LBM_ERR_STATE : LBM_OK;
}

int lbm_selfcheck_psi(const lbm_lattice_desc* d, const float* rho, int64_t n, float* psi,
                      double* radicand) {
    return guarded([&] { return lbm_selfcheck_psi_body(d, rho, n, psi, radicand); });
}

static int lbm_selfcheck_body(char* report, int32_t report_len) {
    std::string msg;
    const int shapes[][2] = {{2, 2},   {3, 5},   {4, 4},    {7, 5},   {31, 33}, {32, 32},
                             {64, 3},  {65, 9},  {100, 37}, {127, 129}, {128, 8}, {200, 120},
                             {257, 63}, {512, 17}, {1000, 3}};
    const int tiles[][2] = {{64, 8}, {64, 16}, {128, 4}, {128, 8}, {32, 16}};
    int64_t checked = 0;
    for (int f16 = 0; f16 < 2 && msg.empty(); ++f16) {
        for (const auto& tt : tiles) {
            for (int wp = 0; wp < 2 && msg.empty(); ++wp) {
                // lay out all shapes in one arena, as a batch handle would
                int64_t pc = 0, qc = 0;
                std::vector<LatDev> lats;
                int idx = 0;
                for (const auto& sh : shapes) {
                    lbm_lattice_desc d;
                    lbm_desc_default(&d, sh[0], sh[1]);
                    d.storage = f16 ? LBM_STORE_F16_DEV : LBM_STORE_F32_DEV;
                    lats.push_back(make_lat(d, idx++, pc, qc));
                }
                const int es = f16 ? 2 : 4;
                for (const LatDev& L : lats) {
                    const int64_t lo = L.off_f[0] * es, hi = (L.off_f[1] + 9 * L.plane) * es;
                    const int64_t plo = L.off_psi * 4,
                                  phi = (L.off_psi + (int64_t)L.pitch_psi * (L.ny + 2 * GY)) * 4;
                    for (int y0 = 0; y0 < L.ny; y0 += tt[1])
                        for (int x0 = 0; x0 < L.nx; x0 += tt[0])
                            for (int par = 0; par < 2; ++par) {
                                std::string e = check_tile_plan(f16, tt[0], tt[1], wp != 0, L, par,
                                                                x0, y0, lo, hi, plo, phi);
                                ++checked;
                                if (!e.empty()) {
                                    msg = e;
                                    goto done;
                                }
                            }
                }
            }
        }
    }
    {
        // the single-pass step's plans
        const int ftiles[][2] = {{64, 8}, {32, 16}, {64, 16}, {128, 8}};
        for (int f16 = 0; f16 < 2 && msg.empty(); ++f16)
            for (const auto& tt : ftiles) {
                int64_t pc = 0, qc = 0;
                std::vector<LatDev> lats;
                int idx = 0;
                for (const auto& sh : shapes) {
                    lbm_lattice_desc d;
                    lbm_desc_default(&d, sh[0], sh[1]);
                    d.storage = f16 ? LBM_STORE_F16_DEV : LBM_STORE_F32_DEV;
                    lats.push_back(make_lat(d, idx++, pc, qc));
                }
                const int es = f16 ? 2 : 4;
                for (const LatDev& L : lats) {
                    const int64_t lo = L.off_f[0] * es, hi = (L.off_f[1] + 9 * L.plane) * es;
                    for (int y0 = 0; y0 < L.ny; y0 += tt[1])
                        for (int x0 = 0; x0 < L.nx; x0 += tt[0])
                            for (int par = 0; par < 2; ++par) {
                                std::string e =
                                    f16 ? check_fused_shape<2>(tt[0], tt[1], L, par, x0, y0, lo, hi)
                                        : check_fused_shape<4>(tt[0], tt[1], L, par, x0, y0, lo, hi);
                                ++checked;
                                if (!e.empty()) {
                                    msg = e;
                                    goto done;
                                }
                            }
                }
            }
    }
    if (msg.empty()) {
        // the single pass's tensor coordinates, one lattice and row spaces
        const int n = (int)(sizeof(shapes) / sizeof(shapes[0]));
        msg = check_tma_layouts<64, 8>(shapes, n, checked);
        if (msg.empty()) msg = check_tma_layouts<32, 16>(shapes, n, checked);
        if (msg.empty()) msg = check_tma_layouts<64, 16>(shapes, n, checked);
        if (msg.empty()) msg = check_tma_layouts<128, 8>(shapes, n, checked);
    }
done:
    if (msg.empty()) msg = "ok: " + std::to_string(checked) + " tile plans checked";
    if (report && report_len > 0) std::snprintf(report, (size_t)report_len, "%s", msg.c_str());
    return msg.rfind("ok:", 0) == 0 ? LBM_OK : LBM_ERR_STATE;
}

int lbm_selfcheck(char* report, int32_t report_len) {
    return guarded([&] { return lbm_selfcheck_body(report, report_len); });
}

}  // extern "C"
