// lbm_server.cu -- continuous-batching server of the C ABI (lbm_server_*,
// lbm_submit, lbm_poll): many independent lattices resident in one device
// arena, stepped together by the same two passes as a batch handle.
//
// One worker thread owns the GPU work.  Its loop:
//   1. admit queued requests (first come first served, skipping those that
//      do not fit yet) while a slot and arena space are free; initialise
//      each at equilibrium in the current population buffer;
//   2. if the resident set changed, rebuild the lattice table and both tile
//      lists (lattice-major, so each lattice's tiles are one range);
//   3. run k = min(chunk_steps, fewest steps left) steps for every resident
//      lattice: two launches per step over the whole tile list;
//   4. read the fault words; copy out the moments of lattices that finished
//      (psi pass over their tiles, moments kernel, device-to-host) and free
//      their space.
// All resident lattices share the buffer parity (each step flips it), so a
// newly admitted lattice is initialised into the buffer the next step reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pplbm.h"
#include "lbm_kernels.h"
#include "lbm_layout.h"

using namespace pplbm;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) in 256-byte units, coalescing on release.
class ArenaAlloc {
  public:
    void reset(size_t n) {
        free_.clear();
        if (n) free_[0] = n;
        in_use_ = 0;
    }
    bool alloc(size_t n, size_t* off) {
        n = (size_t)round_up((int64_t)n, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            in_use_ += n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (size_t)round_up((int64_t)n, 256);
        in_use_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t in_use() const { return in_use_; }

  private:
    std::map<size_t, size_t> free_;
    size_t in_use_ = 0;
};

enum { ST_QUEUED = 0, ST_RESIDENT = 1, ST_DONE = 2 };

struct Request {
    uint64_t ticket = 0;
    lbm_lattice_desc d{};
    std::vector<double> rho;  // initial field until admitted, then the result
    std::vector<double> ux, uy;
    int64_t nsteps = 0, remaining = 0;
    int state = ST_QUEUED;
    int status = LBM_OK;
    size_t pop_off = 0, psi_off = 0, pop_bytes = 0, psi_bytes = 0;
    LatDev L{};
    Clock::time_point t_submit, t_done;
};

struct PassState {
    int variant = LBM_KERNEL_PLAIN, tx = 64, ty = 4, spt = 2;
    int4* tiles = nullptr;
    size_t cap = 0;
    int ntiles = 0;
    std::vector<int> begin, count;
};

}  // namespace

struct lbm_server {
    lbm_server_opts o{};
    int device = 0, sm_count = 0, f16 = 0, es = 4;
    cudaStream_t stream = nullptr;
    void* arena = nullptr;
    double* staging = nullptr;  // rho, ux, uy of one request
    LatDev* lat_dev = nullptr;  // max_resident entries
    uint32_t* status = nullptr; // max_resident words
    uint32_t* status_host = nullptr;
    PassState pass[2];
    ArenaAlloc alloc;
    int parity = 0;
    // shared with the API threads
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request> reqs;
    std::vector<uint64_t> resident;
    uint64_t next_ticket = 1;
    bool stop = false;
    lbm_server_stats st{};
    std::thread worker;
};

namespace {

void free_server(lbm_server* S) {
    for (auto& P : S->pass)
        if (P.tiles) cudaFree(P.tiles);
    if (S->status_host) cudaFreeHost(S->status_host);
    if (S->status) cudaFree(S->status);
    if (S->lat_dev) cudaFree(S->lat_dev);
    if (S->staging) cudaFree(S->staging);
    if (S->arena) cudaFree(S->arena);
    if (S->stream) cudaStreamDestroy(S->stream);
}

int pass_grid(lbm_server* S, int k) {
    const PassState& P = S->pass[k];
    int occ;
    if (P.variant == LBM_KERNEL_TMA)
        occ = k == 0 ? occupancy_psi_tma(S->f16, S->o.eos_precision, P.tx, P.ty)
                     : occupancy_collide_tma(S->f16, P.tx, P.ty);
    else
        occ = k == 0 ? occupancy_psi(S->f16, S->o.eos_precision, P.spt, P.tx * (P.ty / P.spt))
                     : occupancy_collide(S->f16, P.spt, P.tx * (P.ty / P.spt),
                                         (size_t)(P.tx + 2) * (P.ty + 2) * sizeof(float));
    return std::max(1, std::min(P.ntiles, S->sm_count * occ));
}

cudaError_t launch(lbm_server* S, int k, const StepArgs& a, int grid) {
    const PassState& P = S->pass[k];
    const dim3 block(P.tx, P.ty / P.spt);
    if (k == 0)
        return P.variant == LBM_KERNEL_TMA
                   ? launch_psi_tma(S->f16, S->o.eos_precision, P.tx, P.ty, a, grid, S->stream)
                   : launch_psi(S->f16, S->o.eos_precision, P.spt, a, dim3(grid), block, S->stream);
    return P.variant == LBM_KERNEL_TMA
               ? launch_collide_tma(S->f16, P.tx, P.ty, a, grid, S->stream)
               : launch_collide(S->f16, P.spt, a, dim3(grid), block,
                                (size_t)(P.tx + 2) * (P.ty + 2) * sizeof(float), S->stream);
}

StepArgs args(lbm_server* S, int k) {
    StepArgs a;
    a.lats = S->lat_dev;
    a.tiles = S->pass[k].tiles;
    a.ntiles = S->pass[k].ntiles;
    a.pop = S->arena;
    a.psi = static_cast<float*>(S->arena);
    a.status = S->status;
    a.parity = S->parity;
    return a;
}

// Rebuild the lattice table and tile lists from the resident requests.
cudaError_t rebuild(lbm_server* S, std::vector<Request*>& res) {
    std::vector<LatDev> lats(res.size());
    for (size_t i = 0; i < res.size(); ++i) {
        res[i]->L.lattice = (int)i;
        lats[i] = res[i]->L;
    }
    cudaError_t e = cudaSuccess;
    if (!lats.empty())
        e = cudaMemcpyAsync(S->lat_dev, lats.data(), lats.size() * sizeof(LatDev),
                            cudaMemcpyHostToDevice, S->stream);
    if (e != cudaSuccess) return e;
    for (auto& P : S->pass) {
        std::vector<int4> t;
        P.begin.assign(res.size(), 0);
        P.count.assign(res.size(), 0);
        for (size_t l = 0; l < res.size(); ++l) {
            P.begin[l] = (int)t.size();
            for (int y0 = 0; y0 < lats[l].ny; y0 += P.ty)
                for (int x0 = 0; x0 < lats[l].nx; x0 += P.tx)
                    t.push_back(make_int4((int)l, x0, y0, 0));
            P.count[l] = (int)t.size() - P.begin[l];
        }
        const size_t bytes = t.size() * sizeof(int4);
        if (bytes > P.cap) {
            if (P.tiles) {
                cudaStreamSynchronize(S->stream);
                cudaFree(P.tiles);
            }
            P.tiles = nullptr;
            P.cap = 0;
            e = cudaMalloc(&P.tiles, std::max<size_t>(bytes * 2, 4096));
            if (e != cudaSuccess) return e;
            P.cap = std::max<size_t>(bytes * 2, 4096);
        }
        if (bytes) e = cudaMemcpyAsync(P.tiles, t.data(), bytes, cudaMemcpyHostToDevice, S->stream);
        if (e != cudaSuccess) return e;
        P.ntiles = (int)t.size();
    }
    // the host staging vectors go out of scope: finish the copies first
    return cudaStreamSynchronize(S->stream);
}

// Moments of resident lattice `l` (index in the current table) into R.
cudaError_t copy_out(lbm_server* S, Request& R, int l) {
    StepArgs a = args(S, 0);
    a.tiles = S->pass[0].tiles + S->pass[0].begin[l];
    a.ntiles = S->pass[0].count[l];
    cudaError_t e = launch(S, 0, a, std::min(pass_grid(S, 0), a.ntiles));
    if (e != cudaSuccess) return e;
    const size_t n = (size_t)R.L.nx * R.L.ny;
    double* dr = S->staging;
    double* dx = dr + S->o.max_request_sites;
    double* dy = dx + S->o.max_request_sites;
    e = launch_moments(S->f16, R.L, S->arena, S->parity, static_cast<float*>(S->arena), dr, dx,
                       dy, S->stream);
    if (e != cudaSuccess) return e;
    R.rho.resize(n);
    R.ux.resize(n);
    R.uy.resize(n);
    cudaMemcpyAsync(R.rho.data(), dr, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    cudaMemcpyAsync(R.ux.data(), dx, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    cudaMemcpyAsync(R.uy.data(), dy, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    return cudaStreamSynchronize(S->stream);
}

void fail_all(lbm_server* S, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& kv : S->reqs)
        if (kv.second.state != ST_DONE) {
            kv.second.state = ST_DONE;
            kv.second.status = status;
            kv.second.t_done = Clock::now();
            S->st.failed++;
        }
    S->queue.clear();
    S->resident.clear();
}

void worker_main(lbm_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> res;  // resident requests in table order (worker's view)
    bool changed = false;
    for (;;) {
        std::vector<Request*> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            if (res.empty() && S->queue.empty()) {
                S->cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            for (auto it = S->queue.begin(); it != S->queue.end();) {
                if ((int)(res.size() + admitted.size()) >= S->o.max_resident) break;
                Request& R = S->reqs[*it];
                size_t po = 0, qo = 0;
                if (S->alloc.alloc(R.pop_bytes, &po)) {
                    if (S->alloc.alloc(R.psi_bytes, &qo)) {
                        R.pop_off = po;
                        R.psi_off = qo;
                        R.state = ST_RESIDENT;
                        admitted.push_back(&R);
                        S->resident.push_back(R.ticket);
                        it = S->queue.erase(it);
                        continue;
                    }
                    S->alloc.release(po, R.pop_bytes);
                }
                ++it;  // does not fit yet: smaller requests behind it may
            }
            S->st.queued = (int)S->queue.size();
            S->st.arena_in_use = (int64_t)S->alloc.in_use();
        }
        const auto t0 = Clock::now();
        cudaError_t e = cudaSuccess;
        for (Request* R : admitted) {
            R->L.off_f[0] = (int64_t)(R->pop_off / S->es);
            R->L.off_f[1] = R->L.off_f[0] + 9 * R->L.plane;
            R->L.off_psi = (int64_t)(R->psi_off / 4);
            const size_t n = (size_t)R->L.nx * R->L.ny;
            if (R->d.storage != LBM_STORE_F32 && R->d.rho0 < 0.0)
                R->L.rho0 = auto_rho0(R->rho.data(), n);
            e = cudaMemcpyAsync(S->staging, R->rho.data(), n * sizeof(double),
                                cudaMemcpyHostToDevice, S->stream);
            if (e == cudaSuccess)
                e = launch_init(S->f16, R->L, S->arena, S->parity, S->staging, nullptr, nullptr,
                                S->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);  // staging reused next
            if (e != cudaSuccess) break;
            std::vector<double>().swap(R->rho);
            res.push_back(R);
            changed = true;
        }
        if (e == cudaSuccess && changed) {
            e = rebuild(S, res);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(S->status, 0, std::max<size_t>(res.size(), 1) * 4, S->stream);
            changed = false;
        }
        if (e != cudaSuccess) {
            fail_all(S, LBM_ERR_CUDA);
            res.clear();
            continue;
        }
        if (res.empty()) continue;
        int64_t k = S->o.chunk_steps;
        for (Request* R : res) k = std::min(k, R->remaining);
        const int g0 = pass_grid(S, 0), g1 = pass_grid(S, 1);
        for (int64_t s = 0; s < k && e == cudaSuccess; ++s) {
            e = launch(S, 0, args(S, 0), g0);
            if (e == cudaSuccess) e = launch(S, 1, args(S, 1), g1);
            S->parity ^= 1;
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->status_host, S->status, res.size() * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, S->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        if (e != cudaSuccess) {
            fail_all(S, LBM_ERR_CUDA);
            res.clear();
            continue;
        }
        int64_t done_sites = 0;
        std::vector<Request*> keep;
        for (size_t l = 0; l < res.size(); ++l) {
            Request* R = res[l];
            R->remaining -= k;
            done_sites += (int64_t)R->L.nx * R->L.ny * k;
            const uint32_t bits = S->status_host[l];
            if (R->remaining > 0 && !bits) {
                keep.push_back(R);
                continue;
            }
            int status = LBM_OK;
            if (bits & 2u) status = LBM_ERR_TIMEOUT;
            else if (bits) status = LBM_ERR_NUMERIC;
            if (status == LBM_OK && copy_out(S, *R, (int)l) != cudaSuccess) status = LBM_ERR_CUDA;
            std::lock_guard<std::mutex> lk(S->mu);
            R->status = status;
            R->state = ST_DONE;
            R->t_done = Clock::now();
            S->alloc.release(R->pop_off, R->pop_bytes);
            S->alloc.release(R->psi_off, R->psi_bytes);
            S->resident.erase(std::find(S->resident.begin(), S->resident.end(), R->ticket));
            if (status == LBM_OK) S->st.completed++;
            else S->st.failed++;
            changed = true;
        }
        res.swap(keep);
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.site_steps += done_sites;
        S->st.busy_s += std::chrono::duration<double>(Clock::now() - t0).count();
        S->st.resident = (int)res.size();
        S->st.arena_in_use = (int64_t)S->alloc.in_use();
    }
}

}  // namespace

extern "C" {

void lbm_server_opts_default(lbm_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->arena_bytes = (size_t)8 << 30;
    o->max_resident = 1024;
    o->chunk_steps = 100;
    o->max_request_sites = (int64_t)2048 * 2048;
    o->storage = LBM_STORE_F32_DEV;
    o->eos_precision = LBM_EOS_DF;
    o->kernel_variant = LBM_KERNEL_AUTO;
}

int lbm_server_create(const lbm_server_opts* opts, lbm_server** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_server_opts o;
    lbm_server_opts_default(&o);
    if (opts) {
        o = *opts;
        lbm_server_opts d;
        lbm_server_opts_default(&d);
        if (!o.arena_bytes) o.arena_bytes = d.arena_bytes;
        if (!o.max_resident) o.max_resident = d.max_resident;
        if (!o.chunk_steps) o.chunk_steps = d.chunk_steps;
        if (!o.max_request_sites) o.max_request_sites = d.max_request_sites;
    }
    if (o.max_resident < 1 || o.chunk_steps < 1 || o.max_request_sites < 4 ||
        o.storage < LBM_STORE_F32 || o.storage > LBM_STORE_F16_DEV ||
        o.eos_precision < LBM_EOS_F64 || o.eos_precision > LBM_EOS_F32)
        return LBM_ERR_ARG;
    lbm_server* S = new (std::nothrow) lbm_server();
    if (!S) return LBM_ERR_OOM;
    S->o = o;
    S->f16 = o.storage == LBM_STORE_F16_DEV;
    S->es = S->f16 ? 2 : 4;
    for (int k = 0; k < 2; ++k) {
        PassState& P = S->pass[k];
        P.variant = kPassDefaults[k].variant;
        P.tx = kPassDefaults[k].tx;
        P.ty = kPassDefaults[k].ty;
        P.spt = kPassDefaults[k].spt;
        if (o.kernel_variant == LBM_KERNEL_TMA) {
            P.variant = LBM_KERNEL_TMA;
            P.tx = 64;
            P.ty = 8;
            P.spt = 1;
        } else if (o.kernel_variant == LBM_KERNEL_PLAIN) {
            P.variant = LBM_KERNEL_PLAIN;
        }
        if (o.tile_x || o.tile_y) {
            P.tx = o.tile_x ? o.tile_x : 64;
            P.ty = o.tile_y ? o.tile_y : 8;
            P.spt = 1;
        }
        const bool ok = P.variant == LBM_KERNEL_TMA
                            ? tma_shape_supported(P.tx, P.ty)
                            : (P.tx % 32 == 0 && P.ty > 0 && P.tx * P.ty <= 512 * P.spt &&
                               P.ty % P.spt == 0);
        if (!ok) {
            delete S;
            return LBM_ERR_ARG;
        }
    }
    auto fail = [&](int rc) {
        free_server(S);
        delete S;
        return rc;
    };
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(LBM_ERR_CUDA);
    if (cudaMalloc(&S->arena, o.arena_bytes) != cudaSuccess ||
        cudaMalloc(&S->staging, 3 * (size_t)o.max_request_sites * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&S->lat_dev, (size_t)o.max_resident * sizeof(LatDev)) != cudaSuccess ||
        cudaMalloc(&S->status, (size_t)o.max_resident * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&S->status_host, (size_t)o.max_resident * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_OOM);
    }
    if (cudaMemset(S->arena, 0, o.arena_bytes) != cudaSuccess) return fail(LBM_ERR_CUDA);
    S->alloc.reset(o.arena_bytes);
    S->st.arena_bytes = (int64_t)o.arena_bytes;
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        return fail(LBM_ERR_OOM);
    }
    *out = S;
    return LBM_OK;
}

int lbm_submit(lbm_server* S, const lbm_lattice_desc* d, const double* rho, int64_t nsteps,
               uint64_t* ticket) {
    if (!S || !d || !rho || !ticket || nsteps < 1) return LBM_ERR_ARG;
    Request R;
    R.d = *d;
    R.d.storage = S->o.storage;
    R.d.eos_precision = S->o.eos_precision;
    std::string why;
    if (validate_desc(R.d, why) != LBM_OK) return LBM_ERR_ARG;
    const size_t n = (size_t)R.d.nx * R.d.ny;
    if ((int64_t)n > S->o.max_request_sites) return LBM_ERR_CAPACITY;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(rho[i])) return LBM_ERR_ARG;
    R.L = lat_layout(R.d, 0);
    R.pop_bytes = (size_t)lat_pop_elems(R.L) * S->es;
    R.psi_bytes = (size_t)lat_psi_elems(R.L) * 4;
    if ((size_t)round_up((int64_t)R.pop_bytes, 256) + (size_t)round_up((int64_t)R.psi_bytes, 256) >
        S->o.arena_bytes)
        return LBM_ERR_CAPACITY;
    R.rho.assign(rho, rho + n);
    R.nsteps = R.remaining = nsteps;
    R.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return LBM_ERR_STATE;
    R.ticket = S->next_ticket++;
    *ticket = R.ticket;
    S->queue.push_back(R.ticket);
    S->reqs.emplace(R.ticket, std::move(R));
    S->st.submitted++;
    S->st.queued = (int)S->queue.size();
    S->cv.notify_one();
    return LBM_OK;
}

int lbm_poll(lbm_server* S, uint64_t ticket, double* rho, double* ux, double* uy,
             double* latency_s) {
    if (!S) return LBM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return LBM_ERR_UNKNOWN_TICKET;
    Request& R = it->second;
    if (R.state != ST_DONE) return LBM_PENDING;
    const int status = R.status;
    if (status == LBM_OK) {
        const size_t n = R.rho.size();
        if (rho) std::memcpy(rho, R.rho.data(), n * sizeof(double));
        if (ux) std::memcpy(ux, R.ux.data(), n * sizeof(double));
        if (uy) std::memcpy(uy, R.uy.data(), n * sizeof(double));
    }
    if (latency_s) *latency_s = std::chrono::duration<double>(R.t_done - R.t_submit).count();
    S->reqs.erase(it);
    return status;
}

int lbm_server_get_stats(lbm_server* S, lbm_server_stats* out) {
    if (!S || !out) return LBM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaStreamSynchronize(S->stream);
    free_server(S);
    delete S;
}

}  // extern "C"
