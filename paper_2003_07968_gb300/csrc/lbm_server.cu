// lbm_server.cu -- continuous-batching server of the C ABI (lbm_server_*,
// lbm_submit, lbm_poll): many independent lattices resident in one device
// arena, stepped together by the same kernels as a batch handle.  The
// arena's population part is one row space: every lattice at the common
// pitch of the widest accepted request, its ny + 2 GY rows (allocated first
// fit) in each of 18 planes, so that one tensor map covers all resident
// lattices and the single pass runs on the TMA kernel.
//
// One worker thread owns the GPU work and keeps two chunks in flight; it
// only enqueues work and waits for the GPU, so that short chunks keep the
// GPU busy.  Large host copies happen elsewhere: lbm_submit copies a field
// into a pinned input slot on the caller's thread, and lbm_poll copies a
// result out of its pinned result slot.  Each turn of the loop:
//   1. finish the requests whose copy-out is done and release the input
//      slots whose upload is done;
//   2. admit queued requests (first come first served, skipping those that
//      do not fit yet) while a slot, arena space and the resident-site
//      target allow; their fields go from their pinned slots to the device
//      on the upload stream (overlapping the chunk in flight) and are
//      initialised at equilibrium on the main stream;
//   3. launch chunk n: update one of two alternating table sets (step
//      quotas; lattice table and tile lists only when the resident lattices
//      changed) through pinned mirrors, then one launch per step over the
//      tile list of every resident lattice.  Each lattice runs min(k, its
//      remaining steps), where k fills about chunk_ms of GPU time at the
//      rate measured on earlier chunks (at most chunk_steps).  The kernels
//      skip the tiles of a lattice whose quota is used up.  Quotas are known
//      on the host, so the lattices that finish in chunk n are known when it
//      is launched and are not part of chunk n + 1;
//   4. retire chunk n - 1 (which ran while the host did 1-3): read its fault
//      words and enqueue the copy-outs of the lattices that finished in it
//      (moments, plus a psi pass when velocities are kept, device to pinned
//      result slot, on the side stream while chunk n runs).  A request is
//      done, and its arena space free, once its copy-out has completed.
// A lattice whose fault bit shows up is dropped one chunk later than it
// faulted (its extra chunk computes garbage that nobody reads).  Every
// lattice still resident after a chunk has run all of its steps, so all
// resident lattices share the buffer parity; a lattice that stops early
// keeps its own final parity for the copy-out.  Bounding the resident sites
// keeps the GPU saturated without stretching every request's latency.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pplbm.h"
#include "lbm_kernels.h"
#include "lbm_host_scan.h"
#include "lbm_layout.h"

using namespace pplbm;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) in units of `granule`, coalescing on
// release (bytes of the psi arena; rows of the population row space).
class ArenaAlloc {
  public:
    void reset(size_t n, size_t granule = 256) {
        free_.clear();
        if (n) free_[0] = n;
        in_use_ = 0;
        granule_ = granule;
    }
    bool alloc(size_t n, size_t* off) {
        n = (size_t)round_up((int64_t)n, (int64_t)granule_);
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
        n = (size_t)round_up((int64_t)n, (int64_t)granule_);
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
    size_t granule_ = 256;
};

enum { ST_QUEUED = 0, ST_RESIDENT = 1, ST_DONE = 2 };
constexpr size_t kNoSlot = ~size_t(0);

struct Request {
    uint64_t ticket = 0;
    lbm_lattice_desc d{};
    std::vector<double> rho;  // initial field (no pinned slot) or result (no result slot)
    std::vector<double> ux, uy;
    // pinned slots: the initial field (from submit until its upload is done)
    // and the result (from its copy-out until it is polled), in doubles
    size_t in_off = kNoSlot, in_n = 0, out_off = kNoSlot, out_n = 0;
    int64_t nsteps = 0, remaining = 0;
    int state = ST_QUEUED;
    int status = LBM_OK;
    size_t row_off = 0, psi_off = 0, rows = 0, psi_bytes = 0;  // rows of the row space
    size_t stage_off = 0;  // doubles into the upload buffers while being admitted
    bool dropped = false;  // faulted: no further chunks, released once its last chunk is done
    LatDev L{};
    Clock::time_point t_submit, t_done;
};

struct PassState {
    int tx = 64, ty = 4, spt = 2;
};

// One set of device tables (lattice table, tile list per pass, quotas,
// fault words).  Two sets alternate between chunks so that the copy-out of
// lattices that finished in chunk n (on the side stream, with set n % 2)
// overlaps chunk n + 1 (main stream, the other set).
struct TableSet {
    LatDev* lat = nullptr;
    int* quota = nullptr;
    uint32_t* status = nullptr;
    int4* tiles[2] = {nullptr, nullptr};
    size_t cap[2] = {0, 0};
    int ntiles[2] = {0, 0};
    std::vector<int> begin[2], count[2];
    // tickets of the lattices (in table order) that the lattice table and
    // tile lists describe; a chunk over the same lattices only rewrites the
    // quotas.  Tickets, not addresses: a new request can occupy the memory of
    // one that was polled
    std::vector<uint64_t> members;
    // pinned mirrors of the tables, so that their uploads are asynchronous
    LatDev* lat_h = nullptr;
    int* quota_h = nullptr;
    int4* tiles_h[2] = {nullptr, nullptr};
    size_t hcap[2] = {0, 0};
};

// A finished request whose copy-out is in flight on the side stream.
struct Drain {
    Request* R;
    cudaEvent_t done;
};

}  // namespace

struct lbm_server {
    lbm_server_opts o{};
    int device = 0, sm_count = 0, f16 = 0, es = 4;
    int fused = 1;  // one launch per step (LBM_SCHED_FUSED)
    cudaStream_t stream = nullptr, side = nullptr, up = nullptr;
    cudaEvent_t chunk_end[2] = {nullptr, nullptr};  // per table set: its last chunk is done
    cudaEvent_t chunk_begin[2] = {nullptr, nullptr};  // ... and where its steps began (timing)
    cudaEvent_t up_done = nullptr;    // the last uploads have read their pinned slots
    cudaEvent_t init_done = nullptr;  // the last inits have read staging
    cudaEvent_t side_done[2] = {nullptr, nullptr};  // copy-outs reading a table set's tiles
    std::vector<cudaEvent_t> spare_events;          // for copy-outs, reused
    // device arena: the population row space (every resident lattice with the
    // common pitch, its ny + 2 GY rows in each of 18 planes), then psi
    void* arena = nullptr;
    float* psi_arena = nullptr;
    int64_t pitch = 0, plane = 0, row_cap = 0;  // of the row space (elements, rows)
    size_t pop_bytes = 0, psi_region = 0;
    bool tma = false;      // single pass on the TMA kernel (one tensor map for the arena)
    CUtensorMap tmap[2]{};  // loads, stores
    size_t up_cap = 0;            // doubles of the device staging buffer
    double* staging = nullptr;    // rho of the requests admitted in one turn (device)
    float* staging32 = nullptr;   // the same rounded to FP32, as lbm_init's init reads it
    double* in_host = nullptr;    // pinned slots of initial fields (in_alloc, doubles)
    double* out_host = nullptr;   // pinned slots of results (out_alloc, doubles)
    double* outbuf = nullptr;     // rho, ux, uy of one finished request (side stream)
    double* down_host = nullptr;  // ... pinned copy when no result slot is free
    uint32_t* status_host = nullptr;  // fault words of both table sets (pinned)
    PassState pass[2];
    TableSet set[2];
    ArenaAlloc rows_alloc, psi_alloc;
    ArenaAlloc in_alloc, out_alloc;  // under mu: submit and poll use them too
    int parity = 0;
    // shared with the API threads
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool dead = false;  // the worker ended on an exception
    lbm_server_stats st{};
    std::thread worker;
};

namespace {

// Device memory of the server: from the caller's allocator when opts give
// one (it must return 256-byte aligned memory), else cudaMalloc.
void* srv_alloc(lbm_server* S, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (S->o.alloc) {
        p = S->o.alloc(bytes, S->o.alloc_ctx);
        if (p && (reinterpret_cast<uintptr_t>(p) & 255u)) {
            S->o.free(p, bytes, S->o.alloc_ctx);
            p = nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void srv_free(lbm_server* S, void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (S->o.alloc)
        S->o.free(p, bytes, S->o.alloc_ctx);
    else
        cudaFree(p);
}

void free_server(lbm_server* S) {
    const size_t nmax = (size_t)S->o.max_request_sites, nres = (size_t)S->o.max_resident;
    for (auto& T : S->set) {
        for (int k = 0; k < 2; ++k) srv_free(S, T.tiles[k], T.cap[k]);
        for (auto& t : T.tiles_h)
            if (t) cudaFreeHost(t);
        srv_free(S, T.lat, nres * sizeof(LatDev));
        srv_free(S, T.quota, nres * sizeof(int));
        srv_free(S, T.status, nres * sizeof(uint32_t));
        if (T.lat_h) cudaFreeHost(T.lat_h);
        if (T.quota_h) cudaFreeHost(T.quota_h);
    }
    if (S->status_host) cudaFreeHost(S->status_host);
    if (S->down_host) cudaFreeHost(S->down_host);
    if (S->in_host) cudaFreeHost(S->in_host);
    if (S->out_host) cudaFreeHost(S->out_host);
    for (auto& e : S->spare_events) cudaEventDestroy(e);
    for (auto& e : S->side_done)
        if (e) cudaEventDestroy(e);
    srv_free(S, S->outbuf, 3 * nmax * sizeof(double));
    srv_free(S, S->staging, S->up_cap * sizeof(double));
    srv_free(S, S->staging32, S->up_cap * sizeof(float));
    srv_free(S, S->arena, S->o.arena_bytes);
    for (auto& e : S->chunk_end)
        if (e) cudaEventDestroy(e);
    for (auto& e : S->chunk_begin)
        if (e) cudaEventDestroy(e);
    if (S->up_done) cudaEventDestroy(S->up_done);
    if (S->init_done) cudaEventDestroy(S->init_done);
    if (S->up) cudaStreamDestroy(S->up);
    if (S->side) cudaStreamDestroy(S->side);
    if (S->stream) cudaStreamDestroy(S->stream);
}

size_t smem_of(const PassState& P) { return (size_t)(P.tx + 2) * (P.ty + 2) * sizeof(float); }

// Pass 0: psi pass (used by the copy-out; and by the two-pass schedule);
// pass 1: the collision pass, or the single-pass step when fused.
int pass_grid(lbm_server* S, int k, int ntiles) {
    const PassState& P = S->pass[k];
    const int thr = P.tx * (P.ty / P.spt);
    const int occ =
        k == 0   ? occupancy_psi(S->f16, S->o.eos_precision, P.spt, thr)
        : S->tma ? occupancy_fused_tma(S->f16, 0, S->o.eos_precision, P.tx, P.ty, true, false)
        : S->fused ? occupancy_fused(S->f16, 0, S->o.eos_precision, P.spt, thr, smem_of(P))
                   : occupancy_collide(S->f16, 0, P.spt, thr, smem_of(P));
    return std::max(1, std::min(ntiles, S->sm_count * occ));
}

cudaError_t launch(lbm_server* S, int k, const StepArgs& a, int grid, cudaStream_t st) {
    const PassState& P = S->pass[k];
    const dim3 block(P.tx, P.ty / P.spt);
    if (k == 0) return launch_psi(S->f16, S->o.eos_precision, P.spt, a, dim3(grid), block, st);
    if (S->tma)
        return launch_fused_tma(S->f16, 0, S->o.eos_precision, P.tx, P.ty, a, S->tmap, nullptr,
                                grid, st);
    if (S->fused)
        return launch_fused(S->f16, 0, S->o.eos_precision, P.spt, a, dim3(grid), block, smem_of(P),
                            st);
    return launch_collide(S->f16, 0, P.spt, a, dim3(grid), block, smem_of(P), st);
}

StepArgs args(lbm_server* S, const TableSet& T, int k, int parity) {
    StepArgs a{};
    a.lats = T.lat;
    a.tiles = T.tiles[k];
    a.ntiles = T.ntiles[k];
    a.pop = S->arena;
    a.psi = S->psi_arena;
    a.status = T.status;
    a.parity = parity;
    a.quota = T.quota;
    a.step = 0;
    return a;
}

// Fill table set T from the resident requests with their chunk quotas,
// through its pinned mirrors (the caller has waited for the set's previous
// chunk, so the mirrors' last uploads are done).
cudaError_t rebuild(lbm_server* S, TableSet& T, std::vector<Request*>& res,
                    const std::vector<int>& quota) {
    std::vector<uint64_t> members(res.size());
    for (size_t i = 0; i < res.size(); ++i) members[i] = res[i]->ticket;
    cudaError_t e = cudaSuccess;
    if (!res.empty()) {
        std::memcpy(T.quota_h, quota.data(), quota.size() * sizeof(int));
        e = cudaMemcpyAsync(T.quota, T.quota_h, quota.size() * sizeof(int),
                            cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(T.status, 0, res.size() * sizeof(uint32_t), S->stream);
    }
    // same lattices in the same order: lattice table and tile lists stand
    if (e != cudaSuccess || (!res.empty() && members == T.members)) return e;
    T.members.clear();
    for (size_t i = 0; i < res.size(); ++i) {
        res[i]->L.lattice = (int)i;
        T.lat_h[i] = res[i]->L;
    }
    if (!res.empty())
        e = cudaMemcpyAsync(T.lat, T.lat_h, res.size() * sizeof(LatDev), cudaMemcpyHostToDevice,
                            S->stream);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < 2; ++k) {
        const PassState& P = S->pass[k];
        size_t nt = 0;
        for (Request* R : res)
            nt += (size_t)((R->L.nx + P.tx - 1) / P.tx) * ((R->L.ny + P.ty - 1) / P.ty);
        const size_t bytes = nt * sizeof(int4);
        if (bytes > T.cap[k]) {
            if (T.tiles[k]) {
                cudaDeviceSynchronize();  // no kernel or copy-out still reads the old list
                srv_free(S, T.tiles[k], T.cap[k]);
            }
            T.tiles[k] = nullptr;
            T.cap[k] = 0;
            const size_t cap = std::max<size_t>(bytes * 2, 4096);
            T.tiles[k] = static_cast<int4*>(srv_alloc(S, cap));
            if (!T.tiles[k]) return cudaErrorMemoryAllocation;
            T.cap[k] = cap;
        }
        if (bytes > T.hcap[k]) {
            if (T.tiles_h[k]) cudaFreeHost(T.tiles_h[k]);
            T.tiles_h[k] = nullptr;
            T.hcap[k] = 0;
            e = cudaMallocHost(&T.tiles_h[k], T.cap[k]);
            if (e != cudaSuccess) return e;
            T.hcap[k] = T.cap[k];
        }
        int4* t = T.tiles_h[k];
        size_t m = 0;
        T.begin[k].assign(res.size(), 0);
        T.count[k].assign(res.size(), 0);
        for (size_t l = 0; l < res.size(); ++l) {
            T.begin[k][l] = (int)m;
            for (int y0 = 0; y0 < res[l]->L.ny; y0 += P.ty)
                for (int x0 = 0; x0 < res[l]->L.nx; x0 += P.tx) t[m++] = make_int4((int)l, x0, y0, 0);
            T.count[k][l] = (int)m - T.begin[k][l];
        }
        if (bytes)
            e = cudaMemcpyAsync(T.tiles[k], t, bytes, cudaMemcpyHostToDevice, S->stream);
        if (e != cudaSuccess) return e;
        T.ntiles[k] = (int)nt;
    }
    T.members = members;
    return cudaSuccess;
}

// Enqueue on the side stream the moments of lattice l of set T (final
// parity `par`) into the pinned host doubles at `host` (rho, then ux and uy
// with the server's with_velocity option): psi pass (velocities only: the
// force-shifted u needs psi), moments into the device buffer, device to
// host.  The side stream serialises the copy-outs over the one buffer.
cudaError_t enqueue_copy_out(lbm_server* S, const TableSet& T, const Request& R, int l, int par,
                             double* host) {
    const bool vel = S->o.with_velocity != 0;
    cudaError_t e = cudaSuccess;
    if (vel) {
        StepArgs a = args(S, T, 0, par);
        a.tiles = T.tiles[0] + T.begin[0][l];
        a.ntiles = T.count[0][l];
        a.quota = nullptr;
        e = launch(S, 0, a, pass_grid(S, 0, a.ntiles), S->side);
        if (e != cudaSuccess) return e;
    }
    const size_t n = (size_t)R.L.nx * R.L.ny;
    double* dr = S->outbuf;
    double* dx = dr + S->o.max_request_sites;
    double* dy = dx + S->o.max_request_sites;
    e = launch_moments(S->f16, R.L, S->arena, par, S->psi_arena, dr, vel ? dx : nullptr,
                       vel ? dy : nullptr, 0, R.L.ny, S->side);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host, dr, n * sizeof(double), cudaMemcpyDeviceToHost, S->side);
    if (e == cudaSuccess && vel)
        e = cudaMemcpyAsync(host + n, dx, n * sizeof(double), cudaMemcpyDeviceToHost, S->side);
    if (e == cudaSuccess && vel)
        e = cudaMemcpyAsync(host + 2 * n, dy, n * sizeof(double), cudaMemcpyDeviceToHost,
                            S->side);
    return e;
}

// When no result slot is free: the same copy-out through the one pinned
// buffer, waited for, into R's vectors.
cudaError_t copy_out_now(lbm_server* S, const TableSet& T, Request& R, int l, int par) {
    cudaError_t e = enqueue_copy_out(S, T, R, l, par, S->down_host);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->side);
    if (e != cudaSuccess) return e;
    const size_t n = (size_t)R.L.nx * R.L.ny;
    const double* h = S->down_host;
    R.rho.assign(h, h + n);
    if (S->o.with_velocity) {
        R.ux.assign(h + n, h + 2 * n);
        R.uy.assign(h + 2 * n, h + 3 * n);
    }
    return cudaSuccess;
}

cudaEvent_t take_event(lbm_server* S) {
    if (!S->spare_events.empty()) {
        cudaEvent_t e = S->spare_events.back();
        S->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
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
    S->st.queued = 0;
    S->st.resident = 0;
}

struct Finished {
    Request* R;
    int l, par, status;
};

// What the worker remembers of a chunk in flight until it retires it.
struct Chunk {
    bool live = false;
    std::vector<Request*> res;       // lattices of the chunk, in table order
    std::vector<int> quota;
    int p0 = 0;                      // buffer parity at its start
    std::vector<Finished> finished;  // ran their last steps in it
    std::vector<Request*> dropped;   // faulted earlier, still part of it: free once it is done
};

int64_t arena_in_use(const lbm_server* S) {
    return (int64_t)(S->rows_alloc.in_use() * (size_t)(18 * S->pitch * S->es) +
                     S->psi_alloc.in_use());
}

void finish(lbm_server* S, Request* R, int status) {
    std::lock_guard<std::mutex> lk(S->mu);
    R->status = status;
    R->state = ST_DONE;
    R->t_done = Clock::now();
    S->rows_alloc.release(R->row_off, R->rows);
    S->psi_alloc.release(R->psi_off, R->psi_bytes);
    if (status == LBM_OK)
        S->st.completed++;
    else
        S->st.failed++;
    S->st.arena_in_use = arena_in_use(S);
}

void worker_loop(lbm_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> res;  // resident and still to run (host view)
    int64_t res_sites = 0;      // sites of the resident lattices still running
    Chunk chunk[2];
    int64_t n = 0;              // chunks launched
    // site updates per second of the chunks so far (CUDA event timings); the
    // first chunks assume a modest rate, so they come out short
    double rate = 2e10;
    std::deque<Drain> drain;                       // copy-outs in flight, in order
    std::vector<std::pair<size_t, size_t>> in_pending;  // input slots being uploaded
    // finish the requests whose copy-out is done, release uploaded input slots
    auto settle = [&]() -> cudaError_t {
        while (!drain.empty()) {
            const cudaError_t q = cudaEventQuery(drain.front().done);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) return q;
            S->spare_events.push_back(drain.front().done);
            finish(S, drain.front().R, LBM_OK);
            drain.pop_front();
        }
        if (!in_pending.empty()) {
            const cudaError_t q = cudaEventQuery(S->up_done);
            if (q == cudaSuccess) {
                std::lock_guard<std::mutex> lk(S->mu);
                for (auto& sl : in_pending) S->in_alloc.release(sl.first, sl.second);
                in_pending.clear();
            } else if (q != cudaErrorNotReady) {
                return q;
            }
        }
        return cudaSuccess;
    };
    for (;;) {
        cudaError_t e = settle();
        // ------------------------------------------------------------ admission
        std::vector<Request*> admitted, to_stage;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            if (res.empty() && S->queue.empty() && !chunk[0].live && !chunk[1].live) {
                if (drain.empty() && in_pending.empty()) {
                    S->cv.wait_for(lk, std::chrono::milliseconds(20));
                    continue;
                }
                // only copy-outs or uploads in flight: wait for the oldest
                lk.unlock();
                if (!drain.empty())
                    cudaEventSynchronize(drain.front().done);
                else
                    cudaEventSynchronize(S->up_done);
                continue;
            }
            // first come first served, skipping requests that do not fit yet,
            // while slots, arena space, the resident-site target and the
            // staging buffer allow (one request is always admitted into an
            // idle GPU); a field without a pinned slot gets one here
            size_t up_used = 0;
            for (auto it = S->queue.begin(); it != S->queue.end();) {
                if ((int)(res.size() + admitted.size()) >= S->o.max_resident) break;
                Request& R = S->reqs[*it];
                const int64_t ns = (int64_t)R.L.nx * R.L.ny;
                const size_t nup = (size_t)round_up(ns, 32);
                if (res_sites + ns > S->o.target_resident_sites && (res_sites > 0 || !admitted.empty()))
                    break;
                if (up_used + nup > S->up_cap) break;
                const bool stage = R.in_off == kNoSlot;
                size_t io = 0;
                if (stage && !S->in_alloc.alloc((size_t)ns, &io)) {
                    ++it;
                    continue;
                }
                size_t po = 0, qo = 0;
                if (S->rows_alloc.alloc(R.rows, &po)) {
                    if (S->psi_alloc.alloc(R.psi_bytes, &qo)) {
                        if (stage) {
                            R.in_off = io;
                            R.in_n = (size_t)ns;
                            to_stage.push_back(&R);
                        }
                        R.row_off = po;
                        R.psi_off = qo;
                        R.stage_off = up_used;
                        up_used += nup;
                        R.state = ST_RESIDENT;
                        admitted.push_back(&R);
                        res_sites += ns;
                        it = S->queue.erase(it);
                        continue;
                    }
                    S->rows_alloc.release(po, R.rows);
                }
                if (stage) S->in_alloc.release(io, (size_t)ns);
                ++it;
            }
            S->st.queued = (int)S->queue.size();
            S->st.arena_in_use = arena_in_use(S);
        }
        int64_t launches = 0;
        if (e == cudaSuccess && !admitted.empty()) {
            // fields that arrived while the pinned slots were full
            for (Request* R : to_stage) {
                std::memcpy(S->in_host + R->in_off, R->rho.data(), R->in_n * sizeof(double));
                std::vector<double>().swap(R->rho);
            }
            // the previous inits have read the staging buffer
            e = cudaStreamWaitEvent(S->up, S->init_done, 0);
            for (Request* R : admitted) {
                if (e != cudaSuccess) break;
                e = cudaMemcpyAsync(S->staging + R->stage_off, S->in_host + R->in_off,
                                    R->in_n * sizeof(double), cudaMemcpyHostToDevice, S->up);
                in_pending.emplace_back(R->in_off, R->in_n);
                R->in_off = kNoSlot;  // the slot now belongs to in_pending
            }
            if (e == cudaSuccess) e = cudaEventRecord(S->up_done, S->up);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(S->stream, S->up_done, 0);
            for (Request* R : admitted) {
                if (e != cudaSuccess) break;
                R->L.pitch = (int32_t)S->pitch;
                R->L.plane = S->plane;
                R->L.row0 = (int32_t)R->row_off;
                R->L.off_f[0] = (int64_t)R->row_off * S->pitch;
                R->L.off_f[1] = R->L.off_f[0] + 9 * S->plane;
                R->L.off_psi = (int64_t)(R->psi_off / 4);
                // the same init arithmetic as lbm_init: neighbours' densities
                // from an FP32 copy of the field
                e = launch_to_f32(S->staging + R->stage_off, (int64_t)R->L.nx * R->L.ny,
                                  S->staging32 + R->stage_off, S->stream);
                if (e == cudaSuccess)
                    e = launch_init(S->f16, R->L, S->arena, S->parity, S->staging + R->stage_off,
                                    S->staging32 + R->stage_off, nullptr, nullptr, S->stream);
                launches += 2;
                res.push_back(R);
            }
            if (e == cudaSuccess) e = cudaEventRecord(S->init_done, S->stream);
        }
        // ------------------------------------------------------------ chunk n
        const int cur = (int)(n & 1);
        if (e == cudaSuccess && !res.empty()) {
            Chunk& C = chunk[cur];
            // the table set's previous chunk (n - 2) is done; its tile lists
            // are rewritten on the GPU after the copy-outs that read them
            e = cudaEventSynchronize(S->chunk_end[cur]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(S->stream, S->side_done[cur], 0);
            C = Chunk{};
            C.live = true;
            C.res = res;
            C.p0 = S->parity;
            C.quota.resize(res.size());
            // steps of this chunk: about chunk_ms of GPU time over the
            // resident sites, at most chunk_steps
            int64_t steps = S->o.chunk_steps;
            if (S->o.chunk_ms > 0.0) {
                const double fit = S->o.chunk_ms * 1e-3 * rate / (double)std::max<int64_t>(res_sites, 1);
                steps = std::max<int64_t>(1, std::min<int64_t>(steps, (int64_t)fit));
            }
            int64_t k = 0;
            std::vector<Request*> keep;
            for (size_t l = 0; l < res.size(); ++l) {
                C.quota[l] = (int)std::min<int64_t>(steps, res[l]->remaining);
                k = std::max<int64_t>(k, C.quota[l]);
                res[l]->remaining -= C.quota[l];
                if (res[l]->remaining > 0)
                    keep.push_back(res[l]);
                else
                    C.finished.push_back(Finished{res[l], (int)l, (C.p0 + C.quota[l]) & 1, LBM_OK});
            }
            TableSet& T = S->set[cur];
            if (e == cudaSuccess) e = rebuild(S, T, C.res, C.quota);
            if (e == cudaSuccess) e = cudaEventRecord(S->chunk_begin[cur], S->stream);
            const int g0 = pass_grid(S, 0, T.ntiles[0]), g1 = pass_grid(S, 1, T.ntiles[1]);
            for (int64_t st = 0; st < k && e == cudaSuccess; ++st) {
                StepArgs a0 = args(S, T, 0, S->parity), a1 = args(S, T, 1, S->parity);
                a0.step = a1.step = (int)st;
                if (!S->fused) e = launch(S, 0, a0, g0, S->stream);
                if (e == cudaSuccess) e = launch(S, 1, a1, g1, S->stream);
                launches += S->fused ? 1 : 2;
                S->parity ^= 1;
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(S->status_host + cur * S->o.max_resident, T.status,
                                    C.res.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                    S->stream);
            if (e == cudaSuccess) e = cudaEventRecord(S->chunk_end[cur], S->stream);
            for (const Finished& f : C.finished) res_sites -= (int64_t)f.R->L.nx * f.R->L.ny;
            res.swap(keep);
            ++n;
        }
        // ------------------------------------------------------------ retire n - 1
        Chunk& P = chunk[cur ^ 1];
        if (e == cudaSuccess && P.live) {
            // copy-outs in flight end before the chunk does: finish their
            // requests as they complete, then wait for the chunk
            while (e == cudaSuccess && !drain.empty() &&
                   cudaEventQuery(S->chunk_end[cur ^ 1]) == cudaErrorNotReady) {
                e = cudaEventSynchronize(drain.front().done);
                if (e == cudaSuccess) e = settle();
            }
            if (e == cudaSuccess) e = cudaEventSynchronize(S->chunk_end[cur ^ 1]);
            float gpu_ms = 0.f;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&gpu_ms, S->chunk_begin[cur ^ 1], S->chunk_end[cur ^ 1]);
            const uint32_t* bits = S->status_host + (cur ^ 1) * S->o.max_resident;
            int64_t done_sites = 0;
            std::vector<Request*> failed_now;
            for (size_t l = 0; l < P.res.size() && e == cudaSuccess; ++l) {
                Request* R = P.res[l];
                done_sites += (int64_t)R->L.nx * R->L.ny * P.quota[l];
                if (!bits[l] || R->dropped) continue;
                const int status = (bits[l] & 2u) ? LBM_ERR_TIMEOUT : LBM_ERR_NUMERIC;
                R->status = status;
                bool fin = false;
                for (Finished& f : P.finished)
                    if (f.R == R) {
                        f.status = status;  // finishes (with the error) below
                        fin = true;
                    }
                if (fin) continue;
                // it went on into chunk n: fail it there
                R->dropped = true;
                Chunk& Cn = chunk[cur];
                bool fin_n = false;
                if (Cn.live)
                    for (Finished& f : Cn.finished)
                        if (f.R == R) {
                            f.status = status;
                            fin_n = true;
                        }
                if (fin_n) continue;
                res.erase(std::remove(res.begin(), res.end(), R), res.end());
                res_sites -= (int64_t)R->L.nx * R->L.ny;
                if (Cn.live)
                    Cn.dropped.push_back(R);  // freed once chunk n is done
                else
                    failed_now.push_back(R);
            }
            // copy-outs into pinned result slots, in flight on the side stream
            // while chunk n runs; a request is done when its copy-out is
            const size_t comps = S->o.with_velocity ? 3 : 1;
            for (Finished& f : P.finished) {
                int status = f.status;
                if (status == LBM_OK && e == cudaSuccess) {
                    const size_t need = comps * (size_t)f.R->L.nx * f.R->L.ny;
                    size_t off = 0;
                    bool slot;
                    {
                        std::lock_guard<std::mutex> lk(S->mu);
                        slot = S->out_alloc.alloc(need, &off);
                    }
                    cudaEvent_t ev = slot ? take_event(S) : nullptr;
                    if (slot && ev) {
                        f.R->out_off = off;
                        f.R->out_n = need;
                        e = enqueue_copy_out(S, S->set[cur ^ 1], *f.R, f.l, f.par,
                                             S->out_host + off);
                        if (e == cudaSuccess) e = cudaEventRecord(ev, S->side);
                        launches += S->o.with_velocity ? 2 : 1;
                        if (e == cudaSuccess) {
                            drain.push_back(Drain{f.R, ev});
                            continue;
                        }
                        S->spare_events.push_back(ev);
                        status = LBM_ERR_CUDA;
                    } else {
                        if (slot) {
                            std::lock_guard<std::mutex> lk(S->mu);
                            S->out_alloc.release(off, need);
                        }
                        e = copy_out_now(S, S->set[cur ^ 1], *f.R, f.l, f.par);
                        launches += S->o.with_velocity ? 2 : 1;
                        if (e != cudaSuccess) status = LBM_ERR_CUDA;
                    }
                }
                finish(S, f.R, status);
            }
            if (e == cudaSuccess) e = cudaEventRecord(S->side_done[cur ^ 1], S->side);
            for (Request* R : P.dropped) finish(S, R, R->status);
            for (Request* R : failed_now) finish(S, R, R->status);
            if (gpu_ms > 0.f && done_sites > 0) {
                const double r = (double)done_sites / (gpu_ms * 1e-3);
                rate = 0.7 * rate + 0.3 * r;
            }
            std::lock_guard<std::mutex> lk(S->mu);
            S->st.site_steps += done_sites;
            S->st.busy_s += gpu_ms * 1e-3;
            S->st.resident = (int)res.size();
            P.live = false;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->st.launches += launches;
        }
        if (e != cudaSuccess) {
            cudaStreamSynchronize(S->stream);
            cudaStreamSynchronize(S->side);
            cudaStreamSynchronize(S->up);
            // copy-outs in flight keep their result slots (released by poll)
            for (Drain& d : drain) S->spare_events.push_back(d.done);
            drain.clear();
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (auto& sl : in_pending) S->in_alloc.release(sl.first, sl.second);
                in_pending.clear();
            }
            fail_all(S, LBM_ERR_CUDA);
            res.clear();
            res_sites = 0;
            chunk[0] = Chunk{};
            chunk[1] = Chunk{};
            S->set[0].members.clear();
            S->set[1].members.clear();
            continue;
        }
    }
    // stopping: wait for the copies in flight, keep their events for reuse
    cudaStreamSynchronize(S->side);
    cudaStreamSynchronize(S->up);
    for (Drain& d : drain) S->spare_events.push_back(d.done);
}

// The worker thread: an exception (an allocation that failed) must not end
// the process; the server fails every request and refuses new ones.
void worker_main(lbm_server* S) {
    try {
        worker_loop(S);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->dead = true;
        }
        cudaStreamSynchronize(S->stream);
        cudaStreamSynchronize(S->side);
        cudaStreamSynchronize(S->up);
        fail_all(S, LBM_ERR_STATE);
    }
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

extern "C" {

void lbm_server_opts_default(lbm_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->arena_bytes = (size_t)8 << 30;
    o->max_resident = 1024;
    o->chunk_steps = 100;
    o->max_request_sites = (int64_t)2048 * 2048;
    o->target_resident_sites = (int64_t)16 << 20;
    o->storage = LBM_STORE_F32_DEV;
    o->eos_precision = LBM_EOS_DF;
    o->kernel_variant = LBM_KERNEL_AUTO;
    o->with_velocity = 1;
    o->max_width = 2048;
    o->chunk_ms = 4.0;
}

static int lbm_server_create_body(const lbm_server_opts* opts, lbm_server** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_server_opts o;
    lbm_server_opts_default(&o);
    if (opts) {
        lbm_server_opts d = o;
        o = *opts;
        if (!o.arena_bytes) o.arena_bytes = d.arena_bytes;
        if (!o.max_resident) o.max_resident = d.max_resident;
        if (!o.chunk_steps) o.chunk_steps = d.chunk_steps;
        if (!o.max_request_sites) o.max_request_sites = d.max_request_sites;
        if (!o.target_resident_sites) o.target_resident_sites = d.target_resident_sites;
        if (!o.max_width) o.max_width = d.max_width;
        if (o.chunk_ms == 0.0) o.chunk_ms = d.chunk_ms;
    }
    if (o.max_resident < 1 || o.chunk_steps < 1 || o.max_request_sites < 4 ||
        o.target_resident_sites < 1 || o.storage < LBM_STORE_F32 ||
        o.storage > LBM_STORE_F16_DEV || o.eos_precision < LBM_EOS_F64 ||
        o.eos_precision > LBM_EOS_F32 || o.max_width < 2 ||
        (o.kernel_variant != LBM_KERNEL_AUTO && o.kernel_variant != LBM_KERNEL_PLAIN &&
         o.kernel_variant != LBM_KERNEL_TMA) ||
        (o.schedule != LBM_SCHED_AUTO && o.schedule != LBM_SCHED_TWO_PASS &&
         o.schedule != LBM_SCHED_FUSED) ||
        (o.kernel_variant == LBM_KERNEL_TMA && o.schedule == LBM_SCHED_TWO_PASS) ||
        (o.alloc == nullptr) != (o.free == nullptr))
        return LBM_ERR_ARG;
    lbm_server* S = new (std::nothrow) lbm_server();
    if (!S) return LBM_ERR_OOM;
    S->o = o;
    S->fused = o.schedule != LBM_SCHED_TWO_PASS;
    S->f16 = o.storage == LBM_STORE_F16_DEV;
    S->es = S->f16 ? 2 : 4;
    // the single pass on the TMA kernel unless plain loads were asked for
    const bool want_tma = S->fused && o.kernel_variant != LBM_KERNEL_PLAIN;
    for (int k = 0; k < 2; ++k) {
        PassState& P = S->pass[k];
        P.tx = kPassDefaults[k].tx;
        P.ty = kPassDefaults[k].ty;
        P.spt = kPassDefaults[k].spt;
        if (k == 1 && want_tma) {
            P.tx = 32;
            P.ty = 16;
            P.spt = 2;
        }
        if (o.tile_x || o.tile_y) {
            P.tx = o.tile_x ? o.tile_x : 64;
            P.ty = o.tile_y ? o.tile_y : 8;
            P.spt = o.sites_per_thread ? o.sites_per_thread : 1;
            if (k == 1 && want_tma) P.spt = P.tx * P.ty / 256;
        }
        const bool bad = (k == 1 && want_tma) ? !fused_tma_shape_supported(P.tx, P.ty)
                                              : (P.tx % 32 || P.ty < 1 || P.spt < 1 ||
                                                 P.tx * (P.ty / P.spt) > 512 || P.ty % P.spt);
        if (bad) {
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
        cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&S->chunk_end[0]) != cudaSuccess ||
        cudaEventCreate(&S->chunk_end[1]) != cudaSuccess ||
        cudaEventCreate(&S->chunk_begin[0]) != cudaSuccess ||
        cudaEventCreate(&S->chunk_begin[1]) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->up_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->init_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->side_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->side_done[1], cudaEventDisableTiming) != cudaSuccess)
        return fail(LBM_ERR_CUDA);
    const size_t nmax = (size_t)o.max_request_sites;
    // one turn admits at most the resident-site target plus one request
    S->up_cap = (size_t)round_up(o.target_resident_sites, 32) + (size_t)round_up((int64_t)nmax, 32);
    // the arena: a population row space with the common pitch of the widest
    // request, then a psi region (a ninth of the arena)
    {
        const int64_t gx = 16 / S->es;
        S->pitch = round_up(o.max_width + 2 * gx, 32 / S->es);
        S->psi_region = (size_t)round_up((int64_t)(o.arena_bytes / 9), 256);
        const size_t pop_budget = o.arena_bytes - S->psi_region;
        S->row_cap = (int64_t)(pop_budget / (size_t)(18 * S->pitch * S->es));
        S->plane = round_up(S->row_cap * S->pitch, 256 / S->es);
        while (S->row_cap > 0 && (size_t)(18 * S->plane * S->es) > pop_budget) {
            --S->row_cap;
            S->plane = round_up(S->row_cap * S->pitch, 256 / S->es);
        }
        if (S->row_cap < 1) return fail(LBM_ERR_ARG);
        S->pop_bytes = (size_t)(18 * S->plane * S->es);
    }
    // pinned slots for fields waiting to be uploaded and results waiting to
    // be polled: room for the staging buffer's worth of sites and one more
    // request, or for everything the arena can hold if that is less
    const size_t arena_sites = (size_t)S->row_cap * (size_t)o.max_width;
    const size_t slot_sites = std::min(S->up_cap, arena_sites) + (size_t)round_up((int64_t)nmax, 32);
    const size_t out_sites = slot_sites * (o.with_velocity ? 3 : 1);
    bool ok = (S->arena = srv_alloc(S, o.arena_bytes)) != nullptr &&
              (S->staging = static_cast<double*>(srv_alloc(S, S->up_cap * sizeof(double)))) &&
              (S->staging32 = static_cast<float*>(srv_alloc(S, S->up_cap * sizeof(float)))) &&
              cudaMallocHost(&S->in_host, slot_sites * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&S->out_host, out_sites * sizeof(double)) == cudaSuccess &&
              (S->outbuf = static_cast<double*>(srv_alloc(S, 3 * nmax * sizeof(double)))) &&
              cudaMallocHost(&S->down_host, 3 * nmax * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&S->status_host, 2 * (size_t)o.max_resident * sizeof(uint32_t)) ==
                  cudaSuccess;
    for (auto& T : S->set)
        ok = ok &&
             (T.lat = static_cast<LatDev*>(srv_alloc(S, (size_t)o.max_resident * sizeof(LatDev)))) &&
             (T.quota = static_cast<int*>(srv_alloc(S, (size_t)o.max_resident * sizeof(int)))) &&
             (T.status =
                  static_cast<uint32_t*>(srv_alloc(S, (size_t)o.max_resident * sizeof(uint32_t)))) &&
             cudaMallocHost(&T.lat_h, (size_t)o.max_resident * sizeof(LatDev)) == cudaSuccess &&
             cudaMallocHost(&T.quota_h, (size_t)o.max_resident * sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(LBM_ERR_OOM);
    }
    if (cudaMemset(S->arena, 0, o.arena_bytes) != cudaSuccess) return fail(LBM_ERR_CUDA);
    S->psi_arena = reinterpret_cast<float*>(static_cast<char*>(S->arena) + S->pop_bytes);
    S->rows_alloc.reset((size_t)S->row_cap, 1);
    S->psi_alloc.reset(o.arena_bytes - S->pop_bytes);
    S->in_alloc.reset(slot_sites, 32);
    S->out_alloc.reset(out_sites, 32);
    // one tensor map for the whole row space (all resident requests)
    if (want_tma)
        S->tma = fused_tma_make_space_map(S->f16, S->pass[1].tx, S->pass[1].ty, S->pitch,
                                          S->plane, S->row_cap, S->arena, S->tmap);
    if (want_tma && !S->tma) {
        if (o.kernel_variant == LBM_KERNEL_TMA) return fail(LBM_ERR_ARG);
        S->pass[1].tx = kPassDefaults[1].tx;  // plain loads instead
        S->pass[1].ty = kPassDefaults[1].ty;
        S->pass[1].spt = kPassDefaults[1].spt;
    }
    S->st.arena_bytes = (int64_t)o.arena_bytes;
    try {
        S->worker = std::thread(worker_main, S);
    } catch (...) {
        return fail(LBM_ERR_OOM);
    }
    *out = S;
    return LBM_OK;
}

int lbm_server_create(const lbm_server_opts* opts, lbm_server** out) {
    return guarded([&] { return lbm_server_create_body(opts, out); });
}

static int lbm_submit_body(lbm_server* S, const lbm_lattice_desc* d, const double* rho, int64_t nsteps,
               uint64_t* ticket) {
    if (!S || !d || !rho || !ticket || nsteps < 1) return LBM_ERR_ARG;
    Request R;
    R.d = *d;
    R.d.storage = S->o.storage;
    R.d.eos_precision = S->o.eos_precision;
    std::string why;
    if (validate_desc(R.d, why) != LBM_OK || R.d.collision != LBM_COLL_BGK) return LBM_ERR_ARG;
    const size_t n = (size_t)R.d.nx * R.d.ny;
    if ((int64_t)n > S->o.max_request_sites) return LBM_ERR_CAPACITY;
    double mn = 0.0;
    if (!field_scan(rho, n, &mn)) return LBM_ERR_ARG;  // every density finite
    if (R.d.nx > S->o.max_width) return LBM_ERR_CAPACITY;
    R.L = lat_layout(R.d, 0);
    R.rows = (size_t)(R.d.ny + 2 * GY);  // of the row space, at the common pitch
    R.psi_bytes = (size_t)lat_psi_elems(R.L) * 4;
    if ((int64_t)R.rows > S->row_cap ||
        (size_t)round_up((int64_t)R.psi_bytes, 256) > S->o.arena_bytes - S->pop_bytes)
        return LBM_ERR_CAPACITY;
    if (R.d.storage != LBM_STORE_F32 && R.d.rho0 < 0.0) R.L.rho0 = auto_rho0_of_min(mn);
    // the field goes to a pinned slot when one is free (the copy runs on the
    // caller's thread), else to the heap until the worker stages it
    size_t off = 0;
    bool slot;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        slot = S->in_alloc.alloc(n, &off);
    }
    if (slot) {
        std::memcpy(S->in_host + off, rho, n * sizeof(double));
        R.in_off = off;
        R.in_n = n;
    } else {
        R.rho.assign(rho, rho + n);
    }
    R.nsteps = R.remaining = nsteps;
    R.t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop || S->dead) {
        if (slot) S->in_alloc.release(off, n);
        return LBM_ERR_STATE;
    }
    R.ticket = S->next_ticket++;
    *ticket = R.ticket;
    S->queue.push_back(R.ticket);
    S->reqs.emplace(R.ticket, std::move(R));
    S->st.submitted++;
    S->st.queued = (int)S->queue.size();
    S->cv.notify_one();
    return LBM_OK;
}

int lbm_submit(lbm_server* S, const lbm_lattice_desc* d, const double* rho, int64_t nsteps,
               uint64_t* ticket) {
    return guarded([&] { return lbm_submit_body(S, d, rho, nsteps, ticket); });
}

static int lbm_poll_body(lbm_server* S, uint64_t ticket, double* rho, double* ux, double* uy,
             double* latency_s) {
    if (!S) return LBM_ERR_ARG;
    // Under the lock: take the finished request out of the table (its result
    // slot stays allocated, so nothing else can reuse it).  The copy of the
    // result runs without the lock, so that the worker is never held up by
    // a poll; the slot is released afterwards.
    int status;
    size_t n = 0, out_off = kNoSlot, out_n = 0;
    std::vector<double> vr, vx, vy;  // a result that had no pinned slot
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return LBM_ERR_UNKNOWN_TICKET;
        Request& R = it->second;
        if (R.state != ST_DONE) return LBM_PENDING;
        status = R.status;
        n = (size_t)R.L.nx * R.L.ny;
        out_off = R.out_off;
        out_n = R.out_n;
        vr.swap(R.rho);
        vx.swap(R.ux);
        vy.swap(R.uy);
        if (latency_s) *latency_s = std::chrono::duration<double>(R.t_done - R.t_submit).count();
        if (R.in_off != kNoSlot) S->in_alloc.release(R.in_off, R.in_n);
        S->reqs.erase(it);
    }
    if (status == LBM_OK) {
        const bool vel = S->o.with_velocity != 0;
        // the result is in its pinned slot, or (no slot was free) in the vectors
        const double* src[3] = {vr.data(), vel ? vx.data() : nullptr, vel ? vy.data() : nullptr};
        if (out_off != kNoSlot) {
            const double* h = S->out_host + out_off;
            src[0] = h;
            src[1] = vel ? h + n : nullptr;
            src[2] = vel ? h + 2 * n : nullptr;
        }
        if (rho) std::memcpy(rho, src[0], n * sizeof(double));
        // without with_velocity the server keeps no velocities: NaN
        for (int c = 1; c < 3; ++c) {
            double* dst = c == 1 ? ux : uy;
            if (!dst) continue;
            if (src[c])
                std::memcpy(dst, src[c], n * sizeof(double));
            else
                std::fill(dst, dst + n, std::numeric_limits<double>::quiet_NaN());
        }
    }
    if (out_off != kNoSlot) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->out_alloc.release(out_off, out_n);
    }
    return status;
}

int lbm_poll(lbm_server* S, uint64_t ticket, double* rho, double* ux, double* uy,
             double* latency_s) {
    return guarded([&] { return lbm_poll_body(S, ticket, rho, ux, uy, latency_s); });
}

static int lbm_server_get_stats_body(lbm_server* S, lbm_server_stats* out) {
    if (!S || !out) return LBM_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    return LBM_OK;
}

int lbm_server_get_stats(lbm_server* S, lbm_server_stats* out) {
    return guarded([&] { return lbm_server_get_stats_body(S, out); });
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
    cudaStreamSynchronize(S->side);
    cudaStreamSynchronize(S->up);
    free_server(S);
    delete S;
}

}  // extern "C"
