// Build server (include/esmf_server.h): admission by device-memory budget, a
// residency cache of per-molecule handles, continuous batching over
// non-blocking streams, optional CUDA-graph replay, optional batched ticks
// (the tensor-path builds admitted together run as one persistent launch),
// latency statistics.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "esmf_internal.cuh"
#include "esmf_server.h"

namespace esmf {
int handle_reserve(esmf_fock_t *h, int m);
}

using namespace esmf;

namespace {

using Clock = std::chrono::steady_clock;

struct Molecule {
    int n = 0;
    std::vector<double> center, exps, coefs;
    std::vector<int32_t> nprim;
    double tol = 0.0;
    esmf_fock_t *h = nullptr;
    int64_t bytes = 0;        // device bytes of the handle
    int64_t known_bytes = 0;  // largest device bytes a handle of this molecule has had (0: never created)
    uint64_t last_use = 0;
    bool busy = false;
    int queued = 0;           // requests waiting for this molecule
};

struct Request {
    char err[256] = "";
    int64_t ticket = 0;
    int mol = 0, m = 0;
    const double *D = nullptr;
    double *J = nullptr, *K = nullptr, *traces = nullptr;
    Clock::time_point t_submit, t_done;
    bool done = false;
    int status = ESMF_OK;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_in = nullptr;     // inputs copied (batched ticks wait on it)
    size_t cap = 0;           // doubles per matrix batch (m * N * N)
    int tcap = 0;
    double *dD = nullptr, *dJ = nullptr, *dK = nullptr, *dt = nullptr;
    double *hD = nullptr, *hJ = nullptr, *hK = nullptr, *ht = nullptr;   // page-locked staging
    std::shared_ptr<Request> req;
};

}  // namespace

struct esmf_server {
    int device = 0;
    int64_t budget = 0;
    int max_inflight = 1;
    int precision = ESMF_PREC_FP16X2;
    bool use_graphs = false;
    bool batch = false;              // batched ticks
    bool evict_largest = false;      // eviction order: largest idle first (else LRU)
    cudaStream_t tick_stream = nullptr;
    cudaEvent_t tick_ev = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::vector<Molecule> mols;
    std::deque<std::shared_ptr<Request>> pending;
    std::map<int64_t, std::shared_ptr<Request>> tickets;
    std::vector<Slot> slots;
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;   // (molecule, m, slot)
    // batched ticks captured once per composition: (molecule, m, slot) of
    // every entry in tick order
    std::map<std::vector<std::tuple<int, int, int>>, cudaGraphExec_t> tick_graphs;
    int64_t next_ticket = 1;
    uint64_t use_clock = 0;
    int inflight = 0;
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0, creates = 0, evictions = 0, graph_launches = 0;
    int64_t batch_launches = 0, batched_builds = 0, tick_graph_launches = 0;
    int64_t peak_inflight = 0;
    std::vector<double> lat_ms;
    Clock::time_point first_submit, last_done;
    bool have_first = false;
};

namespace {

int64_t resident_bytes(const esmf_server *s) {
    int64_t b = 0;
    for (const auto &m : s->mols) if (m.h) b += m.bytes;
    return b;
}

// Captured graphs hold the device addresses of a molecule's work memory and of
// a slot's I/O buffers: drop them whenever either is reallocated or freed.
// (Only called for an idle molecule or a free slot, so none of them runs.)
// Batched-tick graphs that contain molecule `mol` (field 0) or slot `slot`
// (field 2) of any entry; a negative argument matches nothing.
void drop_tick_graphs(esmf_server *s, int mol, int slot) {
    for (auto it = s->tick_graphs.begin(); it != s->tick_graphs.end();) {
        bool hit = false;
        for (const auto &e : it->first) hit |= std::get<0>(e) == mol || std::get<2>(e) == slot;
        if (hit) {
            cudaGraphExecDestroy(it->second);
            it = s->tick_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

void drop_graphs_of(esmf_server *s, int mol) {
    for (auto it = s->graphs.begin(); it != s->graphs.end();) {
        if (std::get<0>(it->first) == mol) {
            cudaGraphExecDestroy(it->second);
            it = s->graphs.erase(it);
        } else {
            ++it;
        }
    }
    drop_tick_graphs(s, mol, -1);
}

void drop_graphs_of_slot(esmf_server *s, int slot) {
    for (auto it = s->graphs.begin(); it != s->graphs.end();) {
        if (std::get<2>(it->first) == slot) {
            cudaGraphExecDestroy(it->second);
            it = s->graphs.erase(it);
        } else {
            ++it;
        }
    }
    drop_tick_graphs(s, -1, slot);
}

void evict(esmf_server *s, int idx) {
    Molecule &m = s->mols[idx];
    drop_graphs_of(s, idx);
    esmf_fock_destroy(m.h);
    m.h = nullptr;
    m.bytes = 0;
    ++s->evictions;
}

// How long a request for a molecule without a handle may wait for room
// rather than evict a molecule that still has queued requests (a bound that
// only guarantees progress: queues of resident molecules drain long before).
constexpr double kPatienceMs = 30000.0;

// Free device memory for a handle of molecule idx: evict idle handles until
// its size fits — the size its handle had before (with 1/16 to spare for a
// larger density count), or, on first creation, the upper bound of its store.  Molecules with no queued request go
// first (the largest or the least recently used first, by the server's
// order); molecules with queued requests only when allow_queued is set, the
// one whose next request comes latest in the queue first (the furthest next
// use, which is the eviction that costs the fewest re-creations).  Returns
// true when the bound fits.
bool make_room(esmf_server *s, int idx, bool allow_queued) {
    const Molecule &mol = s->mols[idx];
    const int64_t np = (mol.n + 7) / 8 * 8;
    const int64_t P = np * (np + 1) / 2;
    const int64_t bound = mol.known_bytes > 0 ? mol.known_bytes + mol.known_bytes / 16
                                              : (P * (P + 1) / 2) * 4 + (P * (P + 1) / 2) / 8 + np * np * 64;
    std::vector<int64_t> next_use;
    for (;;) {
        const int64_t freeb = s->budget - resident_bytes(s);
        if (freeb >= bound) return true;
        int victim = -1;
        for (size_t i = 0; i < s->mols.size(); ++i) {
            const Molecule &c = s->mols[i];
            if ((int)i == idx || !c.h || c.busy || c.queued > 0) continue;
            if (victim < 0) { victim = (int)i; continue; }
            const Molecule &v = s->mols[victim];
            const bool better = s->evict_largest ? (c.bytes > v.bytes || (c.bytes == v.bytes && c.last_use < v.last_use))
                                                 : c.last_use < v.last_use;
            if (better) victim = (int)i;
        }
        if (victim < 0 && allow_queued) {
            if (next_use.empty()) {
                next_use.assign(s->mols.size(), INT64_MAX);
                int64_t pos = 0;
                for (const auto &r : s->pending) {
                    if (next_use[r->mol] == INT64_MAX) next_use[r->mol] = pos;
                    ++pos;
                }
            }
            for (size_t i = 0; i < s->mols.size(); ++i) {
                const Molecule &c = s->mols[i];
                if ((int)i == idx || !c.h || c.busy) continue;
                if (victim < 0 || next_use[i] > next_use[victim] ||
                    (next_use[i] == next_use[victim] && c.bytes > s->mols[victim].bytes))
                    victim = (int)i;
            }
        }
        if (victim < 0) return false;
        evict(s, victim);
    }
}

int ensure_slot(esmf_server *s, int slot_idx, size_t cnt, int m) {
    Slot &sl = s->slots[slot_idx];
    if (cnt <= sl.cap && m <= sl.tcap) return ESMF_OK;
    drop_graphs_of_slot(s, slot_idx);
    cudaFree(sl.dD); cudaFree(sl.dJ); cudaFree(sl.dK); cudaFree(sl.dt);
    cudaFreeHost(sl.hD); cudaFreeHost(sl.hJ); cudaFreeHost(sl.hK); cudaFreeHost(sl.ht);
    sl.dD = sl.dJ = sl.dK = sl.dt = sl.hD = sl.hJ = sl.hK = sl.ht = nullptr;
    sl.cap = 0; sl.tcap = 0;
    const size_t b = cnt * sizeof(double), tb = (size_t)m * sizeof(double);
    if (cudaMalloc(&sl.dD, b) || cudaMalloc(&sl.dJ, b) || cudaMalloc(&sl.dK, b) || cudaMalloc(&sl.dt, tb) ||
        cudaMallocHost(&sl.hD, b) || cudaMallocHost(&sl.hJ, b) || cudaMallocHost(&sl.hK, b) ||
        cudaMallocHost(&sl.ht, tb)) {
        cudaGetLastError();
        set_error("server slot allocation of %zu bytes failed", b);
        return ESMF_ERR_OOM;
    }
    sl.cap = cnt;
    sl.tcap = m;
    return ESMF_OK;
}

void finish(esmf_server *s, Slot &sl, int status) {
    std::shared_ptr<Request> r = sl.req;
    Molecule &mol = s->mols[r->mol];
    if (status == ESMF_OK) {
        const size_t cnt = (size_t)r->m * mol.n * mol.n;
        std::memcpy(r->J, sl.hJ, cnt * sizeof(double));
        std::memcpy(r->K, sl.hK, cnt * sizeof(double));
        if (r->traces) std::memcpy(r->traces, sl.ht, r->m * sizeof(double));
        if (mol.h && esmf_fock_device_error(mol.h, 1) != 0) status = ESMF_ERR_TIMEOUT;
    }
    r->status = status;
    r->t_done = Clock::now();
    r->done = true;
    mol.busy = false;
    mol.last_use = ++s->use_clock;
    sl.req.reset();
    --s->inflight;
    if (status == ESMF_OK) {
        ++s->completed;
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        s->last_done = r->t_done;
    } else {
        ++s->failed;
    }
    s->cv_done.notify_all();
}

int issue_build(esmf_server *s, int slot_idx, Molecule &mol, int mol_idx, int m) {
    Slot &sl = s->slots[slot_idx];
    if (!s->use_graphs)
        return esmf_fock_build(mol.h, m, sl.dD, sl.dJ, sl.dK, nullptr, sl.dt, sl.stream);
    auto key = std::make_tuple(mol_idx, m, slot_idx);
    auto it = s->graphs.find(key);
    if (it == s->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        if (cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            set_error("begin capture failed");
            return ESMF_ERR_CUDA;
        }
        const int rc = esmf_fock_build(mol.h, m, sl.dD, sl.dJ, sl.dK, nullptr, sl.dt, sl.stream);
        const cudaError_t e = cudaStreamEndCapture(sl.stream, &g);
        if (rc != ESMF_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (rc == ESMF_OK) set_error("stream capture failed");
            return rc != ESMF_OK ? rc : ESMF_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            cudaGetLastError();
            set_error("graph instantiate failed");
            return ESMF_ERR_CUDA;
        }
        it = s->graphs.emplace(key, ge).first;
    }
    if (cudaGraphLaunch(it->second, sl.stream) != cudaSuccess) {
        cudaGetLastError();
        set_error("graph launch failed");
        return ESMF_ERR_CUDA;
    }
    ++s->graph_launches;
    return ESMF_OK;
}

// results back to the slot's page-locked buffers, then the completion event
int issue_outputs(Slot &sl, size_t cnt, int m) {
    if (cudaMemcpyAsync(sl.hJ, sl.dJ, cnt * sizeof(double), cudaMemcpyDeviceToHost, sl.stream) ||
        cudaMemcpyAsync(sl.hK, sl.dK, cnt * sizeof(double), cudaMemcpyDeviceToHost, sl.stream) ||
        cudaMemcpyAsync(sl.ht, sl.dt, m * sizeof(double), cudaMemcpyDeviceToHost, sl.stream) ||
        cudaEventRecord(sl.ev, sl.stream))
        return ESMF_ERR_CUDA;
    return ESMF_OK;
}

void fail_slot(esmf_server *s, int slot_idx, int rc) {
    Slot &sl = s->slots[slot_idx];
    std::snprintf(sl.req->err, sizeof(sl.req->err), "%s", esmf_last_error());
    cudaGetLastError();
    cudaStreamSynchronize(sl.stream);
    finish(s, sl, rc);
}

bool on_tensor_path(esmf_fock_t *h) {
    esmf_stats_t st;
    return esmf_fock_stats(h, &st) == ESMF_OK && st.mode == ESMF_MODE_STORED && is_split16(st.precision);
}

// Most batched-tick compositions kept as instantiated graphs; beyond it the
// cache starts over (a stream of ever-new compositions then costs a capture
// per tick, as many as without the cache).
constexpr size_t kMaxTickGraphs = 128;

// The batched build of one tick from its captured graph: captured on first
// use of this composition (molecules, density counts and slots), replayed
// after.  The handles' work memory for these m was reserved at admission, so
// the captured build allocates nothing.
int launch_tick_graph(esmf_server *s, const std::vector<std::tuple<int, int, int>> &key, int count,
                      esmf_fock_t *const *hs, const int *ms, const double *const *Ds, double *const *Js,
                      double *const *Ks, double *const *ts) {
    auto it = s->tick_graphs.find(key);
    if (it == s->tick_graphs.end()) {
        if (s->tick_graphs.size() >= kMaxTickGraphs) {
            for (auto &g : s->tick_graphs) cudaGraphExecDestroy(g.second);
            s->tick_graphs.clear();
        }
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        if (cudaStreamBeginCapture(s->tick_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            set_error("begin capture of a batched tick failed");
            return ESMF_ERR_CUDA;
        }
        const int rc = esmf_fock_build_batch(count, hs, ms, Ds, Js, Ks, nullptr, ts, s->tick_stream);
        const cudaError_t e = cudaStreamEndCapture(s->tick_stream, &g);
        if (rc != ESMF_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (rc == ESMF_OK) set_error("capture of a batched tick failed");
            return rc != ESMF_OK ? rc : ESMF_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            cudaGetLastError();
            set_error("instantiating a batched tick failed");
            return ESMF_ERR_CUDA;
        }
        it = s->tick_graphs.emplace(key, ge).first;
    }
    if (cudaGraphLaunch(it->second, s->tick_stream) != cudaSuccess) {
        cudaGetLastError();
        set_error("launching a batched tick graph failed");
        return ESMF_ERR_CUDA;
    }
    ++s->tick_graph_launches;
    return ESMF_OK;
}

// One batched tick: the builds of the slots in `tick` (distinct molecules on
// the tensor path, inputs being copied on their own streams) as one
// esmf_fock_build_batch call on the tick stream, i.e. one persistent launch
// per pass of 16 densities for all of them, replayed from a CUDA graph when
// graphs are on; each slot's result copies wait for the tick.
void issue_tick(esmf_server *s, const std::vector<int> &tick) {
    const int count = (int)tick.size();
    esmf_fock_t *hs[ESMF_MAX_BATCH] = {};
    int ms[ESMF_MAX_BATCH] = {};
    const double *Ds[ESMF_MAX_BATCH] = {};
    double *Js[ESMF_MAX_BATCH] = {}, *Ks[ESMF_MAX_BATCH] = {}, *ts[ESMF_MAX_BATCH] = {};
    int rc = ESMF_OK;
    std::vector<std::tuple<int, int, int>> key;
    for (int i = 0; i < count && rc == ESMF_OK; ++i) {
        Slot &sl = s->slots[tick[i]];
        hs[i] = s->mols[sl.req->mol].h;
        ms[i] = sl.req->m;
        Ds[i] = sl.dD; Js[i] = sl.dJ; Ks[i] = sl.dK; ts[i] = sl.dt;
        key.emplace_back(sl.req->mol, sl.req->m, tick[i]);
        if (cudaStreamWaitEvent(s->tick_stream, sl.ev_in, 0) != cudaSuccess) rc = ESMF_ERR_CUDA;
    }
    if (rc == ESMF_OK) {
        rc = s->use_graphs ? launch_tick_graph(s, key, count, hs, ms, Ds, Js, Ks, ts)
                           : esmf_fock_build_batch(count, hs, ms, Ds, Js, Ks, nullptr, ts, s->tick_stream);
    }
    if (rc == ESMF_OK && cudaEventRecord(s->tick_ev, s->tick_stream) != cudaSuccess) rc = ESMF_ERR_CUDA;
    if (rc == ESMF_OK) {
        ++s->batch_launches;
        s->batched_builds += count;
    } else {
        cudaStreamSynchronize(s->tick_stream);
    }
    for (int i = 0; i < count; ++i) {
        Slot &sl = s->slots[tick[i]];
        int r = rc;
        if (r == ESMF_OK && cudaStreamWaitEvent(sl.stream, s->tick_ev, 0) != cudaSuccess) r = ESMF_ERR_CUDA;
        if (r == ESMF_OK) {
            const Molecule &mol = s->mols[sl.req->mol];
            r = issue_outputs(sl, (size_t)sl.req->m * mol.n * mol.n, sl.req->m);
        }
        if (r != ESMF_OK) fail_slot(s, tick[i], r);
    }
}

// try to start request r in a free slot; returns false if it must wait.  With
// batched ticks, a tensor-path build is not issued here: its slot joins
// `tick` once its inputs are on their way.
bool try_admit(esmf_server *s, const std::shared_ptr<Request> &r, std::vector<int> &tick) {
    Molecule &mol = s->mols[r->mol];
    if (mol.busy) return false;
    int slot_idx = -1;
    for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].req) { slot_idx = (int)i; break; }
    if (slot_idx < 0) return false;
    if (!mol.h) {
        // While other builds are in flight (so the server makes progress) a
        // new handle waits, up to kPatienceMs, rather than evict a molecule
        // that still has queued requests: that eviction would only be undone
        // by a re-creation a few requests later.
        const double waited = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
        const bool patient = s->inflight > 0 && waited < kPatienceMs;
        if (!make_room(s, r->mol, !patient) && patient) return false;
    }
    Slot &sl = s->slots[slot_idx];
    sl.req = r;
    ++s->inflight;
    s->peak_inflight = std::max<int64_t>(s->peak_inflight, s->inflight);
    int rc = ESMF_OK;
    if (!mol.h) {
        esmf_basis_t b;
        b.n_basis = mol.n; b.center = mol.center.data(); b.n_prim = mol.nprim.data();
        b.exps = mol.exps.data(); b.coefs = mol.coefs.data();
        const int64_t freeb = std::max<int64_t>(1, s->budget - resident_bytes(s));
        rc = esmf_fock_create(&b, mol.tol, ESMF_MODE_AUTO, s->precision, s->device, freeb, &mol.h);
        if (rc == ESMF_OK) ++s->creates;
    }
    if (rc == ESMF_OK) {
        esmf_stats_t before, after;
        esmf_fock_stats(mol.h, &before);
        rc = handle_reserve(mol.h, r->m);
        esmf_fock_stats(mol.h, &after);
        if (after.device_bytes != before.device_bytes) drop_graphs_of(s, r->mol);   // work memory moved
        mol.bytes = after.device_bytes;
        mol.known_bytes = std::max(mol.known_bytes, mol.bytes);
    }
    if (rc == ESMF_OK) rc = ensure_slot(s, slot_idx, (size_t)r->m * mol.n * mol.n, r->m);
    mol.busy = true;
    if (rc == ESMF_OK) {
        const size_t cnt = (size_t)r->m * mol.n * mol.n;
        std::memcpy(sl.hD, r->D, cnt * sizeof(double));
        if (cudaMemcpyAsync(sl.dD, sl.hD, cnt * sizeof(double), cudaMemcpyHostToDevice, sl.stream)) rc = ESMF_ERR_CUDA;
        if (rc == ESMF_OK && s->batch && on_tensor_path(mol.h)) {
            if (cudaEventRecord(sl.ev_in, sl.stream) != cudaSuccess) {
                rc = ESMF_ERR_CUDA;
            } else {
                tick.push_back(slot_idx);
                if ((int)tick.size() == ESMF_MAX_BATCH) {
                    issue_tick(s, tick);
                    tick.clear();
                }
                return true;
            }
        }
        if (rc == ESMF_OK) rc = issue_build(s, slot_idx, mol, r->mol, r->m);
        if (rc == ESMF_OK) rc = issue_outputs(sl, cnt, r->m);
    }
    if (rc != ESMF_OK) fail_slot(s, slot_idx, rc);
    return true;
}

void worker_main(esmf_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->stop && s->pending.empty() && s->inflight == 0) break;
        // completions
        for (auto &sl : s->slots) {
            if (!sl.req) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaSuccess) finish(s, sl, ESMF_OK);
            else if (q != cudaErrorNotReady) {
                std::snprintf(sl.req->err, sizeof(sl.req->err), "build: %s", cudaGetErrorString(q));
                cudaGetLastError();
                finish(s, sl, ESMF_ERR_CUDA);
            }
        }
        // admissions: first, in arrival order, requests whose molecule is
        // resident (no integral evaluation needed); then the others, which
        // may create handles and evict idle molecules.  A request whose
        // molecule is busy waits without blocking the requests behind it.
        // With batched ticks, the tensor-path builds admitted in this pass
        // run together as one batched build.
        std::vector<int> tick;
        for (int pass = 0; pass < 2; ++pass) {
            for (auto it = s->pending.begin(); it != s->pending.end();) {
                if (s->inflight >= s->max_inflight) break;
                Molecule &mol = s->mols[(*it)->mol];
                if (pass == 0 && !mol.h) { ++it; continue; }
                --mol.queued;
                if (try_admit(s, *it, tick)) {
                    it = s->pending.erase(it);
                } else {
                    ++mol.queued;
                    ++it;
                }
            }
        }
        if (!tick.empty()) issue_tick(s, tick);
        if (s->inflight > 0) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
}

}  // namespace

extern "C" {

int esmf_server_create(int device, int64_t budget_bytes, int max_inflight, int precision, int flags,
                       esmf_server_t **out) {
    if (!out || budget_bytes <= 0 || max_inflight < 1 || max_inflight > 64 || precision < ESMF_PREC_FP64 ||
        precision > ESMF_PREC_F32X2 ||
        (flags & ~(ESMF_SERVER_GRAPHS | ESMF_SERVER_BATCH | ESMF_SERVER_EVICT_LARGEST)) != 0) {
        set_error("bad server arguments");
        return ESMF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("device %d not available", device);
        return ESMF_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    esmf_server *s = new (std::nothrow) esmf_server();
    if (!s) { set_error("host allocation failed"); return ESMF_ERR_OOM; }
    s->device = device; s->budget = budget_bytes; s->max_inflight = max_inflight;
    s->precision = precision;
    s->use_graphs = (flags & ESMF_SERVER_GRAPHS) != 0;
    s->batch = (flags & ESMF_SERVER_BATCH) != 0;
    s->evict_largest = (flags & ESMF_SERVER_EVICT_LARGEST) != 0;
    s->slots.resize(max_inflight);
    if (s->batch && (cudaStreamCreateWithFlags(&s->tick_stream, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaEventCreateWithFlags(&s->tick_ev, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        set_error("stream creation failed");
        esmf_server_destroy(s);
        cudaSetDevice(prev);
        return ESMF_ERR_CUDA;
    }
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev_in, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            set_error("stream creation failed");
            esmf_server_destroy(s);
            cudaSetDevice(prev);
            return ESMF_ERR_CUDA;
        }
    }
    s->worker = std::thread(worker_main, s);
    cudaSetDevice(prev);
    *out = s;
    return ESMF_OK;
}

int esmf_server_register(esmf_server_t *s, const esmf_basis_t *basis, double tol, int *basis_id) {
    if (!s || !basis || !basis_id || basis->n_basis <= 0 || !basis->center || !basis->n_prim || !basis->exps ||
        !basis->coefs || !(tol >= 0.0)) {
        set_error("bad register arguments");
        return ESMF_ERR_INVALID_ARG;
    }
    Molecule mol;
    mol.n = basis->n_basis;
    mol.tol = tol;
    int64_t np = 0;
    for (int i = 0; i < mol.n; ++i) {
        if (basis->n_prim[i] < 1 || basis->n_prim[i] > ESMF_MAX_PRIM) { set_error("bad n_prim"); return ESMF_ERR_INVALID_ARG; }
        np += basis->n_prim[i];
    }
    mol.center.assign(basis->center, basis->center + 3 * mol.n);
    mol.nprim.assign(basis->n_prim, basis->n_prim + mol.n);
    mol.exps.assign(basis->exps, basis->exps + np);
    mol.coefs.assign(basis->coefs, basis->coefs + np);
    std::lock_guard<std::mutex> lk(s->mu);
    s->mols.push_back(std::move(mol));
    *basis_id = (int)s->mols.size() - 1;
    return ESMF_OK;
}

int esmf_server_submit(esmf_server_t *s, int basis_id, int m, const double *D, double *J, double *K,
                       double *traces, int64_t *ticket) {
    if (!s || !D || !J || !K || !ticket || m < 1 || m > ESMF_MAX_DENSITIES) {
        set_error("bad submit arguments");
        return ESMF_ERR_INVALID_ARG;
    }
    auto r = std::make_shared<Request>();
    r->m = m; r->D = D; r->J = J; r->K = K; r->traces = traces;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (basis_id < 0 || basis_id >= (int)s->mols.size()) { set_error("unknown basis id %d", basis_id); return ESMF_ERR_INVALID_ARG; }
        r->mol = basis_id;
        r->ticket = s->next_ticket++;
        s->tickets[r->ticket] = r;
        s->pending.push_back(r);
        ++s->mols[basis_id].queued;
        ++s->submitted;
        if (!s->have_first) { s->first_submit = r->t_submit; s->have_first = true; }
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return ESMF_OK;
}

int esmf_server_wait(esmf_server_t *s, int64_t ticket, int timeout_ms) {
    if (!s) { set_error("server is NULL"); return ESMF_ERR_INVALID_ARG; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) { set_error("unknown ticket"); return ESMF_ERR_INVALID_ARG; }
    std::shared_ptr<Request> r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        set_error("ticket %lld not finished", (long long)ticket);
        return ESMF_ERR_TIMEOUT;
    }
    s->tickets.erase(ticket);
    if (r->status != ESMF_OK) set_error("request %lld: %s", (long long)ticket, r->err);
    return r->status;
}

int esmf_server_stats(esmf_server_t *s, esmf_server_stats_t *out) {
    if (!s || !out) { set_error("NULL argument"); return ESMF_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted; out->completed = s->completed; out->failed = s->failed;
    out->creates = s->creates; out->evictions = s->evictions; out->graph_launches = s->graph_launches;
    out->batch_launches = s->batch_launches; out->batched_builds = s->batched_builds;
    out->tick_graph_launches = s->tick_graph_launches;
    out->resident_bytes = resident_bytes(s);
    out->peak_inflight = s->peak_inflight;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            size_t i = (size_t)(q * (double)(v.size() - 1) + 0.5);
            return v[std::min(i, v.size() - 1)];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
        out->max_ms = v.back();
        if (s->have_first) out->span_s = std::chrono::duration<double>(s->last_done - s->first_submit).count();
    }
    return ESMF_OK;
}

int esmf_server_reset_stats(esmf_server_t *s) {
    if (!s) { set_error("server is NULL"); return ESMF_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(s->mu);
    s->submitted = s->completed = s->failed = s->creates = s->evictions = s->graph_launches = 0;
    s->batch_launches = s->batched_builds = s->tick_graph_launches = 0;
    s->peak_inflight = s->inflight;
    s->lat_ms.clear();
    s->have_first = false;
    return ESMF_OK;
}

void esmf_server_destroy(esmf_server_t *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto &g : s->graphs) cudaGraphExecDestroy(g.second);
    for (auto &g : s->tick_graphs) cudaGraphExecDestroy(g.second);
    for (auto &mol : s->mols) if (mol.h) esmf_fock_destroy(mol.h);
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        cudaFree(sl.dD); cudaFree(sl.dJ); cudaFree(sl.dK); cudaFree(sl.dt);
        cudaFreeHost(sl.hD); cudaFreeHost(sl.hJ); cudaFreeHost(sl.hK); cudaFreeHost(sl.ht);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.ev_in) cudaEventDestroy(sl.ev_in);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->tick_stream) {
        cudaStreamSynchronize(s->tick_stream);
        cudaStreamDestroy(s->tick_stream);
    }
    if (s->tick_ev) cudaEventDestroy(s->tick_ev);
    cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
