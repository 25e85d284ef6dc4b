// vor_server.cu -- request server with continuous batching (vor_server_*).
//
// One dispatcher thread owns every CUDA call of a server.  Clients only
// touch host state under the server mutex: submit copies the sites into the
// pinned block and queues the request; poll/wait/release read or drop it.
//
// A wave is the batch of a prefix of the waiting requests (vor_sched.h):
//   launch    take a device block (workspace + sites + set offsets + boxes +
//             worst-case outputs + the per-request cell offsets), copy the
//             staged sites in, vor_build_batch_async, rebase the cell
//             offsets per request, copy the error word and the totals out,
//             record an event;
//   sizes     (event done) read status and totals; on an error split the
//             wave into single-request waves; else take an exact host result
//             block, copy the results out, record the event again;
//   results   (event done) point every request at its slices, free the
//             device block and the stream.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "vor.h"
#include "vor_internal.h"
#include "vor_sched.h"

namespace vor {
namespace {

constexpr uint64_t kAlign = 256;

uint64_t al(uint64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Per request, the cell offsets rebased to its own first edge: out[j][k] =
// cell_ptr[set_ptr[j] + k] - cell_ptr[set_ptr[j]] for k = 0..n_j, stored at
// out + set_ptr[j] + j; edge_base[j] = cell_ptr[set_ptr[j]] (j = S: total).
__global__ void k_rebase(const long long *__restrict__ cell_ptr, const long long *__restrict__ set_ptr,
                         int S, long long total, long long *__restrict__ out,
                         long long *__restrict__ edge_base, const WsHeader *hdr) {
    if (hdr->err) return;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q <= S) edge_base[q] = cell_ptr[set_ptr[q]];
    if (q >= total) return;
    int lo = 0, hi = S;                    // largest j with set_ptr[j] + j <= q
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (set_ptr[mid] + mid <= q) lo = mid;
        else hi = mid;
    }
    const long long k = q - (set_ptr[lo] + lo);
    out[q] = cell_ptr[set_ptr[lo] + k] - cell_ptr[set_ptr[lo]];
}

struct HostResult {        // one wave's results in the pinned block
    uint64_t off = 0;
    int refs = 0;
};

struct Request {
    uint64_t id = 0;
    int64_t n = 0;
    vor_box box{0, 0};
    uint64_t in_off = 0;   // staged sites (pinned block)
    bool staged = false;
    int status = VOR_PENDING;
    bool solo = false;     // run in a wave of its own (after a failed wave)
    bool cancelled = false;
    bool running = false;
    double t_submit = 0, t_start = 0, t_done = 0;
    int wave_requests = 0;
    std::shared_ptr<HostResult> res;
    const int64_t *cell_ptr = nullptr;
    const int32_t *labels = nullptr;
    const double *vx = nullptr, *vy = nullptr;
    const int32_t *del = nullptr;
    int64_t n_edges = 0, n_del = 0;
};

// device layout of a wave
struct WaveLayout {
    uint64_t ws, ws_bytes, sites, set_ptr, boxes, cell_ptr, labels, vx, vy, del, del_set_ptr, totals,
        rebased, edge_base, total;
    int64_t edge_cap, del_cap;
};

// pinned layout of a wave's small block: the status word and totals, then
// the set offsets and boxes handed to the device
struct SmallLayout { uint64_t err, totals, set_ptr, boxes, total; };

SmallLayout small_layout(int S) {
    SmallLayout L;
    uint64_t at = 0;
    L.err = at;     at = al(at + 8);
    L.totals = at;  at = al(at + 16);
    L.set_ptr = at; at = al(at + (uint64_t)(S + 1) * 8);
    L.boxes = at;   at = al(at + (uint64_t)S * 8);
    L.total = at;
    return L;
}

struct Wave {
    std::vector<Request *> reqs;
    std::vector<int64_t> set_ptr;
    std::vector<vor_box> boxes;
    int64_t N = 0;
    int S = 0;
    int stream = -1;
    cudaEvent_t ev = nullptr;
    int phase = 0;                 // 1: building, 2: copying results out
    uint64_t dev_off = 0, small_off = 0;
    WaveLayout L{};
    SmallLayout SL{};
    std::shared_ptr<HostResult> res;
    int64_t E = 0, D = 0;
    uint64_t r_cell = 0, r_lab = 0, r_vx = 0, r_vy = 0, r_del = 0, r_dsp = 0, r_eb = 0;
};

}  // namespace
}  // namespace vor

using namespace vor;

struct vor_server {
    vor_server_config cfg{};
    int device = 0;
    char *dev_base = nullptr;
    char *host_base = nullptr;
    Arena dev_arena, host_arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::vector<cudaEvent_t> events;
    std::mutex mu;
    std::condition_variable cv_work;   // dispatcher: new requests or stop
    std::condition_variable cv_done;   // clients: completions, room in the pinned block
    std::deque<Request *> pending;
    std::vector<std::unique_ptr<Wave>> inflight;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread thr;
    std::chrono::steady_clock::time_point t0;
    int64_t host_allocs = 0;
    vor_server_stats st{};

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // device bytes of a wave of the first k pending requests
    bool wave_layout(const std::vector<Request *> &rs, int k, WaveLayout &L,
                     std::vector<int64_t> &ptr, std::vector<vor_box> &bx) const {
        ptr.assign(k + 1, 0);
        bx.resize(k);
        for (int j = 0; j < k; j++) {
            ptr[j + 1] = ptr[j] + rs[j]->n;
            bx[j] = rs[j]->box;
        }
        const int64_t ws = vor_batch_workspace_bytes(ptr.data(), k, bx.data(), &cfg.opts);
        if (ws < 0) return false;
        const int64_t N = ptr[k];
        L.edge_cap = vor_batch_edge_capacity(N, k);
        L.del_cap = vor_batch_delaunay_capacity(N, k);
        uint64_t at = 0;
        L.ws = at;          at = al(at + (uint64_t)ws);
        L.ws_bytes = (uint64_t)ws;
        L.sites = at;       at = al(at + (uint64_t)N * 8);
        L.set_ptr = at;     at = al(at + (uint64_t)(k + 1) * 8);
        L.boxes = at;       at = al(at + (uint64_t)k * 8);
        L.cell_ptr = at;    at = al(at + (uint64_t)(N + 1) * 8);
        L.labels = at;      at = al(at + (uint64_t)L.edge_cap * 4);
        L.vx = at;          at = al(at + (uint64_t)L.edge_cap * 8);
        L.vy = at;          at = al(at + (uint64_t)L.edge_cap * 8);
        L.del = at;         at = al(at + (uint64_t)L.del_cap * 8);
        L.del_set_ptr = at; at = al(at + (uint64_t)(k + 1) * 8);
        L.totals = at;      at = al(at + 16);
        L.rebased = at;     at = al(at + (uint64_t)(N + k) * 8);
        L.edge_base = at;   at = al(at + (uint64_t)(k + 1) * 8);
        L.total = at;
        return true;
    }

    void finish_request(Request *r, int status) {
        r->status = r->cancelled ? VOR_E_CANCELLED : status;
        r->running = false;
        r->t_done = now();
        if (r->status == VOR_OK) st.completed++;
        else if (r->status == VOR_E_CANCELLED) st.cancelled++;
        else st.failed++;
        if (r->status != VOR_OK && r->res) {
            drop_result(r);
        }
    }

    void drop_result(Request *r) {
        if (!r->res) return;
        if (--r->res->refs == 0) host_arena.release(r->res->off);
        r->res.reset();
        r->cell_ptr = nullptr;
        r->labels = nullptr;
        r->vx = r->vy = nullptr;
        r->del = nullptr;
    }

    void unstage(Request *r) {
        if (r->staged) {
            host_arena.release(r->in_off);
            r->staged = false;
        }
    }

    void release_wave(Wave &w) {
        dev_arena.release(w.dev_off);
        host_arena.release(w.small_off);
        stream_busy[w.stream] = false;
    }

    // launch a wave of the first k pending requests (lock held)
    bool launch(int k) {
        std::unique_ptr<Wave> w(new Wave);
        for (int j = 0; j < k; j++) w->reqs.push_back(pending[j]);
        if (!wave_layout(w->reqs, k, w->L, w->set_ptr, w->boxes)) return false;
        w->S = k;
        w->N = w->set_ptr[k];
        w->SL = small_layout(k);
        if (!dev_arena.alloc(w->L.total, &w->dev_off)) return false;
        if (!host_arena.alloc(w->SL.total, &w->small_off)) {
            dev_arena.release(w->dev_off);
            return false;
        }
        int si = -1;
        for (int i = 0; i < (int)streams.size(); i++)
            if (!stream_busy[i]) { si = i; break; }
        if (si < 0) {
            dev_arena.release(w->dev_off);
            host_arena.release(w->small_off);
            return false;
        }
        stream_busy[si] = true;
        w->stream = si;
        w->ev = events[si];
        for (int j = 0; j < k; j++) pending.pop_front();
        cudaStream_t stm = streams[si];
        char *d = dev_base + w->dev_off;
        char *hs = host_base + w->small_off;
        std::memcpy(hs + w->SL.set_ptr, w->set_ptr.data(), (size_t)(k + 1) * 8);
        std::memcpy(hs + w->SL.boxes, w->boxes.data(), (size_t)k * 8);
        const double t = now();
        for (Request *r : w->reqs) {
            r->running = true;
            r->t_start = t;
            r->wave_requests = k;
        }
        st.waves++;
        if (k > st.max_wave_requests_seen) st.max_wave_requests_seen = k;
        bool ok = cudaMemcpyAsync(d + w->L.set_ptr, hs + w->SL.set_ptr, (size_t)(k + 1) * 8,
                                  cudaMemcpyHostToDevice, stm) == cudaSuccess &&
                  cudaMemcpyAsync(d + w->L.boxes, hs + w->SL.boxes, (size_t)k * 8,
                                  cudaMemcpyHostToDevice, stm) == cudaSuccess;
        for (int j = 0; j < k && ok; j++) {
            Request *r = w->reqs[j];
            if (r->n > 0)
                ok = cudaMemcpyAsync(d + w->L.sites + (size_t)w->set_ptr[j] * 8, host_base + r->in_off,
                                     (size_t)r->n * 8, cudaMemcpyHostToDevice, stm) == cudaSuccess;
        }
        int rc = VOR_OK;
        if (ok) {
            vor_out out;
            out.cell_ptr = (int64_t *)(d + w->L.cell_ptr);
            out.edge_label = (int32_t *)(d + w->L.labels);
            out.vx = (double *)(d + w->L.vx);
            out.vy = (double *)(d + w->L.vy);
            out.del_edge = (int32_t *)(d + w->L.del);
            out.totals = (int64_t *)(d + w->L.totals);
            out.edge_cap = w->L.edge_cap;
            out.del_cap = w->L.del_cap;
            rc = vor_build_batch_async((const vor_site *)(d + w->L.sites),
                                       (const int64_t *)(d + w->L.set_ptr), w->set_ptr.data(), k,
                                       (const vor_box *)(d + w->L.boxes), w->boxes.data(), &cfg.opts,
                                       d + w->L.ws, (int64_t)w->L.ws_bytes, &out,
                                       (int64_t *)(d + w->L.del_set_ptr), stm);
            if (rc == VOR_OK) {
                const long long items = w->N + k;
                const int T = 256;
                const long long blocks = (std::max(items, (long long)k + 1) + T - 1) / T;
                k_rebase<<<(unsigned)blocks, T, 0, stm>>>(
                    (const long long *)(d + w->L.cell_ptr), (const long long *)(d + w->L.set_ptr), k,
                    items, (long long *)(d + w->L.rebased), (long long *)(d + w->L.edge_base),
                    (const WsHeader *)(d + w->L.ws));
                ok = cudaGetLastError() == cudaSuccess &&
                     cudaMemcpyAsync(hs + w->SL.err, d + w->L.ws, 4, cudaMemcpyDeviceToHost, stm) ==
                         cudaSuccess &&
                     cudaMemcpyAsync(hs + w->SL.totals, d + w->L.totals, 16, cudaMemcpyDeviceToHost,
                                     stm) == cudaSuccess;
            }
        }
        if (!ok || rc != VOR_OK) {
            // the wave never ran: its requests fail (argument errors) or are
            // retried alone (CUDA errors of a batch)
            cudaStreamSynchronize(stm);
            release_wave(*w);
            for (Request *r : w->reqs) {
                unstage(r);
                finish_request(r, ok ? rc : VOR_E_CUDA);
            }
            cv_done.notify_all();
            return true;
        }
        cudaEventRecord(w->ev, stm);
        w->phase = 1;
        inflight.push_back(std::move(w));
        return true;
    }

    // a wave's build finished: status, sizes, results out (lock held)
    void on_built(Wave &w) {
        const char *hs = host_base + w.small_off;
        unsigned err = 0;
        std::memcpy(&err, hs + w.SL.err, 4);
        int64_t tot[2];
        std::memcpy(tot, hs + w.SL.totals, 16);
        const int status = status_of_error_bits(err);
        if (status != VOR_OK) {
            release_wave(w);
            w.phase = 3;
            if (w.S > 1) {
                // split: every request again, alone, at the head of the queue
                // (their sites are still staged)
                st.split_waves++;
                for (int j = w.S - 1; j >= 0; j--) {
                    Request *r = w.reqs[j];
                    r->running = false;
                    r->solo = true;
                    if (r->cancelled) {
                        unstage(r);
                        finish_request(r, VOR_E_CANCELLED);
                        continue;
                    }
                    pending.push_front(r);
                }
            } else {
                unstage(w.reqs[0]);
                finish_request(w.reqs[0], status);
            }
            cv_done.notify_all();
            return;
        }
        for (Request *r : w.reqs) unstage(r);
        w.E = tot[0];
        w.D = tot[1];
        uint64_t at = 0;
        w.r_cell = at; at = al(at + (uint64_t)(w.N + w.S) * 8);
        w.r_lab = at;  at = al(at + (uint64_t)w.E * 4);
        w.r_vx = at;   at = al(at + (uint64_t)w.E * 8);
        w.r_vy = at;   at = al(at + (uint64_t)w.E * 8);
        w.r_del = at;  at = al(at + (uint64_t)w.D * 8);
        w.r_dsp = at;  at = al(at + (uint64_t)(w.S + 1) * 8);
        w.r_eb = at;   at = al(at + (uint64_t)(w.S + 1) * 8);
        uint64_t off = 0;
        host_allocs++;
        const bool injected = cfg.fail_host_alloc_at > 0 && host_allocs == cfg.fail_host_alloc_at;
        if (injected || !host_arena.alloc(at, &off)) {
            if (!injected && host_arena.size() >= at) {
                // no room yet: retry when clients release results
                w.phase = 4;
                return;
            }
            release_wave(w);
            w.phase = 3;
            for (Request *r : w.reqs) finish_request(r, VOR_E_OOM);
            cv_done.notify_all();
            return;
        }
        w.res = std::make_shared<HostResult>();
        w.res->off = off;
        w.res->refs = w.S;
        char *h = host_base + off;
        const char *d = dev_base + w.dev_off;
        cudaStream_t stm = streams[w.stream];
        bool ok =
            cudaMemcpyAsync(h + w.r_cell, d + w.L.rebased, (size_t)(w.N + w.S) * 8,
                            cudaMemcpyDeviceToHost, stm) == cudaSuccess &&
            (w.E == 0 ||
             (cudaMemcpyAsync(h + w.r_lab, d + w.L.labels, (size_t)w.E * 4, cudaMemcpyDeviceToHost, stm) ==
                  cudaSuccess &&
              cudaMemcpyAsync(h + w.r_vx, d + w.L.vx, (size_t)w.E * 8, cudaMemcpyDeviceToHost, stm) ==
                  cudaSuccess &&
              cudaMemcpyAsync(h + w.r_vy, d + w.L.vy, (size_t)w.E * 8, cudaMemcpyDeviceToHost, stm) ==
                  cudaSuccess)) &&
            (w.D == 0 || cudaMemcpyAsync(h + w.r_del, d + w.L.del, (size_t)w.D * 8,
                                         cudaMemcpyDeviceToHost, stm) == cudaSuccess) &&
            cudaMemcpyAsync(h + w.r_dsp, d + w.L.del_set_ptr, (size_t)(w.S + 1) * 8,
                            cudaMemcpyDeviceToHost, stm) == cudaSuccess &&
            cudaMemcpyAsync(h + w.r_eb, d + w.L.edge_base, (size_t)(w.S + 1) * 8,
                            cudaMemcpyDeviceToHost, stm) == cudaSuccess &&
            cudaEventRecord(w.ev, stm) == cudaSuccess;
        if (!ok) {
            cudaStreamSynchronize(stm);
            host_arena.release(off);
            w.res.reset();
            release_wave(w);
            w.phase = 3;
            for (Request *r : w.reqs) finish_request(r, VOR_E_CUDA);
            cv_done.notify_all();
            return;
        }
        w.phase = 2;
    }

    // a wave's results are on the host (lock held)
    void on_copied(Wave &w) {
        const char *h = host_base + w.res->off;
        const int64_t *eb = (const int64_t *)(h + w.r_eb);
        const int64_t *dsp = (const int64_t *)(h + w.r_dsp);
        for (int j = 0; j < w.S; j++) {
            Request *r = w.reqs[j];
            r->res = w.res;
            r->cell_ptr = (const int64_t *)(h + w.r_cell) + w.set_ptr[j] + j;
            r->labels = (const int32_t *)(h + w.r_lab) + eb[j];
            r->vx = (const double *)(h + w.r_vx) + eb[j];
            r->vy = (const double *)(h + w.r_vy) + eb[j];
            r->del = (const int32_t *)(h + w.r_del) + 2 * dsp[j];
            r->n_edges = eb[j + 1] - eb[j];
            r->n_del = dsp[j + 1] - dsp[j];
            finish_request(r, VOR_OK);
        }
        release_wave(w);
        w.phase = 3;
        cv_done.notify_all();
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lock(mu);
        while (true) {
            bool progress = false;
            for (auto &wp : inflight) {
                Wave &w = *wp;
                if (w.phase == 4) {                      // waiting for host room
                    w.phase = 1;
                    on_built(w);
                    if (w.phase != 4) progress = true;
                    continue;
                }
                if (w.phase != 1 && w.phase != 2) continue;
                const cudaError_t q = cudaEventQuery(w.ev);
                if (q == cudaErrorNotReady) continue;
                progress = true;
                if (q != cudaSuccess) {
                    cudaStreamSynchronize(streams[w.stream]);
                    if (w.res) { host_arena.release(w.res->off); w.res.reset(); }
                    for (Request *r : w.reqs) { unstage(r); finish_request(r, VOR_E_CUDA); }
                    release_wave(w);
                    w.phase = 3;
                    cv_done.notify_all();
                    continue;
                }
                if (w.phase == 1) on_built(w);
                else on_copied(w);
            }
            inflight.erase(std::remove_if(inflight.begin(), inflight.end(),
                                          [](const std::unique_ptr<Wave> &w) { return w->phase == 3; }),
                           inflight.end());
            // new waves while streams are free
            while (!pending.empty() && (int)inflight.size() < cfg.max_inflight) {
                std::vector<int64_t> sizes;
                const int lim = pending.front()->solo ? 1 : cfg.max_wave_requests;
                for (int j = 0; j < (int)pending.size() && j < lim; j++) {
                    if (j > 0 && pending[j]->solo) break;
                    sizes.push_back(pending[j]->n);
                }
                std::vector<Request *> head(pending.begin(), pending.begin() + sizes.size());
                WaveLimits wl{lim, cfg.max_wave_sites};
                const uint64_t room = dev_arena.largest_free();
                const int k = plan_wave(sizes, wl, room, [&](int kk) -> uint64_t {
                    WaveLayout L;
                    std::vector<int64_t> p;
                    std::vector<vor_box> b;
                    return wave_layout(head, kk, L, p, b) ? L.total : ~0ull;
                });
                if (k == 0 || !launch(k)) break;
                progress = true;
            }
            st.pending = (int64_t)pending.size();
            st.inflight = (int64_t)inflight.size();
            if (stop && inflight.empty() && pending.empty()) break;
            if (!progress) {
                if (inflight.empty() && pending.empty()) cv_work.wait(lock);
                else cv_work.wait_for(lock, std::chrono::microseconds(20));
            }
        }
    }
};

extern "C" {

void vor_server_config_default(vor_server_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->device_bytes = (int64_t)16 << 30;
    c->host_bytes = (int64_t)4 << 30;
    c->max_inflight = 4;
    c->max_wave_requests = 64;
    c->max_wave_sites = (int64_t)8 << 20;
    vor_opts_default(&c->opts);
    c->fail_host_alloc_at = 0;
}

int vor_server_create(const vor_server_config *cfg, vor_server **out) {
    if (!cfg || !out) return VOR_E_INVALID_ARG;
    *out = nullptr;
    if (cfg->device_bytes < (1 << 20) || cfg->host_bytes < (1 << 20) || cfg->max_inflight < 1 ||
        cfg->max_inflight > 64 || cfg->max_wave_requests < 1 || cfg->max_wave_sites < 1)
        return VOR_E_INVALID_ARG;
    {
        vor_box b{1 << 20, 1 << 20};
        if (vor_workspace_bytes(1, b, &cfg->opts) < 0) return VOR_E_INVALID_ARG;
    }
    std::unique_ptr<vor_server> s(new vor_server);
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) return VOR_E_CUDA;
    if (cudaMalloc((void **)&s->dev_base, (size_t)cfg->device_bytes) != cudaSuccess) {
        cudaGetLastError();
        return VOR_E_OOM;
    }
    if (cudaHostAlloc((void **)&s->host_base, (size_t)cfg->host_bytes, cudaHostAllocDefault) !=
        cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->dev_base);
        return VOR_E_OOM;
    }
    s->dev_arena.reset((uint64_t)cfg->device_bytes, kAlign);
    s->host_arena.reset((uint64_t)cfg->host_bytes, kAlign);
    for (int i = 0; i < cfg->max_inflight; i++) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            for (auto x : s->events) cudaEventDestroy(x);
            cudaFree(s->dev_base);
            cudaFreeHost(s->host_base);
            return VOR_E_CUDA;
        }
        s->streams.push_back(st);
        s->events.push_back(ev);
        s->stream_busy.push_back(false);
    }
    s->t0 = std::chrono::steady_clock::now();
    vor_server *raw = s.release();
    raw->thr = std::thread([raw] { raw->loop(); });
    *out = raw;
    return VOR_OK;
}

int vor_server_submit(vor_server *s, const vor_site *h_sites, int64_t n, vor_box box,
                      double timeout_s, uint64_t *ticket) {
    if (!s || !ticket || n < 0 || (n > 0 && !h_sites)) return VOR_E_INVALID_ARG;
    if (box.w < 2 || box.h < 2 || box.w > (1 << 20) || box.h > (1 << 20)) return VOR_E_BOX_TOO_LARGE;
    if (n > (1 << 27)) return VOR_E_SERVER_FULL;
    // the request alone must fit both budgets
    {
        std::vector<Request *> one;
        Request probe;
        probe.n = n;
        probe.box = box;
        one.push_back(&probe);
        WaveLayout L;
        std::vector<int64_t> p;
        std::vector<vor_box> b;
        if (!s->wave_layout(one, 1, L, p, b)) return VOR_E_INVALID_ARG;
        const uint64_t host_need = al((uint64_t)n * 8) + small_layout(1).total +
                                   al((uint64_t)(n + 1) * 8) + (uint64_t)L.edge_cap * 20 +
                                   (uint64_t)L.del_cap * 8 + 8 * kAlign;
        if (L.total > s->dev_arena.size() || host_need > s->host_arena.size()) return VOR_E_SERVER_FULL;
    }
    std::unique_ptr<Request> r(new Request);
    r->n = n;
    r->box = box;
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    while (!s->host_arena.alloc((uint64_t)(n > 0 ? n : 1) * 8, &r->in_off)) {
        if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
            if (!s->host_arena.alloc((uint64_t)(n > 0 ? n : 1) * 8, &r->in_off))
                return VOR_E_SERVER_FULL;
            break;
        }
    }
    r->staged = true;
    if (n > 0) std::memcpy(s->host_base + r->in_off, h_sites, (size_t)n * 8);
    r->id = s->next_id++;
    r->t_submit = s->now();
    *ticket = r->id;
    s->pending.push_back(r.get());
    s->reqs[r->id] = std::move(r);
    s->st.submitted++;
    s->cv_work.notify_one();
    return VOR_OK;
}

static void fill_result(const Request *r, vor_request_result *res) {
    if (!res) return;
    std::memset(res, 0, sizeof(*res));
    res->status = r->status;
    res->wave_requests = r->wave_requests;
    res->n = r->n;
    res->t_submit = r->t_submit;
    res->t_start = r->t_start;
    res->t_done = r->t_done;
    if (r->status == VOR_OK) {
        res->n_edges = r->n_edges;
        res->n_del = r->n_del;
        res->cell_ptr = r->cell_ptr;
        res->edge_label = r->labels;
        res->vx = r->vx;
        res->vy = r->vy;
        res->del_edge = r->del;
    }
}

int vor_server_poll(vor_server *s, uint64_t ticket, vor_request_result *res) {
    if (!s) return VOR_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VOR_E_INVALID_ARG;
    fill_result(it->second.get(), res);
    return it->second->status;
}

int vor_server_wait(vor_server *s, uint64_t ticket, double timeout_s, vor_request_result *res) {
    if (!s) return VOR_E_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    while (true) {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return VOR_E_INVALID_ARG;
        if (it->second->status != VOR_PENDING) {
            fill_result(it->second.get(), res);
            return it->second->status;
        }
        if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
            auto it2 = s->reqs.find(ticket);
            if (it2 != s->reqs.end() && it2->second->status != VOR_PENDING) {
                fill_result(it2->second.get(), res);
                return it2->second->status;
            }
            if (it2 == s->reqs.end()) return VOR_E_INVALID_ARG;
            fill_result(it2->second.get(), res);
            return VOR_E_TIMEOUT;
        }
    }
}

int vor_server_cancel(vor_server *s, uint64_t ticket) {
    if (!s) return VOR_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VOR_E_INVALID_ARG;
    Request *r = it->second.get();
    if (r->status != VOR_PENDING) return VOR_OK;        // already final
    r->cancelled = true;
    if (!r->running) {
        auto p = std::find(s->pending.begin(), s->pending.end(), r);
        if (p != s->pending.end()) s->pending.erase(p);
        s->unstage(r);
        s->finish_request(r, VOR_E_CANCELLED);
        s->cv_done.notify_all();
    }
    return VOR_OK;
}

int vor_server_release(vor_server *s, uint64_t ticket) {
    if (!s) return VOR_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VOR_E_INVALID_ARG;
    Request *r = it->second.get();
    if (r->status == VOR_PENDING) return VOR_PENDING;
    s->drop_result(r);
    s->reqs.erase(it);
    s->cv_done.notify_all();
    s->cv_work.notify_one();                             // a wave may wait for host room
    return VOR_OK;
}

int vor_server_statistics(vor_server *s, vor_server_stats *out) {
    if (!s || !out) return VOR_E_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    out->pending = (int64_t)s->pending.size();
    out->inflight = (int64_t)s->inflight.size();
    out->device_free = (int64_t)s->dev_arena.free_bytes();
    out->device_largest_free = (int64_t)s->dev_arena.largest_free();
    out->host_free = (int64_t)s->host_arena.free_bytes();
    return VOR_OK;
}

double vor_server_now(const vor_server *s) { return s ? s->now() : 0.0; }

int vor_server_destroy(vor_server *s) {
    if (!s) return VOR_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        // waiting requests are cancelled; running waves finish
        while (!s->pending.empty()) {
            Request *r = s->pending.front();
            s->pending.pop_front();
            r->cancelled = true;
            s->unstage(r);
            s->finish_request(r, VOR_E_CANCELLED);
        }
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->thr.join();
    for (auto x : s->streams) cudaStreamDestroy(x);
    for (auto x : s->events) cudaEventDestroy(x);
    cudaFree(s->dev_base);
    cudaFreeHost(s->host_base);
    delete s;
    return VOR_OK;
}

}  // extern "C"
