// apax_server.cu -- request serving with continuous batching.
//
// Requests (encode or decode of one array) are queued on the host.  Each
// poll retires the steps whose CUDA event has completed, then admits queued
// requests (first come, first served) while a step slot is free and the
// device arena has room for their outputs and workspace, and launches them
// as one step: one batched encode launch and one batched decode launch on
// the slot's stream.  Steps on different slots overlap on the device, so
// requests that arrive while others run join the next step instead of
// waiting for the GPU to drain.  The arena is caller-owned device memory
// (its size is the admission cap); job tables go up from pinned staging
// with asynchronous copies, and results come back through mapped pinned
// memory, so a poll never blocks on the device.
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <vector>

#include "apax_plan.h"

using namespace apax;
using namespace apax::host;

namespace {

constexpr uint64_t kArenaAlign = 256;

// First-fit allocator over [0, size) with coalescing of free ranges.
struct Arena {
    uint64_t size = 0, used = 0, peak = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> length
    void init(uint64_t s)
    {
        size = s;
        used = peak = 0;
        free_.clear();
        if (s) free_[0] = s;
    }
    bool alloc(uint64_t want, uint64_t &off)
    {
        want = (want + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        if (want == 0) want = kArenaAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= want) {
                off = it->first;
                const uint64_t rest = it->second - want;
                free_.erase(it);
                if (rest) free_[off + want] = rest;
                used += want;
                if (used > peak) peak = used;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t want)
    {
        want = (want + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        if (want == 0) want = kArenaAlign;
        used -= want;
        auto it = free_.emplace(off, want).first;
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
};

struct Req {
    apax_request r;
    double t_submit;
    uint64_t out_bytes;   // bytes to allocate for the output (0: caller's buffer)
    uint64_t ws_est;      // batch workspace share
    uint64_t out_off;     // arena offset of a server-allocated output
    void *out;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t *pinned = nullptr;      // job-table staging
    uint64_t pinned_bytes = 0;
    apax_result *res_host = nullptr;  // mapped pinned results
    apax_result *res_dev = nullptr;
    bool busy = false;
    std::vector<Req> reqs;
    uint64_t ws_off = 0, ws_bytes = 0;
    apax_batch *enc = nullptr, *dec = nullptr;
    double t_launch = 0;
};

double now_s(const std::chrono::steady_clock::time_point &t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct apax_server {
    apax_server_config cfg;
    uint8_t *arena_base;
    Arena arena;
    std::deque<Req> queue;
    std::vector<Slot> slots;
    std::deque<apax_completion> done;
    std::map<void *, std::pair<uint64_t, uint64_t>> outputs;  // server-allocated outputs
    std::chrono::steady_clock::time_point t0;
    uint64_t steps = 0, admitted = 0, completed = 0;
};

namespace {

// Output bytes and a batch-workspace bound of one request (host checks of
// the single-array call).
int size_request(const apax_request &r, uint64_t &out_bytes, uint64_t &ws_est)
{
    if (r.op == APAX_OP_ENCODE) {
        uint64_t cap;
        int st = apax_encoded_size(r.dtype, r.n, &r.p, &cap);
        if (st) return st;
        if (r.out && r.out_capacity < cap) return APAX_ERR_CAPACITY;
        out_bytes = r.out ? 0 : cap;
        apax_encode_job j;
        memset(&j, 0, sizeof j);
        j.x = r.in ? r.in : (const void *)(uintptr_t)256;
        j.dtype = r.dtype;
        j.n = r.n;
        j.p = r.p;
        j.out = r.out ? r.out : (void *)(uintptr_t)256;
        j.out_capacity = cap;
        j.res = (apax_result *)(uintptr_t)256;
        if (!r.in && r.n) return APAX_ERR_INVALID_ARG;
        ws_est = batch_workspace_bytes(0, &j, 1);
        return ws_est ? APAX_OK : APAX_ERR_INVALID_ARG;
    }
    if (r.op == APAX_OP_DECODE) {
        Fmt f;
        int st = fmt_of(r.dtype, f);
        if (st) return st;
        if (!block_size_ok(r.p.block_size)) return APAX_ERR_BLOCK_SIZE;
        if ((!r.in && r.in_bytes) || ((uintptr_t)r.in & 3)) return APAX_ERR_INVALID_ARG;
        const uint64_t need = r.n * (uint64_t)f.size;
        if (r.out && r.out_capacity < need) return APAX_ERR_CAPACITY;
        out_bytes = r.out ? 0 : need;
        apax_decode_job j;
        memset(&j, 0, sizeof j);
        j.in = r.in;
        j.in_bytes = r.in_bytes;
        j.y = r.out ? r.out : (void *)(uintptr_t)256;
        j.dtype = r.dtype;
        j.block_size = r.p.block_size;
        j.n = r.n;
        j.res = (apax_result *)(uintptr_t)256;
        ws_est = batch_workspace_bytes(1, &j, 1);
        return ws_est ? APAX_OK : APAX_ERR_INVALID_ARG;
    }
    return APAX_ERR_INVALID_ARG;
}

void retire(apax_server *s, Slot &sl)
{
    const double t = now_s(s->t0);
    const int k = (int)sl.reqs.size();
    int ie = 0, id = 0;
    const int ne = [&] {
        int c = 0;
        for (const Req &q : sl.reqs) c += q.r.op == APAX_OP_ENCODE;
        return c;
    }();
    for (int i = 0; i < k; ++i) {
        const Req &q = sl.reqs[i];
        const int slot = q.r.op == APAX_OP_ENCODE ? ie++ : ne + id++;
        volatile apax_result *rr = sl.res_host + slot;
        apax_completion c;
        memset(&c, 0, sizeof c);
        c.id = q.r.id;
        c.op = q.r.op;
        c.status = rr->status;
        c.bytes = rr->bytes;
        c.out = q.out;
        c.t_arrival = q.r.t_arrival > 0 ? q.r.t_arrival : q.t_submit;
        c.t_submit = q.t_submit;
        c.t_launch = sl.t_launch;
        c.t_done = t;
        s->done.push_back(c);
        if (q.out_bytes) {
            if (c.status != APAX_OK) {
                s->arena.release(q.out_off, q.out_bytes);  // nothing to hand over
                s->done.back().out = nullptr;
            } else {
                s->outputs[q.out] = std::make_pair(q.out_off, q.out_bytes);
            }
        }
    }
    s->completed += k;
    if (sl.enc) apax_batch_destroy(sl.enc);
    if (sl.dec) apax_batch_destroy(sl.dec);
    sl.enc = sl.dec = nullptr;
    if (sl.ws_bytes) s->arena.release(sl.ws_off, sl.ws_bytes);
    sl.ws_bytes = 0;
    sl.reqs.clear();
    sl.busy = false;
}

// Admit queued requests into one step on a free slot.  Returns the number
// admitted (0: nothing fits or nothing queued), or a negative status.
int admit(apax_server *s, Slot &sl)
{
    std::vector<Req> take;
    while (!s->queue.empty() && (int)take.size() < (int)s->cfg.max_batch) {
        Req q = s->queue.front();
        uint64_t off = 0;
        if (q.out_bytes && !s->arena.alloc(q.out_bytes, off)) break;
        q.out_off = off;
        q.out = q.out_bytes ? (void *)(s->arena_base + off) : q.r.out;
        take.push_back(q);
        s->queue.pop_front();
    }
    // jobs: encodes first, then decodes (result slots in that order); the
    // step's exact workspace, giving back the newest requests until it fits
    std::vector<apax_encode_job> ej;
    std::vector<apax_decode_job> dj;
    uint64_t ws_enc = 0, ws_dec = 0;
    while (!take.empty()) {
        ej.clear();
        dj.clear();
        for (const Req &q : take) {
            if (q.r.op != APAX_OP_ENCODE) continue;
            apax_encode_job j;
            memset(&j, 0, sizeof j);
            j.x = q.r.in;
            j.dtype = q.r.dtype;
            j.n = q.r.n;
            j.p = q.r.p;
            j.out = q.out;
            j.out_capacity = q.out_bytes ? q.out_bytes : q.r.out_capacity;
            ej.push_back(j);
        }
        for (const Req &q : take) {
            if (q.r.op != APAX_OP_DECODE) continue;
            apax_decode_job j;
            memset(&j, 0, sizeof j);
            j.in = q.r.in;
            j.in_bytes = q.r.in_bytes;
            j.y = q.out;
            j.dtype = q.r.dtype;
            j.block_size = q.r.p.block_size;
            j.n = q.r.n;
            dj.push_back(j);
        }
        for (size_t i = 0; i < ej.size(); ++i) ej[i].res = sl.res_dev + i;
        for (size_t i = 0; i < dj.size(); ++i) dj[i].res = sl.res_dev + ej.size() + i;
        ws_enc = ej.empty() ? 0 : batch_workspace_bytes(0, ej.data(), (int)ej.size());
        ws_dec = dj.empty() ? 0 : batch_workspace_bytes(1, dj.data(), (int)dj.size());
        const uint64_t want = ws_enc + ws_dec + 2 * kArenaAlign;
        uint64_t off;
        if (s->arena.alloc(want, off)) {
            sl.ws_off = off;
            sl.ws_bytes = want;
            break;
        }
        Req q = take.back();
        take.pop_back();
        if (q.out_bytes) s->arena.release(q.out_off, q.out_bytes);
        s->queue.push_front(q);
    }
    if (take.empty()) return 0;
    uint8_t *ws = s->arena_base + sl.ws_off;
    uint8_t *ws_e = (uint8_t *)(((uintptr_t)ws + kArenaAlign - 1) / kArenaAlign * kArenaAlign);
    uint8_t *ws_d = ws_e + (ws_enc + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    int st_e = APAX_OK, st_d = APAX_OK;
    const uint64_t half = sl.pinned_bytes / 2;
    if (!ej.empty()) {
        st_e = batch_create(0, ej.data(), (int)ej.size(), ws_e, ws_enc, sl.pinned, half, sl.stream,
                            true, &sl.enc);
        if (!st_e) st_e = apax_batch_run(sl.enc, sl.stream);
    }
    if (!dj.empty()) {
        st_d = batch_create(1, dj.data(), (int)dj.size(), ws_d, ws_dec, sl.pinned + half, half,
                            sl.stream, true, &sl.dec);
        if (!st_d) st_d = apax_batch_run(sl.dec, sl.stream);
    }
    sl.reqs.swap(take);
    sl.busy = true;
    sl.t_launch = now_s(s->t0);
    s->steps += 1;
    s->admitted += sl.reqs.size();
    const bool rec_ok = cudaEventRecord(sl.done, sl.stream) == cudaSuccess;
    if (st_e || st_d || !rec_ok) {
        // drain what was enqueued, then report the part that was not
        cudaStreamSynchronize(sl.stream);
        const int st_r = rec_ok ? APAX_OK : APAX_ERR_CUDA;
        for (size_t i = 0; i < ej.size() + dj.size(); ++i) {
            const int st = i < ej.size() ? (st_e ? st_e : st_r) : (st_d ? st_d : st_r);
            if (st) {
                sl.res_host[i].status = st;
                sl.res_host[i].bytes = 0;
            }
        }
        if (!rec_ok) retire(s, sl);
        return st_e ? st_e : (st_d ? st_d : (rec_ok ? (int)sl.reqs.size() : APAX_ERR_CUDA));
    }
    return (int)sl.reqs.size();
}

void destroy_server(apax_server *s)
{
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.enc) apax_batch_destroy(sl.enc);
        if (sl.dec) apax_batch_destroy(sl.dec);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        if (sl.res_host) cudaFreeHost(sl.res_host);
    }
    delete s;
}

}  // namespace

extern "C" {

int apax_server_create(const apax_server_config *cfg, apax_server **out)
{
    if (!cfg || !out) return APAX_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg->arena || !cfg->arena_bytes || ((uintptr_t)cfg->arena % kArenaAlign))
        return APAX_ERR_INVALID_ARG;
    if (cfg->slots < 1 || cfg->slots > 64 || cfg->max_batch < 1 || cfg->max_batch > 65536)
        return APAX_ERR_INVALID_ARG;
    apax_server *s = new apax_server();
    s->cfg = *cfg;
    s->arena_base = (uint8_t *)cfg->arena;
    s->arena.init(cfg->arena_bytes);
    s->t0 = std::chrono::steady_clock::now();
    s->slots.resize(cfg->slots);
    // per slot: job-table staging (encode and decode halves) and results
    const uint64_t table = (uint64_t)cfg->max_batch * (sizeof(EncArgs) + 64) + (1 << 16);
    for (Slot &sl : s->slots) {
        sl.pinned_bytes = 2 * table;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.pinned, sl.pinned_bytes, cudaHostAllocDefault) !=
                cudaSuccess ||
            cudaHostAlloc((void **)&sl.res_host, sizeof(apax_result) * cfg->max_batch,
                          cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&sl.res_dev, sl.res_host, 0) != cudaSuccess) {
            destroy_server(s);
            return APAX_ERR_CUDA;
        }
    }
    *out = s;
    return APAX_OK;
}

int apax_server_submit(apax_server *s, const apax_request *r)
{
    if (!s || !r) return APAX_ERR_INVALID_ARG;
    Req q;
    memset(&q, 0, sizeof q);
    q.r = *r;
    int st = size_request(*r, q.out_bytes, q.ws_est);
    if (st) return st;
    // a request that could never fit the arena is refused at once
    if (q.out_bytes + q.ws_est + 4 * kArenaAlign > s->arena.size) return APAX_ERR_CAPACITY;
    q.t_submit = now_s(s->t0);
    s->queue.push_back(q);
    return APAX_OK;
}

int apax_server_poll(apax_server *s, apax_completion *out, int max_out, int *n_out)
{
    if (!s || (max_out > 0 && !out) || !n_out) return APAX_ERR_INVALID_ARG;
    int st = APAX_OK;
    for (Slot &sl : s->slots) {
        if (!sl.busy) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaSuccess) retire(s, sl);
        else if (e != cudaErrorNotReady) st = APAX_ERR_CUDA;
    }
    for (Slot &sl : s->slots) {
        if (sl.busy || s->queue.empty()) continue;
        const int a = admit(s, sl);
        if (a < 0) st = a;
        if (a == 0) break;  // the queue head does not fit yet
    }
    int k = 0;
    while (k < max_out && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = k;
    return st;
}

int apax_server_release(apax_server *s, void *out)
{
    if (!s) return APAX_ERR_INVALID_ARG;
    auto it = s->outputs.find(out);
    if (it == s->outputs.end()) return APAX_ERR_INVALID_ARG;
    s->arena.release(it->second.first, it->second.second);
    s->outputs.erase(it);
    return APAX_OK;
}

int apax_server_stats(const apax_server *s, apax_server_stats_t *st)
{
    if (!s || !st) return APAX_ERR_INVALID_ARG;
    memset(st, 0, sizeof *st);
    st->queued = s->queue.size();
    for (const Slot &sl : s->slots) {
        if (!sl.busy) continue;
        st->inflight += sl.reqs.size();
        st->busy_slots += 1;
    }
    st->arena_used = s->arena.used;
    st->arena_peak = s->arena.peak;
    st->steps = s->steps;
    st->admitted = s->admitted;
    st->completed = s->completed;
    st->undelivered = s->done.size();
    return APAX_OK;
}

void apax_server_destroy(apax_server *s)
{
    if (s) destroy_server(s);
}

}  // extern "C"
