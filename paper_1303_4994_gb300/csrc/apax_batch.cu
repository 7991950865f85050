// apax_batch.cu -- batched codec: many arrays of mixed dtype, length and
// parameters in one persistent launch, with a plan that lives in a
// caller-owned workspace and an autotuner for its launch geometry.
//
// A plan is built once on the host (validation, per-array tile counts, the
// descriptor table copied into the workspace).  Running it is one memset of
// the plan's counters and one kernel launch on the caller's stream, so it
// can be captured into a CUDA graph and replayed.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "apax_plan.h"

using namespace apax;
using namespace apax::host;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Launch geometries the tuner may pick for teams of 8 (blocks per tile =
// threads / 8) and teams of 32 (one block per warp).
struct Geo {
    int ts, threads;
};

}  // namespace

struct apax_batch {
    int op;  // 0 encode, 1 decode, 2 profile
    int count;
    std::vector<EncArgs> jobs;     // encode: per-array arguments, workspace pointers unset
    std::vector<DecArgs> djobs;    // decode: per-container arguments
    std::vector<uint32_t> dN;      // decode: declared block sizes
    std::vector<ProfArgs> pjobs;   // profile: per-array arguments
    ProfArgs *d_pjobs;
    int max_ncand;
    DecArgs *d_djobs;
    uint64_t *d_tiles_of;
    uint32_t *d_bsize;
    std::vector<uint32_t> gp8, gp32;
    uint32_t pkt_words, ebuf_words;
    bool need32;                   // some packet only fits teams of 32
    uint8_t *ws;
    uint64_t ws_bytes;
    // layout
    EncArgs *d_jobs;
    uint64_t *d_prefix;
    uint8_t *d_zero;               // start of the region cleared per run
    uint64_t zero_bytes;
    uint64_t total_tiles;
    apax_batch_config cfg;
    int sms;
    int dev;
    std::string key;               // tuner cache key
    // table upload: synchronous (plans), or from pinned staging on a stream
    uint8_t *pinned;
    uint64_t pinned_bytes, pinned_used;
    cudaStream_t up_stream;
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, apax_batch_config> g_tune_cache;

// Copy one table into the workspace.  A plan's copy from pageable memory
// can return before its DMA lands: the wait after it lets work on any
// stream (non-blocking ones too) see the table.
bool upload(apax_batch *b, void *dst, const void *src, size_t bytes)
{
    if (!b->pinned)
        return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaStreamSynchronize(0) == cudaSuccess;
    const size_t off = align_up(b->pinned_used, 16);
    if (off + bytes > b->pinned_bytes) return false;
    memcpy(b->pinned + off, src, bytes);
    b->pinned_used = off + bytes;
    return cudaMemcpyAsync(dst, b->pinned + off, bytes, cudaMemcpyHostToDevice, b->up_stream) ==
           cudaSuccess;
}

Geo geo_of(const apax_batch *b, const apax_batch_config &c)
{
    Geo g;
    if (b->need32) {
        g.ts = 32;
        g.threads = (int)c.threads;
    } else {
        g.ts = 8;
        g.threads = (int)c.threads;
    }
    return g;
}

// Fixed-rate arrays with blocks of at most 1024 samples are encoded one
// block per thread (the search runs without team exchanges).
bool t1_job(const EncArgs &a)
{
    return a.mode == APAX_FIXED_RATE && a.N <= kT1MaxBlock && !a.gsh && !a.sum;  // version 1 only
}

size_t pkt_smem_of(const apax_batch *b, const Geo &g)
{
    return (size_t)(g.threads / g.ts) * (b->pkt_words + b->ebuf_words) * 4;
}

// Staging of a tile for the largest block (elements x element size) of the
// batch, or 0.
size_t stage_of(const apax_batch *b, const Geo &g)
{
    bool any_fr = false;
    for (const EncArgs &a : b->jobs) any_fr |= a.mode == APAX_FIXED_RATE && !t1_job(a);
    if (!any_fr) return 0;
    uint64_t mx = 0;
    for (const EncArgs &a : b->jobs) {
        Fmt f;
        fmt_of(a.dtype, f);
        const uint64_t v = (uint64_t)a.N * f.size;
        mx = v > mx ? v : mx;
    }
    const size_t ps = pkt_smem_of(b, g);
    return stage_bytes(1, (uint32_t)mx, g.threads / g.ts, (ps + 15) / 16 * 16);
}

size_t smem_of(const apax_batch *b, const Geo &g)
{
    const size_t ps = pkt_smem_of(b, g), sb = stage_of(b, g);
    size_t sm = sb ? (ps + 15) / 16 * 16 + sb : ps;
    for (const EncArgs &a : b->jobs)  // the exponent columns of block-per-thread tiles
        if (t1_job(a)) sm = std::max(sm, (size_t)g.threads * (a.N / 4));
    return sm;
}

bool config_ok(const apax_batch *b, const apax_batch_config &c)
{
    if (b->need32) {
        if (c.threads < 32 || c.threads > 128 || (c.threads % 32)) return false;
    } else {
        if (c.threads != 64 && c.threads != 128) return false;
    }
    Geo g = geo_of(b, c);
    return pkt_smem_of(b, g) <= kEncSmemCap;
}

// Smallest tile of any allowed geometry (sizes the look-back arrays).
int min_tile_blocks(const apax_batch *b) { return b->need32 ? 1 : 8; }

// Workspace: [job table][tile prefix][ticket | done+status per job | tiles]
struct Layout {
    size_t jobs, prefix, zero, counters, tiles, total;
};

Layout layout_of(int count, const std::vector<EncArgs> &jobs, int min_tile)
{
    Layout L;
    L.jobs = 0;
    L.prefix = align_up(L.jobs + (size_t)count * sizeof(EncArgs), kAlign);
    L.zero = align_up(L.prefix + (size_t)(count + 1) * 8, kAlign);
    L.counters = L.zero + 64;  // the ticket and padding
    size_t t = align_up(L.counters + (size_t)count * 16, kAlign);
    L.tiles = t;
    uint64_t words = 0;
    for (const EncArgs &a : jobs)
        if (a.mode == APAX_FIXED_QUALITY) words += a.nb ? (a.nb + min_tile - 1) / min_tile : 1;
    L.total = align_up(t + words * 8, kAlign);
    return L;
}

int apply_decode_config(apax_batch *b, const apax_batch_config &c);
int apply_profile_config(apax_batch *b, const apax_batch_config &c);

// Rebuild the device table for a geometry (synchronous; not on a hot path).
int apply_config(apax_batch *b, const apax_batch_config &c)
{
    if (b->op == 1) return apply_decode_config(b, c);
    if (b->op == 2) return apply_profile_config(b, c);
    if (!config_ok(b, c)) return APAX_ERR_INVALID_ARG;
    const Geo g = geo_of(b, c);
    const int nteams = g.threads / g.ts;
    const Layout L = layout_of(b->count, b->jobs, min_tile_blocks(b));
    std::vector<EncArgs> tab(b->jobs);
    std::vector<uint64_t> prefix((size_t)b->count + 1, 0);
    uint64_t tiles_words = 0;
    for (int i = 0; i < b->count; ++i) {
        EncArgs &a = tab[i];
        a.pkt_words = b->pkt_words;
        a.ebuf_words = b->ebuf_words;
        a.stage_off = stage_of(b, g) ? (uint32_t)((pkt_smem_of(b, g) + 15) / 16 * 16) : 0;
        a.gp = (int)(g.ts == 8 ? b->gp8[i] : b->gp32[i]);
        a.ntiles = a.nb ? (a.nb + nteams - 1) / nteams : 1;
        a.t1 = t1_job(a) ? 1 : 0;
        if (a.t1) {  // a block per thread: tiles of `threads` blocks
            a.gp = (int)(a.N / 4);
            a.ntiles = a.nb ? (a.nb + g.threads - 1) / g.threads : 1;
        }
        a.ticket = nullptr;
        a.done = (unsigned *)(b->ws + L.counters + 16 * (size_t)i);
        a.status = (int *)(b->ws + L.counters + 16 * (size_t)i + 4);
        if (a.mode == APAX_FIXED_QUALITY) {
            a.tiles = (unsigned long long *)(b->ws + L.tiles + 8 * tiles_words);
            tiles_words += a.ntiles;
        } else {
            a.tiles = nullptr;
        }
        prefix[i + 1] = prefix[i] + a.ntiles;
    }
    b->total_tiles = prefix[b->count];
    b->d_jobs = (EncArgs *)(b->ws + L.jobs);
    b->d_prefix = (uint64_t *)(b->ws + L.prefix);
    b->d_zero = b->ws + L.zero;
    b->zero_bytes = L.tiles + 8 * tiles_words - L.zero;
    if (!upload(b, b->d_jobs, tab.data(), tab.size() * sizeof(EncArgs)) ||
        !upload(b, b->d_prefix, prefix.data(), prefix.size() * 8))
        return APAX_ERR_CUDA;
    b->cfg = c;
    if (b->cfg.ctas_per_sm == 0) {
        const int occ = encode_batch_occupancy(g.ts, g.threads, smem_of(b, g));
        b->cfg.ctas_per_sm = occ > 0 ? (uint32_t)occ : 1;
    }
    return APAX_OK;
}

apax_batch_config default_config(const apax_batch *b)
{
    apax_batch_config c;
    if (b->op != 0) {
        c.threads = 128;
        c.ctas_per_sm = 0;
        return c;
    }
    c.threads = b->need32 ? 32 : 128;
    if (b->need32) {
        const size_t per = (size_t)(b->pkt_words + b->ebuf_words) * 4;
        int w = 4;
        while (w > 1 && (size_t)w * per > kEncSmemCap) --w;
        c.threads = 32 * w;
    }
    c.ctas_per_sm = 0;
    return c;
}

int validate_encode_jobs(const apax_encode_job *jobs, int count, std::vector<EncArgs> &out,
                         std::vector<uint32_t> &gp8, std::vector<uint32_t> &gp32,
                         uint32_t &pkt_words, uint32_t &ebuf_words, bool &need32)
{
    if (count <= 0 || !jobs) return APAX_ERR_INVALID_ARG;
    out.resize(count);
    gp8.resize(count);
    gp32.resize(count);
    pkt_words = 0;
    ebuf_words = 0;
    for (int i = 0; i < count; ++i) {
        const apax_encode_job &j = jobs[i];
        uint32_t pw, ew;
        int st = fill_enc_args(j.x, j.dtype, j.n, &j.p, j.code_dev, j.out, j.out_capacity, j.res,
                               out[i], pw, ew);
        if (st) return st;
        if (!j.res) return APAX_ERR_INVALID_ARG;
        pkt_words = pw > pkt_words ? pw : pkt_words;
        ebuf_words = ew > ebuf_words ? ew : ebuf_words;
        const int gs = (j.p.format & APAX_FORMAT_GROUP8) ? 8 : 4;
        gp8[i] = (uint32_t)groups_per_thread(j.p.block_size, gs, 8);
        gp32[i] = (uint32_t)groups_per_thread(j.p.block_size, gs, 32);
    }
    need32 = 16ull * (pkt_words + ebuf_words) * 4 > kEncSmemCap;
    return APAX_OK;
}

// ---- decode plans
// Workspace: [job table][tile prefix][tiles per job][block sizes]
//            [ticket | done+status per job]
struct DLayout {
    size_t jobs, prefix, tiles_of, bsize, zero, counters, total;
};

DLayout dlayout_of(int count)
{
    DLayout L;
    L.jobs = 0;
    L.prefix = align_up((size_t)count * sizeof(DecArgs), kAlign);
    L.tiles_of = align_up(L.prefix + (size_t)(count + 1) * 8, kAlign);
    L.bsize = align_up(L.tiles_of + (size_t)count * 8, kAlign);
    L.zero = align_up(L.bsize + (size_t)count * 4, kAlign);
    L.counters = L.zero + 64;
    L.total = align_up(L.counters + (size_t)count * 16, kAlign);
    return L;
}

int validate_decode_jobs(const apax_decode_job *jobs, int count, std::vector<DecArgs> &out,
                         std::vector<uint32_t> &bs, bool &need32)
{
    if (count <= 0 || !jobs) return APAX_ERR_INVALID_ARG;
    out.resize(count);
    bs.resize(count);
    need32 = false;
    for (int i = 0; i < count; ++i) {
        const apax_decode_job &j = jobs[i];
        Fmt f;
        int st = fmt_of(j.dtype, f);
        if (st) return st;
        if (!block_size_ok(j.block_size)) return APAX_ERR_BLOCK_SIZE;
        if ((!j.in && j.in_bytes) || (!j.y && j.n) || !j.res) return APAX_ERR_INVALID_ARG;
        if (((uintptr_t)j.in & 3) || ((uintptr_t)j.y % f.size)) return APAX_ERR_INVALID_ARG;
        DecArgs &a = out[i];
        memset(&a, 0, sizeof a);
        a.in = (const uint8_t *)j.in;
        a.in_bytes = j.in_bytes;
        a.y = j.y;
        a.dtype = j.dtype;
        a.n = j.n;
        a.ranged = false;
        a.res = j.res;
        bs[i] = j.block_size;
        if (j.block_size / 4 > 1024) need32 = true;
    }
    return APAX_OK;
}

int apply_decode_config(apax_batch *b, const apax_batch_config &c)
{
    if (b->need32 ? (c.threads < 32 || c.threads > 128 || (c.threads % 32))
                  : (c.threads != 64 && c.threads != 128))
        return APAX_ERR_INVALID_ARG;
    const int ts = b->need32 ? 32 : 8;
    const int nteams = (int)c.threads / ts;
    const DLayout L = dlayout_of(b->count);
    std::vector<DecArgs> tab(b->djobs);
    std::vector<uint64_t> prefix((size_t)b->count + 1, 0), tiles((size_t)b->count, 0);
    for (int i = 0; i < b->count; ++i) {
        DecArgs &a = tab[i];
        const uint64_t nb = (a.n + b->dN[i] - 1) / b->dN[i];
        // blocks of up to 1024 samples: one per thread, tiles of `threads` blocks
        const uint64_t per = b->dN[i] <= kT1MaxBlock ? c.threads : (uint64_t)nteams;
        tiles[i] = nb ? (nb + per - 1) / per : 1;
        a.done = (unsigned *)(b->ws + L.counters + 16 * (size_t)i);
        a.status = (int *)(b->ws + L.counters + 16 * (size_t)i + 4);
        prefix[i + 1] = prefix[i] + tiles[i];
    }
    b->total_tiles = prefix[b->count];
    b->d_djobs = (DecArgs *)(b->ws + L.jobs);
    b->d_prefix = (uint64_t *)(b->ws + L.prefix);
    b->d_tiles_of = (uint64_t *)(b->ws + L.tiles_of);
    b->d_bsize = (uint32_t *)(b->ws + L.bsize);
    b->d_zero = b->ws + L.zero;
    b->zero_bytes = L.total - L.zero;
    if (!upload(b, b->d_djobs, tab.data(), tab.size() * sizeof(DecArgs)) ||
        !upload(b, b->d_prefix, prefix.data(), prefix.size() * 8) ||
        !upload(b, b->d_tiles_of, tiles.data(), tiles.size() * 8) ||
        !upload(b, b->d_bsize, b->dN.data(), b->dN.size() * 4))
        return APAX_ERR_CUDA;
    b->cfg = c;
    if (b->cfg.ctas_per_sm == 0) {
        const int occ = decode_batch_occupancy(ts, (int)c.threads);
        b->cfg.ctas_per_sm = occ > 0 ? (uint32_t)occ : 1;
    }
    return APAX_OK;
}

// ---- profile plans (runs of 16 blocks: the tree's level-1 nodes)
// Workspace: [job table][run prefix][ticket | done+status per job |
//            candidate bytes per job][run sums and tree scratch per job]
struct PLayout {
    size_t jobs, prefix, zero, counters, bytes, sums, total;
    std::vector<size_t> sums_of;
};

uint64_t prof_sums_words(const ProfArgs &a)
{
    const uint64_t Qn = 2 + 4 * (uint64_t)a.ncand;
    return Qn * (a.nruns ? a.nruns : 1) + Qn * 2 * (((a.nruns + 15) / 16) + 1);
}

PLayout playout_of(const std::vector<ProfArgs> &jobs)
{
    const size_t count = jobs.size();
    PLayout L;
    L.jobs = 0;
    L.prefix = align_up(count * sizeof(ProfArgs), kAlign);
    L.zero = align_up(L.prefix + (count + 1) * 8, kAlign);
    L.counters = L.zero + 64;
    L.bytes = align_up(L.counters + count * 16, kAlign);
    L.sums = align_up(L.bytes + count * 8 * 32, kAlign);
    size_t off = L.sums;
    L.sums_of.resize(count);
    for (size_t i = 0; i < count; ++i) {
        L.sums_of[i] = off;
        off = align_up(off + 8 * prof_sums_words(jobs[i]), 16);
    }
    L.total = align_up(off, kAlign);
    return L;
}

int validate_profile_jobs(const apax_profile_job *jobs, int count, std::vector<ProfArgs> &out,
                          int &max_ncand)
{
    if (count <= 0 || !jobs) return APAX_ERR_INVALID_ARG;
    out.resize(count);
    max_ncand = 1;
    for (int i = 0; i < count; ++i) {
        const apax_profile_job &j = jobs[i];
        int st = fill_prof_args(j.x, j.dtype, j.n, j.block_size, j.format, j.candidates, j.ncand,
                                j.target, j.points, j.summary, out[i]);
        if (st) return st;
        if (j.ncand > max_ncand) max_ncand = j.ncand;
    }
    return APAX_OK;
}

int apply_profile_config(apax_batch *b, const apax_batch_config &c)
{
    if (c.threads != 128) return APAX_ERR_INVALID_ARG;
    const PLayout L = playout_of(b->pjobs);
    std::vector<ProfArgs> tab(b->pjobs);
    std::vector<uint64_t> prefix((size_t)b->count + 1, 0);
    for (int i = 0; i < b->count; ++i) {
        ProfArgs &a = tab[i];
        a.done = (unsigned *)(b->ws + L.counters + 16 * (size_t)i);
        a.status = (int *)(b->ws + L.counters + 16 * (size_t)i + 4);
        a.bytes = (unsigned long long *)(b->ws + L.bytes + 256 * (size_t)i);
        a.run_sums = (double *)(b->ws + L.sums_of[i]);
        const uint64_t Qn = 2 + 4 * (uint64_t)a.ncand;
        a.scratch = a.run_sums + Qn * (a.nruns ? a.nruns : 1);
        prefix[i + 1] = prefix[i] + (a.nruns ? a.nruns : 1);
    }
    b->total_tiles = prefix[b->count];
    b->d_pjobs = (ProfArgs *)(b->ws + L.jobs);
    b->d_prefix = (uint64_t *)(b->ws + L.prefix);
    b->d_zero = b->ws + L.zero;
    b->zero_bytes = L.sums - L.zero;
    if (!upload(b, b->d_pjobs, tab.data(), tab.size() * sizeof(ProfArgs)) ||
        !upload(b, b->d_prefix, prefix.data(), prefix.size() * 8))
        return APAX_ERR_CUDA;
    b->cfg = c;
    if (b->cfg.ctas_per_sm == 0) {
        const int occ = profile_batch_occupancy(b->max_ncand);
        b->cfg.ctas_per_sm = occ > 0 ? (uint32_t)occ : 1;
    }
    return APAX_OK;
}

std::string make_key(const apax_batch *b)
{
    // arrays, total samples (log2 bucket), dtype/mode mix, largest packet
    uint64_t n = 0;
    unsigned mix = 0;
    for (const EncArgs &a : b->jobs) {
        n += a.n;
        mix |= 1u << (2 * a.dtype + a.mode);
    }
    for (const DecArgs &a : b->djobs) {
        n += a.n;
        mix |= 1u << (16 + a.dtype);
    }
    for (const ProfArgs &a : b->pjobs) {
        n += a.n;
        mix |= 1u << (24 + a.dtype);
    }
    int lg = 0;
    while ((n >> lg) > 1) ++lg;
    char buf[128];
    static const char *ops[3] = {"enc", "dec", "prof"};
    snprintf(buf, sizeof buf, "%s:%d:%d:%x:%u:%u:%d:%d", ops[b->op], b->count, lg, mix,
             b->pkt_words, b->ebuf_words, (int)b->need32, b->dev);
    return buf;
}

}  // namespace

namespace apax {
namespace host {

int batch_create(int op, const void *jobs, int count, void *workspace, uint64_t workspace_bytes,
                 uint8_t *pinned, uint64_t pinned_bytes, cudaStream_t stream, bool use_tuned,
                 apax_batch **plan)
{
    if (!plan) return APAX_ERR_INVALID_ARG;
    *plan = nullptr;
    apax_batch *b = new apax_batch();
    b->op = op;
    b->count = count;
    b->pkt_words = b->ebuf_words = 0;
    b->need32 = false;
    b->pinned = pinned;
    b->pinned_bytes = pinned_bytes;
    b->pinned_used = 0;
    b->up_stream = stream;
    int st;
    uint64_t need = 0;
    if (op == 0) {
        st = validate_encode_jobs((const apax_encode_job *)jobs, count, b->jobs, b->gp8, b->gp32,
                                  b->pkt_words, b->ebuf_words, b->need32);
        if (!st) need = layout_of(count, b->jobs, min_tile_blocks(b)).total;
    } else if (op == 1) {
        st = validate_decode_jobs((const apax_decode_job *)jobs, count, b->djobs, b->dN, b->need32);
        if (!st) need = dlayout_of(count).total;
    } else {
        st = validate_profile_jobs((const apax_profile_job *)jobs, count, b->pjobs, b->max_ncand);
        if (!st) need = playout_of(b->pjobs).total;
    }
    if (!st && (!workspace || ((uintptr_t)workspace % kAlign))) st = APAX_ERR_INVALID_ARG;
    if (!st && workspace_bytes < need) st = APAX_ERR_CAPACITY;
    if (!st && (cudaGetDevice(&b->dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev) !=
                    cudaSuccess))
        st = APAX_ERR_CUDA;
    if (st) {
        delete b;
        return st;
    }
    b->ws = (uint8_t *)workspace;
    b->ws_bytes = workspace_bytes;
    b->key = make_key(b);
    apax_batch_config c = default_config(b);
    if (use_tuned) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(b->key);
        if (it != g_tune_cache.end()) c = it->second;
    }
    st = apply_config(b, c);
    if (st) {
        delete b;
        return st;
    }
    *plan = b;
    return APAX_OK;
}

uint64_t batch_workspace_bytes(int op, const void *jobs, int count)
{
    uint64_t v = 0;
    int st = op == 0 ? apax_batch_encode_workspace_size((const apax_encode_job *)jobs, count, &v)
           : op == 1 ? apax_batch_decode_workspace_size((const apax_decode_job *)jobs, count, &v)
                     : apax_batch_profile_workspace_size((const apax_profile_job *)jobs, count, &v);
    return st ? 0 : v;
}

}  // namespace host
}  // namespace apax

extern "C" {

int apax_batch_encode_workspace_size(const apax_encode_job *jobs, int count, uint64_t *bytes)
{
    if (!bytes) return APAX_ERR_INVALID_ARG;
    std::vector<EncArgs> v;
    std::vector<uint32_t> g8, g32;
    uint32_t pw, ew;
    bool n32;
    int st = validate_encode_jobs(jobs, count, v, g8, g32, pw, ew, n32);
    if (st) return st;
    *bytes = layout_of(count, v, n32 ? 1 : 8).total;
    return APAX_OK;
}

int apax_batch_encode_create(const apax_encode_job *jobs, int count, void *workspace,
                             uint64_t workspace_bytes, apax_batch **plan)
{
    return apax::host::batch_create(0, jobs, count, workspace, workspace_bytes, nullptr, 0, nullptr,
                                    true, plan);
}

int apax_batch_decode_workspace_size(const apax_decode_job *jobs, int count, uint64_t *bytes)
{
    if (!bytes) return APAX_ERR_INVALID_ARG;
    std::vector<DecArgs> v;
    std::vector<uint32_t> bs;
    bool n32;
    int st = validate_decode_jobs(jobs, count, v, bs, n32);
    if (st) return st;
    *bytes = dlayout_of(count).total;
    return APAX_OK;
}

int apax_batch_decode_create(const apax_decode_job *jobs, int count, void *workspace,
                             uint64_t workspace_bytes, apax_batch **plan)
{
    return apax::host::batch_create(1, jobs, count, workspace, workspace_bytes, nullptr, 0, nullptr,
                                    true, plan);
}

int apax_batch_profile_workspace_size(const apax_profile_job *jobs, int count, uint64_t *bytes)
{
    if (!bytes) return APAX_ERR_INVALID_ARG;
    std::vector<ProfArgs> v;
    int mx;
    int st = validate_profile_jobs(jobs, count, v, mx);
    if (st) return st;
    *bytes = playout_of(v).total;
    return APAX_OK;
}

int apax_batch_profile_create(const apax_profile_job *jobs, int count, void *workspace,
                              uint64_t workspace_bytes, apax_batch **plan)
{
    return apax::host::batch_create(2, jobs, count, workspace, workspace_bytes, nullptr, 0, nullptr,
                                    true, plan);
}

int apax_batch_run(apax_batch *b, void *stream)
{
    if (!b) return APAX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = cuda_fail(cudaMemsetAsync(b->d_zero, 0, b->zero_bytes, s));
    if (st) return st;
    const uint64_t want = (uint64_t)b->sms * b->cfg.ctas_per_sm;
    const unsigned ctas = (unsigned)(want < b->total_tiles ? want : b->total_tiles);
    if (b->op == 2) {
        ProfBatchArgs pa;
        pa.jobs = b->d_pjobs;
        pa.run_prefix = b->d_prefix;
        pa.count = b->count;
        pa.total_runs = b->total_tiles;
        pa.ticket = (unsigned long long *)b->d_zero;
        return cuda_fail(launch_profile_batch(pa, b->max_ncand, ctas, s));
    }
    if (b->op == 1) {
        DecBatchArgs da;
        da.jobs = b->d_djobs;
        da.tile_prefix = b->d_prefix;
        da.tiles_of = b->d_tiles_of;
        da.block_size = b->d_bsize;
        da.count = b->count;
        da.total_tiles = b->total_tiles;
        da.ticket = (unsigned long long *)b->d_zero;
        return cuda_fail(launch_decode_batch(da, b->need32 ? 32 : 8, (int)b->cfg.threads, ctas, s));
    }
    const Geo g = geo_of(b, b->cfg);
    EncBatchArgs ba;
    ba.jobs = b->d_jobs;
    ba.tile_prefix = b->d_prefix;
    ba.count = b->count;
    ba.total_tiles = b->total_tiles;
    ba.ticket = (unsigned long long *)b->d_zero;
    return cuda_fail(launch_encode_batch(ba, g.ts, g.threads, smem_of(b, g), ctas, s));
}

int apax_batch_get_config(const apax_batch *b, apax_batch_config *c)
{
    if (!b || !c) return APAX_ERR_INVALID_ARG;
    *c = b->cfg;
    return APAX_OK;
}

int apax_batch_set_config(apax_batch *b, const apax_batch_config *c)
{
    if (!b || !c) return APAX_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return APAX_ERR_CUDA;
    return apply_config(b, *c);
}

int apax_batch_tune(apax_batch *b, int reps, void *stream)
{
    if (!b || reps < 1) return APAX_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<apax_batch_config> cands;
    const int thr8[2] = {64, 128};
    for (int t = 0; t < (b->op == 2 ? 1 : (b->need32 ? 4 : 2)); ++t) {
        apax_batch_config c;
        c.threads = b->op == 2 ? 128u : (b->need32 ? 32u * (t + 1) : (uint32_t)thr8[t]);
        int occ;
        if (b->op == 2) {
            occ = profile_batch_occupancy(b->max_ncand);
        } else if (b->op == 1) {
            occ = decode_batch_occupancy(b->need32 ? 32 : 8, (int)c.threads);
        } else {
            if (!config_ok(b, c)) continue;
            const Geo g = geo_of(b, c);
            occ = encode_batch_occupancy(g.ts, g.threads, smem_of(b, g));
        }
        for (int k = 1; k <= occ; k = k < 2 ? k + 1 : k * 2) {
            c.ctas_per_sm = (uint32_t)k;
            cands.push_back(c);
        }
        if (occ > 2 && (occ & (occ - 1))) {
            c.ctas_per_sm = (uint32_t)occ;
            cands.push_back(c);
        }
    }
    if (cands.empty()) return APAX_ERR_INVALID_ARG;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return APAX_ERR_CUDA;
    float best = 0.f;
    apax_batch_config bestc = b->cfg;
    int st = APAX_OK;
    for (const apax_batch_config &c : cands) {
        if ((st = cuda_fail(cudaStreamSynchronize(s))) != APAX_OK) break;
        if ((st = apply_config(b, c)) != APAX_OK) break;
        if ((st = apax_batch_run(b, s)) != APAX_OK) break;  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == APAX_OK; ++r) st = apax_batch_run(b, s);
        cudaEventRecord(e1, s);
        if (st || (st = cuda_fail(cudaEventSynchronize(e1))) != APAX_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0.f || ms < best) {
            best = ms;
            bestc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    st = apply_config(b, bestc);
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[b->key] = b->cfg;
    return APAX_OK;
}

uint64_t apax_batch_tiles(const apax_batch *b) { return b ? b->total_tiles : 0; }

void apax_batch_destroy(apax_batch *b) { delete b; }

}  // extern "C"
