// apax_host.cu -- C ABI of the codec: argument validation, container sizes,
// workspace layout, launch planning.  No allocation, no stream sync.
#include <math.h>
#include <string.h>

#include <array>
#include <map>
#include <mutex>

#include "apax_team.cuh"
#include "apax_kernels.h"
#include "apax_plan.h"

using namespace apax;

using namespace apax::host;

namespace {

}  // namespace

namespace apax {
namespace host {

int fill_enc_args(const void *x, int dtype, uint64_t n, const apax_params *p,
                  const uint32_t *code_dev, void *out, uint64_t cap, apax_result *res, EncArgs &a,
                  uint32_t &pkt_words, uint32_t &ebuf_words)
{
    Fmt f;
    int st = check(dtype, p, f);
    if (st) return st;
    if ((!x && n) || !out) return APAX_ERR_INVALID_ARG;
    // the container is written as 32-bit words; inputs at element alignment
    if (((uintptr_t)out & 3) || ((uintptr_t)x % f.size)) return APAX_ERR_INVALID_ARG;
    const uint32_t N = p->block_size;
    const uint64_t nb = (n + N - 1) / N;
    const uint64_t B = p->mode == APAX_FIXED_RATE ? budget(f, N, p->rate_num, p->rate_den) : 0;
    team_words(f, N, B, pkt_words, ebuf_words);
    memset(&a, 0, sizeof a);
    a.x = x;
    a.n = n;
    a.N = N;
    a.nb = nb;
    a.dtype = dtype;
    a.mode = p->mode;
    a.code = p->atten_code;
    a.code_dev = code_dev;
    a.out = (uint8_t *)out;
    a.cap = cap;
    a.res = res;
    a.n_hdr = n;
    a.gsh = f.gs == 8 ? 1 : 0;
    a.sum = (f.opts & APAX_FORMAT_SUM_STREAM) ? 1 : 0;
    a.spin_limit = 1ll << 31;
    a.test_stall_tile = -1;
    if (p->mode == APAX_FIXED_RATE) {
        a.rate_num = p->rate_num;
        a.rate_den = p->rate_den;
        a.search = (int)p->search;
        a.B = (uint32_t)B;
        uint64_t total;
        apax_encoded_size(dtype, n, p, &total);
        if (cap < total) return APAX_ERR_CAPACITY;
        a.fr_payload = total - 40;
        a.poff = 40;
    } else {
        a.poff = 40 + table_bytes(nb);
        if (cap < a.poff) return APAX_ERR_CAPACITY;
    }
    return APAX_OK;
}

int fill_prof_args(const void *x, int dtype, uint64_t n, uint32_t block_size, uint32_t format,
                   const uint16_t *candidates, int ncand, double target,
                   apax_profile_point *points, apax_profile_summary *summary, ProfArgs &a)
{
    Fmt f;
    int st = fmt_of(dtype, f);
    if (st) return st;
    if (!block_size_ok(block_size)) return APAX_ERR_BLOCK_SIZE;
    st = fmt_opts(format, block_size, f);
    if (st) return st;
    uint16_t def[16];
    if (!candidates) {
        if (ncand != APAX_PROFILE_DEFAULT_CANDIDATES) return APAX_ERR_INVALID_ARG;
        for (int i = 0; i < 16; ++i) def[i] = (uint16_t)(256 * i);
        candidates = def;
    }
    if (ncand < 1 || ncand > 32 || (!x && n) || !points || !summary) return APAX_ERR_INVALID_ARG;
    if (((uintptr_t)x % f.size) || ((uintptr_t)points & 7) || ((uintptr_t)summary & 7))
        return APAX_ERR_INVALID_ARG;
    for (int i = 0; i < ncand; ++i) {
        // strictly increasing codes of 0..4095
        if (candidates[i] > 4095) return APAX_ERR_INVALID_ARG;
        if (i && candidates[i] <= candidates[i - 1]) return APAX_ERR_INVALID_ARG;
    }
    if (!(target == target)) return APAX_ERR_INVALID_ARG;
    const uint64_t nb = (n + block_size - 1) / block_size;
    memset(&a, 0, sizeof a);
    a.x = x;
    a.n = n;
    a.N = block_size;
    a.nb = nb;
    a.dtype = dtype;
    a.ncand = ncand;
    for (int i = 0; i < ncand; ++i) a.codes[i] = candidates[i];
    a.nruns = (nb + 15) / 16;
    a.gp = groups_per_thread(block_size, f.gs, kProfTS);
    a.gsh = f.gs == 8 ? 1 : 0;
    a.sum = (f.opts & APAX_FORMAT_SUM_STREAM) ? 1 : 0;
    a.target = target;
    a.points = points;
    a.summary = summary;
    return APAX_OK;
}

}  // namespace host
}  // namespace apax

namespace {

// A whole array, or (shard) the blocks [b0, b1) of an array of n_all
// elements, x pointing at block b0 - 1 (b0 > 0: the lag decision's halo) or
// at block 0; the container then describes the sub-array of those blocks.
int encode_impl(const void *x, int dtype, uint64_t n, const apax_params *p,
                const uint32_t *code_dev, void *out, uint64_t cap, void *ws, uint64_t wsb,
                apax_result *res, int64_t stall, int64_t spin, void *stream,
                bool shard = false, uint64_t n_all = 0, uint64_t b0 = 0, uint64_t b1 = 0)
{
    EncArgs a;
    uint32_t pw, ew;
    int st = fill_enc_args(x, dtype, n, p, code_dev, out, cap, res, a, pw, ew);
    if (st) return st;
    if (!ws || ((uintptr_t)ws & 7)) return APAX_ERR_INVALID_ARG;
    uint64_t need_ws;
    apax_workspace_size(dtype, n, p, &need_ws);
    if (wsb < need_ws) return APAX_ERR_CAPACITY;
    int ts, threads;
    Plan pl;
    Fmt f;
    fmt_of(dtype, f);
    fmt_opts(p->format, p->block_size, f);
    if (p->mode == APAX_FIXED_RATE && a.N <= kT1MaxBlock && a.nb >= kT1MinBlocks && !p->format) {
        // fixed rate, a block per thread: its 13-step search runs without
        // team exchanges (measured faster); fixed quality keeps teams, whose
        // packets leave through coalesced stores.  Format options take teams.
        pl = plan_geometry(a.N, a.nb, 0, 0, 1, 128);
        pl.smem = (size_t)128 * (a.N / 4);
    } else {
        default_geometry((size_t)(pw + ew) * 4, a.nb, ts, threads);
        pl = plan_geometry(a.N, a.nb, pw, ew, ts, threads, f.gs);
    }
    a.pkt_words = pl.pkt_words;
    a.ebuf_words = pl.ebuf_words;
    // staging of the tile in shared memory: on for the fixed-rate search by
    // teams (13 passes over a block), off for fixed quality, whose occupancy
    // matters more than its few L2 re-reads (measured on GB300)
    const bool want = p->mode == APAX_FIXED_RATE;
    // blocks that fit a team's registers are read from global memory once
    const bool in_regs = pl.ts != 1 && encode_res_eligible(dtype, p->mode, a.N, pl.ts);
    const size_t sb = (want && pl.ts != 1 && !in_regs) ? stage_bytes(f.size, a.N, pl.threads / pl.ts, pl.smem) : 0;
    a.stage_off = sb ? (uint32_t)((pl.smem + 15) / 16 * 16) : 0;
    if (sb) pl.smem = a.stage_off + sb;
    a.gp = pl.gp;
    a.ntiles = pl.ntiles;
    a.spin_limit = spin;
    a.test_stall_tile = stall;
    uint8_t *w = (uint8_t *)ws;
    a.ticket = (unsigned *)(w + 0);
    a.done = (unsigned *)(w + 4);
    a.status = (int *)(w + 8);
    a.tiles = (unsigned long long *)(w + kWsHead);
    if (shard) {
        // blocks keep their global numbers: the halo block j - 1 of the first
        // one is read, and x is placed so that block j sits at x + j N
        const uint64_t xb0 = b0 ? b0 - 1 : 0;
        a.x = (const void *)((uintptr_t)x - (uintptr_t)(xb0 * (uint64_t)a.N * f.size));
        a.n = n_all;
        a.jb0 = b0;
        a.nb = b1;
        a.n_hdr = n;
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_fail(cudaMemsetAsync(ws, 0, need_ws, s));
    if (st) return st;
    if (a.sum) {
        // the stream decisions of the call's blocks, in the workspace's tail
        const uint64_t cnt = a.nb - a.jb0;
        uint8_t *sel = w + need_ws - (cnt + 15) / 16 * 16;
        SelArgs sa;
        sa.x = a.x;
        sa.n = a.n;
        sa.N = a.N;
        sa.nb = a.nb;
        sa.j0 = a.jb0;
        sa.count = cnt;
        sa.dtype = dtype;
        sa.gsh = a.gsh;
        sa.gp = 0;
        sa.sel = sel;
        st = cuda_fail(launch_best_streams(sa, s));
        if (st) return st;
        a.sel = sel;
    }
    if (in_regs) return cuda_fail(launch_encode_res(a, pl.threads, pl.smem, s));
    return cuda_fail(launch_encode(a, pl.ts, pl.threads, pl.smem, s));
}

int decode_impl(const void *in, uint64_t in_bytes, uint64_t b0, uint64_t b1, bool ranged,
                void *y, int dtype, uint64_t n, void *ws, uint64_t wsb, apax_result *res,
                void *stream)
{
    Fmt f;
    int st = fmt_of(dtype, f);
    if (st) return st;
    const bool need_y = ranged ? b1 > b0 : n > 0;
    if ((!in && in_bytes) || (!y && need_y) || !ws) return APAX_ERR_INVALID_ARG;
    if (((uintptr_t)in & 3) || ((uintptr_t)ws & 7) || ((uintptr_t)y % f.size))
        return APAX_ERR_INVALID_ARG;
    if (wsb < apax_decode_workspace_size()) return APAX_ERR_CAPACITY;
    if (b0 > b1) return APAX_ERR_INVALID_ARG;
    DecArgs a;
    memset(&a, 0, sizeof a);
    a.in = (const uint8_t *)in;
    a.in_bytes = in_bytes;
    a.y = y;
    a.dtype = dtype;
    a.n = n;
    a.b0 = b0;
    a.b1 = b1;
    a.ranged = ranged;
    uint8_t *w = (uint8_t *)ws;
    a.done = (unsigned *)(w + 16);
    a.ticket = (unsigned long long *)(w + 24);
    a.status = (int *)(w + 8);
    a.res = res;
    const int sms = sm_count();
    // Grid-stride over blocks.  The small-block launch (16 teams of 8 per
    // CTA) sizes its grid for the smallest legal block size; the large-block
    // launch (4 teams of 32) for blocks of more than 4096 samples.
    const uint64_t blocks = ranged ? (b1 - b0) : (n + 63) / 64;
    uint64_t ctas = (blocks + 15) / 16;
    const uint64_t cap = (uint64_t)sms * 8;
    if (ctas > cap) ctas = cap;
    if (ctas == 0) ctas = 1;
    a.nctas = (unsigned)ctas;
    // the teams-of-32 launch: blocks above 4096 samples, or at most
    // kTeam32MaxBlocks blocks of any size (n / 64 bounds the block count)
    const uint64_t few = (n + 63) / 64 < kTeam32MaxBlocks ? (n + 63) / 64 : kTeam32MaxBlocks;
    const uint64_t lblocks = ranged ? (b1 - b0) : ((n + 4095) / 4096 > few ? (n + 4095) / 4096 : few);
    uint64_t lctas = (lblocks + 3) / 4;
    if (lctas > (uint64_t)sms * 4) lctas = (uint64_t)sms * 4;
    if (lctas == 0) lctas = 1;
    a.nctas_large = (unsigned)lctas;
    // at most kTeam32MaxBlocks blocks whatever the block size: every
    // container is the teams-of-32 launch's, so the other one is not enqueued
    a.small_launched = blocks > kTeam32MaxBlocks;
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_fail(cudaMemsetAsync(ws, 0, apax_decode_workspace_size(), s));
    if (st) return st;
    return cuda_fail(launch_decode(a, s));
}

// Streams on which the host-input sweep runs its pieces: created once per
// device (non-blocking, for the life of the process's CUDA context) and
// reused.
constexpr int kSweepStreams = 16;
static bool sweep_streams(cudaStream_t (&out)[kSweepStreams])
{
    static std::mutex mu;
    static std::map<int, std::array<cudaStream_t, kSweepStreams>> pool;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pool.find(dev);
    if (it == pool.end()) {
        std::array<cudaStream_t, kSweepStreams> a{};
        for (int k = 0; k < kSweepStreams; ++k) {
            if (cudaStreamCreateWithFlags(&a[k], cudaStreamNonBlocking) != cudaSuccess) {
                for (int i = 0; i < k; ++i) cudaStreamDestroy(a[i]);
                return false;
            }
        }
        it = pool.emplace(dev, a).first;
    }
    for (int k = 0; k < kSweepStreams; ++k) out[k] = it->second[k];
    return true;
}

// Workspace layout of a profile: head (done, status), per-candidate byte
// counters, the run sums, then the tree scratch.
static void place_profile_workspace(ProfArgs &a, void *workspace)
{
    uint8_t *w = (uint8_t *)workspace;
    a.done = (unsigned *)(w + 4);
    a.status = (int *)(w + 8);
    a.bytes = (unsigned long long *)(w + kWsHead);
    const uint64_t Qn = 2 + 4 * (uint64_t)a.ncand;
    a.run_sums = (double *)(w + kWsHead + 8 * 32);
    a.scratch = a.run_sums + Qn * (a.nruns ? a.nruns : 1);
    a.run_flags = (uint8_t *)(a.scratch + Qn * 2 * (((a.nruns + 15) / 16) + 1));
    a.sel = a.sum ? a.run_flags + (a.nruns + 15) / 16 * 16 : nullptr;
}

}  // namespace

namespace apax {
int encode_with_workspace(const void *x, int dtype, uint64_t n, const apax_params *p, void *out,
                          uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                          apax_result *res, void *stream)
{
    return encode_impl(x, dtype, n, p, nullptr, out, out_capacity, workspace, workspace_bytes, res,
                       -1, 1ll << 31, stream);
}
}  // namespace apax

extern "C" {

int apax_encoded_size(int dtype, uint64_t n, const apax_params *p, uint64_t *bytes)
{
    Fmt f;
    int st = check(dtype, p, f);
    if (st) return st;
    if (!bytes) return APAX_ERR_INVALID_ARG;
    const uint32_t N = p->block_size;
    const uint64_t nb = (n + N - 1) / N;
    if (nb == 0) {
        *bytes = 40;
        return APAX_OK;
    }
    const uint64_t Lend = n - (nb - 1) * N;
    if (p->mode == APAX_FIXED_RATE) {
        *bytes = 40 + (nb - 1) * budget(f, N, p->rate_num, p->rate_den) +
                 budget(f, Lend, p->rate_num, p->rate_den);
    } else {
        // every exponent absolute (8 bits) at the full width W
        const uint64_t gs = (uint64_t)f.gs;
        const uint64_t full = pad32((uint64_t)f.H + 8ull * (N / gs) + (uint64_t)f.W * N);
        const uint64_t Gl = (Lend + gs - 1) / gs;
        const uint64_t last = pad32((uint64_t)f.H + 8ull * Gl + (uint64_t)f.W * gs * Gl);
        *bytes = 40 + table_bytes(nb) + (nb - 1) * full + last;
    }
    return APAX_OK;
}

int apax_copy_container(const void *src, const apax_result *res, void *dst, uint64_t capacity,
                        void *stream)
{
    if (!src || !res || !dst || ((uintptr_t)src & 3) || ((uintptr_t)dst & 3) || ((uintptr_t)res & 7))
        return APAX_ERR_INVALID_ARG;
    const uintptr_t s0 = (uintptr_t)src, d0 = (uintptr_t)dst;
    if (capacity && s0 < d0 + capacity && d0 < s0 + capacity) return APAX_ERR_INVALID_ARG;
    if (!capacity) return APAX_OK;
    return cuda_fail(launch_copy_sized(src, res, dst, capacity, (cudaStream_t)stream));
}

int apax_workspace_size(int dtype, uint64_t n, const apax_params *p, uint64_t *bytes)
{
    Fmt f;
    int st = check(dtype, p, f);
    if (st) return st;
    if (!bytes) return APAX_ERR_INVALID_ARG;
    const uint64_t nb = (n + p->block_size - 1) / p->block_size;
    const uint64_t B =
        p->mode == APAX_FIXED_RATE ? budget(f, p->block_size, p->rate_num, p->rate_den) : 0;
    const Plan pl = plan_encode(f, p->block_size, nb, B);
    *bytes = kWsHead + (p->mode == APAX_FIXED_QUALITY ? 8 * pl.ntiles : 0);
    // the sum stream: one stream decision byte per block
    if (f.opts & APAX_FORMAT_SUM_STREAM) *bytes = (*bytes + 15) / 16 * 16 + (nb + 15) / 16 * 16;
    return APAX_OK;
}

int apax_encode(const void *x, int dtype, uint64_t n, const apax_params *p, void *out,
                uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                apax_result *res, void *stream)
{
    return encode_impl(x, dtype, n, p, nullptr, out, out_capacity, workspace, workspace_bytes,
                       res, -1, 1ll << 31, stream);
}

int apax_encode_recommended(const void *x, int dtype, uint64_t n, const apax_params *p,
                            const struct apax_profile_summary *summary, void *out,
                            uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                            apax_result *res, void *stream)
{
    if (!p || p->mode != APAX_FIXED_QUALITY || !summary) return APAX_ERR_INVALID_ARG;
    return encode_impl(x, dtype, n, p, &summary->recommended_code, out, out_capacity, workspace,
                       workspace_bytes, res, -1, 1ll << 31, stream);
}

int apax_encode_test_stall(const void *x, int dtype, uint64_t n, const apax_params *p, void *out,
                           uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                           apax_result *res, int64_t stall_tile, int64_t spin_cycles,
                           void *stream)
{
    if (!p || p->mode != APAX_FIXED_QUALITY || spin_cycles <= 0) return APAX_ERR_INVALID_ARG;
    return encode_impl(x, dtype, n, p, nullptr, out, out_capacity, workspace, workspace_bytes,
                       res, stall_tile, spin_cycles, stream);
}

int apax_shard_elements(uint64_t n, uint32_t block_size, uint64_t block_begin, uint64_t block_end,
                        uint64_t *elements)
{
    if (!block_size_ok(block_size)) return APAX_ERR_BLOCK_SIZE;
    const uint64_t nb = (n + block_size - 1) / block_size;
    if (!elements || block_begin >= block_end || block_end > nb) return APAX_ERR_INVALID_ARG;
    const uint64_t e1 = block_end * (uint64_t)block_size < n ? block_end * (uint64_t)block_size : n;
    *elements = e1 - block_begin * (uint64_t)block_size;
    return APAX_OK;
}

int apax_encode_shard(const void *x, int dtype, uint64_t n, const apax_params *p,
                      uint64_t block_begin, uint64_t block_end, void *out, uint64_t out_capacity,
                      void *workspace, uint64_t workspace_bytes, apax_result *res, void *stream)
{
    if (!p) return APAX_ERR_INVALID_ARG;
    uint64_t n_sub;
    int st = apax_shard_elements(n, p->block_size, block_begin, block_end, &n_sub);
    if (st) return st;
    return encode_impl(x, dtype, n_sub, p, nullptr, out, out_capacity, workspace, workspace_bytes,
                       res, -1, 1ll << 31, stream, true, n, block_begin, block_end);
}

int apax_shard_rebase(void *container, uint64_t block_count, uint64_t add_words, void *stream)
{
    if (!container || ((uintptr_t)container & 3)) return APAX_ERR_INVALID_ARG;
    uint32_t *t = (uint32_t *)((uint8_t *)container + 40);
    return cuda_fail(launch_table_rebase(t, t, block_count, add_words, (cudaStream_t)stream));
}

int apax_merge_shards(const apax_shard *shards, int count, int dtype, uint64_t n,
                      const apax_params *p, void *out, uint64_t out_capacity, apax_result *res,
                      void *stream)
{
    Fmt f;
    int st = check(dtype, p, f);
    if (st) return st;
    if (!shards || count < 1 || !out || ((uintptr_t)out & 3)) return APAX_ERR_INVALID_ARG;
    const uint32_t N = p->block_size;
    const uint64_t nb = (n + N - 1) / N;
    const bool fq = p->mode == APAX_FIXED_QUALITY;
    // the shards tile [0, nb) in order; their payload sizes from their byte counts
    uint64_t next = 0, payload = 0;
    for (int i = 0; i < count; ++i) {
        const apax_shard &sh = shards[i];
        if (!sh.container || ((uintptr_t)sh.container & 3) || sh.block_begin != next ||
            sh.block_end <= sh.block_begin || sh.block_end > nb)
            return APAX_ERR_INVALID_ARG;
        const uint64_t head = 40 + (fq ? table_bytes(sh.block_end - sh.block_begin) : 0);
        if (sh.bytes < head || ((sh.bytes - head) & 3)) return APAX_ERR_INVALID_ARG;
        payload += sh.bytes - head;
        next = sh.block_end;
    }
    if (next != nb) return APAX_ERR_INVALID_ARG;
    if (fq && payload / 4 > 0xffffffffull) return APAX_ERR_TOO_LARGE;
    const uint64_t poff = 40 + (fq ? table_bytes(nb) : 0);
    if (out_capacity < poff + payload) return APAX_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *o = (uint8_t *)out;
    uint64_t at = 0;
    for (int i = 0; i < count; ++i) {
        const apax_shard &sh = shards[i];
        const uint64_t nbs = sh.block_end - sh.block_begin;
        const uint64_t head = 40 + (fq ? table_bytes(nbs) : 0);
        const uint8_t *src = (const uint8_t *)sh.container;
        if (fq) {
            st = cuda_fail(launch_table_rebase((const uint32_t *)(src + 40),
                                               (uint32_t *)(o + 40) + sh.block_begin, nbs, at / 4, s));
            if (st) return st;
        }
        if (sh.bytes > head) {
            st = cuda_fail(cudaMemcpyAsync(o + poff + at, src + head, sh.bytes - head,
                                           cudaMemcpyDeviceToDevice, s));
            if (st) return st;
        }
        at += sh.bytes - head;
    }
    if (fq && (nb & 1)) {  // the table's padding word
        st = cuda_fail(cudaMemsetAsync(o + 40 + 4 * nb, 0, 4, s));
        if (st) return st;
    }
    EncArgs a;
    memset(&a, 0, sizeof a);
    a.out = o;
    a.dtype = dtype;
    a.mode = p->mode;
    a.N = N;
    a.code = p->atten_code;
    a.B = p->mode == APAX_FIXED_RATE ? (uint32_t)budget(f, N, p->rate_num, p->rate_den) : 0;
    a.n_hdr = n;
    a.poff = poff;
    a.gsh = f.gs == 8 ? 1 : 0;
    a.sum = (f.opts & APAX_FORMAT_SUM_STREAM) ? 1 : 0;
    a.res = res;
    return cuda_fail(launch_merged_header(a, payload, s));
}

namespace {
// Spectral segment length for n elements (0 below 4 samples).
int quality_L(uint64_t n, int &logL)
{
    if (n < 4) {
        logL = 0;
        return 0;
    }
    int L = 4096;
    while ((uint64_t)L > n) L >>= 1;
    logL = 0;
    while ((1 << logL) < L) ++logL;
    return L;
}

struct QLayout {
    uint64_t state, hist, keys, tw, part, P, total;
};

QLayout quality_layout(uint64_t n)
{
    int logL;
    const int L = quality_L(n, logL);
    const uint64_t H = (uint64_t)L / 2, segs = L ? n / (uint64_t)L : 0;
    auto up = [](uint64_t v) { return (v + 255) / 256 * 256; };
    QLayout q;
    q.state = 0;
    q.hist = 256;
    q.keys = q.hist + up(256 * 8);
    q.tw = q.keys + up(8 * n);
    q.part = q.tw + up(16 * H);
    q.P = q.part + up(8 * 3 * H * quality_spectral_ctas(segs));
    q.total = q.P + up(8 * 3 * H);
    return q;
}
}  // namespace

int apax_quality_workspace_size(int dtype, uint64_t n, uint64_t *bytes)
{
    Fmt f;
    int st = fmt_of(dtype, f);
    if (st) return st;
    if (!bytes) return APAX_ERR_INVALID_ARG;
    *bytes = quality_layout(n).total;
    return APAX_OK;
}

int apax_quality_metrics(const void *x, const void *y, int dtype, uint64_t n, void *workspace,
                         uint64_t workspace_bytes, apax_quality *q, void *stream)
{
    Fmt f;
    int st = fmt_of(dtype, f);
    if (st) return st;
    if ((n && (!x || !y)) || !q || !workspace || ((uintptr_t)workspace & 255) ||
        ((uintptr_t)x % f.size) || ((uintptr_t)y % f.size) || ((uintptr_t)q & 7))
        return APAX_ERR_INVALID_ARG;
    const QLayout lay = quality_layout(n);
    if (workspace_bytes < lay.total) return APAX_ERR_CAPACITY;
    uint8_t *w = (uint8_t *)workspace;
    QualityArgs a;
    memset(&a, 0, sizeof a);
    a.x = x;
    a.y = y;
    a.dtype = dtype;
    a.n = n;
    a.state = (SelState *)(w + lay.state);
    a.hist = (unsigned long long *)(w + lay.hist);
    a.keys = (unsigned long long *)(w + lay.keys);
    a.L = quality_L(n, a.logL);
    a.segs = a.L ? n / (uint64_t)a.L : 0;
    a.tw = (double2 *)(w + lay.tw);
    a.part = (double *)(w + lay.part);
    a.P = (double *)(w + lay.P);
    a.q = q;
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_fail(cudaMemsetAsync(w, 0, lay.keys, s));  // state and counters
    if (st) return st;
    apax_quality head;
    memset(&head, 0, sizeof head);
    head.s2r_ratio = __builtin_nan("");
    head.n = n;
    head.L = (uint32_t)a.L;
    head.segments = (uint32_t)a.segs;
    // the header fields known on the host go in with a small kernel-free copy
    // of the whole record's defaults through the memset-cleared workspace:
    // the kernels overwrite the computed fields
    st = cuda_fail(launch_quality_header(q, head, s));
    if (st) return st;
    return cuda_fail(launch_quality(a, s));
}

void apax_quality_db(const apax_quality *q, double *out)
{
    auto db = [](double p) { return p > 0.0 ? 10.0 * log10(p) : (p == 0.0 ? -INFINITY : NAN); };
    const double r = q->s2r_ratio;
    out[0] = r != r ? r : (r == 0.0 ? -INFINITY : (isinf(r) ? INFINITY : 20.0 * log10(r)));
    out[1] = db(q->peak_x);
    out[2] = db(q->floor_x);
    out[3] = db(q->peak_y);
    out[4] = db(q->floor_y);
    out[5] = db(q->peak_d);
    out[6] = db(q->floor_d);
    out[7] = q->mean_d_db;
    out[8] = out[1] - out[2];
    out[9] = out[1] - out[7];
    out[10] = out[2] - out[7];
    if (!q->segments)
        for (int i = 1; i < 11; ++i) out[i] = NAN;
}

uint64_t apax_decode_workspace_size(void) { return kWsHead; }

int apax_decode(const void *in, uint64_t in_bytes, void *y, int dtype, uint64_t n,
                void *workspace, uint64_t workspace_bytes, apax_result *res, void *stream)
{
    // block count is unknown on the host (N is in the container): the kernel
    // bounds the range by the container's block count
    return decode_impl(in, in_bytes, 0, ~0ull, false, y, dtype, n, workspace, workspace_bytes,
                       res, stream);
}

int apax_decode_blocks(const void *in, uint64_t in_bytes, uint64_t block_begin,
                       uint64_t block_end, void *y, int dtype, uint64_t n, void *workspace,
                       uint64_t workspace_bytes, apax_result *res, void *stream)
{
    return decode_impl(in, in_bytes, block_begin, block_end, true, y, dtype, n, workspace,
                       workspace_bytes, res, stream);
}

int apax_profile_workspace_size(int dtype, uint64_t n, uint32_t block_size, int ncand,
                                uint64_t *bytes)
{
    Fmt f;
    int st = fmt_of(dtype, f);
    if (st) return st;
    if (!block_size_ok(block_size)) return APAX_ERR_BLOCK_SIZE;
    if (ncand < 1 || ncand > 32 || !bytes) return APAX_ERR_INVALID_ARG;
    const uint64_t nb = (n + block_size - 1) / block_size;
    const uint64_t nruns = (nb + 15) / 16;
    const uint64_t Qn = 2 + 4 * (uint64_t)ncand;
    const uint64_t head = kWsHead + 8 * 32;
    const uint64_t runs = 8 * Qn * (nruns ? nruns : 1);
    const uint64_t scratch = 8 * Qn * 2 * (((nruns + 15) / 16) + 1);
    const uint64_t flags = (nruns + 15) / 16 * 16;  // runs left to the team sweep
    const uint64_t sel = (nb + 15) / 16 * 16;       // stream decisions (the sum stream)
    *bytes = head + runs + scratch + flags + sel;
    return APAX_OK;
}

int apax_profile(const void *x, int dtype, uint64_t n, uint32_t block_size,
                 const uint16_t *candidates, int ncand, double target, void *workspace,
                 uint64_t workspace_bytes, apax_profile_point *points,
                 apax_profile_summary *summary, void *stream)
{
    return apax_profile_format(x, dtype, n, block_size, 0, candidates, ncand, target, workspace,
                               workspace_bytes, points, summary, stream);
}

int apax_profile_format(const void *x, int dtype, uint64_t n, uint32_t block_size,
                        uint32_t format, const uint16_t *candidates, int ncand, double target,
                        void *workspace, uint64_t workspace_bytes, apax_profile_point *points,
                        apax_profile_summary *summary, void *stream)
{
    ProfArgs a;
    int st = fill_prof_args(x, dtype, n, block_size, format, candidates, ncand, target, points,
                            summary, a);
    if (st) return st;
    if (!workspace || ((uintptr_t)workspace & 15)) return APAX_ERR_INVALID_ARG;
    uint64_t need;
    st = apax_profile_workspace_size(dtype, n, block_size, ncand, &need);
    if (st) return st;
    if (workspace_bytes < need) return APAX_ERR_CAPACITY;
    place_profile_workspace(a, workspace);
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_fail(cudaMemsetAsync(workspace, 0, kWsHead + 8 * 32, s));
    if (st) return st;
    return cuda_fail(launch_profile(a, s));
}

int apax_profile_from_host(const void *x_host, void *x_dev, int dtype, uint64_t n,
                           uint32_t block_size, const uint16_t *candidates, int ncand,
                           double target, int chunks, void *workspace, uint64_t workspace_bytes,
                           apax_profile_point *points, apax_profile_summary *summary,
                           void *stream, void *copy_stream)
{
    ProfArgs a;
    int st = fill_prof_args(x_dev, dtype, n, block_size, 0, candidates, ncand, target, points,
                            summary, a);
    if (st) return st;
    if ((!x_host && n) || chunks < 1 || chunks > 64 || stream == copy_stream)
        return APAX_ERR_INVALID_ARG;
    if (!workspace || ((uintptr_t)workspace & 15)) return APAX_ERR_INVALID_ARG;
    uint64_t need;
    st = apax_profile_workspace_size(dtype, n, block_size, ncand, &need);
    if (st) return st;
    if (workspace_bytes < need) return APAX_ERR_CAPACITY;
    place_profile_workspace(a, workspace);
    Fmt f;
    fmt_of(dtype, f);
    cudaStream_t s = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
    st = cuda_fail(cudaMemsetAsync(workspace, 0, kWsHead + 8 * 32, s));
    if (st) return st;
    // Fork: the copies and the sweep streams wait for the work already
    // queued on `stream` (which may still read x_dev).  Piece c goes over on
    // copy_stream; its runs go on sweep stream c mod kSweepStreams once the
    // piece is there, so pieces' sweeps overlap one another as well as the
    // later copies (a piece is a fraction of a wave).  Join: `stream` waits
    // for every sweep stream, then sums the tree.
    cudaStream_t ss[kSweepStreams];
    if (!sweep_streams(ss)) return APAX_ERR_CUDA;
    cudaEvent_t ev[2 + 64 + kSweepStreams];
    int nev = 0;
    auto fail = [&](cudaError_t e) {
        for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
        return cuda_fail(e);
    };
    auto event = [&](cudaEvent_t *out) {
        const cudaError_t e = cudaEventCreateWithFlags(&ev[nev], cudaEventDisableTiming);
        if (e == cudaSuccess) *out = ev[nev++];
        return e;
    };
    cudaEvent_t fork;
    cudaError_t e = event(&fork);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaEventRecord(fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, fork, 0)) != cudaSuccess)
        return fail(e);
    const int nss = chunks < kSweepStreams ? chunks : kSweepStreams;
    for (int k = 0; k < nss; ++k)
        if ((e = cudaStreamWaitEvent(ss[k], fork, 0)) != cudaSuccess) return fail(e);
    const uint64_t R = a.nruns, per_run = 16ull * block_size;
    for (int c = 0; c < chunks; ++c) {
        const uint64_t r0 = R * (uint64_t)c / (uint64_t)chunks, r1 = R * (uint64_t)(c + 1) / (uint64_t)chunks;
        if (r1 <= r0) continue;
        const uint64_t e0 = r0 * per_run, e1 = r1 * per_run < n ? r1 * per_run : n;
        e = cudaMemcpyAsync((uint8_t *)x_dev + e0 * f.size, (const uint8_t *)x_host + e0 * f.size,
                            (e1 - e0) * f.size, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return fail(e);
        cudaEvent_t landed;
        if ((e = event(&landed)) != cudaSuccess) return fail(e);
        cudaStream_t sk = ss[c % nss];
        if ((e = cudaEventRecord(landed, cs)) != cudaSuccess || (e = cudaStreamWaitEvent(sk, landed, 0)) != cudaSuccess)
            return fail(e);
        ProfArgs b = a;
        b.run0 = r0;
        b.run1 = r1;
        // with more than one piece every piece takes the team sweep (no run
        // flags): its runs end soon after the piece lands, where the
        // one-block-per-thread sweep's long per-thread walks outlast the copy
        // and hold the SMs' registers while later pieces wait (64 MiB float32
        // in 8 pieces: 0.574 ms with it on every piece, 0.57 on the first
        // quarter only, 0.512 never).  One piece overlaps nothing inside the
        // call, so it keeps the faster sweep.
        if (chunks > 1) b.run_flags = nullptr;
        if ((e = launch_profile_runs(b, sk)) != cudaSuccess) return fail(e);
    }
    // join: the copy stream (every piece is on the device) and the sweeps
    cudaEvent_t jc;
    if ((e = event(&jc)) != cudaSuccess) return fail(e);
    if ((e = cudaEventRecord(jc, cs)) != cudaSuccess || (e = cudaStreamWaitEvent(s, jc, 0)) != cudaSuccess)
        return fail(e);
    for (int k = 0; k < nss; ++k) {
        cudaEvent_t j;
        if ((e = event(&j)) != cudaSuccess) return fail(e);
        if ((e = cudaEventRecord(j, ss[k])) != cudaSuccess || (e = cudaStreamWaitEvent(s, j, 0)) != cudaSuccess)
            return fail(e);
    }
    e = launch_profile_tree(a, s);
    // events recorded and waited on are released by CUDA once complete
    for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    return cuda_fail(e);
}

static double corr_host(double sxx, double sxy, double syy)
{
    if (!isfinite(sxx) || !isfinite(sxy) || !isfinite(syy)) {
        const uint64_t b = 0x7ff8000000000000ull;
        double r;
        memcpy(&r, &b, sizeof r);
        return r;
    }
    if (sxx == 0.0 && syy == 0.0) return 1.0;
    if (sxx == 0.0 || syy == 0.0) return 0.0;
    double p = sxx * syy;
    if (isfinite(p) && p >= 2.2250738585072014e-308) return sxy / sqrt(p);
    return (sxy / sqrt(sxx)) / sqrt(syy);
}

void apax_derived_metrics(const apax_profile_point *pt, uint64_t n, double *out)
{
    const double sx = pt->sx, sy = pt->sy, sxx = pt->sxx, sxy = pt->sxy, syy = pt->syy,
                 sdd = pt->sdd;
    out[0] = corr_host(sxx, sxy, syy);
    if (n == 0) {
        for (int i = 1; i < 11; ++i) out[i] = 0.0;
        return;
    }
    const double nn = (double)n;
    const double vx = sxx - sx * sx / nn, vy = syy - sy * sy / nn, cv = sxy - sx * sy / nn;
    if (vx <= 0.0 && vy <= 0.0) out[1] = 1.0;
    else if (vx <= 0.0 || vy <= 0.0) out[1] = 0.0;
    else out[1] = cv / sqrt(vx * vy);
    if (sdd == 0.0) {
        out[2] = INFINITY;
        out[3] = 0.0;
        out[4] = -INFINITY;
    } else if (sxx == 0.0) {
        out[2] = -INFINITY;
        out[3] = INFINITY;
        out[4] = INFINITY;
    } else {
        out[2] = 10.0 * log10(sxx / sdd);
        out[3] = 100.0 * sqrt(sdd / sxx);
        out[4] = 20.0 * log10(out[3] / 100.0);
    }
    const double mx = sx / nn, my = sy / nn, md = (sx - sy) / nn;
    out[5] = mx;
    out[6] = my;
    out[7] = md;
    double t = sxx / nn - mx * mx;
    out[8] = sqrt(t > 0.0 ? t : 0.0);
    t = syy / nn - my * my;
    out[9] = sqrt(t > 0.0 ? t : 0.0);
    t = sdd / nn - md * md;
    out[10] = sqrt(t > 0.0 ? t : 0.0);
}

const char *apax_status_string(int status)
{
    switch (status) {
    case APAX_OK: return "ok";
    case APAX_ERR_INVALID_ARG: return "invalid argument";
    case APAX_ERR_BLOCK_SIZE: return "block size outside 64..16384 or not a multiple of 4";
    case APAX_ERR_DTYPE: return "unknown element type";
    case APAX_ERR_RATE: return "fixed rate outside the representable packet sizes";
    case APAX_ERR_CAPACITY: return "output or workspace too small";
    case APAX_ERR_TOO_LARGE: return "payload beyond 2^32 words";
    case APAX_ERR_CUDA: return "CUDA runtime error";
    case APAX_ERR_NONFINITE: return "non-finite float input";
    case APAX_ERR_CORRUPT: return "corrupt stream";
    case APAX_ERR_TIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
    }
}

const char *apax_build_info(void) { return "apax-gb300 1.0 sm_103a"; }

}  // extern "C"
