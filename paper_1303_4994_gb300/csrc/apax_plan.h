// apax_plan.h -- host-side validation, container sizes and launch planning
// shared by the single-array and batched entry points (internal).
#pragma once

#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

#include "apax_team.cuh"
#include "apax_kernels.h"

namespace apax {
namespace host {

struct Fmt {
    int size = 0, W = 0, F = 0, H = 0;  // zero until fmt_of fills them
    int gs = 4;          // BFPE group size (8 with APAX_FORMAT_GROUP8)
    uint32_t opts = 0;   // APAX_FORMAT_* bits
};

inline int fmt_of(int dtype, Fmt &f)
{
    switch (dtype) {
    case APAX_I8: f = {1, 8, 0, 32}; return APAX_OK;
    case APAX_I16: f = {2, 16, 0, 32}; return APAX_OK;
    case APAX_I32: f = {4, 32, 0, 32}; return APAX_OK;
    case APAX_F32: f = {4, 32, 1, 48}; return APAX_OK;
    case APAX_F64: f = {8, 32, 1, 48}; return APAX_OK;
    default: return APAX_ERR_DTYPE;
    }
}

inline bool block_size_ok(uint32_t N) { return N >= 64 && N <= 16384 && (N % 4) == 0; }

// Format options: known bits only; groups of 8 need whole groups per block.
inline int fmt_opts(uint32_t format, uint32_t N, Fmt &f)
{
    if (format & ~(uint32_t)(APAX_FORMAT_GROUP8 | APAX_FORMAT_SUM_STREAM)) return APAX_ERR_INVALID_ARG;
    f.opts = format;
    f.gs = (format & APAX_FORMAT_GROUP8) ? 8 : 4;
    if (N % (uint32_t)f.gs) return APAX_ERR_BLOCK_SIZE;
    return APAX_OK;
}

// Groups of 4 samples per team thread.  With groups of 8 a thread owns an
// even number of them (whole groups of 8).
inline int groups_per_thread(uint32_t N, int gs, int ts)
{
    return gs == 8 ? 2 * (int)((N / 8 + ts - 1) / ts) : (int)((N / 4 + ts - 1) / ts);
}

inline uint64_t pad32(uint64_t bits) { return 4 * ((bits + 31) / 32); }

inline uint64_t minpacket(const Fmt &f, uint64_t L)
{
    uint64_t G = (L + f.gs - 1) / f.gs;
    return pad32((uint64_t)f.H + 8 + 4 * ((G - 1 + 1) / 2));
}

inline uint64_t budget(const Fmt &f, uint64_t L, uint32_t num, uint32_t den)
{
    uint64_t b = (L * (uint64_t)f.size * den / (4ull * num)) * 4;
    uint64_t mp = minpacket(f, L);
    return b > mp ? b : mp;
}

inline uint64_t table_bytes(uint64_t nb) { return ((4 * nb) + 7) / 8 * 8; }

inline int check(int dtype, const apax_params *p, Fmt &f)
{
    if (!p) return APAX_ERR_INVALID_ARG;
    int st = fmt_of(dtype, f);
    if (st) return st;
    if (!block_size_ok(p->block_size)) return APAX_ERR_BLOCK_SIZE;
    st = fmt_opts(p->format, p->block_size, f);
    if (st) return st;
    if (p->search > APAX_SEARCH_PREDICT) return APAX_ERR_INVALID_ARG;
    if (p->mode == APAX_FIXED_RATE) {
        if (p->rate_num == 0 || p->rate_den == 0) return APAX_ERR_RATE;
        uint64_t B = ((uint64_t)p->block_size * f.size * p->rate_den / (4ull * p->rate_num)) * 4;
        if (B < minpacket(f, p->block_size) || B >= (1u << 18)) return APAX_ERR_RATE;
    } else if (p->mode == APAX_FIXED_QUALITY) {
        if (p->atten_code > 4095) return APAX_ERR_INVALID_ARG;
    } else {
        return APAX_ERR_INVALID_ARG;
    }
    return APAX_OK;
}

// Encoder launch plan.  A team of TS threads owns a block; its shared
// memory holds the block's packet image and exponent bytes.  Teams of 8
// (16 per 128-thread CTA) when that fits, else teams of 32 (one per warp).
struct Plan {
    int ts, threads;
    uint32_t pkt_words, ebuf_words;
    int gp;
    size_t smem;
    uint64_t ntiles;
};

// Shared-memory words of one team: the largest possible packet, or the
// whole fixed-rate budget when that is larger (packets are padded to it),
// then the exponent bytes.
inline void team_words(const Fmt &f, uint32_t N, uint64_t fr_budget_bytes, uint32_t &pkt_words,
                       uint32_t &ebuf_words)
{
    pkt_words = max_packet_words(f.H, f.W, N);
    if (fr_budget_bytes / 4 > pkt_words) pkt_words = (uint32_t)(fr_budget_bytes / 4);
    ebuf_words = ((N / 4) + 3) / 4;
}

constexpr size_t kEncSmemCap = 200 * 1024;

// Geometry for a given team size and CTA size.
inline Plan plan_geometry(uint32_t N, uint64_t nb, uint32_t pkt_words, uint32_t ebuf_words, int ts,
                          int threads, int gs = 4)
{
    Plan pl;
    pl.ts = ts;
    pl.threads = threads;
    pl.pkt_words = pkt_words;
    pl.ebuf_words = ebuf_words;
    const int nteams = threads / ts;
    pl.gp = groups_per_thread(N, gs, ts);
    pl.smem = (size_t)nteams * (pkt_words + ebuf_words) * 4;
    pl.ntiles = nb ? (nb + nteams - 1) / nteams : 1;
    return pl;
}

// Team size and CTA size of a single-array encode (the workspace size and
// the launch both come from here): teams of 8, 16 per 128-thread CTA, when
// their packets fit and the array is large; teams of 32 for small arrays (4
// per CTA) and for packets too large for 16 teams (as many warps as fit).
inline void default_geometry(size_t per_team_bytes, uint64_t nb, int &ts, int &threads)
{
    if (16 * per_team_bytes <= kEncSmemCap) {
        ts = nb <= kTeam32MaxBlocks ? 32 : 8;
        threads = 128;
    } else {
        ts = 32;
        int warps = 4;
        while (warps > 1 && (size_t)warps * per_team_bytes > kEncSmemCap) --warps;
        threads = 32 * warps;
    }
}

// Shared-memory staging of a tile (its blocks and the one before): the
// bytes, or 0 when it would not leave room for enough CTAs per SM.
constexpr size_t kStageCap = 48 * 1024, kStageTotalCap = 100 * 1024;

inline size_t stage_bytes(int elem_size, uint32_t N, int nteams, size_t smem_before)
{
    const size_t b = ((size_t)(nteams + 1) * N * elem_size + 15) / 16 * 16;
    return (b <= kStageCap && smem_before + b <= kStageTotalCap) ? b : 0;
}

inline Plan plan_encode(const Fmt &f, uint32_t N, uint64_t nb, uint64_t fr_budget_bytes)
{
    uint32_t pw, ew;
    team_words(f, N, fr_budget_bytes, pw, ew);
    int ts, threads;
    default_geometry((size_t)(pw + ew) * 4, nb, ts, threads);
    return plan_geometry(N, nb, pw, ew, ts, threads, f.gs);
}

constexpr uint64_t kWsHead = 64;  // ticket, done, status (+ padding)

// Validate one encode call and fill its per-array arguments (everything
// but the team geometry and the workspace pointers).
int fill_enc_args(const void *x, int dtype, uint64_t n, const apax_params *p,
                  const uint32_t *code_dev, void *out, uint64_t cap, apax_result *res, EncArgs &a,
                  uint32_t &pkt_words, uint32_t &ebuf_words);

// Validate one profile call and fill its arguments (all but the workspace
// pointers).
int fill_prof_args(const void *x, int dtype, uint64_t n, uint32_t block_size, uint32_t format,
                   const uint16_t *candidates, int ncand, double target,
                   apax_profile_point *points, apax_profile_summary *summary, ProfArgs &a);

// Batch plans (apax_batch.cu).  op: 0 encode, 1 decode, 2 profile; jobs
// points at apax_encode_job / apax_decode_job / apax_profile_job.  With
// `pinned` the plan's tables are copied from that pinned host staging on
// `stream` (asynchronously) instead of with a synchronous copy.
int batch_create(int op, const void *jobs, int count, void *workspace, uint64_t workspace_bytes,
                 uint8_t *pinned, uint64_t pinned_bytes, cudaStream_t stream, bool use_tuned,
                 apax_batch **plan);
uint64_t batch_workspace_bytes(int op, const void *jobs, int count);  // 0 on error

inline int cuda_fail(cudaError_t e) { return e == cudaSuccess ? APAX_OK : APAX_ERR_CUDA; }


}  // namespace host
}  // namespace apax
