// apax_kernels.h -- argument blocks and launchers shared by the host layer
// and the kernel translation units (internal; not part of the C ABI).
#pragma once

#include <stdint.h>
#include <atomic>
#include <cuda_runtime.h>

#include "../../include/apax.h"

namespace apax {

// Block-per-thread paths (decode and the fixed-rate search): block sizes up
// to kT1MaxBlock samples; a single array takes them when it has at least
// kT1MinBlocks blocks (fewer leave SMs idle, so teams are used), a batch
// always does.
constexpr uint32_t kT1MaxBlock = 1024;
constexpr uint64_t kT1MinBlocks = 32768;

// Arrays (or decoded block ranges) of at most this many blocks run with
// teams of 32, a block per warp: they do not fill the GPU, so the per-lane
// sequential chain (8 samples of a 256-sample block instead of 32) sets the
// time.  Measured on the int16 sensor trace (1024 blocks at 4:1): encode
// 52 -> 33 us; at 8192 blocks teams of 8 are faster again (66 vs 74 us).
constexpr uint64_t kTeam32MaxBlocks = 4096;

// Raises kernel K's dynamic shared-memory limit on the current device to at
// least `bytes`, calling the runtime only when the limit has to grow: the
// attribute call costs host time between a call's first and last launch,
// which single small calls feel.  The cache assumes one CUDA context per
// device for the life of the process (no cudaDeviceReset in between).
template <auto K>
inline cudaError_t smem_limit(size_t bytes)
{
    constexpr int kDevs = 64;
    static std::atomic<int> have[kDevs];  // static storage: starts at zero
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool known = dev >= 0 && dev < kDevs;
    if (known && have[dev].load(std::memory_order_acquire) >= (int)bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && known) {
        int cur = have[dev].load(std::memory_order_relaxed);
        while (cur < (int)bytes && !have[dev].compare_exchange_weak(cur, (int)bytes)) {
        }
    }
    return e;
}

// Multiprocessor count of the current device, read once per device.
inline int sm_count()
{
    constexpr int kDevs = 64;
    static std::atomic<int> count[kDevs];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev >= 0 && dev < kDevs) {
        const int c = count[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return 152;
    if (dev >= 0 && dev < kDevs) count[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

struct EncArgs {
    const void *x;      // element 0 of the array (a shard's x is offset so that
                        // its blocks sit at their global places)
    uint64_t n;
    uint32_t N;
    uint64_t nb;        // blocks (the end of the encoded range)
    uint64_t jb0;       // first block encoded (0, or a shard's first block)
    uint64_t n_hdr;     // elements named in the container header
    int dtype;
    int mode;           // 0 fixed rate, 1 fixed quality
    uint32_t code;      // fixed-quality code
    const uint32_t *code_dev;  // if set: code read on the device
    uint32_t B;         // fixed-rate budget of a full block
    uint32_t rate_num, rate_den;
    int search;         // fixed-rate search policy (APAX_SEARCH_*)
    uint64_t fr_payload; // fixed-rate payload bytes (exact, host computed)
    uint8_t *out;
    uint64_t cap;
    uint64_t poff;      // payload offset in the container
    uint32_t pkt_words, ebuf_words;  // per-team shared-memory layout
    uint32_t stage_off; // byte offset of the staged tile in shared memory (0: none)
    int t1;             // batches: this array is encoded one block per thread
    int gp;             // groups of 4 per team thread (even with groups of 8)
    int gsh;            // log2(BFPE group size / 4): 0, or 1 for groups of 8
    int sum;            // the sum stream is a candidate (format version 2)
    const uint8_t *sel; // single arrays with the sum stream: the stream of block
                        // jb0 + i at sel[i] (launch_best_streams), else NULL
    uint64_t ntiles;
    // workspace
    unsigned *ticket;
    unsigned *done;
    int *status;
    unsigned long long *tiles;
    long long spin_limit;      // clock cycles of a bounded wait
    long long test_stall_tile; // test hook: this tile never publishes (-1: off)
    apax_result *res;
};

// Many arrays in one launch: jobs[i] owns global tiles
// [tile_prefix[i], tile_prefix[i + 1]).
struct EncBatchArgs {
    const EncArgs *jobs;
    const uint64_t *tile_prefix;  // count + 1 entries
    int count;
    uint64_t total_tiles;
    unsigned long long *ticket;
};

struct DecArgs {
    const uint8_t *in;
    uint64_t in_bytes;
    void *y;
    int dtype;
    uint64_t n;
    uint64_t b0, b1;    // block range to decode
    bool ranged;        // y receives blocks [b0, b1) from y[0]
    unsigned *done;     // two completion counters (one per size class)
    unsigned long long *ticket;  // tile counter of the block-per-thread mode
    int *status;
    unsigned nctas, nctas_large;
    bool small_launched;  // the teams-of-8 / block-per-thread launch runs (else
                          // every container belongs to the teams-of-32 one)
    apax_result *res;
};

// Many containers in one launch: jobs[i] owns global tiles
// [tile_prefix[i], tile_prefix[i + 1]) of its declared block size.
struct DecBatchArgs {
    const DecArgs *jobs;
    const uint64_t *tile_prefix;  // count + 1 entries
    const uint64_t *tiles_of;     // tiles per job
    const uint32_t *block_size;   // declared block size per job
    int count;
    uint64_t total_tiles;
    unsigned long long *ticket;
};

// Profiler team size: threads per codec block (16 blocks per CTA).
constexpr int kProfTS = 8;

struct ProfArgs {
    const void *x;
    uint64_t n;
    uint32_t N;
    uint64_t nb;
    int dtype;
    int ncand;
    uint32_t codes[32];
    uint64_t nruns;     // level-1 nodes (16 blocks each)
    uint64_t run0, run1; // runs swept by one launch of the run kernel
    uint32_t stage_off; // byte offset of the staged run in shared memory (0: none)
    int gp;             // groups of 4 per team thread (even with groups of 8)
    int gsh;            // log2(BFPE group size / 4) of the byte counts
    int sum;            // the sum stream is a candidate of the byte counts
    const uint8_t *sel; // single arrays with the sum stream: block j's stream at
                        // sel[j] (launch_best_streams), else NULL
    double *run_sums;   // [nruns][2 + 4*ncand]: sx, sxx, then (sy, sxy, syy, sdd) per candidate
    unsigned long long *bytes;  // [ncand] payload bytes (atomic)
    int *status;
    unsigned *done;
    unsigned nctas;
    double target;
    double *scratch;    // tree levels
    apax_profile_point *points;
    apax_profile_summary *summary;
    uint8_t *run_flags;  // [nruns] runs left to the team kernel by the one-block-per-thread
                         // sweep (NULL: that sweep is not used)
};

// Signal-quality metrics (apax_quality.cu).
struct SelState {
    unsigned long long prefix;  // key bits chosen so far
    unsigned long long k;       // rank still to find among the keys matching prefix
    int shift;                  // bit position of the byte being counted
    int pad;
};
struct QualityArgs {
    const void *x, *y;
    int dtype;
    uint64_t n;
    SelState *state;
    unsigned long long *hist;  // 256 counters
    unsigned long long *keys;  // n
    int L, logL;               // spectral segment length (0: no spectrum)
    uint64_t segs;
    double2 *tw;               // L/2 twiddles
    double *part;              // per-CTA periodogram sums
    double *P;                 // 3 * L/2 averaged bins
    apax_quality *q;
};
uint64_t quality_spectral_ctas(uint64_t segs);
cudaError_t launch_quality(const QualityArgs &a, cudaStream_t s);
cudaError_t launch_quality_header(apax_quality *q, const apax_quality &h, cudaStream_t s);

// The one-block-per-thread float32 sweep (apax_profile_t1.cu): arrays of at
// least this many blocks of at most 256 samples, candidates 0 then
// power-of-two attenuations.
constexpr uint64_t kProfT1MinBlocks = 16384;
bool profile_t1_eligible(const ProfArgs &a);
cudaError_t launch_profile_t1(const ProfArgs &a, cudaStream_t s);

cudaError_t launch_encode(const EncArgs &a, int ts, int threads, size_t smem, cudaStream_t s);
// Single arrays whose blocks fit the registers of a team of 8 (fixed
// quality, at most 256 samples of int8, int16 or float32): apax_encode_res.cu.
bool encode_res_eligible(int dtype, int mode, uint32_t N, int ts);
cudaError_t launch_encode_res(const EncArgs &a, int threads, size_t smem, cudaStream_t s);

// Stream decisions of blocks [j0, j0 + count) of an array with the sum
// stream into sel[0, count) (apax_select.cu).
struct SelArgs {
    const void *x;   // block j at x + j N
    uint64_t n;
    uint32_t N;
    uint64_t nb;     // blocks of the array (or the end of a shard's range)
    uint64_t j0, count;
    int dtype;
    int gsh;
    int gp;          // set by the launcher
    uint8_t *sel;
};
cudaError_t launch_best_streams(const SelArgs &a, cudaStream_t s);
// Shard merging: dst[i] = src[i] + add for i < count; the merged header
// (a.out, a.n_hdr, a.mode, a.code, a.B, a.poff) and a.res.
cudaError_t launch_table_rebase(const uint32_t *src, uint32_t *dst, uint64_t count, uint64_t add,
                                cudaStream_t s);
cudaError_t launch_merged_header(const EncArgs &a, uint64_t payload, cudaStream_t s);
// dst[0, min(res->bytes, cap)) = src[...], the size read on the device.
cudaError_t launch_copy_sized(const void *src, const apax_result *res, void *dst, uint64_t cap,
                              cudaStream_t s);
cudaError_t launch_encode_batch(const EncBatchArgs &b, int ts, int threads, size_t smem,
                               unsigned ctas, cudaStream_t s);
int encode_batch_occupancy(int ts, int threads, size_t smem);  // CTAs per SM
cudaError_t launch_decode(const DecArgs &a, cudaStream_t s);
cudaError_t launch_decode_batch(const DecBatchArgs &b, int ts, int threads, unsigned ctas,
                               cudaStream_t s);
int decode_batch_occupancy(int ts, int threads);
cudaError_t launch_profile(const ProfArgs &a, cudaStream_t s);       // all runs, then the tree
cudaError_t launch_profile_runs(const ProfArgs &a, cudaStream_t s);  // runs [a.run0, a.run1)
cudaError_t launch_profile_tree(const ProfArgs &a, cudaStream_t s);  // tree and finalisation

// Many arrays' profiler sweeps in one launch: jobs[i] owns global runs
// [run_prefix[i], run_prefix[i + 1]) (at least one, to finalise empty arrays).
struct ProfBatchArgs {
    const ProfArgs *jobs;
    const uint64_t *run_prefix;
    int count;
    uint64_t total_runs;
    unsigned long long *ticket;
};
cudaError_t launch_profile_batch(const ProfBatchArgs &b, int max_ncand, unsigned ctas,
                                 cudaStream_t s);
int profile_batch_occupancy(int max_ncand);

// apax_encode with an already-sized workspace supplied by another entry point.
int encode_with_workspace(const void *x, int dtype, uint64_t n, const apax_params *p, void *out,
                          uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                          apax_result *res, void *stream);

}  // namespace apax
