/*
 * apax.h -- C ABI of the GB300 APAX codec library (libapax_gb300.so).
 *
 * The library implements the data-parallel hot path of the APAX universal
 * numerical encoder and profiler of Wegener, "Universal Numerical Encoder and
 * Profiler Reduces Computing's Memory Wall with Software, FPGA, and SoC
 * Implementations" (arXiv 1303.4994):
 *   - Sec. 6 (encoder block diagram): blocks of 64..16384 samples, a per-block
 *     attenuator, a redundancy remover choosing among the data and its
 *     derivatives with the decision of block j carried in block j+1's header,
 *     and a 4-byte (integer) or 6-byte (float) block header;
 *   - Sec. 6 (bit packer): block floating point with one exponent per group of
 *     4 samples (or 8, an option) and joint exponent encoding of the
 *     exponents;
 *   - Sec. 6 (signal monitor) and Sec. 5 (Fig. 3b): as an option, the sum of
 *     neighbouring samples as a fourth stream, for data near the Nyquist
 *     frequency;
 *   - Sec. 4 (profiler): a sweep over encoding settings reporting
 *     r = sum(xy) / sqrt(sum(x^2) sum(y^2)) and a recommended setting at a
 *     correlation target.
 * The exact bitstream (field layout, derivative set, attenuation values,
 * rounding, fixed-rate search, container) follows the readings listed with
 * the project's design notes; the paper leaves those open.
 *
 * Conventions for every call:
 *   - Pointers named x, y, out, in, workspace, res, points and summary are
 *     DEVICE pointers unless the comment says host.  res / points / summary
 *     may also be host-pinned memory mapped into the device address space.
 *   - The caller owns every buffer.  The library never allocates device
 *     memory and never synchronises the stream inside an asynchronous call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - The return value reports argument errors found on the host (0 = the
 *     work was enqueued).  Errors that depend on the data (non-finite input,
 *     corrupt stream, output capacity, timeout) are written by the kernels to
 *     res->status when the work completes; read it after synchronising.
 *   - Asynchronous calls only enqueue kernels and cudaMemsetAsync; they may be
 *     captured in a CUDA graph.
 */
#ifndef APAX_GB300_H
#define APAX_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types (Sec. 7 datasets: int8/16/32 and 32/64-bit floats). */
typedef enum { APAX_I8 = 1, APAX_I16 = 2, APAX_I32 = 3, APAX_F32 = 4, APAX_F64 = 5 } apax_dtype;

/* Encoding modes (Sec. 6 adaptive loop: a target packet size, or a fixed
 * attenuation for a quality target). */
typedef enum { APAX_FIXED_RATE = 0, APAX_FIXED_QUALITY = 1 } apax_mode;

/* Status codes: returned by calls (host-side checks) and written to
 * apax_result.status (data-dependent errors). */
enum {
    APAX_OK = 0,
    APAX_ERR_INVALID_ARG = -1, /* bad pointer, count, mode, code, or dtype/n mismatch on decode */
    APAX_ERR_BLOCK_SIZE = -2,  /* block size outside 64..16384 or not a multiple of the group size (Sec. 6) */
    APAX_ERR_DTYPE = -3,       /* unknown element type */
    APAX_ERR_RATE = -4,        /* fixed-rate budget below the all-zero packet or above 2^18 B */
    APAX_ERR_CAPACITY = -5,    /* output or workspace smaller than required */
    APAX_ERR_TOO_LARGE = -6,   /* payload beyond 2^32 words (offset table limit) */
    APAX_ERR_CUDA = -7,        /* a CUDA runtime call failed */
    APAX_ERR_NONFINITE = -8,   /* NaN or infinity in a float input */
    APAX_ERR_CORRUPT = -9,     /* malformed stream (header, tokens, offsets, lengths) */
    APAX_ERR_TIMEOUT = -10     /* a bounded device wait expired (offset scan) */
};

/* Fixed-rate search policies (Sec. 6 adaptive loop: the attenuation of each
 * block is adjusted until its packet meets the rate).  The policy is the
 * encoder's: it is not stored in the stream, and any decoder reads either.
 *   APAX_SEARCH_BISECT   code 0 if it fits, else bisection of [0, 4095]
 *                        keeping the upper end fitting (13 packet sizings).
 *   APAX_SEARCH_PREDICT  code 0 if it fits, else a start code predicted from
 *                        the code-0 exponents (the bits an attenuation of
 *                        2^-k removes from each group, interpolated in 1/16
 *                        octave steps), then up the ladder of codes
 *                        128 k + M[f] until the packet fits (usually 1-3
 *                        sizings).  The codes, and so the bytes, differ
 *                        from BISECT's. */
typedef enum { APAX_SEARCH_BISECT = 0, APAX_SEARCH_PREDICT = 1 } apax_search;

/* Format options (bits of apax_params.format).  With none the container is
 * version 1; with any it is version 2, which names the options in its flags
 * byte so that a decoder needs no parameter.
 *   APAX_FORMAT_GROUP8      BFPE groups of 8 samples instead of 4 (Sec. 6
 *                           bit packer: "groups of 4 or 8"): one exponent
 *                           and token per 8 samples.  The block size must
 *                           be a multiple of 8.
 *   APAX_FORMAT_SUM_STREAM  the redundancy remover also considers the sum
 *                           stream u_0 = q_0, u_i = q_i + q_{i-1} (block
 *                           header selector 3), small where the data
 *                           alternate in sign (a spectrum near the Nyquist
 *                           frequency, Sec. 5 Fig. 3b).  The stream of
 *                           fewest code-0 bits is chosen, as for the others
 *                           (Sec. 6 signal monitor and redundancy remover).
 * The options change how q is packed, never q: decoded values are the same
 * with every format. */
enum { APAX_FORMAT_GROUP8 = 1, APAX_FORMAT_SUM_STREAM = 2 };

/* Encoding parameters.
 *   block_size  N, 64..16384, multiple of 4 (Sec. 6).  256 is the default.
 *   mode        APAX_FIXED_RATE or APAX_FIXED_QUALITY.
 *   rate_num, rate_den   fixed rate num:den (e.g. 4:1): every full block's
 *               packet is exactly floor(N*size*den / (4*num))*4 bytes.
 *   atten_code  fixed-quality attenuation code c in 0..4095: k = c >> 7,
 *               m = c & 127, a(c) = (256 - m) 2^-(8+k); 4095 zeroes the data;
 *               0 is lossless for integer types.
 *   search      fixed-rate search policy (apax_search; ignored for fixed
 *               quality); other values give APAX_ERR_INVALID_ARG.
 *   format      format options (APAX_FORMAT_* bits; 0 = version 1); other
 *               bits give APAX_ERR_INVALID_ARG.
 */
typedef struct {
    uint32_t block_size;
    int32_t mode;
    uint32_t rate_num;
    uint32_t rate_den;
    uint32_t atten_code;
    uint32_t search;
    uint32_t format;
} apax_params;

/* Completion record written by the device when a call's work finishes:
 * status (APAX_OK or a negative code) and, for encode, the container size in
 * bytes; for decode, the number of elements written. */
typedef struct {
    int32_t status;
    uint32_t pad;
    uint64_t bytes;
} apax_result;

/* Size of the encoded container in bytes (host call, no device work).
 * Fixed rate: the exact size, 40 + (nblocks-1)*B + B_last.  Fixed quality:
 * a worst-case bound to size the output allocation.  Returns a status. */
int apax_encoded_size(int dtype, uint64_t n, const apax_params *p, uint64_t *bytes /* host */);

/* Device workspace bytes that apax_encode needs for these arguments
 * (fixed quality: the tile status words of the offset scan). */
int apax_workspace_size(int dtype, uint64_t n, const apax_params *p, uint64_t *bytes /* host */);

/* Encode n elements of x (C order, element type dtype) into out, a container
 * of at most out_capacity bytes: a 40-byte header, for fixed quality an
 * offset table of nblocks 32-bit word offsets (padded to 8 bytes), then one
 * packet per block.  workspace must hold apax_workspace_size() bytes; it is
 * cleared on the stream before use.  res receives the status and the
 * container size.  Calls that overlap in time on the device must use
 * distinct workspaces. */
int apax_encode(const void *x, int dtype, uint64_t n, const apax_params *p, void *out,
                uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                apax_result *res, void *stream);

/* Fixed-quality encode whose attenuation code is read on the device from
 * summary->recommended_code (written by apax_profile), so that a
 * profile -> encode -> decode pipeline needs no host round trip.
 * p->mode must be APAX_FIXED_QUALITY; p->atten_code is ignored. */
struct apax_profile_summary;
int apax_encode_recommended(const void *x, int dtype, uint64_t n, const apax_params *p,
                            const struct apax_profile_summary *summary, void *out,
                            uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                            apax_result *res, void *stream);

/* Copy a container out without a host round trip: the first
 * min(res->bytes, capacity) bytes of src (as apax_encode and
 * apax_encode_recommended leave them: res->bytes is read on the device when
 * the copy runs) to dst, by a kernel on `stream`.  dst may be device memory
 * or page-locked host memory mapped into the device address space (the
 * kernel then writes it over the host link), so a caller need not wait for
 * the encode to learn the size before moving the container to the host.
 * src and dst must be 4-byte aligned and must not overlap; enqueue the copy
 * after the encode that wrote src and res (same stream, or an event).  Not
 * a step of the paper's method: a transfer helper for its output. */
int apax_copy_container(const void *src, const apax_result *res, void *dst, uint64_t capacity,
                        void *stream);

/* Device workspace bytes of apax_decode / apax_decode_blocks (a status word,
 * one completion counter per launch and the block-per-thread tile counter). */
uint64_t apax_decode_workspace_size(void);

/* Decode a container of in_bytes bytes into y (n elements of dtype).  The
 * container header is checked on the device: a dtype or n different from the
 * arguments gives APAX_ERR_INVALID_ARG in res->status, a malformed stream
 * APAX_ERR_CORRUPT.  Never reads past in_bytes.  workspace: at least
 * apax_decode_workspace_size() bytes, cleared on the stream before use. */
int apax_decode(const void *in, uint64_t in_bytes, void *y, int dtype, uint64_t n,
                void *workspace, uint64_t workspace_bytes, apax_result *res, void *stream);

/* Random access (the offset table of fixed-quality containers, j*B for
 * fixed rate): decode only blocks [block_begin, block_end) into y, which
 * receives the elements of those blocks starting at y[0].  block_end must
 * not exceed the container's block count (else APAX_ERR_INVALID_ARG in
 * res->status). */
int apax_decode_blocks(const void *in, uint64_t in_bytes, uint64_t block_begin,
                       uint64_t block_end, void *y, int dtype, uint64_t n, void *workspace,
                       uint64_t workspace_bytes, apax_result *res, void *stream);

/* Profiler (Sec. 4).  One point per candidate code: the fixed-quality
 * container size at that code and the reconstruction sums of the decoded y
 * against x.  Each block's sums are exact and rounded once to binary64; the
 * array totals add the block values in a fixed fan-in-16 tree, so the
 * numbers are reproducible bit for bit. */
typedef struct {
    uint32_t code;   /* candidate attenuation code */
    uint32_t flags;  /* bit 0: r >= target */
    uint64_t bytes;  /* fixed-quality container size at this code */
    double sx, sy, sxx, sxy, syy, sdd; /* sums of x, y, x^2, xy, y^2, (x-y)^2 */
    double r;        /* sum(xy) / sqrt(sum(x^2) sum(y^2)) (Sec. 4) */
} apax_profile_point;

typedef struct apax_profile_summary {
    int32_t status;            /* APAX_OK or a data error (e.g. non-finite input) */
    int32_t recommended;       /* index of the recommended candidate */
    uint32_t recommended_code; /* its code */
    uint32_t flags;            /* bit 0: even the first candidate misses the target */
    uint64_t n;                /* elements profiled */
} apax_profile_summary;

/* Default candidate ladder: c_i = 256 i, i = 0..15 (a = 4^-i, 12 dB steps). */
#define APAX_PROFILE_DEFAULT_CANDIDATES 16

/* Workspace bytes apax_profile needs for n elements, block size N and ncand
 * candidates. */
int apax_profile_workspace_size(int dtype, uint64_t n, uint32_t block_size, int ncand,
                                uint64_t *bytes /* host */);

/* Sweep ncand candidate codes over x.  candidates (host) must be strictly
 * increasing codes of 0..4095; NULL selects the default ladder (ncand must
 * then be 16).  Power-of-two attenuations (codes that are multiples of 128)
 * take the fast exact-sum path; float candidates with m != 0 are summed by
 * an exact superaccumulator per block and sweep markedly slower.  The recommended
 * candidate is the largest i with r_j >= target for every j <= i, else 0
 * with summary->flags bit 0 set.  points (ncand entries) and summary are
 * written by the device; the call is asynchronous. */
int apax_profile(const void *x, int dtype, uint64_t n, uint32_t block_size,
                 const uint16_t *candidates /* host */, int ncand, double target,
                 void *workspace, uint64_t workspace_bytes, apax_profile_point *points,
                 apax_profile_summary *summary, void *stream);

/* apax_profile for containers with format options (APAX_FORMAT_* bits, as
 * in apax_params.format): each point's byte count is the size of the
 * fixed-quality container apax_encode writes with that format; the sums and
 * r depend only on the decoded values and equal apax_profile's.  Same
 * workspace size.  Format 0 is apax_profile. */
int apax_profile_format(const void *x, int dtype, uint64_t n, uint32_t block_size,
                        uint32_t format, const uint16_t *candidates /* host */, int ncand,
                        double target, void *workspace, uint64_t workspace_bytes,
                        apax_profile_point *points, apax_profile_summary *summary,
                        void *stream);

/* apax_profile for an array in page-locked host memory (x_host, e.g. from
 * cudaHostAlloc), leaving its copy in x_dev (device, n elements of dtype):
 * the array goes to the device in `chunks` pieces (1..64, whole runs of 16
 * blocks each) with cudaMemcpyAsync on copy_stream, and each piece is swept
 * (with more than one piece by the sweep with a team of threads per block,
 * whose short per-block latency ends each piece's sweep soon after it
 * lands; one piece takes apax_profile's own sweep once it is there)
 * as soon as it is there, on one of sixteen library-owned streams (created on
 * first use per device and kept for the process's CUDA context, so not
 * valid across cudaDeviceReset), so the copy hides behind the sweep.  The copies and
 * sweeps first wait for the work queued on `stream` before the call; work
 * queued on `stream` after it sees x_dev, points and summary.  Results are
 * identical to apax_profile on x_dev.  copy_stream must differ from stream.
 * Asynchronous: no host synchronisation; the events it uses are released by
 * CUDA once complete. */
int apax_profile_from_host(const void *x_host, void *x_dev, int dtype, uint64_t n,
                           uint32_t block_size, const uint16_t *candidates /* host */, int ncand,
                           double target, int chunks, void *workspace, uint64_t workspace_bytes,
                           apax_profile_point *points, apax_profile_summary *summary,
                           void *stream, void *copy_stream);

/* Derived metrics of one profile point (host call): r, centred Pearson r,
 * time-domain SNR in dB = 10 log10(sum x^2 / sum d^2), RMS residual in
 * percent and in dB (Table 3's two RMS columns), and means and population
 * standard deviations of x, y and d.  out receives 11 doubles in that
 * order. */
void apax_derived_metrics(const apax_profile_point *pt, uint64_t n, double *out /* host */);

/* ---------------------------------------------------------------- shards
 * One array split over several devices (Sec. 6: every block is coded on its
 * own; only the best-stream decision looks at the block before).  A shard is
 * a contiguous range of blocks [block_begin, block_end).  Its container is
 * an ordinary container of the sub-array of those blocks' elements, so it
 * decodes on its own with apax_decode; its packets are exactly the
 * whole-array packets of those blocks because the first block's stream
 * decision reads the block before the range (the halo).  The shards of one
 * array merge into the whole-array container with apax_merge_shards (one
 * device), or stay distributed: fixed rate needs no exchange (packet j sits
 * at j*B); fixed quality needs the payload word counts of the shards before
 * it (an exclusive scan of one number per shard), which apax_shard_rebase
 * adds to a shard's offset-table slice. */

/* Elements of the sub-array of blocks [block_begin, block_end) of an array
 * of n elements (host call). */
int apax_shard_elements(uint64_t n, uint32_t block_size, uint64_t block_begin, uint64_t block_end,
                        uint64_t *elements /* host */);

/* Encode blocks [block_begin, block_end) of an array of n elements.  x
 * (device) holds the shard's elements preceded by the whole halo block
 * block_begin - 1 when block_begin > 0: x points at element
 * (block_begin - 1) * N, or at element 0 for the first shard.  out receives
 * the sub-array's container (apax_encoded_size / apax_workspace_size of
 * apax_shard_elements() elements give its capacity and workspace); res its
 * status and size.  Errors as apax_encode; a range outside the array is
 * APAX_ERR_INVALID_ARG. */
int apax_encode_shard(const void *x, int dtype, uint64_t n, const apax_params *p,
                      uint64_t block_begin, uint64_t block_end, void *out, uint64_t out_capacity,
                      void *workspace, uint64_t workspace_bytes, apax_result *res, void *stream);

/* Adds add_words to the block_count offset-table entries of a fixed-quality
 * shard container (device), in place on the stream: its packets then sit at
 * their word offsets in the whole array's payload, add_words being the
 * payload words of all earlier shards. */
int apax_shard_rebase(void *container, uint64_t block_count, uint64_t add_words, void *stream);

/* One shard's container: device pointer, its byte count (apax_result.bytes
 * of its encode) and its block range. */
typedef struct {
    const void *container;
    uint64_t bytes;
    uint64_t block_begin, block_end;
} apax_shard;

/* Merge the containers of count shards that tile the blocks of an array of
 * n elements, in block order (host array of descriptors, containers on this
 * device, not yet rebased), into out: the container apax_encode writes for
 * the whole array, byte for byte.  Asynchronous on the stream (kernels and
 * device-to-device copies); res receives the status and size. */
int apax_merge_shards(const apax_shard *shards, int count, int dtype, uint64_t n,
                      const apax_params *p, void *out, uint64_t out_capacity, apax_result *res,
                      void *stream);

/* ---------------------------------------------------------------- quality
 * The profiler's windows 3 and 4 (Sec. 4) for an array x and its decoded y
 * (e.g. at the recommended code): the 2-sigma S2R margin -- the level that
 * 95.5% of the samples' signal-to-residual ratios 20 log10(|x|/|x - y|)
 * reach -- and the spectral levels: peaks and floors of x, y and d = x - y,
 * the residual spectrum's mean level, the dynamic range DR = peak - floor of
 * x, the SRR = peak of x - residual mean, and the FFT S2R margin = floor of
 * x - residual mean.  Readings (the paper gives no estimator): d is x - y
 * rounded once to binary64; the margin's ratio is the floor(45 n / 1000)-th
 * smallest per-sample |x| / |d| (0-based; +inf where d = 0, 0 where x = 0
 * and d != 0); spectra average full segments of 4096 samples (the largest
 * power of two <= n below that), each mean-removed and multiplied by the
 * periodic Hann window, as |FFT|^2 / sum(w^2) over bins 1..L/2; peak = max,
 * floor = lower median, residual mean = mean of 10 log10 over the bins. */
typedef struct {
    double s2r_ratio;        /* the 2-sigma S2R margin as an amplitude ratio */
    uint64_t n;
    uint32_t L, segments;    /* spectral segment length and count (0: no spectrum) */
    double peak_x, floor_x, peak_y, floor_y, peak_d, floor_d; /* bin powers */
    double mean_d_db;        /* mean of 10 log10 of the residual's bins */
} apax_quality;

/* Workspace bytes of apax_quality_metrics for n elements (host call). */
int apax_quality_workspace_size(int dtype, uint64_t n, uint64_t *bytes /* host */);

/* Compute the metrics of x against y (device, n elements of dtype each,
 * finite) into q (device), asynchronously on the stream: kernels and one
 * cudaMemsetAsync of the workspace.  The margin's ratio is exact (the same
 * bits as sorting the ratios); the spectral levels are binary64 FFT sums
 * added in an order that does not depend on the device. */
int apax_quality_metrics(const void *x, const void *y, int dtype, uint64_t n, void *workspace,
                         uint64_t workspace_bytes, apax_quality *q, void *stream);

/* The metrics in dB (host call): out = [2-sigma S2R margin, peak_x, floor_x,
 * peak_y, floor_y, peak_d, floor_d, residual mean, DR, SRR, FFT S2R margin]. */
void apax_quality_db(const apax_quality *q, double *out /* host, 11 */);

/* Encode without any allocation (no counterpart in the paper: this entry
 * exists for callers that cannot allocate device memory at all -- code
 * running inside another runtime's allocator or memory-pool hook, paths that
 * must never block on the CUDA driver's allocator, or plug-ins whose host owns
 * every device buffer).  Same arguments and results as apax_encode, minus
 * the workspace: the scratch lives in one fixed device array of
 * APAX_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  Limit: the call must need no more scratch than that
 * (apax_workspace_size() <= APAX_NOALLOC_SCRATCH_BYTES: 64 bytes plus 8 per
 * tile of up to 16 blocks for fixed quality, i.e. about 134 million elements
 * at block size 256; fixed rate always fits); larger calls return
 * APAX_ERR_CAPACITY without touching the device.  The first call on each
 * device looks up the array's device address (once, with that device
 * current); with CUDA's lazy module loading that first call may also load
 * the library's device code and so allocate the fixed array itself, which
 * can block on the driver.  Make the first call at start-up, outside any
 * allocator hook and before capturing any stream into a graph.  The address
 * is kept for the life of the process: do not call this entry point after
 * cudaDeviceReset on that device.  Each call
 * clears the scratch words it uses on its stream; all calls share the one
 * array, so calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller. */
#define APAX_NOALLOC_SCRATCH_BYTES (256u << 10)
int apax_encode_noalloc(const void *x, int dtype, uint64_t n, const apax_params *p, void *out,
                        uint64_t out_capacity, apax_result *res, void *stream);

/* Test hook for the bounded device waits (no counterpart in the paper):
 * a fixed-quality apax_encode in which tile `stall_tile` (a tile is a group
 * of consecutive blocks) never publishes its offset, so that its successor's
 * wait expires after about spin_cycles clock cycles and res->status becomes
 * APAX_ERR_TIMEOUT.  The kernel still terminates; the output is invalid. */
int apax_encode_test_stall(const void *x, int dtype, uint64_t n, const apax_params *p, void *out,
                           uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                           apax_result *res, int64_t stall_tile, int64_t spin_cycles,
                           void *stream);

/* ---------------------------------------------------------------- batches
 * Many arrays in one launch (no counterpart in the paper, which codes one
 * stream at a time): thousands of arrays of uneven length, mixed element
 * types and per-array parameters are encoded by one persistent kernel whose
 * CTAs take tiles of consecutive blocks from a global ticket.  The bytes of
 * every container are exactly those apax_encode writes for the same array.
 *
 * Usage: size the workspace, build a plan (host call; validates every job
 * with apax_encode's rules and copies the plan's tables into the workspace
 * with a synchronous copy), then run it any number of times.  A run is one
 * cudaMemsetAsync of the plan's counters plus one kernel launch, so it may
 * be captured into a CUDA graph.  The jobs' buffers and the workspace must
 * stay valid while the plan is used; one plan must not run twice at the
 * same time (its counters live in the workspace). */
typedef struct {
    const void *x;              /* device: n samples of dtype */
    int32_t dtype;              /* apax_dtype */
    uint32_t reserved0;         /* 0 */
    uint64_t n;
    apax_params p;              /* block size, mode, rate or code of this array */
    const uint32_t *code_dev;   /* device or NULL: fixed-quality code read on the
                                   device at run time (e.g. &summary->recommended_code) */
    void *out;                  /* device: the array's container (4-byte aligned) */
    uint64_t out_capacity;      /* >= apax_encoded_size() of this array */
    apax_result *res;           /* device: this array's status and container bytes */
} apax_encode_job;

typedef struct apax_batch apax_batch;   /* opaque host-side plan */
typedef struct apax_server apax_server; /* opaque request server */

/* Launch geometry of a plan: CTA size (teams of 8 threads: 64 or 128, i.e.
 * 8 or 16 blocks per tile; teams of 32 -- one block per warp -- when a
 * block size needs them: 32..128) and persistent CTAs per SM (0 = the
 * occupancy maximum). */
typedef struct {
    uint32_t threads;
    uint32_t ctas_per_sm;
} apax_batch_config;

/* Workspace bytes for a batch of `count` jobs (host call). */
int apax_batch_encode_workspace_size(const apax_encode_job *jobs, int count, uint64_t *bytes);

/* Build a plan (host call, synchronous copy into `workspace`, which must be
 * 256-byte aligned).  The geometry is the tuner's last choice for a batch of
 * the same shape in this process, else a default. */
int apax_batch_encode_create(const apax_encode_job *jobs, int count, void *workspace,
                             uint64_t workspace_bytes, apax_batch **plan);

/* One container to decode in a batch.  `block_size` is the block size the
 * container was encoded with (the plan sizes its tiles from it; a container
 * whose header says otherwise is reported as APAX_ERR_CORRUPT). */
typedef struct {
    const void *in;             /* device: container (4-byte aligned) */
    uint64_t in_bytes;
    void *y;                    /* device: n elements of dtype */
    int32_t dtype;
    uint32_t block_size;
    uint64_t n;
    apax_result *res;           /* device: this container's status; bytes = n */
} apax_decode_job;

/* Workspace bytes and plan of a decode batch (host calls; the same rules
 * as the encode batch; apax_decode's checks per job). */
int apax_batch_decode_workspace_size(const apax_decode_job *jobs, int count, uint64_t *bytes);
int apax_batch_decode_create(const apax_decode_job *jobs, int count, void *workspace,
                             uint64_t workspace_bytes, apax_batch **plan);

/* One array to profile in a batch: apax_profile's arguments. */
typedef struct {
    const void *x;                  /* device: n samples of dtype */
    int32_t dtype;
    uint32_t block_size;
    uint64_t n;
    const uint16_t *candidates;     /* host (read when the plan is built), or NULL
                                       with ncand = APAX_PROFILE_DEFAULT_CANDIDATES */
    int32_t ncand;
    uint32_t format;                /* APAX_FORMAT_* bits (apax_profile_format) */
    double target;
    apax_profile_point *points;     /* device: ncand points */
    apax_profile_summary *summary;  /* device */
} apax_profile_job;

/* Workspace bytes and plan of a profile batch: every array's sweep in one
 * persistent launch (runs of 16 blocks as work items; the CTA finishing an
 * array's last run adds up its fan-in-16 tree, in the same order as
 * apax_profile, and writes its points and summary).  CTA size is fixed at
 * 128; the tuner picks CTAs per SM. */
int apax_batch_profile_workspace_size(const apax_profile_job *jobs, int count, uint64_t *bytes);
int apax_batch_profile_create(const apax_profile_job *jobs, int count, void *workspace,
                              uint64_t workspace_bytes, apax_batch **plan);

/* Enqueue one run on `stream`: every job's output and result. */
int apax_batch_run(apax_batch *plan, void *stream);

/* Read or set the geometry (setting rewrites the plan's tables after a
 * device synchronisation; APAX_ERR_INVALID_ARG for a geometry the plan
 * cannot use). */
int apax_batch_get_config(const apax_batch *plan, apax_batch_config *cfg);
int apax_batch_set_config(apax_batch *plan, const apax_batch_config *cfg);

/* Autotuner: runs the plan `reps` times under every allowed geometry (CTA
 * size = blocks per tile and look-back granularity; CTAs per SM = tiles in
 * flight per SM), keeps the fastest by CUDA-event time, and remembers it
 * for later plans of the same shape in this process.  Synchronous; it
 * performs real runs, so the jobs' outputs are written. */
int apax_batch_tune(apax_batch *plan, int reps, void *stream);

/* Tiles of the plan's current geometry (work items of one run). */
uint64_t apax_batch_tiles(const apax_batch *plan);

void apax_batch_destroy(apax_batch *plan);

/* ---------------------------------------------------------------- serving
 * A request server with continuous batching (no counterpart in the paper).
 * Requests queue on the host; every apax_server_poll retires finished steps
 * and admits queued requests, first come first served, while a step slot is
 * free and the device arena has room for their outputs and workspace; the
 * admitted requests run as one step (one batched encode launch and one
 * batched decode launch on the slot's stream).  Steps on different slots
 * overlap on the device.  The arena is caller-owned device memory and its
 * size is the admission cap; the server allocates pinned host memory for
 * its job-table staging and results.  Every output is byte-identical to the
 * single-array call on the same request.  Host calls on one server must
 * not run concurrently. */
enum { APAX_OP_ENCODE = 0, APAX_OP_DECODE = 1 };

typedef struct {
    void *arena;                /* device, 256-byte aligned */
    uint64_t arena_bytes;       /* admission cap */
    uint32_t slots;             /* steps in flight at once (1..64) */
    uint32_t max_batch;         /* requests per step (1..65536) */
} apax_server_config;

typedef struct {
    uint64_t id;                /* caller's tag, returned in the completion */
    int32_t op;                 /* APAX_OP_ENCODE / APAX_OP_DECODE */
    int32_t dtype;
    uint64_t n;                 /* elements */
    apax_params p;              /* encode: all fields; decode: block_size */
    const void *in;             /* device: samples (encode) or container (decode) */
    uint64_t in_bytes;          /* decode: container bytes */
    void *out;                  /* device output, or NULL: allocated from the arena
                                   (give it back with apax_server_release) */
    uint64_t out_capacity;
    double t_arrival;           /* seconds on the server clock, or 0: submit time */
} apax_request;

typedef struct {
    uint64_t id;
    int32_t op;
    int32_t status;             /* apax_result status of the request */
    uint64_t bytes;             /* container bytes (encode) or elements (decode) */
    void *out;                  /* where the output is */
    double t_arrival, t_submit, t_launch, t_done;  /* server clock, seconds */
} apax_completion;

typedef struct {
    uint64_t queued, inflight, busy_slots;
    uint64_t arena_used, arena_peak;
    uint64_t steps, admitted, completed, undelivered;
} apax_server_stats_t;

int apax_server_create(const apax_server_config *cfg, apax_server **srv);
/* Queue a request (host checks of the single-array call; a request that
 * could never fit the arena returns APAX_ERR_CAPACITY). */
int apax_server_submit(apax_server *srv, const apax_request *req);
/* Retire finished steps, admit queued requests, and return up to max_out
 * completions (never waits for the device). */
int apax_server_poll(apax_server *srv, apax_completion *out, int max_out, int *n_out);
/* Give a server-allocated output back to the arena. */
int apax_server_release(apax_server *srv, void *out);
int apax_server_stats(const apax_server *srv, apax_server_stats_t *stats);
/* Waits for the steps in flight, then frees the server's host resources. */
void apax_server_destroy(apax_server *srv);

/* Human-readable text of a status code. */
const char *apax_status_string(int status);

/* Library version and the device architecture it was compiled for. */
const char *apax_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* APAX_GB300_H */
