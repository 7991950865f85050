// apax_encode.cu -- block encoder kernels (Sec. 6 encoder and bit packer).
//
// One warp encodes one block; a CTA of WPC warps is one tile of WPC
// consecutive blocks.  Each warp
//   1. decides its stream from the predecessor block at code 0 (the
//      one-block lag of Sec. 6: block j+1 carries block j's best stream),
//   2. picks the attenuation code (fixed quality: given; fixed rate: the
//      BISECT search against the block budget),
//   3. computes exponents, JEE tokens and mantissas into a shared-memory
//      packet.
// Fixed-rate packets land at j*B.  Fixed-quality packet offsets come from a
// device-wide exclusive scan over tiles with decoupled look-back (Merrill &
// Garland 2016): tiles take tickets in launch order, publish their word
// count, and walk back over predecessors with a bounded spin.
#include "apax_block.cuh"
#include "apax_kernels.h"

namespace apax {

constexpr uint64_t kFlagA = 1ull << 62, kFlagP = 2ull << 62, kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void set_status(int *st, int code) { atomicMin(st, code); }

__device__ __forceinline__ void put_le(uint8_t *p, uint64_t v, int nb)
{
    for (int i = 0; i < nb; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

// Container header (40 bytes, little endian): "APX1", version 1, dtype,
// mode, flags (bit 0: offset table), N, fixed-quality code, reserved,
// fixed-rate budget B, n, payload bytes (written last), 4 reserved bytes.
__device__ void write_container_header(const EncArgs &a, int code)
{
    uint8_t *h = a.out;
    h[0] = 'A'; h[1] = 'P'; h[2] = 'X'; h[3] = '1';
    h[4] = 1;
    h[5] = (uint8_t)a.dtype;
    h[6] = (uint8_t)a.mode;
    h[7] = a.mode == 1 ? 1 : 0;
    put_le(h + 8, a.N, 4);
    put_le(h + 12, a.mode == 1 ? (uint64_t)code : 0, 2);
    put_le(h + 14, 0, 2);
    put_le(h + 16, a.mode == 0 ? a.B : 0, 4);
    put_le(h + 20, a.n, 8);
    put_le(h + 36, 0, 4);
}

// Bounded wait on a predecessor tile's status word.
__device__ __forceinline__ uint64_t wait_tile(unsigned long long *tiles, uint64_t t,
                                              long long limit, int *status, bool &timed_out)
{
    volatile unsigned long long *p = tiles + t;
    uint64_t v = *p;
    if (v) return v;
    const long long t0 = clock64();
    while (true) {
        __nanosleep(64);
        v = *p;
        if (v) return v;
        if (clock64() - t0 > limit) {
            timed_out = true;
            set_status(status, -10);
            return kFlagP;  // treat as a zero prefix so successors finish
        }
    }
}

template <int DT, int MODE>
__global__ void __launch_bounds__(256) k_encode(EncArgs a)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint64_t s_tile;
    __shared__ uint32_t s_words[8];
    __shared__ uint64_t s_base;
    const int wid = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    using raw = typename DT_<DT>::raw;
    constexpr int H = DT_<DT>::H;

    if (threadIdx.x == 0) s_tile = MODE == 1 ? (uint64_t)atomicAdd(a.ticket, 1u) : blockIdx.x;
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t j = tile * (uint64_t)wpc + (uint64_t)wid;
    const bool active = j < a.nb;
    int code = (int)a.code;
    if (a.code_dev) code = (int)*a.code_dev;

    uint32_t *pkt = smem + (size_t)wid * (a.pkt_words + a.ebuf_words);
    uint8_t *ebuf = reinterpret_cast<uint8_t *>(pkt + a.pkt_words);

    if (tile == 0 && threadIdx.x == 0) write_container_header(a, code);

    uint32_t words = 0;  // packet words of this warp's block
    if (active) {
        const raw *x = reinterpret_cast<const raw *>(a.x);
        BlockView<DT> prev, cur;
        // stream decision: best(j-1) (block 0 uses its own best)
        open_block<DT>(prev, x, a.n, a.N, j == 0 ? 0 : j - 1);
        open_block<DT>(cur, x, a.n, a.N, j);
        if (cur.bad && lane == 0) set_status(a.status, -8);
        const int s = best_stream<DT>(prev);
        uint32_t plen;
        if (MODE == 0) {
            const uint32_t budget = cur.L == (int)a.N ? a.B : fr_budget<DT>(cur.L, a.rate_num, a.rate_den);
            code = fr_search<DT>(cur, s, budget);
            plen = budget;
        }
        int32_t u[8];
        int sume, nib;
        final_pass<DT>(cur, code, s, ebuf, u, sume, nib);
        const uint32_t bits = (uint32_t)H + 4u * (uint32_t)nib + 4u * (uint32_t)sume;
        if (MODE == 1) plen = pad32_bytes(bits);
        words = plen >> 2;
        for (uint32_t t = lane; t < words; t += 32) pkt[t] = 0;
        __syncwarp();
        if (lane == 0) {
            uint32_t h0 = (uint32_t)s | ((uint32_t)code << 2) | (plen << 14);
            atomicOr(&pkt[0], h0);
            if (H == 48) atomicOr(&pkt[1], (uint32_t)(uint16_t)(int16_t)cur.Eb);
        }
        write_tokens(ebuf, cur.G, H, pkt);
        write_mantissas<DT>(cur, code, s, ebuf, (uint32_t)H + 4u * (uint32_t)nib, u, pkt);
        __syncwarp();
    }

    uint64_t off_words;  // packet start in payload words
    if (MODE == 1) {
        if (lane == 0) s_words[wid] = words;
        __syncthreads();
        if (wid == 0) {
            uint32_t v = lane < wpc ? s_words[lane] : 0;
            uint32_t incl = warp_incl_scan(v);
            uint32_t total = __shfl_sync(kFull, incl, 31);
            if (lane < wpc) s_words[lane] = incl - v;
            if (lane == 0) {
                bool to = false;
                uint64_t excl = 0;
                const bool hook = a.test_stall_tile == (long long)tile;
                if (tile == 0) {
                    if (!hook) atomicExch(a.tiles, kFlagP | total);
                } else {
                    if (!hook) atomicExch(a.tiles + tile, kFlagA | total);
                    int64_t t = (int64_t)tile - 1;
                    while (t >= 0) {
                        uint64_t st = wait_tile(a.tiles, (uint64_t)t, a.spin_limit, a.status, to);
                        excl += st & kValMask;
                        if ((st & ~kValMask) == kFlagP) break;
                        --t;
                    }
                    if (!hook) atomicExch(a.tiles + tile, kFlagP | ((excl + total) & kValMask));
                }
                s_base = excl;
            }
        }
        __syncthreads();
        off_words = s_base + s_words[wid];
    } else {
        off_words = j * (uint64_t)(a.B >> 2);
    }

    if (active) {
        const uint64_t start = a.poff + 4ull * off_words;
        if (MODE == 1) {
            if (off_words > 0xffffffffull) {
                if (lane == 0) set_status(a.status, -6);
            } else if (lane == 0) {
                reinterpret_cast<uint32_t *>(a.out + 40)[j] = (uint32_t)off_words;
                if (j == a.nb - 1 && (a.nb & 1)) reinterpret_cast<uint32_t *>(a.out + 40)[j + 1] = 0;
            }
        }
        if (start + 4ull * words > a.cap) {
            if (lane == 0) set_status(a.status, -5);
        } else {
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.out + start);
            for (uint32_t t = lane; t < words; t += 32) dst[t] = pkt[t];
        }
    }

    // completion: the last CTA to finish writes the payload size and result
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(a.done, 1u);
        if (prev == a.ntiles - 1) {
            __threadfence();
            uint64_t payload;
            if (MODE == 1) {
                volatile unsigned long long *last = a.tiles + (a.ntiles - 1);
                payload = 4ull * ((uint64_t)(*last) & kValMask);
            } else {
                payload = a.fr_payload;
            }
            put_le(a.out + 28, payload, 8);
            volatile int *st = a.status;
            if (a.res) {
                a.res->bytes = a.poff + payload;
                a.res->status = *st;
            }
        }
    }
}

template <int DT>
static cudaError_t launch_dt(const EncArgs &a, int wpc, size_t smem, cudaStream_t s)
{
    if (a.mode == 1) {
        auto k = k_encode<DT, 1>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)a.ntiles, 32 * wpc, smem, s>>>(a);
    } else {
        auto k = k_encode<DT, 0>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)a.ntiles, 32 * wpc, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_encode(const EncArgs &a, int wpc, size_t smem, cudaStream_t s)
{
    switch (a.dtype) {
    case 1: return launch_dt<1>(a, wpc, smem, s);
    case 2: return launch_dt<2>(a, wpc, smem, s);
    case 3: return launch_dt<3>(a, wpc, smem, s);
    case 4: return launch_dt<4>(a, wpc, smem, s);
    default: return launch_dt<5>(a, wpc, smem, s);
    }
}

}  // namespace apax
