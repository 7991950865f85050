// apax_encode.cuh -- device helpers of the block encoder shared by its
// kernels (container header, look-back, PREDICT search, token and field
// writers; internal).
#pragma once

#include "apax_team.cuh"
#include "apax_kernels.h"

namespace apax {
constexpr uint64_t kFlagA = 1ull << 62, kFlagP = 2ull << 62, kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void set_status(int *st, int code) { atomicMin(st, code); }

__device__ __forceinline__ void put_le(uint8_t *p, uint64_t v, int nb)
{
    for (int i = 0; i < nb; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

// Container header (40 bytes, little endian): "APX1", version (1, or 2 with
// a format option), dtype, mode, flags (bit 0: offset table; bit 1: BFPE
// groups of 8; bit 2: the sum stream), N, fixed-quality code, reserved,
// fixed-rate budget B, n, payload bytes (written last), 4 reserved bytes.
static __device__ void write_container_header(const EncArgs &a, int code)
{
    uint8_t *h = a.out;
    h[0] = 'A'; h[1] = 'P'; h[2] = 'X'; h[3] = '1';
    h[4] = (a.gsh || a.sum) ? 2 : 1;
    h[5] = (uint8_t)a.dtype;
    h[6] = (uint8_t)a.mode;
    h[7] = (uint8_t)((a.mode == 1 ? 1 : 0) | (a.gsh ? 2 : 0) | (a.sum ? 4 : 0));
    put_le(h + 8, a.N, 4);
    put_le(h + 12, a.mode == 1 ? (uint64_t)code : 0, 2);
    put_le(h + 14, 0, 2);
    put_le(h + 16, a.mode == 0 ? a.B : 0, 4);
    put_le(h + 20, a.n_hdr, 8);
    put_le(h + 36, 0, 4);
}

// Bounded wait on a predecessor tile's status word.
__device__ __forceinline__ uint64_t wait_tile(unsigned long long *tiles, uint64_t t,
                                              long long limit, int *status)
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
            set_status(status, -10);
            return kFlagP;  // treat as a zero prefix so successors finish
        }
    }
}

__device__ __forceinline__ uint32_t pad32_bytes(uint32_t bits) { return 4u * ((bits + 31u) >> 5); }

// ---------------------------------------------------------------- PREDICT search
// The ladder of the PREDICT fixed-rate search: codes 128 k + M[f] with
// M[f] = RNE(256 (1 - 2^(-f/16))), so that a(128 k + M[f]) is 2^-(k + f/16)
// on the attenuator's grid; 4095 follows the last rung.
__device__ __forceinline__ int ladder_m(int f)
{
    // M[0..15] = 0 11 21 31 41 50 59 67 | 75 83 90 97 104 110 116 122, a byte each
    const uint64_t lo = 0x433B32291F150B00ull, hi = 0x7A746E68615A534Bull;
    return (int)(((f < 8 ? lo >> (8 * f) : hi >> (8 * (f - 8)))) & 0xffu);
}

__device__ __forceinline__ int ladder_next(int c)
{
    const int k = c >> 7, m = c & 127;
#pragma unroll 1
    for (int f = 0; f < 16; ++f)
        if (ladder_m(f) > m) return 128 * k + ladder_m(f);
    return k < 31 ? 128 * (k + 1) : 4095;
}

// Start code of the PREDICT search: D = packet bits at code 0 minus the
// budget's bits; red(k) = 4 sum_g min(e_g, k) are the bits an attenuation of
// 2^-k is predicted to remove; k1 = the least k in 1..31 with red(k) >= D
// (31 if none); f = ceil(16 (D - red(k1-1)) / (red(k1) - red(k1-1)))
// clamped to 1..16 (16 for a zero denominator); start = 128 (k1-1) + M[f]
// for f < 16, else 128 k1.  rprev = red(k1-1), rk = red(k1).
__device__ __forceinline__ int predict_from_red(int D, int k1, int rprev, int rk)
{
    const int num = 16 * (D - rprev), den = rk - rprev;
    int f = 16;
    if (den != 0) {
        f = num / den;  // truncation toward zero, then the ceiling
        if (f * den < num) ++f;
    }
    f = f < 1 ? 1 : (f > 16 ? 16 : f);
    return f < 16 ? 128 * (k1 - 1) + ladder_m(f) : 128 * k1;
}

// The start for one thread: red(k) = red(k-1) + 4 cnt_ge(k), where
// cnt_ge(k) = #{g : e_g >= k}.
template <class CntGe>
__device__ __forceinline__ int predict_start(int D, CntGe &&cnt_ge)
{
    int rprev = 0, rk = 0, k1 = 31;
#pragma unroll 1
    for (int k = 1; k <= 31; ++k) {
        rk = rprev + 4 * cnt_ge(k);
        if (rk >= D) {
            k1 = k;
            break;
        }
        if (k < 31) rprev = rk;
    }
    return predict_from_red(D, k1, rprev, rk);
}

// The smallest packet of L samples in BFPE groups of 4 << gsh: header, the
// first exponent absolute, one joint token per two further groups.
template <int DT>
__device__ __forceinline__ uint32_t min_packet(int L, int gsh)
{
    const int G = gsh ? (L + 7) >> 3 : (L + 3) >> 2;
    return pad32_bytes((uint32_t)DT_<DT>::H + 8u + 4u * (uint32_t)((G - 1 + 1) >> 1));
}

template <int DT>
__device__ __forceinline__ uint32_t fr_budget(int L, uint32_t num, uint32_t den, int gsh)
{
    const uint64_t b = ((uint64_t)L * DT_<DT>::S * den / (4ull * num)) * 4ull;
    const uint32_t mp = min_packet<DT>(L, gsh);
    return b > mp ? (uint32_t)b : mp;
}

__device__ __forceinline__ uint32_t abs_token(int e)
{
    const int v = e >= 31 ? 31 : e;
    return (uint32_t)(14 + (v >> 4)) | ((uint32_t)(v & 15) << 4);
}

// Append `cnt` nibbles (value tok) to the thread's token bit stream at
// nibble position *pos, flushing complete words into pkt.
struct NibWriter {
    uint64_t acc;
    int fill;       // bits in acc
    uint32_t word;  // packet word index acc starts at
    uint32_t *pkt;
    __device__ __forceinline__ void start(uint32_t *p, uint32_t bit)
    {
        pkt = p;
        word = bit >> 5;
        fill = (int)(bit & 31);
        acc = 0;
    }
    __device__ __forceinline__ void put(uint32_t v, int nbits)
    {
        acc |= (uint64_t)v << fill;
        fill += nbits;
        if (fill >= 32) {
            atomicOr(&pkt[word], (uint32_t)acc);
            acc >>= 32;
            fill -= 32;
            ++word;
        }
    }
    __device__ __forceinline__ void flush()
    {
        if (fill > 0 && acc) atomicOr(&pkt[word], (uint32_t)acc);
    }
};

// Decoupled look-back, in two steps so that a tile's aggregate is visible
// early: publish_aggregate (one lane) as soon as the tile's size is known,
// lookback_prefix (warp 0, every lane) after the tile's other work.
__device__ __forceinline__ void publish_aggregate(const EncArgs &a, uint64_t tile, uint32_t total)
{
    if (a.test_stall_tile == (long long)tile) return;  // test hook: never publishes
    atomicExch(a.tiles + tile, (tile == 0 ? kFlagP : kFlagA) | total);
}

// Reads 32 predecessors per probe (lane l reads tile base - l); the nearest
// inclusive prefix ends the walk.  Returns the exclusive prefix and
// publishes this tile's inclusive prefix.
__device__ __forceinline__ uint64_t lookback_prefix(const EncArgs &a, uint64_t tile, uint32_t total)
{
    const int l = threadIdx.x & 31;
    if (tile == 0) return 0;
    const bool hook = a.test_stall_tile == (long long)tile;
    uint64_t excl = 0;
    int64_t base = (int64_t)tile - 1;
    while (true) {
        const int64_t tt = base - l;
        const uint64_t st = tt >= 0 ? wait_tile(a.tiles, (uint64_t)tt, a.spin_limit, a.status) : kFlagP;
        const unsigned pm = __ballot_sync(kFull, (st & ~kValMask) == kFlagP);
        const int near = pm ? __ffs(pm) - 1 : 31;
        uint64_t val = l <= near ? (st & kValMask) : 0;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) val += __shfl_xor_sync(kFull, val, m);
        excl += val;
        if (pm) break;
        base -= 32;
    }
    if (l == 0 && !hook) atomicExch(a.tiles + tile, kFlagP | ((excl + total) & kValMask));
    return excl;
}

// Writes the Sec. 6 JEE tokens of groups [g0, g1) of a block of G groups
// whose exponents are eb[g * est]; s_in: the group before g0 opened a joint
// token that g0 completes.
template <class Wr>
__device__ __forceinline__ void write_tokens(Wr &nw, const uint8_t *eb, int est, int g0, int g1, int G,
                                             bool s_in)
{
    bool st = s_in;
    int eprev = g0 > 0 && g0 < G ? eb[(size_t)(g0 - 1) * est] : 0;
#pragma unroll 1
    for (int g = g0; g < g1; ++g) {
        const int e = eb[(size_t)g * est];
        if (g == 0) {
            nw.put(abs_token(e), 8);
            st = false;
        } else {
            const int d = e - eprev;
            if ((unsigned)(d + 1) <= 2u) {
                if (st) {
                    st = false;  // second diff of the previous joint token
                } else {
                    const int dn = g + 1 < G ? (int)eb[(size_t)(g + 1) * est] - e : 99;
                    if ((unsigned)(dn + 1) <= 2u) nw.put((uint32_t)(3 * (d + 1) + (dn + 1)), 4);
                    else nw.put((uint32_t)(11 + d), 4);
                    st = true;
                }
            } else {
                if ((unsigned)(d + 2) <= 4u) nw.put((uint32_t)(11 + d), 4);
                else nw.put(abs_token(e), 8);
                st = false;
            }
        }
        eprev = e;
    }
}

// Appends one group's four e-bit fields in as few wide pieces as fit.
template <class Wr>
__device__ __forceinline__ void write_group_fields(Wr &mw, int e, const int32_t (&u)[4])
{
    if (!e) return;
    const uint32_t m = e >= 32 ? 0xffffffffu : ((1u << e) - 1u);
    const uint32_t f0 = (uint32_t)u[0] & m, f1 = (uint32_t)u[1] & m, f2 = (uint32_t)u[2] & m,
                   f3 = (uint32_t)u[3] & m;
    if (e <= 8) {
        mw.put(f0 | (f1 << e) | (f2 << (2 * e)) | (f3 << (3 * e)), 4 * e);
    } else if (e <= 16) {
        mw.put(f0 | (f1 << e), 2 * e);
        mw.put(f2 | (f3 << e), 2 * e);
    } else {
        mw.put(f0, e);
        mw.put(f1, e);
        mw.put(f2, e);
        mw.put(f3, e);
    }
}

// A packet written by its only owner straight to global memory: complete
// words are stored as they fill.
struct GWriter {
    uint32_t *dst;
    uint64_t acc;
    int fill;
    uint32_t w;
    __device__ __forceinline__ void start(uint32_t *d)
    {
        dst = d;
        acc = 0;
        fill = 0;
        w = 0;
    }
    __device__ __forceinline__ void put(uint32_t v, int nbits)
    {
        acc |= (uint64_t)v << fill;
        fill += nbits;
        if (fill >= 32) {
            dst[w++] = (uint32_t)acc;
            acc >>= 32;
            fill -= 32;
        }
    }
    __device__ __forceinline__ void flush()
    {
        if (fill > 0) dst[w++] = (uint32_t)acc;
        acc = 0;
        fill = 0;
    }
};

}  // namespace apax
