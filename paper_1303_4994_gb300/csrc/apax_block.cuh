// apax_block.cuh -- per-block warp routines shared by the encode and profile
// kernels: loading a block, its float exponent, packet-size evaluation of the
// three derivative streams, and the exponent/token/mantissa writers.
#pragma once

#include "apax_device.cuh"

namespace apax {

template <int DT>
struct BlockView {
    using raw = typename DT_<DT>::raw;
    using lt = typename LaneT<DT>::t;
    const raw *p;  // first sample of the block
    int L, G, nch; // samples, groups, chunks of 256
    int Eb;        // float block exponent
    bool bad;      // non-finite sample seen
    lt x0[8];      // chunk 0 (cached when nch == 1)
};

// Load lane samples [base + 8 lane, +8) of a block of L samples (zero past L).
template <int DT>
__device__ __forceinline__ void load_lane(const typename DT_<DT>::raw *p, int L, int chunk,
                                          typename LaneT<DT>::t (&x)[8])
{
    using raw = typename DT_<DT>::raw;
    using lt = typename LaneT<DT>::t;
    const int i0 = chunk * kChunk + 8 * (int)lane_id();
    const raw *q = p + i0;
    constexpr int BYTES = 8 * sizeof(raw);
    if (i0 + 8 <= L && (((uintptr_t)q) % (BYTES >= 16 ? 16 : BYTES)) == 0) {
        if constexpr (BYTES == 8) {
            uint2 v = __ldg(reinterpret_cast<const uint2 *>(q));
            uint32_t w[2] = {v.x, v.y};
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = (int8_t)(w[t >> 2] >> (8 * (t & 3)));
        } else if constexpr (BYTES == 16) {
            uint4 v = __ldg(reinterpret_cast<const uint4 *>(q));
            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = (int16_t)(w[t >> 1] >> (16 * (t & 1)));
        } else if constexpr (BYTES == 32) {
            uint4 a = __ldg(reinterpret_cast<const uint4 *>(q));
            uint4 b = __ldg(reinterpret_cast<const uint4 *>(q) + 1);
            uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = (lt)w[t];
        } else {
            const ulonglong2 *r = reinterpret_cast<const ulonglong2 *>(q);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ulonglong2 v = __ldg(r + t);
                x[2 * t] = v.x;
                x[2 * t + 1] = v.y;
            }
        }
    } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (i0 + t < L) {
                if constexpr (DT_<DT>::F) {
                    using B = typename DT_<DT>::bits;
                    x[t] = __ldg(reinterpret_cast<const B *>(q + t));
                } else {
                    x[t] = (lt)__ldg(q + t);
                }
            } else {
                x[t] = 0;
            }
        }
    }
}

// Open a block view: samples, groups, chunk count, float exponent.
template <int DT>
__device__ __forceinline__ void open_block(BlockView<DT> &b, const typename DT_<DT>::raw *x,
                                           uint64_t n, uint32_t N, uint64_t j)
{
    uint64_t off = j * (uint64_t)N;
    uint64_t rem = n - off;
    b.p = x + off;
    b.L = (int)(rem < N ? rem : N);
    b.G = (b.L + 3) >> 2;
    b.nch = (b.L + kChunk - 1) / kChunk;
    b.Eb = 0;
    b.bad = false;
    if (b.nch == 1) load_lane<DT>(b.p, b.L, 0, b.x0);
    if constexpr (DT_<DT>::F) {
        using T = DT_<DT>;
        using B = typename T::bits;
        constexpr B absm = ~((B)1 << (sizeof(B) * 8 - 1));
        constexpr B expm = (B)T::EMAX << T::MB;
        uint64_t mx = 0;
        bool bad = false;
        for (int ch = 0; ch < b.nch; ++ch) {
            typename LaneT<DT>::t xv[8];
            if (b.nch == 1) {
#pragma unroll
                for (int t = 0; t < 8; ++t) xv[t] = b.x0[t];
            } else {
                load_lane<DT>(b.p, b.L, ch, xv);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                B a = xv[t] & absm;
                bad |= (a & expm) == expm;
                mx = (uint64_t)a > mx ? (uint64_t)a : mx;
            }
        }
        if constexpr (sizeof(B) == 4) {
            mx = __reduce_max_sync(kFull, (uint32_t)mx);
        } else {
            mx = warp_max_u64(mx);
        }
        b.bad = __any_sync(kFull, bad);
        b.Eb = b.bad ? 0 : block_exp_from_maxbits<DT>(mx);
    }
}

template <int DT>
__device__ __forceinline__ void chunk_x(const BlockView<DT> &b, int ch, typename LaneT<DT>::t (&x)[8])
{
    if (b.nch == 1) {
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = b.x0[t];
    } else {
        load_lane<DT>(b.p, b.L, ch, x);
    }
}

// Quantise the lane's samples of chunk ch; samples past L repeat q[L-1]
// (the padding of the last group).  Returns the count of valid groups in the
// chunk.  carry_q1/q2 receive the chunk's last two q values (for the next
// chunk's derivatives).
template <int DT>
__device__ __forceinline__ int chunk_quantise(const BlockView<DT> &b, int ch, const Code &c,
                                              int32_t (&q)[8])
{
    typename LaneT<DT>::t x[8];
    chunk_x<DT>(b, ch, x);
    const int i0 = ch * kChunk + 8 * (int)lane_id();
#pragma unroll
    for (int t = 0; t < 8; ++t) q[t] = quantise<DT>(x[t], c, b.Eb);
    const int last = b.L - 1;
    if (last < (ch + 1) * kChunk) {  // the last chunk: pad with q[L-1]
        int li = last - ch * kChunk;
        int32_t ql = __shfl_sync(kFull, q[li & 7], li >> 3);
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (i0 + t > last) q[t] = ql;
    }
    int gc = b.G - ch * (kChunk / 4);
    return gc > 64 ? 64 : gc;
}

// Packet bits (unpadded) of the block at code c for the streams in smask
// (bit s set -> bits[s] computed).  Sec. 6 packet: header, JEE tokens, 4 e_g
// mantissa bits per group.
template <int DT>
__device__ __forceinline__ void eval_block(const BlockView<DT> &b, int code, unsigned smask,
                                           uint32_t (&bits)[3])
{
    constexpr int W = DT_<DT>::W;
    const Code c(code);
    int32_t p1 = 0, p2 = 0;  // last two q of the previous chunk (lane 0 only)
    int eprev[3] = {0, 0, 0};
    bool carry[3] = {false, false, false};
    int nib[3] = {0, 0, 0}, sume[3] = {0, 0, 0};
    for (int ch = 0; ch < b.nch; ++ch) {
        int32_t q[8];
        int gc = chunk_quantise<DT>(b, ch, c, q);
        int32_t u1 = __shfl_up_sync(kFull, q[7], 1), u2 = __shfl_up_sync(kFull, q[6], 1);
        if (lane_id() == 0) { u1 = p1; u2 = p2; }
        const bool bstart = (ch == 0) && lane_id() == 0;
        const int g0 = 2 * (int)lane_id();
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (!((smask >> s) & 1)) continue;
            int32_t u[8];
            derive<W>(q, s, u1, u2, bstart, u);
            int e0 = g0 < gc ? group_exp(u[0], u[1], u[2], u[3]) : 0;
            int e1 = g0 + 1 < gc ? group_exp(u[4], u[5], u[6], u[7]) : 0;
            ChunkTok tk = chunk_tokens(e0, e1, gc, ch == 0, eprev[s], carry[s]);
            nib[s] += tk.nib;
            sume[s] += warp_sum(e0 + e1);
            eprev[s] = tk.last_e;
            carry[s] = tk.carry;
        }
        p1 = __shfl_sync(kFull, q[7], 31);
        p2 = __shfl_sync(kFull, q[6], 31);
    }
#pragma unroll
    for (int s = 0; s < 3; ++s)
        bits[s] = (uint32_t)DT_<DT>::H + 4u * (uint32_t)nib[s] + 4u * (uint32_t)sume[s];
}

// best(j): stream with the fewest packet bits at code 0, ties to the lower.
template <int DT>
__device__ __forceinline__ int best_stream(const BlockView<DT> &b)
{
    uint32_t bits[3];
    eval_block<DT>(b, 0, 7u, bits);
    int s = 0;
    if (bits[1] < bits[s]) s = 1;
    if (bits[2] < bits[s]) s = 2;
    return s;
}

__device__ __forceinline__ uint32_t pad32_bytes(uint32_t bits) { return 4u * ((bits + 31u) >> 5); }

// Minimum packet (all exponents zero) of a block of L samples.
template <int DT>
__device__ __forceinline__ uint32_t min_packet(int L)
{
    int G = (L + 3) >> 2;
    return pad32_bytes((uint32_t)DT_<DT>::H + 8u + 4u * (uint32_t)((G - 1 + 1) >> 1));
}

// Fixed-rate budget of a block of L samples.
template <int DT>
__device__ __forceinline__ uint32_t fr_budget(int L, uint32_t num, uint32_t den)
{
    uint64_t b = ((uint64_t)L * DT_<DT>::S * den / (4ull * num)) * 4ull;
    uint32_t mp = min_packet<DT>(L);
    return b > mp ? (uint32_t)b : mp;
}

// Fixed-rate search, policy BISECT: code 0 if it fits, else bisection on
// [0, 4095] keeping the upper end fitting (4095, the zero attenuator, always
// fits).
template <int DT>
__device__ __forceinline__ int fr_search(const BlockView<DT> &b, int s, uint32_t budget)
{
    uint32_t bits[3];
    eval_block<DT>(b, 0, 1u << s, bits);
    if (pad32_bytes(bits[s]) <= budget) return 0;
    int lo = 0, hi = 4095;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        eval_block<DT>(b, mid, 1u << s, bits);
        if (pad32_bytes(bits[s]) <= budget) hi = mid;
        else lo = mid;
    }
    return hi;
}

// ---------------------------------------------------------------- writer
// Computes the chosen stream's group exponents into ebuf (one byte per
// group) and returns (sum of exponents, JEE nibble count).  For a one-chunk
// block the stream values stay in u (registers).
template <int DT>
__device__ __forceinline__ void final_pass(const BlockView<DT> &b, int code, int s, uint8_t *ebuf,
                                           int32_t (&u)[8], int &sume, int &nib)
{
    constexpr int W = DT_<DT>::W;
    const Code c(code);
    int32_t p1 = 0, p2 = 0;
    int eprev = 0;
    bool carry = false;
    sume = 0;
    nib = 0;
    const int g0l = 2 * (int)lane_id();
    for (int ch = 0; ch < b.nch; ++ch) {
        int32_t q[8];
        int gc = chunk_quantise<DT>(b, ch, c, q);
        int32_t u1 = __shfl_up_sync(kFull, q[7], 1), u2 = __shfl_up_sync(kFull, q[6], 1);
        if (lane_id() == 0) { u1 = p1; u2 = p2; }
        derive<W>(q, s, u1, u2, (ch == 0) && lane_id() == 0, u);
        int e0 = g0l < gc ? group_exp(u[0], u[1], u[2], u[3]) : 0;
        int e1 = g0l + 1 < gc ? group_exp(u[4], u[5], u[6], u[7]) : 0;
        ChunkTok tk = chunk_tokens(e0, e1, gc, ch == 0, eprev, carry);
        nib += tk.nib;
        sume += warp_sum(e0 + e1);
        eprev = tk.last_e;
        carry = tk.carry;
        const int gb = ch * 64 + g0l;
        if (g0l < gc) ebuf[gb] = (uint8_t)e0;
        if (g0l + 1 < gc) ebuf[gb + 1] = (uint8_t)e1;
        p1 = __shfl_sync(kFull, q[7], 31);
        p2 = __shfl_sync(kFull, q[6], 31);
    }
    __syncwarp();
}

__device__ __forceinline__ uint32_t abs_token(int e)
{
    int v = e >= 31 ? 31 : e;
    return (uint32_t)(14 + (v >> 4)) | ((uint32_t)(v & 15) << 4);
}

// Writes the JEE token section (Sec. 6) from ebuf into the packet words pkt
// (zeroed), starting at bit H.  Tokens: first exponent absolute; greedy
// joint nibble 3(d1+1)+(d2+1) for two diffs in [-1,1]; single nibble 11+d for
// a diff in [-2,2]; else absolute 14+(v>>4), v&15.
__device__ __forceinline__ void write_tokens(const uint8_t *ebuf, int G, int H, uint32_t *pkt)
{
    const int l = (int)lane_id();
    bool carry = false;
    int nbase = 0;
    const int nch = (G + 63) >> 6;
    for (int ch = 0; ch < nch; ++ch) {
        const int g0 = ch * 64 + 2 * l, g1 = g0 + 1;
        const bool v0 = g0 < G, v1 = g1 < G;
        const int e0 = v0 ? ebuf[g0] : 0, e1 = v1 ? ebuf[g1] : 0;
        const int em = (g0 >= 1 && v0) ? ebuf[g0 - 1] : 0;
        const bool v2 = g1 + 1 < G;
        const int e2 = v2 ? ebuf[g1 + 1] : 0;
        const int d0 = e0 - em, d1 = e1 - e0, d2 = e2 - e1;
        const bool pos0 = g0 >= 1;
        const bool s0 = v0 && pos0 && d0 >= -1 && d0 <= 1;
        const bool s1 = v1 && d1 >= -1 && d1 <= 1;
        const bool s2 = v2 && d2 >= -1 && d2 <= 1;
        const uint64_t S = ballot64(s0, s1);
        const uint64_t E = jee_even_offsets(S, carry && ch > 0);
        const bool E0 = (E >> (2 * l)) & 1, E1 = (E >> (2 * l + 1)) & 1;
        uint32_t tok = 0;
        int cnt = 0;
        if (v0) {
            if (!pos0) {
                tok = abs_token(e0);
                cnt = 2;
            } else if (s0) {
                if (E0) {
                    tok = s1 ? (uint32_t)(3 * (d0 + 1) + (d1 + 1)) : (uint32_t)(11 + d0);
                    cnt = 1;
                }
            } else if (d0 >= -2 && d0 <= 2) {
                tok = (uint32_t)(11 + d0);
                cnt = 1;
            } else {
                tok = abs_token(e0);
                cnt = 2;
            }
        }
        if (v1) {
            uint32_t t1 = 0;
            int c1 = 0;
            if (s1) {
                if (E1) {
                    t1 = s2 ? (uint32_t)(3 * (d1 + 1) + (d2 + 1)) : (uint32_t)(11 + d1);
                    c1 = 1;
                }
            } else if (d1 >= -2 && d1 <= 2) {
                t1 = (uint32_t)(11 + d1);
                c1 = 1;
            } else {
                t1 = abs_token(e1);
                c1 = 2;
            }
            tok |= t1 << (4 * cnt);
            cnt += c1;
        }
        const int incl = warp_incl_scan(cnt);
        const int t0 = nbase + incl - cnt;
        if (cnt) {
            const uint32_t bit = (uint32_t)H + 4u * (uint32_t)t0;
            const uint32_t w = bit >> 5, sh = bit & 31;
            atomicOr(&pkt[w], tok << sh);
            if (sh + 4u * cnt > 32u) atomicOr(&pkt[w + 1], tok >> (32 - sh));
        }
        nbase += __shfl_sync(kFull, incl, 31);
        const int lastg = (G - ch * 64 < 64 ? G - ch * 64 : 64) - 1;
        carry = ((E & S) >> lastg) & 1;
    }
}

// Packs the lane's 8 stream values (two groups of widths e0, e1) at bit
// offset `bit` of the packet (LSB first).
__device__ __forceinline__ void pack_lane(uint32_t *pkt, uint32_t bit, const int32_t (&u)[8], int e0,
                                          int e1)
{
    if (e0 + e1 == 0) return;
    uint32_t w = bit >> 5;
    uint32_t fill = bit & 31;
    uint64_t acc = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int e = t < 4 ? e0 : e1;
        if (e == 0) continue;
        const uint64_t mask = e >= 32 ? 0xffffffffull : ((1ull << e) - 1);
        acc |= ((uint64_t)(uint32_t)u[t] & mask) << fill;
        fill += (uint32_t)e;
        if (fill >= 32) {
            atomicOr(&pkt[w], (uint32_t)acc);
            acc >>= 32;
            fill -= 32;
            ++w;
        }
    }
    if (fill) atomicOr(&pkt[w], (uint32_t)acc);
}

// Writes the mantissa section.  For one-chunk blocks u holds the stream
// values; longer blocks recompute each chunk.
template <int DT>
__device__ __forceinline__ void write_mantissas(const BlockView<DT> &b, int code, int s,
                                                const uint8_t *ebuf, uint32_t mbase,
                                                const int32_t (&u_cached)[8], uint32_t *pkt)
{
    constexpr int W = DT_<DT>::W;
    const int g0l = 2 * (int)lane_id();
    if (b.nch == 1) {
        const int e0 = g0l < b.G ? ebuf[g0l] : 0;
        const int e1 = g0l + 1 < b.G ? ebuf[g0l + 1] : 0;
        const int w4 = 4 * (e0 + e1);
        const int incl = warp_incl_scan(w4);
        pack_lane(pkt, mbase + (uint32_t)(incl - w4), u_cached, e0, e1);
        return;
    }
    const Code c(code);
    int32_t p1 = 0, p2 = 0;
    uint32_t base = mbase;
    for (int ch = 0; ch < b.nch; ++ch) {
        int32_t q[8], u[8];
        int gc = chunk_quantise<DT>(b, ch, c, q);
        int32_t u1 = __shfl_up_sync(kFull, q[7], 1), u2 = __shfl_up_sync(kFull, q[6], 1);
        if (lane_id() == 0) { u1 = p1; u2 = p2; }
        derive<W>(q, s, u1, u2, (ch == 0) && lane_id() == 0, u);
        const int gb = ch * 64 + g0l;
        const int e0 = g0l < gc ? ebuf[gb] : 0;
        const int e1 = g0l + 1 < gc ? ebuf[gb + 1] : 0;
        const int w4 = 4 * (e0 + e1);
        const int incl = warp_incl_scan(w4);
        pack_lane(pkt, base + (uint32_t)(incl - w4), u, e0, e1);
        base += (uint32_t)__shfl_sync(kFull, incl, 31);
        p1 = __shfl_sync(kFull, q[7], 31);
        p2 = __shfl_sync(kFull, q[6], 31);
    }
}

// Largest packet of a block of N samples (all widths W, all tokens absolute).
__host__ __device__ inline uint32_t max_packet_words(int H, int W, uint32_t N)
{
    uint32_t G = (N + 3) / 4;
    uint64_t bits = (uint64_t)H + 8ull * G + (uint64_t)W * 4ull * G;
    return (uint32_t)((bits + 31) / 32);
}

}  // namespace apax
