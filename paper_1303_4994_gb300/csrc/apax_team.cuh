// apax_team.cuh -- team-per-block building blocks of the codec kernels.
//
// A team of TS threads (8, or 32 for very large blocks) owns one codec
// block.  Team thread t owns a contiguous range of BFPE groups (Sec. 6: one
// exponent per group of 4 samples) and walks it one group (4 samples) at a
// time in a rolled loop (small code; the samples come from L1 on re-reads).
// Per-block work that does not parallelise well -- the greedy JEE pairing,
// the exponent bookkeeping -- runs as a short sequential state machine inside
// each thread; the team combines the threads' results with log2(TS) shuffle
// steps.
#pragma once

#include "apax_device.cuh"

namespace apax {


template <int TS>
__device__ __forceinline__ int tlane() { return (int)(lane_id() & (TS - 1)); }

template <int TS, typename T>
__device__ __forceinline__ T tshfl(T v, int src) { return __shfl_sync(kFull, v, src, TS); }
template <int TS, typename T>
__device__ __forceinline__ T tshfl_up(T v, int d) { return __shfl_up_sync(kFull, v, d, TS); }
template <int TS, typename T>
__device__ __forceinline__ T tshfl_down(T v, int d) { return __shfl_down_sync(kFull, v, d, TS); }
template <int TS, typename T>
__device__ __forceinline__ T tshfl_xor(T v, int m) { return __shfl_xor_sync(kFull, v, m, TS); }

template <int TS, typename T>
__device__ __forceinline__ T team_sum(T v)
{
#pragma unroll
    for (int m = TS / 2; m >= 1; m >>= 1) v += tshfl_xor<TS>(v, m);
    return v;
}

template <int TS, typename T>
__device__ __forceinline__ T team_incl_scan(T v)
{
    const int t = tlane<TS>();
#pragma unroll
    for (int d = 1; d < TS; d <<= 1) {
        T o = tshfl_up<TS>(v, d);
        if (t >= d) v += o;
    }
    return v;
}

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// bits() of a W-bit value held sign-extended in 32 bits (Sec. 6 BFPE width:
// least b with -2^(b-1) <= v < 2^(b-1), 0 for v = 0): 32 - clz(v ^ (v << 1)).
// The OR over a group gives the group's widest value directly.
__device__ __forceinline__ uint32_t bits_term(int32_t v) { return (uint32_t)v ^ ((uint32_t)v << 1); }

__device__ __forceinline__ int exp_from_or(uint32_t acc)
{
    int e = 32 - __clz(acc);
    return e + (e == 31);  // a width of 31 is promoted to 32
}

// ---------------------------------------------------------------- geometry
// A team's view of one block.
template <int DT>
struct TBlock {
    using raw = typename DT_<DT>::raw;
    const raw *p;  // first sample of the block
    int L, G;      // samples, groups
    int g0, g1;    // this thread's groups [g0, g1) (empty if g1 <= g0)
    int Eb;        // float block exponent
    bool bad;      // a non-finite sample
    bool active;   // the block exists
};

// Load the 4 samples of the group starting at sample s (zeros past L):
// one vector load when the group is whole and aligned.
template <int DT>
__device__ __forceinline__ void load4(const TBlock<DT> &b, int s, typename LaneT<DT>::t (&x)[4])
{
    using raw = typename DT_<DT>::raw;
    using lt = typename LaneT<DT>::t;
    const raw *q = b.p + s;
    constexpr int ES = sizeof(raw);
    if (b.active && s + 4 <= b.L && ((uintptr_t)q & (4 * ES - 1)) == 0) {
        if constexpr (ES == 1) {
            const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(q));
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = (int8_t)(w >> (8 * j));
        } else if constexpr (ES == 2) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(q));
            x[0] = (int16_t)w.x; x[1] = (int16_t)(w.x >> 16);
            x[2] = (int16_t)w.y; x[3] = (int16_t)(w.y >> 16);
        } else if constexpr (ES == 4) {
            const uint4 w = __ldg(reinterpret_cast<const uint4 *>(q));
            x[0] = (lt)w.x; x[1] = (lt)w.y; x[2] = (lt)w.z; x[3] = (lt)w.w;
        } else {
            const ulonglong2 *r = reinterpret_cast<const ulonglong2 *>(q);
            const ulonglong2 w0 = __ldg(r), w1 = __ldg(r + 1);
            x[0] = w0.x; x[1] = w0.y; x[2] = w1.x; x[3] = w1.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (b.active && s + j < b.L) {
                if constexpr (DT_<DT>::F)
                    x[j] = __ldg(reinterpret_cast<const typename DT_<DT>::bits *>(q + j));
                else
                    x[j] = (lt)__ldg(q + j);
            } else {
                x[j] = 0;
            }
        }
    }
}

template <int DT>
__device__ __forceinline__ typename LaneT<DT>::t load1(const TBlock<DT> &b, int s)
{
    using lt = typename LaneT<DT>::t;
    if (!b.active || s < 0 || s >= b.L) return 0;
    if constexpr (DT_<DT>::F)
        return __ldg(reinterpret_cast<const typename DT_<DT>::bits *>(b.p + s));
    else
        return (lt)__ldg(b.p + s);
}

// ---------------------------------------------------------------- quantiser
// Per (block, code) quantiser.  Floats with a power-of-two code (m = 0) use
// one fused multiply-add: x 2^(Q-Eb-k) is exact, adding 1.5 2^23 (k >= 1, so
// |value| < 2^22) rounds it to the nearest integer with ties to even in the
// binade [2^23, 2^24), whose bit patterns then differ from that of 1.5 2^23
// by exactly the integer.  For k = 0 the addend carries the value's sign
// (|value| < 2^23).  Everything else uses exact integer significand
// arithmetic (Sec. 6 attenuator, one rounding of the exact product).
template <int DT>
struct Quant {
    Code c;
    int Eb;
    int mode;     // 0 integer, 1 fused (k >= 1), 2 fused signed (k == 0)
    float scale;  // 2^(Q - Eb - k)
    __device__ __forceinline__ Quant(int code, int eb) : c(code), Eb(eb), mode(0), scale(0.f)
    {
        if constexpr (DT == 4) {
            const int se = 23 - eb - c.k;
            if (!c.zero && c.m == 0 && se >= -126 && se <= 127) {
                mode = c.k >= 1 ? 1 : 2;
                scale = __int_as_float((se + 127) << 23);
            }
        }
    }
    __device__ __forceinline__ int32_t operator()(typename LaneT<DT>::t v) const
    {
        if constexpr (DT == 4) {
            if (mode == 1) {
                const float t = __fmaf_rn(__uint_as_float(v), scale, 12582912.0f);
                return __float_as_int(t) - 0x4B400000;
            }
            if (mode == 2) {
                const uint32_t sg = v & 0x80000000u;
                const float t = __fmaf_rn(__uint_as_float(v), scale, __uint_as_float(sg | 0x4B000000u));
                const int32_t a = (__float_as_int(t) & 0x7fffffff) - 0x4B000000;
                return sg ? -a : a;
            }
        }
        return quantise<DT>(v, c, Eb);
    }
};

// ---------------------------------------------------------------- token counter
// Greedy JEE (Sec. 6) over one thread's groups.  The first group of the
// thread waits for its predecessor's exponent (exchanged afterwards); the
// machine runs from the second group assuming it enters in state "free"
// (the previous group does not start a token that could absorb it), and
// records the length of its leading run of small diffs, which is all that
// changes when it enters "pending" instead.
struct TokCount {
    int nib;       // nibbles from the second group on (entering "free")
    int lead;      // leading small diffs from the second group on
    bool leading;  // still in the leading run
    bool st;       // pending state after the last group
    int e_first, e_last;
    int sume;
    bool any;      // at least one group
    __device__ __forceinline__ void init()
    {
        nib = 0; lead = 0; leading = true; st = false; e_first = 0; e_last = 0; sume = 0;
        any = false;
    }
    __device__ __forceinline__ void push(int e, bool valid)
    {
        if (!valid) return;
        sume += e;
        if (!any) {
            any = true;
            e_first = e;
            e_last = e;
            return;
        }
        const int d = e - e_last;
        const bool sm = (unsigned)(d + 1) <= 2u;
        nib += sm ? (st ? 0 : 1) : ((unsigned)(d + 2) <= 4u ? 1 : 2);
        st = sm && !st;
        if (leading) {
            if (sm) ++lead;
            else leading = false;
        }
        e_last = e;
    }
};

// Team combination of the threads' counters: total nibbles and exponent sum
// of the block, and (optionally) each thread's entering state and nibble
// count.  block_first: this thread owns group 0 of the block.
template <int TS>
__device__ __forceinline__ void team_tokens(const TokCount &c, bool block_first, int &nib_total,
                                            int &sume_total, bool *s_in_out = nullptr,
                                            int *nib_mine = nullptr)
{
    const int t = tlane<TS>();
    int e_prev = tshfl_up<TS>(c.e_last, 1);
    // contribution of the first group and the state entering the second,
    // for an entering state F (a) or T (b)
    int n0a = 0, n0b = 0;
    bool s1a = false, s1b = false;
    if (c.any) {
        if (block_first || t == 0) {
            n0a = n0b = 2;  // absolute first exponent
        } else {
            const int d = c.e_first - e_prev;
            const bool sm = (unsigned)(d + 1) <= 2u;
            if (sm) {
                n0a = 1; s1a = true;   // starts a token
                n0b = 0; s1b = false;  // absorbed by the predecessor's joint token
            } else {
                n0a = n0b = (unsigned)(d + 2) <= 4u ? 1 : 2;
            }
        }
    }
    // rest of the thread entering state s1: nib_T = nib_F - (lead odd)
    const bool all_small = c.leading;  // every diff after the first group is small
    auto rest_nib = [&](bool s1) { return s1 ? c.nib - (c.lead & 1) : c.nib; };
    auto rest_out = [&](bool s1) { return (s1 && all_small) ? !c.st : c.st; };
    const int na = c.any ? n0a + rest_nib(s1a) : 0, nb = c.any ? n0b + rest_nib(s1b) : 0;
    const bool oa = c.any ? rest_out(s1a) : false, ob = c.any ? rest_out(s1b) : true;
    // out-state function as 2 bits: bit0 = f(F), bit1 = f(T); identity for no groups
    uint32_t f = (uint32_t)oa | ((uint32_t)ob << 1);
    uint32_t inc = f;
#pragma unroll
    for (int d = 1; d < TS; d <<= 1) {
        uint32_t o = tshfl_up<TS>(inc, d);
        if (t >= d) {
            // inc after o: (inc o o)(s) = inc(o(s))
            const uint32_t i0 = (inc >> (o & 1)) & 1, i1 = (inc >> ((o >> 1) & 1)) & 1;
            inc = i0 | (i1 << 1);
        }
    }
    uint32_t exc = tshfl_up<TS>(inc, 1);
    const bool s_in = t == 0 ? false : (bool)(exc & 1);
    const int mine = s_in ? nb : na;
    nib_total = team_sum<TS>(mine);
    sume_total = team_sum<TS>(c.sume);
    if (s_in_out) *s_in_out = s_in;
    if (nib_mine) *nib_mine = mine;
}

// ---------------------------------------------------------------- block walk
// Open block j for a team: geometry of this thread's groups, float exponent.
template <int DT, int TS>
__device__ __forceinline__ void open_team_block(TBlock<DT> &b, const typename DT_<DT>::raw *x,
                                                uint64_t n, uint32_t N, uint64_t nb, uint64_t j,
                                                int gp)
{
    using T = DT_<DT>;
    b.active = j < nb;
    const uint64_t off = j * (uint64_t)N;
    b.p = x + (b.active ? off : 0);
    b.L = b.active ? (int)((n - off) < N ? (n - off) : N) : 0;
    b.G = (b.L + 3) >> 2;
    const int t = tlane<TS>();
    b.g0 = t * gp;
    b.g1 = min(b.g0 + gp, b.G);
    b.Eb = 0;
    b.bad = false;
    if constexpr (T::F) {
        using B = typename T::bits;
        constexpr B absm = ~((B)1 << (sizeof(B) * 8 - 1));
        constexpr B expm = (B)T::EMAX << T::MB;
        uint64_t mx = 0;
        bool bad = false;
#pragma unroll 1
        for (int g = b.g0; g < b.g1; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT>(b, 4 * g, xv);  // zeros past L do not change the maximum
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const B a = xv[i] & absm;
                bad |= (a & expm) == expm;
                mx = umax64(mx, (uint64_t)a);
            }
        }
#pragma unroll
        for (int m = TS / 2; m >= 1; m >>= 1) mx = umax64(mx, tshfl_xor<TS>(mx, m));
        b.bad = team_sum<TS>((int)bad) > 0;
        b.Eb = b.bad ? 0 : block_exp_from_maxbits<DT>(mx);
    }
}

// Derivative carry at a thread's first sample s0: the previous sample's q
// and first difference (Sec. 5/6 streams live within a block).
template <int DT>
__device__ __forceinline__ void seg_carry(const TBlock<DT> &b, const Quant<DT> &Q, int s0,
                                          int32_t &qp, int32_t &s1p)
{
    if (s0 == 0) {
        qp = 0;
        s1p = 0;
        return;
    }
    const int32_t a = Q(load1<DT>(b, s0 - 1));
    const int32_t c = s0 >= 2 ? Q(load1<DT>(b, s0 - 2)) : 0;
    qp = a;
    s1p = s0 - 1 == 0 ? 0 : (int32_t)((uint32_t)a - (uint32_t)c);
}

// Quantise group g (samples xv) and derive its three streams (S0 the data,
// S1 first differences, S2 second differences with u_1 = q_1 - q_0; mod
// 2^W, sign-extended).  Samples past L repeat q[L-1] (last-group padding).
// qp / s1p carry the previous sample's q and first difference.
template <int DT>
__device__ __forceinline__ void group_streams(const TBlock<DT> &b, const Quant<DT> &Q, int g,
                                              const typename LaneT<DT>::t (&xv)[4], int32_t &qp,
                                              int32_t &s1p, int32_t (&q)[4], int32_t (&v0)[4],
                                              int32_t (&v1)[4], int32_t (&v2)[4])
{
    constexpr int W = DT_<DT>::W;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int idx = 4 * g + i;
        const int32_t qi = idx < b.L ? Q(xv[i]) : qp;
        const int32_t d1 = (int32_t)((uint32_t)qi - (uint32_t)qp);
        int32_t d2 = (int32_t)((uint32_t)d1 - (uint32_t)s1p);
        if (idx == 1) d2 = d1;
        q[i] = qi;
        v0[i] = sext_w((uint32_t)qi, W);
        v1[i] = sext_w((uint32_t)d1, W);
        v2[i] = sext_w((uint32_t)d2, W);
        s1p = idx == 0 ? 0 : d1;
        qp = qi;
    }
}

__device__ __forceinline__ uint32_t or4(const int32_t (&v)[4])
{
    return bits_term(v[0]) | bits_term(v[1]) | bits_term(v[2]) | bits_term(v[3]);
}

// Packet bits (unpadded) of the team's block at `code` for the streams in
// smask.  Sec. 6 packet: header, JEE tokens, 4 e_g mantissa bits per group.
template <int DT, int TS>
__device__ __forceinline__ void team_eval(const TBlock<DT> &b, int code, unsigned smask,
                                          uint32_t (&bits)[3])
{
    const Quant<DT> Q(code, b.Eb);
    TokCount tc[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) tc[s].init();
    int32_t qp, s1p;
    seg_carry<DT>(b, Q, 4 * b.g0, qp, s1p);
#pragma unroll 1
    for (int g = b.g0; g < b.g1; ++g) {
        typename LaneT<DT>::t xv[4];
        load4<DT>(b, 4 * g, xv);
        int32_t q[4], v0[4], v1[4], v2[4];
        group_streams<DT>(b, Q, g, xv, qp, s1p, q, v0, v1, v2);
        tc[0].push(exp_from_or(or4(v0)), true);
        tc[1].push(exp_from_or(or4(v1)), true);
        tc[2].push(exp_from_or(or4(v2)), true);
    }
    const bool first = b.g0 == 0;
    // Every stream's team exchange runs on every lane (the teams of a warp may
    // ask for different streams; shuffles need the whole warp).
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        int nib, sume;
        team_tokens<TS>(tc[s], first, nib, sume);
        bits[s] = ((smask >> s) & 1) ? (uint32_t)DT_<DT>::H + 4u * (uint32_t)nib + 4u * (uint32_t)sume : 0u;
    }
}

// Largest packet of a block of N samples (all widths W, all tokens absolute).
__host__ __device__ inline uint32_t max_packet_words(int H, int W, uint32_t N)
{
    const uint32_t G = (N + 3) / 4;
    const uint64_t bits = (uint64_t)H + 8ull * G + (uint64_t)W * 4ull * G;
    return (uint32_t)((bits + 31) / 32);
}

}  // namespace apax
