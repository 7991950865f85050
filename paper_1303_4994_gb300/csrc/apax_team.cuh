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

// Team shuffles (width TS, every lane of the warp takes part).  A team of
// one thread exchanges nothing: its shuffles are the identity, so code that
// runs per thread (and may diverge) calls no warp collective.
template <int TS, typename T>
__device__ __forceinline__ T tshfl(T v, int src)
{
    if constexpr (TS == 1) return v;
    else return __shfl_sync(kFull, v, src, TS);
}
template <int TS, typename T>
__device__ __forceinline__ T tshfl_up(T v, int d)
{
    if constexpr (TS == 1) return v;
    else return __shfl_up_sync(kFull, v, d, TS);
}
template <int TS, typename T>
__device__ __forceinline__ T tshfl_down(T v, int d)
{
    if constexpr (TS == 1) return v;
    else return __shfl_down_sync(kFull, v, d, TS);
}
template <int TS, typename T>
__device__ __forceinline__ T tshfl_xor(T v, int m)
{
    if constexpr (TS == 1) return v;
    else return __shfl_xor_sync(kFull, v, m, TS);
}

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
    int L, G;      // samples, groups of 4 (padded to whole BFPE groups)
    int g0, g1;    // this thread's groups of 4 [g0, g1) (empty if g1 <= g0)
    int gsh;       // log2(BFPE group size / 4): with groups of 8 (gsh = 1)
                   // G, g0 and g1 are even, so a thread owns whole groups
    int Eb;        // float block exponent
    bool bad;      // a non-finite sample
    bool active;   // the block exists
};

// Load the 4 samples of the group starting at sample s: one vector load
// when the group is whole and aligned.  Plain (generic) loads: the block
// may sit in global memory or in a shared-memory staging copy.  Past L the group is padded with
// zeros, or (PAD) with x[L-1], whose quantised value is the last-group
// padding of Sec. 6 packets (the replicated q[L-1]).
template <int DT, bool PAD = false>
__device__ __forceinline__ void load4(const TBlock<DT> &b, int s, typename LaneT<DT>::t (&x)[4])
{
    using raw = typename DT_<DT>::raw;
    using lt = typename LaneT<DT>::t;
    const raw *q = b.p + s;
    constexpr int ES = sizeof(raw);
    if (b.active && s + 4 <= b.L && ((uintptr_t)q & (4 * ES - 1)) == 0) {
        if constexpr (ES == 1) {
            const uint32_t w = *reinterpret_cast<const uint32_t *>(q);
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = (int8_t)(w >> (8 * j));
        } else if constexpr (ES == 2) {
            const uint2 w = *reinterpret_cast<const uint2 *>(q);
            x[0] = (int16_t)w.x; x[1] = (int16_t)(w.x >> 16);
            x[2] = (int16_t)w.y; x[3] = (int16_t)(w.y >> 16);
        } else if constexpr (ES == 4) {
            const uint4 w = *reinterpret_cast<const uint4 *>(q);
            x[0] = (lt)w.x; x[1] = (lt)w.y; x[2] = (lt)w.z; x[3] = (lt)w.w;
        } else {
            const ulonglong2 *r = reinterpret_cast<const ulonglong2 *>(q);
            const ulonglong2 w0 = r[0], w1 = r[1];
            x[0] = w0.x; x[1] = w0.y; x[2] = w1.x; x[3] = w1.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int i = s + j;
            if (PAD && i >= b.L) i = b.L - 1;
            if (b.active && i >= 0 && i < b.L) {
                if constexpr (DT_<DT>::F)
                    x[j] = *reinterpret_cast<const typename DT_<DT>::bits *>(b.p + i);
                else
                    x[j] = (lt)b.p[i];
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
        return *reinterpret_cast<const typename DT_<DT>::bits *>(b.p + s);
    else
        return (lt)b.p[s];
}

// ---------------------------------------------------------------- quantiser
// Per (block, code) quantiser (Sec. 6 attenuator: q = RNE(x a(c) 2^(Q-Eb)),
// one rounding of the exact product).
//   float32: with b = (256 - m) 2^(Q-Eb-8-k), an 8-bit integer times a power
//   of two and so exact in float32, q = RNE(x b).  A fused multiply-add
//   forms x b exactly and rounds x b + c once.  For k >= 1, |x b| < 2^22 and
//   c = 1.5 2^23 puts the sum in the binade [2^23, 2^24), whose unit is 1:
//   the rounding is RNE to an integer (c is even), and the result's bit
//   pattern differs from c's by exactly q.  For k = 0, |x b| < 2^23 and
//   c = +-2^23 with the sign of x does the same in magnitude; with m = 0 as
//   well b is a power of two, x b is exact in float32 (or below the normal
//   range, where it and q are 0), and one conversion with RNE gives q.
//   Blocks whose b leaves the normal range take the exact integer path.
//   int8/int16: the product x (256 - m) and the rounding shift by 8 + k in
//   32 bits.  Everything else: exact integer significand arithmetic.
template <int DT>
struct Quant {
    Code c;
    int Eb;
    int mode;     // 0 exact integer, 1 fused (k >= 1), 2 convert (k = 0, m = 0),
                  // 3 small int, 4 fused signed (k = 0, m > 0)
    float scale;  // b
    __device__ __forceinline__ Quant(int code, int eb) : c(code), Eb(eb), mode(0), scale(0.f)
    {
        if constexpr (DT == 4) {
            const int se = 15 - eb - c.k;  // b = (256 - m) 2^se; 2^(se+8) for m = 0
            if (!c.zero && se + 8 >= -126 && se + 8 <= 127 && se >= -126) {
                mode = c.k >= 1 ? 1 : (c.m == 0 ? 2 : 4);
                scale = __fmul_rn((float)(256 - c.m), __int_as_float((se + 127) << 23));
            }
        }
        if constexpr (DT == 1 || DT == 2) {
            // a = (256 - m) 2^-(8+k) as a float (exact, normal for k <= 31);
            // x a has at most 24 significant bits and |x a| <= 2^15, so one
            // FMA with 1.5 2^23 rounds it to the nearest integer, ties to even
            mode = 3;
            scale = c.zero ? 0.f : __fmul_rn((float)(256 - c.m), __int_as_float((119 - c.k) << 23));
        }
    }
    __device__ __forceinline__ int32_t operator()(typename LaneT<DT>::t v) const
    {
        if constexpr (DT == 4) {
            if (mode == 1) {
                const float t = __fmaf_rn(__uint_as_float(v), scale, 12582912.0f);
                return __float_as_int(t) - 0x4B400000;
            }
            if (mode == 2) return __float2int_rn(__fmul_rn(__uint_as_float(v), scale));
            if (mode == 4) {
                const uint32_t sg = v & 0x80000000u;
                const float t = __fmaf_rn(__uint_as_float(v), scale, __uint_as_float(sg | 0x4B000000u));
                const int32_t a = (__float_as_int(t) & 0x7fffffff) - 0x4B000000;
                return sg ? -a : a;
            }
        }
        if constexpr (DT == 1 || DT == 2) {
            const float t = __fmaf_rn((float)(int32_t)v, scale, 12582912.0f);
            return __float_as_int(t) - 0x4B400000;
        }
        return quantise<DT>(v, c, Eb);
    }
};

// The quantiser with its mode fixed at compile time (no per-sample mode
// test), and the dispatch that picks it once per (block, code).  Callers
// keep warp collectives outside the dispatched function: teams of one warp
// may take different modes.
template <int DT, int M>
struct QuantM {
    static constexpr int kMode = M;
    const Quant<DT> &Q;
    __device__ __forceinline__ explicit QuantM(const Quant<DT> &q) : Q(q) {}
    __device__ __forceinline__ int32_t operator()(typename LaneT<DT>::t v) const
    {
        if constexpr (DT == 4 && M == 1) {
            const float t = __fmaf_rn(__uint_as_float(v), Q.scale, 12582912.0f);
            return __float_as_int(t) - 0x4B400000;
        } else if constexpr (DT == 4 && M == 2) {
            return __float2int_rn(__fmul_rn(__uint_as_float(v), Q.scale));
        } else if constexpr (DT == 4 && M == 4) {
            const uint32_t sg = v & 0x80000000u;
            const float t = __fmaf_rn(__uint_as_float(v), Q.scale, __uint_as_float(sg | 0x4B000000u));
            const int32_t a = (__float_as_int(t) & 0x7fffffff) - 0x4B000000;
            return sg ? -a : a;
        } else if constexpr ((DT == 1 || DT == 2) && M == 3) {
            const float t = __fmaf_rn((float)(int32_t)v, Q.scale, 12582912.0f);
            return __float_as_int(t) - 0x4B400000;
        } else {
            return quantise<DT>(v, Q.c, Q.Eb);
        }
    }
};

template <int DT, class F>
__device__ __forceinline__ void with_quant(const Quant<DT> &Q, F &&f)
{
    if constexpr (DT == 4) {
        switch (Q.mode) {
        case 1: f(QuantM<DT, 1>(Q)); break;
        case 2: f(QuantM<DT, 2>(Q)); break;
        case 4: f(QuantM<DT, 4>(Q)); break;
        default: f(QuantM<DT, 0>(Q)); break;
        }
    } else if constexpr (DT == 1 || DT == 2) {
        f(QuantM<DT, 3>(Q));
    } else {
        f(QuantM<DT, 0>(Q));
    }
}

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
    // one team sum of both counts: nibbles < 2^14, exponent bits < 2^18
    const uint32_t both = team_sum<TS>((uint32_t)mine | ((uint32_t)c.sume << 14));
    nib_total = (int)(both & 0x3fffu);
    sume_total = (int)(both >> 14);
    if (s_in_out) *s_in_out = s_in;
    if (nib_mine) *nib_mine = mine;
}

// ---------------------------------------------------------------- block walk
// Open block j for a team: geometry of this thread's groups, float exponent.
template <int DT, int TS>
__device__ __forceinline__ void open_team_block(TBlock<DT> &b, const typename DT_<DT>::raw *x,
                                                uint64_t n, uint32_t N, uint64_t nb, uint64_t j,
                                                int gp, uint64_t base_block = 0, int gsh = 0)
{
    using T = DT_<DT>;
    b.active = j < nb;
    const uint64_t off = j * (uint64_t)N;
    // x holds blocks from base_block on (the array itself, or a staged tile)
    b.p = x + (b.active ? off - base_block * (uint64_t)N : 0);
    b.L = b.active ? (int)((n - off) < N ? (n - off) : N) : 0;
    b.gsh = gsh;
    b.G = gsh ? 2 * ((b.L + 7) >> 3) : (b.L + 3) >> 2;
    const int t = tlane<TS>();
    b.g0 = t * gp;
    b.g1 = min(b.g0 + gp, b.G);
    b.Eb = 0;
    b.bad = false;
    if constexpr (T::F) {
        // the largest magnitude's bit pattern; NaN and infinities have all
        // exponent bits set and so compare above every finite magnitude
        using B = typename T::bits;
        constexpr B absm = ~((B)1 << (sizeof(B) * 8 - 1));
        constexpr B expm = (B)T::EMAX << T::MB;
        B mx = 0;
#pragma unroll 1
        for (int g = b.g0; g < b.g1; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT>(b, 4 * g, xv);  // zeros past L do not change the maximum
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const B a = xv[i] & absm;
                mx = a > mx ? a : mx;
            }
        }
#pragma unroll
        for (int m = TS / 2; m >= 1; m >>= 1) {
            const B o = tshfl_xor<TS>(mx, m);
            mx = o > mx ? o : mx;
        }
        b.bad = mx >= expm;
        b.Eb = b.bad ? 0 : block_exp_from_maxbits<DT>((uint64_t)mx);
    }
}

// ---------------------------------------------------------------- streams (carried)
// The derivative streams of Sec. 6 from carried predecessors, with no
// per-sample position tests: S1 u_i = q_i - qp1, S2 u_i = q_i - 2 qp2 + qpp2
// (mod 2^W).  At the block start qp1 = 0, qp2 = q_0 and qpp2 = 2 q_0, which
// give u_0 = q_0 (both streams) and S2's u_1 = q_1 - q_0 through the same
// formulas; elsewhere the carries are the two preceding q.
struct Carry {
    uint32_t qp1, qp2, qpp2;
};

template <int DT, class QF>
__device__ __forceinline__ Carry carry_in(const TBlock<DT> &b, const QF &Q, int s0)
{
    Carry c;
    if (s0 == 0) {
        const uint32_t q0 = (uint32_t)Q(load1<DT>(b, 0));
        c.qp1 = 0;
        c.qp2 = q0;
        c.qpp2 = 2u * q0;
    } else {
        const uint32_t a = (uint32_t)Q(load1<DT>(b, s0 - 1));
        c.qp1 = a;
        c.qp2 = a;
        c.qpp2 = (uint32_t)Q(load1<DT>(b, s0 - 2));
    }
    return c;
}

// One group, all three streams (and the sum stream S3 when SUM): OR of
// the width terms of each stream.
template <int DT, bool SUM = false, class QF>
__device__ __forceinline__ void group3(const QF &Q, const typename LaneT<DT>::t (&xv)[4],
                                       Carry &c, uint32_t &o0, uint32_t &o1, uint32_t &o2,
                                       uint32_t *o3 = nullptr)
{
    constexpr int W = DT_<DT>::W;
    o0 = o1 = o2 = 0;
    uint32_t s3 = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t q = (uint32_t)Q(xv[i]);
        const uint32_t u1 = q - c.qp1, u2 = q - 2u * c.qp2 + c.qpp2;
        o0 |= bits_term((int32_t)q);  // q is already a W-bit value
        o1 |= bits_term(sext_w(u1, W));
        o2 |= bits_term(sext_w(u2, W));
        if constexpr (SUM) s3 |= bits_term(sext_w(q + c.qp1, W));
        c.qp1 = q;
        c.qpp2 = c.qp2;
        c.qp2 = q;
    }
    if constexpr (SUM) *o3 = s3;
}

// One stream s: coefficients of u = q - a qp + bb qpp and its carries.
// S3, the sum stream, is a = -1 on the S1 carry: u_0 = q_0, u_i = q_i + q_{i-1}.
struct Stream1 {
    uint32_t a, bb, qp, qpp;
    __device__ __forceinline__ Stream1(int s, const Carry &c)
    {
        a = s == 0 ? 0u : (s == 1 ? 1u : (s == 2 ? 2u : 0xffffffffu));
        bb = s == 2 ? 1u : 0u;
        qp = (s == 1 || s == 3) ? c.qp1 : c.qp2;
        qpp = c.qpp2;
    }
};

// One group, one stream: the quantised values, the stream values
// (sign-extended) and their OR of width terms.
template <int DT, class QF>
__device__ __forceinline__ uint32_t group1q(const QF &Q, const typename LaneT<DT>::t (&xv)[4],
                                            Stream1 &st, int32_t (&qv)[4], int32_t (&u)[4])
{
    constexpr int W = DT_<DT>::W;
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t q = (uint32_t)Q(xv[i]);
        qv[i] = (int32_t)q;
        u[i] = sext_w(q - st.a * st.qp + st.bb * st.qpp, W);
        o |= bits_term(u[i]);
        st.qpp = st.qp;
        st.qp = q;
    }
    return o;
}

template <int DT, class QF>
__device__ __forceinline__ uint32_t group1(const QF &Q, const typename LaneT<DT>::t (&xv)[4],
                                           Stream1 &st, int32_t (&u)[4])
{
    int32_t qv[4];
    return group1q<DT>(Q, xv, st, qv, u);
}

// Greedy JEE counters of the three streams at once (SIMD within a register:
// one 10-bit lane per stream; exponents <= 32, counts < 1024 per thread).
// Same transitions as TokCount::push.
struct Tok3 {
    static constexpr uint32_t L1 = 0x00100401u, L2 = 0x00200802u, L3 = 0x00300C03u,
                              B9 = 0x20080200u;
    uint32_t nib, lead, leading, st, e_first, e_last;
    int sume0, sume1, sume2;
    bool any;
    __device__ __forceinline__ void init()
    {
        nib = lead = st = e_first = e_last = 0;
        leading = L1;
        sume0 = sume1 = sume2 = 0;
        any = false;
    }
    __device__ __forceinline__ void push(int e0, int e1, int e2)
    {
        sume0 += e0;
        sume1 += e1;
        sume2 += e2;
        const uint32_t E = (uint32_t)e0 | ((uint32_t)e1 << 10) | ((uint32_t)e2 << 20);
        if (!any) {
            any = true;
            e_first = e_last = E;
            return;
        }
        const uint32_t D = E + B9 - e_last;  // 512 + e - e_prev per lane
        const uint32_t sm = (((D + L1) & ~(D - L2)) & B9) >> 9;  // |d| <= 1
        const uint32_t s2 = (((D + L2) & ~(D - L3)) & B9) >> 9;  // |d| <= 2
        nib = nib + L2 - s2 - (sm & st);
        st = sm & ~st;
        leading &= sm;
        lead += leading;
        e_last = E;
    }
    __device__ __forceinline__ TokCount lane(int s) const
    {
        TokCount t;
        const int sh = 10 * s;
        t.nib = (int)((nib >> sh) & 1023u);
        t.lead = (int)((lead >> sh) & 1023u);
        t.leading = (leading >> sh) & 1u;
        t.st = (st >> sh) & 1u;
        t.e_first = (int)((e_first >> sh) & 1023u);
        t.e_last = (int)((e_last >> sh) & 1023u);
        t.sume = s == 0 ? sume0 : (s == 1 ? sume1 : sume2);
        t.any = any;
        return t;
    }
};

// Unpadded packet bits of the team's block for streams S0-S2 (and S3 when
// SUM) at `code` (the stream decision of Sec. 6 evaluates them at code 0).
// With groups of 8 the width terms of two groups of 4 are ORed before an
// exponent is counted.
template <int DT, int TS, bool SUM>
__device__ __forceinline__ void team_eval_streams(const TBlock<DT> &b, int code, uint32_t (&bits)[4])
{
    const Quant<DT> Q(code, b.Eb);
    Tok3 tk;
    tk.init();
    TokCount t3;
    t3.init();
    with_quant<DT>(Q, [&](const auto &qf) {
        Carry c = carry_in<DT>(b, qf, 4 * b.g0);
        uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 1
        for (int g = b.g0; g < b.g1; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT, true>(b, 4 * g, xv);
            uint32_t o0, o1, o2, o3 = 0;
            group3<DT, SUM>(qf, xv, c, o0, o1, o2, &o3);
            a0 |= o0;
            a1 |= o1;
            a2 |= o2;
            a3 |= o3;
            if (!b.gsh || (g & 1)) {
                tk.push(exp_from_or(a0), exp_from_or(a1), exp_from_or(a2));
                if constexpr (SUM) t3.push(exp_from_or(a3), true);
                a0 = a1 = a2 = a3 = 0;
            }
        }
    });
    const bool first = b.g0 == 0;
    const uint32_t wm = 4u << b.gsh;  // mantissa bits per exponent unit
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        int nib, sume;
        team_tokens<TS>(tk.lane(s), first, nib, sume);
        bits[s] = (uint32_t)DT_<DT>::H + 4u * (uint32_t)nib + wm * (uint32_t)sume;
    }
    bits[3] = 0xffffffffu;
    if constexpr (SUM) {
        int nib, sume;
        team_tokens<TS>(t3, first, nib, sume);
        bits[3] = (uint32_t)DT_<DT>::H + 4u * (uint32_t)nib + wm * (uint32_t)sume;
    }
}

template <int DT, int TS>
__device__ __forceinline__ uint32_t team_eval1(const TBlock<DT> &b, int code, int s);

// The stream of fewest code-0 bits among S0-S2, and S3 when `sum` (ties to
// the lower index).  Warp-uniform `sum`.  S3 is sized by a second pass over
// the block (version-2 containers only), which keeps the version-1 pass's
// registers.
template <int DT, int TS>
__device__ __forceinline__ int team_best_stream(const TBlock<DT> &b, bool sum)
{
    uint32_t bb[4];
    team_eval_streams<DT, TS, false>(b, 0, bb);
    if (sum) bb[3] = team_eval1<DT, TS>(b, 0, 3);
    int s = 0;
    if (bb[1] < bb[s]) s = 1;
    if (bb[2] < bb[s]) s = 2;
    if (bb[3] < bb[s]) s = 3;
    return s;
}

// Unpadded packet bits of the team's block for stream s at `code`.
template <int DT, int TS>
__device__ __forceinline__ uint32_t team_eval1(const TBlock<DT> &b, int code, int s)
{
    const Quant<DT> Q(code, b.Eb);
    TokCount tc;
    tc.init();
    with_quant<DT>(Q, [&](const auto &qf) {
        Stream1 st(s, carry_in<DT>(b, qf, 4 * b.g0));
        uint32_t acc = 0;
#pragma unroll 1
        for (int g = b.g0; g < b.g1; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT, true>(b, 4 * g, xv);
            int32_t u[4];
            acc |= group1<DT>(qf, xv, st, u);
            if (!b.gsh || (g & 1)) {
                tc.push(exp_from_or(acc), true);
                acc = 0;
            }
        }
    });
    int nib, sume;
    team_tokens<TS>(tc, b.g0 == 0, nib, sume);
    return (uint32_t)DT_<DT>::H + 4u * (uint32_t)nib + (4u << b.gsh) * (uint32_t)sume;
}

// team_eval1 at code 0 that also leaves each BFPE group's exponent in
// ebuf[g >> gsh] (this thread's groups; the team's groups together).
template <int DT, int TS>
__device__ __forceinline__ uint32_t team_exps(const TBlock<DT> &b, int s, uint8_t *ebuf)
{
    const Quant<DT> Q(0, b.Eb);
    TokCount tc;
    tc.init();
    with_quant<DT>(Q, [&](const auto &qf) {
        Stream1 st(s, carry_in<DT>(b, qf, 4 * b.g0));
        uint32_t acc = 0;
#pragma unroll 1
        for (int g = b.g0; g < b.g1; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT, true>(b, 4 * g, xv);
            int32_t u[4];
            acc |= group1<DT>(qf, xv, st, u);
            if (!b.gsh || (g & 1)) {
                const int e = exp_from_or(acc);
                ebuf[g >> b.gsh] = (uint8_t)e;
                tc.push(e, true);
                acc = 0;
            }
        }
    });
    int nib, sume;
    team_tokens<TS>(tc, b.g0 == 0, nib, sume);
    return (uint32_t)DT_<DT>::H + 4u * (uint32_t)nib + (4u << b.gsh) * (uint32_t)sume;
}

// ---------------------------------------------------------------- staging
// Bulk (TMA) copies global -> shared memory completed on an mbarrier, in
// inline PTX.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_shared(void *dst, const void *src, uint32_t bytes, uint64_t *m)
{
    uint64_t g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(g), "r"(bytes), "r"(smem_addr(m))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_inval(uint64_t *m)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(m)) : "memory");
}

// Copy blocks [b0, b1) of the array into shared memory (all threads of the
// CTA call it; zeros past n), so that the codec's repeated passes over a
// block read shared memory instead of L2.  The 16-byte aligned bulk of the
// range moves with one TMA bulk copy; the rest (an unaligned source, the
// ragged tail, the zeros past n) with vector loads.  The wait on the copy is
// bounded: past `spin` clock cycles the status becomes APAX_ERR_TIMEOUT and
// the copy is waited for once more (bounded).  Returns true (the same value
// in every thread) when the staged copy is complete; false when a wait ran
// out, in which case the caller must not read xs (it reads the array from
// global memory instead) and the barrier, which may still expect bytes, is
// left as it is.
template <int DT>
__device__ __forceinline__ bool stage_blocks(typename DT_<DT>::raw *xs, const typename DT_<DT>::raw *x,
                                             uint64_t n, uint32_t N, uint64_t b0, uint64_t b1,
                                             int *status, long long spin)
{
    using raw = typename DT_<DT>::raw;
    constexpr int ES = sizeof(raw);
    __shared__ __align__(8) uint64_t s_mbar;
    const uint64_t s0 = b0 * (uint64_t)N;
    const uint64_t s1 = min(b1 * (uint64_t)N, n);
    const uint64_t send = b1 * (uint64_t)N;  // staged samples end (zeros from s1)
    const bool al16 = (((uintptr_t)(x + s0)) & 15) == 0 && (((uintptr_t)xs) & 15) == 0;
    // bulk part: whole 16-byte chunks of real samples
    const uint64_t bulk_bytes = al16 && s1 > s0 ? (((s1 - s0) * ES) / 16) * 16 : 0;
    const uint64_t bulk_elems = bulk_bytes / ES;
    if (bulk_bytes) {
        if (threadIdx.x == 0) {
            mbar_init(&s_mbar, 1);
            mbar_expect_tx(&s_mbar, (uint32_t)bulk_bytes);
            bulk_to_shared(xs, x + s0, (uint32_t)bulk_bytes, &s_mbar);
        }
    }
    // the rest, element by element (disjoint from the bulk part)
    for (uint64_t i = s0 + bulk_elems + threadIdx.x; i < send; i += blockDim.x)
        xs[i - s0] = i < s1 ? x[i] : (raw)0;
    if (!bulk_bytes) return true;
    __syncthreads();  // the barrier is initialised before anyone waits on it
    const long long t0 = clock64();
    bool done = mbar_try_wait(&s_mbar, 0);
    while (!done && clock64() - t0 <= spin) done = mbar_try_wait(&s_mbar, 0);
    if (!done) {
        atomicMin(status, -10);
        const long long t1 = clock64();
        while (!done && clock64() - t1 <= spin) done = mbar_try_wait(&s_mbar, 0);
    }
    const bool all = __syncthreads_and(done) != 0;
    if (all && threadIdx.x == 0) mbar_inval(&s_mbar);
    return all;
}

// Largest packet of a block of N samples (all widths W, all tokens absolute).
__host__ __device__ inline uint32_t max_packet_words(int H, int W, uint32_t N)
{
    const uint32_t G = (N + 3) / 4;
    const uint64_t bits = (uint64_t)H + 8ull * G + (uint64_t)W * 4ull * G;
    return (uint32_t)((bits + 31) / 32);
}

}  // namespace apax
