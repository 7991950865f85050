// apax_decode.cu -- block decoder (inverse of the Sec. 6 encoder).
//
// A team of 8 threads decodes one block: header -> JEE tokens (parallel
// parse: every thread takes 16 nibbles of a 128-nibble window; the
// token/continuation state of its first nibble comes from a team scan of
// two-state transition functions) -> exponents (each thread resolves its own
// groups after a segmented team scan) -> mantissas (each thread unpacks its
// contiguous groups) -> inverse derivatives (S1: prefix sum; S2: u_0 plus a
// double prefix sum of the remaining values; S3, the sum stream of version-2
// containers: an alternating-sign prefix sum; team-scanned as (sum, sum of
// prefixes, length) triples, all mod 2^W) -> dequantisation with the
// reciprocal table, rounded once to the output type.  Version-2 containers
// with BFPE groups of 8 keep one exponent per 8 samples (two groups of 4 of
// one width).  Teams stride over blocks; fixed-rate packets sit at j*B,
// fixed-quality ones at the offset table's word offsets, so any block range
// can be decoded on its own.
#include "apax_team.cuh"
#include "apax_kernels.h"

namespace apax {

namespace {

__device__ __forceinline__ void set_status(int *st, int code) { atomicMin(st, code); }

// Bounded word reader over one packet.
struct PktReader {
    const uint32_t *w;
    uint32_t nwords;
    __device__ __forceinline__ uint32_t get(uint32_t i, bool &oob) const
    {
        if (i >= nwords) {
            oob = true;
            return 0;
        }
        return __ldg(w + i);
    }
    // 64 bits starting at bit b (zero past the packet; the caller checks the
    // extent of what it consumes)
    __device__ __forceinline__ uint64_t bits64(uint32_t b) const
    {
        bool dummy = false;
        const uint32_t i = b >> 5, sh = b & 31;
        const uint64_t lo = (uint64_t)get(i, dummy) | ((uint64_t)get(i + 1, dummy) << 32);
        const uint64_t hi = get(i + 2, dummy);
        return sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
    }
};

// Sequential reader of e-bit two's-complement fields.
struct FieldReader {
    const PktReader *pr;
    uint32_t wi;
    int sh;
    uint64_t acc;
    int fill;
    bool started;
    __device__ __forceinline__ void init(const PktReader *p, uint32_t bit)
    {
        pr = p;
        wi = bit >> 5;
        sh = bit & 31;
        acc = 0;
        fill = 0;
        started = false;
    }
    __device__ __forceinline__ int32_t get(int e, bool &oob)
    {
        if (e == 0) return 0;
        if (!started) {
            acc = (uint64_t)pr->get(wi, oob) >> sh;
            fill = 32 - sh;
            started = true;
        }
        if (fill < e) {
            acc |= (uint64_t)pr->get(++wi, oob) << fill;
            fill += 32;
        }
        const uint32_t m = e >= 32 ? 0xffffffffu : ((1u << e) - 1u);
        const uint32_t v = (uint32_t)acc & m;
        acc >>= e;
        fill -= e;
        return e >= 32 ? (int32_t)v : ((int32_t)(v << (32 - e)) >> (32 - e));
    }
};

// two-state function composition, 2 bits: bit s = image of state s
// (state 0: a token starts here; 1: second nibble of an absolute token)
__device__ __forceinline__ uint32_t fafter(uint32_t f, uint32_t g)  // g after f
{
    const uint32_t i0 = (g >> (f & 1)) & 1, i1 = (g >> ((f >> 1) & 1)) & 1;
    return i0 | (i1 << 1);
}

template <int TS, typename T>
__device__ __forceinline__ T team_max(T v)
{
#pragma unroll
    for (int m = TS / 2; m >= 1; m >>= 1) {
        const T o = tshfl_xor<TS>(v, m);
        v = o > v ? o : v;
    }
    return v;
}

// Parse the JEE token section (Sec. 6) into ebuf: G exponents.  Returns the
// nibble count, or -1 for a malformed section.  Warp-collective: every team
// of the warp calls it (a team with G = 0 just follows along).
template <int TS>
__device__ int parse_tokens(const PktReader &pr, int H, int G, int W, uint8_t *ebuf, int g0, int g1)
{
    const int t = tlane<TS>();
    constexpr int WIN = 16 * TS;
    int done_g = 0, tpos = 0;
    bool bad = false;
    // pass 1: one entry per group: 0x80|v (absolute) or 8+d (diff)
    while (__any_sync(kFull, done_g < G && !bad)) {
        const bool need = done_g < G && !bad;
        const uint64_t v64 = need ? pr.bits64((uint32_t)H + 4u * (uint32_t)(tpos + 16 * t)) : 0;
        uint32_t F = 2u;  // identity
#pragma unroll
        for (int i = 0; i < 16; ++i) F = fafter(F, ((v64 >> (4 * i)) & 15) >= 14 ? 1u : 0u);
        uint32_t inc = F;
#pragma unroll
        for (int d = 1; d < TS; d <<= 1) {
            const uint32_t o = tshfl_up<TS>(inc, d);
            if (t >= d) inc = fafter(o, inc);
        }
        uint32_t exc = tshfl_up<TS>(inc, 1);
        if (t == 0) exc = 2u;
        const uint32_t next_first = (uint32_t)tshfl_down<TS>((int)(v64 & 15), 1);
        // my 16 nibbles: complete tokens (the window's last nibble may open an
        // absolute token that ends in the next window)
        uint32_t state = exc & 1, startmask = 0;
        int lg = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const uint32_t nb = (v64 >> (4 * i)) & 15;
            if (state == 0 && 16 * t + i + (nb >= 14 ? 2 : 1) <= WIN) {
                startmask |= 1u << i;
                lg += nb <= 8 ? 2 : 1;
            }
            state = state == 0 ? (nb >= 14 ? 1u : 0u) : 0u;
        }
        const int incl = team_incl_scan<TS>(lg);
        int gpos = done_g + incl - lg;
        int used_end = 0;
        if (need) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (!((startmask >> i) & 1)) continue;
                const uint32_t nb = (v64 >> (4 * i)) & 15;
                if (gpos < G) {
                    if (nb >= 14) {
                        const uint32_t lo = i < 15 ? (uint32_t)((v64 >> (4 * (i + 1))) & 15) : next_first;
                        ebuf[gpos] = (uint8_t)(0x80u | (((nb - 14) << 4) | lo));
                    } else if (gpos == 0) {
                        bad = true;  // the first exponent must be absolute
                    } else if (nb <= 8) {
                        if (gpos + 1 >= G) {
                            bad = true;  // a joint token needs two diffs
                        } else {
                            ebuf[gpos] = (uint8_t)(8 + (int)(nb / 3) - 1);
                            ebuf[gpos + 1] = (uint8_t)(8 + (int)(nb % 3) - 1);
                        }
                    } else {
                        ebuf[gpos] = (uint8_t)(8 + (int)nb - 11);
                    }
                    used_end = max(used_end, 16 * t + i + (nb >= 14 ? 2 : 1));
                }
                gpos += nb <= 8 ? 2 : 1;
            }
        }
        used_end = team_max<TS>(used_end);
        bad = team_sum<TS>((int)bad) > 0;
        const int avail = tshfl<TS>(incl, TS - 1);
        if (need) {
            if (avail <= 0) bad = true;
            done_g += min(avail, G - done_g);
            tpos += used_end;
        }
    }
    __syncwarp();
    // (no early return: the shuffles below need every lane of the warp)
    bad = team_sum<TS>((int)bad) > 0;
    if (bad) g1 = g0;  // a malformed team resolves nothing
    // pass 2: resolve my groups (segmented scan of "absolute resets, diffs add")
    bool f = false;
    int v = 0;
    for (int g = g0; g < g1; ++g) {
        const uint32_t a = ebuf[g];
        if (a & 0x80) {
            f = true;
            v = (a & 31) == 31 ? 32 : (int)(a & 31);
        } else {
            v += (int)a - 8;
        }
    }
    bool sf = f;
    int sv = v;
#pragma unroll
    for (int d = 1; d < TS; d <<= 1) {
        const bool of = tshfl_up<TS>((int)sf, d) != 0;
        const int ov = tshfl_up<TS>(sv, d);
        if (t >= d && !sf) {
            sv += ov;
            sf = of;
        }
    }
    const int e_before = tshfl_up<TS>(sv, 1);  // exponent of group g0 - 1
    __syncwarp();
    const int lim = W >= 32 ? 32 : W;
    int e = e_before;
    for (int g = g0; g < g1; ++g) {
        const uint32_t a = ebuf[g];
        e = (a & 0x80) ? ((a & 31) == 31 ? 32 : (int)(a & 31)) : e + (int)a - 8;
        bad |= e < 0 || e > lim || e == 31;
        ebuf[g] = (uint8_t)(e < 0 ? 0 : (e > 32 ? 32 : e));
    }
    __syncwarp();
    bad = team_sum<TS>((int)bad) > 0;
    return bad ? -1 : tpos;
}

template <int DT>
__device__ __forceinline__ void store4(typename DT_<DT>::raw *y, int s0, int lim,
                                       const typename LaneT<DT>::t (&v)[4])
{
    using raw = typename DT_<DT>::raw;
    raw *q = y + s0;
    constexpr int ES = sizeof(raw);
    if (s0 + 4 <= lim && ((uintptr_t)q & (4 * ES - 1)) == 0) {
        if constexpr (ES == 1) {
            *reinterpret_cast<uint32_t *>(q) = ((uint32_t)v[0] & 0xffu) | (((uint32_t)v[1] & 0xffu) << 8) |
                                              (((uint32_t)v[2] & 0xffu) << 16) | ((uint32_t)v[3] << 24);
        } else if constexpr (ES == 2) {
            *reinterpret_cast<uint2 *>(q) =
                make_uint2(((uint32_t)v[0] & 0xffffu) | ((uint32_t)v[1] << 16),
                           ((uint32_t)v[2] & 0xffffu) | ((uint32_t)v[3] << 16));
        } else if constexpr (ES == 4) {
            *reinterpret_cast<uint4 *>(q) = make_uint4((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2], (uint32_t)v[3]);
        } else {
            ulonglong2 *o = reinterpret_cast<ulonglong2 *>(q);
            o[0] = make_ulonglong2(v[0], v[1]);
            o[1] = make_ulonglong2(v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (s0 + i < lim) {
                if constexpr (DT_<DT>::F)
                    reinterpret_cast<typename DT_<DT>::bits *>(q)[i] = v[i];
                else
                    q[i] = (raw)v[i];
            }
        }
    }
}

// Dequantiser of one block (Sec. 6 attenuator inverse with the decoder's
// reciprocal table R[m] = RNE(2^32 / (256 - m))).  Floats with m = 0 whose
// results are normal take y = float(q) * 2^(Eb - Q + k), which is exact.
template <int DT>
struct Dequant {
    Code c;
    int Eb;
    uint32_t R;
    bool fast;
    float scale;
    __device__ __forceinline__ Dequant(int code, int eb)
        : c(code), Eb(eb), R(recip_entry(code & 127)), fast(false), scale(0.f)
    {
        if constexpr (DT == 4) {
            const int se = eb - 23 + c.k;
            if (!c.zero && c.m == 0 && se >= -126 && eb + c.k <= 127) {
                fast = true;
                scale = __int_as_float((se + 127) << 23);
            }
        }
    }
    __device__ __forceinline__ typename LaneT<DT>::t operator()(int32_t qi) const
    {
        using T = DT_<DT>;
        using lt = typename LaneT<DT>::t;
        if constexpr (!T::F) {
            int64_t yv = 0;
            if (!c.zero && qi != 0) {
                const int64_t V = (int64_t)qi * (int64_t)R;
                if (c.k <= 23) {
                    yv = rne_shift_s64(V, 24 - c.k);
                } else {
                    const int sh2 = c.k - 24;
                    const int64_t lim = (int64_t)1 << (62 - sh2);
                    yv = V >= lim ? INT64_MAX : (V <= -lim ? INT64_MIN : V * ((int64_t)1 << sh2));
                }
            }
            constexpr int64_t lo = DT == 1 ? -128 : (DT == 2 ? -32768 : -2147483648ll);
            constexpr int64_t hi = DT == 1 ? 127 : (DT == 2 ? 32767 : 2147483647ll);
            yv = yv < lo ? lo : (yv > hi ? hi : yv);
            return (lt)yv;
        } else {
            if (c.zero || qi == 0) return (lt)0;
            if constexpr (DT == 4) {
                if (fast) return __float_as_uint(__fmul_rn(__int2float_rn(qi), scale));
            }
            return round_to_format<DT>((int64_t)qi * (int64_t)R, Eb - T::Q + c.k - 24);
        }
    }
};

// Container header fields (40 bytes, little endian; see the encoder).
struct DecHdr {
    uint32_t N, B;
    uint64_t n, payload, poff, nb;
    int mode;
    int gsh;  // version 2: log2(BFPE group size / 4)
    int sum;  // version 2: selector 3 (the sum stream) is valid
    int err;  // 0, or the status a malformed or mismatched header gives
};

__device__ __forceinline__ DecHdr read_header(const DecArgs &a)
{
    DecHdr h;
    h.N = h.B = 0;
    h.n = h.payload = h.poff = h.nb = 0;
    h.mode = 0;
    h.gsh = h.sum = 0;
    h.err = -9;
    const uint8_t *in = a.in;
    if (!(in && a.in_bytes >= 40 && in[0] == 'A' && in[1] == 'P' && in[2] == 'X' && in[3] == '1'))
        return h;
    // version 1: no format option; version 2: at least one (flags bits 1-2)
    const int fmt = (in[7] >> 1) & 0x7f;
    if (!((in[4] == 1 && fmt == 0) || (in[4] == 2 && fmt >= 1 && fmt <= 3))) return h;
    h.gsh = fmt & 1;
    h.sum = (fmt >> 1) & 1;
    auto le = [&](int o, int k) {
        uint64_t v = 0;
        for (int i = 0; i < k; ++i) v |= (uint64_t)in[o + i] << (8 * i);
        return v;
    };
    h.mode = in[6];
    h.N = (uint32_t)le(8, 4);
    h.B = (uint32_t)le(16, 4);
    h.n = le(20, 8);
    h.payload = le(28, 8);
    if (in[5] != a.dtype || h.n != a.n) {
        h.err = -1;
        return h;
    }
    if (h.N < 64 || h.N > 16384 || (h.N & (h.gsh ? 7u : 3u)) || (h.mode != 0 && h.mode != 1)) return h;
    h.nb = (h.n + h.N - 1) / h.N;
    h.poff = 40 + (h.mode == 1 ? ((4 * h.nb + 7) / 8) * 8 : 0);
    if (h.poff > a.in_bytes || h.payload > a.in_bytes - h.poff) return h;
    if (h.mode == 0 && ((h.B & 3) || h.B == 0)) return h;
    if (a.ranged && (a.b1 > h.nb || a.b0 > a.b1)) {
        h.err = -1;
        return h;
    }
    h.err = 0;
    return h;
}

// One tile: the CTA's teams decode blocks jb + tile * nteams + team of the
// array (jb = the first block of the requested range).  Teams of TS threads
// with EB bytes of exponent buffer each: (8, 1024) for block sizes up to
// 4096, (32, 4096) above.
template <int DT, int TS, int EB>
__device__ __forceinline__ void decode_tile(const DecArgs &a, const DecHdr &hd, uint64_t tile,
                                            uint8_t *dsm)
{
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    constexpr int W = T::W, H = T::H;
    const int team = threadIdx.x / TS, t = tlane<TS>();
    const int nteams = blockDim.x / TS;
    uint8_t *ebuf = dsm + (size_t)team * EB;
    const uint8_t *in = a.in;
    const uint32_t N = hd.N, B = hd.B;
    const uint64_t n = hd.n, payload = hd.payload, poff = hd.poff, nb = hd.nb;
    const int mode = hd.mode;
    const int gsh = hd.gsh;
    // groups of 4 per thread; with groups of 8 an even count (whole groups)
    const int gp = gsh ? 2 * (int)((N / 8 + TS - 1) / TS) : (int)((N / 4 + TS - 1) / TS);
    const uint64_t jb = a.ranged ? a.b0 : 0, je = a.ranged ? a.b1 : nb;
    const uint32_t *tab = reinterpret_cast<const uint32_t *>(in + 40);
    {
        const uint64_t j = jb + tile * (uint64_t)nteams + (uint64_t)team;
        const bool active = j < je;
        int L = 0, G = 0;
        bool bad = false;
        PktReader pr;
        pr.w = reinterpret_cast<const uint32_t *>(in + poff);
        pr.nwords = 0;
        if (active) {
            const uint64_t start = mode == 1 ? 4ull * (uint64_t)__ldg(tab + j) : j * (uint64_t)B;
            const uint64_t off = j * (uint64_t)N;
            L = (int)((n - off) < N ? (n - off) : N);
            G = gsh ? 2 * ((L + 7) >> 3) : (L + 3) >> 2;
            bad = start >= payload || (start & 3);
            if (!bad) {
                pr.w = reinterpret_cast<const uint32_t *>(in + poff + start);
                const uint64_t aw = (payload - start) >> 2;
                pr.nwords = (uint32_t)(aw > 0xffffffffull ? 0xffffffffull : aw);
            }
        }
        bool oob = false;
        const uint32_t h0 = active && !bad ? pr.get(0, oob) : 0;
        const int s = h0 & 3, code = (h0 >> 2) & 4095;
        const uint32_t plen = h0 >> 14;
        if (active) {
            bad |= oob || (s == 3 && !hd.sum) || plen < 4 || (plen & 3) ||
                   (uint64_t)plen > 4ull * pr.nwords;
            if (mode == 0 && j + 1 < nb && plen != B) bad = true;
        }
        int Eb = 0;
        if (active && !bad) {
            pr.nwords = plen >> 2;
            if (T::F) Eb = (int)(int16_t)(pr.get(1, oob) & 0xffffu);
        }
        bad = team_sum<TS>((int)bad) > 0;
        if (active && bad && t == 0) set_status(a.status, -9);
        const bool go0 = active && !bad;
        const int Gt = go0 ? G : 0;
        const int g0 = t * gp, g1 = min(g0 + gp, Gt);
        // one exponent per BFPE group: ebuf[g >> gsh] for the groups of 4 g
        const int nib = parse_tokens<TS>(pr, H, Gt >> gsh, W, ebuf, g0 >> gsh, g1 >> gsh);
        const bool go = go0 && nib >= 0;
        if (go0 && nib < 0 && t == 0) set_status(a.status, -9);
        // mantissa bit offset of my groups
        int mysum = 0;
        if (go)
            for (int g = g0; g < g1; ++g) mysum += ebuf[g >> gsh];
        const int incl4 = team_incl_scan<TS>(4 * mysum);
        const int total4 = tshfl<TS>(incl4, TS - 1);
        if (go && t == 0 && (uint64_t)H + 4ull * (uint64_t)nib + (uint64_t)total4 > 8ull * plen)
            set_status(a.status, -9);
        const uint32_t bit0 = (uint32_t)H + 4u * (uint32_t)(go ? nib : 0) + (uint32_t)(incl4 - 4 * mysum);
        const Dequant<DT> DQ(code, Eb);
        raw *yb = reinterpret_cast<raw *>(a.y) +
                  (a.ranged ? (j - a.b0) * (uint64_t)N : j * (uint64_t)N);
        const int lim = min(L, 4 * g1);  // my samples end here
        const int ge = go ? g1 : g0;      // my groups [g0, ge)
        // totals of my samples for the team scan: S = sum w, D = sum of
        // prefixes of w, len = count; w = u except u_0 of an S2 block, and
        // w_i = (-1)^i u_i for S3, whose inverse q_i = u_i - q_{i-1} is
        // q_i = (-1)^i (w_0 + ... + w_i)
        uint32_t S = 0, D = 0, u0 = 0;
        int len = 0;
        FieldReader fr;
        if (s != 0) {
            fr.init(&pr, bit0);
#pragma unroll 1
            for (int g = g0; g < ge; ++g) {
                const int e = ebuf[g >> gsh];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int32_t uv = fr.get(e, oob);
                    const int idx = 4 * g + i;
                    if (idx == 0) u0 = (uint32_t)uv;
                    S += (s == 2 && idx == 0) ? 0u
                                              : ((s == 3 && (i & 1)) ? 0u - (uint32_t)uv : (uint32_t)uv);
                    D += S;
                }
            }
            len = 4 * (ge - g0);
        }
        // team scan of (S, D, len): A then B -> (SA+SB, DA+DB+lenB*SA, lenA+lenB)
        uint32_t sS = S, sD = D;
        int sl = len;
#pragma unroll
        for (int d = 1; d < TS; d <<= 1) {
            const uint32_t oS = tshfl_up<TS>(sS, d), oD = tshfl_up<TS>(sD, d);
            const int ol = tshfl_up<TS>(sl, d);
            if (t >= d) {
                sD = oD + sD + (uint32_t)sl * oS;
                sS = oS + sS;
                sl = ol + sl;
            }
        }
        uint32_t runS = tshfl_up<TS>(sS, 1), runD = tshfl_up<TS>(sD, 1);
        if (t == 0) runS = runD = 0;
        const uint32_t u0b = tshfl<TS>(u0, 0);
        // values: inverse derivatives, dequantised, stored 4 at a time
        fr.init(&pr, bit0);
#pragma unroll 1
        for (int g = g0; g < ge; ++g) {
            const int e = ebuf[g >> gsh];
            lt out[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int32_t uv = fr.get(e, oob);
                const int idx = 4 * g + i;
                uint32_t q;
                if (s == 0) {
                    q = (uint32_t)uv;
                } else if (s == 1) {
                    runS += (uint32_t)uv;
                    q = runS;
                } else if (s == 2) {
                    runS += idx == 0 ? 0u : (uint32_t)uv;
                    runD += runS;
                    q = u0b + runD;
                } else {
                    runS += (i & 1) ? 0u - (uint32_t)uv : (uint32_t)uv;
                    q = (i & 1) ? 0u - runS : runS;
                }
                out[i] = DQ(sext_w(q, W));
            }
            store4<DT>(yb, 4 * g, lim, out);
        }
        const int any_oob = team_sum<TS>((int)(go && oob));
        if (go && any_oob > 0 && t == 0) set_status(a.status, -9);
    }
}

// One block by one thread (block sizes up to kT1MaxBlock): header, the JEE
// tokens in order, then the mantissas, inverse derivatives and
// dequantisation in one sequential pass -- no team scans.  eb is this
// thread's column of exponent bytes (stride est).

template <int DT>
__device__ __forceinline__ void decode_block_t1(const DecArgs &a, const DecHdr &hd, uint64_t j,
                                                uint8_t *eb, int est)
{
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    constexpr int W = T::W, H = T::H;
    const uint32_t N = hd.N;
    const uint64_t off = j * (uint64_t)N;
    const int L = (int)((hd.n - off) < N ? (hd.n - off) : N);
    const int gsh = hd.gsh;
    const int G = gsh ? 2 * ((L + 7) >> 3) : (L + 3) >> 2;  // groups of 4
    const int GX = G >> gsh;                                // BFPE groups
    const uint8_t *in = a.in;
    const uint64_t start = hd.mode == 1
                               ? 4ull * (uint64_t)__ldg(reinterpret_cast<const uint32_t *>(in + 40) + j)
                               : j * (uint64_t)hd.B;
    if (start >= hd.payload || (start & 3)) {
        set_status(a.status, -9);
        return;
    }
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(in + hd.poff + start);
    const uint64_t aw = (hd.payload - start) >> 2;
    uint32_t nwords = (uint32_t)(aw > 0xffffffffull ? 0xffffffffull : aw);
    bool bad = false;
    auto word = [&](uint32_t i) -> uint32_t {
        if (i >= nwords) {
            bad = true;
            return 0u;
        }
        return __ldg(pw + i);
    };
    const uint32_t h0 = word(0);
    const int s = h0 & 3, code = (h0 >> 2) & 4095;
    const uint32_t plen = h0 >> 14;
    bad |= (s == 3 && !hd.sum) || plen < 4 || (plen & 3) || (uint64_t)plen > 4ull * nwords;
    if (hd.mode == 0 && j + 1 < hd.nb && plen != hd.B) bad = true;
    if (bad) {
        set_status(a.status, -9);
        return;
    }
    nwords = plen >> 2;
    int Eb = 0;
    if (T::F) Eb = (int)(int16_t)(word(1) & 0xffffu);
    // LSB-first bit reader: bits [p, p + 32) of the packet are the funnel
    // shift of the word pair (c0, c1); the three words after c1 are loaded
    // ahead, so a load's latency overlaps about ten fields before its word
    // is needed.  Words past the packet read as zero; the bit count is
    // checked against the packet length before any field is read.
    uint32_t p = 0, wi = 0, c0 = 0, c1 = 0, n0 = 0, n1 = 0, n2 = 0;
    auto peek = [&](uint32_t i) -> uint32_t { return i < nwords ? __ldg(pw + i) : 0u; };
    auto seek = [&](uint32_t bit) {
        p = bit;
        wi = bit >> 5;
        c0 = peek(wi);
        c1 = peek(wi + 1);
        n0 = peek(wi + 2);
        n1 = peek(wi + 3);
        n2 = peek(wi + 4);
    };
    // the next 32 bits (a field of k <= 32 bits is their low k bits), then
    // moves k bits on: at most one word boundary is crossed
    auto take = [&](uint32_t k) -> uint32_t {
        const uint32_t v = __funnelshift_r(c0, c1, p);
        const uint32_t np = p + k;
        if ((np ^ p) >= 32u) {
            c0 = c1;
            c1 = n0;
            n0 = n1;
            n1 = n2;
            ++wi;
            n2 = peek(wi + 4);
        }
        p = np;
        return v;
    };
    // tokens (Sec. 6 JEE): absolute first, then joint / single / absolute
    constexpr int lim = W >= 32 ? 32 : W;
    seek((uint32_t)H);
    int g = 0, ep = 0, nib = 0, sume = 0;
    auto put = [&](int e) {
        bad |= e < 0 || e > lim || e == 31;
        e = e < 0 ? 0 : (e > 32 ? 32 : e);
        eb[(size_t)g * est] = (uint8_t)e;
        sume += e;
        ep = e;
        ++g;
    };
    while (g < GX && !bad) {
        const int nb = (int)(take(4) & 15u);
        ++nib;
        if (nb >= 14) {
            const int v = ((nb - 14) << 4) | (int)(take(4) & 15u);
            ++nib;
            put(v == 31 ? 32 : v);
        } else if (g == 0) {
            bad = true;  // the first exponent is absolute
        } else if (nb <= 8) {
            if (g + 1 >= GX) {
                bad = true;  // a joint token needs two diffs
            } else {
                const int d1 = (nb * 11) >> 5;  // nb / 3 for nb <= 8
                const int e1 = ep + d1 - 1;
                put(e1);
                put(e1 + (nb - 3 * d1) - 1);
            }
        } else {
            put(ep + nb - 11);
        }
    }
    if (!bad && (uint64_t)H + 4ull * (uint64_t)nib + (4ull << gsh) * (uint64_t)sume > 8ull * plen)
        bad = true;
    if (bad) {
        set_status(a.status, -9);
        return;
    }
    // values: fields, inverse derivative, dequantisation, 4 at a time
    const Dequant<DT> DQ(code, Eb);
    raw *yb = reinterpret_cast<raw *>(a.y) + (a.ranged ? (j - a.b0) * (uint64_t)N : off);
    seek((uint32_t)H + 4u * (uint32_t)nib);
    // the four fields of a group, sign-extended from e bits (e = 0: zeros);
    // two fields per read when they fit in 32 bits
    auto fields = [&](int gg, int32_t (&u)[4]) {
        const uint32_t e = eb[(size_t)(gg >> gsh) * est];
        if (e <= 16) {
            const uint32_t v0 = take(2 * e), v1 = take(2 * e);
            u[0] = bfe_s32(v0, 0, e);
            u[1] = bfe_s32(v0, e, e);
            u[2] = bfe_s32(v1, 0, e);
            u[3] = bfe_s32(v1, e, e);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) u[i] = bfe_s32(take(e), 0, e);
        }
    };
    auto emit = [&](int gg, const uint32_t (&q)[4]) {
        lt out[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = DQ(sext_w(q[i], W));
        store4<DT>(yb, 4 * gg, L, out);
    };
    // One loop per stream selector when every converged lane has the same
    // one (lanes decode different blocks: mixed selectors would run the
    // loops one after another), else one loop that branches per sample.
    // float64 keeps the one loop: its dequantiser makes copies costly.
    const unsigned am = __activemask();
    const bool uniform = DT != 5 && __all_sync(am, s == __shfl_sync(am, s, __ffs(am) - 1));
    if (!uniform) {
        uint32_t run = 0, runD = 0, u0 = 0;
#pragma unroll 1
        for (int gg = 0; gg < G; ++gg) {
            int32_t u[4];
            fields(gg, u);
            uint32_t q[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t uv = (uint32_t)u[i];
                if (s == 0) {
                    q[i] = uv;
                } else if (s == 1) {
                    run += uv;
                    q[i] = run;
                } else if (s == 2) {
                    if (gg == 0 && i == 0) u0 = uv;  // second differences start from the first value
                    else run += uv;
                    runD += run;
                    q[i] = u0 + runD;
                } else {
                    run = uv - run;  // the sum stream: q_i = u_i - q_{i-1}
                    q[i] = run;
                }
            }
            emit(gg, q);
        }
    } else if (s == 0) {
#pragma unroll 1
        for (int gg = 0; gg < G; ++gg) {
            int32_t u[4];
            fields(gg, u);
            const uint32_t q[4] = {(uint32_t)u[0], (uint32_t)u[1], (uint32_t)u[2], (uint32_t)u[3]};
            emit(gg, q);
        }
    } else if (s == 1) {
        uint32_t run = 0;
#pragma unroll 1
        for (int gg = 0; gg < G; ++gg) {
            int32_t u[4];
            fields(gg, u);
            uint32_t q[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = run += (uint32_t)u[i];
            emit(gg, q);
        }
    } else if (s == 3) {
        // the sum stream: q_i = u_i - q_{i-1}
        uint32_t run = 0;
#pragma unroll 1
        for (int gg = 0; gg < G; ++gg) {
            int32_t u[4];
            fields(gg, u);
            uint32_t q[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = run = (uint32_t)u[i] - run;
            emit(gg, q);
        }
    } else {
        // second differences: the first field is the first value itself
        uint32_t run = 0, runD = 0, u0 = 0;
#pragma unroll 1
        for (int gg = 0; gg < G; ++gg) {
            int32_t u[4];
            fields(gg, u);
            if (gg == 0) {
                u0 = (uint32_t)u[0];
                u[0] = 0;
            }
            uint32_t q[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                run += (uint32_t)u[i];
                runD += run;
                q[i] = u0 + runD;
            }
            emit(gg, q);
        }
    }
}

// Size class of a container: teams of 32 for blocks above 4096 samples and
// for ranges of at most kTeam32MaxBlocks blocks, else teams of 8 (or a block
// per thread); header errors are reported by the small class.
template <int EB>
__device__ __forceinline__ bool my_class(const DecArgs &a, const DecHdr &h)
{
    constexpr bool LARGE = EB > 1024;
    if (h.err) return a.small_launched ? !LARGE : LARGE;  // reported once
    const uint64_t blocks = a.ranged ? a.b1 - a.b0 : h.nb;
    return (h.N / 4 > 1024 || blocks <= kTeam32MaxBlocks) == LARGE;
}

// One array: CTAs stride over tiles of the requested block range.  Both
// size classes are enqueued; each decodes only the containers of its class.
template <int DT, int TS, int EB>
__global__ void __launch_bounds__(128) k_decode(DecArgs a)
{
    extern __shared__ uint8_t dsm[];
    __shared__ DecHdr s_h;
    if (threadIdx.x == 0) s_h = read_header(a);
    __syncthreads();
    const DecHdr hd = s_h;
    constexpr bool LARGE = EB > 1024;
    // the other size class's container: this launch has nothing to do (its
    // completion counter is only read by the class that owns the container)
    if (!my_class<EB>(a, hd)) return;
    {
        if (hd.err) {
            if (threadIdx.x == 0) set_status(a.status, hd.err);
        } else if (!LARGE && hd.N <= kT1MaxBlock &&
                   (a.ranged ? a.b1 - a.b0 : hd.nb) >= kT1MinBlocks) {
            // a block per thread, tiles of blockDim.x blocks.  A CTA's first
            // tile is its own index (the block scheduler spreads CTAs evenly
            // over the SMs; first-come tickets piled the tiles onto the SMs
            // whose CTAs started first); later tiles come from a counter
            // (blocks differ in cost, a static stride leaves a tail).
            const uint64_t jb = a.ranged ? a.b0 : 0, je = a.ranged ? a.b1 : hd.nb;
            const uint64_t per = blockDim.x;
            const uint64_t ntiles = (je - jb + per - 1) / per;
            __shared__ uint64_t s_tile;
            uint64_t tile = blockIdx.x;
            while (tile < ntiles) {
                const uint64_t j = jb + tile * per + threadIdx.x;
                if (j < je) decode_block_t1<DT>(a, hd, j, dsm + threadIdx.x, (int)blockDim.x);
                __syncthreads();
                if (threadIdx.x == 0) s_tile = gridDim.x + atomicAdd(a.ticket, 1ull);
                __syncthreads();
                tile = s_tile;
            }
        } else {
            const int nteams = blockDim.x / TS;
            const uint64_t jb = a.ranged ? a.b0 : 0, je = a.ranged ? a.b1 : hd.nb;
            const uint64_t ntiles = (je - jb + nteams - 1) / nteams;
            for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
                decode_tile<DT, TS, EB>(a, hd, tile, dsm);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned *done = LARGE ? a.done + 1 : a.done;
        const unsigned prev = atomicAdd(done, 1u);
        if (prev == gridDim.x - 1 && my_class<EB>(a, hd)) {
            __threadfence();
            volatile int *st = a.status;
            if (a.res) {
                a.res->bytes = a.ranged ? 0 : a.n;
                a.res->status = *st;
            }
        }
    }
}

template <int DT>
__device__ __noinline__ void decode_t1_call(const DecArgs &a, const DecHdr &hd, uint64_t j, uint8_t *eb,
                                            int est)
{
    decode_block_t1<DT>(a, hd, j, eb, est);
}

template <int DT, int TS, int EB>
__device__ __noinline__ void decode_tile_call(const DecArgs &a, const DecHdr &hd, uint64_t tile,
                                              uint8_t *dsm)
{
    decode_tile<DT, TS, EB>(a, hd, tile, dsm);
}

// Many arrays in one persistent launch: global tile tickets, owning array
// by binary search, per-array completion.  The plan sizes each array's tiles
// from its declared block size; a container whose header disagrees is
// reported as corrupt.
template <int TS, int EB>
__global__ void __launch_bounds__(128) k_decode_batch(DecBatchArgs ba)
{
    extern __shared__ uint8_t dsm[];
    __shared__ uint64_t s_tile;
    __shared__ int s_job;
    __shared__ __align__(16) DecArgs s_args;
    __shared__ DecHdr s_h;
    while (true) {
        if (threadIdx.x == 0) {
            const uint64_t g = atomicAdd(ba.ticket, 1ull);
            int lo = 0, hi = ba.count;
            if (g < ba.total_tiles) {
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (ba.tile_prefix[mid] <= g) lo = mid;
                    else hi = mid;
                }
                s_tile = g - ba.tile_prefix[lo];
            } else {
                s_tile = ~0ull;
            }
            s_job = lo;
        }
        __syncthreads();
        if (s_tile == ~0ull) break;
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(ba.jobs + s_job);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&s_args);
            for (int i = threadIdx.x; i < (int)(sizeof(DecArgs) / 4); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            DecHdr h = read_header(s_args);
            if (h.err == 0 && h.N != ba.block_size[s_job]) h.err = -9;
            s_h = h;
            if (h.err) set_status(s_args.status, h.err);
        }
        __syncthreads();
        const DecHdr hd = s_h;
        if (hd.err == 0 && ba.block_size[s_job] <= kT1MaxBlock) {
            // a block per thread: the plan made this array's tiles blockDim.x blocks
            const uint64_t j = s_tile * blockDim.x + threadIdx.x;
            if (j < hd.nb) {
                uint8_t *eb = dsm + threadIdx.x;
                switch (s_args.dtype) {
                case 1: decode_t1_call<1>(s_args, hd, j, eb, (int)blockDim.x); break;
                case 2: decode_t1_call<2>(s_args, hd, j, eb, (int)blockDim.x); break;
                case 3: decode_t1_call<3>(s_args, hd, j, eb, (int)blockDim.x); break;
                case 4: decode_t1_call<4>(s_args, hd, j, eb, (int)blockDim.x); break;
                default: decode_t1_call<5>(s_args, hd, j, eb, (int)blockDim.x); break;
                }
            }
        } else if (hd.err == 0) {
            switch (s_args.dtype) {
            case 1: decode_tile_call<1, TS, EB>(s_args, hd, s_tile, dsm); break;
            case 2: decode_tile_call<2, TS, EB>(s_args, hd, s_tile, dsm); break;
            case 3: decode_tile_call<3, TS, EB>(s_args, hd, s_tile, dsm); break;
            case 4: decode_tile_call<4, TS, EB>(s_args, hd, s_tile, dsm); break;
            default: decode_tile_call<5, TS, EB>(s_args, hd, s_tile, dsm); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(s_args.done, 1u);
            if (prev == ba.tiles_of[s_job] - 1) {
                __threadfence();
                volatile int *st = s_args.status;
                if (s_args.res) {
                    s_args.res->bytes = s_args.n;
                    s_args.res->status = *st;
                }
            }
        }
        __syncthreads();
    }
}

template <int DT, int TS, int EB>
static cudaError_t launch_one(const DecArgs &a, unsigned ctas, cudaStream_t s)
{
    constexpr int threads = 128;
    size_t smem = (size_t)(threads / TS) * EB;
    if (EB <= 1024 && smem < (size_t)threads * (kT1MaxBlock / 4)) smem = (size_t)threads * (kT1MaxBlock / 4);
    auto k = k_decode<DT, TS, EB>;
    const cudaError_t e = smem_limit<k_decode<DT, TS, EB>>(smem);
    if (e != cudaSuccess) return e;
    k<<<ctas, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t launch_dt(const DecArgs &a, cudaStream_t s)
{
    if (a.small_launched) {
        const cudaError_t e = launch_one<DT, 8, 1024>(a, a.nctas, s);
        if (e != cudaSuccess) return e;
    }
    return launch_one<DT, 32, 4096>(a, a.nctas_large, s);
}

}  // namespace

static size_t decode_batch_smem(int ts, int threads)
{
    const size_t teams = (size_t)(threads / ts) * (ts == 8 ? 1024 : 4096);
    const size_t cols = (size_t)threads * (kT1MaxBlock / 4);  // block-per-thread exponent columns
    return teams > cols ? teams : cols;
}

cudaError_t launch_decode_batch(const DecBatchArgs &b, int ts, int threads, unsigned ctas,
                               cudaStream_t s)
{
    const size_t smem = decode_batch_smem(ts, threads);
    auto k = ts == 8 ? k_decode_batch<8, 1024> : k_decode_batch<32, 4096>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ctas) k<<<ctas, threads, smem, s>>>(b);
    return cudaGetLastError();
}

int decode_batch_occupancy(int ts, int threads)
{
    const size_t smem = decode_batch_smem(ts, threads);
    auto k = ts == 8 ? k_decode_batch<8, 1024> : k_decode_batch<32, 4096>;
    int nb = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_decode(const DecArgs &a, cudaStream_t s)
{
    switch (a.dtype) {
    case 1: return launch_dt<1>(a, s);
    case 2: return launch_dt<2>(a, s);
    case 3: return launch_dt<3>(a, s);
    case 4: return launch_dt<4>(a, s);
    default: return launch_dt<5>(a, s);
    }
}

}  // namespace apax
