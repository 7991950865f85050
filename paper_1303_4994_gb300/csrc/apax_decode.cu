// apax_decode.cu -- block decoder (inverse of the Sec. 6 encoder).
//
// One warp decodes one block: header -> JEE tokens (parallel parse: the
// token/continuation state of every nibble comes from a warp scan of
// two-state transition functions) -> exponents (segmented scan of absolute
// values and diffs) -> mantissas (each lane unpacks its two groups) ->
// inverse derivatives (warp prefix sums mod 2^W) -> dequantisation with the
// reciprocal table, rounded once to the output type.  Warps stride over the
// blocks; fixed-rate packets sit at j*B, fixed-quality ones at the offset
// table's word offsets, so any block range can be decoded on its own.
#include "apax_device.cuh"
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
        if (i >= nwords) { oob = true; return 0; }
        return __ldg(w + i);
    }
    // 16 bits starting at bit b
    __device__ __forceinline__ uint32_t bits16(uint32_t b, bool &oob) const
    {
        uint32_t i = b >> 5, sh = b & 31;
        uint64_t v = get(i, oob);
        if (sh > 16) v |= (uint64_t)get(i + 1, oob) << 32;
        return (uint32_t)(v >> sh) & 0xffffu;
    }
};

// Composition of two-state functions coded as 2 bits: bit s = image of s
// (state 0: token start, state 1: continuation of an absolute token).
__device__ __forceinline__ uint32_t fcomp(uint32_t f, uint32_t g)  // g after f
{
    uint32_t i0 = (g >> (f & 1)) & 1, i1 = (g >> ((f >> 1) & 1)) & 1;
    return i0 | (i1 << 1);
}
__device__ __forceinline__ uint32_t nib_fn(uint32_t nib)
{
    // start -> continuation for an escape nibble (14, 15); continuation -> start
    return nib >= 14 ? 1u : 0u;  // image(start) = nib>=14, image(cont) = start (0)
}

// Parse the JEE token section: fills ebuf with the G exponents, returns the
// nibble count or -1 for a malformed section.
__device__ int parse_tokens(const PktReader &pr, int H, int G, int W, uint8_t *ebuf)
{
    // Nibbles read past the packet inside a window are zero and harmless:
    // the caller checks that the consumed section and the mantissas fit.
    bool oob = false;
    const int l = (int)lane_id();
    int done_g = 0;
    int tpos = 0;  // nibbles consumed
    bool bad = false;
    // entries: 0x80|v absolute (v in 0..31), 8+d diff
    while (done_g < G) {
        // lane's 4 nibbles of this window of 128
        const uint32_t b = (uint32_t)H + 4u * (uint32_t)(tpos + 4 * l);
        const uint32_t v16 = pr.bits16(b, oob);
        uint32_t nb[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) nb[t] = (v16 >> (4 * t)) & 15u;
        // composed lane function
        uint32_t F = 2u;  // identity: image(0)=0, image(1)=1
#pragma unroll
        for (int t = 0; t < 4; ++t) F = fcomp(F, nib_fn(nb[t]));
        // exclusive scan of functions across lanes
        uint32_t inc = F;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t o = __shfl_up_sync(kFull, inc, d);
            if (l >= d) inc = fcomp(o, inc);
        }
        uint32_t exc = __shfl_up_sync(kFull, inc, 1);
        if (l == 0) exc = 2u;
        uint32_t state = exc & 1;  // image of "start" at the window start
        const uint32_t next_first = __shfl_down_sync(kFull, nb[0], 1);
        int gcnt[4], tlen[4];
        bool start[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            start[t] = state == 0;
            tlen[t] = start[t] ? (nb[t] >= 14 ? 2 : 1) : 0;
            gcnt[t] = start[t] ? (nb[t] <= 8 ? 2 : 1) : 0;
            state = state == 0 ? (nb[t] >= 14 ? 1u : 0u) : 0u;
        }
        // a token is complete if its last nibble is inside the window
        const int wpos0 = 4 * l;
        bool complete[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) complete[t] = start[t] && (wpos0 + t + tlen[t] <= 128);
        // groups before each token: exclusive scan (complete tokens only)
        int lg = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) lg += complete[t] ? gcnt[t] : 0;
        int incl = warp_incl_scan(lg);
        int gpos = done_g + incl - lg;
        // first incomplete token start (window position) bounds consumption
        int first_inc = 128;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (start[t] && !complete[t]) first_inc = min(first_inc, wpos0 + t);
        first_inc = __reduce_min_sync(kFull, first_inc);
        int used_end = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int wp = wpos0 + t;
            if (complete[t] && wp < first_inc && gpos < G) {
                const uint32_t a = nb[t];
                if (a >= 14) {
                    const uint32_t lo = t < 3 ? nb[t + 1] : next_first;
                    const uint32_t v = ((a - 14) << 4) | lo;
                    ebuf[gpos] = (uint8_t)(0x80u | v);
                } else if (gpos == 0) {
                    bad = true;
                } else if (a <= 8) {
                    if (gpos + 1 >= G) bad = true;
                    else {
                        ebuf[gpos] = (uint8_t)(8 + (int)(a / 3) - 1);
                        ebuf[gpos + 1] = (uint8_t)(8 + (int)(a % 3) - 1);
                    }
                } else {
                    ebuf[gpos] = (uint8_t)(8 + (int)a - 11);
                }
                used_end = max(used_end, wp + tlen[t]);
            }
            gpos += (complete[t] && wp < first_inc) ? gcnt[t] : 0;
        }
        used_end = __reduce_max_sync(kFull, used_end);
        // every complete token precedes the first incomplete one (an escape
        // nibble in the window's last position), so the scan total counts
        // exactly the groups this window can supply
        const int gained = min(__shfl_sync(kFull, incl, 31), G - done_g);
        if (gained <= 0 || used_end == 0) { bad = true; break; }
        done_g += gained;
        tpos += used_end;
        if (__any_sync(kFull, bad)) break;
    }
    bad = __any_sync(kFull, bad);
    __syncwarp();
    if (bad) return -1;
    // resolve entries into exponents: segmented scan over groups
    int carry_e = 0;
    bool anybad = false;
    for (int base = 0; base < G; base += 64) {
        const int g0 = base + 2 * l, g1 = g0 + 1;
        const uint32_t a0 = g0 < G ? ebuf[g0] : 8u, a1 = g1 < G ? ebuf[g1] : 8u;
        // (is_abs, value) pairs; combine lane's two entries
        bool f0 = a0 & 0x80, f1 = a1 & 0x80;
        int v0 = f0 ? (int)(a0 & 31) : (int)a0 - 8, v1 = f1 ? (int)(a1 & 31) : (int)a1 - 8;
        if (f0 && v0 == 31) v0 = 32;
        if (f1 && v1 == 31) v1 = 32;
        bool F = f0 || f1;
        int V = f1 ? v1 : v0 + v1;
        // inclusive segmented scan across lanes
        bool sF = F;
        int sV = V;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            bool oF = __shfl_up_sync(kFull, sF, d);
            int oV = __shfl_up_sync(kFull, sV, d);
            if (l >= d) {
                if (!sF) sV += oV;
                sF = sF || oF;
            }
        }
        bool xF = __shfl_up_sync(kFull, sF, 1);
        int xV = __shfl_up_sync(kFull, sV, 1);
        if (l == 0) { xF = false; xV = 0; }
        const int before = xF ? xV : carry_e + xV;  // exponent of group g0-1
        const int e0 = f0 ? v0 : before + v0;
        const int e1 = f1 ? v1 : e0 + v1;
        const int lim = W >= 32 ? 32 : W;
        if (g0 < G) {
            anybad |= e0 < 0 || e0 > lim || e0 == 31;
            ebuf[g0] = (uint8_t)e0;
        }
        if (g1 < G) {
            anybad |= e1 < 0 || e1 > lim || e1 == 31;
            ebuf[g1] = (uint8_t)e1;
        }
        const int lastg = min(G - base, 64) - 1;
        carry_e = __shfl_sync(kFull, (lastg & 1) ? e1 : e0, lastg >> 1);
    }
    __syncwarp();
    if (__any_sync(kFull, anybad)) return -1;
    return tpos;
}

template <int DT>
__device__ __forceinline__ void store_lane(typename DT_<DT>::raw *y, int i0, int L,
                                           const typename LaneT<DT>::t (&v)[8])
{
    using raw = typename DT_<DT>::raw;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (i0 + t < L) {
            if constexpr (DT_<DT>::F) {
                using B = typename DT_<DT>::bits;
                reinterpret_cast<B *>(y)[i0 + t] = v[t];
            } else {
                y[i0 + t] = (raw)v[t];
            }
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(256) k_decode(DecArgs a)
{
    extern __shared__ uint8_t dsm[];
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    constexpr int W = T::W, H = T::H;
    const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
    uint8_t *ebuf = dsm + (size_t)wid * 4096;

    // container header (checked by every warp)
    const uint8_t *in = a.in;
    bool ok = in && a.in_bytes >= 40 && in[0] == 'A' && in[1] == 'P' && in[2] == 'X' && in[3] == '1' &&
              in[4] == 1;
    int err = -9;
    uint32_t N = 0, B = 0;
    uint64_t n = 0, payload = 0, poff = 0, nb = 0;
    int mode = 0;
    if (ok) {
        auto le = [&](int o, int k) {
            uint64_t v = 0;
            for (int i = 0; i < k; ++i) v |= (uint64_t)in[o + i] << (8 * i);
            return v;
        };
        mode = in[6];
        N = (uint32_t)le(8, 4);
        B = (uint32_t)le(16, 4);
        n = le(20, 8);
        payload = le(28, 8);
        if (in[5] != a.dtype || n != a.n) { ok = false; err = -1; }
        else if (N < 64 || N > 16384 || (N & 3) || (mode != 0 && mode != 1)) ok = false;
        else {
            nb = (n + N - 1) / N;
            poff = 40 + (mode == 1 ? ((4 * nb + 7) / 8) * 8 : 0);
            if (poff > a.in_bytes || payload > a.in_bytes - poff) ok = false;
            if (mode == 0 && ((B & 3) || B == 0)) ok = false;
            if (a.ranged && (a.b1 > nb || a.b0 > a.b1)) { ok = false; err = -1; }
        }
    }
    if (!ok) {
        if (l == 0) set_status(a.status, err);
    } else {
        const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wid;
        const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
        const uint32_t *tab = reinterpret_cast<const uint32_t *>(in + 40);
        const uint64_t jb = a.ranged ? a.b0 : 0, je = a.ranged ? a.b1 : nb;
        for (uint64_t j = jb + gw; j < je; j += nw) {
            const uint64_t start = mode == 1 ? 4ull * (uint64_t)__ldg(tab + j) : j * (uint64_t)B;
            const uint64_t off = j * (uint64_t)N;
            const int L = (int)((n - off) < N ? (n - off) : N);
            const int G = (L + 3) >> 2;
            bool bad = start >= payload || (start & 3);
            PktReader pr;
            pr.w = reinterpret_cast<const uint32_t *>(in + poff + (bad ? 0 : start));
            uint64_t availw = bad ? 0 : (payload - start) >> 2;
            pr.nwords = (uint32_t)(availw > 0xffffffffull ? 0xffffffffull : availw);
            bool oob = false;
            const uint32_t h0 = pr.get(0, oob);
            const int s = h0 & 3, code = (h0 >> 2) & 4095;
            const uint32_t plen = h0 >> 14;
            bad |= oob || s == 3 || plen < 4 || (plen & 3) || (uint64_t)plen > 4ull * pr.nwords;
            if (mode == 0 && j + 1 < nb && plen != B) bad = true;
            int Eb = 0;
            if (!bad) {
                pr.nwords = plen >> 2;
                if (T::F) Eb = (int)(int16_t)(pr.get(1, oob) & 0xffffu);
            }
            int nib = -1;
            if (!bad) nib = parse_tokens(pr, H, G, W, ebuf);
            if (nib < 0) bad = true;
            if (bad) {
                if (l == 0) set_status(a.status, -9);
                continue;
            }
            const Code c(code);
            const uint32_t R = recip_entry(c.m);
            raw *yb = reinterpret_cast<raw *>(a.y) + (a.ranged ? (j - a.b0) * (uint64_t)N : off);
            uint32_t mbit = (uint32_t)H + 4u * (uint32_t)nib;
            uint32_t P = 0, Qs = 0, u0 = 0;  // running prefix sums (mod 2^32), first value
            const int nch = (L + kChunk - 1) / kChunk;
            for (int ch = 0; ch < nch; ++ch) {
                const int g0 = ch * 64 + 2 * l;
                const int e0 = g0 < G ? ebuf[g0] : 0, e1 = g0 + 1 < G ? ebuf[g0 + 1] : 0;
                const int w4 = 4 * (e0 + e1);
                const int incl = warp_incl_scan(w4);
                uint32_t bit = mbit + (uint32_t)(incl - w4);
                // unpack 8 values
                int32_t u[8];
                {
                    uint32_t wi = bit >> 5;
                    uint32_t sh = bit & 31;
                    uint64_t acc = 0;
                    int fill = 0;
                    if (w4) {
                        acc = (uint64_t)pr.get(wi, oob) >> sh;
                        fill = 32 - (int)sh;
                    }
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const int e = t < 4 ? e0 : e1;
                        if (e == 0) { u[t] = 0; continue; }
                        if (fill < e) {
                            acc |= (uint64_t)pr.get(++wi, oob) << fill;
                            fill += 32;
                        }
                        uint32_t v = (uint32_t)acc & (e >= 32 ? 0xffffffffu : ((1u << e) - 1));
                        acc >>= e;
                        fill -= e;
                        u[t] = e >= 32 ? (int32_t)v : ((int32_t)(v << (32 - e)) >> (32 - e));
                    }
                }
                mbit += (uint32_t)__shfl_sync(kFull, incl, 31);
                // inverse streams mod 2^32 (reduced to W bits at the end)
                uint32_t q[8];
                if (s == 0) {
#pragma unroll
                    for (int t = 0; t < 8; ++t) q[t] = (uint32_t)u[t];
                } else {
                    if (ch == 0) u0 = __shfl_sync(kFull, (uint32_t)u[0], 0);
                    uint32_t pl[8], acc = 0;
#pragma unroll
                    for (int t = 0; t < 8; ++t) { acc += (uint32_t)u[t]; pl[t] = acc; }
                    uint32_t li = warp_incl_scan(acc);
                    uint32_t ex = P + li - acc;
                    P += __shfl_sync(kFull, li, 31);
                    if (s == 1) {
#pragma unroll
                        for (int t = 0; t < 8; ++t) q[t] = ex + pl[t];
                    } else {
                        // v_i = P_i - u_0 for i >= 1, v_0 = u_0; q = prefix of v
                        uint32_t vv[8], a2 = 0;
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const bool first = ch == 0 && l == 0 && t == 0;
                            vv[t] = first ? u0 : (ex + pl[t] - u0);
                            a2 += vv[t];
                            vv[t] = a2;
                        }
                        uint32_t li2 = warp_incl_scan(a2);
                        uint32_t ex2 = Qs + li2 - a2;
                        Qs += __shfl_sync(kFull, li2, 31);
#pragma unroll
                        for (int t = 0; t < 8; ++t) q[t] = ex2 + vv[t];
                    }
                }
                // dequantise (Sec. 6 attenuator inverse with the reciprocal table)
                lt out[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int32_t qi = sext_w(q[t], W);
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
                        out[t] = (lt)yv;
                    } else {
                        out[t] = (c.zero || qi == 0)
                                     ? (lt)0
                                     : round_to_format<DT>((int64_t)qi * (int64_t)R, Eb - T::Q + c.k - 24);
                    }
                }
                if (__any_sync(kFull, oob)) {
                    if (l == 0) set_status(a.status, -9);
                    break;
                }
                store_lane<DT>(yb, ch * kChunk + 8 * l, L, out);
            }
            const uint32_t endbit = mbit;
            if (endbit > 8u * plen && l == 0) set_status(a.status, -9);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(a.done, 1u);
        if (prev == a.nctas - 1) {
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
static cudaError_t launch_dt(const DecArgs &a, int wpc, cudaStream_t s)
{
    const size_t smem = (size_t)wpc * 4096;
    auto k = k_decode<DT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<a.nctas, 32 * wpc, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decode(const DecArgs &a, int wpc, cudaStream_t s)
{
    switch (a.dtype) {
    case 1: return launch_dt<1>(a, wpc, s);
    case 2: return launch_dt<2>(a, wpc, s);
    case 3: return launch_dt<3>(a, wpc, s);
    case 4: return launch_dt<4>(a, wpc, s);
    default: return launch_dt<5>(a, wpc, s);
    }
}

}  // namespace apax
