// apax_encode.cu -- block encoder kernels (Sec. 6 encoder and bit packer).
//
// A team of TS threads encodes one block; a CTA's teams form one tile of
// consecutive blocks.  Each team
//   1. decides its stream from the predecessor block at code 0 (the
//      one-block lag of Sec. 6: block j+1 carries block j's best stream),
//   2. picks the attenuation code (fixed quality: given; fixed rate: the
//      BISECT or PREDICT search against the block budget),
//   3. writes exponents, JEE tokens and mantissas into a shared-memory
//      packet image, which is then copied out with coalesced word stores.
// Fixed-rate packets land at j*B.  Fixed-quality packet offsets come from a
// device-wide exclusive scan over tiles with decoupled look-back (Merrill &
// Garland 2016): tiles take tickets in launch order, publish their word
// count, and walk back over predecessors with a bounded spin.
#include "apax_team.cuh"
#include "apax_kernels.h"
#include "apax_encode.cuh"

namespace apax {

// ---------------------------------------------------------------- tile body
// One tile (nteams consecutive blocks) of the array described by `a`.
// Called by every thread of the CTA; `smem` holds the teams' packet images.
// INL: the tile sizes the sum stream itself for the stream decision (the
// batched kernels); single-array kernels read a.sel instead, which keeps
// the sizing's registers out of them.
template <int DT, int TS, int MODE, bool INL>
__device__ __forceinline__ void encode_tile(const EncArgs &a, uint64_t tile, uint32_t *smem)
{
    __shared__ uint32_t s_words[32];
    __shared__ uint32_t s_total;
    __shared__ uint64_t s_base;
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    constexpr int H = T::H;
    const int team = threadIdx.x / TS, t = tlane<TS>();
    const int nteams = blockDim.x / TS;
    const int gp = a.gp;

    // block j of the array; jl = j - jb0 its place in this container
    const uint64_t j = a.jb0 + tile * (uint64_t)nteams + (uint64_t)team;
    const uint64_t jl = j - a.jb0, nbl = a.nb - a.jb0;
    int code = (int)a.code;
    if (a.code_dev) code = (int)*a.code_dev;
    uint32_t *pkt = smem + (size_t)team * (a.pkt_words + a.ebuf_words);
    uint8_t *ebuf = reinterpret_cast<uint8_t *>(pkt + a.pkt_words);
    if (tile == 0 && threadIdx.x == 0) write_container_header(a, code);

    const raw *x = reinterpret_cast<const raw *>(a.x);
    // the tile's blocks and the one before it (the lag decision's halo) in
    // shared memory, when the plan has room for them
    uint64_t base = 0;
    if (a.stage_off) {
        raw *xs = reinterpret_cast<raw *>(reinterpret_cast<uint8_t *>(smem) + a.stage_off);
        const uint64_t jb0 = a.jb0 + tile * (uint64_t)nteams;
        base = jb0 ? jb0 - 1 : 0;
        const uint64_t bend = min(jb0 + (uint64_t)nteams, a.nb);
        if (stage_blocks<DT>(xs, x, a.n, a.N, base, bend > base ? bend : base, a.status, a.spin_limit))
            x = xs;  // else (a wait ran out) read the blocks from global memory
        else
            base = 0;
        __syncthreads();
    }
    // stream decision: best(j-1) at code 0 (block 0 uses its own)
    int s;
    if (!INL && a.sel) {
        s = jl < nbl ? a.sel[jl] : 0;
    } else {
        TBlock<DT> pv;
        open_team_block<DT, TS>(pv, x, a.n, a.N, a.nb, j == 0 ? 0 : j - 1, gp, base, a.gsh);
        s = team_best_stream<DT, TS>(pv, INL && a.sum != 0);
    }
    TBlock<DT> b;
    open_team_block<DT, TS>(b, x, a.n, a.N, a.nb, j, gp, base, a.gsh);
    const int gsh = b.gsh;
    if (b.active && b.bad && t == 0) set_status(a.status, -8);
    uint32_t plen = 0;
    if (MODE == 0) {
        const uint32_t budget = b.L == (int)a.N ? a.B : fr_budget<DT>(b.L, a.rate_num, a.rate_den, gsh);
        if (a.search == APAX_SEARCH_PREDICT) {
            // the code-0 exponents of stream s into ebuf, the packet bits
            const uint32_t bits0 = team_exps<DT, TS>(b, s, ebuf);
            __syncwarp();
            const bool fits0 = pad32_bytes(bits0) <= budget;
            // every team of the warp steps through the same loops (their
            // shuffles are shared); a team that is done follows along
            const int D = (int)bits0 - 8 * (int)budget;
            const int ge = b.active ? b.g1 : b.g0;
            // red(k) for k = 1, 2, ... until every team of the warp has its k1
            // (a group of 4 << gsh samples loses that many bits per unit of k)
            int rprev = 0, rk = 0, k1 = 0;
#pragma unroll 1
            for (int k = 1; k <= 31 && __any_sync(kFull, !fits0 && k1 == 0); ++k) {
                int cnt = 0;
                for (int g = b.g0 >> gsh; g < (ge >> gsh); ++g) cnt += ebuf[g] >= k;
                cnt = team_sum<TS>(cnt);
                if (k1 == 0) {
                    rk = rprev + (4 << gsh) * cnt;
                    if (rk >= D) k1 = k;
                    else if (k < 31) rprev = rk;
                }
            }
            int c = predict_from_red(D, k1 ? k1 : 31, rprev, rk);
            bool need = !fits0 && c < 4095;
#pragma unroll 1
            while (__any_sync(kFull, need)) {
                const uint32_t bm = team_eval1<DT, TS>(b, need ? c : 0, s);
                if (need) {
                    if (pad32_bytes(bm) <= budget) need = false;
                    else c = ladder_next(c);
                    need = need && c < 4095;
                }
            }
            code = fits0 ? 0 : c;
        } else {
            const bool fits0 = pad32_bytes(team_eval1<DT, TS>(b, 0, s)) <= budget;
            int lo = 0, hi = 4095;
            // Teams of one warp share shuffles, so every team runs the same 12
            // halvings unless all of them already fit at code 0.
            if (!__all_sync(kFull, fits0)) {
#pragma unroll 1
                for (int it = 0; it < 12; ++it) {  // at most 12 halvings close [0, 4095]
                    const int mid = (lo + hi) >> 1;
                    const uint32_t bm = team_eval1<DT, TS>(b, mid, s);
                    if (hi - lo > 1) {
                        if (pad32_bytes(bm) <= budget) hi = mid;
                        else lo = mid;
                    }
                }
            }
            code = fits0 ? 0 : hi;
        }
        plen = budget;
    }

    // final pass: the chosen stream's exponents into ebuf (one per BFPE
    // group: ebuf[g >> gsh] for the groups of 4 g), token counts
    const Quant<DT> Q(code, b.Eb);
    TokCount tc;
    tc.init();
    with_quant<DT>(Q, [&](const auto &qf) {
        Stream1 st(s, carry_in<DT>(b, qf, 4 * b.g0));
        uint32_t acc = 0;
#pragma unroll 1
        for (int g = b.g0; g < b.g1; ++g) {
            lt xv[4];
            load4<DT, true>(b, 4 * g, xv);
            int32_t u[4];
            acc |= group1<DT>(qf, xv, st, u);
            if (!gsh || (g & 1)) {
                const int e = exp_from_or(acc);
                ebuf[g >> gsh] = (uint8_t)e;
                tc.push(e, true);
                acc = 0;
            }
        }
    });
    int nib_total, sume_total, nib_mine;
    bool s_in;
    team_tokens<TS>(tc, b.g0 == 0, nib_total, sume_total, &s_in, &nib_mine);
    const uint32_t wm = 4u << gsh;  // mantissa bits per exponent unit
    const uint32_t bits = (uint32_t)H + 4u * (uint32_t)nib_total + wm * (uint32_t)sume_total;
    if (MODE == 1) plen = pad32_bytes(bits);
    const uint32_t words = b.active ? plen >> 2 : 0;
    if (MODE == 1) {
        // the tile's size is known: scan it and publish the aggregate now,
        // so that successors' look-backs find it while this tile assembles
        if (t == 0) s_words[team] = words;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            const uint32_t v = l < nteams ? s_words[l] : 0;
            const uint32_t incl = warp_incl_scan(v);
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            __syncwarp();
            if (l < nteams) s_words[l] = incl - v;
            if (l == 0) {
                s_total = total;
                publish_aggregate(a, tile, total);
            }
        }
    }
    for (uint32_t w = t; w < words; w += TS) pkt[w] = 0;
    __syncwarp();
    // team scans before any divergence: every lane of the warp takes part
    const int nib_before = team_incl_scan<TS>(nib_mine) - nib_mine;
    const int sume_before = team_incl_scan<TS>(tc.sume) - tc.sume;
    if (b.active) {
        if (t == 0) {
            atomicOr(&pkt[0], (uint32_t)s | ((uint32_t)code << 2) | (plen << 14));
            if (H == 48) atomicOr(&pkt[1], (uint32_t)(uint16_t)(int16_t)b.Eb);
        }
        // tokens of my groups (Sec. 6 JEE), starting at my nibble offset
        NibWriter nw;
        nw.start(pkt, (uint32_t)H + 4u * (uint32_t)nib_before);
        write_tokens(nw, ebuf, 1, b.g0 >> gsh, b.g1 >> gsh, b.G >> gsh, s_in);
        nw.flush();
        // mantissas of my groups after the token section (a group of 8 is
        // two groups of 4 of its one width)
        NibWriter mw;
        mw.start(pkt, (uint32_t)H + 4u * (uint32_t)nib_total + wm * (uint32_t)sume_before);
        with_quant<DT>(Q, [&](const auto &qf) {
            Stream1 sm(s, carry_in<DT>(b, qf, 4 * b.g0));
#pragma unroll 1
            for (int g = b.g0; g < b.g1; ++g) {
                lt xv[4];
                load4<DT, true>(b, 4 * g, xv);
                int32_t u[4];
                group1<DT>(qf, xv, sm, u);
                write_group_fields(mw, ebuf[g >> gsh], u);
            }
        });
        mw.flush();
    }
    __syncthreads();

    uint64_t off_words;  // packet start in payload words
    if (MODE == 1) {
        if (threadIdx.x < 32) {
            const uint64_t excl = lookback_prefix(a, tile, s_total);
            if (threadIdx.x == 0) s_base = excl;
        }
        __syncthreads();
        off_words = s_base + s_words[team];
    } else {
        off_words = jl * (uint64_t)(a.B >> 2);
    }

    if (b.active) {
        const uint64_t start = a.poff + 4ull * off_words;
        if (MODE == 1 && t == 0) {
            if (off_words > 0xffffffffull) {
                set_status(a.status, -6);
            } else {
                reinterpret_cast<uint32_t *>(a.out + 40)[jl] = (uint32_t)off_words;
                if (jl == nbl - 1 && (nbl & 1)) reinterpret_cast<uint32_t *>(a.out + 40)[jl + 1] = 0;
            }
        }
        if (start + 4ull * words > a.cap) {
            if (t == 0) set_status(a.status, -5);
        } else {
            uint32_t *dst = reinterpret_cast<uint32_t *>(a.out + start);
            for (uint32_t w = t; w < words; w += TS) dst[w] = pkt[w];
        }
    }

    // completion: the CTA that finishes the array's last tile writes the
    // payload size and the result
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(a.done, 1u);
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

// Does block b fit `budget` bytes at `code` on stream s (one thread owns the
// block)?  The running packet size -- header, the first absolute token, the
// nibbles and exponent bits so far -- only grows, so a pass stops as soon as
// it exceeds the budget: the answer is the same as from the full size.
template <int DT>
__device__ __forceinline__ bool fits_t1(const TBlock<DT> &b, int code, int s, uint32_t budget)
{
    constexpr int H = DT_<DT>::H;
    const Quant<DT> Q(code, b.Eb);
    // the greedy JEE count of one whole block in one thread: the first
    // exponent is absolute (2 nibbles), then the TokCount transitions
    int nib = 0, sume = 0, e_last = 0;
    bool st = false;
    const uint32_t limit = 8u * budget;  // bits; budget is a multiple of 4 bytes
    bool over = false;
    with_quant<DT>(Q, [&](const auto &qf) {
        Stream1 sm(s, carry_in<DT>(b, qf, 0));
#pragma unroll 1
        for (int g = 0; g < b.G; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT, true>(b, 4 * g, xv);
            int32_t u[4];
            const int e = exp_from_or(group1<DT>(qf, xv, sm, u));
            const int d = e - e_last;
            const bool small = (unsigned)(d + 1) <= 2u;
            const int inc = small ? (st ? 0 : 1) : ((unsigned)(d + 2) <= 4u ? 1 : 2);
            nib += g == 0 ? 2 : inc;
            st = g != 0 && small && !st;
            sume += e;
            e_last = e;
            if ((g & 7) == 7 && (uint32_t)H + 4u * (uint32_t)nib + 4u * (uint32_t)sume > limit) {
                over = true;
                break;
            }
        }
    });
    if (over) return false;
    return pad32_bytes((uint32_t)H + 4u * (uint32_t)nib + 4u * (uint32_t)sume) <= budget;
}

// Exponents of block b at code 0 on stream s into the column eb (stride
// nt), and the unpadded packet bits (one thread owns the block).
template <int DT>
__device__ __forceinline__ uint32_t exps_t1(const TBlock<DT> &b, int s, uint8_t *eb, int nt)
{
    constexpr int H = DT_<DT>::H;
    const Quant<DT> Q(0, b.Eb);
    int nib = 0, sume = 0, e_last = 0;
    bool st = false;
    with_quant<DT>(Q, [&](const auto &qf) {
        Stream1 sm(s, carry_in<DT>(b, qf, 0));
#pragma unroll 1
        for (int g = 0; g < b.G; ++g) {
            typename LaneT<DT>::t xv[4];
            load4<DT, true>(b, 4 * g, xv);
            int32_t u[4];
            const int e = exp_from_or(group1<DT>(qf, xv, sm, u));
            eb[(size_t)g * nt] = (uint8_t)e;
            const int d = e - e_last;
            const bool small = (unsigned)(d + 1) <= 2u;
            const int inc = small ? (st ? 0 : 1) : ((unsigned)(d + 2) <= 4u ? 1 : 2);
            nib += g == 0 ? 2 : inc;
            st = g != 0 && small && !st;
            sume += e;
            e_last = e;
        }
    });
    return (uint32_t)H + 4u * (uint32_t)nib + 4u * (uint32_t)sume;
}

// ---------------------------------------------------------------- block per thread
// Fixed rate, a tile of blockDim.x blocks, one per thread (block sizes up to
// kT1MaxBlock): the team functions run with a team of one, exponents sit in
// a lane-interleaved shared-memory column (smem bytes g * blockDim.x +
// thread), and each thread writes its own packet straight to its place j*B.

template <int DT>
__device__ __forceinline__ void encode_tile_t1(const EncArgs &a, uint64_t tile, uint8_t *smem)
{
    using T = DT_<DT>;
    using raw = typename T::raw;
    using lt = typename LaneT<DT>::t;
    constexpr int H = T::H;
    const int tid = threadIdx.x, nt = blockDim.x;
    const uint64_t j = a.jb0 + tile * (uint64_t)nt + (uint64_t)tid;  // block of the array
    uint8_t *eb = smem + tid;  // exponent of group g at eb[g * nt]
    if (tile == 0 && tid == 0) write_container_header(a, 0);
    const raw *x = reinterpret_cast<const raw *>(a.x);
    // stream decision: best(j-1) at code 0 (block 0 uses its own)
    int s;
    {
        TBlock<DT> pv;
        open_team_block<DT, 1>(pv, x, a.n, a.N, a.nb, j == 0 ? 0 : j - 1, a.gp);
        s = team_best_stream<DT, 1>(pv, false);  // version-1 containers only
    }
    TBlock<DT> b;
    open_team_block<DT, 1>(b, x, a.n, a.N, a.nb, j, a.gp);
    if (b.active && b.bad) set_status(a.status, -8);
    // the search against the block budget (Sec. 6 adaptive loop)
    const uint32_t budget = b.L == (int)a.N ? a.B : fr_budget<DT>(b.L, a.rate_num, a.rate_den, 0);
    int code = 0;
    if (a.search == APAX_SEARCH_PREDICT) {
        // the code-0 exponents of stream s into the column, the packet bits
        const uint32_t bits0 = exps_t1<DT>(b, s, eb, nt);
        if (pad32_bytes(bits0) > budget) {
            int c = predict_start((int)bits0 - 8 * (int)budget, [&](int k) {
                int cnt = 0;
                for (int g = 0; g < b.G; ++g) cnt += eb[(size_t)g * nt] >= k;
                return cnt;
            });
            while (c < 4095 && !fits_t1<DT>(b, c, s, budget)) c = ladder_next(c);
            code = c;
        }
    } else {
        const bool fits0 = fits_t1<DT>(b, 0, s, budget);
        int lo = 0, hi = 4095;
        if (!fits0) {
#pragma unroll 1
            for (int it = 0; it < 12 && hi - lo > 1; ++it) {  // 12 halvings close [0, 4095]
                const int mid = (lo + hi) >> 1;
                if (fits_t1<DT>(b, mid, s, budget)) hi = mid;
                else lo = mid;
            }
        }
        code = fits0 ? 0 : hi;
    }
    const uint32_t plen = budget;
    // final pass: exponents into the column
    const Quant<DT> Q(code, b.Eb);
    with_quant<DT>(Q, [&](const auto &qf) {
        Stream1 st(s, carry_in<DT>(b, qf, 0));
#pragma unroll 1
        for (int g = 0; g < b.G; ++g) {
            lt xv[4];
            load4<DT, true>(b, 4 * g, xv);
            int32_t u[4];
            eb[(size_t)g * nt] = (uint8_t)exp_from_or(group1<DT>(qf, xv, st, u));
        }
    });
    const uint32_t words = b.active ? plen >> 2 : 0;
    if (b.active) {
        const uint64_t start = a.poff + (j - a.jb0) * a.B;
        if (start + 4ull * words > a.cap) {
            set_status(a.status, -5);
        } else {
            GWriter w;
            w.start(reinterpret_cast<uint32_t *>(a.out + start));
            w.put((uint32_t)s | ((uint32_t)code << 2) | (plen << 14), 32);
            if (H == 48) w.put((uint32_t)(uint16_t)(int16_t)b.Eb, 16);
            write_tokens(w, eb, nt, 0, b.G, b.G, false);
            with_quant<DT>(Q, [&](const auto &qf) {
                Stream1 sm(s, carry_in<DT>(b, qf, 0));
#pragma unroll 1
                for (int g = 0; g < b.G; ++g) {
                    lt xv[4];
                    load4<DT, true>(b, 4 * g, xv);
                    int32_t u[4];
                    group1<DT>(qf, xv, sm, u);
                    write_group_fields(w, eb[(size_t)g * nt], u);
                }
            });
            w.flush();
            while (w.w < words) w.dst[w.w++] = 0u;  // padding to the budget
        }
    }

    // completion: the CTA that finishes the array's last tile writes the
    // payload size and the result
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(a.done, 1u);
        if (prev == a.ntiles - 1) {
            __threadfence();
            put_le(a.out + 28, a.fr_payload, 8);
            volatile int *st = a.status;
            if (a.res) {
                a.res->bytes = a.poff + a.fr_payload;
                a.res->status = *st;
            }
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(128) k_encode_t1(EncArgs a)
{
    extern __shared__ uint32_t smem[];
    encode_tile_t1<DT>(a, blockIdx.x, reinterpret_cast<uint8_t *>(smem));
}

// ---------------------------------------------------------------- kernels
// One array: fixed quality takes tiles by ticket (launch order, which the
// look-back relies on), fixed rate by CTA index.
template <int DT, int TS, int MODE>
__global__ void __launch_bounds__(128) k_encode(EncArgs a)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint64_t s_tile;
    if (threadIdx.x == 0) s_tile = MODE == 1 ? (uint64_t)atomicAdd(a.ticket, 1u) : blockIdx.x;
    __syncthreads();
    encode_tile<DT, TS, MODE, false>(a, s_tile, smem);
}

template <int DT, int TS, int MODE>
__device__ __noinline__ void encode_tile_call(const EncArgs &a, uint64_t tile, uint32_t *smem)
{
    encode_tile<DT, TS, MODE, true>(a, tile, smem);
}

template <int DT>
__device__ __noinline__ void encode_tile_t1_call(const EncArgs &a, uint64_t tile, uint32_t *smem)
{
    encode_tile_t1<DT>(a, tile, reinterpret_cast<uint8_t *>(smem));
}

template <int TS>
__device__ __forceinline__ void encode_tile_any(const EncArgs &a, uint64_t tile, uint32_t *smem)
{
    if (a.t1) {  // fixed rate, a block per thread
        switch (a.dtype) {
        case 1: encode_tile_t1_call<1>(a, tile, smem); break;
        case 2: encode_tile_t1_call<2>(a, tile, smem); break;
        case 3: encode_tile_t1_call<3>(a, tile, smem); break;
        case 4: encode_tile_t1_call<4>(a, tile, smem); break;
        default: encode_tile_t1_call<5>(a, tile, smem); break;
        }
        return;
    }
    const int k = 2 * a.dtype + a.mode;
    switch (k) {
    case 2: encode_tile_call<1, TS, 0>(a, tile, smem); break;
    case 3: encode_tile_call<1, TS, 1>(a, tile, smem); break;
    case 4: encode_tile_call<2, TS, 0>(a, tile, smem); break;
    case 5: encode_tile_call<2, TS, 1>(a, tile, smem); break;
    case 6: encode_tile_call<3, TS, 0>(a, tile, smem); break;
    case 7: encode_tile_call<3, TS, 1>(a, tile, smem); break;
    case 8: encode_tile_call<4, TS, 0>(a, tile, smem); break;
    case 9: encode_tile_call<4, TS, 1>(a, tile, smem); break;
    case 10: encode_tile_call<5, TS, 0>(a, tile, smem); break;
    default: encode_tile_call<5, TS, 1>(a, tile, smem); break;
    }
}

// Many arrays in one persistent launch: CTAs take global tile tickets in
// order (so each array's tiles start in order, as its look-back needs),
// find the owning array by binary search over the tile prefix, and run
// that array's tile body.
template <int TS>
__global__ void __launch_bounds__(128) k_encode_batch(EncBatchArgs ba)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint64_t s_tile;
    __shared__ int s_job;
    __shared__ __align__(16) EncArgs s_args;
    while (true) {
        if (threadIdx.x == 0) {
            const uint64_t g = atomicAdd(ba.ticket, 1ull);
            int lo = 0, hi = ba.count;  // jobs[lo] owns g: prefix[lo] <= g < prefix[lo + 1]
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
            // the job's descriptor into shared memory
            const uint32_t *src = reinterpret_cast<const uint32_t *>(ba.jobs + s_job);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&s_args);
            for (int i = threadIdx.x; i < (int)(sizeof(EncArgs) / 4); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        encode_tile_any<TS>(s_args, s_tile, smem);
        __syncthreads();
    }
}

template <int DT, int TS>
static cudaError_t launch_ts(const EncArgs &a, int threads, size_t smem, cudaStream_t s)
{
    auto k = a.mode == 1 ? k_encode<DT, TS, 1> : k_encode<DT, TS, 0>;
    const cudaError_t e =
        a.mode == 1 ? smem_limit<k_encode<DT, TS, 1>>(smem) : smem_limit<k_encode<DT, TS, 0>>(smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)a.ntiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t launch_t1(const EncArgs &a, int threads, size_t smem, cudaStream_t s)
{
    auto k = k_encode_t1<DT>;  // fixed rate only
    const cudaError_t e = smem_limit<k_encode_t1<DT>>(smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)a.ntiles, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t launch_dt(const EncArgs &a, int ts, int threads, size_t smem, cudaStream_t s)
{
    if (ts == 1) return launch_t1<DT>(a, threads, smem, s);
    return ts == 8 ? launch_ts<DT, 8>(a, threads, smem, s) : launch_ts<DT, 32>(a, threads, smem, s);
}

cudaError_t launch_encode_batch(const EncBatchArgs &b, int ts, int threads, size_t smem,
                               unsigned ctas, cudaStream_t s)
{
    auto k = ts == 8 ? k_encode_batch<8> : k_encode_batch<32>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ctas) k<<<ctas, threads, smem, s>>>(b);
    return cudaGetLastError();
}

int encode_batch_occupancy(int ts, int threads, size_t smem)
{
    int nb = 0;
    auto k = ts == 8 ? k_encode_batch<8> : k_encode_batch<32>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_encode(const EncArgs &a, int ts, int threads, size_t smem, cudaStream_t s)
{
    switch (a.dtype) {
    case 1: return launch_dt<1>(a, ts, threads, smem, s);
    case 2: return launch_dt<2>(a, ts, threads, smem, s);
    case 3: return launch_dt<3>(a, ts, threads, smem, s);
    case 4: return launch_dt<4>(a, ts, threads, smem, s);
    default: return launch_dt<5>(a, ts, threads, smem, s);
    }
}


// ---------------------------------------------------------------- shards
// One container from the containers of contiguous block ranges (shards):
// each shard's offset table slice moves to its place with its payload's word
// offset added; the header names the whole array.
namespace {
__global__ void k_table_rebase(const uint32_t *src, uint32_t *dst, uint64_t count, uint64_t add)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = (uint32_t)((uint64_t)src[i] + add);  // the host checked the 2^32-word limit
}

// The first min(res->bytes, cap) bytes of src to dst (both 4-byte aligned,
// containers are whole words); 16-byte pieces when both are 16-byte aligned.
__global__ void k_copy_sized(const uint8_t *src, const apax_result *res, uint8_t *dst, uint64_t cap)
{
    const uint64_t rb = *(const volatile uint64_t *)&res->bytes;
    const uint64_t bytes = (rb < cap ? rb : cap) & ~3ull;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    uint64_t done = 0;
    if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
        const uint64_t n16 = bytes >> 4;
        for (uint64_t i = t0; i < n16; i += step)
            reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
        done = n16 << 4;
    }
    for (uint64_t i = (done >> 2) + t0; i < (bytes >> 2); i += step)
        reinterpret_cast<uint32_t *>(dst)[i] = reinterpret_cast<const uint32_t *>(src)[i];
}

__global__ void k_merged_header(EncArgs a, uint64_t payload)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        write_container_header(a, (int)a.code);
        put_le(a.out + 28, payload, 8);
        if (a.res) {
            a.res->bytes = a.poff + payload;
            a.res->status = 0;
        }
    }
}
}  // namespace

cudaError_t launch_table_rebase(const uint32_t *src, uint32_t *dst, uint64_t count, uint64_t add,
                                cudaStream_t s)
{
    if (count) {
        const uint64_t g = (count + 255) / 256;
        k_table_rebase<<<(unsigned)(g < 4096 ? g : 4096), 256, 0, s>>>(src, dst, count, add);
    }
    return cudaGetLastError();
}

cudaError_t launch_merged_header(const EncArgs &a, uint64_t payload, cudaStream_t s)
{
    k_merged_header<<<1, 32, 0, s>>>(a, payload);
    return cudaGetLastError();
}

cudaError_t launch_copy_sized(const void *src, const apax_result *res, void *dst, uint64_t cap,
                              cudaStream_t s)
{
    const uint64_t need = (cap + 16 * 256 - 1) / (16 * 256);  // CTAs for one 16-byte piece a thread
    const uint64_t most = 4ull * (uint64_t)sm_count();
    const unsigned ctas = (unsigned)(need < most ? (need ? need : 1) : most);
    k_copy_sized<<<ctas, 256, 0, s>>>(reinterpret_cast<const uint8_t *>(src), res,
                                      reinterpret_cast<uint8_t *>(dst), cap);
    return cudaGetLastError();
}

}  // namespace apax
